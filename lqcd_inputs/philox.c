/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) over arrays of 64-bit indices, for the
 * seeded input generators of large lattices.  Same words as the numpy version in philox.py:
 * counter = (index low word, index high word, purpose, 0), key = (seed low, seed high); ten
 * rounds, each multiplying counter words 0 and 2 by the published multipliers and mixing the
 * high halves with words 1 and 3 and the key, the key advanced by the Weyl increments. */
#include <stdint.h>

static void philox_one(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; r++) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

/* out[4 i + w] = word w of Philox(index[i]) for i < n. */
void philox_words(const uint64_t* index, long n, uint32_t purpose, uint64_t seed, uint32_t* out) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) {
    uint32_t c[4] = {(uint32_t)index[i], (uint32_t)(index[i] >> 32), purpose, 0u};
    philox_one(c, k0, k1);
    out[4 * i] = c[0];
    out[4 * i + 1] = c[1];
    out[4 * i + 2] = c[2];
    out[4 * i + 3] = c[3];
  }
}
