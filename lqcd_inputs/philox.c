/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) over arrays of 64-bit indices, for the
 * seeded input generators of large lattices.  Same words as the numpy version in philox.py:
 * counter = (index low word, index high word, purpose, 0), key = (seed low, seed high); ten
 * rounds, each multiplying counter words 0 and 2 by the published multipliers and mixing the
 * high halves with words 1 and 3 and the key, the key advanced by the Weyl increments. */
#include <math.h>
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

/* Uniforms of the seeded generators: two numbers in (0, 1) with 53-bit resolution per index, from
 * the four words (27 high bits of one word, 26 of the next, + 0.5, over 2^53). */
static void uniform_pair(uint64_t index, uint32_t purpose, uint64_t seed, double* u1, double* u2) {
  uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), purpose, 0u};
  philox_one(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  *u1 = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6) + 0.5) / 9007199254740992.0;
  *u2 = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6) + 0.5) / 9007199254740992.0;
}

/* Box-Muller: out[2 i], out[2 i + 1] = r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 ln u1). */
void gaussian_pairs(const uint64_t* index, long n, uint32_t purpose, uint64_t seed, double* out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) {
    double u1, u2;
    uniform_pair(index[i], purpose, seed, &u1, &u2);
    const double r = sqrt(-2.0 * log(u1)), th = 6.283185307179586476925286766559 * u2;
    out[2 * i] = r * cos(th);
    out[2 * i + 1] = r * sin(th);
  }
}

/* Eigen-decomposition of a 3x3 complex Hermitian matrix by cyclic Jacobi rotations (each rotation
 * zeroes one off-diagonal pair exactly; sweeps until the off-diagonal norm is below 1e-30 of the
 * matrix norm).  a: row-major (re, im) pairs, overwritten; w: eigenvalues; q: columns are the
 * eigenvectors. */
static void herm3_eig(double a[3][3][2], double w[3], double q[3][3][2]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      q[i][j][0] = i == j ? 1.0 : 0.0;
      q[i][j][1] = 0.0;
    }
  double norm = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) norm += a[i][j][0] * a[i][j][0] + a[i][j][1] * a[i][j][1];
  for (int sweep = 0; sweep < 50; sweep++) {
    double off = 0.0;
    for (int i = 0; i < 3; i++)
      for (int j = i + 1; j < 3; j++) off += a[i][j][0] * a[i][j][0] + a[i][j][1] * a[i][j][1];
    if (off <= 1e-30 * norm || off == 0.0) break;
    for (int p = 0; p < 2; p++)
      for (int r = p + 1; r < 3; r++) {
        const double ar = a[p][r][0], ai = a[p][r][1];
        const double mag = sqrt(ar * ar + ai * ai);
        if (mag == 0.0) continue;
        /* a_pr = mag e^{i phi}: the rotation J = [[c, -s e^{i phi}], [s e^{-i phi}, c]] on (p, r)
         * with tan(2 theta) = 2 mag / (a_pp - a_rr) zeroes a_pr in J^H A J */
        const double er = ar / mag, ei = ai / mag;
        const double app = a[p][p][0], arr = a[r][r][0];
        const double theta = 0.5 * atan2(2.0 * mag, app - arr);
        const double c = cos(theta), s = sin(theta);
        /* columns p, r of A <- A J */
        for (int k = 0; k < 3; k++) {
          const double kp0 = a[k][p][0], kp1 = a[k][p][1], kr0 = a[k][r][0], kr1 = a[k][r][1];
          /* new_kp = c a_kp + s e^{-i phi} a_kr ; new_kr = -s e^{i phi} a_kp + c a_kr */
          a[k][p][0] = c * kp0 + s * (er * kr0 + ei * kr1);
          a[k][p][1] = c * kp1 + s * (er * kr1 - ei * kr0);
          a[k][r][0] = c * kr0 - s * (er * kp0 - ei * kp1);
          a[k][r][1] = c * kr1 - s * (er * kp1 + ei * kp0);
          const double qp0 = q[k][p][0], qp1 = q[k][p][1], qr0 = q[k][r][0], qr1 = q[k][r][1];
          q[k][p][0] = c * qp0 + s * (er * qr0 + ei * qr1);
          q[k][p][1] = c * qp1 + s * (er * qr1 - ei * qr0);
          q[k][r][0] = c * qr0 - s * (er * qp0 - ei * qp1);
          q[k][r][1] = c * qr1 - s * (er * qp1 + ei * qp0);
        }
        /* rows p, r of A <- J^H A */
        for (int k = 0; k < 3; k++) {
          const double pk0 = a[p][k][0], pk1 = a[p][k][1], rk0 = a[r][k][0], rk1 = a[r][k][1];
          /* new_pk = c a_pk + s e^{i phi} a_rk ; new_rk = -s e^{-i phi} a_pk + c a_rk */
          a[p][k][0] = c * pk0 + s * (er * rk0 - ei * rk1);
          a[p][k][1] = c * pk1 + s * (er * rk1 + ei * rk0);
          a[r][k][0] = c * rk0 - s * (er * pk0 + ei * pk1);
          a[r][k][1] = c * rk1 - s * (er * pk1 - ei * pk0);
        }
        a[p][r][0] = a[p][r][1] = a[r][p][0] = a[r][p][1] = 0.0;
        a[p][p][1] = a[r][r][1] = 0.0;
      }
  }
  for (int i = 0; i < 3; i++) w[i] = a[i][i][0];
}

/* SU(3) links of the seeded recipe: for link id l, h_1..h_8 are the Box-Muller pairs of the
 * Philox indices 4 l + j (j = 0..3: h_{2j+1}, h_{2j+2}); H = sum_a h_a lambda_a / 2 with the
 * Gell-Mann matrices; U = exp(i eps H) = Q diag(exp(i eps w)) Q^H from the eigen-decomposition of
 * H.  out: n x 9 complex (row-major (re, im) pairs). */
void su3_links(const uint64_t* link_ids, long n, uint32_t purpose, uint64_t seed, double eps, double* out) {
  const double r3 = 1.0 / sqrt(3.0);
#pragma omp parallel for schedule(static)
  for (long l = 0; l < n; l++) {
    double h[8];
    for (int j = 0; j < 4; j++) {
      double u1, u2;
      uniform_pair(link_ids[l] * 4 + (uint64_t)j, purpose, seed, &u1, &u2);
      const double r = sqrt(-2.0 * log(u1)), th = 6.283185307179586476925286766559 * u2;
      h[2 * j] = r * cos(th);
      h[2 * j + 1] = r * sin(th);
    }
    double a[3][3][2] = {{{0}}};
    /* lambda_1..8 / 2 */
    a[0][1][0] += 0.5 * h[0]; a[1][0][0] += 0.5 * h[0];
    a[0][1][1] -= 0.5 * h[1]; a[1][0][1] += 0.5 * h[1];
    a[0][0][0] += 0.5 * h[2]; a[1][1][0] -= 0.5 * h[2];
    a[0][2][0] += 0.5 * h[3]; a[2][0][0] += 0.5 * h[3];
    a[0][2][1] -= 0.5 * h[4]; a[2][0][1] += 0.5 * h[4];
    a[1][2][0] += 0.5 * h[5]; a[2][1][0] += 0.5 * h[5];
    a[1][2][1] -= 0.5 * h[6]; a[2][1][1] += 0.5 * h[6];
    a[0][0][0] += 0.5 * r3 * h[7]; a[1][1][0] += 0.5 * r3 * h[7]; a[2][2][0] -= r3 * h[7];
    double w[3], q[3][3][2];
    herm3_eig(a, w, q);
    double* U = out + 18 * l;
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < 3; m++) {
          const double er = cos(eps * w[m]), ei = sin(eps * w[m]);
          /* q_im e^{i eps w_m} conj(q_km) */
          const double t0 = q[i][m][0] * er - q[i][m][1] * ei, t1 = q[i][m][0] * ei + q[i][m][1] * er;
          re += t0 * q[k][m][0] + t1 * q[k][m][1];
          im += t1 * q[k][m][0] - t0 * q[k][m][1];
        }
        U[2 * (3 * i + k)] = re;
        U[2 * (3 * i + k) + 1] = im;
      }
  }
}
