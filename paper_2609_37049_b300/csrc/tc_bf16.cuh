// Fifth-generation tensor-core building blocks (sm_100 family, tcgen05) for small BF16 GEMM tiles
// with FP32 accumulation in tensor memory, used by the network preconditioner (nn.cu).
//
// One CTA computes D[128 x N] = A[128 x K] B[K x N]: A and B sit in shared memory in the
// canonical K-major layout without swizzle ("core matrices" of 8 rows x 16 bytes = 8 x 8 BF16;
// element (r, k) at (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2 bytes), B stored as
// its transpose (N rows of K).  One elected thread issues the MMAs (K / 16 of them, accumulating
// in tensor memory); their completion is signalled on an mbarrier with tcgen05.commit; each warp
// of the CTA's first warpgroup then reads its 32 rows of D with tcgen05.ld (row r of D is tensor
// memory lane r, column j is column j of the allocation).
//
// Descriptor formats (PTX ISA, tcgen05 shared-memory descriptor and kind::f16 instruction
// descriptor):
//   smem descriptor: [0,14) address >> 4, [16,30) leading-dimension byte offset >> 4,
//                    [32,46) stride-dimension byte offset >> 4, [46,48) version 1,
//                    [49,52) base offset 0, [52] LBO mode 0, [61,64) layout 0 (no swizzle);
//   instruction descriptor: [4,6) D format (1 = F32), [7,10) A format (1 = BF16),
//                    [10,13) B format (1 = BF16), [15] A major (0 = K), [16] B major (0 = K),
//                    [17,23) N >> 3, [24,29) M >> 4.
// Every wait on an mbarrier has an iteration limit and a time limit; a wait that runs out sets a flag the kernel
// reports, and the kernel still deallocates its tensor memory before it returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace lqcd {
namespace tc {

LQCD_D uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

LQCD_D uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
  return d;                // base offset 0, LBO mode 0, no swizzle
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, both operands K-major, M x N tile.
constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Allocate ncols (power of two >= 32) tensor-memory columns for this CTA; one full warp executes
// it and the base address lands in *dst (shared memory).
LQCD_D void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

LQCD_D void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (+)= A B for one K = 16 step (single thread).
LQCD_D void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// Arrive on mbar once every MMA issued so far by this thread has completed.
LQCD_D void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

LQCD_D void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
LQCD_D void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes of shared memory made visible to the tensor cores (async proxy)
LQCD_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

LQCD_D void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// One arrival on mbar (release: this thread's earlier writes are visible to whoever sees the
// phase complete).
LQCD_D void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Wait for phase `parity` of mbar to complete; false if it did not within `limit` polls or
// about two seconds (global timer), whichever comes first.  Each poll may suspend the thread for
// up to kSuspendNs (it resumes as soon as the phase completes), so a waiting warp takes no issue
// slots from the warps it waits for.
constexpr uint32_t kSuspendNs = 20000;
LQCD_D bool mbar_wait(uint64_t* mbar, uint32_t parity, int limit) {
  const uint32_t a = smem_u32(mbar);
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < limit; i++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if ((i & 15) == 15) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) return false;
    }
  }
  return false;
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (lane = row within the warp's
// quarter); taddr carries the lane quarter in bits 16+ and the column in bits 0..15.
LQCD_D void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (r, k) of a K-major BF16 operand in the canonical no-swizzle layout
// with core matrices packed K-fastest: LBO = 128 bytes (next 8 k), SBO = (K / 8) * 128 bytes
// (next 8 rows).
LQCD_HD uint32_t kmajor_offset(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

}  // namespace tc
}  // namespace lqcd
