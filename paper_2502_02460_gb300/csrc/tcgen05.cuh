// Building blocks shared by the tcgen05 matrix-product kernels (ozaki.cu, tc_gemm.cu): shared-memory
// descriptors for 16-deep K-major operand slices, the kind::f16 MMA, commits and bounded mbarrier
// waits, bulk copies and tensor-memory loads.  All inline PTX for sm_103a.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace gev {
namespace tc {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major 16-deep operand slice: 8 x 8 core matrices of 16-byte
// rows, the two k-halves adjacent (leading offset 128 B), 8-row groups 256 B apart
__host__ __device__ __forceinline__ int toff16(int r, int k) {
  return ((r >> 3) * 2 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor of such a slice (no swizzle, descriptor version 1)
__device__ __forceinline__ uint64_t sdesc16(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on mbar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; gives up early once another role has recorded an error in *err
__device__ __forceinline__ bool bar_wait(uint32_t mbar, uint32_t parity, volatile int* err) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (try_wait(mbar, parity)) return true;
    if ((it & 255) == 255 && *err) return false;
    __nanosleep(32);
  }
  return false;
}

// bounded wait without the early exit (draining after an error)
__device__ __forceinline__ bool bar_wait_plain(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (try_wait(mbar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_smem), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// zero-pattern masks of a product: op(A)[i,k] = 0 for k > i (tri_a 1) or k < i (tri_a 2);
// op(B)[k,j] = 0 for k < j (tri_b 1) or k > j (tri_b 2).  As "keep" codes over (vector r, element k):
// 1 keeps k <= r, 2 keeps k >= r.
__host__ __device__ __forceinline__ bool kept(int keep, long long r, long long k) {
  return keep == 0 || (keep == 1 ? k <= r : k >= r);
}

// k range [kb, ke) of a tile (rows m0 .. m0+TM-1 of op(A), columns n0 .. n0+TN-1 of op(B)) holding
// non-zero products; k absolute = local + koff
__device__ __forceinline__ void tile_k_range(int tri_a, int tri_b, int m0, int TM, int n0, int TN, int K, int koff,
                                             long long& kb, long long& ke) {
  kb = 0;
  ke = K;
  if (tri_a == 1) ke = ke < (long long)m0 + TM - koff ? ke : (long long)m0 + TM - koff;
  else if (tri_a == 2) kb = kb > (long long)m0 - koff ? kb : (long long)m0 - koff;
  if (tri_b == 1) kb = kb > (long long)n0 - koff ? kb : (long long)n0 - koff;
  else if (tri_b == 2) ke = ke < (long long)n0 + TN - koff ? ke : (long long)n0 + TN - koff;
}

}  // namespace tc
}  // namespace gev
