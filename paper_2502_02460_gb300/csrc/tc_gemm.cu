// FP32 GEMM from BF16x3 products on the 5th-generation tensor cores (tcgen05, kind::f16, FP32
// accumulation in tensor memory), for the FP32 stages of the mixed form.
//
//   a = a_hi + a_lo,  b = b_hi + b_lo  (a_hi = bf16(a), a_lo = bf16(a - a_hi))
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (three MMAs into one accumulator)
//
// One CTA (128 threads) owns a 128 x 128 tile of C.  Producer: all threads load the FP32 (or FP64)
// operand tiles with any transpose / triangular mask, split them into hi/lo BF16 and store them in
// the canonical K-major, no-swizzle layout (core matrices of 8 rows x 16 bytes; LBO = 128 B between
// core matrices along K, SBO = 1024 B along M/N).  One elected thread issues the MMAs of the 64-deep
// slice (4 k-steps x 3 products) and commits them to an mbarrier; the next slice is staged into the
// other buffer while they run.  Epilogue: the 4 warps read their 32 TMEM lanes (tcgen05.ld 32x32b)
// and write C.  Every wait on the mbarrier is bounded; on expiry the kernel records ST_TIMEOUT,
// waits (bounded) for its MMAs and frees its tensor memory before returning.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace gev {

namespace {

constexpr int TM = 128, TN = 128, TK = 64, NTH = 128;
constexpr int TMEM_COLS = 256;                      // >= TN (headroom keeps any N field in range)
constexpr int OP_BYTES = TM * TK * 2;               // one BF16 operand tile: 16 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;           // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;  // two stages + barriers

template <class TI, class TO> struct TcP {
  int M, N, K, ta, tb, tri_a, tri_b, c_lower;
  float alpha, beta;
  const TI* A;
  long long lda;
  const TI* B;
  long long ldb;
  TO* C;
  long long ldc;
  int* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// offset (bytes) of element (r, k) of a 128 x 64 K-major tile in the no-swizzle canonical layout
__device__ __forceinline__ int tile_off(int r, int k) {
  return ((r >> 3) * (TK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (TK / 8) * 128;
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(lbo >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, relative LBO mode, no swizzle (bits 61-63 = 0)
  return d;
}

// kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the given phase parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    __nanosleep(20);
  }
  return false;
}

template <class TI, class TO>
__device__ __forceinline__ float load_a(const TcP<TI, TO>& p, int gi, int gk) {
  if (gi >= p.M || gk >= p.K) return 0.f;
  if ((p.tri_a == 1 && gk > gi) || (p.tri_a == 2 && gk < gi)) return 0.f;
  return (float)((p.ta == 0) ? p.A[gi + gk * p.lda] : p.A[gk + gi * p.lda]);
}
template <class TI, class TO>
__device__ __forceinline__ float load_b(const TcP<TI, TO>& p, int gk, int gj) {
  if (gj >= p.N || gk >= p.K) return 0.f;
  if ((p.tri_b == 1 && gk < gj) || (p.tri_b == 2 && gk > gj)) return 0.f;
  return (float)((p.tb == 0) ? p.B[gk + gj * p.ldb] : p.B[gj + gk * p.ldb]);
}

__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int off, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
}

template <class TI, class TO>
__global__ void __launch_bounds__(NTH, 1) tc_gemm_kernel(TcP<TI, TO> p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (p.c_lower && n0 > m0 + TM - 1) return;
  int kb = 0, ke = p.K;
  if (p.tri_a == 1) ke = min(ke, m0 + TM);
  else if (p.tri_a == 2) kb = max(kb, m0);
  if (p.tri_b == 1) kb = max(kb, n0);
  else if (p.tri_b == 2) ke = min(ke, n0 + TN);
  kb = kb / TK * TK;
  unsigned char* stage0 = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);       // 2 barriers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE_BYTES + 64);
  int* flag = reinterpret_cast<int*>(smem + 2 * STAGE_BYTES + 128);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(TM, TN);

  const int nslices = (ke > kb) ? (ke - kb + TK - 1) / TK : 0;
  uint32_t phase[2] = {0, 0};
  int pending[2] = {0, 0};  // MMAs committed to barrier s and not yet waited for
  bool ok = true;
  for (int sl = 0; sl < nslices && ok; ++sl) {
    const int s = sl & 1;
    unsigned char* st = stage0 + s * STAGE_BYTES;
    // the MMAs that last read this stage must be done before it is overwritten (thread 0 waits,
    // the outcome is shared so every thread takes the same branch)
    if (pending[s]) {
      if (tid == 0) *flag = mbar_wait(smem_u32(&mbar[s]), phase[s]) ? 0 : 1;
      __syncthreads();
      const int expired = *flag;
      __syncthreads();
      if (expired) { ok = false; break; }
      phase[s] ^= 1;
      pending[s] = 0;
    }
    const int k0 = kb + sl * TK;
    // producer: 128 x 64 tiles of op(A) and op(B)^T, split into hi / lo
    for (int e = tid; e < TM * TK; e += NTH) {
      int r, k;
      if (p.ta == 0) { r = e % TM; k = e / TM; } else { k = e % TK; r = e / TK; }
      int gk = k0 + k;
      float v = (gk < ke) ? load_a(p, m0 + r, gk) : 0.f;
      split_store(st, st + OP_BYTES, tile_off(r, k), v);
      int c, kk;
      if (p.tb == 0) { kk = e % TK; c = e / TK; } else { c = e % TN; kk = e / TN; }
      gk = k0 + kk;
      v = (gk < ke) ? load_b(p, gk, n0 + c) : 0.f;
      split_store(st + 2 * OP_BYTES, st + 3 * OP_BYTES, tile_off(c, kk), v);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + OP_BYTES, b_hi = a_hi + 2 * OP_BYTES,
                     b_lo = a_hi + 3 * OP_BYTES;
#pragma unroll
      for (int ks = 0; ks < TK / 16; ++ks) {
        const uint32_t koff = ks * 2 * 128;  // 16 BF16 along K = two core matrices = 2 * LBO
        const int first = (sl == 0 && ks == 0) ? 0 : 1;
        mma_bf16(tmem, smem_desc(a_hi + koff), smem_desc(b_hi + koff), idesc, first);
        mma_bf16(tmem, smem_desc(a_hi + koff), smem_desc(b_lo + koff), idesc, 1);
        mma_bf16(tmem, smem_desc(a_lo + koff), smem_desc(b_hi + koff), idesc, 1);
      }
      mma_commit(smem_u32(&mbar[s]));
    }
    pending[s] = 1;
  }
  // drain: wait for every committed batch (bounded, thread 0)
  if (tid == 0) {
    bool good = ok;
    for (int s = 0; s < 2; ++s)
      if (pending[s] && !mbar_wait(smem_u32(&mbar[s]), phase[s])) good = false;
    *flag = good ? 0 : 1;
    if (!good) atomicCAS(&p.status[ST_TIMEOUT], 0, 401);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool any_mma = nslices > 0 && *flag == 0;
  // epilogue: warp w owns rows 32w .. 32w+31 (TMEM lanes), 16 columns per load
  const int row = m0 + warp * 32 + lane;
  for (int cb = 0; cb < TN; cb += 16) {
    uint32_t r[16];
    if (any_mma) {
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) r[q] = 0u;
    }
    if (row < p.M) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int col = n0 + cb + q;
        if (col >= p.N || (p.c_lower && row < col)) continue;
        TO* c = &p.C[row + (long long)col * p.ldc];
        const TO out = (TO)(p.alpha * __uint_as_float(r[q]));
        *c = (p.beta != 0.f) ? out + (TO)p.beta * (*c) : out;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

// C = alpha op(A) op(B) + beta C with BF16x3 tensor-core products (FP32 accumulation).  Falls back to
// the FP32 SIMT GEMM (gemm32) when the output has too few tiles to fill the GPU (split K there).
template <class TI, class TO> void gemm_bf16x3(Sys& s, const GemmP<TI>& q, TO* C, float alpha, float beta) {
  if (q.M <= 0 || q.N <= 0) return;
  const long long tiles = (long long)cdiv(q.M, TM) * cdiv(q.N, TN);
  if (tiles * 2 < s.sms && q.K >= 512) {
    gemm32<TI, TO>(s, q, C, alpha, beta);
    return;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute((const void*)tc_gemm_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM_BYTES);
    attr = true;
  }
  TcP<TI, TO> p{};
  p.M = q.M; p.N = q.N; p.K = q.K; p.ta = q.ta; p.tb = q.tb; p.tri_a = q.tri_a; p.tri_b = q.tri_b;
  p.c_lower = q.c_lower; p.alpha = alpha; p.beta = beta; p.A = q.A; p.lda = q.lda; p.B = q.B; p.ldb = q.ldb;
  p.C = C; p.ldc = q.ldc; p.status = s.status;
  dim3 grid(cdiv(q.M, TM), cdiv(q.N, TN));
  GEV_COUNT(s);
  tc_gemm_kernel<TI, TO><<<grid, NTH, SMEM_BYTES, s.stream>>>(p);
}

template void gemm_bf16x3<float, float>(Sys&, const GemmP<float>&, float*, float, float);
template void gemm_bf16x3<float, double>(Sys&, const GemmP<float>&, double*, float, float);
template void gemm_bf16x3<double, double>(Sys&, const GemmP<double>&, double*, float, float);

}  // namespace gev

extern "C" int gev_gemm_f32(int M, int N, int K, int ta, int tb, float alpha, const float* A, int lda,
                            const float* B, int ldb, float beta, float* C, int ldc, int engine, void* stream,
                            int* status_dev) {
  using namespace gev;
  if (M < 0) return -1;
  if (N < 0) return -2;
  if (K < 0) return -3;
  if (ta < 0 || ta > 1) return -4;
  if (tb < 0 || tb > 1) return -5;
  if (!A && M > 0 && K > 0) return -7;
  if (lda < std::max(1, ta ? K : M)) return -8;
  if (!B && K > 0 && N > 0) return -9;
  if (ldb < std::max(1, tb ? N : K)) return -10;
  if (!C && M > 0 && N > 0) return -12;
  if (ldc < std::max(1, M)) return -13;
  if (engine < 0 || engine > 1) return -14;
  if (!status_dev) return -16;
  Sys s;
  s.stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  GEV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s.sms = sms > 0 ? sms : 152;
  s.status = status_dev;
  s.splitws = nullptr;
  s.splitws_bytes = 0;
  GemmP<float> g = gp<float>(M, N, K, ta, tb, alpha, A, lda, B, ldb, beta, C, ldc);
  if (engine == 1) gemm_bf16x3<float, float>(s, g, C, alpha, beta);
  else gemm32<float, float>(s, g, C, alpha, beta);
  GEV_TRY(last_error());
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}
