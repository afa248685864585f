// FP64 GEMM emulated on the BF16 tensor cores (tcgen05), for the FP64 stages of the mixed form.
//
// GB300 executes FP64 at ~1 TFLOP/s (DMMA and DFMA alike) but BF16 at ~1.9 PFLOP/s, so an FP64
// product is formed from exact BF16 pieces (an error-free splitting in the manner of Ozaki, Ogita,
// Oishi and Rump):
//
//   row i of op(A) is scaled by 2^-E_i, column j of op(B) by 2^-F_j (E, F: exponents just above the
//   largest magnitude), so every scaled entry x lies in (-1, 1);  x = sum_{p=1..8} a_p 2^-7p with
//   integer digits |a_p| <= 127 taken from the bits of x (integer arithmetic only, truncated below
//   2^-56);  a_p 2^-7p is stored as BF16, exactly.
//
//   A B = 2^(E_i+F_j) sum_{p,q} (a_p 2^-7p)(b_q 2^-7q); pairs with p + q >= 10 (< 2^-56 relative)
//   are dropped.  For d = p + q <= 7 the products of one diagonal d are integers times 2^-7d below
//   2^14: summed over a K chunk of 128 with at most 6 pairs they stay below 2^24, so the FP32
//   tensor-memory accumulator holds them exactly; after each chunk these exact sums are added to
//   one FP64 accumulator per output in registers (6 additions per 128 of K: fewer roundings than an
//   FP64 dot product of length K).  The diagonals d = 8, 9 share one FP32 accumulator over all of
//   K; its roundings stay near 2^-51 of the result.
//
// CTA tile 128 x 64 (TMEM: 6 exact accumulators + 1 shared, 64 columns each), 128 threads; the 8
// digit planes of the 128 x 64 A slice and the 64 x 64 B slice occupy 192 KB of shared memory
// (canonical K-major layout without swizzle, as in tc_gemm.cu).  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gev {

namespace {

constexpr int OM = 128, ON = 64, OK_ = 64, NTH = 128, NSLICE = 8, DMAX = 9, DEXACT = 7;
constexpr int A_PLANE = OM * OK_ * 2;  // 16 KB
constexpr int B_PLANE = ON * OK_ * 2;  // 8 KB
constexpr int SMEM_OZ = NSLICE * (A_PLANE + B_PLANE) + 1024;
constexpr int TMEM_COLS_OZ = 512;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int toff(int r, int k) {
  return ((r >> 3) * (OK_ / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (OK_ / 8) * 128;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | ((uint64_t)1 << 46);
}

__host__ __device__ constexpr uint32_t idesc_oz() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ON >> 3) << 17) | ((uint32_t)(OM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ bool bar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(20);
  }
  return false;
}

// exponent E with |x| < 2^E for a finite x != 0 (0 for x == 0)
__device__ __forceinline__ int exp_above(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be == 0) return (b << 1) ? -1022 : -100000;  // subnormal / zero
  return be - 1022;  // |x| < 2^(be - 1023 + 1)
}

// per-row exponents of op(A) (mask applied): one thread per row
__global__ void k_row_exp(int M, int K, const double* A, long long lda, int ta, int tri, int* E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int e = -100000;
  const int k0 = (tri == 2) ? min(i, K) : 0, k1 = (tri == 1) ? min(i + 1, K) : K;
  for (int k = k0; k < k1; ++k) e = max(e, exp_above(ta == 0 ? A[i + k * lda] : A[k + i * lda]));
  E[i] = (e == -100000) ? 0 : e;
}

// per-column exponents of op(B) (mask applied): one thread per column
__global__ void k_col_exp(int N, int K, const double* B, long long ldb, int tb, int tri, int* F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  int e = -100000;
  const int k0 = (tri == 1) ? min(j, K) : 0, k1 = (tri == 2) ? min(j + 1, K) : K;
  for (int k = k0; k < k1; ++k) e = max(e, exp_above(tb == 0 ? B[k + j * ldb] : B[j + k * ldb]));
  F[j] = (e == -100000) ? 0 : e;
}

// the 8 digit planes of x * 2^-E, as BF16 with their scale 2^-7p
__device__ __forceinline__ void split_digits(double x, int E, unsigned char* planes, int plane_bytes, int off) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (be != 0 || (bits << 1) != 0) {
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int ex;
    if (be == 0) { ex = -1022; } else { m |= (1ull << 52); ex = be - 1023; }
    const int s = ex - E + 4;  // X = |x| 2^(56-E) = m 2^(ex - 52 + 56 - E)
    if (s >= 0) X = m << s;            // s <= 3 since |x| < 2^E
    else if (s > -64) X = m >> (-s);   // digits below 2^-56 are dropped
  }
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int p = 1; p <= NSLICE; ++p) {
    const int dig = (int)((X >> (56 - 7 * p)) & 127ull);
    float v = __int2float_rn(neg ? -dig : dig);
    v = ldexpf(v, -7 * p);  // exact: a power-of-two scale of a 7-bit integer
    *reinterpret_cast<__nv_bfloat16*>(planes + (p - 1) * plane_bytes + off) = __float2bfloat16_rn(v);
  }
}

struct OzP {
  int M, N, K, ta, tb, tri_a, tri_b, c_lower;
  double alpha, beta;
  const double* A;
  long long lda;
  const double* B;
  long long ldb;
  double* C;
  long long ldc;
  const int* E;
  const int* F;
  int* status;
};

__global__ void __launch_bounds__(NTH, 1) ozaki_kernel(OzP p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * OM, n0 = blockIdx.y * ON;
  if (p.c_lower && n0 > m0 + OM - 1) return;
  int kb = 0, ke = p.K;
  if (p.tri_a == 1) ke = min(ke, m0 + OM);
  else if (p.tri_a == 2) kb = max(kb, m0);
  if (p.tri_b == 1) kb = max(kb, n0);
  else if (p.tri_b == 2) ke = min(ke, n0 + ON);
  kb = kb / OK_ * OK_;
  unsigned char* Ap = smem;                                // 8 planes x 16 KB
  unsigned char* Bp = smem + NSLICE * A_PLANE;              // 8 planes x 8 KB
  unsigned char* ctrl = smem + NSLICE * (A_PLANE + B_PLANE);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ctrl);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctrl + 64);
  int* flag = reinterpret_cast<int*>(ctrl + 128);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                 "r"(TMEM_COLS_OZ));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc_oz();
  // TMEM accumulators: exact diagonals d = 2..7 at columns (d-2)*64, the shared one at 6*64
  constexpr int SHARED_SLOT = DEXACT - 1;
  double acc[ON];
#pragma unroll
  for (int c = 0; c < ON; ++c) acc[c] = 0.0;
  const int row = warp * 32 + lane;  // TMEM lane = tile row owned by this thread
  const int nsteps = (ke > kb) ? (ke - kb + OK_ - 1) / OK_ : 0;
  uint32_t phase = 0;
  bool ok = true;
  for (int st = 0; st < nsteps && ok; ++st) {
    const int k0 = kb + st * OK_;
    // ---- producer: digit planes of the 128 x 64 A slice and the 64 x 64 B slice
    for (int e = tid; e < OM * OK_; e += NTH) {
      int r, k;
      if (p.ta == 0) { r = e % OM; k = e / OM; } else { k = e % OK_; r = e / OK_; }
      const int gi = m0 + r, gk = k0 + k;
      double v = 0.0;
      int E = 0;
      if (gi < p.M && gk < ke && !((p.tri_a == 1 && gk > gi) || (p.tri_a == 2 && gk < gi))) {
        v = (p.ta == 0) ? p.A[gi + gk * p.lda] : p.A[gk + gi * p.lda];
        E = p.E[gi];
      }
      split_digits(v, E, Ap, A_PLANE, toff(r, k));
    }
    for (int e = tid; e < ON * OK_; e += NTH) {
      int c, k;
      if (p.tb == 0) { k = e % OK_; c = e / OK_; } else { c = e % ON; k = e / ON; }
      const int gj = n0 + c, gk = k0 + k;
      double v = 0.0;
      int F = 0;
      if (gj < p.N && gk < ke && !((p.tri_b == 1 && gk < gj) || (p.tri_b == 2 && gk > gj))) {
        v = (p.tb == 0) ? p.B[gk + gj * p.ldb] : p.B[gj + gk * p.ldb];
        F = p.F[gj];
      }
      split_digits(v, F, Bp, B_PLANE, toff(c, k));
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    // ---- MMAs of this 64-deep slice: 4 k-steps x 36 digit pairs
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const bool chunk_start = (st & 1) == 0;  // exact diagonals restart every 128 of K
      const uint32_t a0 = su32(Ap), b0 = su32(Bp);
      for (int ks = 0; ks < OK_ / 16; ++ks) {
        const uint32_t koff = ks * 256;
        bool first_exact[DEXACT + 1] = {true, true, true, true, true, true, true, true};
        for (int pa = 1; pa <= NSLICE; ++pa) {
          for (int qb = 1; qb + pa <= DMAX; ++qb) {
            const int d = pa + qb;
            int slot, en;
            if (d <= DEXACT) {
              slot = d - 2;
              en = (chunk_start && ks == 0 && first_exact[d]) ? 0 : 1;
              first_exact[d] = false;
            } else {
              slot = SHARED_SLOT;
              en = (st == 0 && ks == 0 && pa == 1 && qb == DEXACT) ? 0 : 1;  // first shared-accumulator MMA
            }
            mma(tmem + slot * ON, sdesc(a0 + (pa - 1) * A_PLANE + koff), sdesc(b0 + (qb - 1) * B_PLANE + koff), id,
                en);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(mbar))
                   : "memory");
      *flag = bar_wait(su32(mbar), phase) ? 0 : 1;
    }
    __syncthreads();
    if (*flag) { ok = false; break; }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // ---- end of a 128-deep chunk (or of K): move the exact diagonals into the integer accumulators
    if ((st & 1) == 1 || st == nsteps - 1) {
#pragma unroll
      for (int d = 2; d <= DEXACT; ++d) {
#pragma unroll
        for (int cb = 0; cb < ON; cb += 16) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((d - 2) * ON + cb);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[cb + q] += (double)__uint_as_float(r[q]);  // exact chunk sums
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();  // the next chunk's first MMAs overwrite these accumulators
    }
  }
  if (!ok && tid == 0) atomicCAS(&p.status[ST_TIMEOUT], 0, 402);
  // ---- epilogue: the shared low-order accumulator, then C = alpha 2^(E+F) sum + beta C
  const bool any = nsteps > 0 && ok;
  const int gi = m0 + row;
  const int Ei = (gi < p.M) ? p.E[gi] : 0;
#pragma unroll
  for (int cb = 0; cb < ON; cb += 16) {
    uint32_t r[16];
    if (any) {
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(SHARED_SLOT * ON + cb);
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
    if (gi < p.M) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int gj = n0 + cb + q;
        if (gj >= p.N || (p.c_lower && gi < gj)) continue;
        const double s = (any ? acc[cb + q] + (double)__uint_as_float(r[q]) : 0.0);
        const double v = p.alpha * ldexp(s, Ei + p.F[gj]);
        double* c = &p.C[gi + gj * p.ldc];
        *c = (p.beta != 0.0) ? v + p.beta * (*c) : v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS_OZ));
}

}  // namespace

// FP64 GEMM on the tensor cores (real data).  Needs 2 * max(M, N) ints of scratch in s.ozws.
void gemm_f64_emulated(Sys& s, const GemmP<double>& q) {
  if (q.M <= 0 || q.N <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute((const void*)ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_OZ);
    attr = true;
  }
  int* E = s.ozws;
  int* F = s.ozws + std::max(q.M, q.N) + 8;
  GEV_COUNT(s);
  k_row_exp<<<cdiv(q.M, 128), 128, 0, s.stream>>>(q.M, q.K, q.A, q.lda, q.ta, q.tri_a, E);
  GEV_COUNT(s);
  k_col_exp<<<cdiv(q.N, 128), 128, 0, s.stream>>>(q.N, q.K, q.B, q.ldb, q.tb, q.tri_b, F);
  OzP p{};
  p.M = q.M; p.N = q.N; p.K = q.K; p.ta = q.ta; p.tb = q.tb; p.tri_a = q.tri_a; p.tri_b = q.tri_b;
  p.c_lower = q.c_lower; p.alpha = q.alpha; p.beta = q.beta; p.A = q.A; p.lda = q.lda; p.B = q.B;
  p.ldb = q.ldb; p.C = q.C; p.ldc = q.ldc; p.E = E; p.F = F; p.status = s.status;
  GEV_COUNT(s);
  ozaki_kernel<<<dim3(cdiv(q.M, OM), cdiv(q.N, ON)), NTH, SMEM_OZ, s.stream>>>(p);
}

}  // namespace gev

extern "C" int gev_gemm_f64(int M, int N, int K, int ta, int tb, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc, int engine, void* stream,
                            int* status_dev, int* scratch_dev) {
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
  if (engine == 1 && !scratch_dev) return -17;
  Sys s;
  s.stream = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  GEV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s.sms = sms > 0 ? sms : 152;
  s.status = status_dev;
  s.ozws = scratch_dev;
  s.emu_fp64 = engine;
  s.splitws = nullptr;
  s.splitws_bytes = 0;
  gemm<double>(s, gp<double>(M, N, K, ta, tb, alpha, A, lda, B, ldb, beta, C, ldc));
  GEV_TRY(last_error());
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}
