// FP32 GEMM on the CUDA cores (FFMA) for the FP32 stages of the mixed form: the full->band updates,
// the back-transforms and the divide-and-conquer merge products.  Operands may be FP32 or FP64
// (converted to FP32 when staged), the result FP32 or FP64.
//
// 128x128 tile (128x64 / 64x128 for thin products), 8-deep k slice, an 8x8 register micro-tile per
// thread (rows ty*4+{0..3} and BM/2+ty*4+{0..3}, columns likewise, so the shared-memory reads are
// float4 and conflict free), a two-stage smem pipeline, the same zero-pattern masks as the FP64
// GEMM and a deterministic split K.  Measured FFMA peak on GB300: 73.9 TFLOP/s.
#include <algorithm>

#include "common.cuh"

namespace gev {

namespace {

constexpr int BK = 8;

template <class TI, class TO> struct G32 {
  int M, N, K, ta, tb, tri_a, tri_b, c_lower;
  float alpha, beta;
  const TI* A;
  long long lda;
  const TI* B;
  long long ldb;
  TO* C;
  long long ldc;
  int ksplit;
  float* ws;
};

template <class TI, class TO>
__device__ __forceinline__ float ld_a(const G32<TI, TO>& p, int gi, int gk, int kb, int ke) {
  if (gi >= p.M || gk >= ke || gk < kb) return 0.f;
  if ((p.tri_a == 1 && gk > gi) || (p.tri_a == 2 && gk < gi)) return 0.f;
  return (float)((p.ta == 0) ? p.A[gi + gk * p.lda] : p.A[gk + gi * p.lda]);
}
template <class TI, class TO>
__device__ __forceinline__ float ld_b(const G32<TI, TO>& p, int gk, int gj, int kb, int ke) {
  if (gj >= p.N || gk >= ke || gk < kb) return 0.f;
  if ((p.tri_b == 1 && gk < gj) || (p.tri_b == 2 && gk > gj)) return 0.f;
  return (float)((p.tb == 0) ? p.B[gk + gj * p.ldb] : p.B[gj + gk * p.ldb]);
}

// BM x BN tile (128 x 128, or 128 x 64 / 64 x 128 for thin products), BM BN / 64 threads with an
// 8 x 8 register micro-tile each: rows ty*4+{0..3} and BM/2+ty*4+{0..3}, columns likewise.
template <class TI, class TO, int BM, int BN>
__global__ void __launch_bounds__(BM * BN / 64) gemm32_kernel(G32<TI, TO> p) {
  constexpr int NT = BM * BN / 64, RA = BM * BK / NT, RB = BN * BK / NT, TXN = BN / 8;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (p.c_lower && n0 > m0 + BM - 1) return;
  int kb = 0, ke = p.K;
  if (p.tri_a == 1) ke = min(ke, m0 + BM);
  else if (p.tri_a == 2) kb = max(kb, m0);
  if (p.tri_b == 1) kb = max(kb, n0);
  else if (p.tri_b == 2) ke = min(ke, n0 + BN);
  if (p.ksplit > 1) {
    const int chunk = ((p.K + p.ksplit - 1) / p.ksplit + BK - 1) / BK * BK;
    const int z0 = blockIdx.z * chunk;
    kb = max(kb, z0);
    ke = min(ke, z0 + chunk);
  }
  kb = kb / BK * BK;
  const int tid = threadIdx.x, tx = tid % TXN, ty = tid / TXN;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float ra[RA], rb[RB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (p.ta == 0) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      ra[r] = ld_a(p, m0 + i, k0 + k, kb, ke);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int e = tid + r * NT;
      int j, kk;
      if (p.tb == 0) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      rb[r] = ld_b(p, k0 + kk, n0 + j, kb, ke);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (p.ta == 0) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      As[buf][k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int e = tid + r * NT;
      int j, kk;
      if (p.tb == 0) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      Bs[buf][kk][j] = rb[r];
    }
  };
  int buf = 0;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][BM / 2 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][BN / 2 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  // epilogue: the 8 loads of C of a row first, so that they overlap
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = m0 + (i < 4 ? ty * 4 + i : BM / 2 + ty * 4 + (i - 4));
    if (gi >= p.M) continue;
    const bool read_c = p.ksplit == 1 && p.beta != 0.f;
    TO cin[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gj = n0 + (j < 4 ? tx * 4 + j : BN / 2 + tx * 4 + (j - 4));
      cin[j] = (read_c && gj < p.N && !(p.c_lower && gi < gj)) ? p.C[gi + gj * p.ldc] : (TO)0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gj = n0 + (j < 4 ? tx * 4 + j : BN / 2 + tx * 4 + (j - 4));
      if (gj >= p.N) continue;
      if (p.c_lower && gi < gj) continue;
      if (p.ksplit > 1) {
        p.ws[(size_t)blockIdx.z * p.M * p.N + gi + (size_t)gj * p.M] = acc[i][j];
      } else {
        const TO out = (TO)(p.alpha * acc[i][j]);  // the accumulation with C happens in TO
        p.C[gi + gj * p.ldc] = read_c ? out + (TO)p.beta * cin[j] : out;
      }
    }
  }
}

template <class TI, class TO>
__global__ void splitk_reduce32(G32<TI, TO> p) {
  const long long total = (long long)p.M * p.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.M), j = (int)(t / p.M);
    if (p.c_lower && i < j) continue;
    float s = 0.f;
    for (int z = 0; z < p.ksplit; ++z) s += p.ws[(size_t)z * total + t];
    TO* c = &p.C[i + (long long)j * p.ldc];
    const TO out = (TO)(p.alpha * s);
    if (p.beta != 0.f) *c = out + (TO)p.beta * (*c);
    else *c = out;
  }
}

}  // namespace

template <class TI, class TO> void gemm32(Sys& s, const GemmP<TI>& q, TO* C, float alpha, float beta) {
  if (q.M <= 0 || q.N <= 0) return;
  // large products go to the tensor cores (BF16 split products, tc_gemm.cu) when enabled
  // (thin products stay on the CUDA cores: the tensor cores' FP32 accumulation is about ten times
  // less accurate over long K, which costs the mixed form refinement iterations)
  if (s.fp32_tc && q.M >= 128 && q.N >= 128 && q.K >= 32 && (double)q.M * q.N * q.K >= 1.0e8 &&
      gemm_tc32<TI, TO>(s, q, C, alpha, beta, s.fp32_tc))
    return;
  G32<TI, TO> p{};
  p.M = q.M; p.N = q.N; p.K = q.K; p.ta = q.ta; p.tb = q.tb; p.tri_a = q.tri_a; p.tri_b = q.tri_b;
  p.c_lower = q.c_lower; p.alpha = alpha; p.beta = beta; p.A = q.A; p.lda = q.lda; p.B = q.B;
  p.ldb = q.ldb; p.C = C; p.ldc = q.ldc;
  // tile shape: thin products (N or M <= 64) use a 64-wide tile so no half of it idles
  const int shape = (p.N <= 64 && p.M > 64) ? 1 : ((p.M <= 64 && p.N > 64) ? 2 : 0);
  const int BM = shape == 2 ? 64 : 128, BN = shape == 1 ? 64 : 128;
  dim3 grid(cdiv(p.M, BM), cdiv(p.N, BN), 1);
  long long tiles = (long long)grid.x * grid.y;
  if (p.c_lower) tiles = (tiles + grid.x) / 2;
  p.ksplit = 1;
  if (tiles < s.sms && p.K >= 512) {
    int want = (int)((2 * s.sms + tiles - 1) / tiles);
    int ks = std::min(want, p.K / 128);
    if (ks > 64) ks = 64;
    while (ks > 1 && (size_t)ks * p.M * p.N * sizeof(float) > s.splitws_bytes) --ks;
    if (ks > 1) {
      p.ksplit = ks;
      p.ws = (float*)s.splitws;
      grid.z = ks;
    }
  }
  GEV_COUNT(s);
  if (shape == 1) gemm32_kernel<TI, TO, 128, 64><<<grid, 128, 0, s.stream>>>(p);
  else if (shape == 2) gemm32_kernel<TI, TO, 64, 128><<<grid, 128, 0, s.stream>>>(p);
  else gemm32_kernel<TI, TO, 128, 128><<<grid, 256, 0, s.stream>>>(p);
  if (p.ksplit > 1) {
    unsigned blocks = cdiv((long long)p.M * p.N, 256);
    if (blocks > 8u * s.sms) blocks = 8u * s.sms;
    GEV_COUNT(s);
    splitk_reduce32<TI, TO><<<blocks, 256, 0, s.stream>>>(p);
  }
}

template <> void gemm<float>(Sys& s, GemmP<float> p) { gemm32<float, float>(s, p, p.C, p.alpha, p.beta); }

template void gemm32<float, float>(Sys&, const GemmP<float>&, float*, float, float);
template void gemm32<float, double>(Sys&, const GemmP<float>&, double*, float, float);
template void gemm32<double, double>(Sys&, const GemmP<double>&, double*, float, float);
template void gemm32<double, float>(Sys&, const GemmP<double>&, float*, float, float);

}  // namespace gev
