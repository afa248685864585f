// FP64 / complex128 GEMM on the FP64 tensor path (DMMA, mma.sync m8n8k4) for every dense
// contraction of the solver: Cholesky trailing updates and panel solves, the inversion, the
// Multiply step A = X H X^H, the two-sided full->band updates, back-transforms and C = X^H Y.
//
// GB300 note: FP64 throughput is ~1 TFLOP/s for both DMMA and DFMA (measured), i.e. ~6.6 GFLOP/s
// per SM.  A 64x64 tile with a 16-deep k-slice performs 131 kFLOP per 16 KB of operands, so shared
// memory and L2 traffic are far below what the FP64 pipe can consume; the kernel is therefore a
// plain two-stage smem pipeline (registers prefetch the next k-slice while the current one runs).
// Triangular operands are handled per element at load time (the zero triangle is never read) and
// per tile (k ranges and output tiles that are identically zero are skipped), which is what makes
// TRMM / SYRK / the Multiply step cost their algorithmic flops.
#include <algorithm>

#include "common.cuh"

namespace gev {

namespace {

constexpr int BM = 64, BN = 64, NT = 128;
// k-depth of a shared-memory slice: 16 for real data, 8 for complex (re and im planes) so the
// double-buffered tiles stay within 48 KB of static shared memory.
template <class T> __host__ __device__ constexpr int bk_of() { return is_cx<T>::value ? 8 : 16; }

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <class T> struct Frag;
template <> struct Frag<double> {
  double acc[4][4][2];
};
template <> struct Frag<zd> {
  double acc[4][4][2];   // real part
  double acci[4][4][2];  // imaginary part
};

template <class T>
__device__ __forceinline__ T load_a(const GemmP<T>& p, int gi, int gk, int kb, int ke) {
  if (gi >= p.M || gk >= ke || gk < kb) return zero_<T>();
  if ((p.tri_a == 1 && gk > gi) || (p.tri_a == 2 && gk < gi)) return zero_<T>();
  T v = (p.ta == 0) ? p.A[gi + gk * p.lda] : p.A[gk + gi * p.lda];
  return p.ta == 2 ? conj_(v) : v;
}
template <class T>
__device__ __forceinline__ T load_b(const GemmP<T>& p, int gk, int gj, int kb, int ke) {
  if (gj >= p.N || gk >= ke || gk < kb) return zero_<T>();
  if ((p.tri_b == 1 && gk < gj) || (p.tri_b == 2 && gk > gj)) return zero_<T>();
  T v = (p.tb == 0) ? p.B[gk + gj * p.ldb] : p.B[gj + gk * p.ldb];
  return p.tb == 2 ? conj_(v) : v;
}


template <class T>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmP<T> p) {
  constexpr bool CX = is_cx<T>::value;
  constexpr int BK = bk_of<T>();
  constexpr int PER = BM * BK / NT;  // elements of each operand staged per thread
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  __shared__ double Asi[CX ? 2 : 1][BK][BM + 1];
  __shared__ double Bsi[CX ? 2 : 1][BK][BN + 1];

  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (p.c_lower && n0 > m0 + BM - 1) return;  // tile strictly above the diagonal

  int kb = 0, ke = p.K;
  if (p.tri_a == 1) ke = min(ke, m0 + BM);
  else if (p.tri_a == 2) kb = max(kb, m0);
  if (p.tri_b == 1) kb = max(kb, n0);
  else if (p.tri_b == 2) ke = min(ke, n0 + BN);
  if (p.ksplit > 1) {
    int chunk = ((p.K + p.ksplit - 1) / p.ksplit + BK - 1) / BK * BK;
    int z0 = blockIdx.z * chunk;
    kb = max(kb, z0);
    ke = min(ke, z0 + chunk);
  }
  kb = kb / BK * BK;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  Frag<T> f;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      f.acc[a][b][0] = f.acc[a][b][1] = 0.0;
      if constexpr (CX) f.acci[a][b][0] = f.acci[a][b][1] = 0.0;
    }

  // register staging of one k-slice
  T ra[PER], rb[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      int e = tid + r * NT;
      int i, k;
      if (p.ta == 0) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      ra[r] = load_a(p, m0 + i, k0 + k, kb, ke);
      int j, kk;
      if (p.tb == 0) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      rb[r] = load_b(p, k0 + kk, n0 + j, kb, ke);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      int e = tid + r * NT;
      int i, k;
      if (p.ta == 0) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      As[buf][k][i] = re_(ra[r]);
      if constexpr (CX) Asi[buf][k][i] = im_(ra[r]);
      int j, kk;
      if (p.tb == 0) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      Bs[buf][kk][j] = re_(rb[r]);
      if constexpr (CX) Bsi[buf][kk][j] = im_(rb[r]);
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
    for (int ks = 0; ks < BK; ks += 4) {
      const int kr = ks + (lane & 3);
      double a[4], b[4], ai[4], bi[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[buf][kr][wm + q * 8 + (lane >> 2)];
        b[q] = Bs[buf][kr][wn + q * 8 + (lane >> 2)];
        if constexpr (CX) {
          ai[q] = Asi[buf][kr][wm + q * 8 + (lane >> 2)];
          bi[q] = Bsi[buf][kr][wn + q * 8 + (lane >> 2)];
        }
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          dmma(f.acc[mi][ni][0], f.acc[mi][ni][1], a[mi], b[ni]);
          if constexpr (CX) {
            dmma(f.acc[mi][ni][0], f.acc[mi][ni][1], -ai[mi], bi[ni]);
            dmma(f.acci[mi][ni][0], f.acci[mi][ni][1], a[mi], bi[ni]);
            dmma(f.acci[mi][ni][0], f.acci[mi][ni][1], ai[mi], b[ni]);
          }
        }
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  // epilogue
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gi = m0 + wm + mi * 8 + (lane >> 2);
        const int gj = n0 + wn + ni * 8 + 2 * (lane & 3) + h;
        if (gi >= p.M || gj >= p.N) continue;
        if (p.c_lower && gi < gj) continue;
        T v;
        if constexpr (CX) v = make_zd(f.acc[mi][ni][h], f.acci[mi][ni][h]);
        else v = f.acc[mi][ni][h];
        if (p.ksplit > 1) {
          p.ws[(size_t)blockIdx.z * p.M * p.N + gi + (size_t)gj * p.M] = v;
        } else {
          T* c = &p.C[gi + gj * p.ldc];
          T out = p.alpha * v;
          if (p.beta != zero_<T>()) out += p.beta * (*c);
          *c = out;
        }
      }
}

// C = alpha * sum_z ws[z] + beta * C (fixed summation order: deterministic)
template <class T>
__global__ void splitk_reduce(GemmP<T> p) {
  const long long total = (long long)p.M * p.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % p.M), j = (int)(t / p.M);
    if (p.c_lower && i < j) continue;
    T s = zero_<T>();
    for (int z = 0; z < p.ksplit; ++z) s += p.ws[(size_t)z * total + t];
    T* c = &p.C[i + (long long)j * p.ldc];
    T out = p.alpha * s;
    if (p.beta != zero_<T>()) out += p.beta * (*c);
    *c = out;
  }
}

// sum over j = 0..J of max(0, min(ah, bh(j)) - max(al, bl(j))): the multiply-adds of one output row
// (bl/bh: the k range allowed by the zero pattern of op(B) in column j).
long double row_fmas(long long al, long long ah, int tri_b, long long J) {
  if (J < 0 || ah <= al) return 0.0L;
  long double s = 0.0L;
  if (tri_b == 0) return (long double)(ah - al) * (long double)(J + 1);
  if (tri_b == 1) {  // op(B)[k,j] = 0 for k < j
    const long long j1 = std::min(J, al);
    if (j1 >= 0) s += (long double)(ah - al) * (long double)(j1 + 1);
    const long long lo = std::max(al + 1, 0LL), hi = std::min(J, ah - 1);
    if (hi >= lo) s += (long double)(hi - lo + 1) * ah - (long double)(lo + hi) * (hi - lo + 1) / 2.0L;
    return s;
  }
  // tri_b == 2: op(B)[k,j] = 0 for k > j
  const long long lo = std::max(al, 0LL), hi = std::min(J, ah - 1);
  if (hi >= lo) s += (long double)(lo + hi) * (hi - lo + 1) / 2.0L + (long double)(1 - al) * (hi - lo + 1);
  const long long lo2 = std::max(ah, 0LL);
  if (J >= lo2) s += (long double)(ah - al) * (long double)(J - lo2 + 1);
  return s;
}

template <class T> double algorithmic_flops(const GemmP<T>& p) {
  long double fma = 0.0L;
  for (long long i = 0; i < p.M; ++i) {
    long long al = (p.tri_a == 2) ? i : 0;
    long long ah = (p.tri_a == 1) ? std::min<long long>(p.K, i + 1) : p.K;
    const long long J = p.c_lower ? std::min<long long>(p.N - 1, i) : p.N - 1;
    fma += row_fmas(al, ah, p.tri_b, J);
  }
  return (double)(fma * (is_cx<T>::value ? 8.0L : 2.0L));
}

}  // namespace

template <class T> void gemm(Sys& s, GemmP<T> p) {
  if (p.M <= 0 || p.N <= 0) return;
  if constexpr (!is_cx<T>::value) {
    if (p.lowp) {  // mixed form: FP64 operands, FP32 arithmetic
      gemm32<double, double>(s, p, p.C, (float)p.alpha, (float)p.beta);
      return;
    }
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (s.account) {
    const size_t need = 2 * (size_t)(s.gemm_used + 1);
    while (s.gemm_ev.size() < need) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      s.gemm_ev.push_back(e);
    }
    ev0 = s.gemm_ev[2 * s.gemm_used];
    ev1 = s.gemm_ev[2 * s.gemm_used + 1];
    if ((int)s.gemm_fl.size() <= s.gemm_used) s.gemm_fl.resize(s.gemm_used + 1);
    s.gemm_fl[s.gemm_used] = algorithmic_flops(p);
    cudaEventRecord(ev0, s.stream);
  }
  bool emulated = false;
  if constexpr (!is_cx<T>::value) {
    if (s.emu_fp64) {  // FP64 product from BF16 digit planes on the tensor cores
      gemm_f64_emulated(s, p);
      emulated = true;
    }
  } else {
    if (s.emu_fp64 && p.alpha.y == 0.0 && p.beta.y == 0.0) {  // through the real embedding
      gemm_c128_emulated(s, p);
      emulated = true;
    }
  }
  if (emulated) {
    if (s.account) {
      cudaEventRecord(ev1, s.stream);
      ++s.gemm_used;
    }
    return;
  }
  dim3 grid(cdiv(p.M, BM), cdiv(p.N, BN), 1);
  long long tiles = (long long)grid.x * grid.y;
  if (p.c_lower) tiles = (tiles + grid.x) / 2;
  p.ksplit = 1;
  p.ws = nullptr;
  // split K when the output has too few tiles to fill the GPU and K is long
  if (tiles < s.sms && p.K >= 512) {
    int want = (int)((2 * s.sms + tiles - 1) / tiles);
    int maxk = p.K / 128;
    int ks = want < maxk ? want : maxk;
    if (ks > 64) ks = 64;
    size_t need = (size_t)ks * p.M * p.N * sizeof(T);
    while (ks > 1 && need > s.splitws_bytes) {
      --ks;
      need = (size_t)ks * p.M * p.N * sizeof(T);
    }
    if (ks > 1) {
      p.ksplit = ks;
      p.ws = (T*)s.splitws;
      grid.z = ks;
    }
  }
  GEV_COUNT(s);
  gemm_kernel<T><<<grid, NT, 0, s.stream>>>(p);
  if (p.ksplit > 1) {
    long long total = (long long)p.M * p.N;
    unsigned blocks = cdiv(total, 256);
    if (blocks > 8u * s.sms) blocks = 8u * s.sms;
    GEV_COUNT(s);
    splitk_reduce<T><<<blocks, 256, 0, s.stream>>>(p);
  }
  if (s.account) {
    cudaEventRecord(ev1, s.stream);
    ++s.gemm_used;
  }
}

// Sum the timed GEMM launches of the current call (stream must be synchronised).
void gemm_account(Sys& s, int* calls, double* ms, double* flops) {
  double tm = 0.0, fl = 0.0;
  for (int i = 0; i < s.gemm_used; ++i) {
    float t = 0.f;
    cudaEventElapsedTime(&t, s.gemm_ev[2 * i], s.gemm_ev[2 * i + 1]);
    tm += t;
    fl += s.gemm_fl[i];
  }
  *calls = s.gemm_used;
  *ms = tm;
  *flops = fl;
}

template void gemm<double>(Sys&, GemmP<double>);
template void gemm<zd>(Sys&, GemmP<zd>);

}  // namespace gev
