// One-stage Householder tridiagonalisation ("ELPA1", section "Usability and Tutorials", where the
// one-stage solver is reported as the faster GPU choice when all, or most, eigenpairs are wanted), and
// its back-transform Y = Q Z.
//
//   A = Q T Q^H,  Q = H_0 H_1 ... H_{n-2},  H_j = I - tau_j v_j v_j^H,  v_j = 0 above row j+1,
//   v_j(j+1) = 1,  H_j^H A(j+1:, j) = (e_j, 0, ..., 0)^T with e_j real.
//
// Blocked in panels of nb columns as in the classical aggregated reduction: inside a panel the
// trailing matrix is left untouched and the panel's reflectors are kept as the pair (V, W) with
//   A_current = A - V W^H - W V^H,
// so each column costs one Hermitian matrix-vector product with the ORIGINAL trailing block plus
// rank-2c corrections:
//   a(j:, j)  -= V(j:, 0:c) W(j, 0:c)^H + W(j:, 0:c) V(j, 0:c)^H         (column update)
//   (v, tau, e_j) from a(j+1:, j)                                         (reflector)
//   p = A(j+1:, j+1:) v - V (W^H v) - W (V^H v)                          (symv + corrections)
//   w = tau p + alpha v,  alpha = -|tau|^2 (v^H p) / 2                    (the new column of W)
// and after the panel the trailing block takes the rank-2nb update A22 -= [V W] [W V]^H as ONE
// product on the tensor-core engine.
//
// GB300 layout: one cooperative kernel per panel.  The trailing block's lower triangle is read in
// 64 x 64 tiles spread over all blocks (each tile serves both the direct product A_IL v_L and the
// reflected one A_IL^H v_I: the lower triangle is read once per column); tile partial sums go to
// one 64-value slot per (row tile, partner tile) and are summed in a fixed order, so the result
// does not depend on timing.  Three bounded grid barriers per column: after the column update
// (norm), after the symv (partials), after the new W column (alpha).  The panel's reflectors go to
// the handle's V1 (unit first entry, zero above) and the panel's compact-WY factor T (Q_panel =
// I - V T V^H, built from the same inner products V^H v) to T1, for the back-transform, which
// applies groups of panels as three tensor-core products each (bt_he2hb).
#include <algorithm>

#include "common.cuh"
#include "coop.cuh"

namespace gev {

namespace {

constexpr int NT = 256;
constexpr int TS = 64;   // symv tile
constexpr int TLD = 65;  // its shared-memory leading dimension

constexpr int STG = TS * TLD + 2 * TS;  // shared-memory elements: the tile and its two 64-entry v segments

template <class T> struct TdArgs {
  int n, j0, pw, nb, npd;
  T* A;
  long long lda;
  T* V1;   // reflectors, n x n (column j = v_j)
  T* YV;   // n x 2nb: [V | W]
  T* VY;   // n x 2nb: [W | V]
  long long ldw;
  double* d;
  double* e;
  T* Tp;       // nb x nb compact-WY factor of the panel
  T* slots;    // symv tile partial sums: ntile^2 x 64
  T* dparts;   // npd x 2nb: V^H v, W^H v partial sums
  double* nparts;  // G: ||x||^2 partial sums
  T* aparts;   // G: w0^H v partial sums
  T* piv;      // w0 at the pivot row of the column just finished
  GridBar gb;
};

__device__ __forceinline__ float shx(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shx(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ zd shx(zd v, int m) {
  return make_zd(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <class T> __device__ __forceinline__ T group_sum(T v, int width) {
  for (int m = width >> 1; m > 0; m >>= 1) v += shx(v, m);
  return v;
}

// sum of f(i) over i = start, start + step, ... < end with U independent accumulators, so that U
// loads are in flight (the terms are L2 reads); the order is fixed by the arguments
template <class T, int U = 4, class F> __device__ __forceinline__ T ssum(int start, int end, int step, F f) {
  T acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc[u] = zero_<T>();
  int i = start;
  for (; i + (U - 1) * step < end; i += U * step) {
    T x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = f(i + u * step);
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] += x[u];
  }
  for (; i < end; i += step) acc[0] += f(i);
  T t = zero_<T>();
#pragma unroll
  for (int u = 0; u < U; ++u) t += acc[u];
  return t;
}

// block-wide sum in a fixed order; the result is returned to every thread
template <class T> __device__ T block_sum_all(T v, T* red) {
  v = group_sum(v, 32);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = zero_<T>();
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// threads per row for row-parallel phases: a power of two <= 32 with (threads per row) * rows ~ NT
__device__ __forceinline__ int rows_tpr(int nrows) {
  int t = 32;
  while (t > 1 && t * nrows > NT) t >>= 1;
  return t;
}

template <class T>
__global__ void __launch_bounds__(NT, 2) k_td_panel(TdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* As = reinterpret_cast<T*>(smraw);  // TS x TLD tile, then the two TS-entry v segments
  T* vI = As + TS * TLD;
  T* vL = vI + TS;
  T* redD = As + STG;  // 4 x TS
  T* redT = redD + 4 * TS;
  __shared__ T s_vj[128], s_wj[128];   // pivot row of V and W (conjugated)
  __shared__ T s_vhv[128], s_whv[128]; // V^H v, W^H v
  __shared__ T s_red[NT / 32];
  __shared__ double s_redd[NT / 32];
  __shared__ T s_tau, s_scale;

  const int n = a.n, j0 = a.j0, nb = a.nb, G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const long long ldw = a.ldw, lda = a.lda;
  T* Vp = a.YV;
  T* Wp = a.YV + (long long)nb * ldw;
  T* Wq = a.VY;                          // second copy of W
  T* Vq = a.VY + (long long)nb * ldw;    // second copy of V
  const int R = (n - j0 + G - 1) / G;
  const int rlo = j0 + g * R, rhi = min(n, rlo + R);
  const T one = from_re<T>(1.0);
  T tau_prev = zero_<T>();

  for (int c = 0; c < a.pw; ++c) {
    const int j = j0 + c;
    // ================= A: finish W(:, c-1); update column j; norm of x = a(j+2:, j)
    // (every load of this phase that does not depend on alpha_{c-1} is issued first, together)
    T part = zero_<T>(), pivv = zero_<T>(), vjl = zero_<T>(), wjl = zero_<T>();
    T wfin = zero_<T>(), vfin = zero_<T>();
    const int ifin = max(rlo, j) + tid;  // this thread's first own row of W(:, c-1)
    if (c > 0) {
      for (int q = tid; q < G; q += NT) part += ldcg_(&a.aparts[q]);
      pivv = ldcg_(a.piv);
      if (ifin < rhi) {
        const long long o = ifin + (long long)(c - 1) * ldw;
        wfin = ldcg_(&Wp[o]);
        vfin = ldcg_(&Vp[o]);
      }
    }
    if (tid < c) {
      vjl = ldcg_(&Vp[j + (long long)tid * ldw]);
      if (tid < c - 1) wjl = ldcg_(&Wp[j + (long long)tid * ldw]);
    }
    if (c > 0) {
      const T dot = block_sum_all(part, s_red);
      const T alpT = from_re<T>(-0.5 * re_(tau_prev * dot));
      for (int i = ifin; i < rhi; i += NT) {
        const long long o = i + (long long)(c - 1) * ldw;
        const T w = (i == ifin ? wfin : ldcg_(&Wp[o])) + alpT * (i == ifin ? vfin : ldcg_(&Vp[o]));
        Wp[o] = w;
        Wq[o] = w;
      }
      if (tid == c - 1) wjl = pivv + alpT;  // v_{c-1}(j) = 1
    }
    if (tid < c) {
      s_vj[tid] = conj_(vjl);
      s_wj[tid] = conj_(wjl);
    }
    __syncthreads();
    double nrm = 0.0;
    {
      const int r0 = max(rlo, j), nr = max(0, rhi - r0);
      const int tpr = rows_tpr(nr), lane = tid % tpr, rpass = NT / tpr;
      for (int base = 0; base < nr; base += rpass) {
        const int i = r0 + base + tid / tpr;
        const bool ok = i < rhi;
        T acc = zero_<T>();
        if (ok)
          acc = ssum<T>(lane, c, tpr, [&](int l) {
            const long long o = i + (long long)l * ldw;
            return ldcg_(&Vp[o]) * s_wj[l] + ldcg_(&Wp[o]) * s_vj[l];
          });
        acc = group_sum(acc, tpr);
        if (ok && lane == 0) {
          T* pa = &a.A[i + (long long)j * lda];
          T x = *pa - acc;
          if (i == j) {
            x = from_re<T>(re_(x));
            a.d[j] = re_(x);
          }
          *pa = x;
          if (i >= j + 2) nrm += abs2_(x);
        }
      }
    }
    if (j == n - 1) break;  // the last diagonal entry: no reflector
    {
      const double tot = block_sum_all(nrm, s_redd);
      if (tid == 0) a.nparts[g] = tot;
    }
    if (!grid_sync(a.gb, 201)) return;
    // ================= B: reflector; symv over the lower tiles; V^H v, W^H v
    {
      double part = 0.0;
      for (int q = tid; q < G; q += NT) part += ldcg_(&a.nparts[q]);
      const double xn = block_sum_all(part, s_redd);
      if (tid == 0) {
        const T alpha = ldcg_(&a.A[(j + 1) + (long long)j * lda]);
        const bool trivial = (xn == 0.0 && im_(alpha) == 0.0);
        double beta;
        if (trivial) {
          beta = re_(alpha);
          s_tau = zero_<T>();
          s_scale = zero_<T>();
        } else {
          const double nr = sqrt(abs2_(alpha) + xn);
          beta = re_(alpha) >= 0.0 ? -nr : nr;
          const T bt = from_re<T>(beta);
          s_tau = div_(bt - alpha, bt);
          s_scale = div_(one, alpha - bt);
        }
        if (g == 0) a.e[j] = beta;
      }
      __syncthreads();
    }
    const T tau = s_tau, scale = s_scale;
    const T* colj = a.A + (long long)j * lda;
    auto vfun = [&](int i) -> T {
      if (i <= j || i >= n) return zero_<T>();
      if (i == j + 1) return one;
      return scale * ldcg_(&colj[i]);
    };
    for (int i = max(rlo, j + 1) + tid; i < rhi; i += NT) {
      const T v = vfun(i);
      a.V1[i + (long long)j * ldw] = v;
      Vp[i + (long long)c * ldw] = v;
      Vq[i + (long long)c * ldw] = v;
    }
    // symv: tiles (I, L), I >= L, of rows/columns [t0*TS, n), entries outside [j+1, n) masked
    const int t0 = (j + 1) / TS;
    const int ntile = (n + TS - 1) / TS - t0;
    const long long ntt = (long long)ntile * (ntile + 1) / 2;
    // tile t -> (I, L) with t = I (I + 1) / 2 + L
    // (the first guess in FP32: FP64 arithmetic is scarce on this part and t < 2^24)
    auto tile_of = [&](long long t, int& I, int& L) {
      I = (int)((__fsqrt_rn(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while ((long long)I * (I + 1) / 2 > t) --I;
      while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
      L = (int)(t - (long long)I * (I + 1) / 2);
    };
    const int gt = g - a.npd, Gt = G - a.npd;  // tile blocks: g >= npd
    // the tile's products from shared memory (tile Ab, v_L / v_I in vl / vi); partial sums to
    // the two slots
    auto tile_products = [&](const T* Ab, const T* vl, const T* vi, int I, int L) {
      const bool diag = (I == L);
      {
        const int x = tid & (TS - 1), q = tid >> 6;
        T sd = zero_<T>(), st = zero_<T>();
#pragma unroll 4
        for (int k = 0; k < 16; ++k) {
          const int y = q * 16 + k;
          sd += Ab[x + y * TLD] * vl[y];                       // row x of the tile
          if (!diag || y > x) st += conj_(Ab[y + x * TLD]) * vi[y];  // column x, reflected
        }
        redD[q * TS + x] = sd;
        redT[q * TS + x] = st;
      }
      __syncthreads();
      // (the next tile's shared-memory stores touch Ab, vl and vi only; the reduction buffers are
      // written again after the next tile's first barrier, when every thread has left this one)
      if (tid < TS) {
        T o = redD[tid] + redD[TS + tid] + redD[2 * TS + tid] + redD[3 * TS + tid];
        if (diag) o += redT[tid] + redT[TS + tid] + redT[2 * TS + tid] + redT[3 * TS + tid];
        a.slots[((long long)I * ntile + L) * TS + tid] = o;
      } else if (!diag && tid < 2 * TS) {
        const int x = tid - TS;
        a.slots[((long long)L * ntile + I) * TS + x] = redT[x] + redT[TS + x] + redT[2 * TS + x] + redT[3 * TS + x];
      }
    };
    {
      // this thread's 16 entries of tile (I, L): row r = tid % 64, columns 16 q .. 16 q + 15
      T nx[16];
      T nvr = zero_<T>();  // threads < 128: the raw column-j entry behind the next tile's v_L / v_I
      auto load_tile = [&](int I, int L) {
        const int r = tid & (TS - 1), q = tid >> 6;
        const int rb = (t0 + I) * TS, cb = (t0 + L) * TS, row = rb + r;
        const bool diag = (I == L), rok = row > j && row < n;
        if (tid < 2 * TS) {
          const int iv = tid < TS ? cb + tid : rb + tid - TS;
          nvr = (iv > j + 1 && iv < n) ? ldcg_(&colj[iv]) : zero_<T>();
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int l = q * 16 + k, col = cb + l;
          T val = zero_<T>();
          if (rok && col > j && col < n && (!diag || r >= l)) {
            val = a.A[row + (long long)col * lda];
            if (diag && r == l) val = from_re<T>(re_(val));
          }
          nx[k] = val;
        }
      };
      if (gt >= 0 && gt < ntt) {
        int I, L;
        tile_of(gt, I, L);
        load_tile(I, L);
      }
      // the next tile's entries are loaded into registers while this one is multiplied from shared memory
      for (long long t = gt; gt >= 0 && t < ntt; t += Gt) {
        int I, L;
        tile_of(t, I, L);
        const int rb = (t0 + I) * TS, cb = (t0 + L) * TS;
        {
          const int r = tid & (TS - 1), q = tid >> 6;
#pragma unroll
          for (int k = 0; k < 16; ++k) As[r + (q * 16 + k) * TLD] = nx[k];
          if (tid < 2 * TS) {
            const int iv = tid < TS ? cb + tid : rb + tid - TS;
            const T v = iv == j + 1 ? one : (iv > j + 1 && iv < n ? scale * nvr : zero_<T>());
            if (tid < TS) vL[tid] = v;
            else vI[tid - TS] = v;
          }
        }
        __syncthreads();
        if (t + Gt < ntt) {
          int I2, L2;
          tile_of(t + Gt, I2, L2);
          load_tile(I2, L2);
        }
        tile_products(As, vL, vI, I, L);
      }
    }
    __syncthreads();
    // V^H v and W^H v over rows [j+1, n) on the npd dot blocks (no tiles): warp w sums values
    // 16 w .. 16 w + 15 (value u < c: column u of V, else column u - c of W), lanes over rows, the
    // sixteen column loads of a row in flight together
    if (g < a.npd && c > 0) {
      const int m = n - (j + 1);
      const int Rd = (m + a.npd - 1) / a.npd;
      const int lo = j + 1 + g * Rd, hi = min(n, lo + Rd);
      const int lane = tid & 31, vb = (tid >> 5) * 16;
      if (vb < 2 * c) {
        T acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = zero_<T>();
        for (int i = lo + lane; i < hi; i += 32) {
          const T vi = vfun(i);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int val = vb + u;
            if (val < 2 * c) {
              const T* col = val < c ? Vp + (long long)val * ldw : Wp + (long long)(val - c) * ldw;
              acc[u] += cmul(ldcg_(&col[i]), vi);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int val = vb + u;
          const T r = group_sum(acc[u], 32);
          if (lane == 0 && val < 2 * c) a.dparts[(long long)g * 2 * nb + (val < c ? val : nb + val - c)] = r;
        }
      }
    }
    if (!grid_sync(a.gb, 202)) return;
    // ================= C: p = slots + corrections; w0 = tau p; T column c
    for (int l = tid; l < 2 * c; l += NT) {
      const int ll = l % c;
      const int off = l < c ? ll : nb + ll;
      const T s = ssum<T, 8>(0, a.npd, 1, [&](int q) { return ldcg_(&a.dparts[(long long)q * 2 * nb + off]); });
      if (l < c) s_vhv[ll] = s;
      else s_whv[ll] = s;
    }
    __syncthreads();
    if (g == 0)  // column c of T, raw: (V^H v_c above the diagonal, tau_c on it), finished at the end
      for (int i = tid; i < nb; i += NT) a.Tp[i + (long long)c * nb] = i < c ? s_vhv[i] : (i == c ? tau : zero_<T>());
    T dotp = zero_<T>();
    {
      const int r0 = max(rlo, j + 1), nr = max(0, rhi - r0);
      const int tpr = rows_tpr(nr), lane = tid % tpr, rpass = NT / tpr;
      for (int base = 0; base < nr; base += rpass) {
        const int i = r0 + base + tid / tpr;
        const bool ok = i < rhi;
        T acc = zero_<T>();
        if (ok) {
          const int Ri = i / TS - t0, r = i % TS;
          const T* sl = a.slots + (long long)Ri * ntile * TS + r;
          acc = ssum<T, 8>(lane, ntile, tpr, [&](int X) { return ldcg_(&sl[(long long)X * TS]); });
          acc -= ssum<T>(lane, c, tpr, [&](int l) {
            const long long o = i + (long long)l * ldw;
            return ldcg_(&Vp[o]) * s_whv[l] + ldcg_(&Wp[o]) * s_vhv[l];
          });
        }
        acc = group_sum(acc, tpr);
        if (ok && lane == 0) {
          const long long o = i + (long long)c * ldw;
          const T w0 = tau * acc;
          Wp[o] = w0;
          Wq[o] = w0;
          if (i == j + 1) *a.piv = w0;
          dotp += cmul(w0, ldcg_(&Vp[o]));
        }
      }
    }
    {
      const T tot = block_sum_all(dotp, s_red);
      if (tid == 0) a.aparts[g] = tot;
    }
    tau_prev = tau;
    if (!grid_sync(a.gb, 203)) return;
    if (c == a.pw - 1) {
      // finish the panel's last W column for the trailing update
      T part = zero_<T>();
      for (int q = tid; q < G; q += NT) part += ldcg_(&a.aparts[q]);
      const T dot = block_sum_all(part, s_red);
      const T alpT = from_re<T>(-0.5 * re_(tau * dot));
      for (int i = max(rlo, j + 1) + tid; i < rhi; i += NT) {
        const long long o = i + (long long)c * ldw;
        const T w = ldcg_(&Wp[o]) + alpT * ldcg_(&Vp[o]);
        Wp[o] = w;
        Wq[o] = w;
      }
    }
  }
  // the panel's compact-WY factor from its raw columns (forward accumulation):
  //   T(0:c, c) = -tau_c T(0:c, 0:c) (V(:, 0:c)^H v_c),   T(c, c) = tau_c
  if (g == 0) {
    const int nr = min(a.pw, n - 1 - j0);  // reflectors in this panel
    T* Ts = As;                            // nb x nb in shared memory (ld nb)
    for (int q = tid; q < nb * nb; q += NT) {
      const int i = q % nb, cc = q / nb;
      Ts[q] = (i < nr && cc < nr) ? a.Tp[i + (long long)cc * nb] : zero_<T>();
    }
    __syncthreads();
    for (int cc = 1; cc < nr; ++cc) {
      if (tid < cc) vI[tid] = Ts[tid + cc * nb];
      __syncthreads();
      const T tc = Ts[cc + cc * nb];
      if (tid < cc) {
        T acc = zero_<T>();
        for (int l = tid; l < cc; ++l) acc += Ts[tid + l * nb] * vI[l];
        Ts[tid + cc * nb] = -(tc * acc);
      }
      __syncthreads();
    }
    for (int q = tid; q < nb * nb; q += NT) a.Tp[q] = Ts[q];
  }
}

template <class T>
__global__ void k_real_to(int n, int k, const double* Z, long long ldz, T* Y, long long ldy) {
  const long long total = (long long)n * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), c = (int)(t / n);
    Y[i + c * ldy] = from_re<T>(Z[i + c * ldz]);
  }
}

template <class T> size_t td_smem() { return sizeof(T) * ((size_t)STG + 8 * TS) + 64; }

}  // namespace

template <class T> int he2td(Sys& s, T* A, int lda) {
  const int n = s.n, nb = s.b;
  if (nb > 64 || (size_t)4 * n * nb > (size_t)8 * s.b * n) return GEV_ERR_UNSUPPORTED;
  const size_t smem = td_smem<T>();
  GEV_TRY(set_dyn_smem((const void*)k_td_panel<T>, smem));
  int per_sm = 0;
  GEV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_td_panel<T>, NT, smem));
  if (per_sm < 1) return GEV_ERR_UNSUPPORTED;
  const int gmax = std::min(per_sm, 2) * s.sms;
  T* V1 = (T*)s.V1;
  GEV_CUDA_TRY(cudaMemsetAsync(V1, 0, sizeof(T) * (size_t)n * n, s.stream));
  GEV_CUDA_TRY(cudaMemsetAsync(s.e, 0, sizeof(double) * n, s.stream));
  T* YV = (T*)s.Pn;
  T* VY = YV + (size_t)n * 2 * nb;
  const size_t ntl = (size_t)(n + TS - 1) / TS;
  if (ntl * ntl * TS * sizeof(T) > s.q_bytes) return GEV_ERR_UNSUPPORTED;
  char* pw_base = (char*)s.panelws;
  TdArgs<T> a{};
  a.n = n;
  a.nb = nb;
  a.A = A;
  a.lda = lda;
  a.V1 = V1;
  a.YV = YV;
  a.VY = VY;
  a.ldw = n;
  a.d = s.d;
  a.e = s.e;
  a.slots = (T*)s.Q;
  a.nparts = (double*)pw_base;                       // gmax doubles
  a.aparts = (T*)(pw_base + 2048 * 8);               // gmax values
  a.piv = (T*)(pw_base + 2048 * 8 + 2048 * 16);
  a.dparts = (T*)(pw_base + 2048 * 8 + 2048 * 16 + 256);  // 32 x 2nb values
  if ((size_t)2048 * 8 + 2048 * 16 + 256 + (size_t)32 * 2 * nb * sizeof(T) > s.panelws_bytes || gmax > 2048 ||
      gmax < 2)
    return GEV_ERR_UNSUPPORTED;
  a.gb = GridBar{(unsigned*)&s.status[ST_BARRIER_CNT], (unsigned*)&s.status[ST_BARRIER_GEN], s.status,
                 &s.status[ST_ABORT]};
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0);
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int pw = std::min(nb, n - j0);
    const long long nt0 = (long long)((n + TS - 1) / TS - (j0 + 1) / TS);
    const long long ntt = nt0 * (nt0 + 1) / 2;
    // dot blocks (V^H v, W^H v over ~128 rows each, at most 32) beside the tile blocks
    const int npd = std::max(1, std::min(32, (n - j0) / 128));
    const int G = npd + (int)std::min<long long>(gmax - npd, std::max<long long>(ntt, 1));
    a.j0 = j0;
    a.pw = pw;
    a.npd = npd;
    a.Tp = (T*)s.T1 + (size_t)(j0 / nb) * nb * nb;
    GEV_CUDA_TRY(cudaMemsetAsync(&s.status[ST_BARRIER_CNT], 0, 2 * sizeof(int), s.stream));
    void* args[] = {&a};
    GEV_COUNT(s);
    GEV_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_td_panel<T>, dim3(G), dim3(NT), args, smem, s.stream));
    if (j0 + pw < n) {
      // A22 -= [V W] [W V]^H over rows/columns [j0 + nb, n), lower triangle
      const int r0 = j0 + nb, m = n - r0;
      GemmP<T> g = gp<T>(m, m, 2 * nb, 0, 2, mone, YV + r0, n, VY + r0, n, one, A + r0 + (long long)r0 * lda, lda);
      g.c_lower = 1;
      gemm(s, g);
    }
  }
  s.q1_pw = nb;
  s.q1_off = 1;
  s.q1_nrefl = n - 1;
  s.nsbr_panels = (n - 1 + nb - 1) / nb;
  s.have_band = false;
  s.have_tridiag_refl = false;
  s.one_stage_used = true;
  return stop_on_timeout(s);
}

// Y = Q Z for the reflectors of the last he2td on this handle (Z real n x k)
template <class T> int back_td(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy) {
  const int n = s.n;
  const long long total = (long long)n * k;
  unsigned blocks = cdiv(total, 256);
  if (blocks > 16u * s.sms) blocks = 16u * s.sms;
  GEV_COUNT(s);
  k_real_to<T><<<blocks, 256, 0, s.stream>>>(n, k, Z, ldz, Y, ldy);
  GEV_TRY(last_error());
  return bt_he2hb<T>(s, Y, ldy, k);
}

template int he2td<float>(Sys&, float*, int);
template int he2td<double>(Sys&, double*, int);
template int he2td<zd>(Sys&, zd*, int);
template int back_td<float>(Sys&, const double*, int, int, float*, int);
template int back_td<double>(Sys&, const double*, int, int, double*, int);
template int back_td<zd>(Sys&, const double*, int, int, zd*, int);

}  // namespace gev
