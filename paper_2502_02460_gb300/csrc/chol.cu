// Reduction steps 1-3 of the section "Current Status of the Implementation" and the final
// back-multiplication (Table 1: Choles., Invert, Multiply, Mult.):
//   potrf : S = L L^H, blocked right-looking; diagonal blocks factored (and inverted) in one CTA,
//           panel solve L21 = A21 L11^{-H} as a GEMM with the inverted diagonal block, trailing
//           update A22 -= L21 L21^H as a lower-only GEMM.
//   trtri : X = L^{-1}, blocked from the last block column: X21 = -X22 L21 X11.
//   hegst : A = X H X^H with H = B + B^H, B = tril(H) with halved diagonal:
//           P = X B (lower x lower -> lower), M = P X^H, A = M + M^H   (N^3 flops in total).
//   mult  : C = X^H Y (upper-triangular operand, N^2 k flops).
#include "common.cuh"

namespace gev {

namespace {

constexpr int NBMAX = 64;
constexpr int LDS = NBMAX + 1;

constexpr int SB = 16;  // sub-block of the blocked leaf factorisation and inverse

template <class T> __device__ __forceinline__ T shfl_(T v, int src);
template <> __device__ __forceinline__ double shfl_<double>(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <> __device__ __forceinline__ zd shfl_<zd>(zd v, int src) {
  return make_zd(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// X <- L^{-1} for the jb x jb lower-triangular L in shared memory (both column-major, ld LDS; X fully
// overwritten, zero above the diagonal), blocked by SB:
//   the diagonal blocks X_ii = L_ii^{-1}: one warp each, lane c forms column c by forward substitution;
//   then by block diagonals d = 1, 2, ...: S = sum_{k=j}^{i-1} L_ik X_kj for every block (i, j = i - d),
//   and X_ij = -X_ii S (block columns are independent; a diagonal needs the previous ones).
// tmp: (NBMAX / SB - 1) SB^2 elements of shared scratch.  Called by all threads of the block.
template <class T>
__device__ void inv_lower_blocked(int jb, const T* L, T* X, T* tmp) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nsb = (jb + SB - 1) / SB;
  for (int t = tid; t < NBMAX * LDS; t += blockDim.x) X[t] = zero_<T>();
  __syncthreads();
  if (warp < nsb) {
    const int k0 = warp * SB, bs = min(SB, jb - k0), c = lane;
    if (c < bs) {
      for (int i = c; i < bs; ++i) {
        T acc = (i == c) ? from_re<T>(1.0) : zero_<T>();
        for (int p = c; p < i; ++p) acc -= L[(k0 + i) + (k0 + p) * LDS] * X[(k0 + p) + (k0 + c) * LDS];
        X[(k0 + i) + (k0 + c) * LDS] = (1.0 / re_(L[(k0 + i) + (k0 + i) * LDS])) * acc;
      }
    }
  }
  __syncthreads();
  for (int d = 1; d < nsb; ++d) {
    const int nblk = nsb - d;  // blocks (i, j) = (j + d, j), j < nblk
    for (int t = tid; t < nblk * SB * SB; t += blockDim.x) {
      const int bj = t / (SB * SB), e = t % (SB * SB), r = e % SB, c = e / SB;
      const int bi = bj + d, i0 = bi * SB, j0 = bj * SB;
      T acc = zero_<T>();
      if (i0 + r < jb && j0 + c < jb)
        for (int k = j0; k < i0; ++k) acc += L[(i0 + r) + k * LDS] * X[k + (j0 + c) * LDS];
      tmp[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < nblk * SB * SB; t += blockDim.x) {
      const int bj = t / (SB * SB), e = t % (SB * SB), r = e % SB, c = e / SB;
      const int bi = bj + d, i0 = bi * SB, j0 = bj * SB;
      if (i0 + r < jb && j0 + c < jb) {
        T acc = zero_<T>();
        for (int q = 0; q <= r; ++q) acc += X[(i0 + r) + (i0 + q) * LDS] * tmp[bj * SB * SB + q + c * SB];
        X[(i0 + r) + (j0 + c) * LDS] = -acc;
      }
    }
    __syncthreads();
  }
}

// Factor the jb x jb diagonal block in place (lower) and write its inverse to Dinv, blocked by SB:
// for each SB-column sub-panel, one warp factors the SB x SB diagonal block in registers (lane i holds
// row i; the pivot column travels by shuffles), all threads solve the rows below against it and update
// the trailing block.  A non-positive pivot records its index (first one, atomicCAS) and stops.
template <class T>
__global__ void k_potrf_diag(int jb, T* A, long long lda, T* Dinv, long long ldd, int* status, int j0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* L = reinterpret_cast<T*>(smraw);
  T* X = L + NBMAX * LDS;
  T* tmp = X + NBMAX * LDS;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) fail = 0;
  for (int t = tid; t < jb * jb; t += blockDim.x) {
    int i = t % jb, j = t / jb;
    L[i + j * LDS] = (i >= j) ? A[i + j * lda] : zero_<T>();
  }
  __syncthreads();
  for (int kb = 0; kb < jb; kb += SB) {
    const int bs = min(SB, jb - kb);
    // (a) the diagonal block, by warp 0
    if (warp == 0) {
      T r[SB];
      const int i = lane;
#pragma unroll
      for (int j = 0; j < SB; ++j) r[j] = (i < bs && j <= i) ? L[(kb + i) + (kb + j) * LDS] : zero_<T>();
      int bad = -1;
#pragma unroll
      for (int p = 0; p < SB; ++p) {
        if (p < bs && bad < 0) {  // uniform over the warp
          const double dpp = re_(shfl_(r[p], p));
          if (!(dpp > 0.0)) {
            bad = p;
          } else {
            const double piv = sqrt(dpp);
            if (i == p) r[p] = from_re<T>(piv);
            else if (i > p) r[p] = (1.0 / piv) * r[p];
#pragma unroll
            for (int j = p + 1; j < SB; ++j) {
              const T ljp = shfl_(r[p], j);
              if (j < bs && i >= j && i < bs) r[j] -= mulc(r[p], ljp);
            }
          }
        }
      }
      if (bad >= 0) {
        if (lane == 0) {
          fail = 1;
          atomicCAS(&status[ST_NOT_SPD], 0, j0 + kb + bad + 1);
        }
      } else {
#pragma unroll
        for (int j = 0; j < SB; ++j)
          if (i < bs && j <= i) L[(kb + i) + (kb + j) * LDS] = r[j];
      }
    }
    __syncthreads();
    if (fail) return;
    const int r0 = kb + bs, nr = jb - r0;
    if (nr <= 0) break;
    // (b) rows below: L21 = A21 L11^{-H}, one thread per row
    for (int i = r0 + tid; i < jb; i += blockDim.x) {
      for (int p = 0; p < bs; ++p) {
        T x = L[i + (kb + p) * LDS];
        for (int q = 0; q < p; ++q) x -= mulc(L[i + (kb + q) * LDS], L[(kb + p) + (kb + q) * LDS]);
        L[i + (kb + p) * LDS] = (1.0 / re_(L[(kb + p) + (kb + p) * LDS])) * x;
      }
    }
    __syncthreads();
    // (c) trailing update A22 -= L21 L21^H (lower triangle)
    for (int t = tid; t < nr * nr; t += blockDim.x) {
      const int i = r0 + t % nr, j = r0 + t / nr;
      if (j <= i) {
        T acc = zero_<T>();
        for (int p = 0; p < bs; ++p) acc += mulc(L[i + (kb + p) * LDS], L[j + (kb + p) * LDS]);
        L[i + j * LDS] -= acc;
      }
    }
    __syncthreads();
  }
  inv_lower_blocked(jb, L, X, tmp);
  for (int t = tid; t < jb * jb; t += blockDim.x) {
    int i = t % jb, j = t / jb;
    A[i + j * lda] = (i >= j) ? L[i + j * LDS] : zero_<T>();
    Dinv[i + j * ldd] = X[i + j * LDS];
  }
}

// Invert every diagonal block of the lower-triangular L: block q -> Dinv[:, q*nb ...] (ld nb).
template <class T>
__global__ void k_inv_diag_blocks(int n, int nb, const T* A, long long lda, T* Dinv) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* L = reinterpret_cast<T*>(smraw);
  T* X = L + NBMAX * LDS;
  const int j0 = blockIdx.x * nb;
  const int jb = min(nb, n - j0);
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) {
    int i = t % jb, j = t / jb;
    L[i + j * LDS] = (i >= j) ? A[(j0 + i) + (long long)(j0 + j) * lda] : zero_<T>();
  }
  __syncthreads();
  inv_lower_blocked(jb, L, X, X + NBMAX * LDS);
  for (int t = threadIdx.x; t < jb * jb; t += blockDim.x) {
    int i = t % jb, j = t / jb;
    Dinv[i + (long long)(j0 + j) * nb] = X[i + j * LDS];
  }
}

template <class T> size_t diag_smem() { return sizeof(T) * (2 * NBMAX * LDS + (NBMAX / SB - 1) * SB * SB); }

template <class T> int set_smem_attrs() {
  GEV_TRY(allow_dyn_smem(k_potrf_diag<T>, diag_smem<T>()));
  GEV_TRY(allow_dyn_smem(k_inv_diag_blocks<T>, diag_smem<T>()));
  return 0;
}

}  // namespace

template <class T> int potrf(Sys& s, T* A, int lda) {
  const int n = s.n, nb = s.nb;
  GEV_TRY(set_smem_attrs<T>());
  T* Dinv = (T*)s.dinv;  // nb x nb (first block slot)
  T* P = (T*)s.Pn;       // n x nb panel
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zero = zero_<T>();
  for (int j = 0; j < n; j += nb) {
    const int jb = nb < n - j ? nb : n - j;
    T* Ajj = A + j + (long long)j * lda;
    GEV_COUNT(s);
    k_potrf_diag<T><<<1, 256, diag_smem<T>(), s.stream>>>(jb, Ajj, lda, Dinv, nb, s.status, j);
    GEV_TRY(last_error());
    const int m = n - j - jb;
    if (m <= 0) break;
    T* A21 = A + (j + jb) + (long long)j * lda;
    T* A22 = A + (j + jb) + (long long)(j + jb) * lda;
    // L21 = A21 L11^{-H}
    GemmP<T> g = gp<T>(m, jb, jb, 0, 2, one, A21, lda, Dinv, nb, zero, P, n);
    g.tri_b = 2;
    gemm(s, g);
    // A22 -= L21 L21^H (lower)
    g = gp<T>(m, m, jb, 0, 2, mone, P, n, P, n, one, A22, lda);
    g.c_lower = 1;
    gemm(s, g);
    GEV_TRY(copy2d<T>(s, m, jb, P, n, A21, lda));
  }
  GEV_TRY(zero_upper<T>(s, n, A, lda));
  return last_error();
}

// In-place inverse of the lower-triangular block A[o:o+sz, o:o+sz] (o, sz multiples of nb except
// at the end): X21 = -X22 (L21 X11) after inverting both diagonal halves, recursively, so the work
// is done by a few large triangular GEMMs instead of a chain of thin ones.
template <class T> void trtri_rec(Sys& s, T* A, int lda, int o, int sz, T* Dinv, T* W) {
  const int nb = s.nb;
  if (sz <= nb) {
    copy2d<T>(s, sz, sz, Dinv + (long long)o * nb, nb, A + o + (long long)o * lda, lda);
    return;
  }
  int n1 = (sz / 2 + nb - 1) / nb * nb;
  if (n1 >= sz) n1 = sz - nb;
  const int n2 = sz - n1;
  trtri_rec(s, A, lda, o, n1, Dinv, W);
  trtri_rec(s, A, lda, o + n1, n2, Dinv, W);
  T* X11 = A + o + (long long)o * lda;
  T* A21 = A + (o + n1) + (long long)o * lda;
  T* X22 = A + (o + n1) + (long long)(o + n1) * lda;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zero = zero_<T>();
  GemmP<T> g = gp<T>(n2, n1, n1, 0, 0, one, A21, lda, X11, lda, zero, W, s.n);  // W = L21 X11
  g.tri_b = 1;
  gemm(s, g);
  g = gp<T>(n2, n1, n2, 0, 0, mone, X22, lda, W, s.n, zero, A21, lda);          // X21 = -X22 W
  g.tri_a = 1;
  gemm(s, g);
}

template <class T> int trtri(Sys& s, T* A, int lda) {
  const int n = s.n, nb = s.nb;
  GEV_TRY(set_smem_attrs<T>());
  T* Dinv = (T*)s.dinv;  // nb x n: all diagonal-block inverses
  const int nblk = (n + nb - 1) / nb;
  GEV_COUNT(s);
  k_inv_diag_blocks<T><<<nblk, 256, diag_smem<T>(), s.stream>>>(n, nb, A, lda, Dinv);
  GEV_TRY(last_error());
  trtri_rec<T>(s, A, lda, 0, n, Dinv, (T*)s.W1);
  GEV_TRY(zero_upper<T>(s, n, A, lda));
  return last_error();
}

// Cholesky factorisation and inversion in one recursion: A (lower triangle of S = L L^H) <- X = L^{-1}.
//   X11 = L11^{-1}                       (recursion on the leading block)
//   L21 = A21 X11^H,  A22 <- A22 - L21 L21^H (lower)
//   X22 = L22^{-1}                       (recursion on the trailing block)
//   X21 = -X22 (L21 X11)
// Every product is a large triangular GEMM (the flat blocked algorithm's are K = nb wide); leaves of
// nb factor and invert a diagonal block.  L itself is not kept.  W: n x n scratch.
template <class T> void potrf_inv_rec(Sys& s, T* A, int lda, int o, int sz, T* W) {
  const int nb = s.nb;
  T* Aoo = A + o + (long long)o * lda;
  if (sz <= nb) {
    GEV_COUNT(s);
    k_potrf_diag<T><<<1, 256, diag_smem<T>(), s.stream>>>(sz, Aoo, lda, (T*)s.dinv, nb, s.status, o);
    copy2d<T>(s, sz, sz, (T*)s.dinv, nb, Aoo, lda);
    return;
  }
  int n1 = (sz / 2 + nb - 1) / nb * nb;
  if (n1 >= sz) n1 = sz - nb;
  const int n2 = sz - n1;
  potrf_inv_rec(s, A, lda, o, n1, W);
  T* X11 = Aoo;
  T* A21 = A + (o + n1) + (long long)o * lda;
  T* A22 = A + (o + n1) + (long long)(o + n1) * lda;
  const T one = from_re<T>(1.0), mone = from_re<T>(-1.0), zero = zero_<T>();
  GemmP<T> g = gp<T>(n2, n1, n1, 0, 2, one, A21, lda, X11, lda, zero, W, s.n);  // L21 = A21 X11^H
  g.tri_b = 2;
  gemm(s, g);
  g = gp<T>(n2, n2, n1, 0, 2, mone, W, s.n, W, s.n, one, A22, lda);             // A22 -= L21 L21^H
  g.c_lower = 1;
  gemm(s, g);
  copy2d<T>(s, n2, n1, W, s.n, A21, lda);
  potrf_inv_rec(s, A, lda, o + n1, n2, W);
  g = gp<T>(n2, n1, n1, 0, 0, one, A21, lda, X11, lda, zero, W, s.n);           // W = L21 X11
  g.tri_b = 1;
  gemm(s, g);
  g = gp<T>(n2, n1, n2, 0, 0, mone, A + (o + n1) + (long long)(o + n1) * lda, lda, W, s.n, zero, A21, lda);
  g.tri_a = 1;                                                                   // X21 = -X22 W
  gemm(s, g);
}

template <class T> int potrf_inv(Sys& s, T* A, int lda) {
  GEV_TRY(set_smem_attrs<T>());
  potrf_inv_rec<T>(s, A, lda, 0, s.n, (T*)s.W1);
  GEV_TRY(zero_upper<T>(s, s.n, A, lda));
  return last_error();
}

template <class T> int hegst(Sys& s, const T* H, int ldh, const T* X, int ldx, T* A, int lda) {
  const int n = s.n;
  T* B = (T*)s.W1;
  const T one = from_re<T>(1.0), zero = zero_<T>();
  GEV_TRY(tril_halfdiag<T>(s, n, H, ldh, B, n));
  // P = X B (both lower -> lower), into A
  GemmP<T> g = gp<T>(n, n, n, 0, 0, one, X, ldx, B, n, zero, A, lda);
  g.tri_a = 1;
  g.tri_b = 1;
  g.c_lower = 1;
  gemm(s, g);
  // M = P X^H, into B (full)
  g = gp<T>(n, n, n, 0, 2, one, A, lda, X, ldx, zero, B, n);
  g.tri_a = 1;
  g.tri_b = 2;
  gemm(s, g);
  GEV_TRY(herm_sum<T>(s, n, B, n, A, lda));
  return last_error();
}

template <class T> int mult(Sys& s, const T* X, int ldx, const T* Y, int ldy, int k, T* C, int ldc) {
  const int n = s.n;
  GemmP<T> g = gp<T>(n, k, n, 2, 0, from_re<T>(1.0), X, ldx, Y, ldy, zero_<T>(), C, ldc);
  g.tri_a = 2;
  gemm(s, g);
  return last_error();
}

#define GEV_INST(T)                                                     \
  template int potrf<T>(Sys&, T*, int);                                 \
  template int potrf_inv<T>(Sys&, T*, int);                             \
  template int trtri<T>(Sys&, T*, int);                                 \
  template int hegst<T>(Sys&, const T*, int, const T*, int, T*, int);   \
  template int mult<T>(Sys&, const T*, int, const T*, int, int, T*, int);
GEV_INST(double)
GEV_INST(zd)
#undef GEV_INST

}  // namespace gev
