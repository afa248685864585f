// Density matrix of the computed orbitals (section "Circumventing the eigenvalue problem") and its
// energy-weighted counterpart (section "ELSI": the interface returns either eigenpairs or these two
// matrices):
//
//   P_ij = sum_l g_l conj(C_il) C_jl,   g_l = f_l (occupation numbers) or f_l lambda_l,
//
// C_il being the coefficient of basis function i in orbital l (column l of C).
//
// One Hermitian rank-k product on the FP64 matrix-product engine per matrix:
//   W = C diag(g)                      (k_scale_cols, n x k in the handle's scratch),
//   M = W C^H, lower triangle only     (c_lower GEMM: n (n+1) k multiply-adds),
//   P = conj(M) = M^T                  (k_conj_mirror: the conjugate lands on the first index as in
//                                       the definition; both triangles written, diagonal real).
// For real data the conjugations are identities and P = M.
#include "common.cuh"

namespace gev {

namespace {

constexpr int TD = 32;

template <class T>
__global__ void k_scale_cols(int n, int k, const T* __restrict__ C, long long ldc, const double* __restrict__ occ,
                             const double* __restrict__ evals, int energy, T* __restrict__ W, long long ldw) {
  const long long total = (long long)n * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), l = (int)(t / n);
    double g = occ[l];
    if (energy) g *= evals[l];
    W[i + l * ldw] = g * C[i + l * ldc];
  }
}

// A holds M in its lower triangle (the upper triangle is not read).  In place, both triangles:
// lower (i > j) <- conj(M(i, j)), upper (i < j) <- M(j, i), diagonal <- Re M(i, i).  One block per
// 32 x 32 tile on or above the diagonal; it owns that upper tile and its transposed lower tile, so
// every element is read and written by one block, reads before the barrier, writes after it.
template <class T>
__global__ void k_conj_mirror(int n, T* A, long long lda) {
  __shared__ T tile[TD][TD + 1];
  const int bi = blockIdx.x * TD, bj = blockIdx.y * TD;
  if (bi > bj) return;
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    const int gi = bj + threadIdx.x, gj = bi + r;  // tile[r][x] = M(bj + x, bi + r)
    tile[r][threadIdx.x] = (gi < n && gj < n) ? A[gi + gj * lda] : zero_<T>();
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    const int ui = bi + threadIdx.x, uj = bj + r;  // upper element (ui, uj) <- M(uj, ui)
    if (ui < n && uj < n) {
      if (ui < uj) A[ui + uj * lda] = tile[threadIdx.x][r];
      else if (ui == uj) A[ui + uj * lda] = from_re<T>(re_(tile[threadIdx.x][r]));
    }
    const int li = bj + threadIdx.x, lj = bi + r;  // lower element (li, lj) <- conj(M(li, lj))
    if (li < n && lj < n && li > lj) A[li + lj * lda] = conj_(tile[r][threadIdx.x]);
  }
}

}  // namespace

template <class T>
int density(Sys& s, int k, const T* C, int ldc, const double* occ, const double* evals, T* P, int ldp, T* PE,
            int ldpe) {
  const int n = s.n;
  T* W = (T*)s.W1;  // n x k (the n x n scratch of the handle)
  const T one = from_re<T>(1.0), zero = zero_<T>();
  const long long total = (long long)n * k;
  unsigned blocks = (unsigned)cdiv(total, 256);
  if (blocks > 8u * s.sms) blocks = 8u * s.sms;
  const dim3 mg(cdiv(n, TD), cdiv(n, TD)), mb(TD, 8);
  for (int energy = 0; energy < (PE ? 2 : 1); ++energy) {
    T* out = energy ? PE : P;
    const int ldo = energy ? ldpe : ldp;
    GEV_COUNT(s);
    k_scale_cols<T><<<blocks, 256, 0, s.stream>>>(n, k, C, ldc, occ, evals, energy, W, n);
    GemmP<T> g = gp<T>(n, n, k, 0, 2, one, W, n, C, ldc, zero, out, ldo);
    g.c_lower = 1;
    gemm(s, g);
    GEV_COUNT(s);
    k_conj_mirror<T><<<mg, mb, 0, s.stream>>>(n, out, ldo);
  }
  return last_error();
}

template int density<double>(Sys&, int, const double*, int, const double*, const double*, double*, int, double*,
                             int);
template int density<zd>(Sys&, int, const zd*, int, const double*, const double*, zd*, int, zd*, int);

}  // namespace gev
