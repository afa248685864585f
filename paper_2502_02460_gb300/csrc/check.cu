// Accuracy of a solve measured on the device (gev_opts.check): the residual
//   ||H C - S C Lambda||_1 / (||H||_1 ||C||_1)
// and the orthogonality ||C^H S C - I||_1 of the solution of Eq. 2, from the caller's H and S (lower
// triangles) with the handle's FP64 product engine.  H C is formed as (B + B^H) C with B = tril(H),
// diagonal halved, so the upper triangle is never read; likewise S C.  The 1-norm of a Hermitian H is
// its largest column sum of moduli, accumulated from the lower triangle (each off-diagonal entry
// counts for its column and, conjugated, for its row's column).
#include "common.cuh"

namespace gev {

namespace {

constexpr int TD = 32;

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;  // thread 0
}

// colsum[j] += sum_i |H(i,j)| of the full Hermitian H, from the lower triangle: tile (bi, bj) with
// bi >= bj adds the column sums of its lower entries to their columns and, for strictly lower
// entries, their row sums to the columns of the mirrored entries.
template <class T>
__global__ void k_herm_colsum(int n, const T* __restrict__ H, long long ldh, double* colsum) {
  const int bi = blockIdx.x * TD, bj = blockIdx.y * TD;
  if (bi + TD - 1 < bj) return;
  __shared__ double rows[TD];
  __shared__ double cols[TD];
  if (threadIdx.y == 0) { rows[threadIdx.x] = 0.0; cols[threadIdx.x] = 0.0; }
  __syncthreads();
  const int i = bi + threadIdx.x;
  double rsum = 0.0;
  for (int jj = threadIdx.y; jj < TD; jj += blockDim.y) {
    const int j = bj + jj;
    double a = 0.0;
    if (i < n && j < n && i >= j) a = abs_(H[i + (long long)j * ldh]);
    // column j gets a (from the lower entry), column i gets a again when i > j (the mirrored entry)
    atomicAdd(&cols[jj], a);
    if (i > j) rsum += a;
  }
  atomicAdd(&rows[threadIdx.x], rsum);
  __syncthreads();
  if (threadIdx.y == 0) {
    const int c = bj + threadIdx.x;
    if (c < n && cols[threadIdx.x] != 0.0) atomicAdd(&colsum[c], cols[threadIdx.x]);
    const int r = bi + threadIdx.x;
    if (r < n && rows[threadIdx.x] != 0.0) atomicAdd(&colsum[r], rows[threadIdx.x]);
  }
}

// out[0] = max_j sum_i |HC(i,j) - w_j SC(i,j)|, out[1] = max_j sum_i |C(i,j)| (one block per column)
template <class T>
__global__ void k_resid_cols(int n, const T* HC, const T* SC, long long ld, const double* w, const T* C,
                             long long ldc, double* out) {
  const int j = blockIdx.x;
  const double lj = w[j];
  double r = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    r += abs_(HC[i + j * ld] - lj * SC[i + j * ld]);
    c += abs_(C[i + j * ldc]);
  }
  r = block_sum(r);
  __syncthreads();
  c = block_sum(c);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&out[0], r);
    atomic_max_nonneg(&out[1], c);
  }
}

// out[2] = max_j sum_i |G(i,j) - delta_ij| (one block per column of the k x k G)
template <class T>
__global__ void k_gram_dev(int k, const T* G, long long ldg, double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    T g = G[i + j * ldg];
    if (i == j) g -= from_re<T>(1.0);
    s += abs_(g);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomic_max_nonneg(&out[2], s);
}

__global__ void k_max_into(int n, const double* v, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&out[3], m);
}

// HB = (B + B^H) C for a Hermitian M given by its lower triangle (B = tril(M), diagonal halved)
template <class T>
int herm_times(Sys& s, const T* M, int ldm, int k, const T* C, int ldc, T* B, T* out) {
  const int n = s.n;
  const T one = from_re<T>(1.0), zero = zero_<T>();
  GEV_TRY(tril_halfdiag<T>(s, n, M, ldm, B, n));
  GemmP<T> g = gp<T>(n, k, n, 0, 0, one, B, n, C, ldc, zero, out, n);
  g.tri_a = 1;
  gemm(s, g);
  g = gp<T>(n, k, n, 2, 0, one, B, n, C, ldc, one, out, n);
  g.tri_a = 2;
  gemm(s, g);
  return last_error();
}

}  // namespace

// resid / ortho of the solution (C, evals) of the pencil (H, S); buffers W1, V1, Yk of the handle
// and s.d / s.e are overwritten (all free once a solve has written C).
template <class T>
int measure(Sys& s, const T* H, int ldh, const T* S, int lds, int k, const double* evals, const T* C, int ldc,
            double* resid, double* ortho) {
  const int n = s.n;
  T* B = (T*)s.W1;
  T* HC = (T*)s.V1;
  T* SC = (T*)s.Yk;
  double* colsum = s.d;
  double* out = s.e;  // [0] max residual column, [1] max |C| column, [2] max Gram column, [3] ||H||_1
  const bool saved_account = s.account;
  s.account = false;  // not part of the solve's product accounting
  GEV_CUDA_TRY(cudaMemsetAsync(out, 0, 4 * sizeof(double), s.stream));
  GEV_CUDA_TRY(cudaMemsetAsync(colsum, 0, sizeof(double) * (size_t)n, s.stream));
  GEV_TRY(herm_times<T>(s, H, ldh, k, C, ldc, B, HC));
  GEV_TRY(herm_times<T>(s, S, lds, k, C, ldc, B, SC));
  GEV_COUNT(s);
  k_resid_cols<T><<<k, 256, 0, s.stream>>>(n, HC, SC, n, evals, C, ldc, out);
  GEV_COUNT(s);
  k_herm_colsum<T><<<dim3(cdiv(n, TD), cdiv(n, TD)), dim3(TD, 8), 0, s.stream>>>(n, H, ldh, colsum);
  GEV_COUNT(s);
  k_max_into<<<1, 1024, 0, s.stream>>>(n, colsum, out);
  // G = C^H (S C) into the (now free) H C buffer
  T* G = HC;
  gemm(s, gp<T>(k, k, n, 2, 0, from_re<T>(1.0), C, ldc, SC, n, zero_<T>(), G, k));
  GEV_COUNT(s);
  k_gram_dev<T><<<k, 256, 0, s.stream>>>(k, G, k, out);
  GEV_TRY(last_error());
  s.account = saved_account;
  double h[4];
  GEV_CUDA_TRY(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s.stream));
  GEV_TRY(sync_status(s));
  s.have_band = false;  // the reflectors of the last reduction were overwritten
  s.have_tridiag_refl = false;
  const double hn = h[3], cn = h[1];
  *resid = (hn > 0 && cn > 0) ? h[0] / (hn * cn) : h[0];
  *ortho = h[2];
  return 0;
}

template int measure<double>(Sys&, const double*, int, const double*, int, int, const double*, const double*, int,
                             double*, double*);
template int measure<zd>(Sys&, const zd*, int, const zd*, int, int, const double*, const zd*, int, double*,
                         double*);

}  // namespace gev
