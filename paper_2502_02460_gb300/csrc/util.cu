// Element-wise helpers of the solver: triangle copies, Hermitian sums and mirrors (32x32 tiles
// through shared memory, so both the read and the transposed write are coalesced), 2-D copies,
// and the per-column phase normalisation of the eigenvectors.
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace gev {

int set_dyn_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes allowed
  int dev = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(func, dev);
  const auto it = done.find(key);
  if (it != done.end() && (bytes < 0 || it->second >= bytes)) return 0;
  int want = bytes;
  if (want < 0) {
    int optin = 0;
    GEV_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    GEV_CUDA_TRY(cudaFuncGetAttributes(&fa, func));
    want = optin - (int)fa.sharedSizeBytes;
  }
  GEV_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, want));
  done[key] = want;
  return 0;
}

int reset_status(Sys& s) {
  GEV_CUDA_TRY(cudaMemsetAsync(s.status, 0, sizeof(int) * ST_COUNT, s.stream));
  if (s.opts.wait_limit > 0) {
    s.spin_h = s.opts.wait_limit;
    GEV_CUDA_TRY(cudaMemcpyAsync(&s.status[ST_SPIN], &s.spin_h, sizeof(int), cudaMemcpyHostToDevice, s.stream));
  }
  return 0;
}

namespace {

constexpr int TD = 32;

// A = tril(S) (upper zeroed); mode 1: diagonal halved (B = tril(H) with H = B + B^H).
template <class T>
__global__ void k_copy_lower(int n, const T* __restrict__ S, long long lds, T* __restrict__ A,
                             long long lda, int half_diag) {
  const int i = blockIdx.x * TD + threadIdx.x;
  for (int jj = threadIdx.y; jj < TD; jj += blockDim.y) {
    const int j = blockIdx.y * TD + jj;
    if (i >= n || j >= n) continue;
    T v = zero_<T>();
    if (i > j) v = S[i + j * lds];
    else if (i == j) v = from_re<T>(half_diag ? 0.5 * re_(S[i + j * lds]) : re_(S[i + j * lds]));
    A[i + j * lda] = v;
  }
}

// A(i,j) = M(i,j) + conj(M(j,i)) for every (i,j): the full Hermitian sum M + M^H.
template <class T>
__global__ void k_herm_sum(int n, const T* __restrict__ M, long long ldm, T* __restrict__ A,
                           long long lda) {
  __shared__ T tile[TD][TD + 1];
  const int bi = blockIdx.x * TD, bj = blockIdx.y * TD;
  // load the transposed tile M(bj + ., bi + .)
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    int gi = bj + threadIdx.x, gj = bi + r;
    tile[r][threadIdx.x] = (gi < n && gj < n) ? M[gi + gj * ldm] : zero_<T>();
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    int gi = bi + threadIdx.x, gj = bj + r;
    if (gi < n && gj < n) {
      T v = M[gi + gj * ldm] + conj_(tile[threadIdx.x][r]);
      if (gi == gj) v = from_re<T>(re_(v));
      A[gi + gj * lda] = v;
    }
  }
}

// upper <- conj(lower) for tiles on or above the diagonal; diagonal imaginary parts cleared.
template <class T>
__global__ void k_mirror(int n, T* A, long long lda) {
  __shared__ T tile[TD][TD + 1];
  const int bi = blockIdx.x * TD, bj = blockIdx.y * TD;  // destination tile (bi <= bj)
  if (bi > bj) return;
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    int gi = bj + threadIdx.x, gj = bi + r;  // source (lower) element (gi, gj)
    tile[r][threadIdx.x] = (gi < n && gj < n) ? A[gi + gj * lda] : zero_<T>();
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TD; r += blockDim.y) {
    int gi = bi + threadIdx.x, gj = bj + r;  // destination (upper) element (gi, gj)
    if (gi < n && gj < n) {
      if (gi < gj) A[gi + gj * lda] = conj_(tile[threadIdx.x][r]);
      else if (gi == gj) A[gi + gj * lda] = from_re<T>(re_(tile[threadIdx.x][r]));
    }
  }
}

template <class T>
__global__ void k_zero_upper(int n, T* A, long long lda) {
  const int i = blockIdx.x * TD + threadIdx.x;
  for (int jj = threadIdx.y; jj < TD; jj += blockDim.y) {
    const int j = blockIdx.y * TD + jj;
    if (i < n && j < n && i < j) A[i + j * lda] = zero_<T>();
  }
}

template <class T>
__global__ void k_copy2d(int m, int n, const T* __restrict__ src, long long lds, T* __restrict__ dst,
                         long long ldd) {
  const long long total = (long long)m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % m), j = (int)(t / m);
    dst[i + j * ldd] = src[i + j * lds];
  }
}

template <class TA, class TB>
__global__ void k_convert2d(int m, int n, const TA* __restrict__ src, long long lds, TB* __restrict__ dst,
                            long long ldd) {
  const long long total = (long long)m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % m), j = (int)(t / m);
    if constexpr (is_cx<TB>::value) {
      const TA a = src[i + j * lds];
      dst[i + j * ldd] = TB{(decltype(TB{}.x))a.x, (decltype(TB{}.x))a.y};
    } else {
      dst[i + j * ldd] = (TB)src[i + j * lds];
    }
  }
}

// One block per column: the entry of largest modulus (first index on ties) becomes real positive.
template <class T>
__global__ void k_normalize_phase(int n, T* C, long long ldc) {
  const int c = blockIdx.x;
  T* col = C + c * ldc;
  double best = -1.0;
  int bidx = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = abs2_(col[i]);
    if (a > best) { best = a; bidx = i; }
  }
  __shared__ double sv[32];
  __shared__ int si[32];
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, best, off);
    int oi = __shfl_down_sync(0xffffffffu, bidx, off);
    if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sv[wid] = best; si[wid] = bidx; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    best = lane < nw ? sv[lane] : -1.0;
    bidx = lane < nw ? si[lane] : 0x7fffffff;
    for (int off = 16; off > 0; off >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, best, off);
      int oi = __shfl_down_sync(0xffffffffu, bidx, off);
      if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if (lane == 0) si[0] = bidx;
  }
  __syncthreads();
  const int piv = si[0];
  const T pv = col[piv];
  const double ap = abs_(pv);
  __syncthreads();
  if (ap == 0.0) return;
  T ph;
  if constexpr (is_cx<T>::value) ph = make_zd(pv.x / ap, -pv.y / ap);
  else ph = pv > 0 ? 1.0 : -1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i == piv) col[i] = from_re<T>(ap);
    else col[i] = ph * col[i];
  }
}

}  // namespace

template <class T> int copy_lower(Sys& s, int n, const T* S, int lds, T* A, int lda) {
  if (n <= 0) return 0;
  dim3 g(cdiv(n, TD), cdiv(n, TD)), b(TD, 8);
  GEV_COUNT(s);
  k_copy_lower<T><<<g, b, 0, s.stream>>>(n, S, lds, A, lda, 0);
  return last_error();
}
template <class T> int tril_halfdiag(Sys& s, int n, const T* H, int ldh, T* B, int ldb) {
  if (n <= 0) return 0;
  dim3 g(cdiv(n, TD), cdiv(n, TD)), b(TD, 8);
  GEV_COUNT(s);
  k_copy_lower<T><<<g, b, 0, s.stream>>>(n, H, ldh, B, ldb, 1);
  return last_error();
}
template <class T> int herm_sum(Sys& s, int n, const T* M, int ldm, T* A, int lda) {
  if (n <= 0) return 0;
  dim3 g(cdiv(n, TD), cdiv(n, TD)), b(TD, 8);
  GEV_COUNT(s);
  k_herm_sum<T><<<g, b, 0, s.stream>>>(n, M, ldm, A, lda);
  return last_error();
}
template <class T> int mirror_lower(Sys& s, int n, T* A, int lda) {
  if (n <= 0) return 0;
  dim3 g(cdiv(n, TD), cdiv(n, TD)), b(TD, 8);
  GEV_COUNT(s);
  k_mirror<T><<<g, b, 0, s.stream>>>(n, A, lda);
  return last_error();
}
template <class T> int zero_upper(Sys& s, int n, T* A, int lda) {
  if (n <= 1) return 0;
  dim3 g(cdiv(n, TD), cdiv(n, TD)), b(TD, 8);
  GEV_COUNT(s);
  k_zero_upper<T><<<g, b, 0, s.stream>>>(n, A, lda);
  return last_error();
}
template <class T> int copy2d(Sys& s, int m, int n, const T* src, long long lds, T* dst, long long ldd) {
  if (m <= 0 || n <= 0) return 0;
  long long total = (long long)m * n;
  unsigned blocks = cdiv(total, 256);
  if (blocks > 16u * s.sms) blocks = 16u * s.sms;
  GEV_COUNT(s);
  k_copy2d<T><<<blocks, 256, 0, s.stream>>>(m, n, src, lds, dst, ldd);
  return last_error();
}
template <class TA, class TB>
int convert2d(Sys& s, int m, int n, const TA* src, long long lds, TB* dst, long long ldd) {
  if (m <= 0 || n <= 0) return 0;
  long long total = (long long)m * n;
  unsigned blocks = cdiv(total, 256);
  if (blocks > 16u * s.sms) blocks = 16u * s.sms;
  GEV_COUNT(s);
  k_convert2d<TA, TB><<<blocks, 256, 0, s.stream>>>(m, n, src, lds, dst, ldd);
  return last_error();
}
template int convert2d<double, float>(Sys&, int, int, const double*, long long, float*, long long);
template int convert2d<float, double>(Sys&, int, int, const float*, long long, double*, long long);
template int convert2d<zd, zf>(Sys&, int, int, const zd*, long long, zf*, long long);
template int convert2d<zf, zd>(Sys&, int, int, const zf*, long long, zd*, long long);

template <class T> int normalize_phase(Sys& s, int n, int k, T* C, int ldc) {
  if (n <= 0 || k <= 0) return 0;
  GEV_COUNT(s);
  k_normalize_phase<T><<<k, 256, 0, s.stream>>>(n, C, ldc);
  return last_error();
}

int sync_status(Sys& s) {
  GEV_CUDA_TRY(cudaMemcpyAsync(s.status_h, s.status, sizeof(int) * ST_COUNT, cudaMemcpyDeviceToHost,
                               s.stream));
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  if (s.status_h[ST_CONFIG]) {
    fprintf(stderr, "gev: a launch could not be configured (site %d)\n", s.status_h[ST_CONFIG]);
    return GEV_ERR_CUDA;
  }
  return 0;
}

#define GEV_INST(T)                                                                   \
  template int copy_lower<T>(Sys&, int, const T*, int, T*, int);                      \
  template int tril_halfdiag<T>(Sys&, int, const T*, int, T*, int);                   \
  template int herm_sum<T>(Sys&, int, const T*, int, T*, int);                        \
  template int mirror_lower<T>(Sys&, int, T*, int);                                   \
  template int zero_upper<T>(Sys&, int, T*, int);                                     \
  template int copy2d<T>(Sys&, int, int, const T*, long long, T*, long long);         \
  template int normalize_phase<T>(Sys&, int, int, T*, int);
GEV_INST(double)
GEV_INST(zd)
GEV_INST(float)
#undef GEV_INST

}  // namespace gev
