// Mixed-precision form of the generalized solve (real data).
//
// FP64: Cholesky of S, inversion, Multiply A = X H X^T (A is kept in FP64), the refinement and
// C = X^T Y.  FP32: full->band and band->tridiagonal of A32 = fl32(A), the eigenvector products of
// the divide-and-conquer merges, both back-transforms; the secular equations stay FP64.  The paper
// states the precision pattern only (single- and double-precision solutions combined during the SCF
// cycle, section "Future Plans and Challenges"); the refinement is an iteration on the standard
// problem (A, Y) in the spirit of Ogita-Aishima, with an FP64 Rayleigh-Ritz step in span(Y):
//
//   AY = A Y,  T = Y^T AY,  G = Y^T Y
//   Rayleigh-Ritz: T W = G W Lambda (k x k pencil, solved by this library in FP64; W^T G W = I);
//     from the second iteration on, one Ogita-Aishima step W = I + E (first-order eigenvector and
//     orthogonality corrections from T and G; pairs within 1e-7 ||A||_1 only orthogonalised)
//     replaces it whenever max |e_ij| <= 1e-2; a run that ends on such a step finishes with a
//     first-order Loewdin orthonormalisation
//   Y <- Y W,  AY <- AY W,  r_j = AY_j - lambda_j Y_j
//   stop when ||r_j||_1 <= tol ||A||_1 ||y_j||_1 for every j, else
//   out of span: W' = V^T r (V: the other n-k FP32 eigenvectors, mu their FP32 eigenvalues),
//                W'_ij /= (lambda_j - mu_i),  Y <- Y + V W'   (FP32 products, FP64 sum)
//
// The FP32 pipeline resolves eigenvalues only to ~1e-7 ||A||, coarser than the valence spacing of
// DFT-like spectra, so its individual vectors inside near-degenerate groups are mixed while the
// spanned subspaces are accurate; the Rayleigh-Ritz step resolves them exactly in FP64, which a
// pairwise first-order correction cannot do in a few steps.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gev {

namespace {

// band width of the k x k Rayleigh-Ritz solve: the caller's choice, else the library default (64; at
// k = 4096 it measured faster than 32 and 16: the narrower band's cheaper bulge-chasing tasks do not pay
// for the extra back-transform levels and thinner products)
int rr_band(int want, int) {
  if (want == 16 || want == 32 || want == 64) return want;
  return 0;
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// out[j] = sum_i |A(i,j)|  (one block per column)
__global__ void k_colabs(int m, const double* A, long long lda, double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += fabs(A[i + j * lda]);
  __shared__ double red[32];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[j] = t;
  }
}

// out[0] = max_i v[i]  (one block)
__global__ void k_vmax(int n, const double* v, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  __shared__ double red[32];
  m = wmax(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

// residual columns r_j = AY_j - lambda_j Y_j: FP32 copy, and the 1-norms of r_j and y_j
__global__ void k_resid(int n, const double* AY, const double* Y, long long ld, const double* lam,
                        float* Rf, long long ldr, double* rn, double* yn) {
  const int j = blockIdx.x;
  const double l = lam[j];
  double sr = 0.0, sy = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double y = Y[i + j * ld];
    const double r = AY[i + j * ld] - l * y;
    Rf[i + j * ldr] = (float)r;
    sr += fabs(r);
    sy += fabs(y);
  }
  __shared__ double r1[32], r2[32];
  sr = wsum(sr);
  sy = wsum(sy);
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = sr; r2[threadIdx.x >> 5] = sy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r1[w]; b += r2[w]; }
    rn[j] = a;
    yn[j] = b;
  }
}

// W_ij /= (lambda_j - mu_i) (out-of-span coefficients); negligible gaps contribute nothing
__global__ void k_scale_w(int m, int k, float* W, long long ldw, const double* lam, const double* mu,
                          double tiny) {
  const long long total = (long long)m * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    const double den = lam[j] - mu[i];
    float& w = W[i + j * ldw];
    w = (fabs(den) > tiny) ? (float)((double)w / den) : 0.f;
  }
}

// One Ogita-Aishima step in span(Y) (their Algorithm 1 on the Gram data T = Y^T A Y,
// G = Y^T Y, lower triangles): lambda_i = T_ii / G_ii and W = I + E with
//   e_ii = (1 - G_ii) / 2,
//   e_ij = (T_ij - lambda_j G_ij) / (lambda_j - lambda_i)   if |lambda_j - lambda_i| > delta,
//   e_ij = -G_ij / 2                                          otherwise.
// *emax receives max |e_ij| (bit pattern of a non-negative double, atomicMax).
__global__ void k_oa_step(int k, const double* T, const double* G, double delta, double* W, double* lam,
                          unsigned long long* emax) {
  const long long total = (long long)k * k;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double li = T[i + (long long)i * k] / G[i + (long long)i * k];
    double e;
    if (i == j) {
      e = 0.5 * (1.0 - G[t]);
      W[t] = 1.0 + e;
      lam[i] = li;
    } else {
      // T and G hold their lower triangles only (exactly symmetric data: the rounding asymmetry of
      // the products, divided by small gaps, would otherwise break e_ij + e_ji = -G_ij)
      const long long tl = (i > j) ? t : j + (long long)i * k;
      const double tij = T[tl], gij = G[tl];
      const double lj = T[j + (long long)j * k] / G[j + (long long)j * k];
      const double gap = lj - li;
      e = (fabs(gap) > delta) ? (tij - lj * gij) / gap : -0.5 * gij;
      W[t] = e;
    }
    m = fmax(m, fabs(e));
  }
  m = wmax(m);
  if ((threadIdx.x & 31) == 0) atomicMax(emax, (unsigned long long)__double_as_longlong(m));
}

// First-order Loewdin orthonormalisation from G = Y^T Y (lower triangle): W = I + (I - G) / 2, so that
// (Y W)^T (Y W) = I + O((G - I)^2).  One block per column j; *dmax receives the largest column
// 1-norm of G - I (bit pattern of a non-negative double, atomicMax).
__global__ void k_lowdin(int k, const double* G, double* W, unsigned long long* dmax) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double g = (i >= j) ? G[i + (long long)j * k] : G[j + (long long)i * k];  // lower triangle
    const double d = (i == j ? 1.0 : 0.0) - g;
    W[i + (long long)j * k] = (i == j ? 1.0 : 0.0) + 0.5 * d;
    s += fabs(d);
  }
  __shared__ double red[32];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicMax(dmax, (unsigned long long)__double_as_longlong(t));
  }
}

// ---- complex data (zd): the same steps with the Hermitian forms of the formulas
__global__ void k_colabs_z(int m, const zd* A, long long lda, double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += abs_(A[i + j * lda]);
  __shared__ double red[32];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[j] = t;
  }
}

// r_j = AY_j - lambda_j Y_j (FP64), and the 1-norms of r_j and y_j
__global__ void k_resid_z(int n, const zd* AY, const zd* Y, long long ld, const double* lam, zd* R, long long ldr,
                          double* rn, double* yn) {
  const int j = blockIdx.x;
  const double l = lam[j];
  double sr = 0.0, sy = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd y = Y[i + j * ld];
    const zd r = AY[i + j * ld] - l * y;
    R[i + j * ldr] = r;
    sr += abs_(r);
    sy += abs_(y);
  }
  __shared__ double r1[32], r2[32];
  sr = wsum(sr);
  sy = wsum(sy);
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = sr; r2[threadIdx.x >> 5] = sy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r1[w]; b += r2[w]; }
    rn[j] = a;
    yn[j] = b;
  }
}

__global__ void k_scale_w_z(int m, int k, zd* W, long long ldw, const double* lam, const double* mu, double tiny) {
  const long long total = (long long)m * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    const double den = lam[j] - mu[i];
    zd& w = W[i + j * ldw];
    w = (fabs(den) > tiny) ? (1.0 / den) * w : make_zd(0.0, 0.0);
  }
}

// Ogita-Aishima step on Hermitian Gram data (lower triangles): lambda_i = Re T_ii / Re G_ii,
// e_ii = (1 - Re G_ii) / 2, e_ij = (T_ij - lambda_j G_ij) / (lambda_j - lambda_i) or -G_ij / 2
__global__ void k_oa_step_z(int k, const zd* T, const zd* G, double delta, zd* W, double* lam,
                            unsigned long long* emax) {
  const long long total = (long long)k * k;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    const double li = T[i + (long long)i * k].x / G[i + (long long)i * k].x;
    double ea;
    if (i == j) {
      const double e = 0.5 * (1.0 - G[t].x);
      W[t] = make_zd(1.0 + e, 0.0);
      lam[i] = li;
      ea = fabs(e);
    } else {
      const bool lo = i > j;  // lower triangles only: the upper entries are the conjugates
      const long long tl = lo ? t : j + (long long)i * k;
      const zd tij = lo ? T[tl] : conj_(T[tl]), gij = lo ? G[tl] : conj_(G[tl]);
      const double lj = T[j + (long long)j * k].x / G[j + (long long)j * k].x;
      const double gap = lj - li;
      const zd e = (fabs(gap) > delta) ? (1.0 / gap) * (tij - lj * gij) : -0.5 * gij;
      W[t] = e;
      ea = abs_(e);
    }
    m = fmax(m, ea);
  }
  m = wmax(m);
  if ((threadIdx.x & 31) == 0) atomicMax(emax, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_lowdin_z(int k, const zd* G, zd* W, unsigned long long* dmax) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const zd g = (i >= j) ? G[i + (long long)j * k] : conj_(G[j + (long long)i * k]);  // lower triangle
    const zd d = make_zd(i == j ? 1.0 : 0.0, 0.0) - g;
    W[i + (long long)j * k] = make_zd(i == j ? 1.0 : 0.0, 0.0) + 0.5 * d;
    s += abs_(d);
  }
  __shared__ double red[32];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicMax(dmax, (unsigned long long)__double_as_longlong(t));
  }
}

}  // namespace

int solve_mixed(Sys& s, const double* H, int ldh, const double* S, int lds, int k, double* evals, double* C,
                int ldc, gev_report* rep) {
  const int n = s.n;
  cudaStream_t st = s.stream;
  s.n_marks = 0;
  s.launches = 0;
  s.gemm_used = 0;
  s.account = s.opts.timing == 2;
  auto mark = [&](int step) { step_mark(s, step); };
  double* A = (double*)s.A;
  double* X = (double*)s.X;
  GEV_TRY(reset_status(s));
  // ---- FP64: Cholesky, inversion, Multiply
  mark(GEV_STEP_CHOLESKY);
  const bool reuse = (S == nullptr);
  if (!reuse) {
    GEV_TRY(copy_lower<double>(s, n, S, lds, X, n));
    // Cholesky and inversion in one recursion (the "invert" step time is included in "cholesky")
    GEV_TRY(potrf_inv<double>(s, X, n));
    GEV_TRY(sync_status(s));
    if (s.status_h[ST_NOT_SPD]) {
      if (rep) rep->info = s.status_h[ST_NOT_SPD];
      s.have_factor = false;
      return GEV_ERR_NOT_SPD;
    }
    mark(GEV_STEP_INVERT);
  }
  if (rep) rep->reused_factor = reuse ? 1 : 0;
  mark(GEV_STEP_MULTIPLY);
  GEV_TRY(hegst<double>(s, H, ldh, X, n, A, n));
  s.have_factor = true;
  s.factor_kind = 0;
  // ---- FP32 reduction of A32 = fl32(A); all n eigenvectors (the refinement uses the complement)
  // (one-stage option: Householder tridiagonalisation of A32 directly, timed as "to_tridiag")
  const bool one = s.opts.one_stage == 1;  // automatic: two-stage (measured faster in FP32 at n = 16384)
  mark(GEV_STEP_TO_BAND);
  float* A32 = (float*)s.W1;
  GEV_TRY((convert2d<double, float>(s, n, n, A, n, A32, n)));
  if (!one) GEV_TRY(he2hb<float>(s, A32, n, s.b));
  mark(GEV_STEP_TO_TRIDIAG);
  if (one) GEV_TRY(he2td<float>(s, A32, n));
  else GEV_TRY(hb2st<float>(s, s.d, s.e));
  GEV_TRY(stop_on_timeout(s));
  mark(GEV_STEP_SOLVE);
  s.dc_lowp = 1;
  int r = stedc(s, s.d, s.e, n, s.w, s.Zk, n, nullptr);
  s.dc_lowp = 0;
  GEV_TRY(r);
  mark(GEV_STEP_BACK_TRIDIAG);
  float* Y32 = (float*)s.Yk;
  s.z_unit = true;  // the divide-and-conquer eigenvectors
  if (one) GEV_TRY(back_td<float>(s, s.Zk, n, n, Y32, n));
  else GEV_TRY(bt_hb2st<float>(s, s.Zk, n, n, Y32, n));
  s.z_unit = false;
  mark(GEV_STEP_BACK_BAND);
  if (!one) GEV_TRY(bt_he2hb<float>(s, Y32, n, n));
  // ---- FP64 refinement of the k lowest pairs
  mark(GEV_STEP_REFINE);
  // buffers (all free or dedicated at this point; every one large enough also for k = n)
  double* Yd = (double*)s.W1;            // n x k current vectors (A32 is no longer needed)
  double* Yn = (double*)s.Q2;            // n x k Ritz vectors
  double* AY = (double*)s.Q;             // n x k
  double* AYn = s.Zk;                    // n x k
  double* T = s.R1;                      // k x k
  double* G = s.R2;                      // k x k
  double* W = s.R3;                      // k x k Ritz coefficients
  double* lam = s.e;                     // k (the tridiagonal is consumed)
  double* rn = s.d;                      // k (after the column sums of A)
  double* yn = (double*)s.phase;         // k
  double* scal = (double*)s.small;       // [0] ||A||_1, [1] max ||r_j||_1, [2] max ||y_j||_1, [3] max |e_ij|
  float* Rf = Y32 + (size_t)n * n;       // n x k, second half of the FP32 eigenvector buffer
  float* Wp = (float*)s.V2;              // (n-k) x k
  const float* Vp = Y32 + (size_t)k * n;
  const double* mu = s.w + k;
  GEV_TRY((convert2d<float, double>(s, n, k, Y32, n, Yd, n)));
  GEV_COUNT(s);
  k_colabs<<<n, 256, 0, st>>>(n, A, n, s.d);
  GEV_COUNT(s);
  k_vmax<<<1, 1024, 0, st>>>(n, s.d, scal);
  double hs[3] = {0, 0, 0};
  GEV_CUDA_TRY(cudaMemcpyAsync(hs, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  GEV_CUDA_TRY(cudaStreamSynchronize(st));
  const double anorm = hs[0] > 0 ? hs[0] : 1.0;
  const double tol = s.opts.refine_tol;
  const int maxit = s.opts.refine_max_iter;
  // the k x k Rayleigh-Ritz pencil is solved by a second (cached) handle of this library
  if (!s.sub || s.sub_n != k) {
    if (s.sub) gev_free((gev_sys*)s.sub);
    s.sub = nullptr;
    gev_opts o = s.opts;
    o.prec = GEV_PLAIN;
    o.timing = 0;
    o.workspace_limit = 0;
    o.band_b = rr_band(s.opts.rr_band_b, k);
    o.fp64_emulation = s.emu_fp64;  // the Ritz pencil's products use the same FP64 engine
    o.check = 0;
    o.one_stage = (s.opts.rr_one_stage == 1 || (s.opts.rr_one_stage == 0 && k >= 2048)) ? 1 : 2;
    o.debug_stall = 0;
    gev_sys* h = nullptr;
    const int rc = gev_setup(&h, k, GEV_F64, &o);
    if (rc) return rc;
    s.sub = h;
    s.sub_n = k;
  }
  int it = 0, oa_steps = 0;
  double resid = 0.0;
  bool converged = false;
  // largest first-order coefficient for which an Ogita-Aishima step is taken instead of the
  // Rayleigh-Ritz solve (its neglected second-order terms are then ~1e-4 and contract
  // quadratically in the following steps)
  constexpr double kOaMaxCorrection = 1e-2;
  // pairs closer than kOaCluster ||A||_1 are only orthogonalised by an Ogita-Aishima step: their
  // coefficients (T_ij - lambda_j G_ij) / gap would divide the ~1e-15 ||A|| rounding of the FP64
  // products by the gap, and the Rayleigh-Ritz step has already resolved them in FP64
  constexpr double kOaCluster = 1e-7;
  for (;; ++it) {
    gemm(s, gp<double>(n, k, n, 0, 0, 1.0, A, n, Yd, n, 0.0, AY, n));   // AY = A Y
    {  // T = Y^T A Y, G = Y^T Y: lower triangles
      GemmP<double> g = gp<double>(k, k, n, 1, 0, 1.0, Yd, n, AY, n, 0.0, T, k);
      g.c_lower = 1;
      gemm(s, g);
      g = gp<double>(k, k, n, 1, 0, 1.0, Yd, n, Yd, n, 0.0, G, k);
      g.c_lower = 1;
      gemm(s, g);
    }
    // after the first iteration the basis is close to the eigenvectors: one Ogita-Aishima step in
    // span(Y) replaces the Rayleigh-Ritz solve while its corrections stay small
    bool oa = false;
    double emax = 0.0;
    if (it > 0 && !s.opts.refine_rr_only) {
      GEV_CUDA_TRY(cudaMemsetAsync(scal + 3, 0, sizeof(double), st));
      GEV_COUNT(s);
      k_oa_step<<<std::min<unsigned>(cdiv((long long)k * k, 256), 16u * s.sms), 256, 0, st>>>(
          k, T, G, kOaCluster * anorm, W, lam, (unsigned long long*)(scal + 3));
      GEV_CUDA_TRY(cudaMemcpyAsync(&emax, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      GEV_CUDA_TRY(cudaStreamSynchronize(st));
      oa = emax <= kOaMaxCorrection;
      if (oa) ++oa_steps;
    }
    if (!oa) {
      gev_report sr;
      const int rc = gev_solve((gev_sys*)s.sub, T, k, G, k, k, lam, W, k, &sr);
      if (rc) return rc;
      s.launches += sr.launches;
    }
    gemm(s, gp<double>(n, k, k, 0, 0, 1.0, Yd, n, W, k, 0.0, Yn, n));   // Ritz vectors
    gemm(s, gp<double>(n, k, k, 0, 0, 1.0, AY, n, W, k, 0.0, AYn, n));  // A times them
    GEV_COUNT(s);
    k_resid<<<k, 256, 0, st>>>(n, AYn, Yn, n, lam, Rf, n, rn, yn);
    GEV_COUNT(s);
    k_vmax<<<1, 1024, 0, st>>>(k, rn, scal + 1);
    GEV_COUNT(s);
    k_vmax<<<1, 1024, 0, st>>>(k, yn, scal + 2);
    GEV_CUDA_TRY(cudaMemcpyAsync(hs, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GEV_CUDA_TRY(cudaStreamSynchronize(st));
    resid = hs[1] / (anorm * (hs[2] > 0 ? hs[2] : 1.0));
    std::swap(Yd, Yn);  // Yd = the Ritz vectors
    if (resid <= tol && !oa) { converged = true; break; }  // Rayleigh-Ritz vectors: orthonormal in FP64
    if (resid <= tol) {
      // an Ogita-Aishima step leaves second-order defects in orthogonality: finish with a
      // first-order Loewdin step; it moves the residuals by at most ||A|| max_j sum_i |G - I|_ij
      {
        GemmP<double> g = gp<double>(k, k, n, 1, 0, 1.0, Yd, n, Yd, n, 0.0, G, k);
        g.c_lower = 1;
        gemm(s, g);
      }
      GEV_CUDA_TRY(cudaMemsetAsync(scal + 3, 0, sizeof(double), st));
      GEV_COUNT(s);
      k_lowdin<<<k, 256, 0, st>>>(k, G, W, (unsigned long long*)(scal + 3));
      double dmax = 0.0;
      GEV_CUDA_TRY(cudaMemcpyAsync(&dmax, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      GEV_CUDA_TRY(cudaStreamSynchronize(st));
      if (resid + dmax <= tol) {
        gemm(s, gp<double>(n, k, k, 0, 0, 1.0, Yd, n, W, k, 0.0, Yn, n));
        std::swap(Yd, Yn);
        resid += dmax;
        converged = true;
        break;
      }
    }
    if (it >= maxit || n == k) break;
    GemmP<float> g = gp<float>(n - k, k, n, 1, 0, 1.0f, Vp, n, Rf, n, 0.0f, Wp, n - k);
    gemm32<float, float>(s, g, Wp, 1.0f, 0.0f);  // W' = V^T r
    GEV_COUNT(s);
    k_scale_w<<<std::min<unsigned>(cdiv((long long)(n - k) * k, 256), 16u * s.sms), 256, 0, st>>>(
        n - k, k, Wp, n - k, lam, mu, 1e-14 * anorm);
    GemmP<float> g2 = gp<float>(n, k, n - k, 0, 0, 1.0f, Vp, n, Wp, n - k, 1.0f, nullptr, n);
    gemm32<float, double>(s, g2, Yd, 1.0f, 1.0f);  // Y += V W' (FP32 products, FP64 sum)
  }
  if (rep) {
    rep->refine_iters = it + 1;
    rep->refine_resid = resid;
    rep->refine_oa_steps = oa_steps;
  }
  // ---- FP64: C = X^T Y
  mark(GEV_STEP_MULT);
  GEV_TRY(mult<double>(s, X, n, Yd, n, k, C, ldc));
  GEV_TRY(normalize_phase<double>(s, n, k, C, ldc));
  GEV_CUDA_TRY(cudaMemcpyAsync(evals, lam, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
  mark(-1);
  GEV_TRY(sync_status(s));
  if (!s.reuse) s.have_factor = false;
  if (rep) {
    rep->launches = s.launches;
    if (s.account) gemm_account(s, &rep->gemm_calls, &rep->gemm_ms, &rep->gemm_flops);
    if (s.opts.timing) step_collect(s, rep->ms);
  }
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  if (!converged) return GEV_ERR_NO_CONVERGENCE;
  return 0;
}

}  // namespace gev

namespace gev {

// Mixed form for complex Hermitian data.  FP64: Cholesky, inversion, Multiply, full->band (its
// products on the tensor cores) and back-transform 1; FP32 (complex64): the bulge chasing of the
// band, the divide-and-conquer merge products and back-transform 2 - the steps whose FP64 form is
// bound by GB300's FP64 pipe.  Then the FP64 refinement of the real form with Hermitian formulas,
// its out-of-span correction using the complement in FP64.
int solve_mixed_cx(Sys& s, const zd* H, int ldh, const zd* S, int lds, int k, double* evals, zd* C, int ldc,
                   gev_report* rep) {
  const int n = s.n;
  cudaStream_t st = s.stream;
  s.n_marks = 0;
  s.launches = 0;
  s.gemm_used = 0;
  s.account = s.opts.timing == 2;
  auto mark = [&](int step) { step_mark(s, step); };
  zd* A = (zd*)s.A;
  zd* X = (zd*)s.X;
  const zd one = make_zd(1.0, 0.0), zero = make_zd(0.0, 0.0);
  GEV_TRY(reset_status(s));
  mark(GEV_STEP_CHOLESKY);
  const bool reuse = (S == nullptr);
  if (!reuse) {
    GEV_TRY(copy_lower<zd>(s, n, S, lds, X, n));
    // Cholesky and inversion in one recursion (the "invert" step time is included in "cholesky")
    GEV_TRY(potrf_inv<zd>(s, X, n));
    GEV_TRY(sync_status(s));
    if (s.status_h[ST_NOT_SPD]) {
      if (rep) rep->info = s.status_h[ST_NOT_SPD];
      s.have_factor = false;
      return GEV_ERR_NOT_SPD;
    }
    mark(GEV_STEP_INVERT);
  }
  if (rep) rep->reused_factor = reuse ? 1 : 0;
  mark(GEV_STEP_MULTIPLY);
  GEV_TRY(hegst<zd>(s, H, ldh, X, n, A, n));
  s.have_factor = true;
  s.factor_kind = 0;
  // ---- full->band in FP64 on a copy of A (A stays for the refinement)
  mark(GEV_STEP_TO_BAND);
  zd* W1 = (zd*)s.W1;
  GEV_TRY(copy2d<zd>(s, n, n, A, n, W1, n));
  GEV_TRY(he2hb<zd>(s, W1, n, s.b));
  // ---- band -> tridiagonal in complex64
  mark(GEV_STEP_TO_TRIDIAG);
  {
    const long long bl = (long long)s.ldband * (n + 2 * s.b);
    zd* tmp = (zd*)s.bandtmp;  // a copy of the FP64 band, sized like it
    GEV_TRY(copy2d<zd>(s, (int)bl, 1, (const zd*)s.band, bl, tmp, bl));
    GEV_TRY((convert2d<zd, zf>(s, (int)bl, 1, tmp, bl, (zf*)s.band, bl)));
  }
  GEV_TRY(hb2st<zf>(s, s.d, s.e));
  GEV_TRY(stop_on_timeout(s));
  mark(GEV_STEP_SOLVE);
  s.dc_lowp = 1;
  int r = stedc(s, s.d, s.e, n, s.w, s.Zk, n, nullptr);
  s.dc_lowp = 0;
  GEV_TRY(r);
  mark(GEV_STEP_BACK_TRIDIAG);
  zf* Y32 = (zf*)s.Yk;
  s.z_unit = true;  // the divide-and-conquer eigenvectors
  GEV_TRY(bt_hb2st<zf>(s, s.Zk, n, n, Y32, n));
  s.z_unit = false;
  mark(GEV_STEP_BACK_BAND);
  zd* Vfull = W1;  // all n approximate eigenvectors in FP64
  GEV_TRY((convert2d<zf, zd>(s, n, n, Y32, n, Vfull, n)));
  GEV_TRY(bt_he2hb<zd>(s, Vfull, n, n));
  // ---- FP64 refinement of the k lowest pairs
  mark(GEV_STEP_REFINE);
  zd* Yd = (zd*)s.Yk;    // n x k current vectors (the complex64 vectors are consumed)
  zd* Yn = (zd*)s.V1;    // n x k (the full->band reflectors are consumed)
  zd* AY = (zd*)s.R1;    // n x k
  zd* AYn = (zd*)s.R2;   // n x k
  zd* Rr = (zd*)s.R3;    // n x k residual columns
  zd* T = (zd*)s.R4;     // k x k
  zd* G = T + (size_t)k * k;
  zd* W = G + (size_t)k * k;
  zd* Wp = (zd*)s.Q2;    // (n - k) x k
  double* lam = s.e;
  double* rn = s.d;
  double* yn = (double*)s.phase;
  double* scal = (double*)s.small;
  const zd* Vp = Vfull + (size_t)k * n;
  const double* mu = s.w + k;
  GEV_TRY(copy2d<zd>(s, n, k, Vfull, n, Yd, n));
  GEV_COUNT(s);
  k_colabs_z<<<n, 256, 0, st>>>(n, A, n, s.d);
  GEV_COUNT(s);
  k_vmax<<<1, 1024, 0, st>>>(n, s.d, scal);
  double hs[3] = {0, 0, 0};
  GEV_CUDA_TRY(cudaMemcpyAsync(hs, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  GEV_CUDA_TRY(cudaStreamSynchronize(st));
  const double anorm = hs[0] > 0 ? hs[0] : 1.0;
  const double tol = s.opts.refine_tol;
  const int maxit = s.opts.refine_max_iter;
  if (!s.sub || s.sub_n != k) {
    if (s.sub) gev_free((gev_sys*)s.sub);
    s.sub = nullptr;
    gev_opts o = s.opts;
    o.prec = GEV_PLAIN;
    o.timing = 0;
    o.workspace_limit = 0;
    o.band_b = rr_band(s.opts.rr_band_b, k);
    o.fp64_emulation = s.emu_fp64;
    o.check = 0;
    o.one_stage = (s.opts.rr_one_stage == 1 || (s.opts.rr_one_stage == 0 && k >= 2048)) ? 1 : 2;
    o.debug_stall = 0;
    gev_sys* h = nullptr;
    const int rc = gev_setup(&h, k, GEV_C128, &o);
    if (rc) return rc;
    s.sub = h;
    s.sub_n = k;
  }
  constexpr double kOaMaxCorrection = 1e-2;
  constexpr double kOaCluster = 1e-7;  // see solve_mixed
  int it = 0, oa_steps = 0;
  double resid = 0.0;
  bool converged = false;
  for (;; ++it) {
    gemm(s, gp<zd>(n, k, n, 0, 0, one, A, n, Yd, n, zero, AY, n));   // AY = A Y
    {  // T = Y^H A Y, G = Y^H Y: lower triangles
      GemmP<zd> g = gp<zd>(k, k, n, 2, 0, one, Yd, n, AY, n, zero, T, k);
      g.c_lower = 1;
      gemm(s, g);
      g = gp<zd>(k, k, n, 2, 0, one, Yd, n, Yd, n, zero, G, k);
      g.c_lower = 1;
      gemm(s, g);
    }
    bool oa = false;
    if (it > 0 && !s.opts.refine_rr_only) {
      double emax = 0.0;
      GEV_CUDA_TRY(cudaMemsetAsync(scal + 3, 0, sizeof(double), st));
      GEV_COUNT(s);
      k_oa_step_z<<<std::min<unsigned>(cdiv((long long)k * k, 256), 16u * s.sms), 256, 0, st>>>(
          k, T, G, kOaCluster * anorm, W, lam, (unsigned long long*)(scal + 3));
      GEV_CUDA_TRY(cudaMemcpyAsync(&emax, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      GEV_CUDA_TRY(cudaStreamSynchronize(st));
      oa = emax <= kOaMaxCorrection;
      if (oa) ++oa_steps;
    }
    if (!oa) {
      gev_report sr;
      const int rc = gev_solve((gev_sys*)s.sub, T, k, G, k, k, lam, W, k, &sr);
      if (rc) return rc;
      s.launches += sr.launches;
    }
    gemm(s, gp<zd>(n, k, k, 0, 0, one, Yd, n, W, k, zero, Yn, n));
    gemm(s, gp<zd>(n, k, k, 0, 0, one, AY, n, W, k, zero, AYn, n));
    GEV_COUNT(s);
    k_resid_z<<<k, 256, 0, st>>>(n, AYn, Yn, n, lam, Rr, n, rn, yn);
    GEV_COUNT(s);
    k_vmax<<<1, 1024, 0, st>>>(k, rn, scal + 1);
    GEV_COUNT(s);
    k_vmax<<<1, 1024, 0, st>>>(k, yn, scal + 2);
    GEV_CUDA_TRY(cudaMemcpyAsync(hs, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GEV_CUDA_TRY(cudaStreamSynchronize(st));
    resid = hs[1] / (anorm * (hs[2] > 0 ? hs[2] : 1.0));
    std::swap(Yd, Yn);
    if (resid <= tol && !oa) { converged = true; break; }
    if (resid <= tol) {  // Loewdin finish after an Ogita-Aishima step (see solve_mixed)
      {
        GemmP<zd> g = gp<zd>(k, k, n, 2, 0, one, Yd, n, Yd, n, zero, G, k);
        g.c_lower = 1;
        gemm(s, g);
      }
      GEV_CUDA_TRY(cudaMemsetAsync(scal + 3, 0, sizeof(double), st));
      GEV_COUNT(s);
      k_lowdin_z<<<k, 256, 0, st>>>(k, G, W, (unsigned long long*)(scal + 3));
      double dmax = 0.0;
      GEV_CUDA_TRY(cudaMemcpyAsync(&dmax, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      GEV_CUDA_TRY(cudaStreamSynchronize(st));
      if (resid + dmax <= tol) {
        gemm(s, gp<zd>(n, k, k, 0, 0, one, Yd, n, W, k, zero, Yn, n));
        std::swap(Yd, Yn);
        resid += dmax;
        converged = true;
        break;
      }
    }
    if (it >= maxit || n == k) break;
    gemm(s, gp<zd>(n - k, k, n, 2, 0, one, Vp, n, Rr, n, zero, Wp, n - k));  // W' = V^H r
    GEV_COUNT(s);
    k_scale_w_z<<<std::min<unsigned>(cdiv((long long)(n - k) * k, 256), 16u * s.sms), 256, 0, st>>>(
        n - k, k, Wp, n - k, lam, mu, 1e-14 * anorm);
    gemm(s, gp<zd>(n, k, n - k, 0, 0, one, Vp, n, Wp, n - k, one, Yd, n));  // Y += V W'
  }
  if (rep) {
    rep->refine_iters = it + 1;
    rep->refine_resid = resid;
    rep->refine_oa_steps = oa_steps;
  }
  mark(GEV_STEP_MULT);
  GEV_TRY(mult<zd>(s, X, n, Yd, n, k, C, ldc));
  GEV_TRY(normalize_phase<zd>(s, n, k, C, ldc));
  GEV_CUDA_TRY(cudaMemcpyAsync(evals, lam, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
  mark(-1);
  GEV_TRY(sync_status(s));
  if (!s.reuse) s.have_factor = false;
  if (rep) {
    rep->launches = s.launches;
    if (s.account) gemm_account(s, &rep->gemm_calls, &rep->gemm_ms, &rep->gemm_flops);
    if (s.opts.timing) step_collect(s, rep->ms);
  }
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  if (!converged) return GEV_ERR_NO_CONVERGENCE;
  return 0;
}

}  // namespace gev
