// Generalized solve for an ill-conditioned (numerically singular) overlap S, the procedure of the
// section "Current Status of the Implementation": transform the pencil to the basis of the
// eigenvectors D_i of S and omit every D_i whose eigenvalue sigma_i is below delta.
//
//   1. S = D diag(sigma) D^H, all n pairs, by this library's standard chain (full -> band, bulge
//      chasing, divide and conquer, both back-transforms) on the handle's workspace;
//   2. X = D_kept diag(sigma_kept)^{-1/2}, m = #{sigma_i >= delta} columns (sigma ascending: the last m),
//      kept resident in the handle's factor slot for later SCF iterations (gev_reuse_factor);
//   3. H~ = X^H H X (m x m): H X = (B + B^H) X with B = tril(H), diagonal halved, then the lower
//      triangle of X^H (H X), mirrored;
//   4. H~ Y = Y Lambda by the same chain on a cached handle of order m, the k lowest pairs;
//   5. C = X Y, phase normalised.
// C^H S C = I on the kept space.  Every product runs on the handle's FP64 product engine.
#include <vector>

#include "common.cuh"

namespace gev {

namespace {

// X(:, c) = D(:, first + c) / sqrt(sigma[first + c]), c < m
template <class T>
__global__ void k_scale_basis(int n, int m, int first, const T* D, long long ldd, const double* sig, T* X,
                              long long ldx) {
  const long long total = (long long)n * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), c = (int)(t / n);
    X[i + c * ldx] = (1.0 / sqrt(sig[first + c])) * D[i + (long long)(first + c) * ldd];
  }
}

}  // namespace

template <class T>
int solve_reduced(Sys& s, const T* H, int ldh, const T* S, int lds, double delta, int k, double* evals, T* C,
                  int ldc, int* m_kept, gev_report* rep) {
  const int n = s.n;
  const T one = from_re<T>(1.0), zero = zero_<T>();
  T* A = (T*)s.A;
  T* X = (T*)s.X;
  s.n_marks = 0;
  s.launches = 0;
  s.gemm_used = 0;
  s.account = s.opts.timing == 2;
  GEV_TRY(reset_status(s));
  const bool reuse = (S == nullptr);
  step_mark(s, GEV_STEP_CHOLESKY);
  if (!reuse) {
    // 1. all eigenpairs of S
    GEV_TRY(copy_lower<T>(s, n, S, lds, A, n));
    GEV_TRY(mirror_lower<T>(s, n, A, n));
    if (one_stage_for(s.opts.one_stage, n, n)) {  // all n pairs of S
      GEV_TRY(he2td<T>(s, A, n));
    } else {
      GEV_TRY(he2hb<T>(s, A, n, s.b));
      GEV_TRY(hb2st<T>(s, s.d, s.e));
    }
    GEV_TRY(stop_on_timeout(s));
    GEV_TRY(stedc(s, s.d, s.e, n, s.w, s.Zk, n, nullptr));
    T* D = (T*)s.Yk;
    s.z_unit = true;  // the divide-and-conquer eigenvectors
    GEV_TRY(back<T>(s, s.Zk, n, n, D, n));
    s.z_unit = false;
    // 2. the kept basis
    std::vector<double> sig(n);
    GEV_CUDA_TRY(cudaMemcpyAsync(sig.data(), s.w, sizeof(double) * n, cudaMemcpyDeviceToHost, s.stream));
    GEV_TRY(sync_status(s));
    if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
    int first = 0;
    while (first < n && !(sig[first] >= delta)) ++first;
    const int m = n - first;
    s.reduced_m = m;
    s.have_factor = false;
    if (m_kept) *m_kept = m;
    if (m < k) return GEV_ERR_RANK;
    GEV_COUNT(s);
    k_scale_basis<T><<<std::min<unsigned>(cdiv((long long)n * m, 256), 16u * s.sms), 256, 0, s.stream>>>(
        n, m, first, D, n, s.w, X, n);
    GEV_TRY(last_error());
  } else if (m_kept) {
    *m_kept = s.reduced_m;
  }
  const int m = s.reduced_m;
  if (m < k) return GEV_ERR_RANK;
  if (rep) rep->reused_factor = reuse ? 1 : 0;
  // 3. H~ = X^H H X (lower triangle, then mirrored), into A
  step_mark(s, GEV_STEP_MULTIPLY);
  T* B = (T*)s.W1;
  T* HX = (T*)s.V1;
  GEV_TRY(tril_halfdiag<T>(s, n, H, ldh, B, n));
  GemmP<T> g = gp<T>(n, m, n, 0, 0, one, B, n, X, n, zero, HX, n);
  g.tri_a = 1;
  gemm(s, g);
  g = gp<T>(n, m, n, 2, 0, one, B, n, X, n, one, HX, n);
  g.tri_a = 2;
  gemm(s, g);
  g = gp<T>(m, m, n, 2, 0, one, X, n, HX, n, zero, A, m);
  g.c_lower = 1;
  gemm(s, g);
  GEV_TRY(mirror_lower<T>(s, m, A, m));
  s.have_factor = true;
  s.factor_kind = 1;
  s.have_band = false;
  // 4. the m x m standard problem on a cached handle of order m
  if (!s.sub || s.sub_n != m) {
    if (s.sub) gev_free((gev_sys*)s.sub);
    s.sub = nullptr;
    gev_opts o = s.opts;
    o.prec = GEV_PLAIN;
    o.timing = 0;
    o.workspace_limit = 0;
    o.check = 0;
    o.debug_stall = 0;
    o.fp64_emulation = s.emu_fp64;
    gev_sys* h = nullptr;
    const int rc = gev_setup(&h, m, s.dtype, &o);
    if (rc) return rc;
    s.sub = h;
    s.sub_n = m;
  }
  gev_sys* hs = (gev_sys*)s.sub;
  Sys& u = sys_of(hs);
  GEV_TRY(sync_status(s));  // A is complete before the sub-handle's stream reads it
  step_mark(s, GEV_STEP_TO_BAND);
  GEV_TRY(reset_status(u));
  T* Au = (T*)u.A;
  GEV_TRY(copy2d<T>(u, m, m, A, m, Au, m));
  if (one_stage_for(u.opts.one_stage, m, k)) {
    GEV_TRY(he2td<T>(u, Au, m));
  } else {
    GEV_TRY(he2hb<T>(u, Au, m, u.b));
    GEV_TRY(hb2st<T>(u, u.d, u.e));
  }
  GEV_TRY(stop_on_timeout(u));
  GEV_TRY(stedc(u, u.d, u.e, k, u.w, u.Zk, m, nullptr));
  T* Yu = (T*)u.Yk;
  u.z_unit = true;
  GEV_TRY(back<T>(u, u.Zk, m, k, Yu, m));
  u.z_unit = false;
  GEV_TRY(sync_status(u));
  s.launches += u.launches;
  if (u.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  if (u.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  // 5. C = X Y
  step_mark(s, GEV_STEP_MULT);
  gemm(s, gp<T>(n, k, m, 0, 0, one, X, n, Yu, m, zero, C, ldc));
  GEV_TRY(normalize_phase<T>(s, n, k, C, ldc));
  GEV_CUDA_TRY(cudaMemcpyAsync(evals, u.w, sizeof(double) * k, cudaMemcpyDeviceToDevice, s.stream));
  step_mark(s, -1);
  GEV_TRY(sync_status(s));
  if (!s.reuse) s.have_factor = false;
  if (rep) {
    rep->launches = s.launches;
    if (s.account) gemm_account(s, &rep->gemm_calls, &rep->gemm_ms, &rep->gemm_flops);
    if (s.opts.timing) step_collect(s, rep->ms);
  }
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  return 0;
}

template int solve_reduced<double>(Sys&, const double*, int, const double*, int, double, int, double*, double*,
                                   int, int*, gev_report*);
template int solve_reduced<zd>(Sys&, const zd*, int, const zd*, int, double, int, double*, zd*, int, int*,
                               gev_report*);

}  // namespace gev
