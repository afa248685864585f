// C ABI of the solver (include/gev.h, include/gev_steps.h): handle set-up, workspace carving,
// the generalized solve that chains the steps of the reduction (section "Current Status of the
// Implementation", steps 1-3 and the back-transformation; Table 1 step names), and the
// per-step entry points.
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"

using namespace gev;

struct gev_sys {
  Sys s;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t off[32];
  int cnt = 0;
  size_t total = 0;
  size_t add(size_t bytes) {
    size_t o = total;
    off[cnt++] = o;
    total += align256(bytes > 0 ? bytes : 1);
    return o;
  }
};

// band width: a power of two in [16, 64] (the bulge-chasing kernel stages three b x b blocks)
int pick_band(int n, int want) {
  int b = want > 0 ? want : 64;
  int p = 16;
  while (p < b && p < 64) p *= 2;
  return p;
}

// Carve the workspace.  With base == nullptr only the size is computed.
size_t carve(Sys& s, char* base) {
  const size_t n = (size_t)s.n, es = s.es(), b = (size_t)s.b, nb = (size_t)s.nb;
  Layout L;
  size_t oA = L.add(n * n * es), oX = L.add(n * n * es), oW1 = L.add(n * n * es),
         oV1 = L.add(n * n * es), oT1 = L.add(b * (n + b) * es), odinv = L.add(nb * (n + nb) * es),
         oPn = L.add(4 * n * 2 * b * es), osmall = L.add(4 * b * b * es);
  size_t split = 4 * n * 2 * b * es;
  if (split < ((size_t)16 << 20)) split = (size_t)16 << 20;
  size_t osplit = L.add(split);
  const int ldband = 3 * s.b + 2;
  const size_t ntask = (n + b - 1) / b + 2;
  size_t oband = L.add((size_t)ldband * (n + 2 * b) * es);
  size_t oV2 = L.add(b * n * ntask * es), otau2 = L.add(n * ntask * es), ophase = L.add(n * 16);
  size_t od = L.add(n * 8), oe = L.add(n * 8), ow = L.add(n * 8);
  const size_t ntl = (n + 63) / 64;
  const size_t qbytes = std::max(n * n * 8, ntl * ntl * 64 * es);
  size_t oQ = L.add(qbytes), oQ2 = L.add(n * n * 8);
  size_t dcws = 64 * n * 8 + ((size_t)1 << 20);
  size_t odc = L.add(dcws);
  size_t oYk = L.add(n * n * es);
  size_t oZk = L.add(n * n * 8);
  size_t oprog = L.add(n * sizeof(int) + 64);
  // panel factorisation partial sums, double-buffered: 2 x 4096 norms, 2 x b pivot row, 2 x 4096 x b
  size_t panel = (size_t)2 * 4096 * 8 + 2 * 128 * es + (size_t)2 * 4096 * b * es + 256;
  size_t opanel = L.add(panel);
  size_t ost = L.add(sizeof(int) * ST_COUNT);
  size_t ozb = 0;
  // inner dimensions reach max(n, 4b): the full->band rank-2b update and the back-transform-1 groups of
  // four panels have K = 2b and 4b, which exceed n for small orders
  const int kmax = std::max((int)n, 4 * (int)b);
  if (s.emu_fp64)  // complex products run in the real embedding: (2n x 2n) (2n x n)
    ozb = s.dtype == GEV_C128 ? gemm_f64_emulated_scratch(2 * (int)n, (int)n, 2 * kmax)
                              : gemm_f64_emulated_scratch((int)n, (int)n, kmax);
  if (s.fp32_tc) ozb = std::max(ozb, gemm_tc32_scratch((int)n, (int)n, kmax));
  size_t ooz = L.add(ozb);
  const bool mixed = s.opts.prec == GEV_MIXED;
  size_t oR1 = L.add(mixed ? n * n * es : 8), oR2 = L.add(mixed ? n * n * es : 8), oR3 = L.add(mixed ? n * n * es : 8);
  size_t oR4 = L.add(mixed && s.dtype == GEV_C128 ? 3 * n * n * es : 8);
  // complex mixed form: staging copy of the FP64 band while it is converted to complex64
  size_t obt = L.add(mixed && s.dtype == GEV_C128 ? (size_t)ldband * (n + 2 * b) * es : 8);
  // back-transform 1 groups of four panels: the group's T, Gram blocks and one block column
  size_t obtg = L.add(36 * b * b * es);
  if (base) {
    s.A = base + oA; s.X = base + oX; s.W1 = base + oW1; s.V1 = base + oV1; s.T1 = base + oT1;
    s.dinv = base + odinv; s.Pn = base + oPn; s.small = base + osmall;
    s.splitws = base + osplit; s.splitws_bytes = split;
    s.band = base + oband; s.ldband = ldband;
    s.V2 = base + oV2; s.tau2 = base + otau2; s.ntask = (int)ntask; s.phase = base + ophase;
    s.d = (double*)(base + od); s.e = (double*)(base + oe); s.w = (double*)(base + ow);
    s.Q = (double*)(base + oQ); s.q_bytes = qbytes; s.Q2 = (double*)(base + oQ2);
    s.dcws = base + odc; s.dcws_bytes = dcws;
    s.Yk = base + oYk;
    s.Zk = (double*)(base + oZk);
    s.prog = (int*)(base + oprog);
    s.panelws = base + opanel; s.panelws_bytes = panel;
    s.status = (int*)(base + ost);
    s.ozws = ozb ? base + ooz : nullptr;
    s.ozws_bytes = ozb;
    s.R1 = (double*)(base + oR1);
    s.R2 = (double*)(base + oR2);
    s.R3 = (double*)(base + oR3);
    s.R4 = (double*)(base + oR4);
    s.bandtmp = base + obt;
    s.btg = base + obtg;
  }
  return L.total;
}

void fill_defaults(gev_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->cuda_stream = nullptr;
  o->prec = GEV_PLAIN;
  o->band_b = 0;
  o->panel_nb = 0;
  o->refine_tol = 1e-11;
  o->refine_max_iter = 4;
  o->workspace_limit = 0;
  o->timing = 0;
  o->fp64_emulation = -1;
  o->fp32_products = -1;
}

int init_sys(Sys& s, int n, int dtype, const gev_opts* opts) {
  s.n = n;
  s.dtype = dtype;
  if (opts) s.opts = *opts; else fill_defaults(&s.opts);
  if (s.opts.refine_tol <= 0) s.opts.refine_tol = 1e-11;
  if (s.opts.refine_max_iter <= 0) s.opts.refine_max_iter = 4;
  s.stream = (cudaStream_t)s.opts.cuda_stream;
  s.nb = 64;
  if (s.opts.panel_nb > 0 && s.opts.panel_nb < 64) s.nb = (s.opts.panel_nb + 7) / 8 * 8;
  s.b = pick_band(n, s.opts.band_b);
  s.emu_fp64 = s.opts.fp64_emulation < 0 ? 1 : (s.opts.fp64_emulation ? 1 : 0);
  s.fp32_tc = 0;
  if (s.opts.prec == GEV_MIXED) {
    const int f = s.opts.fp32_products;
    s.fp32_tc = (f < 0 || f == 6) ? 6 : (f == 3 ? 3 : 0);
  }
  return 0;
}

template <class T> int solve_t(Sys& s, const T* H, int ldh, const T* S, int lds, int k, double* evals,
                               T* C, int ldc, gev_report* rep);

}  // namespace

namespace gev {
Sys& sys_of(gev_sys* h) { return h->s; }
}  // namespace gev

extern "C" {

void gev_default_opts(gev_opts* opts) {
  if (opts) fill_defaults(opts);
}

const char* gev_strerror(int code) {
  switch (code) {
    case GEV_OK: return "ok";
    case GEV_ERR_NOT_SPD: return "S is not positive definite";
    case GEV_ERR_NO_CONVERGENCE: return "iteration cap reached without convergence";
    case GEV_ERR_TIMEOUT: return "a bounded device wait timed out";
    case GEV_ERR_OOM: return "device workspace allocation failed or exceeds the limit";
    case GEV_ERR_CUDA: return "CUDA runtime error";
    case GEV_ERR_REUSE_WITHOUT_FACTOR: return "S == NULL but no resident factor is held";
    case GEV_ERR_UNSUPPORTED: return "unsupported option combination";
    case GEV_ERR_RANK: return "fewer than k eigenvalues of S reach delta";
    default: return code < 0 ? "invalid argument" : "unknown error";
  }
}

size_t gev_workspace_bytes(int n, int dtype, const gev_opts* opts) {
  if (n < 1 || (dtype != GEV_F64 && dtype != GEV_C128)) return 0;
  Sys s;
  init_sys(s, n, dtype, opts);
  return carve(s, nullptr);
}

int gev_setup(gev_sys** out, int n, int dtype, const gev_opts* opts) {
  if (!out) return -1;
  *out = nullptr;
  if (n < 1) return -2;
  if (dtype != GEV_F64 && dtype != GEV_C128) return -3;
  gev_sys* h = new (std::nothrow) gev_sys();
  if (!h) return GEV_ERR_OOM;
  Sys& s = h->s;
  init_sys(s, n, dtype, opts);
  if (cudaSetDevice(s.opts.device) != cudaSuccess) {
    delete h;
    return -4;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s.opts.device);
  if (sms > 0) s.sms = sms;
  size_t bytes = carve(s, nullptr);
  if (s.opts.workspace_limit && bytes > s.opts.workspace_limit) {
    delete h;
    return GEV_ERR_OOM;
  }
  if (cudaMalloc((void**)&s.base, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GEV_ERR_OOM;
  }
  s.bytes = bytes;
  carve(s, s.base);
  if (cudaMallocHost((void**)&s.status_h, sizeof(int) * ST_COUNT) != cudaSuccess) {
    cudaFree(s.base);
    delete h;
    return GEV_ERR_OOM;
  }
  for (int i = 0; i < 2 * GEV_NSTEPS + 2; ++i) cudaEventCreate(&s.ev[i]);
  if (cudaMemsetAsync(s.status, 0, sizeof(int) * ST_COUNT, s.stream) != cudaSuccess ||
      cudaStreamSynchronize(s.stream) != cudaSuccess) {
    gev_free(h);
    return GEV_ERR_CUDA;
  }
  *out = h;
  return 0;
}

int gev_free(gev_sys* h) {
  if (!h) return 0;
  Sys& s = h->s;
  if (s.sub) {
    gev_free((gev_sys*)s.sub);
    s.sub = nullptr;
  }
  cudaSetDevice(s.opts.device);
  if (s.stream) cudaStreamSynchronize(s.stream);
  else cudaDeviceSynchronize();
  for (int i = 0; i < 2 * GEV_NSTEPS + 2; ++i)
    if (s.ev[i]) cudaEventDestroy(s.ev[i]);
  for (cudaEvent_t e : s.gemm_ev) cudaEventDestroy(e);
  if (s.base) cudaFree(s.base);
  if (s.status_h) cudaFreeHost(s.status_h);
  delete h;
  return 0;
}

int gev_reuse_factor(gev_sys* h, int enable) {
  if (!h) return -1;
  h->s.reuse = enable != 0;
  if (!enable) h->s.have_factor = false;
  return 0;
}

int gev_solve(gev_sys* h, const void* H, int ldh, const void* S, int lds, int k, double* evals,
              void* C, int ldc, gev_report* rep) {
  if (!h) return -1;
  Sys& s = h->s;
  const int n = s.n;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (S && lds < n) return -5;
  if (k < 1 || k > n) return -6;
  if (!evals) return -7;
  if (!C) return -8;
  if (ldc < n) return -9;
  if (!S && !(s.reuse && s.have_factor && s.factor_kind == 0)) return GEV_ERR_REUSE_WITHOUT_FACTOR;
  if (cudaSetDevice(s.opts.device) != cudaSuccess) return GEV_ERR_CUDA;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  if (s.opts.one_stage == 1 && s.opts.prec == GEV_MIXED && s.dtype == GEV_C128) return GEV_ERR_UNSUPPORTED;
  int r;
  if (s.opts.prec == GEV_MIXED && s.dtype == GEV_C128)
    r = solve_mixed_cx(s, (const zd*)H, ldh, (const zd*)S, lds, k, evals, (zd*)C, ldc, rep);
  else if (s.dtype == GEV_C128)
    r = solve_t<zd>(s, (const zd*)H, ldh, (const zd*)S, lds, k, evals, (zd*)C, ldc, rep);
  else if (s.opts.prec == GEV_MIXED)
    r = solve_mixed(s, (const double*)H, ldh, (const double*)S, lds, k, evals, (double*)C, ldc, rep);
  else
    r = solve_t<double>(s, (const double*)H, ldh, (const double*)S, lds, k, evals, (double*)C, ldc, rep);
  if (rep) {
    rep->workspace_bytes = s.bytes;
    rep->resid = -1.0;
    rep->ortho = -1.0;
  }
  if (r == 0 && s.opts.check && S && rep) {
    // the accuracy of the returned pencil solution, on the device (two more products with C)
    const int rc = s.dtype == GEV_C128
                       ? measure<zd>(s, (const zd*)H, ldh, (const zd*)S, lds, k, evals, (const zd*)C, ldc,
                                     &rep->resid, &rep->ortho)
                       : measure<double>(s, (const double*)H, ldh, (const double*)S, lds, k, evals,
                                         (const double*)C, ldc, &rep->resid, &rep->ortho);
    if (rc) return rc;
  }
  return r;
}

int gev_solve_reduced(gev_sys* h, const void* H, int ldh, const void* S, int lds, double delta, int k,
                      double* evals, void* C, int ldc, int* m_kept, gev_report* rep) {
  if (!h) return -1;
  Sys& s = h->s;
  const int n = s.n;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (S && lds < n) return -5;
  if (!(delta >= 0.0) || delta > 1e300) return -6;
  if (k < 1 || k > n) return -7;
  if (!evals) return -8;
  if (!C) return -9;
  if (ldc < n) return -10;
  if (!S && !(s.reuse && s.have_factor && s.factor_kind == 1)) return GEV_ERR_REUSE_WITHOUT_FACTOR;
  if (cudaSetDevice(s.opts.device) != cudaSuccess) return GEV_ERR_CUDA;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  const int r = s.dtype == GEV_C128
                    ? solve_reduced<zd>(s, (const zd*)H, ldh, (const zd*)S, lds, delta, k, evals, (zd*)C, ldc,
                                        m_kept, rep)
                    : solve_reduced<double>(s, (const double*)H, ldh, (const double*)S, lds, delta, k, evals,
                                            (double*)C, ldc, m_kept, rep);
  if (rep) {
    rep->workspace_bytes = s.bytes;
    rep->resid = -1.0;
    rep->ortho = -1.0;
  }
  if (r == 0 && s.opts.check && S && rep) {
    const int rc = s.dtype == GEV_C128
                       ? measure<zd>(s, (const zd*)H, ldh, (const zd*)S, lds, k, evals, (const zd*)C, ldc,
                                     &rep->resid, &rep->ortho)
                       : measure<double>(s, (const double*)H, ldh, (const double*)S, lds, k, evals,
                                         (const double*)C, ldc, &rep->resid, &rep->ortho);
    if (rc) return rc;
  }
  return r;
}

int gev_check(gev_sys* h, const void* H, int ldh, const void* S, int lds, int k, const double* evals,
              const void* C, int ldc, double* resid, double* ortho) {
  if (!h) return -1;
  Sys& s = h->s;
  const int n = s.n;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (!S) return -4;
  if (lds < n) return -5;
  if (k < 1 || k > n) return -6;
  if (!evals) return -7;
  if (!C) return -8;
  if (ldc < n) return -9;
  if (!resid) return -10;
  if (!ortho) return -11;
  if (cudaSetDevice(s.opts.device) != cudaSuccess) return GEV_ERR_CUDA;
  GEV_TRY(reset_status(s));
  return s.dtype == GEV_C128 ? measure<zd>(s, (const zd*)H, ldh, (const zd*)S, lds, k, evals, (const zd*)C, ldc,
                                           resid, ortho)
                             : measure<double>(s, (const double*)H, ldh, (const double*)S, lds, k, evals,
                                               (const double*)C, ldc, resid, ortho);
}

int gev_density(gev_sys* h, int k, const void* C, int ldc, const double* occ, const double* evals, void* P,
                int ldp, void* PE, int ldpe) {
  if (!h) return -1;
  Sys& s = h->s;
  const int n = s.n;
  if (k < 1 || k > n) return -2;
  if (!C) return -3;
  if (ldc < n) return -4;
  if (!occ) return -5;
  if (PE && !evals) return -6;
  if (!P) return -7;
  if (ldp < n) return -8;
  if (PE == P) return -9;
  if (PE && ldpe < n) return -10;
  if (cudaSetDevice(s.opts.device) != cudaSuccess) return GEV_ERR_CUDA;
  s.account = false;
  GEV_TRY(reset_status(s));
  int r = s.dtype == GEV_C128
              ? density<zd>(s, k, (const zd*)C, ldc, occ, evals, (zd*)P, ldp, (zd*)PE, ldpe)
              : density<double>(s, k, (const double*)C, ldc, occ, evals, (double*)P, ldp, (double*)PE, ldpe);
  if (r) return r;
  GEV_TRY(sync_status(s));
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  return 0;
}

// ------------------------------------------------------------------------------ step entries --
#define STEP_PROLOGUE(h)                                            \
  if (!h) return -1;                                                \
  Sys& s = h->s;                                                    \
  if (cudaSetDevice(s.opts.device) != cudaSuccess) return GEV_ERR_CUDA;

int gev_step_potrf(gev_sys* h, void* A, int lda, int* info) {
  STEP_PROLOGUE(h)
  if (!A) return -2;
  if (lda < s.n) return -3;
  GEV_TRY(reset_status(s));
  int r = s.dtype == GEV_C128 ? potrf<zd>(s, (zd*)A, lda) : potrf<double>(s, (double*)A, lda);
  if (r) return r;
  GEV_TRY(sync_status(s));
  if (info) *info = s.status_h[ST_NOT_SPD];
  return s.status_h[ST_NOT_SPD] ? GEV_ERR_NOT_SPD : 0;
}

int gev_step_trtri(gev_sys* h, void* A, int lda) {
  STEP_PROLOGUE(h)
  if (!A) return -2;
  if (lda < s.n) return -3;
  int r = s.dtype == GEV_C128 ? trtri<zd>(s, (zd*)A, lda) : trtri<double>(s, (double*)A, lda);
  if (r) return r;
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}

int gev_step_hegst(gev_sys* h, const void* H, int ldh, const void* X, int ldx, void* A, int lda) {
  STEP_PROLOGUE(h)
  if (!H) return -2;
  if (ldh < s.n) return -3;
  if (!X) return -4;
  if (ldx < s.n) return -5;
  if (!A) return -6;
  if (lda < s.n) return -7;
  int r = s.dtype == GEV_C128
              ? hegst<zd>(s, (const zd*)H, ldh, (const zd*)X, ldx, (zd*)A, lda)
              : hegst<double>(s, (const double*)H, ldh, (const double*)X, ldx, (double*)A, lda);
  if (r) return r;
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}

int gev_step_he2hb(gev_sys* h, void* A, int lda, int b, int* b_used) {
  STEP_PROLOGUE(h)
  if (!A) return -2;
  if (lda < s.n) return -3;
  if (b != 0 && (b < 16 || b > 64)) return -4;
  int bb = b ? pick_band(s.n, b) : s.b;
  if (bb > s.b) return GEV_ERR_UNSUPPORTED;  // workspace sized for the handle's band width
  int r = s.dtype == GEV_C128 ? he2hb<zd>(s, (zd*)A, lda, bb) : he2hb<double>(s, (double*)A, lda, bb);
  if (r) return r;
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  if (b_used) *b_used = s.band_b_used;
  return 0;
}

int gev_step_he2td(gev_sys* h, void* A, int lda, double* d, double* e) {
  STEP_PROLOGUE(h)
  if (!A) return -2;
  if (lda < s.n) return -3;
  if (!d) return -4;
  if (!e && s.n > 1) return -5;
  GEV_TRY(reset_status(s));
  int r = s.dtype == GEV_C128 ? he2td<zd>(s, (zd*)A, lda) : he2td<double>(s, (double*)A, lda);
  if (r) return r;
  GEV_TRY(sync_status(s));
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  GEV_CUDA_TRY(cudaMemcpyAsync(d, s.d, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, s.stream));
  if (s.n > 1)
    GEV_CUDA_TRY(cudaMemcpyAsync(e, s.e, sizeof(double) * (s.n - 1), cudaMemcpyDeviceToDevice, s.stream));
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}

int gev_step_hb2st(gev_sys* h, double* d, double* e) {
  STEP_PROLOGUE(h)
  if (!d) return -2;
  if (!e && s.n > 1) return -3;
  if (!s.have_band) return GEV_ERR_UNSUPPORTED;
  GEV_TRY(reset_status(s));
  int r = s.dtype == GEV_C128 ? hb2st<zd>(s, d, e) : hb2st<double>(s, d, e);
  if (r) return r;
  GEV_TRY(sync_status(s));
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  return 0;
}

int gev_step_stedc(gev_sys* h, const double* d, const double* e, int k, double* w, double* Z, int ldz,
                   int* deflated) {
  STEP_PROLOGUE(h)
  if (!d) return -2;
  if (!e && s.n > 1) return -3;
  if (k < 1 || k > s.n) return -4;
  if (!w) return -5;
  if (!Z) return -6;
  if (ldz < s.n) return -7;
  GEV_TRY(reset_status(s));
  int r = stedc(s, d, e, k, w, Z, ldz, deflated);
  if (r) return r;
  GEV_TRY(sync_status(s));
  if (deflated) *deflated = s.status_h[ST_DEFLATED];
  if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  return 0;
}

int gev_step_back(gev_sys* h, const double* Z, int ldz, int k, void* Y, int ldy) {
  STEP_PROLOGUE(h)
  if (!Z) return -2;
  if (ldz < s.n) return -3;
  if (k < 1 || k > s.n) return -4;
  if (!Y) return -5;
  if (ldy < s.n) return -6;
  if (!s.one_stage_used && (!s.have_band || !s.have_tridiag_refl)) return GEV_ERR_UNSUPPORTED;
  s.z_unit = false;  // the caller's Z: no bound on its entries is assumed
  int r = s.dtype == GEV_C128 ? back<zd>(s, Z, ldz, k, (zd*)Y, ldy) : back<double>(s, Z, ldz, k, (double*)Y, ldy);
  if (r) return r;
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}

int gev_step_mult(gev_sys* h, const void* X, int ldx, const void* Y, int ldy, int k, void* C, int ldc) {
  STEP_PROLOGUE(h)
  if (!X) return -2;
  if (ldx < s.n) return -3;
  if (!Y) return -4;
  if (ldy < s.n) return -5;
  if (k < 1 || k > s.n) return -6;
  if (!C) return -7;
  if (ldc < s.n) return -8;
  int r = s.dtype == GEV_C128 ? mult<zd>(s, (const zd*)X, ldx, (const zd*)Y, ldy, k, (zd*)C, ldc)
                              : mult<double>(s, (const double*)X, ldx, (const double*)Y, ldy, k, (double*)C, ldc);
  if (r) return r;
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  return 0;
}

}  // extern "C"

namespace {

template <class T> int solve_t(Sys& s, const T* H, int ldh, const T* S, int lds, int k, double* evals,
                               T* C, int ldc, gev_report* rep) {
  const int n = s.n;
  const bool timing = s.opts.timing != 0;
  s.n_marks = 0;
  auto mark = [&](int step) { step_mark(s, step); };
  T* A = (T*)s.A;
  T* X = (T*)s.X;
  s.launches = 0;
  s.gemm_used = 0;
  s.account = s.opts.timing == 2;
  GEV_TRY(reset_status(s));
  mark(GEV_STEP_CHOLESKY);
  const bool reuse = (S == nullptr);
  if (!reuse) {
    // steps 1-2: X = L^{-1}, S = L L^H
    GEV_TRY(copy_lower<T>(s, n, S, lds, X, n));
    // Cholesky and inversion in one recursion (the "invert" step time is included in "cholesky")
    GEV_TRY(potrf_inv<T>(s, X, n));
    GEV_TRY(sync_status(s));
    if (s.status_h[ST_NOT_SPD]) {
      if (rep) rep->info = s.status_h[ST_NOT_SPD];
      s.have_factor = false;
      return GEV_ERR_NOT_SPD;
    }
    mark(GEV_STEP_INVERT);
  } else {
    mark(GEV_STEP_INVERT);
  }
  if (rep) rep->reused_factor = reuse ? 1 : 0;
  // step 3: A = X H X^H
  mark(GEV_STEP_MULTIPLY);
  GEV_TRY(hegst<T>(s, H, ldh, X, n, A, n));
  s.have_factor = true;
  s.factor_kind = 0;
  const bool one = one_stage_for(s.opts.one_stage, n, k);
  // steps 4a / 4b: two-stage tridiagonalisation (or the one-stage reduction, timed as "to_tridiag")
  mark(GEV_STEP_TO_BAND);
  if (!one) GEV_TRY(he2hb<T>(s, A, n, s.b));
  mark(GEV_STEP_TO_TRIDIAG);
  if (one) GEV_TRY(he2td<T>(s, A, n));
  else GEV_TRY(hb2st<T>(s, s.d, s.e));
  GEV_TRY(stop_on_timeout(s));
  // step 5: divide and conquer, k lowest vectors
  mark(GEV_STEP_SOLVE);
  GEV_TRY(stedc(s, s.d, s.e, k, s.w, s.Zk, n, nullptr));
  // step 6: Y = Q1 Q2 Z (one stage: Y = Q Z, timed as "back_tridiag")
  mark(GEV_STEP_BACK_TRIDIAG);
  T* Y = (T*)s.Yk;
  s.z_unit = true;  // the divide-and-conquer eigenvectors
  if (one) GEV_TRY(back_td<T>(s, s.Zk, n, k, Y, n));
  else GEV_TRY(bt_hb2st<T>(s, s.Zk, n, k, Y, n));
  s.z_unit = false;
  mark(GEV_STEP_BACK_BAND);
  if (!one) GEV_TRY(bt_he2hb<T>(s, Y, n, k));
  // step 7: C = X^H Y
  mark(GEV_STEP_MULT);
  GEV_TRY(mult<T>(s, X, n, Y, n, k, C, ldc));
  GEV_TRY(normalize_phase<T>(s, n, k, C, ldc));
  GEV_CUDA_TRY(cudaMemcpyAsync(evals, s.w, sizeof(double) * k, cudaMemcpyDeviceToDevice, s.stream));
  mark(-1);
  GEV_TRY(sync_status(s));
  if (!s.reuse) s.have_factor = false;
  if (rep) {
    rep->deflated = s.status_h[ST_DEFLATED];
    rep->launches = s.launches;
    if (s.account) gemm_account(s, &rep->gemm_calls, &rep->gemm_ms, &rep->gemm_flops);
    if (timing) step_collect(s, rep->ms);
  }
  if (s.status_h[ST_TIMEOUT]) return GEV_ERR_TIMEOUT;
  if (s.status_h[ST_NOCONV]) return GEV_ERR_NO_CONVERGENCE;
  return 0;
}

}  // namespace
