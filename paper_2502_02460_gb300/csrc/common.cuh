// Shared definitions of the GB300 generalized eigensolver: scalar types, the handle, launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "gev.h"
#include "gev_steps.h"

namespace gev {

// ------------------------------------------------------------------------------ scalar types --
// complex128, interleaved (re, im) like C99 double complex.
struct alignas(16) zd {
  double x, y;
};

__host__ __device__ __forceinline__ zd make_zd(double a, double b) { return zd{a, b}; }
__host__ __device__ __forceinline__ zd operator+(zd a, zd b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ zd operator-(zd a, zd b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ zd operator-(zd a) { return {-a.x, -a.y}; }
__host__ __device__ __forceinline__ zd operator*(zd a, zd b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ zd operator*(double s, zd a) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zd operator*(zd a, double s) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zd& operator+=(zd& a, zd b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ zd& operator-=(zd& a, zd b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ __forceinline__ bool operator==(zd a, zd b) { return a.x == b.x && a.y == b.y; }
__host__ __device__ __forceinline__ bool operator!=(zd a, zd b) { return !(a == b); }

// complex64, interleaved (re, im): the FP32 stages of the complex mixed form
struct alignas(8) zf {
  float x, y;
};

__host__ __device__ __forceinline__ zf make_zf(float a, float b) { return zf{a, b}; }
__host__ __device__ __forceinline__ zf operator+(zf a, zf b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ zf operator-(zf a, zf b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ zf operator-(zf a) { return {-a.x, -a.y}; }
__host__ __device__ __forceinline__ zf operator*(zf a, zf b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ zf operator*(float s, zf a) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zf operator*(zf a, float s) { return {s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zf& operator+=(zf& a, zf b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ zf& operator-=(zf& a, zf b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ __forceinline__ bool operator==(zf a, zf b) { return a.x == b.x && a.y == b.y; }
__host__ __device__ __forceinline__ bool operator!=(zf a, zf b) { return !(a == b); }
__host__ __device__ __forceinline__ zf conj_(zf a) { return {a.x, -a.y}; }
__host__ __device__ __forceinline__ float re_(zf a) { return a.x; }
__host__ __device__ __forceinline__ float im_(zf a) { return a.y; }
__host__ __device__ __forceinline__ float abs2_(zf a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float abs_(zf a) { return hypotf(a.x, a.y); }
__host__ __device__ __forceinline__ zf mulc(zf a, zf b) { return a * conj_(b); }
__host__ __device__ __forceinline__ zf cmul(zf a, zf b) { return conj_(a) * b; }
__host__ __device__ __forceinline__ zf div_(zf a, zf b) {
  float d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

__host__ __device__ __forceinline__ float conj_(float a) { return a; }
__host__ __device__ __forceinline__ float re_(float a) { return a; }
__host__ __device__ __forceinline__ float im_(float) { return 0.0f; }
__host__ __device__ __forceinline__ float abs2_(float a) { return a * a; }
__host__ __device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__host__ __device__ __forceinline__ float mulc(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ float cmul(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ float div_(float a, float b) { return a / b; }
__host__ __device__ __forceinline__ double conj_(double a) { return a; }
__host__ __device__ __forceinline__ zd conj_(zd a) { return {a.x, -a.y}; }
__host__ __device__ __forceinline__ double re_(double a) { return a; }
__host__ __device__ __forceinline__ double re_(zd a) { return a.x; }
__host__ __device__ __forceinline__ double im_(double) { return 0.0; }
__host__ __device__ __forceinline__ double im_(zd a) { return a.y; }
__host__ __device__ __forceinline__ double abs2_(double a) { return a * a; }
__host__ __device__ __forceinline__ double abs2_(zd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double abs_(double a) { return fabs(a); }
__host__ __device__ __forceinline__ double abs_(zd a) { return hypot(a.x, a.y); }
template <class T> __host__ __device__ __forceinline__ T from_re(double a);
template <> __host__ __device__ __forceinline__ double from_re<double>(double a) { return a; }
template <> __host__ __device__ __forceinline__ float from_re<float>(double a) { return (float)a; }
template <> __host__ __device__ __forceinline__ zd from_re<zd>(double a) { return {a, 0.0}; }
template <> __host__ __device__ __forceinline__ zf from_re<zf>(double a) { return {(float)a, 0.0f}; }
template <class T> __host__ __device__ __forceinline__ T zero_() { return from_re<T>(0.0); }
// a * conj(b) and conj(a) * b
__host__ __device__ __forceinline__ double mulc(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ zd mulc(zd a, zd b) { return a * conj_(b); }
__host__ __device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ zd cmul(zd a, zd b) { return conj_(a) * b; }
__host__ __device__ __forceinline__ zd div_(zd a, zd b) {
  double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__host__ __device__ __forceinline__ double div_(double a, double b) { return a / b; }

// L2-coherent loads/stores (bypass L1) for data another block may have written during the kernel.
__device__ __forceinline__ float ldcg_(const float* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg_(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ double ldcg_(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zd ldcg_(const zd* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return make_zd(v.x, v.y);
}
__device__ __forceinline__ void stcg_(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stcg_(zd* p, zd v) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v.x, v.y));
}
__device__ __forceinline__ zf ldcg_(const zf* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return make_zf(v.x, v.y);
}
__device__ __forceinline__ void stcg_(zf* p, zf v) { __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y)); }

template <class T> struct is_cx { static constexpr bool value = false; };
template <> struct is_cx<zd> { static constexpr bool value = true; };
template <> struct is_cx<zf> { static constexpr bool value = true; };
// real type of a scalar type, and the FP64 type of the same field
template <class T> struct real_of { using type = double; };
template <> struct real_of<float> { using type = float; };
template <> struct real_of<zf> { using type = float; };

// ------------------------------------------------------------------------- status word slots --
enum StatusSlot {
  ST_NOT_SPD = 0,       // pivot index + 1 of the first non-positive Cholesky pivot
  ST_TIMEOUT = 1,       // non-zero: a bounded device wait gave up (value = site code)
  ST_NOCONV = 2,        // non-zero: an iteration cap was hit (value = site code)
  ST_DEFLATED = 3,      // eigenpairs deflated in the top merge
  ST_BARRIER_GEN = 4,   // grid-barrier generation counter (cooperative kernels)
  ST_BARRIER_CNT = 5,   // grid-barrier arrival counter
  ST_ABORT = 6,         // non-zero once a cooperative kernel gave up waiting
  ST_CONFIG = 7,        // non-zero: a launch could not be configured (site code); reported as GEV_ERR_CUDA
  ST_SPIN = 8,          // iteration limit of every bounded device wait (0: kSpinLimit); set by the host
  ST_STALL = 9,         // a flag nothing ever sets: the bulge chase waits on it when asked to stall
  ST_COUNT = 16
};

// Bounded spin limit for every device-side wait (iterations of a ~100 ns nanosleep loop).
constexpr long long kSpinLimit = 20000000;  // ~2 s

// The wait limit of the current launch: status[ST_SPIN] when the host set one (gev_opts.wait_limit),
// else kSpinLimit.  Read once per wait, through L2.
__device__ __forceinline__ long long spin_limit(const int* status) {
  const int v = status ? __ldcg(&status[ST_SPIN]) : 0;
  return v > 0 ? (long long)v : kSpinLimit;
}

// -------------------------------------------------------------------------------------- GEMM --
// C[M x N] = alpha op(A) op(B) + beta C, column-major.
//   ta/tb: 0 = N, 1 = T, 2 = C (conjugate transpose)
//   tri_a: 1 -> op(A)[i,k] = 0 for k > i (lower); 2 -> zero for k < i (upper)
//   tri_b: 1 -> op(B)[k,j] = 0 for k < j (lower); 2 -> zero for k > j (upper)
//   c_lower: only entries i >= j of C are computed and written.
// Zero patterns are applied element by element when loading, so the stored "zero" triangle of a
// triangular operand is never read.
template <class T> struct GemmP {
  int M, N, K;
  int ta, tb;
  int tri_a, tri_b, c_lower;
  T alpha, beta;
  const T* A;
  long long lda;
  const T* B;
  long long ldb;
  T* C;
  long long ldc;
  int ksplit;  // set by the launcher
  T* ws;       // split-K partials (launcher-owned)
  int lowp;    // 1: FP64 operands, products and sums in FP32 (mixed form); 0: native precision
};

struct Sys;

template <class T> void gemm(Sys& s, GemmP<T> p);
// FP32 SIMT GEMM (gemm32.cu): inputs TI (float or double, converted on load), output TO.
template <class TI, class TO> void gemm32(Sys& s, const GemmP<TI>& p, TO* C, float alpha, float beta);
// FP32 GEMM from BF16 split products on tcgen05 (tc_gemm.cu); false when s.ozws is too small
template <class TI, class TO>
bool gemm_tc32(Sys& s, const GemmP<TI>& q, TO* C, float alpha, float beta, int nprod);
size_t gemm_tc32_scratch(int M, int N, int K);  // bytes of s.ozws for an M x N x K product
template <> void gemm<float>(Sys& s, GemmP<float> p);  // FP32: gemm32<float, float>
void gemm_account(Sys& s, int* calls, double* ms, double* flops);
void gemm_f64_emulated(Sys& s, const GemmP<double>& p);
void gemm_c128_emulated(Sys& s, const GemmP<zd>& p);  // real alpha, beta
size_t gemm_f64_emulated_scratch(int M, int N, int K);  // bytes of s.ozws for an M x N x K product

// A block-diagonal operand of the back-transform-2 products: the reflector blocks
// D_j = H(s0) H(s0 + 1) ... H(s0 + b - 1) = I - V_j T_j V_j^H of one level of the band -> tridiagonal
// back-transform (block j: group g = g_lo + j, task t = L - (ngroups - 1 - g), sweeps s0 = g b ..;
// it acts on rows [w00 + 2 b j, w00 + 2 b j + 2 b)).
//   kind 1: op(A) = blockdiag(V_j^H), b x 2b blocks (row q: the reflector of sweep s0 + q, read from
//           the bulge-chasing store V2 / tau2; a reflector with tau = 0 counts as zero)
//   kind 2: op(A) = blockdiag(W_j), 2b x b blocks, W_j = V_j T_j stored column-major at W + j 2b b
// Complex data (cx) enter through the real 2 x 2 embedding like every emulated complex product.
struct BdOp {
  int kind, cx, b, n, ntask, g_lo, L, ngroups, nblk, w00;
  const void* V2;
  const void* tau2;
  const void* W;
};
// C (M x N) = alpha op(A) B + beta C, op(A) the block-diagonal operand (blocks bm x bk; M, K, bm, bk in
// complex units for complex data), B (K x N, ld ldb) and C (ld ldc) as stored, on the emulated FP64
// product engine; each output tile reads only its blocks' K range.  b_below_two: the caller
// guarantees every entry (real and imaginary part) of B is below 2 in magnitude, so the column
// scales are fixed at 2 without a pass over B.  Returns false (nothing launched) when s.ozws is too
// small: gemm_f64_bdiag_scratch gives the bytes.
bool gemm_f64_bdiag(Sys& s, int M, int N, int K, const BdOp& a, int bm, int bk, const void* B, long long ldb,
                    double alpha, double beta, void* C, long long ldc, bool b_below_two);
size_t gemm_f64_bdiag_scratch(int M, int N, int K, int bm, int bk, int cx);
// The same in FP32 from BF16x6 (or x3, s.fp32_tc) split products on the tensor cores (tc_gemm.cu);
// real data only.
bool gemm_f32_bdiag(Sys& s, int M, int N, int K, const BdOp& a, int bm, int bk, const float* B, long long ldb,
                    float alpha, float beta, float* C, long long ldc);
size_t gemm_f32_bdiag_scratch(int M, int N, int K, int bm, int bk);
template <class T> GemmP<T> gp(int M, int N, int K, int ta, int tb, T alpha, const T* A, long long lda,
                               const T* B, long long ldb, T beta, T* C, long long ldc) {
  GemmP<T> p{};
  p.M = M; p.N = N; p.K = K; p.ta = ta; p.tb = tb; p.alpha = alpha; p.beta = beta;
  p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc;
  return p;
}

// ---------------------------------------------------------------------------------- the handle --
struct Sys {
  int n = 0;
  int dtype = GEV_F64;
  gev_opts opts{};
  cudaStream_t stream = nullptr;
  int nb = 64;      // Cholesky / inversion block
  int b = 64;       // band width of the full -> band step
  int sms = 152;

  // workspace (device)
  char* base = nullptr;
  size_t bytes = 0;
  void* A = nullptr;      // n x n working matrix (element size es)
  void* X = nullptr;      // n x n resident L^{-1}
  void* W1 = nullptr;     // n x n scratch
  void* V1 = nullptr;     // n x n compact-WY vectors of the full -> band step
  void* T1 = nullptr;     // b x n triangular factors of the full -> band step
  void* dinv = nullptr;   // nb x n inverted diagonal blocks (Cholesky / inversion)
  void* Pn = nullptr;     // n x 2b panel scratch (x 4 buffers)
  void* small = nullptr;  // b x b scratch (x 4)
  void* splitws = nullptr;  // split-K partials
  size_t splitws_bytes = 0;
  void* band = nullptr;   // compact band, ldband x n
  void* bandtmp = nullptr;  // complex mixed form: FP64 copy of the band during its conversion
  void* btg = nullptr;      // back-transform 1: T, Gram blocks and a block column of a 4-panel group (36 b^2)
  int ldband = 0;
  void* V2 = nullptr;     // bulge-chasing reflectors, b x (n * ntask)
  void* tau2 = nullptr;   // (n * ntask)
  int ntask = 0;          // max tasks per sweep
  void* phase = nullptr;  // complex: diagonal phases folded into back-transform 2 (n)
  double* d = nullptr;    // tridiagonal diagonal (n)
  double* e = nullptr;    // off-diagonal (n)
  double* w = nullptr;    // eigenvalues (n)
  double* Q = nullptr;    // n x n divide-and-conquer eigenvectors (one-stage reduction: symv partial sums)
  size_t q_bytes = 0;
  double* Q2 = nullptr;   // n x n divide-and-conquer scratch
  void* dcws = nullptr;   // divide-and-conquer per-level workspace
  size_t dcws_bytes = 0;
  void* Yk = nullptr;     // n x n back-transformed vectors (element size es)
  double* Zk = nullptr;   // n x n eigenvectors of the tridiagonal (divide-and-conquer output)
  int* prog = nullptr;    // n per-sweep progress counters of the bulge chasing
  int nsbr_panels = 0;    // panels of the last full -> band (or one-stage) reduction
  int q1_pw = 0;          // their width (reflectors per panel)
  int q1_off = 0;         // first row of panel p's block: p * q1_pw + q1_off (b, or 1 for one stage)
  int q1_nrefl = 0;       // reflectors in all (the last panel may be narrower)
  bool one_stage_used = false;  // the last reduction was the one-stage one (no band, no Q2)
  int dc_lowp = 0;        // 1: divide-and-conquer merge products in FP32 (mixed form)
  double* R1 = nullptr;   // mixed form: n x n FP64 refinement buffers (R1..R3)
  double* R2 = nullptr;
  double* R3 = nullptr;
  double* R4 = nullptr;   // complex mixed form: the k x k Gram and coefficient matrices
  void* sub = nullptr;    // mixed form: handle of the k x k Rayleigh-Ritz pencil (gev_sys*)
  int emu_fp64 = 0;       // 1: real FP64 GEMMs formed on the tensor cores (ozaki.cu)
  int fp32_tc = 0;        // FP32 GEMMs: 6 / 3 = BF16x6 / BF16x3 tensor products when large (tc_gemm.cu), 0 = CUDA cores
  void* ozws = nullptr;   // emulated FP64 GEMM: exponents + digit planes (gemm_f64_emulated_scratch)
  size_t ozws_bytes = 0;
  int sub_n = 0;
  void* panelws = nullptr;  // cooperative panel partial sums
  size_t panelws_bytes = 0;
  int* status = nullptr;  // device status words (ST_COUNT ints)
  cudaEvent_t ev[2 * GEV_NSTEPS + 2] = {};
  int ev_step[2 * GEV_NSTEPS + 2] = {};  // step id of each recorded mark (-1: end)
  int n_marks = 0;
  int* status_h = nullptr;  // pinned host mirror
  int spin_h = 0;           // host copy of the wait limit written to status[ST_SPIN]

  // accounting of the current call
  long long launches = 0;
  bool account = false;                 // opts.timing == 2
  std::vector<cudaEvent_t> gemm_ev;     // start/stop pairs
  std::vector<double> gemm_fl;          // algorithmic flops per timed GEMM
  int gemm_used = 0;

  bool have_factor = false;
  int factor_kind = 0;    // resident factor: 0 = X = L^{-1} (Cholesky route), 1 = reduced basis (n x m)
  int reduced_m = 0;      // kept basis size of the reduced route
  bool z_unit = false;    // back-transform input: orthonormal columns (the divide-and-conquer output)
  bool reuse = false;
  bool have_band = false;
  bool have_tridiag_refl = false;
  int band_b_used = 0;

  size_t es() const { return dtype == GEV_C128 ? 16 : 8; }
};

// CUDA error handling: every launcher returns a gev error code.
#define GEV_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      fprintf(stderr, "gev: CUDA error %s at %s:%d\n", cudaGetErrorString(_e), __FILE__, \
              __LINE__);                                                            \
      return GEV_ERR_CUDA;                                                          \
    }                                                                               \
  } while (0)

#define GEV_TRY(expr)        \
  do {                       \
    int _r = (expr);         \
    if (_r != 0) return _r;  \
  } while (0)

inline int last_error() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "gev: CUDA launch error %s\n", cudaGetErrorString(e));
    return GEV_ERR_CUDA;
  }
  return 0;
}

#define GEV_COUNT(s) (++(s).launches)

// Per-step timing with CUDA events on the solve stream: mark(step) starts a step (and ends the
// previous one); the durations are summed per step id after the stream is synchronised.
inline void step_mark(Sys& s, int step);
inline void step_collect(Sys& s, double* ms);

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit on the CURRENT device, once per (kernel, device).
// cudaFuncSetAttribute acts on the current device only, and one process may drive several devices
// (gev_opts.device) from several host threads, so the bookkeeping is per device and under a lock
// (util.cu).  bytes < 0: the most the device allows beside the kernel's static shared memory.
// Returns 0 or GEV_ERR_CUDA (the failing call is reported on stderr).
int set_dyn_smem(const void* func, int bytes);
template <class F> int allow_max_dyn_smem(F* func) { return set_dyn_smem((const void*)func, -1); }
template <class F> int allow_dyn_smem(F* func, size_t bytes) { return set_dyn_smem((const void*)func, (int)bytes); }

// ---------------------------------------------------------------------------- step launchers --
template <class T> int potrf_inv(Sys& s, T* A, int lda);  // S (lower) -> L^{-1}, one recursion
template <class T> int potrf(Sys& s, T* A, int lda);
template <class T> int trtri(Sys& s, T* A, int lda);
template <class T> int hegst(Sys& s, const T* H, int ldh, const T* X, int ldx, T* A, int lda);
template <class T> int mult(Sys& s, const T* X, int ldx, const T* Y, int ldy, int k, T* C, int ldc);
template <class T> int he2hb(Sys& s, T* A, int lda, int b);
template <class T> int hb2st(Sys& s, double* d, double* e);
int stedc(Sys& s, const double* d, const double* e, int k, double* w, double* Z, int ldz, int* deflated);
template <class T> int back(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy);
template <class T> int bt_he2hb(Sys& s, T* Y, int ldy, int k);
// the route of a plain-form solve of order n for k pairs (gev_opts.one_stage: 1 / 2 forced, 0 automatic)
inline bool one_stage_for(int opt, int n, int k) {
  if (opt == 1) return true;
  if (opt == 2) return false;
  return n >= 2048 && (n <= 8192 || 2 * (long long)k >= n);
}
// one-stage Householder tridiagonalisation into s.d / s.e, and Y = Q Z for it (td1.cu)
template <class T> int he2td(Sys& s, T* A, int lda);
template <class T> int back_td(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy);
template <class T> int bt_hb2st(Sys& s, const double* Z, int ldz, int k, T* Y, int ldy);
// P (and PE when non-null) = sum_l g_l conj(C_il) C_jl, g = occ (and occ * evals), both triangles
template <class T>
int density(Sys& s, int k, const T* C, int ldc, const double* occ, const double* evals, T* P, int ldp, T* PE,
            int ldpe);

// element-wise helpers (kernels in util.cu)
template <class T> int copy_lower(Sys& s, int n, const T* S, int lds, T* A, int lda);   // A = tril(S), upper 0
template <class T> int tril_halfdiag(Sys& s, int n, const T* H, int ldh, T* B, int ldb); // B = tril(H), diag/2
template <class T> int herm_sum(Sys& s, int n, const T* M, int ldm, T* A, int lda);     // A = M + M^H (full)
template <class T> int mirror_lower(Sys& s, int n, T* A, int lda);                        // upper <- conj(lower)
template <class T> int zero_upper(Sys& s, int n, T* A, int lda);                          // strict upper <- 0
template <class T> int copy2d(Sys& s, int m, int n, const T* src, long long lds, T* dst, long long ldd);
template <class TA, class TB>
int convert2d(Sys& s, int m, int n, const TA* src, long long lds, TB* dst, long long ldd);
template <class T> int normalize_phase(Sys& s, int n, int k, T* C, int ldc);
int sync_status(Sys& s);  // synchronise the stream, copy the status words to the host mirror
int reset_status(Sys& s);  // zero the status words (and set the wait limit of opts.wait_limit)
// After a step with bounded waits: synchronise, and return GEV_ERR_TIMEOUT when a wait gave up (the
// later steps would only work on the abandoned data).
inline int stop_on_timeout(Sys& s) {
  GEV_TRY(sync_status(s));
  return s.status_h[ST_TIMEOUT] ? GEV_ERR_TIMEOUT : 0;
}
Sys& sys_of(gev_sys* h);  // the handle's state (gev.cu)
// ill-conditioned overlap: the reduced solve in the eigenbasis of S (reduced.cu)
template <class T>
int solve_reduced(Sys& s, const T* H, int ldh, const T* S, int lds, double delta, int k, double* evals, T* C,
                  int ldc, int* m_kept, gev_report* rep);
// gev_opts.check: residual and orthogonality of a solution, on the device (check.cu)
template <class T>
int measure(Sys& s, const T* H, int ldh, const T* S, int lds, int k, const double* evals, const T* C, int ldc,
            double* resid, double* ortho);
// mixed form (mixed.cu): FP32 reduction, FP64 Ogita-Aishima refinement of the standard problem
int solve_mixed(Sys& s, const double* H, int ldh, const double* S, int lds, int k, double* evals,
                double* C, int ldc, gev_report* rep);
int solve_mixed_cx(Sys& s, const zd* H, int ldh, const zd* S, int lds, int k, double* evals, zd* C, int ldc,
                   gev_report* rep);

inline void step_mark(Sys& s, int step) {
  if (!s.opts.timing || s.n_marks >= 2 * GEV_NSTEPS + 2) return;
  s.ev_step[s.n_marks] = step;
  cudaEventRecord(s.ev[s.n_marks], s.stream);
  ++s.n_marks;
}
inline void step_collect(Sys& s, double* ms) {
  for (int i = 0; i < GEV_NSTEPS; ++i) ms[i] = 0.0;
  for (int m = 0; m + 1 < s.n_marks; ++m) {
    const int st = s.ev_step[m];
    if (st < 0 || st >= GEV_NSTEPS) continue;
    float t = 0.f;
    cudaEventElapsedTime(&t, s.ev[m], s.ev[m + 1]);
    ms[st] += t;
  }
}

}  // namespace gev
