/*
 * gev.h -- C ABI of the GB300 dense generalized Hermitian eigensolver.
 *
 * Problem (Eq. 2): H C = S C Lambda with H Hermitian and S Hermitian positive definite, N x N,
 * real FP64 or complex128.  The k lowest eigenpairs are returned.  The path follows the reduction
 * of the section "Current Status of the Implementation" (steps 1-3 and the back-transformation
 * C = U^{-1} C~; Table 1 names the steps Choles., Invert, Multiply, Tridiag., Solve, Back, Mult.):
 *
 *   1  Cholesky          S = L L^H                      (L = U^H; the paper writes S = U^T U)
 *   2  Invert            X = L^{-1}                      (kept resident for SCF reuse)
 *   3  Multiply          A = X H X^H
 *   4a full -> band      A = Q1 B Q1^H   (two-stage tridiagonalisation, "ELPA2")
 *   4b band -> tridiag   B = Q2 T Q2^H   (bulge chasing; T real symmetric)
 *   5  Solve             T = Z Lambda Z^T by divide and conquer
 *   6  Back              Y = Q1 Q2 Z
 *   7  Mult.             C = X^H Y
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major DEVICE pointers with a leading dimension ld >= max(1, n).  Complex
 *     data are interleaved (re, im) doubles (the layout of C99 double complex / complex128).
 *   - Only the lower triangle of H and S is read; the caller's H and S are never written.
 *   - The caller owns H, S, the eigenvalue array and C.  The handle owns its workspace and the
 *     resident factor X = L^{-1}.
 *   - All work is issued on the stream given in gev_opts (0 = legacy default stream) of the device
 *     given there.  Entry points that return results synchronise that stream before returning.
 *   - Eigenvalues ascend.  C is S-orthonormal (C^H S C = I).  In each column the entry of largest
 *     modulus (first index on exact ties) is real and positive.
 *   - Return value 0 = success, -i = the i-th argument is invalid (nothing was launched), or one of
 *     the positive GEV_ERR_* codes below.  After an error the outputs are unspecified, but the handle
 *     stays usable; GEV_ERR_CUDA means the CUDA context itself reported an error.
 */
#ifndef GEV_H
#define GEV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gev_sys gev_sys; /* opaque, one per system (k-point / spin channel) */

typedef enum { GEV_F64 = 0, GEV_C128 = 1 } gev_dtype;
typedef enum { GEV_PLAIN = 0, GEV_MIXED = 1 } gev_precision;

enum {
  GEV_OK = 0,
  GEV_ERR_NOT_SPD = 1,               /* S not positive definite; report.info = pivot index + 1 */
  GEV_ERR_NO_CONVERGENCE = 2,        /* an iteration cap was hit (secular roots, refinement) */
  GEV_ERR_TIMEOUT = 3,               /* a bounded device wait gave up; the kernel returned */
  GEV_ERR_OOM = 4,                   /* workspace allocation failed or exceeds workspace_limit */
  GEV_ERR_CUDA = 5,                  /* a CUDA runtime call failed */
  GEV_ERR_REUSE_WITHOUT_FACTOR = 6,  /* S == NULL but no resident factor is held */
  GEV_ERR_UNSUPPORTED = 7,           /* option combination not available */
  GEV_ERR_RANK = 9                   /* gev_solve_reduced: fewer than k eigenvalues of S reach delta */
};

/* Steps timed in gev_report.ms (milliseconds, CUDA events on the solve stream). */
enum {
  GEV_STEP_CHOLESKY = 0,
  GEV_STEP_INVERT = 1,
  GEV_STEP_MULTIPLY = 2,
  GEV_STEP_TO_BAND = 3,
  GEV_STEP_TO_TRIDIAG = 4,
  GEV_STEP_SOLVE = 5,
  GEV_STEP_BACK_TRIDIAG = 6,
  GEV_STEP_BACK_BAND = 7,
  GEV_STEP_MULT = 8,
  GEV_STEP_REFINE = 9,
  GEV_NSTEPS = 10
};

typedef struct {
  int device;            /* CUDA device ordinal */
  void* cuda_stream;     /* cudaStream_t on that device (NULL = legacy default stream) */
  int prec;              /* gev_precision */
  int band_b;            /* band width of the full->band step (0 = automatic; rounded up to 16, 32 or 64) */
  int panel_nb;          /* block size of Cholesky / inversion (0 = automatic) */
  double refine_tol;     /* mixed form: target residual (0 = 1e-11) */
  int refine_max_iter;   /* mixed form: refinement iteration cap (0 = 4) */
  size_t workspace_limit;/* bytes; 0 = no limit */
  int timing;            /* 1: record per-step times into gev_report.ms; 2: also time every GEMM
                            launch (CUDA events) and sum its algorithmic flops (gemm_ms/gemm_flops) */
  int fp64_emulation;    /* FP64 matrix products: 1 = formed from exact BF16 digit planes on the tensor
                            cores (error below about K 2^-52 times the largest magnitudes of the row of
                            A and the column of B that meet in an entry; complex data
                            through the real 2x2 embedding), 0 = native FP64 DMMA, -1 = automatic (1) */
  int refine_rr_only;    /* mixed form: 1 = a Rayleigh-Ritz solve in every refinement iteration;
                            0 = Ogita-Aishima steps once the basis is close (default) */
  int fp32_products;     /* mixed form, FP32 matrix products: 6 = BF16x6 split products on the tensor
                            cores (FP32-level accuracy), 3 = BF16x3 (about 16 bits), 0 = FP32 CUDA
                            cores, -1 = automatic (6) */
  int wait_limit;        /* iteration limit of the bounded waits of the cooperative kernels (the grid
                            barriers of the full->band panel factorisation, the progress flags of the
                            bulge chasing; one iteration sleeps ~0.1 us); 0 = default (about 2 s).
                            A wait that reaches it gives up: the call returns GEV_ERR_TIMEOUT and the
                            handle stays usable */
  int check;             /* 1: gev_solve also measures its result on the device, gev_report.resid and
                            .ortho (two more products of H and S with C: about 4 n^2 k + 2 n k^2 flops);
                            0 = off (both report -1) */
  int debug_stall;       /* failure-path tests only: 1 = the bulge chasing waits on a flag that nothing
                            sets, so its bounded wait expires (GEV_ERR_TIMEOUT); 0 = off */
  int rr_band_b;         /* mixed form: band width of the FP64 Rayleigh-Ritz solve of the refinement
                            (16, 32 or 64; 0 = automatic: 64) */
  int one_stage;         /* tridiagonalisation route.  1: one-stage Householder reduction (the ELPA1 form
                            of the section "Usability and Tutorials", reported there as the faster GPU
                            choice when all or most eigenpairs are wanted) with a single
                            back-transform, in FP64 (plain form) or FP32 (real mixed form; the complex
                            mixed form returns GEV_ERR_UNSUPPORTED); panel width = the band width.
                            2: two-stage (full -> band, bulge chasing, two back-transforms).
                            0 = automatic (default): plain form one-stage for 2048 <= n <= 8192, or for
                            n >= 2048 with k >= n/2 (where it measured faster on GB300: its
                            matrix-vector products are bound by the FP64 pipe, the two-stage route's
                            products run on the tensor cores), else two-stage; mixed forms two-stage */
  int rr_one_stage;      /* mixed form, the FP64 Rayleigh-Ritz solve of the refinement (all k pairs of
                            a k x k pencil): 1 = one-stage, 2 = two-stage, 0 = automatic (one-stage for
                            k >= 2048) */
} gev_opts;

typedef struct {
  int info;                 /* NOT_SPD: pivot index + 1; otherwise 0 */
  int deflated;             /* eigenpairs deflated in the top divide-and-conquer merge */
  int refine_iters;         /* mixed form: refinement iterations performed */
  int reused_factor;        /* 1 when the resident L^{-1} was used */
  double refine_resid;      /* mixed form: last refinement residual ||A Y - Y L||_1/(||A||_1) */
  double ms[GEV_NSTEPS];    /* per-step times when opts.timing != 0 */
  size_t workspace_bytes;   /* device bytes held by the handle */
  long long launches;       /* kernels launched by the last call */
  int gemm_calls;           /* timing == 2: GEMM launches timed */
  double gemm_ms;           /* timing == 2: summed GEMM durations (ms, CUDA events) */
  double gemm_flops;        /* timing == 2: summed algorithmic GEMM flops (triangles excluded) */
  int refine_oa_steps;      /* mixed form: iterations that took an Ogita-Aishima step in span(Y)
                               instead of the Rayleigh-Ritz solve */
  double resid;             /* opts.check: ||H C - S C Lambda||_1 / (||H||_1 ||C||_1), computed on the
                               device from the caller's H and S (the accuracy measure of Eq. 2's
                               solution); -1 when not computed (opts.check == 0, or S == NULL) */
  double ortho;             /* opts.check: ||C^H S C - I||_1; -1 when not computed */
} gev_report;

/* Fill *opts with the defaults (device 0, default stream, GEV_PLAIN, automatic sizes). */
void gev_default_opts(gev_opts* opts);

/* Create a handle for problems of order n (1 <= n) and the given dtype; allocates the device
   workspace on opts->device.  *out receives the handle (NULL on failure).  opts may be NULL
   (defaults).  Returns GEV_ERR_OOM when the workspace does not fit (or exceeds workspace_limit).
   The handle plays the part of the elsi_handle of the section "Current Status of the
   Implementation" (ELSI): one per k-point / spin channel, carrying the solver settings, the
   workspace and the factor of S that later SCF iterations reuse. */
int gev_setup(gev_sys** out, int n, int dtype, const gev_opts* opts);

/* Solve H C = S C Lambda for the k lowest eigenpairs, 1 <= k <= n.
   H, S   : device, lower triangles read (ldh, lds >= n).  S may be NULL after gev_reuse_factor(s,1)
            and one successful solve: the resident L^{-1} of the last S is then reused.
   evals  : device, k doubles, ascending.
   C      : device, n x k, ldc >= n.
   rep    : optional host struct.
   Synchronises the handle's stream before returning. */
int gev_solve(gev_sys* s, const void* H, int ldh, const void* S, int lds, int k, double* evals,
              void* C, int ldc, gev_report* rep);

/* Generalized solve for an ill-conditioned overlap (section "Current Status of the Implementation":
   when S is numerically singular, the pencil is transformed to the basis of the eigenvectors D_i of S,
   omitting every D_i whose eigenvalue sigma_i is smaller than a small positive delta, typically
   delta <= 1e-5, as ELSI does).  On the device: S = D diag(sigma) D^H (all n pairs, by the same
   two-stage chain as gev_solve), X = D_kept diag(sigma_kept)^{-1/2} (n x m, m = the number of
   sigma_i >= delta), H~ = X^H H X (m x m), H~ Y = Y Lambda for the k lowest pairs, C = X Y.  C^H S C = I
   on the kept space; C has no component along the omitted D_i.
   H, S   : device, lower triangles read (ldh, lds >= n).  S may be NULL after gev_reuse_factor(s, 1)
            and a successful reduced solve: the resident X of the last S is reused (not the factor
            of gev_solve, and vice versa).
   delta  : threshold on the eigenvalues of S, >= 0 and finite (delta = 0 also keeps zero
            eigenvalues: use a positive delta for a singular S).
   k      : 1 <= k <= n; evals (device, k doubles) ascending; C (device, n x k, ldc >= n).
   m_kept : optional host int receiving m.  rep: optional host report (per-step times: the
            eigendecomposition of S under "cholesky", H~ under "multiply", the reduced solve under
            "to_band", C = X Y under "mult").
   Runs the plain FP64 path whatever opts.prec says (the reduced problem is solved once per S in
   FP64).  Returns 0, -i for an invalid i-th argument, GEV_ERR_RANK when m < k (nothing written to
   evals / C), GEV_ERR_REUSE_WITHOUT_FACTOR, GEV_ERR_NO_CONVERGENCE, GEV_ERR_TIMEOUT, GEV_ERR_OOM (the
   order-m handle of the reduced problem could not be allocated) or GEV_ERR_CUDA.  Synchronises the
   handle's stream before returning. */
int gev_solve_reduced(gev_sys* s, const void* H, int ldh, const void* S, int lds, double delta, int k,
                      double* evals, void* C, int ldc, int* m_kept, gev_report* rep);

/* Density matrix of k orbitals (section "Circumventing the eigenvalue problem") and, optionally,
   its energy-weighted counterpart (section "ELSI"):
       P_ij  = sum_l f_l conj(C_il) C_jl,      PE_ij = sum_l f_l lambda_l conj(C_il) C_jl,
   C_il being the coefficient of basis function i in orbital l (column l of C, as gev_solve returns).
   k      : 1 <= k <= n columns of C are used.
   C      : device, n x k, ldc >= n.
   occ    : device, k doubles f_l (occupation numbers; any real values).
   evals  : device, k doubles lambda_l; read only when PE != NULL (may be NULL otherwise).
   P      : device, n x n, ldp >= n; receives the full Hermitian P (both triangles, real diagonal).
   PE     : device n x n with ldpe >= n, or NULL; must not be P.
   C, occ and evals are not modified and must not overlap P or PE.  The products run on the FP64
   matrix-product engine of the handle (opts.fp64_emulation), also on a GEV_MIXED handle.  Uses the
   handle's scratch workspace only: the resident factor and the data kept by the step entry points
   stay valid.  Returns 0, -i for an invalid i-th argument, GEV_ERR_TIMEOUT or GEV_ERR_CUDA.
   Synchronises the handle's stream before returning. */
int gev_density(gev_sys* s, int k, const void* C, int ldc, const double* occ, const double* evals, void* P,
                int ldp, void* PE, int ldpe);

/* Accuracy of k eigenpairs (evals, C) of the pencil (H, S), measured on the device with the handle's
   FP64 product engine: *resid = ||H C - S C Lambda||_1 / (||H||_1 ||C||_1) and
   *ortho = ||C^H S C - I||_1, the two measures of a solution of Eq. 2 (H C = S C Lambda with
   S-orthonormal C).  H, S: device, lower triangles read (ldh, lds >= n); evals: device, k doubles;
   C: device, n x k (ldc >= n); resid, ortho: host.  1 <= k <= n.  Overwrites the handle's scratch
   workspace (the resident factor stays valid; the reflectors kept by gev_step_he2hb / hb2st do not).
   Returns 0, -i for an invalid i-th argument, or GEV_ERR_CUDA.  Synchronises the handle's stream. */
int gev_check(gev_sys* s, const void* H, int ldh, const void* S, int lds, int k, const double* evals,
              const void* C, int ldc, double* resid, double* ortho);

/* enable != 0: keep L^{-1} resident after each solve so the next gev_solve may pass S = NULL
   (SCF iterations with fixed overlap).  enable == 0 drops the resident factor.  Steps 1-2 of the
   reduction (section "Current Status of the Implementation") depend on S only; the ELSI interface
   of the same section reuses them across the SCF cycle of one k-point, which this call enables.
   Returns 0, or -1 for a NULL handle. */
int gev_reuse_factor(gev_sys* s, int enable);

/* Release the handle and its workspace (s may be NULL): the end of an elsi_handle's life (section
   "Current Status of the Implementation", ELSI).  Synchronises the handle's stream first.
   Returns 0. */
int gev_free(gev_sys* s);

/* Device bytes the handle would need for (n, dtype, opts); 0 on invalid arguments. */
size_t gev_workspace_bytes(int n, int dtype, const gev_opts* opts);

/* Error text for a return code (static string). */
const char* gev_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GEV_H */
