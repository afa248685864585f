/*
 * gev_steps.h -- the individual transformation steps of the solver as separate C entry points.
 *
 * The section "Current Status of the Implementation" notes that besides the complete generalized
 * solve, an interface for each individual transformation step is provided (so a caller can run,
 * e.g., only the reduction to the standard problem).  These calls expose the same kernels that
 * gev_solve chains, on the handle's device, stream and workspace.
 *
 * Conventions are those of gev.h: column-major device pointers, complex interleaved, n = the
 * handle's order, lower triangles of Hermitian inputs read.  Each call synchronises the handle's
 * stream and returns 0, -i for an invalid i-th argument, or a GEV_ERR_* code.  None of them
 * allocates device memory; all scratch comes from the handle's workspace.
 */
#ifndef GEV_STEPS_H
#define GEV_STEPS_H

#include "gev.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Step 1 (Cholesky, reduction step 1): A <- L with A = L L^H, lower triangle of A read and
   overwritten, strict upper triangle set to zero.  *info (host) = 0, or pivot index + 1 when the
   matrix is not positive definite (then GEV_ERR_NOT_SPD is returned). */
int gev_step_potrf(gev_sys* s, void* A, int lda, int* info);

/* Step 2 (Invert, reduction step 2): A <- L^{-1} for a lower-triangular A with a positive real
   diagonal; strict upper triangle set to zero. */
int gev_step_trtri(gev_sys* s, void* A, int lda);

/* Step 3 (Multiply, reduction step 3): A = X H X^H, X lower triangular (the inverted factor),
   H Hermitian (lower triangle read).  A receives the full Hermitian result (both triangles). */
int gev_step_hegst(gev_sys* s, const void* H, int ldh, const void* X, int ldx, void* A, int lda);

/* Step 4a (full -> band, two-stage tridiagonalisation stage 1): A (full Hermitian, both
   triangles, overwritten) = Q1 B Q1^H with B of lower band width b (16, 32 or 64; 0 =
   handle default).  The compact-WY blocks of Q1 and the band B stay in the handle for steps 4b
   and 6.  *b_used (host, optional) receives b. */
int gev_step_he2hb(gev_sys* s, void* A, int lda, int b, int* b_used);

/* Step 4b (band -> tridiagonal, stage 2): bulge chasing on the band held by the handle after
   gev_step_he2hb.  d (n) and e (n-1) are device doubles receiving the real tridiagonal T.  The
   reflectors of Q2 (and, for complex data, the diagonal phase matrix) stay in the handle. */
int gev_step_hb2st(gev_sys* s, double* d, double* e);

/* Step 4 in one stage (the ELPA1 form, section "Usability and Tutorials"): A (Hermitian, lower
   triangle read, overwritten) = Q T Q^H with T real symmetric tridiagonal, Q = H_0 ... H_{n-2}
   Householder reflectors kept in the handle for gev_step_back.  d (n) and e (n-1) are device
   doubles receiving T.  Panel width = the handle's band width. */
int gev_step_he2td(gev_sys* s, void* A, int lda, double* d, double* e);

/* Step 5 (Solve): divide and conquer on the real symmetric tridiagonal (d, e) (device, n and
   n-1 doubles, not modified).  w (device, n) receives all eigenvalues ascending; Z (device, real
   n x k, ldz >= n) the eigenvectors of the k lowest.  *deflated (host, optional) = number of
   eigenpairs deflated in the top merge. */
int gev_step_stedc(gev_sys* s, const double* d, const double* e, int k, double* w, double* Z,
                   int ldz, int* deflated);

/* Step 6 (Back): Y = Q1 Q2 Z for real Z (n x k, device) using the reflectors kept by steps 4a and
   4b on this handle (or Y = Q Z after the one-stage step 4, whichever ran last); Y has the handle's
   dtype. */
int gev_step_back(gev_sys* s, const double* Z, int ldz, int k, void* Y, int ldy);

/* Step 7 (Mult.): C = X^H Y, X lower triangular (n x n), Y n x k. */
int gev_step_mult(gev_sys* s, const void* X, int ldx, const void* Y, int ldy, int k, void* C,
                  int ldc);

#ifdef __cplusplus
}
#endif
#endif /* GEV_STEPS_H */
