/*
 * gev_kernels.h -- the matrix products of the mixed-precision form, as C entry points.
 *
 * The mixed form runs its reduction and back-transforms in FP32 (the single/double-precision pattern
 * named in the section "Future Plans and Challenges").  Its products are formed on the tensor cores
 * from BF16 splits: a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi), and
 * a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation (about 16 correct bits per
 * product); the result is then refined in FP64 by the solver.
 */
#ifndef GEV_KERNELS_H
#define GEV_KERNELS_H

#include "gev.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha op(A) op(B) + beta C, FP32, column-major device pointers on the current device.
     ta, tb     : 0 = as stored, 1 = transposed
     engine     : 1 = BF16x3 tensor-core products (tcgen05), 0 = FP32 CUDA-core FMAs
     stream     : cudaStream_t (NULL = legacy default), synchronised before return
     status_dev : device pointer to 16 ints the kernel may write (a bounded wait that expired writes
                  a non-zero code to status_dev[1]); the caller zeroes and reads it
   Returns 0, -i for an invalid i-th argument, or GEV_ERR_CUDA.  Allocates nothing. */
int gev_gemm_f32(int M, int N, int K, int ta, int tb, float alpha, const float* A, int lda,
                 const float* B, int ldb, float beta, float* C, int ldc, int engine, void* stream,
                 int* status_dev);

/* C = alpha op(A) op(B) + beta C in FP64 (real), column-major device pointers, current device.
     engine        : 0 = native FP64 tensor path (DMMA), 1 = emulated on the BF16 tensor cores: every
                     row of op(A) / column of op(B) is scaled by a power of two, split into 8 exact
                     balanced 7-bit digit planes stored as BF16, and the digit products with
                     p + q <= 9 are summed on the tensor cores (exactly, per 512-deep chunk of K, for
                     p + q <= 7), so the error stays below about 2^-50 (|A| |B|)_ij
     status_dev    : device pointer to 16 ints (a bounded wait that expired writes status_dev[1])
     scratch_dev   : engine 1: device scratch of scratch_bytes >= gev_gemm_f64_scratch_bytes(M, N, K)
                     (digit planes: about 16 (M + N) min(K, 32768) bytes, plus split-K partials)
   Returns 0, -i for an invalid i-th argument, or GEV_ERR_CUDA.  Allocates nothing.  An Inf or NaN
   entry of op(A) / op(B) makes every output of its row / column NaN (engine 1). */
int gev_gemm_f64(int M, int N, int K, int ta, int tb, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc, int engine, void* stream,
                 int* status_dev, void* scratch_dev, size_t scratch_bytes);

/* Bytes of scratch gev_gemm_f64 needs for engine 1 (0 for negative sizes). */
size_t gev_gemm_f64_scratch_bytes(int M, int N, int K);

#ifdef __cplusplus
}
#endif
#endif /* GEV_KERNELS_H */
