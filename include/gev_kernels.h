/*
 * gev_kernels.h -- the matrix products of the mixed-precision form, as C entry points.
 *
 * The mixed form runs its reduction and back-transforms in FP32 (the single/double-precision pattern
 * named in the section "Future Plans and Challenges").  Its large FP32 products are formed on the
 * tensor cores from BF16 splits (gev_gemm_f32, engines 1 and 2); its FP64 products from exact BF16
 * digit planes (gev_gemm_f64, engine 1).  The result is refined in FP64 by the solver.
 */
#ifndef GEV_KERNELS_H
#define GEV_KERNELS_H

#include "gev.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha op(A) op(B) + beta C, FP32, column-major device pointers on the current device.
     ta, tb        : 0 = as stored, 1 = transposed
     engine        : 0 = FP32 CUDA-core FMAs; on the tensor cores (tcgen05), from the BF16 split
                     x = x1 + x2 + x3 (exact for FP32 x): 1 = BF16x6, the 6 split products with
                     p + q <= 4 (FP32-level accuracy), 2 = BF16x3, the products x1y1 + x1y2 + x2y1
                     (about 16 significant bits); FP32 accumulation in tensor memory
     stream        : cudaStream_t (NULL = legacy default), synchronised before return
     status_dev    : device pointer to 16 ints the kernel may write (a bounded wait that expired writes
                     a non-zero code to status_dev[1]); the caller zeroes and reads it
     scratch_dev   : engines 1, 2: device scratch of scratch_bytes >= gev_gemm_f32_scratch_bytes(M, N, K)
                     (split planes, about 6 (M + N) K bytes, plus split-K partials); ignored by engine 0
   Returns 0, -i for an invalid i-th argument, or GEV_ERR_CUDA.  Allocates nothing. */
int gev_gemm_f32(int M, int N, int K, int ta, int tb, float alpha, const float* A, int lda,
                 const float* B, int ldb, float beta, float* C, int ldc, int engine, void* stream,
                 int* status_dev, void* scratch_dev, size_t scratch_bytes);

/* Bytes of scratch gev_gemm_f32 needs for engines 1 and 2 (0 for negative sizes). */
size_t gev_gemm_f32_scratch_bytes(int M, int N, int K);

/* C = alpha op(A) op(B) + beta C in FP64 (real), column-major device pointers, current device.
     engine        : 0 = native FP64 tensor path (DMMA), 1 = emulated on the BF16 tensor cores: every
                     row of op(A) / column of op(B) is scaled by a power of two, split into 8 exact
                     balanced 7-bit digit planes stored as BF16, and the digit products with
                     p + q <= 9 are summed on the tensor cores (exactly, per 512-deep chunk of K, for
                     p + q <= 7).  The error is bounded relative to the row and column scales:
                     |err_ij| <= K s_i t_j (2^-52.6 + 2^-53 + K 2^-62.2), s_i (t_j) the power of two
                     just above the largest magnitude of row i of op(A) (column j of op(B)).  For
                     entries of similar magnitude this is the order of a native FP64 product's
                     K 2^-53 (|A| |B|)_ij; entries far below their row's or column's largest keep
                     fewer bits.
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
