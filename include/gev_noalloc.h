/*
 * gev_noalloc.h -- one entry point that allocates no device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers of this library that
 * cannot call cudaMalloc: for example a process whose device memory is owned by another memory
 * manager (a caching allocator or pool with a fixed budget that forbids raw allocations), or a
 * latency-critical loop that cannot afford the implicit device synchronisation of an allocation.
 * Such a caller passes its own input/output buffer; all scratch comes from one fixed array compiled
 * into the library.
 */
#ifndef GEV_NOALLOC_H
#define GEV_NOALLOC_H

#include "gev.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest order accepted, and the size of the fixed scratch array (bytes).  Every GPU on which
   the library is loaded holds GEV_NOALLOC_SCRATCH_BYTES of device memory for it until the
   process exits. */
#define GEV_NOALLOC_MAX_N 4096
#define GEV_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u + 64u * 1024u)

/* Returned when n exceeds GEV_NOALLOC_MAX_N. */
#define GEV_ERR_TOO_LARGE 8

/* Cholesky factorisation S = L L^T of a real symmetric positive definite matrix, in place, with no
   device allocation: the same kernels as gev_step_potrf (gev_steps.h) on the current CUDA device.
     n      : order, 1 <= n <= GEV_NOALLOC_MAX_N (larger n: GEV_ERR_TOO_LARGE, nothing launched)
     A      : device pointer, column-major, lower triangle read, overwritten by L; the strict upper
              triangle is set to zero
     lda    : leading dimension >= n
     stream : cudaStream_t to run on (NULL = legacy default stream); synchronised before return
     info   : optional host pointer; 0, or pivot index + 1 when A is not positive definite (then
              GEV_ERR_NOT_SPD is returned)
   Returns 0, -i for an invalid i-th argument, GEV_ERR_TOO_LARGE, GEV_ERR_NOT_SPD or GEV_ERR_CUDA.
   Set-up: the first call on a device looks up the device address of the scratch array
   (cudaGetSymbolAddress) with that device current, once; make that first call before any stream
   capture begins.  Every call synchronises `stream` and copies one status word to the host before
   it returns.  All calls on a device share its one array and each call clears what must start at
   zero, but nothing else is kept between calls: calls whose work overlaps on the same GPU (issued
   on different streams, or from different host threads) race on the array and must be serialised
   by the caller.  The products of this path run on the native FP64 tensor path (DMMA): the
   emulated FP64 products of a handle need digit-plane workspace that only a handle allocates.
   No cudaMalloc, cudaFree or allocating library routine is called. */
int gev_potrf_noalloc(int n, double* A, int lda, void* stream, int* info);

#ifdef __cplusplus
}
#endif
#endif /* GEV_NOALLOC_H */
