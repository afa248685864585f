// gev_potrf_noalloc: the blocked Cholesky factorisation (the same kernels as gev_step_potrf) for
// callers that cannot allocate device memory.  Its scratch lives in one file-scope __device__ array
// instead of a handle's cudaMalloc'ed workspace.
#include <mutex>

#include "common.cuh"
#include "gev_noalloc.h"

namespace {

// inverted diagonal block (nb x nb) + panel (n_max x nb) + status words, real FP64
constexpr int kNb = 64;
constexpr size_t kDinvBytes = sizeof(double) * kNb * kNb;
constexpr size_t kPanelBytes = sizeof(double) * (size_t)GEV_NOALLOC_MAX_N * kNb;
constexpr size_t kStatusBytes = 256;
static_assert(kDinvBytes + kPanelBytes + kStatusBytes <= GEV_NOALLOC_SCRATCH_BYTES, "scratch size");

// Every device that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GEV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device; the name
// g_noalloc_scratch in host code is only a host-side stand-in and must never reach a kernel).
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return GEV_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "gev: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return GEV_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return 0;
}

}  // namespace

extern "C" int gev_potrf_noalloc(int n, double* A, int lda, void* cuda_stream, int* info) {
  if (info) *info = 0;
  if (n < 1) return -1;
  if (n > GEV_NOALLOC_MAX_N) {
    fprintf(stderr, "gev_potrf_noalloc: n = %d exceeds the fixed scratch limit %d\n", n,
            GEV_NOALLOC_MAX_N);
    return GEV_ERR_TOO_LARGE;
  }
  if (!A) return -2;
  if (lda < n) return -3;
  int dev = 0;
  GEV_CUDA_TRY(cudaGetDevice(&dev));
  void* base = nullptr;
  GEV_TRY(scratch_address(dev, &base));
  // A view of the fixed scratch, no workspace of its own.  A default Sys has emu_fp64 = 0, so every
  // product of the path runs on the native FP64 tensor path (DMMA): the emulated FP64 products need
  // digit-plane scratch (ozws) of the size of the operands, which only a handle allocates.  With
  // splitws empty no product splits K (the panel products have K = nb anyway).
  gev::Sys s;
  s.n = n;
  s.dtype = GEV_F64;
  s.nb = kNb;
  s.stream = (cudaStream_t)cuda_stream;
  int sms = 0;
  GEV_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  s.sms = sms > 0 ? sms : 152;
  char* p = (char*)base;
  s.dinv = p;
  s.Pn = p + kDinvBytes;
  s.status = (int*)(p + kDinvBytes + kPanelBytes);
  s.splitws = nullptr;  // no split-K partials: every GEMM runs unsplit
  s.splitws_bytes = 0;
  GEV_CUDA_TRY(cudaMemsetAsync(s.status, 0, sizeof(int) * gev::ST_COUNT, s.stream));
  int r = gev::potrf<double>(s, A, lda);
  if (r) return r;
  int piv = 0;
  GEV_CUDA_TRY(cudaMemcpyAsync(&piv, &s.status[gev::ST_NOT_SPD], sizeof(int), cudaMemcpyDeviceToHost,
                               s.stream));
  GEV_CUDA_TRY(cudaStreamSynchronize(s.stream));
  if (info) *info = piv;
  return piv ? GEV_ERR_NOT_SPD : 0;
}
