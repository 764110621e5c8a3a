// mgw_response_moments_tda_noalloc: the TDA response moments with all
// scratch in a fixed, statically allocated device array, for callers that
// cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is unavailable or
// forbidden -- inside a host callback or a region that must not
// synchronise, in a process whose device memory is owned by another
// allocator (a framework's pool it may not bypass), or in embedded callers
// that size all memory up front.  They pass the inputs and the output and
// get the same result as mgw_response_moments with screening = TDA.
//
// The scratch lives in `g_tda_scratch`, a file-scope __device__ array, so
// every GPU that loads the library holds it until the process exits.  Host
// code must not use the array's name as a pointer (on the host it is a
// stand-in symbol, not a device address); the device address is fetched once
// per device with cudaGetSymbolAddress, with that device current, the first
// time the entry point runs on that device.  That first call should
// therefore come before any stream capture.
#include "mgw_internal.h"

#include <atomic>

namespace mgw {

// 4 Mi doubles = 32 MiB: D[ov] followed by T[naux][ov]
constexpr long kNoallocScratchDoubles = 4L * 1024 * 1024;
static __device__ __align__(256) double g_tda_scratch[kNoallocScratchDoubles];

// device address of the array per device, published once looked up; two host
// threads making their first call on one device at the same time both look it
// up and store the same address
constexpr int kMaxDevices = 64;
static std::atomic<double*> g_scratch_ptr[kMaxDevices];

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_response_moments_tda_noalloc(void* cuda_stream, int nocc, int nvir, int naux, int nmom,
                                                       const double* eps_W, const double* Lov, double* Wmom) {
  if (nocc < 1 || nvir < 1 || naux < 1 || nmom < 1 || nmom > 64 || !eps_W || !Lov || !Wmom) return MGW_ERR_ARG;
  const long ov = (long)nocc * nvir;
  // D and T must fit the static scratch
  if (ov + (long)naux * ov > kNoallocScratchDoubles) return MGW_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MGW_ERR_CUDA;
  double* D = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!D) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tda_scratch) != cudaSuccess || !p) return MGW_ERR_CUDA;
    D = static_cast<double*>(p);
    g_scratch_ptr[dev].store(D, std::memory_order_release);
  }
  double* T = D + ((ov + 31) / 32) * 32;  // keep T 256-byte aligned
  if ((T - D) + (long)naux * ov > kNoallocScratchDoubles) return MGW_ERR_UNSUPPORTED;

  // a handle on the stack: stream only, no solver, no workspace; its error
  // text goes with it, so callers get the status code alone
  mgw_handle hs;
  mgw_handle* h = &hs;
  h->device = dev;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  const long na2 = (long)naux * naux;
  MGW_TRY(energy_differences(h, nocc, nvir, eps_W, D));
  MGW_CUDA(h, cudaMemcpyAsync(T, Lov, sizeof(double) * naux * ov, cudaMemcpyDeviceToDevice, h->stream));
  for (int n = 0; n < nmom; ++n) {
    double* Wn = Wmom + (long)n * na2;
    MGW_TRY((dgemm<64, 64>(h, naux, naux, ov, 1, ARowMajor{T, ov, 0}, BNMajor{Lov, ov, 0},
                           EpiStore{Wn, naux, 0, 1.0, 0.0}, "w_gemm", /*tri=*/1)));
    if (n + 1 < nmom)
      MGW_TRY((dgemm<64, 64>(h, naux, ov, naux, 1, ARowMajor{Wn, naux, 0}, BRowMajor{Lov, ov, 0},
                             EpiDiagUpdate{T, ov, D, 2.0}, "t_update")));
  }
  return MGW_OK;
}
