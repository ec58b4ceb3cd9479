// bin_static.cu -- mpm_bin_static: the per-cell binning of mpm_bin with its sort scratch in a
// fixed file-scope device array instead of memory allocated per call.
//
// The scratch holds two key and two value buffers of the LSD radix sort plus its per-CTA
// digit histogram, for at most kBinStaticMax particles (4 MiB + 64 KiB).  Its device address
// is taken with cudaGetSymbolAddress once per device, on the first call made with that device
// current, and kept for the process; that first call should come before any stream capture.
// A cudaDeviceReset unloads the module and leaves the kept address stale, so the entry point
// is not for a device that has been reset.  Every call shares the one
// array and finds the previous call's contents in it: nothing there is read before this call
// writes it (each sort pass overwrites every histogram entry it later reads, and only the
// first n keys and values are touched), so no part of it needs clearing.  Calls whose work
// overlaps on the GPU (different streams, or different host threads on one stream without
// ordering) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "mpm.h"

namespace {

constexpr int kBinStaticMax = 1 << 18;     // particles per call
constexpr int kSortTileKeys = 4096;        // keys per sort CTA (radix_sort's tile)
constexpr int kScanTileCounters = 4096;    // counters per scan CTA (radix_sort's scan)
constexpr int kDigitCounters = 256 * ((kBinStaticMax + kSortTileKeys - 1) / kSortTileKeys);
constexpr int kHistEntries = kDigitCounters + (kDigitCounters + kScanTileCounters - 1) / kScanTileCounters;
constexpr size_t kScratchWords = 4 * (size_t)kBinStaticMax + kHistEntries;

static __device__ __align__(256) unsigned g_bin_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned* g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's copy of the scratch (set up on first use).
cudaError_t scratch_for_current_device(unsigned** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

int32_t mpm_bin_static_max(void) { return kBinStaticMax; }

mpm_status mpm_bin_static(const float* x, int32_t n, int32_t grid_res, uint32_t* keys, uint32_t* perm,
                          void* stream) {
  if (!x || !keys || !perm || n < 0 || grid_res < 8 || grid_res > 128 || grid_res % 4) return MPM_ERR_INVALID_ARG;
  if (n > kBinStaticMax) return MPM_ERR_INVALID_ARG;  // beyond the fixed scratch
  if (n == 0) return MPM_OK;
  if (mpm::radix_hist_entries(n) > kHistEntries) return MPM_ERR_INVALID_ARG;  // scratch layout check
  // An error already pending on this thread belongs to an earlier call of the caller's: leave
  // it in place and launch nothing, so that every error reported below is this call's own.
  if (cudaPeekAtLastError() != cudaSuccess) return MPM_ERR_CUDA;
  unsigned* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return MPM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* k1 = base;
  unsigned* k2 = base + kBinStaticMax;
  unsigned* v1 = base + 2 * (size_t)kBinStaticMax;
  unsigned* v2 = base + 3 * (size_t)kBinStaticMax;
  unsigned* hist = base + 4 * (size_t)kBinStaticMax;
  mpm::launch_bin_keys_plain(x, n, grid_res, k1, v1, st);
  if (cudaPeekAtLastError() != cudaSuccess) return (void)cudaGetLastError(), MPM_ERR_CUDA;
  if (cudaMemcpyAsync(keys, k1, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return MPM_ERR_CUDA;
  int bits = 0;
  for (unsigned long long v = (unsigned long long)(grid_res / 4) * (grid_res / 4) * (grid_res / 4) * 64ull - 1ull; v;
       v >>= 1)
    ++bits;
  unsigned* kk[2] = {k1, k2};
  unsigned* vv[2] = {v1, v2};
  const int cur = mpm::radix_sort(kk, vv, n, bits, hist, st);
  if (cudaPeekAtLastError() != cudaSuccess) return (void)cudaGetLastError(), MPM_ERR_CUDA;
  if (cudaMemcpyAsync(perm, vv[cur], sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return MPM_ERR_CUDA;
  return MPM_OK;
}

}  // extern "C"
