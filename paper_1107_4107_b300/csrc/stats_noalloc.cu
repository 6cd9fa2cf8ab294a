// Ensemble statistics without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs after another framework's
// caching allocator has reserved nearly all of the GPU's memory, code that must
// not trigger the device-wide synchronisation cudaMalloc/cudaFree may cause,
// or a service whose device-memory budget is fixed when it starts.  For them,
// arnold_stats_arrays_noalloc() runs the same two-pass statistics reduction as
// arnold_stats_arrays() but keeps its block partials in the fixed array below,
// which is part of the library image: every GPU that loads libarnold.so holds
// it (about 1.7 MB) until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Nothing in it has to start at zero: each call's first kernel
// overwrites every partial slot that its second kernel reads, and the second
// kernel overwrites the result slot.  Calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on the array.
#include <math.h>
#include <string.h>

#include <mutex>

#include "kernels.cuh"

namespace arnold {

namespace {

constexpr int kNoAllocMaxBlocks = 1024;   // block partials; slot kNoAllocMaxBlocks holds the merged result
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) StatsPartial g_noalloc_scratch[kNoAllocMaxBlocks + 1];

// Host-side device address of g_noalloc_scratch per device.  The symbol's name
// in host code is only a host stand-in; the address must come from
// cudaGetSymbolAddress with the device current.
std::mutex g_noalloc_mu;
StatsPartial* g_noalloc_ptr[kNoAllocMaxDevices] = {};

cudaError_t noalloc_scratch(int device, StatsPartial** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<StatsPartial*>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

int to_status(cudaError_t e) {
  if (e == cudaSuccess) return ARNOLD_OK;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ARNOLD_EUNSUPPORTED;
  return ARNOLD_ECUDA;
}

// Makes `device` current for the call and gives the caller back its own
// current device on every return path.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope() { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; }
  ~DeviceScope() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

}  // namespace arnold

extern "C" int arnold_stats_arrays_noalloc(int device, void* cuda_stream, int64_t n, const double* chi,
                                           const double* dE, const double* p, double t, double kappa,
                                           arnold_stats* out) {
  using namespace arnold;
  if (!out || !chi || !p || n <= 0 || !(kappa > 0.0) || t == 0.0) return ARNOLD_EINVAL;
  if (n > ARNOLD_NOALLOC_MAX_N) return ARNOLD_EINVAL;
  if (device < 0 || device >= kNoAllocMaxDevices) return ARNOLD_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return ARNOLD_EUNSUPPORTED;
  if (device >= ndev) return ARNOLD_EINVAL;
  DeviceScope keep;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return to_status(e);
  StatsPartial* scratch = nullptr;
  e = noalloc_scratch(device, &scratch);
  if (e != cudaSuccess) return to_status(e);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long g = (n + 255) / 256;
  const int grid = (int)(g < kNoAllocMaxBlocks ? g : kNoAllocMaxBlocks);
  const double tt = fabs(t);
  const double thr = kappa * log(tt > M_E ? tt : M_E) / tt;
  e = launch_stats(n, chi, dE, p, thr, scratch, grid, scratch + kNoAllocMaxBlocks, st);
  if (e != cudaSuccess) return to_status(e);
  StatsPartial h;
  e = cudaMemcpyAsync(&h, scratch + kNoAllocMaxBlocks, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return to_status(e);
  memcpy(out->hist, h.hist, sizeof out->hist);
  out->under = h.under;
  out->over = h.over;
  out->chaotic = h.chaotic;
  out->n = h.n;
  out->dE_max = h.dE_max;
  for (int k = 0; k < 3; ++k) {
    out->p_mean[k] = h.mean[k];
    out->p_var[k] = h.n ? h.m2[k] / (double)h.n : 0.0;
  }
  out->t = t;
  return ARNOLD_OK;
}
