// noalloc.cu -- a dot product that allocates nothing.
//
// Some callers cannot allocate device memory at the time they need a
// reduction:
//   * serving or real-time loops that reserve all their device memory at
//     start-up and must not allocate afterwards, because an allocation can
//     block, synchronise the device, or fail under a memory budget;
//   * plug-ins hosted by a framework that owns every device allocation
//     through its own allocator and gives them none.
// For them this file provides dfs_dot_noalloc: the same per-point reduction
// scheme as the runtime's generated DOT kernels (one partial per 4096-element
// point, a fixed tree inside the block, the last CTA to finish sums the
// partials in point order), with its scratch in a file-scope device array
// instead of memory the runtime allocates.  The caller still passes the
// inputs and the output.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/diffuse.h"
#include "dfs_device.cuh"

namespace {

constexpr long long kTile = DFS_NOALLOC_TILE;
constexpr long long kMaxPoints = DFS_NOALLOC_MAX_N / DFS_NOALLOC_TILE;
constexpr int kBlock = 256;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: one partial per point, then the
// exit counter of the last-CTA protocol.  Every GPU that loads this library
// holds it until the process exits.
static __device__ __align__(256) double g_partials[kMaxPoints];
static __device__ __align__(256) dfs::Ctl g_ctl;

__global__ void __launch_bounds__(kBlock) dot_noalloc_kernel(const double* __restrict__ x,
                                                             const double* __restrict__ y, long long n,
                                                             double* out, double* partials, dfs::Ctl* ctl) {
  __shared__ double buf[kBlock];
  const long long npts = (n + kTile - 1) / kTile;
  for (long long pt = blockIdx.x; pt < npts; pt += gridDim.x) {
    const long long lo = pt * kTile;
    const long long hi = lo + kTile < n ? lo + kTile : n;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kBlock) acc = dfs::red_fma(__ldg(x + i), __ldg(y + i), acc);
    const double tot = dfs::block_sum(acc, buf);
    if (threadIdx.x == 0) partials[pt] = tot;
  }
  if (dfs::last_cta(ctl)) {
    const double s = dfs::sum_partials(partials, npts);
    if (threadIdx.x == 0) *out = s;
    dfs::ctl_reset(ctl);
  }
}

// Device addresses of the scratch on one device.  The plain fields are
// written once, under g_mu, before `ready` is set with release ordering; a
// caller that loads `ready` as true with acquire ordering therefore sees them
// complete, without taking the lock (host threads may call concurrently).
struct DeviceScratch {
  double* partials = nullptr;
  dfs::Ctl* ctl = nullptr;
  int sms = 0;
  std::atomic<bool> ready{false};
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// Host code cannot use g_partials / g_ctl directly: their names denote
// host-side stand-ins, not device addresses.  Resolve the device addresses
// once per device, with that device current.
int setup(int dev, DeviceScratch& s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (s.ready.load(std::memory_order_relaxed)) return DFS_OK;   // set by another thread under g_mu
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return DFS_ERR_CUDA;
  s.partials = static_cast<double*>(p);
  p = nullptr;
  if (cudaGetSymbolAddress(&p, g_ctl) != cudaSuccess || !p) return DFS_ERR_CUDA;
  s.ctl = static_cast<dfs::Ctl*>(p);
  if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DFS_ERR_CUDA;
  s.ready.store(true, std::memory_order_release);
  return DFS_OK;
}

}  // namespace

extern "C" int dfs_dot_noalloc(const double* x, const double* y, int64_t n, double* out, void* stream) {
  if (!out || n < 0 || (n > 0 && (!x || !y))) return DFS_ERR_INVALID;
  if (n > DFS_NOALLOC_MAX_N) return DFS_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DFS_ERR_CUDA;
  DeviceScratch& s = g_dev[dev];
  if (!s.ready.load(std::memory_order_acquire)) {
    const int rc = setup(dev, s);
    if (rc) return rc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the exit counter must start at zero; a launch always leaves it at zero,
  // but clear it in case an earlier launch was aborted
  if (cudaMemsetAsync(s.ctl, 0, sizeof(dfs::Ctl), st) != cudaSuccess) return DFS_ERR_CUDA;
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(double), st) == cudaSuccess ? DFS_OK : DFS_ERR_CUDA;
  const long long npts = (n + kTile - 1) / kTile;
  const long long cap = 4LL * s.sms;
  const int grid = (int)(npts < cap ? npts : cap);
  dot_noalloc_kernel<<<grid, kBlock, 0, st>>>(x, y, (long long)n, out, s.partials, s.ctl);
  return cudaGetLastError() == cudaSuccess ? DFS_OK : DFS_ERR_CUDA;
}
