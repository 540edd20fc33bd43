// gather.cu -- reads many 0-d stores in one launch (dfs_read_scalars).
//
// A serving loop checks the residual norm of every active solve after each
// tick; one kernel gathers those scalars (any dtype, converted to double)
// into a contiguous buffer so that a single device-to-host copy brings them
// all back.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/diffuse.h"

namespace {

// desc[2*i] = device address of scalar i, desc[2*i+1] = its dfs_dtype
__global__ void gather_scalars_kernel(const int64_t* __restrict__ desc, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const void* p = reinterpret_cast<const void*>(desc[2 * i]);
  double v = 0.0;
  switch ((int)desc[2 * i + 1]) {
    case DFS_F32: v = (double)*static_cast<const float*>(p); break;
    case DFS_F64: v = *static_cast<const double*>(p); break;
    case DFS_I32: v = (double)*static_cast<const int32_t*>(p); break;
    case DFS_I64: v = (double)*static_cast<const int64_t*>(p); break;
    default: break;
  }
  out[i] = v;
}

}  // namespace

namespace dfs {

// desc_dev and out_dev: device buffers of 2n int64 and n doubles
cudaError_t launch_gather_scalars(const int64_t* desc_dev, int n, double* out_dev, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int block = 128;
  gather_scalars_kernel<<<(n + block - 1) / block, block, 0, s>>>(desc_dev, n, out_dev);
  return cudaGetLastError();
}

}  // namespace dfs
