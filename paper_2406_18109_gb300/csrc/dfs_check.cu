// dfs_check.cu -- ahead-of-time instantiation of every device template for
// sm_103a.  The templates are normally compiled at run time by NVRTC inside
// generated kernels; compiling them here with nvcc at build time catches
// errors before any GPU run.  The kernel is never launched.
#include "dfs_device.cuh"

using namespace dfs;

template <typename T>
__device__ T all_ops(T a, T b) {
  T r = op_add(a, b);
  r = op_sub(r, op_mul(a, b));
  r = op_div(r, op_max(op_min(a, b), T(1)));
  r = op_add(r, op_pow(op_abs(a), b));
  r = op_add(r, op_exp(op_neg(a)));
  r = op_add(r, op_log(op_sqrt(op_abs(b))));
  r = op_add(r, op_erf(a));
  r = op_add(r, op_ncdf(b));
  return op_copy(r);
}

extern "C" __global__ void dfs_template_check(const float* x, const double* y, const int* rowptr, const int* col,
                                              float* out32, double* out64, Ctl* ctl, long long n) {
  __shared__ double buf[1024];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float a = 0.f;
  double b = 0.0;
  if (i + 4 <= n) {
    f32x4 v = ld4ro(x + i);
    a = all_ops(v.v[0], v.v[1]);
    f64x2 w = ld2(y + i);
    b = all_ops(w.v[0], w.v[1]);
    b = op_add(b, spmv_row<double>(rowptr, col, y, y, i));
  }
  a = block_sum(a, (float*)buf);
  b = block_sum(b, buf);
  if (!grid_barrier(ctl, 1u, 1000000ull)) return;
  b = op_add(b, sum_partials(y, n));
  if (threadIdx.x == 0) {
    out32[blockIdx.x] = a;
    out64[blockIdx.x] = b;
  }
  if (last_cta(ctl)) ctl_reset(ctl);
}
