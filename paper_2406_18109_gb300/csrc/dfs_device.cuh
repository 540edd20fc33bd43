// dfs_device.cuh -- per-operator device templates composed by the code
// generator into one sm_103a kernel per launch group.
//
// The paper builds a fused task body by composing the bodies of the tasks of
// a fusible prefix in program order, then fusing their loops and keeping the
// temporaries local (Section 6.3, Fig. 8).  Here each task body is one of the
// device functions below applied to one element (or one CSR row); the
// generator emits one loop nest per run of tasks with the same iteration
// space, in which temporaries are registers.
//
// Rounding: every element operation rounds once to its dtype through the
// explicitly rounded intrinsics (__fadd_rn, __dmul_rn, ...).  The compiler
// never contracts those into FMAs, so a fused kernel computes exactly what
// the unfused kernels compute through memory.  Library math functions
// (expf, powf, erf, ...) are called, never re-implemented.
//
// The exceptions are the FP32 erf (erf_mag) and the FP32 log (log_f32), this
// library's own approximations with stated error bounds.
//
// This file is embedded in the library and handed to NVRTC; it is also
// compiled by nvcc at build time as a syntax and target check.
#pragma once

namespace dfs {

typedef long long i64;
typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------- element ops
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float op_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double op_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float op_pow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double op_pow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float op_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double op_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float op_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double op_min(double a, double b) { return fmin(a, b); }

__device__ __forceinline__ float op_copy(float a) { return a; }
__device__ __forceinline__ double op_copy(double a) { return a; }
__device__ __forceinline__ float op_neg(float a) { return -a; }
__device__ __forceinline__ double op_neg(double a) { return -a; }
__device__ __forceinline__ float op_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double op_abs(double a) { return fabs(a); }
__device__ __forceinline__ float op_exp(float a) { return expf(a); }
__device__ __forceinline__ double op_exp(double a) { return exp(a); }
__device__ __forceinline__ double op_log(double a) { return log(a); }
__device__ __forceinline__ float op_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double op_sqrt(double a) { return __dsqrt_rn(a); }
// erf is odd, and ERF is defined as the odd extension of the library's erf on
// [0, inf]: op_erf(a) = copysign(erf(|a|), a).  Any two arguments of equal
// magnitude then share erf_mag exactly, which lets a fused body evaluate
// N(d) and N(-d) with one erf (the code generator's sharing of negations).
// erf(|a|) in FP32 is this library's own approximation, written from the
// mathematics (coefficients fitted by csrc/erf_f32_fit.py, weighted least
// squares on Chebyshev nodes against 40-digit erf):
//   x = |a| < 1:        erf(x) = x + x q(x^2), q of degree 6 fitted to erf(x)/x - 1
//   1 <= x < 3.92:      erf(x) = 1 - 2^p(x),  p of degree 6 fitted to log2 erfc(x),
//                       weighted by erfc(x) (the error that reaches erf)
//   x >= 3.92, inf:     1 (erfc(x) < 2^-25 there); NaN stays NaN
// Its error bound is 2 ulp, the bound CUDA documents for erff (in float32
// emulation of these steps, with the hardware exp2 off by up to 2 ulp either
// way: 1.83 ulp at most over [0, 4.2]); the GPU tests check it against erf in
// FP64 over dense grids and random arguments.  erf_mag2 evaluates two lanes
// with the packed forms of the same operations, each rounded as the scalar
// one, so both give the same bits; the polynomials are evaluated in x itself
// (x only ever a multiplicand), so no product of the caller can be contracted
// into them.
__device__ __forceinline__ float ex2_ftz(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
#define DFS_ERF_A0 0x1.06eba8p-3f
#define DFS_ERF_A1 -0x1.81273ep-2f
#define DFS_ERF_A2 0x1.ce2cf0p-4f
#define DFS_ERF_A3 -0x1.b7f88cp-6f
#define DFS_ERF_A4 0x1.5401dcp-8f
#define DFS_ERF_A5 -0x1.a3dc18p-11f
#define DFS_ERF_A6 0x1.49234ep-14f
#define DFS_ERF_B0 -0x1.041348p-11f
#define DFS_ERF_B1 -0x1.a043c8p+0f
#define DFS_ERF_B2 -0x1.d76156p-1f
#define DFS_ERF_B3 -0x1.309f10p-3f
#define DFS_ERF_B4 0x1.021102p-5f
#define DFS_ERF_B5 -0x1.16abccp-8f
#define DFS_ERF_B6 0x1.19f63ep-12f
__device__ __forceinline__ float erf_mag(float a) {
  const float x = fabsf(a);
  const float t = __fmul_rn(x, x);
  float q = DFS_ERF_A6;
  q = __fmaf_rn(q, t, DFS_ERF_A5);
  q = __fmaf_rn(q, t, DFS_ERF_A4);
  q = __fmaf_rn(q, t, DFS_ERF_A3);
  q = __fmaf_rn(q, t, DFS_ERF_A2);
  q = __fmaf_rn(q, t, DFS_ERF_A1);
  q = __fmaf_rn(q, t, DFS_ERF_A0);
  const float ra = __fmaf_rn(x, q, x);
  float p = DFS_ERF_B6;
  p = __fmaf_rn(p, x, DFS_ERF_B5);
  p = __fmaf_rn(p, x, DFS_ERF_B4);
  p = __fmaf_rn(p, x, DFS_ERF_B3);
  p = __fmaf_rn(p, x, DFS_ERF_B2);
  p = __fmaf_rn(p, x, DFS_ERF_B1);
  p = __fmaf_rn(p, x, DFS_ERF_B0);
  const float rb = __fadd_rn(1.0f, -ex2_ftz(p));
  const float r = x < 1.0f ? ra : rb;
  return x >= 3.92f ? 1.0f : r;
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 erf_mag2(float a0, float a1) {
  const float2 x = make_float2(fabsf(a0), fabsf(a1));
  const float2 t = __fmul2_rn(x, x);
  float2 q = f2(DFS_ERF_A6);
  q = __ffma2_rn(q, t, f2(DFS_ERF_A5));
  q = __ffma2_rn(q, t, f2(DFS_ERF_A4));
  q = __ffma2_rn(q, t, f2(DFS_ERF_A3));
  q = __ffma2_rn(q, t, f2(DFS_ERF_A2));
  q = __ffma2_rn(q, t, f2(DFS_ERF_A1));
  q = __ffma2_rn(q, t, f2(DFS_ERF_A0));
  const float2 ra = __ffma2_rn(x, q, x);
  float2 p = f2(DFS_ERF_B6);
  p = __ffma2_rn(p, x, f2(DFS_ERF_B5));
  p = __ffma2_rn(p, x, f2(DFS_ERF_B4));
  p = __ffma2_rn(p, x, f2(DFS_ERF_B3));
  p = __ffma2_rn(p, x, f2(DFS_ERF_B2));
  p = __ffma2_rn(p, x, f2(DFS_ERF_B1));
  p = __ffma2_rn(p, x, f2(DFS_ERF_B0));
  const float2 rb = __fadd2_rn(f2(1.0f), make_float2(-ex2_ftz(p.x), -ex2_ftz(p.y)));
  float2 r;
  r.x = x.x >= 3.92f ? 1.0f : (x.x < 1.0f ? ra.x : rb.x);
  r.y = x.y >= 3.92f ? 1.0f : (x.y < 1.0f ? ra.y : rb.y);
  return r;
}
// log(a) in FP32, this library's own approximation, written from the
// mathematics (coefficients fitted by csrc/log_f32_fit.py, weighted least
// squares on Chebyshev nodes against 40-digit log1p):
//   a = 2^k m with m in [sqrt(1/2), sqrt(2)), read from the bits of a
//   f = m - 1                      (exact: m lies within a factor 2 of 1)
//   log(m) = f + f^2 Q(f)          Q of degree 8 fitted to (log1p(f) - f) / f^2,
//                                  weighted by |f| (the error that reaches log)
//   log(a) = k ln2_hi + (k ln2_lo + log(m)), ln2 split so that k ln2_hi is exact
// Positive normal arguments take these steps directly; the others take them
// after a subnormal is scaled by 2^23 (k lowered by 23), or are 0, negative,
// inf or NaN, where the hardware log2 gives the IEEE result (-inf, NaN, inf,
// NaN).  Error bound: 1 ulp, the bound CUDA documents for logf (in float32
// emulation of these steps: 0.92 ulp at most over every float in [1/16, 16)
// and 4 M random normal floats); the GPU tests check it against log in FP64.
// log_f32x2 takes the same steps for two lanes with the packed operations,
// each rounded as the scalar one, so both give the same bits; a pair with an
// argument that is not positive normal goes through log_f32 lane by lane.
#define DFS_LOG_C0 -0x1.fffff8p-2f
#define DFS_LOG_C1 0x1.555550p-2f
#define DFS_LOG_C2 -0x1.000428p-2f
#define DFS_LOG_C3 0x1.99a46ap-3f
#define DFS_LOG_C4 -0x1.54279ep-3f
#define DFS_LOG_C5 0x1.226922p-3f
#define DFS_LOG_C6 -0x1.0f2d10p-3f
#define DFS_LOG_C7 0x1.08782ap-3f
#define DFS_LOG_C8 -0x1.38d522p-4f
#define DFS_LN2_HI 0x1.62e400p-1f
#define DFS_LN2_LO 0x1.7f7d1cp-20f
#define DFS_SQRT_HALF_BITS 0x3f3504f3
__device__ __forceinline__ float lg2_ftz(float v) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
// positive, normal and finite
__device__ __forceinline__ bool log_plain(float a) { return (u32)__float_as_int(a) - 0x00800000u < 0x7f000000u; }
// k and m of a positive normal a (d: the bits of a less those of sqrt(1/2))
__device__ __forceinline__ float log_k(int d) { return (float)(d >> 23); }
__device__ __forceinline__ float log_m(int d) { return __int_as_float((d & 0x007fffff) + DFS_SQRT_HALF_BITS); }
__device__ __forceinline__ float log_mk(float f, float kf) {
  const float f2 = __fmul_rn(f, f);
  float q = DFS_LOG_C8;
  q = __fmaf_rn(q, f, DFS_LOG_C7);
  q = __fmaf_rn(q, f, DFS_LOG_C6);
  q = __fmaf_rn(q, f, DFS_LOG_C5);
  q = __fmaf_rn(q, f, DFS_LOG_C4);
  q = __fmaf_rn(q, f, DFS_LOG_C3);
  q = __fmaf_rn(q, f, DFS_LOG_C2);
  q = __fmaf_rn(q, f, DFS_LOG_C1);
  q = __fmaf_rn(q, f, DFS_LOG_C0);
  const float lm = __fmaf_rn(f2, q, f);
  return __fmaf_rn(kf, DFS_LN2_HI, __fmaf_rn(kf, DFS_LN2_LO, lm));
}
static __device__ __noinline__ float log_rare(float a) {
  const bool sub = a < 0x1p-126f;                 // subnormals of either sign become normal
  const float x = sub ? __fmul_rn(a, 0x1p23f) : a;
  if (!log_plain(x)) return lg2_ftz(x);           // +-0 -> -inf, < 0 -> NaN, inf -> inf, NaN -> NaN
  const int d = __float_as_int(x) - DFS_SQRT_HALF_BITS;  // x: a positive subnormal scaled by 2^23
  return log_mk(__fsub_rn(log_m(d), 1.0f), __fsub_rn(log_k(d), 23.0f));
}
__device__ __forceinline__ float log_f32(float a) {
  if (!log_plain(a)) return log_rare(a);
  const int d = __float_as_int(a) - DFS_SQRT_HALF_BITS;
  return log_mk(__fsub_rn(log_m(d), 1.0f), log_k(d));
}
__device__ __forceinline__ float2 log_f32x2(float a0, float a1) {
  if (!(log_plain(a0) && log_plain(a1))) return make_float2(log_f32(a0), log_f32(a1));
  const int d0 = __float_as_int(a0) - DFS_SQRT_HALF_BITS, d1 = __float_as_int(a1) - DFS_SQRT_HALF_BITS;
  const float2 kf = make_float2(log_k(d0), log_k(d1));
  const float2 f = __fadd2_rn(make_float2(log_m(d0), log_m(d1)), f2(-1.0f));
  const float2 ff = __fmul2_rn(f, f);
  float2 q = f2(DFS_LOG_C8);
  q = __ffma2_rn(q, f, f2(DFS_LOG_C7));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C6));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C5));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C4));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C3));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C2));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C1));
  q = __ffma2_rn(q, f, f2(DFS_LOG_C0));
  const float2 lm = __ffma2_rn(ff, q, f);
  return __ffma2_rn(kf, f2(DFS_LN2_HI), __ffma2_rn(kf, f2(DFS_LN2_LO), lm));
}
__device__ __forceinline__ float op_log(float a) { return log_f32(a); }
__device__ __forceinline__ double erf_mag(double a) { return erf(fabs(a)); }
__device__ __forceinline__ float erf_sign(float m, float a) { return copysignf(m, a); }
__device__ __forceinline__ double erf_sign(double m, double a) { return copysign(m, a); }
__device__ __forceinline__ float op_erf(float a) { return erf_sign(erf_mag(a), a); }
__device__ __forceinline__ double op_erf(double a) { return erf_sign(erf_mag(a), a); }
// Standard normal CDF through erf: 0.5 * (1 + erf(x * (1/sqrt 2))), in steps:
// the scaled argument, erf of it, then the affine map.
__device__ __forceinline__ float ncdf_arg(float a) { return op_mul(a, 0.70710678118654752440f); }
__device__ __forceinline__ double ncdf_arg(double a) { return op_mul(a, 0.70710678118654752440); }
__device__ __forceinline__ float ncdf_of_erf(float e) { return op_mul(0.5f, op_add(1.0f, e)); }
__device__ __forceinline__ double ncdf_of_erf(double e) { return op_mul(0.5, op_add(1.0, e)); }
__device__ __forceinline__ float op_ncdf(float a) { return ncdf_of_erf(op_erf(ncdf_arg(a))); }
__device__ __forceinline__ double op_ncdf(double a) { return ncdf_of_erf(op_erf(ncdf_arg(a))); }

// Two FP32 lanes per instruction (the packed add and multiply of sm_100 and
// later): each lane is rounded to nearest exactly as op_add / op_mul round
// it.  The compiler may contract a packed product whose only use is a packed
// or scalar sum into one fused multiply-add, whatever rounding the source
// asks for (measured on GB300), which rounds once where the unfused tasks
// round twice; so the code generator pairs an operation only when no product
// of the body feeds a sum of the body (add, subtract, SUM reduction).
__device__ __forceinline__ float2 pk_add(float a0, float a1, float b0, float b1) {
  return __fadd2_rn(make_float2(a0, a1), make_float2(b0, b1));
}
// ncdf_arg and ncdf_of_erf of two lanes
__device__ __forceinline__ float2 pk_ncdf_arg(float a0, float a1) {
  return __fmul2_rn(make_float2(a0, a1), make_float2(0.70710678118654752440f, 0.70710678118654752440f));
}
__device__ __forceinline__ float2 pk_ncdf_of_erf(float e0, float e1) {
  return __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(e0, e1)));
}

// Reduction step and CSR row product: contraction into FMA is intended here
// (one task's own arithmetic).
__device__ __forceinline__ float red_fma(float a, float b, float acc) { return fmaf(a, b, acc); }
__device__ __forceinline__ double red_fma(double a, double b, double acc) { return fma(a, b, acc); }

// ------------------------------------------------------------ memory access
// Plain (coherent) loads: data written by an earlier phase of the same kernel
// must not be served by the non-coherent read-only path.
template <typename T> __device__ __forceinline__ T ld(const T* p) { return *p; }
// Read-only path, for stores nothing in the kernel writes.
template <typename T> __device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

struct f32x4 { float v[4]; };
struct f64x2 { double v[2]; };

__device__ __forceinline__ f32x4 ld4(const float* p) {
  float4 t = *reinterpret_cast<const float4*>(p);
  f32x4 r; r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w; return r;
}
__device__ __forceinline__ f32x4 ld4ro(const float* p) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  f32x4 r; r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w; return r;
}
// Streaming load (evict-first): inputs read exactly once.
__device__ __forceinline__ f32x4 ld4cs(const float* p) {
  float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  f32x4 r; r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w; return r;
}
__device__ __forceinline__ void st4(float* p, const f32x4& r) {
  *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
}
__device__ __forceinline__ void st4cs(float* p, const f32x4& r) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
}
__device__ __forceinline__ f64x2 ld2(const double* p) {
  double2 t = *reinterpret_cast<const double2*>(p);
  f64x2 r; r.v[0] = t.x; r.v[1] = t.y; return r;
}
__device__ __forceinline__ f64x2 ld2ro(const double* p) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  f64x2 r; r.v[0] = t.x; r.v[1] = t.y; return r;
}
__device__ __forceinline__ f64x2 ld2cs(const double* p) {
  double2 t = __ldcs(reinterpret_cast<const double2*>(p));
  f64x2 r; r.v[0] = t.x; r.v[1] = t.y; return r;
}
// Vectors that start S elements past a 16-byte boundary: p is that
// boundary; two aligned vector loads, the wanted elements picked in
// registers.  Used for views whose column origin is not vector-aligned (the
// shifted views of a stencil) when every root row is a whole number of
// vectors, so both aligned loads stay inside the row of the used elements.
template <int S> __device__ __forceinline__ f32x4 ld4s(const float* p) {
  const f32x4 a = ld4(p), b = ld4(p + 4);
  f32x4 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.v[k] = (S + k < 4) ? a.v[S + k] : b.v[S + k - 4];
  return r;
}
template <int S> __device__ __forceinline__ f32x4 ld4sro(const float* p) {
  const f32x4 a = ld4ro(p), b = ld4ro(p + 4);
  f32x4 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.v[k] = (S + k < 4) ? a.v[S + k] : b.v[S + k - 4];
  return r;
}
template <int S> __device__ __forceinline__ f64x2 ld2s(const double* p) {
  const f64x2 a = ld2(p), b = ld2(p + 2);
  f64x2 r;
#pragma unroll
  for (int k = 0; k < 2; ++k) r.v[k] = (S + k < 2) ? a.v[S + k] : b.v[S + k - 2];
  return r;
}
template <int S> __device__ __forceinline__ f64x2 ld2sro(const double* p) {
  const f64x2 a = ld2ro(p), b = ld2ro(p + 2);
  f64x2 r;
#pragma unroll
  for (int k = 0; k < 2; ++k) r.v[k] = (S + k < 2) ? a.v[S + k] : b.v[S + k - 2];
  return r;
}
__device__ __forceinline__ void st2(double* p, const f64x2& r) {
  *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
}
__device__ __forceinline__ void st2cs(double* p, const f64x2& r) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
}

// ---------------------------------------------------------------- CSR row
// y_r = sum_k val[k] * x[col[k]] over k in [rowptr[r], rowptr[r+1]).
template <typename T>
__device__ __forceinline__ T spmv_row(const int* __restrict__ rowptr, const int* __restrict__ col,
                                      const T* __restrict__ val, const T* x, i64 r) {
  const int k0 = __ldg(rowptr + r), k1 = __ldg(rowptr + r + 1);
  T acc = T(0);
  int k = k0;
  for (; k + 1 < k1; k += 2) {
    const int c0 = __ldg(col + k), c1 = __ldg(col + k + 1);
    const T v0 = __ldg(val + k), v1 = __ldg(val + k + 1);
    const T x0 = ld(x + c0), x1 = ld(x + c1);
    acc = red_fma(v0, x0, acc);
    acc = red_fma(v1, x1, acc);
  }
  if (k < k1) acc = red_fma(__ldg(val + k), ld(x + __ldg(col + k)), acc);
  return acc;
}

// Rows of y = A x for the 32 lanes of a warp, K lanes per row (K a power of
// two, 1..32).  In round t (0 <= t < K) the lanes of group g = lane / K
// compute the row of lane t * (32 / K) + g: lane q of the group sums the
// entries k0 + q, k0 + q + K, ... in order with fma, and the group combines
// its K partial sums with a xor butterfly (every lane of the group ends with
// the same bits, since each level adds the same two values).  Each round's
// loads of col and val are K consecutive entries per row, so dense-ish rows
// are read with few memory transactions per instruction.  Every lane of the
// warp must call it with the same K (warp-uniform control flow); a lane with
// act false owns no row and gets 0.  K = 1 is spmv_row on every lane.
template <typename T>
__device__ __forceinline__ T spmv_warp(const int* __restrict__ rowptr, const int* __restrict__ col,
                                       const T* __restrict__ val, const T* x, i64 r, bool act, int K) {
  if (K <= 1) return act ? spmv_row<T>(rowptr, col, val, x, r) : T(0);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int rpr = 32 / K, g = lane / K, q = lane & (K - 1);
  T mine = T(0);
  for (int t = 0; t < K; ++t) {
    const int src = t * rpr + g;
    const i64 rr = __shfl_sync(full, r, src);
    const int ra = __shfl_sync(full, act ? 1 : 0, src);
    T acc = T(0);
    if (ra) {
      const int k0 = __ldg(rowptr + rr), k1 = __ldg(rowptr + rr + 1);
      for (int k = k0 + q; k < k1; k += K) acc = red_fma(__ldg(val + k), ld(x + __ldg(col + k)), acc);
    }
    for (int m = 1; m < K; m <<= 1) acc = op_add(acc, __shfl_xor_sync(full, acc, m));
    const T got = __shfl_sync(full, acc, (lane % rpr) * K);
    if (t == lane / rpr) mine = got;
  }
  return act ? mine : T(0);
}

// ----------------------------------------------------------- control block
// One per context, zero-initialised; every kernel leaves it zeroed on exit.
constexpr int kTickets = 16;
struct Ctl {
  u32 bar_arrive;   // grid-barrier arrivals (monotone within a launch)
  u32 exit_arrive;  // CTAs that finished the launch
  int err;          // first device error (0 = none)
  int err_where;    // barrier index that timed out
  u64 pad[2];
  u64 ticket[kTickets];  // work-queue counters, one per dynamically dealt phase
};

__device__ __forceinline__ u64 globaltimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ u32 ld_acquire_u32(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

enum { ERR_BARRIER_TIMEOUT = 1 };

__device__ __forceinline__ void red_release_add_u32(u32* p, u32 v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ u32 atom_acq_rel_add_u32(u32* p, u32 v) {
  u32 old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier among the co-resident CTAs of a cooperative launch.
// Arrivals count up; barrier k of the launch completes when gridDim.x * k
// CTAs have arrived.  The CTA's writes are ordered before its arrival by the
// block barrier and the arrival's release; the acquire load that sees the
// last arrival orders every CTA's writes before the reads that follow (the
// PTX memory model's release/acquire pattern at gpu scope).  Measured on
// GB300 over 128 CTAs: 1.28 us per barrier, against 1.43 us with a 64 ns
// sleep between polls and 1.54 us with full fences around a relaxed add; one
// flag per CTA polled by every CTA (1.3-7.8 us from 128 to 608 CTAs) or by a
// master that then releases the rest (2.9-4.7 us) was slower.  The wait
// gives up after `timeout_ns` (or as soon as any CTA has recorded an error),
// records the failure and returns false; callers then skip the rest of the
// kernel, so no CTA ever waits forever.
// `arrive` is false only under the test hook that withholds one arrival.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, u32 k, u64 timeout_ns, bool arrive = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (arrive) red_release_add_u32(&ctl->bar_arrive, 1u);
    const u32 target = gridDim.x * k;
    const u64 t0 = globaltimer_ns();
    while (ld_acquire_u32(&ctl->bar_arrive) < target) {
      if (ld_relaxed_int(&ctl->err) != 0) { ok = 0; break; }
      if (globaltimer_ns() - t0 > timeout_ns) {
        if (atomicCAS(&ctl->err, 0, (int)ERR_BARRIER_TIMEOUT) == 0) ctl->err_where = (int)k;
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Kernel exit: returns true in exactly one CTA -- the last to arrive -- after
// every other CTA's writes are visible.  That CTA finishes pending
// reductions, writes the 0-d results and then calls ctl_reset().
__device__ __forceinline__ bool last_cta(Ctl* ctl) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const u32 n = atom_acq_rel_add_u32(&ctl->exit_arrive, 1u);
    s_last = (n + 1 == gridDim.x);
  }
  __syncthreads();
  return s_last != 0;
}
__device__ __forceinline__ void ctl_reset(Ctl* ctl) {
  if (threadIdx.x == 0) {
    ctl->bar_arrive = 0;
    ctl->exit_arrive = 0;
    for (int i = 0; i < kTickets; ++i) ctl->ticket[i] = 0;
    __threadfence();
  }
}

// Next point of a dynamically dealt phase: thread 0 takes a ticket from the
// phase's counter and the block reads it.  Which CTA runs a point does not
// change any result (reductions keep one partial per point).
__device__ __forceinline__ i64 take_ticket(Ctl* ctl, int q, i64* s_ticket) {
  if (threadIdx.x == 0) *s_ticket = (i64)atomicAdd((unsigned long long*)&ctl->ticket[q], 1ull);
  __syncthreads();
  const i64 t = *s_ticket;
  __syncthreads();
  return t;
}

// ------------------------------------------------ staged SpMV x windows
// An SpMV point (a tile of rows) reads x at the columns of its rows.  When the
// task carries a window argument, up to three windows [lo_k, lo_k + len_k) of
// x covering most of those columns are copied into shared memory by the bulk
// copy engine (TMA, cp.async.bulk) at the start of the point, completing on
// one mbarrier; the rows then read x from shared memory inside the windows
// and from global memory outside them.  The values are the same either way,
// so results do not depend on the staging.  Windows come from host data:
// every field is checked here (bounds, 16-byte alignment of source and size,
// the shared-memory capacity) and a point whose record fails the checks is
// simply not staged.
struct XWin {
  int lo[3];
  int len[3];
};

enum { ERR_COPY_TIMEOUT = 2 };

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// Once per CTA, by every thread, before the first xstage.
__device__ __forceinline__ void xstage_init(u64* mbar) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
}

__device__ __forceinline__ bool mbar_try(u64* mbar, u32 phase) {
  u32 done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(phase)
      : "memory");
  return done != 0;
}

// Stages the point's windows (record w: lo0, len0, lo1, len1, lo2, len2 in
// elements of x, whose extent is xlen) into xs (cap elements).  Called by
// every thread of the CTA at the same point.  Returns the windows in use (all
// lengths 0 when nothing is staged).  The wait for the bytes gives up after
// timeout_ns: the CTA then records ERR_COPY_TIMEOUT, waits once more (bounded)
// for its copy, and stops staging for the rest of the launch (`live`).
template <typename T>
__device__ __forceinline__ XWin xstage(T* xs, int cap, const T* x, i64 xlen, const int* w, u64* mbar, u32& phase,
                                       bool& live, Ctl* ctl, u64 timeout_ns) {
  XWin win;
  i64 tot = 0;
  bool ok = live;
  for (int k = 0; k < 3; ++k) {
    const int lo = ldro(w + 2 * k), len = ldro(w + 2 * k + 1);
    const bool good = len >= 0 && len <= cap && lo >= 0 && (i64)lo + len <= xlen &&
                      ((unsigned long long)(x + lo) & 15ull) == 0 && ((len * (int)sizeof(T)) & 15) == 0;
    ok = ok && good;
    win.lo[k] = lo;
    win.len[k] = good ? len : 0;
    tot += good ? len : 0;
  }
  if (!ok || tot == 0 || tot > cap) {
    for (int k = 0; k < 3; ++k) win.len[k] = 0;
    return win;
  }
  __syncthreads();  // every read of the previous point's windows is done
  if (threadIdx.x == 0) {
    // the generic-proxy writes of x (earlier phases, ordered by the grid
    // barrier) and of xs (the previous point) before the async-proxy copy
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"((u32)tot * (u32)sizeof(T))
                 : "memory");
    int off = 0;
    for (int k = 0; k < 3; ++k) {
      if (win.len[k] > 0)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(xs + off)),
                     "l"(x + win.lo[k]), "r"(win.len[k] * (int)sizeof(T)), "r"(smem_u32(mbar))
                     : "memory");
      off += win.len[k];
    }
  }
  bool done = mbar_try(mbar, phase);
  const u64 t0 = globaltimer_ns();
  while (!done && globaltimer_ns() - t0 <= timeout_ns) done = mbar_try(mbar, phase);
  if (!__syncthreads_and(done ? 1 : 0)) {
    if (threadIdx.x == 0 && atomicCAS(&ctl->err, 0, (int)ERR_COPY_TIMEOUT) == 0) ctl->err_where = -1;
    const u64 t1 = globaltimer_ns();
    while (!mbar_try(mbar, phase) && globaltimer_ns() - t1 <= timeout_ns) {
    }
    __syncthreads();
    live = false;
    for (int k = 0; k < 3; ++k) win.len[k] = 0;
    return win;
  }
  phase ^= 1u;
  return win;
}

// x[c] from the staged windows when c falls in one, else from global memory.
template <typename T>
__device__ __forceinline__ T xsv(const T* x, const T* xs, const XWin& w, int c) {
  unsigned d;
  if ((d = (unsigned)(c - w.lo[0])) < (unsigned)w.len[0]) return xs[d];
  if ((d = (unsigned)(c - w.lo[1])) < (unsigned)w.len[1]) return xs[w.len[0] + d];
  if ((d = (unsigned)(c - w.lo[2])) < (unsigned)w.len[2]) return xs[w.len[0] + w.len[1] + d];
  return ld(x + c);
}

// spmv_row with x read through the staged windows: the same entries in the
// same order with the same fma, so the same bits.
template <typename T>
__device__ __forceinline__ T spmv_row_xs(const int* __restrict__ rowptr, const int* __restrict__ col,
                                         const T* __restrict__ val, const T* x, i64 r, const T* xs, const XWin& w) {
  const int k0 = __ldg(rowptr + r), k1 = __ldg(rowptr + r + 1);
  T acc = T(0);
  int k = k0;
  for (; k + 1 < k1; k += 2) {
    const int c0 = __ldg(col + k), c1 = __ldg(col + k + 1);
    const T v0 = __ldg(val + k), v1 = __ldg(val + k + 1);
    const T x0 = xsv(x, xs, w, c0), x1 = xsv(x, xs, w, c1);
    acc = red_fma(v0, x0, acc);
    acc = red_fma(v1, x1, acc);
  }
  if (k < k1) acc = red_fma(__ldg(val + k), xsv(x, xs, w, __ldg(col + k)), acc);
  return acc;
}

// --------------------------------------------------------------- reductions
template <typename T> __device__ __forceinline__ T warp_sum_xor(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread in a fixed order; the result is returned to
// thread 0 only.  `buf` holds blockDim.x values.  Every thread parks its value
// in shared memory and warp 0 alone adds: lane l sums the values of lanes l of
// warps 0, 1, ... in order, then a xor butterfly combines the 32 lane sums.
// FP64 adds are scarce on GB300 (about two lane operations per SM and clock):
// a butterfly in every warp cost 45 warp instructions per 256-thread block,
// this 12.
template <typename T> __device__ __forceinline__ T block_sum(T v, T* buf) {
  buf[threadIdx.x] = v;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    r = buf[threadIdx.x];
    for (int w = 1; w < nw; ++w) r += buf[threadIdx.x + 32 * w];
    r = warp_sum_xor(r);
  }
  __syncthreads();
  return r;
}

// Sum of partials[0..n) in a fixed order (lane-strided, then a butterfly);
// every thread of every warp computes the same value, so any CTA may use it.
template <typename T> __device__ __forceinline__ T sum_partials(const T* partials, i64 n) {
  const int l = threadIdx.x & 31;
  T acc = T(0);
  for (i64 i = l; i < n; i += 32) acc += ld(partials + i);
  return warp_sum_xor(acc);
}

}  // namespace dfs
