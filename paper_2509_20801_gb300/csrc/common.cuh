// Shared device-side definitions: complex arithmetic on double2 / float2,
// the device descriptors of strips and fronts, and launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace stdd {

// ---------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

__host__ __device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 cmk(float r, float i) { return make_float2(r, i); }

template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// acc + a*b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc - a*b
template <typename C> __host__ __device__ __forceinline__ C cfms(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// conj(a)*b
template <typename C> __host__ __device__ __forceinline__ C cconjmul(C a, C b) {
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) {
  return a.x * a.x + a.y * a.y;
}
// 1/a in complex128: conj(a) / |a|^2, one real reciprocal and three
// multiplies (the schoolbook complex division).  R. L. Smith's scaled form
// (CACM 5(8), 1962) costs two more divisions, and on a part whose FP64 pipe
// retires one warp instruction per 64 cycles per scheduler -- 1.25 TFLOP/s
// over 152 SMs -- even one thread's scalar FP64 work costs what a full
// warp's does.  |a|^2 must neither overflow nor underflow: |a| between
// 2^-511 and 2^511, far outside the stencil scale of these operators;
// callers flag pivots outside it (pivot_ok).
__device__ __forceinline__ double2 crecip(double2 a) {
  const double s = __drcp_rn(a.x * a.x + a.y * a.y);
  return make_double2(a.x * s, -a.y * s);
}
// 1/a in complex64 by Smith's algorithm: the FP32 pipe is not the limit,
// and the scaling keeps the reciprocal accurate over float's narrower range.
__device__ __forceinline__ float2 crecip(float2 a) {
  float2 r;
  if (fabsf(a.x) >= fabsf(a.y)) {
    const float t = a.y / a.x, d = a.x + a.y * t;
    r.x = 1.0f / d;
    r.y = -t / d;
  } else {
    const float t = a.x / a.y, d = a.x * t + a.y;
    r.x = t / d;
    r.y = -1.0f / d;
  }
  return r;
}
// v or -v by the sign bits alone (exactly -v: IEEE negation flips the sign)
__device__ __forceinline__ double2 cneg_if(double2 v, bool neg) {
  const long long m = neg ? (long long)(1ull << 63) : 0ll;
  v.x = __longlong_as_double(__double_as_longlong(v.x) ^ m);
  v.y = __longlong_as_double(__double_as_longlong(v.y) ^ m);
  return v;
}
__device__ __forceinline__ float2 cneg_if(float2 v, bool neg) {
  const int m = neg ? (int)(1u << 31) : 0;
  v.x = __int_as_float(__float_as_int(v.x) ^ m);
  v.y = __int_as_float(__float_as_int(v.y) ^ m);
  return v;
}
// |a|^2 is a usable pivot modulus: positive and finite (in complex128 also
// large enough for conj(a) / |a|^2 to stay finite)
template <typename R> __device__ __forceinline__ bool pivot_ok(R d2) {
  const R lo = sizeof(R) == 8 ? (R)1.0e-300 : (R)0;
  return d2 > lo && d2 < (R)INFINITY;
}

__device__ __forceinline__ double2 to_c(double2 a, double2) { return a; }
__device__ __forceinline__ float2 to_c(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }

template <typename C> __device__ __forceinline__ C shfl(C v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}

// ---------------------------------------------------------- descriptors
// One subdomain of the decomposition: an x-strip spanning every row, or a
// box of a 2-D (checkerboard) decomposition.  Its local field is W x Hl
// nodes, local node (lx, ly) at lx * Hl + ly, W = x1 - x0, Hl = y1 - y0.
struct StripDev {
  int x0, x1;          // local box columns [x0, x1) of the global grid
  int c0, c1;          // owned columns [c0, c1)
  int64_t vec_off;     // offset of the strip's local field in the local buffer
  int64_t coef_off;    // offset of the strip's x coefficients (W entries)
  int64_t fac_off;     // offset of the strip's factor block (complex entries)
  int y0, y1;          // local box rows [y0, y1) (0, ny for a strip)
  int r0, r1;          // owned rows [r0, r1)
  int64_t ycoef_off;   // offset of the local box's y coefficients (Hl entries)
};

// One front instance (a symbolic front of some strip shape in some strip).
struct FrontDev {
  int p, b;            // pivots, border
  int strip;
  int child[2];        // front instance ids (same strip), -1 if none
  int64_t node_off;    // into the shape node array (local node ids x*H + y)
  int64_t cmap_off[2]; // child's ring index -> this front's index
  int64_t inv_off[2];  // this front's index -> child's ring index or -1
  int64_t fac_off;     // absolute offset of [F11 F12] (p x n, col-major, ld p) then F21 (b x p, ld b)
  int64_t s_off;       // offset of F22 (b x b, col-major) in the level-parity workspace
  int64_t u_off;       // update vector (b x nrhs) at u_off * nrhs in the solve parity buffer
  int64_t piv_off;     // front-restricted pivoting: the front's p-entry column -> pivot map in MfArgs::pcol
  int64_t pan_off;     // and its pivot-panel scratch (p x MF_NB complex, per level) in MfArgs::panel
};

}  // namespace stdd
