// device_common.cuh -- device helpers shared by the particle kernels (forces,
// binning) and their adjoints: exact element location, the Lagrange basis,
// the closures' elementary functions per precision and the force parameters.
#pragma once
#include <cstdint>

#include "internal.h"
#include "df64.cuh"

namespace cfdem {

// ----------------------------------------------------------------------------
// exact location arithmetic (no contraction into FMA: same rounding as the
// plain IEEE definition)

__device__ __forceinline__ bool in_box(double x, double x0, double L) {
  double slack = __dmul_rn(1e-12, L);
  double lo = __dsub_rn(x0, slack);
  double hi = __dadd_rn(__dadd_rn(x0, L), slack);
  return x >= lo && x <= hi;  // false for NaN
}

// element index along one axis and the reference coordinate; caller checked
// in_box so t is finite
__device__ __forceinline__ int elem_axis(double x, double x0, double h, int N, double* xi) {
  double t = __ddiv_rn(__dsub_rn(x, x0), h);
  double f = floor(t);
  int i = (int)f;
  i = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
  *xi = __dsub_rn(t, (double)i);
  return i;
}

// element index and reference coordinate from a multiplication by 1/h; the
// IEEE division of the definition is redone only when the product lies
// within 1e-9 of an element face, where the two could round to different
// sides.  xi is then within a few ulps of the divided value.
__device__ __forceinline__ int elem_axis_fast(double x, double x0, double h, double inv_h, int N,
                                              double* xi) {
  double t = (x - x0) * inv_h;
  double f = floor(t);
  double fr = t - f;
  if (fr < 1e-9 || fr > 1.0 - 1e-9) {
    t = __ddiv_rn(__dsub_rn(x, x0), h);
    f = floor(t);
  }
  int i = (int)f;
  i = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
  *xi = t - (double)i;
  return i;
}


// bin index along one axis, floor((x - x0) / be) clamped to [0, nb-1], from a
// multiplication by 1/be; the IEEE division of the definition is redone only
// within 1e-9 of a bin face, where the two could round to different sides
__device__ __forceinline__ int bin_axis_fast(double x, double x0, double be, double inv_be,
                                             int nb) {
  double t = (x - x0) * inv_be;
  double f = floor(t);
  double fr = t - f;
  if (fr < 1e-9 || fr > 1.0 - 1e-9) {
    t = __ddiv_rn(__dsub_rn(x, x0), be);
    f = floor(t);
  }
  if (!(f >= 0.0)) return 0;
  if (f > (double)(nb - 1)) return nb - 1;
  return (int)f;
}

// bin_axis_fast behind a real call, for the rare particles near a bin face
// (inlined, its FP64 instructions would be predicated into every thread)
static __device__ __noinline__ int bin_axis_slow(double x, double x0, double be, double inv_be,
                                                 int nb) {
  return bin_axis_fast(x, x0, be, inv_be, nb);
}

// elem_axis_fast behind a real call, for the same reason
static __device__ __noinline__ int elem_axis_slow(double x, double x0, double h, double inv_h,
                                                  int N, double* xi) {
  return elem_axis_fast(x, x0, h, inv_h, N, xi);
}

// the integer key of a double whose signed order is the order of the values
// (NaNs fall outside every finite interval); the host computes the same keys
// for the in_box bounds, so that the mixed path tests the box without FP64
// instructions
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ bool in_box_key(double v, long long lo, long long hi) {
  const long long k = order_key(v);
  return k >= lo && k <= hi;
}

// floor of t for 0 <= t < 2^22 and its integer value with FP32 additions
// only (adding 2^23 rounds t to an integer held in the low significand
// bits); conversions between integer and floating types issue on this
// part's narrow FP64 pipe
__device__ __forceinline__ float floor_small(float t, int* k) {
  const float y = t + 8388608.0f;
  float r = y - 8388608.0f;
  int i = __float_as_int(y) - 0x4B000000;
  if (r > t) {
    r -= 1.0f;
    i -= 1;
  }
  *k = i;
  return r;
}

// Cell index floor(t), t = (x - x0) / edge, on a grid of n cells, from the
// double-float split of x (t to ~2^-46 |x| / edge), and the fraction t -
// floor(t) as double-float.  Returns -1 when t lies within 1e-5 of a cell
// face or outside [0, n): there the caller's FP64 rule decides, so the cell
// is the one the IEEE definition gives.  nm1f = n - 1 as a float.
__device__ __forceinline__ int cell_df(double x, float x0_hi, float x0_lo, float inv_hi,
                                       float inv_lo, float nm1f, df64* frac) {
  const df64 d = df_from_double_int(x) - df64(x0_hi, x0_lo);
  const df64 t = d * df64(inv_hi, inv_lo);
  if (!(t.hi >= 0.0f && t.hi < nm1f + 1.0f)) return -1;
  int i;
  const float fl = floor_small(t.hi, &i);
  const float fr = (t.hi - fl) + t.lo;
  if (!(fr >= 1e-5f && fr <= 1.0f - 1e-5f && fl <= nm1f)) return -1;
  if (frac) *frac = df_renorm(t.hi - fl, t.lo);  // t.hi - fl is exact
  return i;
}

__device__ __forceinline__ void report_bad(DevStatus* st, int64_t i) {
  atomicMin(&st->first_bad, (unsigned long long)i);
}

template <typename T>
__device__ __forceinline__ T t_sqrt(T v);
template <>
__device__ __forceinline__ double t_sqrt<double>(double v) { return sqrt(v); }
template <>
__device__ __forceinline__ float t_sqrt<float>(float v) { return sqrtf(v); }

// Lagrange basis of degree D on nodes z and its derivative at t; lw[a] =
// 1 / prod_{b != a} (z_a - z_b) comes from the host so that no division is
// done here
template <int D, typename T, typename Z>
__device__ __forceinline__ void lagrange(const Z* zz, const Z* lw, T t, T* l, T* dl) {
  T d[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) d[a] = t - (T)zz[a];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    T v = (T)1, dv = (T)0;
#pragma unroll
    for (int b = 0; b <= D; ++b) {
      if (b == a) continue;
      dv = dv * d[b] + v;
      v = v * d[b];
    }
    l[a] = v * (T)lw[a];
    if (dl) dl[a] = dv * (T)lw[a];
  }
}

// Lagrange basis with its first, second and (if d3 is given) third
// derivatives at t: the product prod_{b != a} (t - z_b) differentiated by
// the Leibniz rule, scaled by the barycentric weight lw[a].
template <int D, typename T, typename Z>
__device__ __forceinline__ void lagrange_d3(const Z* zz, const Z* lw, T t, T* l, T* d1, T* d2,
                                            T* d3) {
  T d[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) d[a] = t - (T)zz[a];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    T v = (T)1, v1 = (T)0, v2 = (T)0, v3 = (T)0;
#pragma unroll
    for (int b = 0; b <= D; ++b) {
      if (b == a) continue;
      v3 = v3 * d[b] + (T)3 * v2;
      v2 = v2 * d[b] + (T)2 * v1;
      v1 = v1 * d[b] + v;
      v = v * d[b];
    }
    l[a] = v * (T)lw[a];
    d1[a] = v1 * (T)lw[a];
    d2[a] = v2 * (T)lw[a];
    if (d3) d3[a] = v3 * (T)lw[a];
  }
}

template <typename T>
struct Closure {
  static __device__ __forceinline__ T log10_(T v);
  static __device__ __forceinline__ T exp_(T v);
  static __device__ __forceinline__ T logn(T v);
  static __device__ __forceinline__ T tiny();
};
template <>
struct Closure<double> {
  static __device__ __forceinline__ double log10_(double v) { return log10(v); }
  static __device__ __forceinline__ double exp_(double v) { return exp(v); }
  static __device__ __forceinline__ double logn(double v) { return log(v); }
  static __device__ __forceinline__ double tiny() { return 1e-300; }
};
template <>
struct Closure<float> {
  static __device__ __forceinline__ float log10_(float v) { return log10f(v); }
  static __device__ __forceinline__ float exp_(float v) { return expf(v); }
  static __device__ __forceinline__ float logn(float v) { return logf(v); }
  static __device__ __forceinline__ float tiny() { return 1e-37f; }
};


}  // namespace cfdem
