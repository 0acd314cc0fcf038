// df64.cuh -- double-float arithmetic: a value carried as an unevaluated sum
// of two FP32 numbers (hi + lo, |lo| <= ulp(hi) / 2), about 48 significant
// bits, on the FP32 pipes.  Addition by Knuth's two-sum, multiplication by
// the FMA-based exact product (Dekker 1971; Shewchuk 1997), square root and
// reciprocal by one Newton step from the FP32 estimate.
#pragma once

namespace cfdem {

struct df64 {
  float hi, lo;
  __host__ __device__ __forceinline__ df64() {}
  __host__ __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ df64(float v) : hi(v), lo(0.f) {}
};
__device__ __forceinline__ df64 df_renorm(float s, float e) {
  float hi = s + e;
  return df64(hi, e - (hi - s));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return df_renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ df64 df_from_double(double v) {
  float h = (float)v;
  return df64(h, (float)(v - (double)h));
}

// The same split without FP64 instructions, for bulk conversions: on this
// part every FP64 instruction -- and the conversions between integer, FP32
// and FP64, and bit scans -- issue on a narrow pipe at about 1/64 of the
// FP32 rate.  hi takes the sign, the exponent and the leading 24
// significand bits of v (truncated); lo the remaining 29 bits m times
// 2^(E - 1075), m made a float by FP32 arithmetic on exact floats 2^23 + k
// (k = m / 64 and m mod 64, each held in the low significand bits) and
// rounded once, so hi + lo = v to 2^-48 |v| and |lo| < ulp(hi).  Zero is
// split as zero; a v whose hi or lo would not be a normal float (|v| <
// 2^-74 or |v| >= 2^128, subnormals, inf, nan) takes the FP64 conversion.
// the two 32-bit halves of the bits of a double, opaque to the compiler:
// tests on them stay integer operations (the compiler otherwise turns a test
// such as (bits << 1) == 0 into an FP64 compare, which issues on the narrow
// FP64 pipe)
__device__ __forceinline__ void double_halves(double v, unsigned* lo, unsigned* hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(*lo), "=r"(*hi) : "d"(v));
}

// the FP64 conversion of the rare values, as a real call: inlined, the
// compiler predicates it into every split and its FP64 instructions issue
// on the narrow pipe even when not taken
static __device__ __noinline__ df64 df_from_double_slow(double v) { return df_from_double(v); }

__device__ __forceinline__ df64 df_from_double_int(double v) {
  unsigned lo32, hi32;
  double_halves(v, &lo32, &hi32);
  const unsigned sign = hi32 & 0x80000000u;
  const int E = (int)((hi32 >> 20) & 0x7ffu);
  // zero and subnormals (the conversion rounds them to a signed zero)
  if (E == 0) return df64(__uint_as_float(sign), 0.f);
  if (E < 949 || E > 1150) return df_from_double_slow(v);
  const float hi = __uint_as_float(sign | ((unsigned)(E - 896) << 23) |
                                   ((hi32 & 0xfffffu) << 3) | (lo32 >> 29));
  const unsigned m = lo32 & 0x1fffffffu;
  const float mh = __uint_as_float(0x4B000000u | (m >> 6)) - 8388608.0f;   // exact
  const float ml = __uint_as_float(0x4B000000u | (m & 63u)) - 8388608.0f;  // exact
  const float mf = fmaf(mh, 64.0f, ml);                                   // m, rounded
  const float lo = mf * __uint_as_float((unsigned)(E - 948) << 23);       // 2^(E - 1075)
  return df64(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

static __device__ __noinline__ double double_from_float_slow(float f) { return (double)f; }

// float -> double by moving the bit fields (exact, as the conversion is);
// subnormals, inf and nan take the conversion instruction (behind a call)
__device__ __forceinline__ double double_from_float_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u << 1) == 0u) return __longlong_as_double((long long)sgn);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0u || ef == 255u) return double_from_float_slow(f);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(ef + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// hi + lo in FP64: one addition after the two exact widenings
__device__ __forceinline__ double double_from_df_int(df64 v) {
  return double_from_float_int(v.hi) + double_from_float_int(v.lo);
}

// Compensated sum of double-float products b_k x_k: the high products are
// added with Knuth's two-sum and every error term (the product errors, the
// cross products b.hi x.lo + b.lo x.hi, the two-sum errors) is gathered in
// one FP32 correction, renormalised once at the end -- 12 FP32 instructions
// per term instead of a double-float multiply (7) and add (11).
struct DfDotAcc {
  float s, c;
  __device__ __forceinline__ void zero() { s = c = 0.f; }
  __device__ __forceinline__ void add(df64 b, df64 x) {
    float p = b.hi * x.hi;
    float e = fmaf(b.hi, x.hi, -p);
    e = fmaf(b.hi, x.lo, e);
    e = fmaf(b.lo, x.hi, e);
    float t = s + p;
    float bb = t - s;
    c += ((s - (t - bb)) + (p - bb)) + e;
    s = t;
  }
  __device__ __forceinline__ df64 get() const { return df_renorm(s, c); }
};

__device__ __forceinline__ bool df_le(df64 a, df64 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
// sqrt(a) for a > 0: x0 = a.hi rsqrt(a.hi), then x0 + (a - x0^2) / (2 x0)
__device__ __forceinline__ df64 df_sqrt(df64 a) {
  float y = rsqrtf(a.hi);
  float x0 = a.hi * y;
  float p = x0 * x0;
  float e = fmaf(x0, x0, -p);
  df64 r = a - df64(p, e);
  return df_renorm(x0, r.hi * (0.5f * y));
}
// 1/b: y0 = 1/b.hi, then y0 + y0 (1 - b y0)
__device__ __forceinline__ df64 df_recip(df64 b) {
  float y0 = 1.0f / b.hi;
  df64 r = df64(1.0f) - b * df64(y0);
  return df_renorm(y0, y0 * r.hi);
}

}  // namespace cfdem
