// drag.cuh -- the drag closures of Sec. 2.3.2 written once for plain
// numbers (float, double) and for dual numbers carrying four derivatives,
// so that the forward force kernel and its adjoint evaluate the same
// expressions.
//
// Every closure returns the scalar coefficient c with f_D = c U, where U =
// u_f - u_p is the slip, eps the clamped fluid fraction, eps_p = 1 - eps,
// d = 2 r_p, V_p = 4/3 pi r_p^3 and Re = rho eps |U| d / mu (Eq. for Re_p):
//   0 Di Felice   1/2 rho C_D pi r_p^2 |U|, C_D = (0.63 + 4.8 / sqrt(Re))^2
//                 eps^(2 - chi), chi = 3.7 - 0.65 exp(-(1.5 - log10 Re)^2 / 2)
//   1 Dallavalle  1/2 rho C_D pi r_p^2 |U|, C_D = (0.63 + 4.8 / sqrt(Re))^2
//   2 Rong        as Di Felice with the exponent 2.65 (eps + 1) - (5.3 -
//                 3.5 eps) eps^2 exp(-(1.5 - log10 Re)^2 / 2)
//   3 Koch-Hill   beta = 18 mu eps^2 eps_p / d^2 (F_0(eps_p) + F_3(eps_p)
//                 Re / 2) V_p / eps_p, evaluated with eps_p cancelled
//   4 Gidaspow    beta V_p / eps_p (the printed beta is per unit volume of
//                 the mixture, a particle takes the share V_p / eps_p):
//                 Ergun below eps = 0.8 with |U| for the printed vector,
//                 Wen-Yu with the Schiller-Naumann C_D from 0.8 up
//   5 Beetstra    3 pi mu d eps F_i(eps, Re), the slip U for the printed u_f
// and c / eps when beta_B = beta_A / eps is asked for (Eq. beta).
//
// C_D |U| products are rewritten so that |U| -> 0 stays finite: the
// Dallavalle square as (0.63 sqrt|U| + 4.8 sqrt(mu / (rho eps d)))^2, the
// Schiller-Naumann C_D eps |U| as 24 mu / (rho d) (1 + 0.15 Re^0.687), and
// Beetstra's Re / (1 + 10^(3 eps_p) Re^-s) as Re^(1+s) / (Re^s + 10^(3 eps_p)).
#pragma once

#include "device_common.cuh"

namespace cfdem {

// ---------------------------------------------------------------- duals

template <typename T>
struct D4 {  // value and derivatives along (U_0, U_1, U_2, eps_c)
  T v, d[4];
};

template <typename T>
__device__ __forceinline__ D4<T> dc(T v) {
  D4<T> r;
  r.v = v;
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = (T)0;
  return r;
}
template <typename T>
__device__ __forceinline__ D4<T> dv(T v, int j) {
  D4<T> r = dc<T>(v);
  r.d[j] = (T)1;
  return r;
}
template <typename T>
__device__ __forceinline__ D4<T> operator+(D4<T> a, D4<T> b) {
#pragma unroll
  for (int j = 0; j < 4; ++j) a.d[j] += b.d[j];
  a.v += b.v;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator-(D4<T> a, D4<T> b) {
#pragma unroll
  for (int j = 0; j < 4; ++j) a.d[j] -= b.d[j];
  a.v -= b.v;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator*(D4<T> a, D4<T> b) {
  D4<T> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = a.d[j] * b.v + a.v * b.d[j];
  return r;
}
template <typename T>
__device__ __forceinline__ D4<T> operator/(D4<T> a, D4<T> b) {
  D4<T> r;
  r.v = a.v / b.v;
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) / b.v;
  return r;
}
template <typename T>
__device__ __forceinline__ D4<T> operator*(T s, D4<T> a) {
  a.v *= s;
#pragma unroll
  for (int j = 0; j < 4; ++j) a.d[j] *= s;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator*(D4<T> a, T s) {
  return s * a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator+(T s, D4<T> a) {
  a.v += s;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator+(D4<T> a, T s) {
  a.v += s;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator-(T s, D4<T> a) {
  D4<T> r;
  r.v = s - a.v;
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = -a.d[j];
  return r;
}
template <typename T>
__device__ __forceinline__ D4<T> operator-(D4<T> a, T s) {
  a.v -= s;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator/(D4<T> a, T s) {
  a.v /= s;
#pragma unroll
  for (int j = 0; j < 4; ++j) a.d[j] /= s;
  return a;
}
template <typename T>
__device__ __forceinline__ D4<T> operator/(T s, D4<T> a) {
  return dc<T>(s) / a;
}

// ------------------------------------------ one interface for T and D4<T>

// constants of a number type (class-template members: inline by definition)
template <typename N>
struct Num;
template <>
struct Num<float> {
  static __device__ __forceinline__ float c(float x) { return x; }
};
template <>
struct Num<double> {
  static __device__ __forceinline__ double c(double x) { return x; }
};
template <typename T>
struct Num<D4<T>> {
  static __device__ __forceinline__ D4<T> c(T x) { return dc<T>(x); }
};

template <typename T>
__device__ __forceinline__ T val(T x) {
  return x;
}
template <typename T>
__device__ __forceinline__ T val(D4<T> x) {
  return x.v;
}

template <typename T>
__device__ __forceinline__ T nsqrt(T x) {
  return t_sqrt<T>(x);
}
template <typename T>
__device__ __forceinline__ D4<T> nsqrt(D4<T> a) {
  D4<T> r;
  r.v = t_sqrt<T>(a.v);
  T k = r.v > (T)0 ? (T)0.5 / r.v : (T)0;
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = k * a.d[j];
  return r;
}
template <typename T>
__device__ __forceinline__ T nexp(T x) {
  return Closure<T>::exp_(x);
}
template <typename T>
__device__ __forceinline__ D4<T> nexp(D4<T> a) {
  D4<T> r;
  r.v = Closure<T>::exp_(a.v);
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = r.v * a.d[j];
  return r;
}
template <typename T>
__device__ __forceinline__ T nlog(T x) {
  return Closure<T>::logn(x);
}
template <typename T>
__device__ __forceinline__ D4<T> nlog(D4<T> a) {
  D4<T> r;
  r.v = Closure<T>::logn(a.v);
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = a.d[j] / a.v;
  return r;
}
template <typename T>
__device__ __forceinline__ T nlog10(T x) {
  return Closure<T>::log10_(x);
}
template <typename T>
__device__ __forceinline__ D4<T> nlog10(D4<T> a) {
  D4<T> r;
  r.v = Closure<T>::log10_(a.v);
  const T k = (T)0.43429448190325182765 / a.v;  // 1 / (a ln 10)
#pragma unroll
  for (int j = 0; j < 4; ++j) r.d[j] = k * a.d[j];
  return r;
}

// ---------------------------------------------------------------- closures

// fluid properties in the precision of the closure
template <typename T>
__device__ __forceinline__ T fp_rho(const ForceParams& fp);
template <>
__device__ __forceinline__ double fp_rho<double>(const ForceParams& fp) { return fp.rho; }
template <>
__device__ __forceinline__ float fp_rho<float>(const ForceParams& fp) { return fp.rho32; }
template <typename T>
__device__ __forceinline__ T fp_mu(const ForceParams& fp);
template <>
__device__ __forceinline__ double fp_mu<double>(const ForceParams& fp) { return fp.mu; }
template <>
__device__ __forceinline__ float fp_mu<float>(const ForceParams& fp) { return fp.mu32; }

// f_D = drag_coef(...) U for |U| = speed > 0; ec the clamped eps.
template <typename N, typename T>
__device__ __forceinline__ N drag_coef(const ForceParams& fp, N speed, N ec, T rp) {
  const T rho = fp_rho<T>(fp), mu = fp_mu<T>(fp), dp = (T)2 * rp;
  const N Re = (rho * dp / mu) * (ec * speed);
  const int model = fp.drag_model;
  N coef;
  if (model <= 2) {
    N a = (T)0.63 * nsqrt(speed) + (T)4.8 * nsqrt(mu / ((rho * dp) * ec));
    N cds = a * a;  // C_D |U| of Dallavalle
    if (model != 1) {
      const N re = val(Re) > Closure<T>::tiny() ? Re : Num<N>::c(Closure<T>::tiny());
      const N tt = (T)1.5 - nlog10(re);
      const N g = nexp((T)(-0.5) * (tt * tt));
      // 2 - chi written out so that its terms are rounded once (no 3.7 or
      // 2.65 (eps + 1) formed first and then subtracted from 2)
      const N two_minus_ex =
          model == 0 ? (T)0.65 * g - (T)1.7
                     : ((T)5.3 - (T)3.5 * ec) * (ec * ec) * g - ((T)2.65 * ec + (T)0.65);
      cds = cds * nexp(two_minus_ex * nlog(ec));
    }
    coef = ((T)0.5 * rho * (T)kPi * rp * rp) * cds;
  } else {
    const N ep = (T)1 - ec;
    const T Vp = (T)(4.0 / 3.0 * kPi) * rp * rp * rp;
    const N e2 = ec * ec;
    if (model == 3) {  // Koch-Hill
      N F0;
      if (val(ep) >= (T)0.4) {
        F0 = (T)10 * ep / (e2 * ec);
      } else {
        const N plogp = val(ep) > (T)0 ? ep * nlog(ep) : Num<N>::c((T)0);
        const N num = (T)1 + (T)3 * nsqrt((T)0.5 * ep) + (T)(135.0 / 64.0) * plogp +
                      (T)16.14 * ep;
        const N den = (T)1 + ep * ((T)0.681 + ep * ((T)8.14 * ep - (T)8.48));
        F0 = num / den;
      }
      const N F3 = (T)0.0673 + (T)0.212 * ep + (T)0.0232 / (e2 * e2 * ec);
      coef = ((T)18 * mu * Vp / (dp * dp)) * (e2 * (F0 + (T)0.5 * F3 * Re));
    } else if (model == 4) {  // Gidaspow
      if (val(ec) < (T)0.8) {
        coef = Vp * (((T)150 * mu / (dp * dp)) * (ep / ec) + ((T)1.75 * rho / dp) * speed);
      } else {
        // C_D eps |U| of Schiller-Naumann
        const N cdu = val(Re) < (T)1000
                          ? ((T)24 * mu / (rho * dp)) * ((T)1 + (T)0.15 * nexp((T)0.687 * nlog(Re)))
                          : (T)0.44 * (ec * speed);
        coef = ((T)0.75 * rho * Vp / dp) * (cdu * nexp((T)(-2.65) * nlog(ec)));
      }
    } else {  // Beetstra
      N F = (T)10 * ep / e2 + e2 * ((T)1 + (T)1.5 * nsqrt(ep));
      if (val(Re) > (T)0) {
        const N lre = nlog(Re);
        const N s = (T)0.5 + (T)2 * ep;
        const N rs = nexp(s * lre);
        const N num = Re / ec + (T)3 * (ep * ec) * Re + (T)8.4 * nexp((T)0.657 * lre);
        const N den = rs + nexp((T)2.30258509299404568402 * ((T)3 * ep));  // 10^(3 eps_p)
        F = F + ((T)(0.413 / 24.0) / e2) * (num * rs / den);
      }
      coef = ((T)3 * (T)kPi * mu * dp) * (ec * F);
    }
  }
  if (fp.beta_over_eps) coef = coef / ec;
  return coef;
}

}  // namespace cfdem
