// adjoint.cu -- gradients of a loss of the coupling step's outputs with
// respect to the particle positions x and the nodal fluid velocities u.
//
// The coupling step maps (x, u) to the forces f (and their drag part f_D)
// and to the projected void fraction eps_h.  Given the gradients of a loss J
// with respect to those outputs (g_f, g_fD per particle, g_eps per node),
// reverse-mode differentiation through the steps of the method gives:
//
//  forces (Sec. 2.3.2): f_D depends on the slip U = u_f(x) - u_p and on the
//    clamped void fraction eps_c(x) at the particle; f_gradp = -V_p grad
//    p(x).  With a_U = (df_D/dU)^T (g_f + g_fD) and a_eps = (df_D/deps_c)^T
//    (g_f + g_fD) (zero where the clamp is active):
//      dJ/du_j    += phi_j(x) a_U                      (scatter to nodes)
//      dJ/deps_h,j += phi_j(x) a_eps                   (scatter to nodes)
//      dJ/dx      += (grad u_f)^T a_U + a_eps grad eps - V_p H_p g_f
//    with H_p the Hessian of the interpolated pressure.  The optional shear
//    force -V_p mu (lap u + grad div u / 3) is linear in the nodal velocities
//    (its weights, second derivatives of the basis, go to dJ/du) and adds
//    third derivatives of the interpolant to dJ/dx.  The 3 x 4 Jacobian
//    of f_D is taken by forward differentiation of the closure on dual
//    numbers carrying four derivatives.
//  projection: eps_h = A^-1 b(eps_q) with A = M + L^2 K symmetric, so the
//    adjoint is lambda = A^-1 dJ/deps_h and dJ/deps_q = w_q |J_e| lambda_h(x_q)
//    (the transpose of the right-hand side's quadrature).
//  quadrature-centred void fraction: eps_q = 1 - sum_i V(R, r_i, d_iq) / V_R
//    with d_iq = |x_i - x_q|.  The lens volume decreases at the rate of the
//    area of the circle in which the two spheres meet, dV/dd = -pi a^2 with
//    a^2 = (4 d^2 R^2 - (d^2 - r^2 + R^2)^2) / (4 d^2) for |R - r| < d <
//    R + r (zero outside: full containment or no contact), so
//      dJ/dx_i += sum_q dJ/deps_q (pi a^2 / V_R) (x_i - x_q) / d_iq.
//    One thread per particle gathers over the Gauss points within R + r_i,
//    in a fixed order, so this part needs no atomics.
// The particle-centroid scheme is piecewise constant in x: it adds nothing.
#include <cstdint>

#include "device_common.cuh"
#include "drag.cuh"
#include "internal.h"

namespace cfdem {
namespace {

// the drag closure of the forward kernel on dual numbers: fd[c] = coef U_c,
// derivatives along (U_0, U_1, U_2, eps_c); eps_c is a constant where the
// clamp is active
template <typename T>
__device__ __forceinline__ void drag_dual(const ForceParams& fp, T rp, T U0v, T U1v, T U2v,
                                          T epscv, bool clamped, D4<T> fd[3]) {
  D4<T> U[3] = {dv<T>(U0v, 0), dv<T>(U1v, 1), dv<T>(U2v, 2)};
  D4<T> ec = clamped ? dc<T>(epscv) : dv<T>(epscv, 3);
  D4<T> speed = nsqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
  if (!(speed.v > (T)0)) {
#pragma unroll
    for (int c = 0; c < 3; ++c) fd[c] = dc<T>((T)0);
    return;
  }
  const D4<T> coef = drag_coef<D4<T>, T>(fp, speed, ec, rp);
#pragma unroll
  for (int c = 0; c < 3; ++c) fd[c] = coef * U[c];
}

// ------------------------------------------------------------ kernels

// Per particle: the force part of the adjoint.  Writes dJ/dx (direct part),
// adds phi_j a_U to dJ/du_j and phi_j a_eps to geps_j.
template <int K, int KP, typename T>
__global__ void __launch_bounds__(128)
k_adj_forces(MeshDev m, Tables tb, ForceParams fp, int64_t n, const double* __restrict__ x,
             const double* __restrict__ r, const double* __restrict__ u_p,
             const double* __restrict__ u_nodal, const double* __restrict__ p_nodal,
             const double* __restrict__ eps_nodal, const double* __restrict__ gf,
             const double* __restrict__ gfd, double* __restrict__ dJdx, double* __restrict__ dJdu,
             double* __restrict__ geps, DevStatus* st) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  if (!(in_box(p[0], m.x0[0], m.L[0]) && in_box(p[1], m.x0[1], m.L[1]) &&
        in_box(p[2], m.x0[2], m.L[2]))) {
    report_bad(st, i);
    dJdx[3 * i] = dJdx[3 * i + 1] = dJdx[3 * i + 2] = 0.0;
    return;
  }
  int ie[3];
  double xid[3];
  for (int a = 0; a < 3; ++a)
    ie[a] = elem_axis_fast(p[a], m.x0[a], m.h[a], fp.inv_h[a], m.ne[a], &xid[a]);
  const double ih[3] = {fp.inv_h[0], fp.inv_h[1], fp.inv_h[2]};

  // u_f, eps and their gradients (Q_k, FP64)
  double lx[K + 1], ly[K + 1], lz[K + 1], dlx[K + 1], dly[K + 1], dlz[K + 1];
  lagrange<K, double>(tb.z, tb.lw, xid[0], lx, dlx);
  lagrange<K, double>(tb.z, tb.lw, xid[1], ly, dly);
  lagrange<K, double>(tb.z, tb.lw, xid[2], lz, dlz);
  int64_t nx = m.nn[0], nxy = (int64_t)m.nn[0] * m.nn[1];
  int64_t base = (int64_t)ie[0] * K + nx * ((int64_t)ie[1] * K) + nxy * ((int64_t)ie[2] * K);
  double uf[3] = {0, 0, 0}, gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double eps = 0, ge[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c <= K; ++c)
#pragma unroll
    for (int b = 0; b <= K; ++b)
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        double phi = lx[a] * ly[b] * lz[c];
        double dphi[3] = {dlx[a] * ly[b] * lz[c] * ih[0], lx[a] * dly[b] * lz[c] * ih[1],
                          lx[a] * ly[b] * dlz[c] * ih[2]};
        int64_t nd = base + a + nx * b + nxy * c;
        double e = __ldg(eps_nodal + nd);
        eps += phi * e;
#pragma unroll
        for (int k = 0; k < 3; ++k) ge[k] += dphi[k] * e;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          double u = __ldg(u_nodal + 3 * nd + comp);
          uf[comp] += phi * u;
#pragma unroll
          for (int k = 0; k < 3; ++k) gu[comp][k] += dphi[k] * u;
        }
      }

  // Hessian of the interpolated pressure (Q_kp, FP64)
  double px[KP + 1], py[KP + 1], pz[KP + 1], dpx[KP + 1], dpy[KP + 1], dpz[KP + 1];
  double ddpx[KP + 1], ddpy[KP + 1], ddpz[KP + 1];
  lagrange_d3<KP, double>(tb.zp, tb.lwp, xid[0], px, dpx, ddpx, (double*)nullptr);
  lagrange_d3<KP, double>(tb.zp, tb.lwp, xid[1], py, dpy, ddpy, (double*)nullptr);
  lagrange_d3<KP, double>(tb.zp, tb.lwp, xid[2], pz, dpz, ddpz, (double*)nullptr);
  int64_t pnx = m.np[0], pnxy = (int64_t)m.np[0] * m.np[1];
  int64_t pbase =
      (int64_t)ie[0] * KP + pnx * ((int64_t)ie[1] * KP) + pnxy * ((int64_t)ie[2] * KP);
  double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int c = 0; c <= KP; ++c)
#pragma unroll
    for (int b = 0; b <= KP; ++b)
#pragma unroll
      for (int a = 0; a <= KP; ++a) {
        double pv = __ldg(p_nodal + pbase + a + pnx * b + pnxy * c);
        H[0][0] += ddpx[a] * py[b] * pz[c] * pv;
        H[1][1] += px[a] * ddpy[b] * pz[c] * pv;
        H[2][2] += px[a] * py[b] * ddpz[c] * pv;
        H[0][1] += dpx[a] * dpy[b] * pz[c] * pv;
        H[0][2] += dpx[a] * py[b] * dpz[c] * pv;
        H[1][2] += px[a] * dpy[b] * dpz[c] * pv;
      }
  H[0][0] *= ih[0] * ih[0];
  H[1][1] *= ih[1] * ih[1];
  H[2][2] *= ih[2] * ih[2];
  H[0][1] *= ih[0] * ih[1];
  H[0][2] *= ih[0] * ih[2];
  H[1][2] *= ih[1] * ih[2];
  H[1][0] = H[0][1];
  H[2][0] = H[0][2];
  H[2][1] = H[1][2];

  // closure Jacobian
  T rp = (T)r[i];
  T U0 = (T)(uf[0] - u_p[3 * i]), U1 = (T)(uf[1] - u_p[3 * i + 1]),
    U2 = (T)(uf[2] - u_p[3 * i + 2]);
  T ev = (T)eps;
  bool clamped = ev < (T)fp.eps_floor || ev > (T)1;
  T epsc = ev < (T)fp.eps_floor ? (T)fp.eps_floor : (ev > (T)1 ? (T)1 : ev);
  D4<T> fd[3];
  drag_dual<T>(fp, rp, U0, U1, U2, epsc, clamped, fd);
  double g_f[3] = {0, 0, 0}, g_d[3];
  if (gf)
    for (int c = 0; c < 3; ++c) g_f[c] = gf[3 * i + c];
  for (int c = 0; c < 3; ++c) g_d[c] = g_f[c] + (gfd ? gfd[3 * i + c] : 0.0);
  double aU[3], aE = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    aU[j] = g_d[0] * (double)fd[0].d[j] + g_d[1] * (double)fd[1].d[j] +
            g_d[2] * (double)fd[2].d[j];
  aE = g_d[0] * (double)fd[0].d[3] + g_d[1] * (double)fd[1].d[3] + g_d[2] * (double)fd[2].d[3];

  // direct gradient with respect to x_i
  const double Vp = 4.0 / 3.0 * kPi * r[i] * r[i] * r[i];
  // shear force f_s,a = c0 (lap u_a + d_a div u / 3), c0 = -V_p mu: linear in
  // the nodal velocities; its x-derivative takes third derivatives of the basis
  const bool shear = fp.shear && gf;
  const double c0 = -Vp * fp.mu;
  double sb[3][K + 1], s1[3][K + 1], s2[3][K + 1], s3[3][K + 1];
  double gs[3] = {0, 0, 0};
  if (shear) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
      lagrange_d3<K, double>(tb.z, tb.lw, xid[ax], sb[ax], s1[ax], s2[ax], s3[ax]);
#pragma unroll
    for (int c = 0; c <= K; ++c)
#pragma unroll
      for (int b = 0; b <= K; ++b)
#pragma unroll
        for (int a = 0; a <= K; ++a) {
          const int id[3] = {a, b, c};
          // D3(p, q, w): d_p d_q d_w of the node's basis function
          auto D3 = [&](int pp, int qq, int ww) {
            double v = 1.0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              const int o = (pp == ax) + (qq == ax) + (ww == ax);
              const double bv = o == 0 ? sb[ax][id[ax]]
                              : o == 1 ? s1[ax][id[ax]] * ih[ax]
                              : o == 2 ? s2[ax][id[ax]] * ih[ax] * ih[ax]
                                       : s3[ax][id[ax]] * ih[ax] * ih[ax] * ih[ax];
              v *= bv;
            }
            return v;
          };
          const int64_t nd = base + a + nx * b + nxy * c;
          const double u[3] = {__ldg(u_nodal + 3 * nd), __ldg(u_nodal + 3 * nd + 1),
                               __ldg(u_nodal + 3 * nd + 2)};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double lapk = D3(k, 0, 0) + D3(k, 1, 1) + D3(k, 2, 2);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
              const double m3 = g_f[0] * D3(k, 0, cc) + g_f[1] * D3(k, 1, cc) +
                                g_f[2] * D3(k, 2, cc);
              gs[k] += u[cc] * (g_f[cc] * lapk + m3 / 3.0);
            }
          }
        }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double g = aE * ge[k] + c0 * gs[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) g += aU[c] * gu[c][k] - Vp * g_f[c] * H[c][k];
    dJdx[3 * i + k] = g;
  }
  // scatter to the nodes
#pragma unroll
  for (int c = 0; c <= K; ++c)
#pragma unroll
    for (int b = 0; b <= K; ++b)
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        double phi = lx[a] * ly[b] * lz[c];
        int64_t nd = base + a + nx * b + nxy * c;
        if (aE != 0.0) atomicAdd(geps + nd, phi * aE);
        if (dJdu) {
          double add[3] = {phi * aU[0], phi * aU[1], phi * aU[2]};
          if (shear) {  // c0 (g_c lap phi + sum_a g_a d_a d_c phi / 3)
            const int id[3] = {a, b, c};
            double D2[3][3];
#pragma unroll
            for (int pp = 0; pp < 3; ++pp)
#pragma unroll
              for (int qq = 0; qq < 3; ++qq) {
                double v = 1.0;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                  const int o = (pp == ax) + (qq == ax);
                  v *= o == 0 ? sb[ax][id[ax]]
                     : o == 1 ? s1[ax][id[ax]] * ih[ax] : s2[ax][id[ax]] * ih[ax] * ih[ax];
                }
                D2[pp][qq] = v;
              }
            const double lap = D2[0][0] + D2[1][1] + D2[2][2];
#pragma unroll
            for (int comp = 0; comp < 3; ++comp)
              add[comp] += c0 * (g_f[comp] * lap + (g_f[0] * D2[0][comp] + g_f[1] * D2[1][comp] +
                                                    g_f[2] * D2[2][comp]) / 3.0);
          }
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) atomicAdd(dJdu + 3 * nd + comp, add[comp]);
        }
      }
}

// g_q = w_q |J_e| lambda_h(x_q) for every Gauss point: the transpose of the
// right-hand side's quadrature, sum-factorised (three contractions of
// (k+1)^4 per element instead of (k+1)^6).  One thread per element.
template <int K>
__global__ void __launch_bounds__(128)
k_adj_interp_q(MeshDev m, Tables tb, const double* __restrict__ lam, double* __restrict__ gq) {
  constexpr int N = K + 1, Q = N * N * N;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const int e32 = (int)e, exy = m.ne[0] * m.ne[1];  // E < 2^31
  int ez = e32 / exy;
  int ey = (e32 - ez * exy) / m.ne[0];
  int ex = e32 - ez * exy - ey * m.ne[0];
  int64_t nx = m.nn[0], nxy = (int64_t)m.nn[0] * m.nn[1];
  int64_t base = (int64_t)ex * K + nx * ((int64_t)ey * K) + nxy * ((int64_t)ez * K);
  double u[N][N][N], v[N][N][N];
#pragma unroll
  for (int c = 0; c < N; ++c)
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) u[c][b][a] = __ldg(lam + base + a + nx * b + nxy * c);
  // x: v[c][b][qx] = sum_a Bw[a][qx] u[c][b][a]
#pragma unroll
  for (int c = 0; c < N; ++c)
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int q = 0; q < N; ++q) {
        double t = 0.0;
#pragma unroll
        for (int a = 0; a < N; ++a) t += tb.Bw[a][q] * u[c][b][a];
        v[c][b][q] = t;
      }
  // y: u[c][qy][qx] = sum_b Bw[b][qy] v[c][b][qx]
#pragma unroll
  for (int c = 0; c < N; ++c)
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < N; ++b) t += tb.Bw[b][q] * v[c][b][qx];
        u[c][q][qx] = t;
      }
  // z: g[qz][qy][qx] = |J| sum_c Bw[c][qz] u[c][qy][qx]
  double* g = gq + e * Q;
#pragma unroll
  for (int q = 0; q < N; ++q)
#pragma unroll
    for (int qy = 0; qy < N; ++qy)
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) t += tb.Bw[c][q] * u[c][qy][qx];
        g[qx + N * (qy + N * q)] = t * m.Ve;
      }
}

// Per particle: sum over the Gauss points q within R + r_i of
// g_q (pi a^2 / V_R) (x_i - x_q) / d, added to dJ/dx_i.  The distance to
// every Gauss point in reach is first tested in FP32 (positions relative to
// the first element in reach, per-axis squares, a margin of 1e-4 on the
// squared cutoff); only the pairs that pass are evaluated, in T, from FP64
// differences.  The derivative vanishes at the cutoff, so the margin only
// adds terms that are zero or nearly so.
template <int K, typename T>
__global__ void __launch_bounds__(128)
k_adj_qcm(MeshDev m, Tables tb, double R, int64_t n, const double* __restrict__ x,
          const double* __restrict__ r, const double* __restrict__ gq, double* __restrict__ dJdx) {
  constexpr int NQ = K + 1, Q = NQ * NQ * NQ;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  if (!(in_box(p[0], m.x0[0], m.L[0]) && in_box(p[1], m.x0[1], m.L[1]) &&
        in_box(p[2], m.x0[2], m.L[2])))
    return;
  const double ri = r[i];
  const double cut = R + ri, cut2 = cut * cut;
  const double dm = R - ri, dm2 = dm * dm;
  const float pre2 = (float)(cut2 * (1.0 + 1e-4));
  const T coef = (T)(kPi / (4.0 / 3.0 * kPi * R * R * R));
  const T R2r2 = (T)(R * R - ri * ri), RR4 = (T)(4.0 * R * R);
  int lo[3], hi[3];
  float rel0[3], hf[3], gf[3][NQ];
  for (int a = 0; a < 3; ++a) {
    double tl = (p[a] - cut - m.x0[a]) / m.h[a], th = (p[a] + cut - m.x0[a]) / m.h[a];
    lo[a] = (int)floor(tl);
    hi[a] = (int)floor(th);
    lo[a] = lo[a] < 0 ? 0 : (lo[a] > m.ne[a] - 1 ? m.ne[a] - 1 : lo[a]);
    hi[a] = hi[a] < 0 ? 0 : (hi[a] > m.ne[a] - 1 ? m.ne[a] - 1 : hi[a]);
    // particle relative to the first element in reach (FP32 for the filter)
    rel0[a] = (float)(p[a] - (m.x0[a] + m.h[a] * (double)lo[a]));
    hf[a] = (float)m.h[a];
#pragma unroll
    for (int q = 0; q < NQ; ++q) gf[a][q] = (float)(m.h[a] * tb.g[q]);
  }
  T g0 = 0, g1 = 0, g2 = 0;
  for (int ez = lo[2]; ez <= hi[2]; ++ez) {
    const float rz = rel0[2] - hf[2] * (float)(ez - lo[2]);
    for (int ey = lo[1]; ey <= hi[1]; ++ey) {
      const float ry = rel0[1] - hf[1] * (float)(ey - lo[1]);
      for (int ex = lo[0]; ex <= hi[0]; ++ex) {
        const float rx = rel0[0] - hf[0] * (float)(ex - lo[0]);
        const int64_t e = ex + (int64_t)m.ne[0] * (ey + (int64_t)m.ne[1] * ez);
        float sx[NQ], sy[NQ], sz[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          float u = rx - gf[0][q], v = ry - gf[1][q], w = rz - gf[2][q];
          sx[q] = u * u;
          sy[q] = v * v;
          sz[q] = w * w;
        }
#pragma unroll
        for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
          for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
              if (sx[qx] + sy[qy] + sz[qz] >= pre2) continue;
              double dx = p[0] - (m.x0[0] + m.h[0] * ((double)ex + tb.g[qx]));
              double dy = p[1] - (m.x0[1] + m.h[1] * ((double)ey + tb.g[qy]));
              double dz = p[2] - (m.x0[2] + m.h[2] * ((double)ez + tb.g[qz]));
              double d2 = dx * dx + dy * dy + dz * dz;
              if (d2 >= cut2 || d2 <= dm2) continue;  // no contact, or full containment
              T d2t = (T)d2;
              T w = d2t + R2r2;
              T a2 = (RR4 * d2t - w * w) / ((T)4 * d2t);
              T s = (T)__ldg(gq + e * Q + qx + NQ * (qy + NQ * qz)) * coef * a2 /
                    t_sqrt<T>(d2t);
              g0 += s * (T)dx;
              g1 += s * (T)dy;
              g2 += s * (T)dz;
            }
      }
    }
  }
  dJdx[3 * i] += (double)g0;
  dJdx[3 * i + 1] += (double)g1;
  dJdx[3 * i + 2] += (double)g2;
}

}  // namespace

cudaError_t launch_adj_forces(const MeshDev& m, const Tables& t, int precision,
                              const ForceParams& fp, int64_t n, const double* x, const double* r,
                              const double* u_p, const double* u_nodal, const double* p_nodal,
                              const double* eps_nodal, const double* gf, const double* gfd,
                              double* dJdx, double* dJdu, double* geps, DevStatus* st,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int bs = 128;
  const unsigned nb = (unsigned)((n + bs - 1) / bs);
#define CFDEM_ADJ(K, KP)                                                                    \
  if (m.k == K && m.kp == KP) {                                                             \
    if (precision == 0)                                                                     \
      k_adj_forces<K, KP, double><<<nb, bs, 0, s>>>(m, t, fp, n, x, r, u_p, u_nodal,        \
                                                    p_nodal, eps_nodal, gf, gfd, dJdx, dJdu, \
                                                    geps, st);                              \
    else                                                                                    \
      k_adj_forces<K, KP, float><<<nb, bs, 0, s>>>(m, t, fp, n, x, r, u_p, u_nodal,         \
                                                   p_nodal, eps_nodal, gf, gfd, dJdx, dJdu,  \
                                                   geps, st);                               \
    count_launches(1);                                                                      \
    return cudaGetLastError();                                                              \
  }
  CFDEM_ADJ(1, 1)
  CFDEM_ADJ(2, 1)
  CFDEM_ADJ(2, 2)
  CFDEM_ADJ(3, 1)
  CFDEM_ADJ(3, 2)
  CFDEM_ADJ(3, 3)
  CFDEM_ADJ(1, 2)
  CFDEM_ADJ(1, 3)
  CFDEM_ADJ(2, 3)
#undef CFDEM_ADJ
  return cudaErrorInvalidValue;
}

cudaError_t launch_adj_qcm(const MeshDev& m, const Tables& t, int precision, double R,
                           const double* lam, double* gq, int64_t n, const double* x,
                           const double* r, double* dJdx, cudaStream_t s) {
  const unsigned eb = (unsigned)((m.E + 127) / 128);
  const unsigned pb = (unsigned)((n + 127) / 128);
#define CFDEM_ADJQ(KK)                                                                \
  if (m.k == KK) {                                                                    \
    k_adj_interp_q<KK><<<eb, 128, 0, s>>>(m, t, lam, gq);                             \
    if (n > 0) {                                                                      \
      if (precision == 0)                                                             \
        k_adj_qcm<KK, double><<<pb, 128, 0, s>>>(m, t, R, n, x, r, gq, dJdx);         \
      else                                                                            \
        k_adj_qcm<KK, float><<<pb, 128, 0, s>>>(m, t, R, n, x, r, gq, dJdx);          \
    }                                                                                 \
    count_launches(n > 0 ? 2 : 1);                                                    \
    return cudaGetLastError();                                                        \
  }
  CFDEM_ADJQ(1)
  CFDEM_ADJQ(2)
  CFDEM_ADJQ(3)
#undef CFDEM_ADJQ
  return cudaErrorInvalidValue;
}

}  // namespace cfdem
