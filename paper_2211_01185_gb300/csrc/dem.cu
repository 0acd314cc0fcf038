// dem.cu -- the DEM step of the particles (Sec. 2.2): Newton's laws for
// translation and rotation (Eqs. newton_law, angular_momentum), soft-sphere
// contacts with the non-linear visco-elastic model of Table (viscoelastic)
// and Velocity Verlet integration, sub-cycled inside one CFD step with the
// fluid force f_fp held (Sec. 2.3, f_coupling = dt_CFD / dt_DEM).
//
// Contact model per pair (unit normal n from i to its partner, overlap
// d_n = r_i + r_j - |x_j - x_i|):
//   k_n = 4/3 Y_e sqrt(R_e d_n), k_t = 8 G_e sqrt(R_e d_n),
//   eta_n = -2 sqrt(5/6) beta sqrt(S_n m_e), eta_t = -2 sqrt(5/6) beta sqrt(S_t m_e),
//   S_n = 2 Y_e sqrt(R_e d_n), S_t = 8 G_e sqrt(R_e d_n), beta = ln e / sqrt(ln^2 e + pi^2),
//   f^n = -k_n d_n n - eta_n v_rn, f^t = -k_t d_t - eta_t v_rt,
// with the effective mass, radius and moduli of the table.  The contact
// point of i lies at r_i n; its velocity relative to the partner is
// v_i - v_j + (r_i w_i + r_j w_j) x n.  The tangential displacement d_t is
// carried per contact, turned onto the current tangent plane and advanced
// by v_rt dt; a Coulomb limit mu_s |f^n| caps f^t (d_t reset to match);
// rolling resistance M^r = -mu_r R_e |f^n| w_rel/|w_rel|; M^t = r_i n x f^t.
// The box faces are walls of infinite mass and radius.
//
// GPU layout.  One thread per particle, in cell order.  A cell list (edge
// >= 2 r_max) is rebuilt by counting sort every sub-step; each particle
// gathers its overlapping partners from the 27 cells around it into a list
// sorted by partner index (capacity C per particle), merges it with its
// previous list to carry d_t, and sums its contacts in that order, then the
// six walls, gravity and the fluid force -- so the forces do not depend on
// the order in which the cell list was filled, and no atomics touch a
// force.  Each particle keeps its own copy of a pair's d_t (the partner's is
// its negative), so i and j never write the same word.  The state is FP64;
// the contact arithmetic is FP64 or, on the mixed path, FP32.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include <type_traits>

#include "cfdem.h"
#include "device_common.cuh"
#include "internal.h"

namespace cfdem {
namespace {

constexpr int kDemMaxCap = 64;

struct DemDev {
  double rho, Y, nu, e, mus, mur;       // particles
  double Yw, nuw, ew, musw, murw;       // walls
  double g[3], lo[3], hi[3];
  double rmax;
  int nc[3];                            // cells per axis
  double inv_ce[3];                     // 1 / cell edge
  int cap;                              // contacts per particle
  // host-computed constants: -2 sqrt(5/6) beta(e) for particle pairs and
  // walls, effective Young's and shear moduli of particle-particle and
  // particle-wall contacts
  double c56, c56w, Ye, Ge, Yew, Gew;
};

__device__ __forceinline__ double d_dot(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// one contact's force (added to F) and torque (added to T) on particle i,
// advancing the carried tangential displacement th in place; T = double
// (FP64 path) or float (mixed path: the overlap arrives from an FP64
// difference, the rest of the contact in FP32)
template <typename R>
__device__ void dem_contact(const R* n, R dn, const R* vrel, const R* wrel, R ri, R me, R Re,
                            R Ye, R Ge, R c56, R mus, R mur, R dt, R* th, R* F, R* Tq) {
  const R vn = n[0] * vrel[0] + n[1] * vrel[1] + n[2] * vrel[2];
  R vrn[3], vrt[3];
  for (int a = 0; a < 3; ++a) {
    vrn[a] = vn * n[a];
    vrt[a] = vrel[a] - vrn[a];
  }
  const R sq = t_sqrt<R>(Re * dn);
  const R kn = (R)(4.0 / 3.0) * Ye * sq;
  const R kt = (R)8 * Ge * sq;
  const R Sn = (R)2 * Ye * sq;
  const R St = (R)8 * Ge * sq;
  const R etan = c56 * t_sqrt<R>(Sn * me);
  const R etat = c56 * t_sqrt<R>(St * me);
  const R hn = th[0] * n[0] + th[1] * n[1] + th[2] * n[2];
  for (int a = 0; a < 3; ++a) th[a] = th[a] - hn * n[a] + vrt[a] * dt;
  R fn[3], ft[3];
  for (int a = 0; a < 3; ++a) {
    fn[a] = -(kn * dn) * n[a] - etan * vrn[a];
    ft[a] = -kt * th[a] - etat * vrt[a];
  }
  const R fnm = t_sqrt<R>(fn[0] * fn[0] + fn[1] * fn[1] + fn[2] * fn[2]);
  const R ftm = t_sqrt<R>(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
  if (ftm > mus * fnm) {
    const R sc = mus * fnm / ftm;
    for (int a = 0; a < 3; ++a) {
      ft[a] = ft[a] * sc;
      th[a] = -(ft[a] + etat * vrt[a]) / kt;
    }
  }
  // (r_i n) x f^t
  const R mt[3] = {ri * (n[1] * ft[2] - n[2] * ft[1]), ri * (n[2] * ft[0] - n[0] * ft[2]),
                   ri * (n[0] * ft[1] - n[1] * ft[0])};
  const R wm = t_sqrt<R>(wrel[0] * wrel[0] + wrel[1] * wrel[1] + wrel[2] * wrel[2]);
  for (int a = 0; a < 3; ++a) {
    F[a] += fn[a] + ft[a];
    Tq[a] += mt[a];
    if (wm > (R)0) Tq[a] += -mur * Re * fnm * wrel[a] / wm;
  }
}

__device__ __forceinline__ int cell_axis(double x, double lo, double inv_ce, int nc) {
  int c = (int)floor((x - lo) * inv_ce);
  return c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
}

// The Velocity Verlet updates, with explicit FMAs so that the fused kernel
// below gives the same bits as the two it replaces.
__device__ __forceinline__ void half_kick(double hdt, double a, double& v) { v = fma(hdt, a, v); }

// first half kick and drift
__global__ void k_dem_kick_drift(int64_t n, double dt, double* __restrict__ x,
                                 double* __restrict__ v, double* __restrict__ w,
                                 const double* __restrict__ acc,
                                 const double* __restrict__ alpha) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  double vt = v[t], wt = w[t];
  half_kick(0.5 * dt, acc[t], vt);
  half_kick(0.5 * dt, alpha[t], wt);
  v[t] = vt;
  w[t] = wt;
  x[t] = fma(dt, vt, x[t]);
}

// second half kick
__global__ void k_dem_kick(int64_t n, double dt, double* __restrict__ v, double* __restrict__ w,
                           const double* __restrict__ acc, const double* __restrict__ alpha) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  double vt = v[t], wt = w[t];
  half_kick(0.5 * dt, acc[t], vt);
  half_kick(0.5 * dt, alpha[t], wt);
  v[t] = vt;
  w[t] = wt;
}

// the second half kick of one sub-step and the first half kick and drift of
// the next, in one pass
__global__ void k_dem_kick_kick_drift(int64_t n, double dt, double* __restrict__ x,
                                      double* __restrict__ v, double* __restrict__ w,
                                      const double* __restrict__ acc,
                                      const double* __restrict__ alpha) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const double a = acc[t], al = alpha[t];
  double vt = v[t], wt = w[t];
  half_kick(0.5 * dt, a, vt);
  half_kick(0.5 * dt, al, wt);
  half_kick(0.5 * dt, a, vt);
  half_kick(0.5 * dt, al, wt);
  v[t] = vt;
  w[t] = wt;
  x[t] = fma(dt, vt, x[t]);
}

// cell of every particle and its slot in the cell (counting sort, pass 1);
// a radius above the stated maximum raises the flag
__global__ void k_dem_cell_count(int64_t n, DemDev p, const double* __restrict__ x,
                                 const double* __restrict__ r, int32_t* __restrict__ cell_of,
                                 int32_t* __restrict__ slot, int32_t* __restrict__ count,
                                 int* __restrict__ flags) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cx = cell_axis(x[3 * i], p.lo[0], p.inv_ce[0], p.nc[0]);
  const int cy = cell_axis(x[3 * i + 1], p.lo[1], p.inv_ce[1], p.nc[1]);
  const int cz = cell_axis(x[3 * i + 2], p.lo[2], p.inv_ce[2], p.nc[2]);
  const int c = cx + p.nc[0] * (cy + p.nc[1] * cz);
  cell_of[i] = c;
  slot[i] = atomicAdd(count + c, 1);
  if (!(r[i] <= p.rmax)) atomicOr(flags, 2);
}

// exclusive scan of count[0..nc) into start[0..nc]: tiles of 1024 cells
// (256 threads x 4) are summed, the tile sums scanned by one block, then
// every tile scans itself from its offset
constexpr int kScanTile = 1024;

__device__ __forceinline__ int32_t block_excl_scan256(int32_t v, int32_t* sh, int32_t* total) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t wsum = lane < 8 ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, wsum, o);
      if (lane >= o) wsum += y;
    }
    if (lane < 8) sh[8 + lane] = wsum;
  }
  __syncthreads();
  const int32_t before = wid > 0 ? sh[8 + wid - 1] : 0;
  *total = sh[15];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(256)
k_dem_scan_tiles(int ncells, const int32_t* __restrict__ count, int32_t* __restrict__ tsum) {
  __shared__ int32_t sh[16];
  const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
  int32_t v = 0;
  for (int q = 0; q < 4; ++q) v += base + q < ncells ? count[base + q] : 0;
  int32_t tot;
  block_excl_scan256(v, sh, &tot);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256)
k_dem_scan_sums(int ntiles, int32_t* __restrict__ tsum) {  // in place, exclusive; tsum[ntiles] = total
  __shared__ int32_t sh[16];
  int32_t run = 0;
  for (int b0 = 0; b0 < ntiles; b0 += 256) {
    const int b = b0 + threadIdx.x;
    const int32_t v = b < ntiles ? tsum[b] : 0;
    int32_t tot;
    const int32_t ex = block_excl_scan256(v, sh, &tot);
    if (b < ntiles) tsum[b] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) tsum[ntiles] = run;
}

__global__ void __launch_bounds__(256)
k_dem_scan_final(int ncells, const int32_t* __restrict__ count,
                 const int32_t* __restrict__ tsum, int32_t* __restrict__ start) {
  __shared__ int32_t sh[16];
  const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
  int32_t c[4], v = 0;
  for (int q = 0; q < 4; ++q) {
    c[q] = base + q < ncells ? count[base + q] : 0;
    v += c[q];
  }
  int32_t tot;
  int32_t run = tsum[blockIdx.x] + block_excl_scan256(v, sh, &tot);
  for (int q = 0; q < 4; ++q) {
    if (base + q < ncells) start[base + q] = run;
    run += c[q];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[ncells] = tsum[gridDim.x];
}

// pass 3: the particle's place in cell order, with an FP32 copy of its
// position (offset from the box's low corner) and radius at that place;
// also FP32 copies of its angular velocity and radius by particle index
__global__ void k_dem_cell_scatter(int64_t n, DemDev p, const double* __restrict__ x,
                                   const double* __restrict__ w, const double* __restrict__ r,
                                   const int32_t* __restrict__ cell_of,
                                   const int32_t* __restrict__ slot,
                                   const int32_t* __restrict__ start, int32_t* __restrict__ perm,
                                   float4* __restrict__ xs, float4* __restrict__ wf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t s = start[cell_of[i]] + slot[i];
  const float rf = (float)r[i];
  perm[s] = (int32_t)i;
  xs[s] = make_float4((float)(x[3 * i] - p.lo[0]), (float)(x[3 * i + 1] - p.lo[1]),
                      (float)(x[3 * i + 2] - p.lo[2]), rf);
  wf[i] = make_float4((float)w[3 * i], (float)w[3 * i + 1], (float)w[3 * i + 2], rf);
}

// max |coordinate| of an FP32 position copy
__device__ __forceinline__ float abs_max3(float4 q) {
  return fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z)));
}

// the FP64 contact test of a screened candidate: d2 < (r_i + r_j)^2, and on
// the FP64 path also 0 < |d| < r_i + r_j on the root (the oracle's test)
template <typename R>
__device__ __forceinline__ bool dem_touch(const double* __restrict__ x,
                                          const double* __restrict__ r, int32_t j,
                                          const double* xi, double ri) {
  const double d[3] = {x[3 * j] - xi[0], x[3 * j + 1] - xi[1], x[3 * j + 2] - xi[2]};
  const double d2 = d_dot(d, d);
  const double rs = ri + r[j];
  if (!(d2 < rs * rs)) return false;
  if (std::is_same<R, double>::value) {
    const double dist = sqrt(d2);
    return dist < rs && dist > 0.0;
  }
  return d2 > 0.0;
}

// forces and torques on every particle; tangential displacements advance by
// dt (0 for the first evaluation of a fresh state).  Thread t takes the
// particle at place t of the cell order, so the threads of a warp share
// most of their 27 cells.  The candidates are screened in FP32 on the
// cell-ordered copy: a stored coordinate is within 2^-24 of its magnitude
// of the FP64 offset and the FP32 difference adds 2^-24 |d|, so
// |d_f - d| <= sqrt(3) 2^-24 (M_i + M_j + |d|) (M = largest |coordinate|);
// the screen passes |d_f| < (r_i + r_j)(1 + 2^-18) + 2^-18 (M_i + M_j), a
// bound more than ten times that error plus the rounding of the squares,
// so no pair the FP64 test accepts is screened out.  The screened
// candidates are kept sorted by index and the FP64 test (dem_touch) runs
// on them afterwards, once per candidate, outside the divergent cell walk.
// The contact arithmetic runs in R (double, or float on the mixed path,
// where the overlap is (rs^2 - d^2) / (rs + d) with the difference of
// squares in FP64, so the small overlap keeps its digits, and the carried
// tangential displacements are stored in FP32).
template <typename R>
__global__ void __launch_bounds__(128)
k_dem_forces(int64_t n, DemDev p, double dt, const double* __restrict__ x,
             const double* __restrict__ v, const double* __restrict__ w,
             const double* __restrict__ r, const double* __restrict__ f_ext,
             const int32_t* __restrict__ start, const int32_t* __restrict__ perm,
             const float4* __restrict__ xs, const float4* __restrict__ wf,
             const int32_t* __restrict__ hj_old, const R* __restrict__ ht_old,
             int32_t* __restrict__ hj_new, R* __restrict__ ht_new, double* __restrict__ wh,
             double* __restrict__ acc, double* __restrict__ alpha, int* __restrict__ flags) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the warp's live threads meet again after each divergent loop: without
  // it they stay split into the groups the cell walk left them in, and every
  // later instruction issues once per group
  const unsigned live = __ballot_sync(0xffffffffu, t < n);
  if (t >= n) return;
  const int64_t i = perm[t];
  const int C = p.cap;
  const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  const double ri = r[i];
  const float4 qi = xs[t];
  const float Mi = abs_max3(qi);
  constexpr float kScreen = 3.814697265625e-06f;  // 2^-18
  // screened partners, sorted by index (insertion into a list of at most
  // kDemMaxCap; a full list drops the screened-in pairs the FP64 test
  // rejects before it takes another)
  int32_t cand[kDemMaxCap];
  int nc = 0;
  const int cx = cell_axis(xi[0], p.lo[0], p.inv_ce[0], p.nc[0]);
  const int cy = cell_axis(xi[1], p.lo[1], p.inv_ce[1], p.nc[1]);
  const int cz = cell_axis(xi[2], p.lo[2], p.inv_ce[2], p.nc[2]);
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= p.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= p.nc[1]) continue;
      // the three cells of a row along x are contiguous in cell order
      const int row = p.nc[0] * (y + p.nc[1] * z);
      const int s0 = start[row + (cx > 0 ? cx - 1 : 0)];
      const int s1 = start[row + (cx < p.nc[0] - 1 ? cx + 2 : p.nc[0])];
      for (int s = s0; s < s1; ++s) {
        if (s == t) continue;
        const float4 qj = xs[s];
        const float ex = qj.x - qi.x, ey = qj.y - qi.y, ez = qj.z - qi.z;
        const float M = Mi + abs_max3(qj);
        const float lim = (qi.w + qj.w) * (1.0f + kScreen) + kScreen * M;
        // positions beyond FP32 range (M not finite) skip the screen
        if (!(ex * ex + ey * ey + ez * ez < lim * lim) && M < 3.0e38f) continue;
        const int32_t j = perm[s];
        if (nc == kDemMaxCap) {
          int m = 0;
          for (int q = 0; q < nc; ++q)
            if (dem_touch<R>(x, r, cand[q], xi, ri)) cand[m++] = cand[q];
          nc = m;
          if (nc == kDemMaxCap) {  // 65 contacts: above any capacity
            if (dem_touch<R>(x, r, j, xi, ri)) atomicOr(flags, 1);
            continue;
          }
        }
        int q = nc++;
        while (q > 0 && cand[q - 1] > j) {
          cand[q] = cand[q - 1];
          --q;
        }
        cand[q] = j;
      }
    }
  }
  __syncwarp(live);
  const double mi = p.rho * (4.0 / 3.0 * kPi) * ri * ri * ri;
  const double Ii = 0.4 * mi * ri * ri;
  const R rir = (R)ri, mir = (R)mi;
  const R mcoef = (R)(p.rho * (4.0 / 3.0 * kPi));
  R F[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
  const R wi[3] = {(R)w[3 * i], (R)w[3 * i + 1], (R)w[3 * i + 2]};
  int o = 0;  // cursor in the previous (sorted) list
  int m = 0;  // contacts kept
  for (int c = 0; c < nc; ++c) {
    const int32_t j = cand[c];
    const double d[3] = {x[3 * j] - xi[0], x[3 * j + 1] - xi[1], x[3 * j + 2] - xi[2]};
    const double d2 = d_dot(d, d);
    const double rjd = r[j];
    const double rs = ri + rjd;
    if (!(d2 < rs * rs)) continue;
    R nrm[3], dn;
    if (std::is_same<R, double>::value) {
      const double dist = sqrt(d2);
      if (!(dist < rs && dist > 0.0)) continue;
      for (int a = 0; a < 3; ++a) nrm[a] = (R)(d[a] / dist);
      dn = (R)(rs - dist);
    } else {
      if (!(d2 > 0.0)) continue;
      const R dist = t_sqrt<R>((R)d2);
      const R inv = (R)1 / dist;
      for (int a = 0; a < 3; ++a) nrm[a] = (R)d[a] * inv;
      dn = (R)(rs * rs - d2) / ((R)rs + dist);
    }
    if (m == C) {
      atomicOr(flags, 1);
      continue;
    }
    R rj, wj[3];
    if (std::is_same<R, double>::value) {
      rj = (R)rjd;
      for (int a = 0; a < 3; ++a) wj[a] = (R)w[3 * j + a];
    } else {
      const float4 q = wf[j];
      rj = (R)q.w;
      wj[0] = (R)q.x;
      wj[1] = (R)q.y;
      wj[2] = (R)q.z;
    }
    const R mj = mcoef * rj * rj * rj;
    const R me = (R)1 / ((R)1 / mir + (R)1 / mj);
    const R Re = (R)1 / ((R)1 / rir + (R)1 / rj);
    const R ws[3] = {rir * wi[0] + rj * wj[0], rir * wi[1] + rj * wj[1], rir * wi[2] + rj * wj[2]};
    const R wxn[3] = {ws[1] * nrm[2] - ws[2] * nrm[1], ws[2] * nrm[0] - ws[0] * nrm[2],
                      ws[0] * nrm[1] - ws[1] * nrm[0]};
    R vrel[3], wrel[3];
    for (int a = 0; a < 3; ++a) {
      vrel[a] = (R)(v[3 * i + a] - v[3 * j + a]) + wxn[a];
      wrel[a] = wi[a] - wj[a];
    }
    R th[3] = {0, 0, 0};
    while (o < C && hj_old[i * C + o] >= 0 && hj_old[i * C + o] < j) ++o;
    if (o < C && hj_old[i * C + o] == j)
      for (int a = 0; a < 3; ++a) th[a] = ht_old[(i * C + o) * 3 + a];
    dem_contact<R>(nrm, dn, vrel, wrel, rir, me, Re, (R)p.Ye, (R)p.Ge, (R)p.c56, (R)p.mus,
                   (R)p.mur, (R)dt, th, F, Tq);
    hj_new[i * C + m] = j;
    for (int a = 0; a < 3; ++a) ht_new[(i * C + m) * 3 + a] = th[a];
    ++m;
  }
  for (int c = m; c < C; ++c) hj_new[i * C + c] = -1;
  __syncwarp(live);
  // walls x-, x+, y-, y+, z-, z+
  for (int wl = 0; wl < 6; ++wl) {
    const int ax = wl / 2;
    R nrm[3] = {0, 0, 0};
    double dnd;
    if (wl % 2 == 0) {
      nrm[ax] = (R)-1;
      dnd = ri - (xi[ax] - p.lo[ax]);
    } else {
      nrm[ax] = (R)1;
      dnd = ri - (p.hi[ax] - xi[ax]);
    }
    double* th = wh + (i * 6 + wl) * 3;
    if (!(dnd > 0.0)) {
      th[0] = th[1] = th[2] = 0.0;
      continue;
    }
    const R rw[3] = {rir * wi[0], rir * wi[1], rir * wi[2]};
    const R wxn[3] = {rw[1] * nrm[2] - rw[2] * nrm[1], rw[2] * nrm[0] - rw[0] * nrm[2],
                      rw[0] * nrm[1] - rw[1] * nrm[0]};
    const R vrel[3] = {(R)v[3 * i] + wxn[0], (R)v[3 * i + 1] + wxn[1], (R)v[3 * i + 2] + wxn[2]};
    R t3[3] = {(R)th[0], (R)th[1], (R)th[2]};
    dem_contact<R>(nrm, (R)dnd, vrel, wi, rir, mir, rir, (R)p.Yew, (R)p.Gew, (R)p.c56w,
                   (R)p.musw, (R)p.murw, (R)dt, t3, F, Tq);
    th[0] = t3[0];
    th[1] = t3[1];
    th[2] = t3[2];
  }
  // two FP64 divisions instead of six (each is a chain on the FP64 pipe)
  const double inv_mi = 1.0 / mi, inv_Ii = 1.0 / Ii;
  for (int a = 0; a < 3; ++a) {
    const double fa = (double)F[a] + mi * p.g[a] + (f_ext ? f_ext[3 * i + a] : 0.0);
    acc[3 * i + a] = fa * inv_mi;
    alpha[3 * i + a] = (double)Tq[a] * inv_Ii;
  }
}

}  // namespace
}  // namespace cfdem

using namespace cfdem;

struct cfdem_dem {
  int device = 0;
  cudaStream_t stream = nullptr;
  cfdem_dem_params prm{};
  bool have_prm = false;
  DemDev dd{};
  int64_t n = -1;        // particle count the state belongs to
  int have_acc = 0;
  int cur = 0;           // which history buffer holds the last lists
  int64_t cap_n = 0, cap_cells = 0, cap_h = 0;
  double *acc = nullptr, *alpha = nullptr, *ht[2] = {nullptr, nullptr}, *wh = nullptr;
  int32_t *hj[2] = {nullptr, nullptr};
  int32_t *cell_of = nullptr, *slot = nullptr, *perm = nullptr, *count = nullptr,
          *start = nullptr, *tsum = nullptr;
  float4* xs = nullptr;  // cell-ordered FP32 positions and radii
  float4* wf = nullptr;  // FP32 angular velocities and radii by particle
  int* flags = nullptr;
  std::string err;
};

namespace {

cfdem_status dfail(cfdem_dem_t d, cfdem_status s, const char* fmt, ...) {
  if (d) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    d->err = buf;
  }
  return s;
}

cfdem_status dcuda(cfdem_dem_t d, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return dfail(d, CFDEM_ENOMEM, "%s: out of device memory", where);
  return dfail(d, CFDEM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define DCK(expr, where)                                  \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return dcuda(d, e_, where);    \
  } while (0)

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

void cfdem_dem_params_default(cfdem_dem_params* p) {
  if (!p) return;
  *p = cfdem_dem_params{};
  p->rho_p = 2500.0;
  p->youngs = 1e7;
  p->poisson = 0.3;
  p->restitution = 0.9;
  p->friction = 0.3;
  p->rolling_friction = 0.0;
  p->wall_youngs = 1e7;
  p->wall_poisson = 0.3;
  p->wall_restitution = 0.9;
  p->wall_friction = 0.3;
  p->wall_rolling_friction = 0.0;
  p->g[2] = -9.81;
  p->capacity = 24;
}

cfdem_status cfdem_dem_create(cfdem_dem_t* out, int device, void* stream) {
  if (!out) return CFDEM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return CFDEM_ECUDA;
  cfdem_dem* d = new cfdem_dem();
  d->device = device;
  d->stream = reinterpret_cast<cudaStream_t>(stream);
  DevGuard g(device);
  if (cudaMalloc(&d->flags, sizeof(int)) != cudaSuccess) {
    delete d;
    return CFDEM_ENOMEM;
  }
  if (cudaMemset(d->flags, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(d->flags);
    delete d;
    return CFDEM_ECUDA;
  }
  *out = d;
  return CFDEM_OK;
}

cfdem_status cfdem_dem_destroy(cfdem_dem_t d) {
  if (!d) return CFDEM_OK;
  DevGuard g(d->device);
  if (d->stream) cudaStreamSynchronize(d->stream);
  else cudaDeviceSynchronize();
  void* ps[] = {d->acc, d->alpha, d->ht[0], d->ht[1], d->wh, d->hj[0], d->hj[1], d->cell_of,
                d->slot, d->perm, d->count, d->start, d->tsum, d->flags, d->xs, d->wf};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete d;
  return CFDEM_OK;
}

cfdem_status cfdem_dem_set_params(cfdem_dem_t d, const cfdem_dem_params* p) {
  if (!d || !p) return dfail(d, CFDEM_EINVAL, "null argument");
  const double vals[] = {p->rho_p, p->youngs, p->wall_youngs, p->max_radius};
  for (double v : vals)
    if (!(v > 0.0) || !std::isfinite(v))
      return dfail(d, CFDEM_EINVAL, "rho_p, youngs, wall_youngs and max_radius must be > 0");
  if (!(p->poisson > -1.0 && p->poisson < 0.5) || !(p->wall_poisson > -1.0 && p->wall_poisson < 0.5))
    return dfail(d, CFDEM_EINVAL, "Poisson ratios must lie in (-1, 0.5)");
  if (!(p->restitution > 0.0 && p->restitution <= 1.0) ||
      !(p->wall_restitution > 0.0 && p->wall_restitution <= 1.0))
    return dfail(d, CFDEM_EINVAL, "coefficients of restitution must lie in (0, 1]");
  if (!(p->friction >= 0.0) || !(p->wall_friction >= 0.0) || !(p->rolling_friction >= 0.0) ||
      !(p->wall_rolling_friction >= 0.0))
    return dfail(d, CFDEM_EINVAL, "friction coefficients must be >= 0");
  if (p->precision < 0 || p->precision > 1)
    return dfail(d, CFDEM_EINVAL, "precision must be 0 (FP64) or 1 (mixed)");
  if (p->capacity < 1 || p->capacity > kDemMaxCap)
    return dfail(d, CFDEM_EINVAL, "capacity must be 1..%d", kDemMaxCap);
  for (int a = 0; a < 3; ++a)
    if (!(p->hi[a] > p->lo[a]) || !std::isfinite(p->lo[a]) || !std::isfinite(p->hi[a]))
      return dfail(d, CFDEM_EINVAL, "box: hi must exceed lo on every axis");
  DemDev& q = d->dd;
  q.rho = p->rho_p;
  q.Y = p->youngs;
  q.nu = p->poisson;
  q.e = p->restitution;
  q.mus = p->friction;
  q.mur = p->rolling_friction;
  q.Yw = p->wall_youngs;
  q.nuw = p->wall_poisson;
  q.ew = p->wall_restitution;
  q.musw = p->wall_friction;
  q.murw = p->wall_rolling_friction;
  q.rmax = p->max_radius;
  auto c56 = [](double e) {
    const double le = std::log(e);
    return -2.0 * std::sqrt(5.0 / 6.0) * (le / std::sqrt(le * le + kPi * kPi));
  };
  q.c56 = c56(p->restitution);
  q.c56w = c56(p->wall_restitution);
  const double nu = p->poisson, nuw = p->wall_poisson;
  q.Ye = 1.0 / ((1.0 - nu * nu) / p->youngs + (1.0 - nu * nu) / p->youngs);
  q.Ge = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / p->youngs + 2.0 * (2.0 - nu) * (1.0 + nu) / p->youngs);
  q.Yew = 1.0 / ((1.0 - nu * nu) / p->youngs + (1.0 - nuw * nuw) / p->wall_youngs);
  q.Gew = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / p->youngs +
                 2.0 * (2.0 - nuw) * (1.0 + nuw) / p->wall_youngs);
  int64_t tot = 1;
  for (int a = 0; a < 3; ++a) {
    q.g[a] = p->g[a];
    q.lo[a] = p->lo[a];
    q.hi[a] = p->hi[a];
    double f = std::floor((p->hi[a] - p->lo[a]) / (2.0 * p->max_radius));
    int nc = f < 1.0 ? 1 : (f > 4096.0 ? 4096 : (int)f);
    q.nc[a] = nc;
    q.inv_ce[a] = nc / (p->hi[a] - p->lo[a]);
    tot *= nc;
  }
  if (tot > ((int64_t)1 << 28)) return dfail(d, CFDEM_EINVAL, "too many cells");
  q.cap = p->capacity;
  // the history layout changes with the capacity and the precision (FP32
  // tangential displacements on the mixed path)
  const bool resize = !d->have_prm || d->prm.capacity != p->capacity ||
                      d->prm.precision != p->precision;
  d->prm = *p;
  d->have_prm = true;
  if (resize) d->n = -1;
  d->have_acc = 0;        // accelerations depend on the parameters
  return CFDEM_OK;
}

cfdem_status cfdem_dem_reset(cfdem_dem_t d) {
  if (!d) return CFDEM_EINVAL;
  d->n = -1;
  d->have_acc = 0;
  return CFDEM_OK;
}

cfdem_status cfdem_dem_step(cfdem_dem_t d, int64_t n, double* x, double* v, double* w,
                            const double* r, const double* f_ext, double dt, int nsub) {
  if (!d) return CFDEM_EINVAL;
  if (!d->have_prm) return dfail(d, CFDEM_ESTATE, "cfdem_dem_set_params first");
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!x || !v || !w || !r)))
    return dfail(d, CFDEM_EINVAL, "null input or bad count");
  if (!(dt > 0.0) || nsub < 0) return dfail(d, CFDEM_EINVAL, "dt must be > 0, nsub >= 0");
  if (n == 0 || nsub == 0) return CFDEM_OK;
  DevGuard g(d->device);
  cudaStream_t s = d->stream;
  const int C = d->prm.capacity;
  const int64_t ncells = (int64_t)d->dd.nc[0] * d->dd.nc[1] * d->dd.nc[2];
  if (n != d->n) {  // a new particle set: fresh state
    if (n > d->cap_n || (int64_t)n * C > d->cap_h) {
      void* old[] = {d->acc, d->alpha, d->wh, d->cell_of, d->slot, d->perm,
                     d->hj[0], d->hj[1], d->ht[0], d->ht[1], d->xs, d->wf};
      for (void* q : old)
        if (q) cudaFree(q);
      d->acc = d->alpha = d->wh = d->ht[0] = d->ht[1] = nullptr;
      d->cell_of = d->slot = d->perm = d->hj[0] = d->hj[1] = nullptr;
      d->xs = d->wf = nullptr;
      d->cap_n = d->cap_h = 0;
      const int64_t cap = n + n / 4 + 256;
      DCK(cudaMalloc(&d->acc, sizeof(double) * 3 * cap), "dem arena");
      DCK(cudaMalloc(&d->alpha, sizeof(double) * 3 * cap), "dem arena");
      DCK(cudaMalloc(&d->wh, sizeof(double) * 18 * cap), "dem arena");
      DCK(cudaMalloc(&d->cell_of, sizeof(int32_t) * cap), "dem arena");
      DCK(cudaMalloc(&d->slot, sizeof(int32_t) * cap), "dem arena");
      DCK(cudaMalloc(&d->perm, sizeof(int32_t) * cap), "dem arena");
      DCK(cudaMalloc(&d->xs, sizeof(float4) * cap), "dem arena");
      DCK(cudaMalloc(&d->wf, sizeof(float4) * cap), "dem arena");
      DCK(cudaMalloc(&d->hj[0], sizeof(int32_t) * cap * C), "dem arena");
      DCK(cudaMalloc(&d->hj[1], sizeof(int32_t) * cap * C), "dem arena");
      DCK(cudaMalloc(&d->ht[0], sizeof(double) * 3 * cap * C), "dem arena");
      DCK(cudaMalloc(&d->ht[1], sizeof(double) * 3 * cap * C), "dem arena");
      d->cap_n = cap;
      d->cap_h = cap * C;
    }
    DCK(cudaMemsetAsync(d->hj[0], 0xff, sizeof(int32_t) * n * C, s), "dem reset");
    DCK(cudaMemsetAsync(d->wh, 0, sizeof(double) * 18 * n, s), "dem reset");
    d->cur = 0;
    d->n = n;
    d->have_acc = 0;
  }
  if (ncells + 1 > d->cap_cells) {
    if (d->count) cudaFree(d->count);
    if (d->start) cudaFree(d->start);
    if (d->tsum) cudaFree(d->tsum);
    d->count = d->start = d->tsum = nullptr;
    d->cap_cells = 0;
    DCK(cudaMalloc(&d->count, sizeof(int32_t) * ncells), "dem cells");
    DCK(cudaMalloc(&d->start, sizeof(int32_t) * (ncells + 1)), "dem cells");
    DCK(cudaMalloc(&d->tsum, sizeof(int32_t) * (ncells / kScanTile + 2)), "dem cells");
    d->cap_cells = ncells + 1;
  }
  const unsigned nb = (unsigned)((n + 127) / 128), nb3 = (unsigned)((3 * n + 255) / 256);
  auto forces = [&](double hdt) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(d->count, 0, sizeof(int32_t) * ncells, s);
    if (e != cudaSuccess) return e;
    k_dem_cell_count<<<nb, 128, 0, s>>>(n, d->dd, x, r, d->cell_of, d->slot, d->count,
                                        d->flags);
    const int ntiles = (int)((ncells + kScanTile - 1) / kScanTile);
    k_dem_scan_tiles<<<ntiles, 256, 0, s>>>((int)ncells, d->count, d->tsum);
    k_dem_scan_sums<<<1, 256, 0, s>>>(ntiles, d->tsum);
    k_dem_scan_final<<<ntiles, 256, 0, s>>>((int)ncells, d->count, d->tsum, d->start);
    k_dem_cell_scatter<<<nb, 128, 0, s>>>(n, d->dd, x, w, r, d->cell_of, d->slot, d->start,
                                          d->perm, d->xs, d->wf);
    const int o = d->cur, nw = 1 - d->cur;
    if (d->prm.precision == 1)  // FP32 tangential history in the same buffers
      k_dem_forces<float><<<nb, 128, 0, s>>>(
          n, d->dd, hdt, x, v, w, r, f_ext, d->start, d->perm, d->xs, d->wf, d->hj[o],
          reinterpret_cast<const float*>(d->ht[o]), d->hj[nw],
          reinterpret_cast<float*>(d->ht[nw]), d->wh, d->acc, d->alpha, d->flags);
    else
      k_dem_forces<double><<<nb, 128, 0, s>>>(n, d->dd, hdt, x, v, w, r, f_ext, d->start,
                                              d->perm, d->xs, d->wf, d->hj[o], d->ht[o],
                                              d->hj[nw], d->ht[nw], d->wh, d->acc, d->alpha,
                                              d->flags);
    count_launches(6);
    d->cur = nw;
    return cudaGetLastError();
  };
  if (!d->have_acc) {
    DCK(forces(0.0), "dem forces");
    d->have_acc = 1;
  }
  k_dem_kick_drift<<<nb3, 256, 0, s>>>(n, dt, x, v, w, d->acc, d->alpha);
  count_launches(1);
  DCK(cudaGetLastError(), "dem drift");
  for (int it = 0; it < nsub; ++it) {
    DCK(forces(dt), "dem forces");
    if (it + 1 < nsub)
      k_dem_kick_kick_drift<<<nb3, 256, 0, s>>>(n, dt, x, v, w, d->acc, d->alpha);
    else
      k_dem_kick<<<nb3, 256, 0, s>>>(n, dt, v, w, d->acc, d->alpha);
    count_launches(1);
    DCK(cudaGetLastError(), "dem kick");
  }
  return CFDEM_OK;
}

cfdem_status cfdem_dem_synchronize(cfdem_dem_t d) {
  if (!d) return CFDEM_EINVAL;
  DevGuard g(d->device);
  int h = 0;
  DCK(cudaMemcpyAsync(&h, d->flags, sizeof(int), cudaMemcpyDeviceToHost, d->stream),
      "dem status");
  DCK(cudaStreamSynchronize(d->stream), "dem synchronize");
  if (h) {
    DCK(cudaMemsetAsync(d->flags, 0, sizeof(int), d->stream), "dem status");
    DCK(cudaStreamSynchronize(d->stream), "dem synchronize");
    if (h & 2) return dfail(d, CFDEM_EINVAL, "a particle radius exceeds max_radius");
    return dfail(d, CFDEM_ECAPACITY, "a particle had more contacts than the capacity");
  }
  return CFDEM_OK;
}

const char* cfdem_dem_last_error(cfdem_dem_t d) { return d ? d->err.c_str() : "null handle"; }

}  // extern "C"
