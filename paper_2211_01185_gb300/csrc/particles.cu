// particles.cu -- per-particle kernels of the coupling step:
//   a1 element location (Sec. 2.3: particles are located on the fluid mesh),
//   a2 stable counting sort into bins and the sorted particle copies,
//   a6 particle-fluid forces (Sec. 2.3.2), a7 fluid source (Eqs. fb, fa).
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "device_common.cuh"
#include "drag.cuh"
#include "df64.cuh"

namespace cfdem {

// ----------------------------------------------------------------------------
// a1: locate

__global__ void k_locate(MeshDev m, int64_t n, const double* __restrict__ x,
                         int32_t* __restrict__ elem, double* __restrict__ xi,
                         DevStatus* st) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  bool ok = in_box(p[0], m.x0[0], m.L[0]) && in_box(p[1], m.x0[1], m.L[1]) &&
            in_box(p[2], m.x0[2], m.L[2]);
  if (!ok) {
    report_bad(st, i);
    if (elem) elem[i] = -1;
    if (xi) xi[3 * i] = xi[3 * i + 1] = xi[3 * i + 2] = 0.0;
    return;
  }
  double t[3];
  int ie[3];
  for (int a = 0; a < 3; ++a) ie[a] = elem_axis(p[a], m.x0[a], m.h[a], m.ne[a], &t[a]);
  if (elem) elem[i] = ie[0] + m.ne[0] * (ie[1] + m.ne[1] * ie[2]);
  if (xi) {
    xi[3 * i] = t[0];
    xi[3 * i + 1] = t[1];
    xi[3 * i + 2] = t[2];
  }
}

cudaError_t launch_locate(const MeshDev& m, int64_t n, const double* x, int32_t* elem,
                          double* xi, DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int bs = 256;
  k_locate<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(m, n, x, elem, xi, st);
  count_launches(1);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// a2: counting sort into bins

__global__ void k_bin_count(MeshDev m, BinDev b, int64_t n, const double* __restrict__ x,
                           const double* __restrict__ r, int32_t* __restrict__ bin_of,
                           int32_t* __restrict__ slot, int32_t* __restrict__ count,
                           DevStatus* st) {
  const double* inv_be = b.inv_be;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool valid = i < n;
  int32_t id = -1;
  double ri = 0.0;
  if (valid) {
    double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    // the box test on integer keys, the bin from a double-float split (the
    // FP64 rule near a bin face): no FP64 instruction for most particles
    if (!(in_box_key(p[0], b.box_lo_key[0], b.box_hi_key[0]) &&
          in_box_key(p[1], b.box_lo_key[1], b.box_hi_key[1]) &&
          in_box_key(p[2], b.box_lo_key[2], b.box_hi_key[2])))
      report_bad(st, i);
    int bq[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      bq[a] = b.loc32 ? cell_df(p[a], b.x0_hi[a], b.x0_lo[a], b.inv_be_hi[a], b.inv_be_lo[a],
                                b.nm1f[a], nullptr)
                      : -1;
      if (bq[a] < 0) bq[a] = bin_axis_slow(p[a], m.x0[a], b.be[a], inv_be[a], b.nb[a]);
    }
    const int bx = bq[0], by = bq[1], bz = bq[2];
    id = bx + b.nb[0] * (by + b.nb[1] * bz);
    bin_of[i] = id;
    if (r) ri = r[i];
  }
  // warp-aggregated counting: one atomic per distinct bin of the warp; the
  // slot order inside a bin is fixed afterwards by k_rank_bins
  unsigned peers = __match_any_sync(FULL, id);
  int leader = __ffs(peers) - 1;
  int rank = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(&count[id], __popc(peers));
  base = __shfl_sync(FULL, base, leader);
  if (valid) slot[i] = base + rank;
  // largest radius: reduced over the warp, then the block, one atomic per
  // block (the bits of a non-negative double order like the value)
  if (r) {
    __shared__ unsigned long long wmax[32];
    // r >= 0 (and not NaN) by integer tests on the bits
    unsigned rl, rh;
    double_halves(ri, &rl, &rh);
    const bool nonneg = !(rh >> 31) && (rh < 0x7ff00000u || (rh == 0x7ff00000u && rl == 0u));
    unsigned long long bits = valid && nonneg ? (unsigned long long)__double_as_longlong(ri) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ob = __shfl_xor_sync(FULL, bits, o);
      bits = ob > bits ? ob : bits;
    }
    const int wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) wmax[wid] = bits;
    __syncthreads();
    if (wid == 0) {
      bits = lane < nw ? wmax[lane] : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ob = __shfl_xor_sync(FULL, bits, o);
        bits = ob > bits ? ob : bits;
      }
      if (lane == 0 && bits) atomicMax(&st->rmax_bits, bits);
    }
  }
}

// exclusive scan of count[0..nb) into start[0..nb], start[nb] = total.
// Two passes: per-tile sums, then the per-tile scan with the tile's offset
// summed from the totals before it.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  // sh: kScanThreads / 32 words
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < kScanThreads / 32 ? sh[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) sh[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) sh[kScanThreads / 32] = wi;
  }
  __syncthreads();
  int32_t res = sh[warp] + inc - v;
  *total = sh[kScanThreads / 32];
  __syncthreads();
  return res;
}

__global__ void k_scan_tiles(const int32_t* __restrict__ in, int64_t nb,
                             int32_t* __restrict__ tile_sum) {
  __shared__ int32_t sh[kScanThreads / 32 + 1];
  int64_t base = blockIdx.x * (int64_t)kScanTile;
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t idx = base + j * kScanThreads + threadIdx.x;
    if (idx < nb) s += in[idx];
  }
  int32_t total;
  block_excl_scan(s, sh, &total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// tile_sum holds each tile's total (k_scan_tiles); this tile's offset is
// the sum of the totals before it, added up here by the block (integers:
// the order does not matter), so no separate scan of the totals is launched
__global__ void k_scan_final(const int32_t* __restrict__ in, int64_t nb,
                             const int32_t* __restrict__ tile_sum, int32_t* __restrict__ out) {
  __shared__ int32_t sh[kScanThreads / 32 + 1];
  int32_t before = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) before += tile_sum[t];
  int32_t off;
  block_excl_scan(before, sh, &off);
  int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * (int64_t)kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t idx = base + j;
    v[j] = idx < nb ? in[idx] : 0;
    s += v[j];
  }
  int32_t total;
  int32_t ex = block_excl_scan(s, sh, &total) + off;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t idx = base + j;
    if (idx < nb) out[idx] = ex;
    ex += v[j];
    if (idx == nb - 1) out[nb] = ex;
  }
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ bin_of,
                          const int32_t* __restrict__ slot, const int32_t* __restrict__ start,
                          int32_t* __restrict__ perm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  perm[start[bin_of[i]] + slot[i]] = (int32_t)i;
}

// restore ascending particle id inside every bin (the atomic slots above
// arrive in any order): a particle's place is the number of particles of its
// bin with a smaller index (one thread per particle; the bins are
// small, and the work of a bin is spread over its particles)
__global__ void k_rank_bins(int64_t n, const int32_t* __restrict__ bin_of,
                            const int32_t* __restrict__ start,
                            const int32_t* __restrict__ unsorted, int32_t* __restrict__ perm) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int32_t i = unsorted[t];
  int32_t b = bin_of[i];
  int32_t s0 = start[b], s1 = start[b + 1];
  int32_t rank = 0;
  for (int32_t j = s0; j < s1; ++j) rank += unsorted[j] < i;
  perm[s0 + rank] = i;
}

// sorted copies: xs64[s] = (x, y, z, r); xs32[s] = float-float split of the
// position relative to the mesh origin and of the radius, hi parts in
// [0..3], lo parts in [4..7]
__global__ void k_gather_sorted(MeshDev m, int64_t n, const int32_t* __restrict__ perm,
                                const double* __restrict__ x, const double* __restrict__ r,
                                double* __restrict__ xs64, float* __restrict__ xs32) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  int64_t i = perm[s];
  double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  double ri = r ? r[i] : 0.0;
  P4 d;
  d.x = p[0];
  d.y = p[1];
  d.z = p[2];
  d.w = ri;
  reinterpret_cast<P4*>(xs64)[s] = d;
  // float-float copies from integer splits (no FP64 instruction): position
  // relative to the origin, radius renormalised (hi the nearest float)
  df64 q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double o = m.x0[a];  // the origin as a float pair, split the same way
    q[a] = df_from_double_int(p[a]) - df_from_double_int(o);
  }
  const df64 rs = df_from_double_int(ri);
  const df64 rr = df_renorm(rs.hi, rs.lo);
  float4* o = reinterpret_cast<float4*>(xs32) + 2 * s;
  o[0] = make_float4(q[0].hi, q[1].hi, q[2].hi, rr.hi);
  o[1] = make_float4(q[0].lo, q[1].lo, q[2].lo, rr.lo);
}

cudaError_t launch_bin(const MeshDev& m, const BinDev& b, int64_t n, const double* x,
                       const double* r, int32_t* bin_of, int32_t* slot, int32_t* bin_count,
                       int32_t* bin_start, int32_t* perm, int32_t* scan_tmp, double* xs64,
                       float* xs32, DevStatus* st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * b.nbins, s);
  if (e != cudaSuccess) return e;
  int bs = 256;
  unsigned gp = (unsigned)((n + bs - 1) / bs);
  if (n > 0) k_bin_count<<<gp, bs, 0, s>>>(m, b, n, x, r, bin_of, slot, bin_count, st);
  int ntiles = (int)((b.nbins + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(bin_count, b.nbins, scan_tmp);
  k_scan_final<<<ntiles, kScanThreads, 0, s>>>(bin_count, b.nbins, scan_tmp, bin_start);
  if (n > 0) {
    // the float-float copy written last by k_gather_sorted holds the
    // unsorted permutation in the meantime (8 floats per particle of room)
    int32_t* unsorted = reinterpret_cast<int32_t*>(xs32);
    k_scatter<<<gp, bs, 0, s>>>(n, bin_of, slot, bin_start, unsorted);
    k_rank_bins<<<gp, bs, 0, s>>>(n, bin_of, bin_start, unsorted, perm);
    k_gather_sorted<<<gp, bs, 0, s>>>(m, n, perm, x, r, xs64, xs32);
  }
  count_launches(n > 0 ? 6 : 2);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// a6: forces

// ---- helpers of the mixed (FP32) path: no FP64 instruction per node

// v as FP32 through its integer double-float split
__device__ __forceinline__ float f32_of(double v) {
  const df64 s = df_from_double_int(v);
  return s.hi + s.lo;
}

// a - b in FP32 from the double-float splits of a and b: the high parts of
// two close values subtract exactly, so the difference carries an FP32
// rounding of itself, not of a or b
__device__ __forceinline__ float df_diff(df64 a, df64 b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// element index and local coordinate (as double-float) along axis a on the
// mixed path: t = (x - x0) / h from the double-float split of x (~2^-46
// |x| / h); where t lies within 1e-5 of an element face (or outside the
// mesh) the FP64 rule of elem_axis_fast decides, so the element is the one
// the definition gives
__device__ __forceinline__ int elem_axis_mixed(double x, const MeshDev& m, const ForceParams& fp,
                                               int a, df64* xi) {
  if (fp.loc32) {
    const int i = cell_df(x, fp.x0_hi[a], fp.x0_lo[a], fp.inv_h_hi[a], fp.inv_h_lo[a],
                          fp.nem1f[a], xi);
    if (i >= 0) return i;
  }
  double xd;
  const int i = elem_axis_slow(x, m.x0[a], m.h[a], fp.inv_h[a], m.ne[a], &xd);
  *xi = df_from_double_int(xd);
  return i;
}

// Lagrange basis of degree D at t in double-float (nodes and barycentric
// weights split on the host)
template <int D>
__device__ __forceinline__ void lagrange_df(const Tables& tb, df64 t, df64* l) {
  df64 d[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) d[a] = t - df64(tb.zf[a], tb.z_lo[a]);
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    df64 v(tb.lwf[a], tb.lw_lo[a]);
#pragma unroll
    for (int b = 0; b <= D; ++b)
      if (b != a) v = v * d[b];
    l[a] = v;
  }
}

// FP64 value written from a T
template <typename T>
__device__ __forceinline__ double out_double(T v);
template <>
__device__ __forceinline__ double out_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ double out_double<float>(float v) { return double_from_float_int(v); }

// Shear force -V_p div tau at local coordinates xi of the element whose first
// velocity node is `base` (Sec. 2.3.2), tau the deviatoric stress of Eq.
// (stress): (div tau)_a = mu (lap u_a + d_a (div u) / 3), second derivatives
// of the Q_k interpolant with the chain rule 1/h per axis.  Nodal values are
// taken relative to the element's first node (FP64 differences, or on the
// mixed path differences of double-float splits) so that the FP32 path does
// not carry the mean velocity through the cancelling weights.
template <int K, typename T>
__device__ __forceinline__ void shear_force(const Tables& tb, const ForceParams& fp,
                                            const double* __restrict__ u_nodal, int64_t base,
                                            int64_t nx, int64_t nxy, const T xi[3], T Vp,
                                            T fs[3]) {
  constexpr bool MIX = std::is_same<T, float>::value;
  T l[3][K + 1], d1[3][K + 1], d2[3][K + 1];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if constexpr (MIX)
      lagrange_d3<K, T>(tb.zf, tb.lwf, xi[ax], l[ax], d1[ax], d2[ax], (T*)nullptr);
    else
      lagrange_d3<K, T>(tb.z, tb.lw, xi[ax], l[ax], d1[ax], d2[ax], (T*)nullptr);
  }
  const T ih0 = MIX ? (T)fp.inv_h32[0] : (T)fp.inv_h[0];
  const T ih1 = MIX ? (T)fp.inv_h32[1] : (T)fp.inv_h[1];
  const T ih2 = MIX ? (T)fp.inv_h32[2] : (T)fp.inv_h[2];
  const T sxx = ih0 * ih0, syy = ih1 * ih1, szz = ih2 * ih2;
  const T sxy = ih0 * ih1, sxz = ih0 * ih2, syz = ih1 * ih2;
  T H[3][6];  // per component: xx, yy, zz, xy, xz, yz
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 6; ++q) H[c][q] = (T)0;
  const double u00 = __ldg(u_nodal + 3 * base), u01 = __ldg(u_nodal + 3 * base + 1),
               u02 = __ldg(u_nodal + 3 * base + 2);
  const df64 r0 = df_from_double_int(u00), r1 = df_from_double_int(u01),
             r2 = df_from_double_int(u02);
#pragma unroll
  for (int c = 0; c <= K; ++c)
#pragma unroll
    for (int b = 0; b <= K; ++b)
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        const int64_t nd = base + a + nx * b + nxy * c;
        T du[3];
        if constexpr (MIX) {
          du[0] = df_diff(df_from_double_int(__ldg(u_nodal + 3 * nd)), r0);
          du[1] = df_diff(df_from_double_int(__ldg(u_nodal + 3 * nd + 1)), r1);
          du[2] = df_diff(df_from_double_int(__ldg(u_nodal + 3 * nd + 2)), r2);
        } else {
          du[0] = (T)(__ldg(u_nodal + 3 * nd) - u00);
          du[1] = (T)(__ldg(u_nodal + 3 * nd + 1) - u01);
          du[2] = (T)(__ldg(u_nodal + 3 * nd + 2) - u02);
        }
        const T w[6] = {d2[0][a] * l[1][b] * l[2][c] * sxx, l[0][a] * d2[1][b] * l[2][c] * syy,
                        l[0][a] * l[1][b] * d2[2][c] * szz, d1[0][a] * d1[1][b] * l[2][c] * sxy,
                        d1[0][a] * l[1][b] * d1[2][c] * sxz, l[0][a] * d1[1][b] * d1[2][c] * syz};
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int q = 0; q < 6; ++q) H[cc][q] += w[q] * du[cc];
      }
  const T mu = MIX ? (T)fp.mu32 : (T)fp.mu;
  const T mu3 = mu / (T)3;
  const T gd[3] = {H[0][0] + H[1][3] + H[2][4], H[0][3] + H[1][1] + H[2][5],
                   H[0][4] + H[1][5] + H[2][2]};  // d_a div u
#pragma unroll
  for (int cc = 0; cc < 3; ++cc)
    fs[cc] = -Vp * (mu * (H[cc][0] + H[cc][1] + H[cc][2]) + mu3 * gd[cc]);
}

// Forces on every particle (Sec. 2.3.2): u_f and eps at the particle by Q_k
// interpolation, grad p by Q_kp, the drag closure, buoyancy and the pressure
// gradient force (and the shear force).  With ps.S, each particle's share of
// the fluid source and its element go to the per-particle records that
// launch_source_sum adds per element.
//
// FP64 path (T = double): location, interpolation and closures in FP64.
// Mixed path (T = float): no FP64 instruction per node.  The element is
// located from a double-float split of x (the FP64 rule only within 1e-5 of
// a face); the slip is interpolated in FP32 from the nodal differences
// u_j - u_p,i formed from double-float splits (the weights sum to one, so
// sum_j phi_j (u_j - u_p) = u_f - u_p, and no FP32 rounding of |u| enters a
// small slip component); pressure differences along each axis likewise; the
// closures in FP32.
template <int K, int KP, typename T, bool SHEAR, bool PRE>
__global__ void __launch_bounds__(128)
k_forces(MeshDev m, Tables tb, ForceParams fp, int64_t n, const double* __restrict__ x,
         const double* __restrict__ r, const double* __restrict__ u_p,
         const double* __restrict__ u_nodal, const double* __restrict__ p_nodal,
         const double* __restrict__ eps_nodal, double* __restrict__ f,
         double* __restrict__ f_drag, PartSrc ps, DevStatus* st) {
  constexpr bool MIX = std::is_same<T, float>::value;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  bool inside;
  if constexpr (MIX)
    inside = in_box_key(p[0], fp.box_lo_key[0], fp.box_hi_key[0]) &&
             in_box_key(p[1], fp.box_lo_key[1], fp.box_hi_key[1]) &&
             in_box_key(p[2], fp.box_lo_key[2], fp.box_hi_key[2]);
  else
    inside = in_box(p[0], m.x0[0], m.L[0]) && in_box(p[1], m.x0[1], m.L[1]) &&
             in_box(p[2], m.x0[2], m.L[2]);
  if (!inside) {
    report_bad(st, i);
    for (int a = 0; a < 3; ++a) {
      f[3 * i + a] = 0.0;
      if (f_drag) f_drag[3 * i + a] = 0.0;
    }
    if (ps.S) ps.elem[i] = -1;
    return;
  }
  int ie[3];
  T xi[3];
  df64 xdf[3];  // mixed path: local coordinates as double-float
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if constexpr (MIX) {
      ie[a] = elem_axis_mixed(p[a], m, fp, a, &xdf[a]);
      xi[a] = xdf[a].hi;
    } else {
      double xd;
      ie[a] = elem_axis_fast(p[a], m.x0[a], m.h[a], fp.inv_h[a], m.ne[a], &xd);
      xi[a] = xd;
    }
  }

  // u_f - u_p and eps at the particle: Q_k interpolation
  T lx[K + 1], ly[K + 1], lz[K + 1];
  df64 lxd[K + 1], lyd[K + 1], lzd[K + 1];
  if constexpr (MIX) {
    lagrange_df<K>(tb, xdf[0], lxd);
    lagrange_df<K>(tb, xdf[1], lyd);
    lagrange_df<K>(tb, xdf[2], lzd);
#pragma unroll
    for (int a = 0; a <= K; ++a) {
      lx[a] = lxd[a].hi;
      ly[a] = lyd[a].hi;
      lz[a] = lzd[a].hi;
    }
  } else {
    lagrange<K, T>(tb.z, tb.lw, xi[0], lx, (T*)nullptr);
    lagrange<K, T>(tb.z, tb.lw, xi[1], ly, (T*)nullptr);
    lagrange<K, T>(tb.z, tb.lw, xi[2], lz, (T*)nullptr);
  }
  const double up0 = u_p[3 * i], up1 = u_p[3 * i + 1], up2 = u_p[3 * i + 2];
  T U0 = 0, U1 = 0, U2 = 0, eps = 0;
  const int64_t nx = m.nn[0], nxy = (int64_t)m.nn[0] * m.nn[1];
  const int64_t base =
      (int64_t)ie[0] * K + nx * ((int64_t)ie[1] * K) + nxy * ((int64_t)ie[2] * K);
  // Mixed path.  The slip u_f - u_p is interpolated in double-float (basis,
  // products and sums, then one subtraction of u_p): a slip component that
  // is small against the nodal velocities (a rough field, u_p of either
  // sign) would otherwise keep an FP32 rounding of the nodal values, ~1e-8
  // m/s.  eps is interpolated in FP32 relative to the element's first node
  // (the weights sum to one), so that FP32 rounds only its variation inside
  // the element.
  df64 uf0(0.f, 0.f), uf1(0.f, 0.f), uf2(0.f, 0.f), re(0.f, 0.f);
  DfDotAcc au0, au1, au2;  // the slip sums (compensated, one renormalisation each)
  au0.zero();
  au1.zero();
  au2.zero();
  if constexpr (MIX) re = df_from_double_int(__ldg(eps_nodal + base));
#pragma unroll
  for (int c = 0; c <= K; ++c) {
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      const T lyz = ly[b] * lz[c];
      df64 lyzd;
      if constexpr (MIX) lyzd = lyd[b] * lzd[c];
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        const int64_t nd = base + a + nx * b + nxy * c;
        if constexpr (MIX) {
          const df64 phid = lxd[a] * lyzd;
          df64 v0, v1, v2, ve;
          if constexpr (PRE) {  // split once per node by launch_split_nodal
            const float4 q0 = __ldg(fp.nodal_df + 2 * nd), q1 = __ldg(fp.nodal_df + 2 * nd + 1);
            v0 = df64(q0.x, q0.y);
            v1 = df64(q0.z, q0.w);
            v2 = df64(q1.x, q1.y);
            ve = df64(q1.z, q1.w);
          } else {
            v0 = df_from_double_int(__ldg(u_nodal + 3 * nd));
            v1 = df_from_double_int(__ldg(u_nodal + 3 * nd + 1));
            v2 = df_from_double_int(__ldg(u_nodal + 3 * nd + 2));
            ve = df_from_double_int(__ldg(eps_nodal + nd));
          }
          au0.add(phid, v0);
          au1.add(phid, v1);
          au2.add(phid, v2);
          eps += phid.hi * df_diff(ve, re);
        } else {
          const T phi = lx[a] * lyz;
          U0 += phi * __ldg(u_nodal + 3 * nd);
          U1 += phi * __ldg(u_nodal + 3 * nd + 1);
          U2 += phi * __ldg(u_nodal + 3 * nd + 2);
          eps += phi * __ldg(eps_nodal + nd);
        }
      }
    }
  }
  if constexpr (MIX) {
    uf0 = au0.get();
    uf1 = au1.get();
    uf2 = au2.get();
    const df64 s0 = uf0 - df_from_double_int(up0), s1 = uf1 - df_from_double_int(up1),
               s2 = uf2 - df_from_double_int(up2);
    U0 = s0.hi + s0.lo;
    U1 = s1.hi + s1.lo;
    U2 = s2.hi + s2.lo;
    eps += re.hi + re.lo;
  } else {  // the FP64 path interpolates u_f, then subtracts u_p
    U0 -= up0;
    U1 -= up1;
    U2 -= up2;
  }
  // grad p at the particle: Q_kp.  Each derivative is taken from nodal
  // differences along its own axis (d/dx uses p_abc - p_0bc, and so on),
  // formed in FP64 or from double-float splits: the shape-function
  // derivatives sum to zero only up to rounding in FP32, so a large pressure
  // varying along one axis would otherwise leak into the other two
  // components of the gradient
  T px[KP + 1], py[KP + 1], pz[KP + 1], dpx[KP + 1], dpy[KP + 1], dpz[KP + 1];
  if constexpr (MIX) {
    lagrange<KP, T>(tb.zpf, tb.lwpf, xi[0], px, dpx);
    lagrange<KP, T>(tb.zpf, tb.lwpf, xi[1], py, dpy);
    lagrange<KP, T>(tb.zpf, tb.lwpf, xi[2], pz, dpz);
  } else {
    lagrange<KP, T>(tb.zp, tb.lwp, xi[0], px, dpx);
    lagrange<KP, T>(tb.zp, tb.lwp, xi[1], py, dpy);
    lagrange<KP, T>(tb.zp, tb.lwp, xi[2], pz, dpz);
  }
  const int64_t pnx = m.np[0], pnxy = (int64_t)m.np[0] * m.np[1];
  const int64_t pbase =
      (int64_t)ie[0] * KP + pnx * ((int64_t)ie[1] * KP) + pnxy * ((int64_t)ie[2] * KP);
  using PV = typename std::conditional<MIX, df64, double>::type;
  PV pv[KP + 1][KP + 1][KP + 1];
#pragma unroll
  for (int c = 0; c <= KP; ++c)
#pragma unroll
    for (int b = 0; b <= KP; ++b)
#pragma unroll
      for (int a = 0; a <= KP; ++a) {
        const double v = __ldg(p_nodal + pbase + a + pnx * b + pnxy * c);
        if constexpr (MIX)
          pv[c][b][a] = df_from_double_int(v);
        else
          pv[c][b][a] = v;
      }
  auto pdiff = [](PV u, PV v) -> T {
    if constexpr (MIX)
      return df_diff(u, v);
    else
      return u - v;
  };
  T gp0 = 0, gp1 = 0, gp2 = 0;
#pragma unroll
  for (int c = 0; c <= KP; ++c) {
#pragma unroll
    for (int b = 0; b <= KP; ++b) {
#pragma unroll
      for (int a = 0; a <= KP; ++a) {
        if (a > 0) gp0 += dpx[a] * py[b] * pz[c] * pdiff(pv[c][b][a], pv[c][b][0]);
        if (b > 0) gp1 += px[a] * dpy[b] * pz[c] * pdiff(pv[c][b][a], pv[c][0][a]);
        if (c > 0) gp2 += px[a] * py[b] * dpz[c] * pdiff(pv[c][b][a], pv[0][b][a]);
      }
    }
  }
  if constexpr (MIX) {
    gp0 *= fp.inv_h32[0];
    gp1 *= fp.inv_h32[1];
    gp2 *= fp.inv_h32[2];
  } else {
    gp0 = gp0 / m.h[0];
    gp1 = gp1 / m.h[1];
    gp2 = gp2 / m.h[2];
  }

  // closures
  const T rp = MIX ? (T)f32_of(r[i]) : (T)r[i];
  const T speed = t_sqrt<T>(U0 * U0 + U1 * U1 + U2 * U2);
  const T floor_ = MIX ? (T)fp.eps_floor32 : (T)fp.eps_floor;
  T epsc = eps < floor_ ? floor_ : eps;
  epsc = epsc > (T)1 ? (T)1 : epsc;
  T fd0 = 0, fd1 = 0, fd2 = 0, coef = 0;
  if (speed > (T)0) {
    coef = drag_coef<T, T>(fp, speed, epsc, rp);
    fd0 = coef * U0;
    fd1 = coef * U1;
    fd2 = coef * U2;
  }
  const T Vp = (T)(4.0 / 3.0 * kPi) * rp * rp * rp;
  T fg0 = -Vp * gp0, fg1 = -Vp * gp1, fg2 = -Vp * gp2;
  if constexpr (SHEAR) {  // the shear force joins the pressure term: f and model B's source
    T fs[3];
    shear_force<K, T>(tb, fp, u_nodal, base, nx, nxy, xi, Vp, fs);
    fg0 += fs[0];
    fg1 += fs[1];
    fg2 += fs[2];
  }
  const T rv = (MIX ? (T)fp.rho32 : (T)fp.rho) * Vp;
  const T g0 = MIX ? (T)fp.g32[0] : (T)fp.g[0];
  const T g1 = MIX ? (T)fp.g32[1] : (T)fp.g[1];
  const T g2 = MIX ? (T)fp.g32[2] : (T)fp.g[2];
  f[3 * i] = out_double<T>(fd0 + (-rv * g0) + fg0);
  f[3 * i + 1] = out_double<T>(fd1 + (-rv * g1) + fg1);
  f[3 * i + 2] = out_double<T>(fd2 + (-rv * g2) + fg2);
  if (f_drag) {
    f_drag[3 * i] = out_double<T>(fd0);
    f_drag[3 * i + 1] = out_double<T>(fd1);
    f_drag[3 * i + 2] = out_double<T>(fd2);
  }
  if (ps.S) {
    // the particle's share of the fluid source: its drag (none when the
    // fluid-side drag form carries it through beta_e), plus for model B the
    // pressure (and shear) part; and its drag coefficient
    T s0 = fd0, s1 = fd1, s2 = fd2;
    if (fp.fluid_drag) s0 = s1 = s2 = (T)0;
    if (fp.vans_model == 1) {
      s0 += fg0;
      s1 += fg1;
      s2 += fg2;
    }
    double* o = ps.S + 4 * i;
    o[0] = out_double<T>(s0);
    o[1] = out_double<T>(s1);
    o[2] = out_double<T>(s2);
    o[3] = out_double<T>(coef);
    ps.elem[i] = (int32_t)(ie[0] + (int64_t)m.ne[0] * (ie[1] + (int64_t)m.ne[1] * ie[2]));
    // the largest magnitudes fix the scale of the fixed-point sums (the bits
    // of non-negative doubles order like their values)
    auto mag = [](double v) {
      return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    };
    unsigned long long mx[3] = {max(mag(o[0]), max(mag(o[1]), mag(o[2]))), mag(o[3]),
                                max(mag(up0), max(mag(up1), mag(up2)))};
    // one atomic per warp and class.  Only the exponent field sets the
    // scale, so the high 32 bits (sign, exponent, leading significand bits)
    // are reduced over the lanes still here (a thread past n or outside the
    // mesh has returned) by the warp's max reduction
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int nc = fp.fluid_drag ? 3 : 1;
    for (int c = 0; c < nc; ++c) {
      const unsigned hi = __reduce_max_sync(act, (unsigned)(mx[c] >> 32));
      if (lane == __ffs(act) - 1) atomicMax(ps.maxbits + c, (unsigned long long)hi << 32);
    }
  }
}

__global__ void k_split_nodal(int64_t n_nodes, const double* __restrict__ u_nodal,
                              const double* __restrict__ eps_nodal, float4* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_nodes;
       j += (int64_t)gridDim.x * blockDim.x) {
    const df64 u0 = df_from_double_int(u_nodal[3 * j]);
    const df64 u1 = df_from_double_int(u_nodal[3 * j + 1]);
    const df64 u2 = df_from_double_int(u_nodal[3 * j + 2]);
    const df64 e = df_from_double_int(eps_nodal[j]);
    out[2 * j] = make_float4(u0.hi, u0.lo, u1.hi, u1.lo);
    out[2 * j + 1] = make_float4(u2.hi, u2.lo, e.hi, e.lo);
  }
}

cudaError_t launch_split_nodal(int64_t n_nodes, const double* u_nodal, const double* eps_nodal,
                               float4* out, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  int64_t b = (n_nodes + 255) / 256;
  k_split_nodal<<<(unsigned)(b < 4864 ? b : 4864), 256, 0, s>>>(n_nodes, u_nodal, eps_nodal, out);
  count_launches(1);
  return cudaGetLastError();
}

template <int K, int KP, typename T>
static void launch_forces_t(const MeshDev& m, const Tables& t, const ForceParams& fp,
                            int64_t n, const double* x, const double* r, const double* u_p,
                            const double* u_nodal, const double* p_nodal,
                            const double* eps_nodal, double* f, double* f_drag, PartSrc ps,
                            DevStatus* st, cudaStream_t s) {
  int bs = 128;
  const unsigned nb = (unsigned)((n + bs - 1) / bs);
  // the pre-split nodal values (mixed path, no shear force) are a separate
  // instantiation, so that the per-particle splits keep their registers
  constexpr bool MIX = std::is_same<T, float>::value;
  if (fp.shear)
    k_forces<K, KP, T, true, false><<<nb, bs, 0, s>>>(m, t, fp, n, x, r, u_p, u_nodal, p_nodal,
                                                      eps_nodal, f, f_drag, ps, st);
  else if (MIX && fp.nodal_df)
    k_forces<K, KP, T, false, MIX><<<nb, bs, 0, s>>>(m, t, fp, n, x, r, u_p, u_nodal, p_nodal,
                                                     eps_nodal, f, f_drag, ps, st);
  else
    k_forces<K, KP, T, false, false><<<nb, bs, 0, s>>>(m, t, fp, n, x, r, u_p, u_nodal,
                                                       p_nodal, eps_nodal, f, f_drag, ps, st);
  count_launches(1);
}

cudaError_t launch_forces(const MeshDev& m, const Tables& t, int precision, const ForceParams& fp,
                          int64_t n, const double* x, const double* r, const double* u_p,
                          const double* u_nodal, const double* p_nodal,
                          const double* eps_nodal, double* f, double* f_drag, PartSrc ps,
                          DevStatus* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define CFDEM_FORCES(K, KP)                                                                  \
  if (m.k == K && m.kp == KP) {                                                              \
    if (precision == 0)                                                                      \
      launch_forces_t<K, KP, double>(m, t, fp, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, \
                                     f_drag, ps, st, s);                                     \
    else                                                                                     \
      launch_forces_t<K, KP, float>(m, t, fp, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f,  \
                                    f_drag, ps, st, s);                                      \
    return cudaGetLastError();                                                               \
  }
  CFDEM_FORCES(1, 1)
  CFDEM_FORCES(2, 1)
  CFDEM_FORCES(2, 2)
  CFDEM_FORCES(3, 1)
  CFDEM_FORCES(3, 2)
  CFDEM_FORCES(3, 3)
  CFDEM_FORCES(1, 2)
  CFDEM_FORCES(1, 3)
  CFDEM_FORCES(2, 3)
#undef CFDEM_FORCES
  return cudaErrorInvalidValue;
}

// Per-element sums of the particle records as exact fixed-point sums: each
// value v of a class (source components, drag coefficients, particle
// velocity components) becomes the integer t = round(v 2^E), E = 61 - the
// exponent of the class's largest |v|, so |t| < 2^62 and the rounding is
// below 2^-62 of that largest value; t is split as hi 2^31 + lo (lo in
// [0, 2^31)) and hi, lo are added by 64-bit integer atomics, which cannot
// overflow for fewer than 2^31 particles.  Integer sums do not depend on the
// order of the additions, so the source has the same bits on every run.

// exponent field of the largest value of a class -> the scale exponent E
__device__ __forceinline__ int fixed_scale(unsigned long long maxbits) {
  const int ex = (int)((maxbits >> 52) & 0x7ff);
  return ex == 0 ? 0 : 1084 - ex;  // 61 - (ex - 1023)
}

// round(v 2^E) by integer operations on the bits of v (rounding half away
// from zero); zero and subnormals give 0
__device__ __forceinline__ long long fixed_of(double v, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return 0;
  const long long M = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = ex - 1075 + E;  // v = M 2^(ex - 1075)
  long long t;
  if (sh >= 0)
    t = M << sh;  // sh <= 9 for the largest value: |t| < 2^62
  else if (sh > -63)
    t = (M + (1ll << (-sh - 1))) >> (-sh);
  else
    t = 0;
  return (b >> 63) ? -t : t;
}

__device__ __forceinline__ void fixed_add(long long* acc, double v, int E) {
  const long long t = fixed_of(v, E);
  const long long hi = t >> 31;            // floor(t / 2^31)
  const long long lo = t - (hi << 31);     // in [0, 2^31)
  atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)hi);
  atomicAdd(reinterpret_cast<unsigned long long*>(acc + 1), (unsigned long long)lo);
}

__device__ __forceinline__ double fixed_value(const long long* acc, int E) {
  // 2^-E as two powers of two built from their bits (0 <= E <= 1084, so
  // each half is a normal number): exact scalings instead of ldexp
  const int e1 = E >> 1, e2 = E - e1;
  const double p1 = __longlong_as_double((long long)(1023 - e1) << 52);
  const double q1 = __longlong_as_double((long long)(1023 - e2) << 52);
  return ((double)acc[0] * 2147483648.0 + (double)acc[1]) * p1 * q1;
}

// acc64: per element S (3 x 2 integers); then, with the fluid-side drag, a
// second block of B (2), U (3 x 2), N (1) and a pad per element
constexpr int kSrcS = 6, kSrcSemi = 10;

__global__ void k_source_accumulate(int64_t n, int64_t E, PartSrc ps,
                                    const double* __restrict__ u_p, int semi,
                                    long long* __restrict__ acc64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t e = ps.elem[i];
  if (e < 0) return;
  long long* a = acc64 + (int64_t)e * kSrcS;
  const double* o = ps.S + 4 * i;
  const int E0 = fixed_scale(ps.maxbits[0]);
  fixed_add(a, o[0], E0);
  fixed_add(a + 2, o[1], E0);
  fixed_add(a + 4, o[2], E0);
  if (semi) {
    long long* b = acc64 + E * kSrcS + (int64_t)e * kSrcSemi;
    fixed_add(b, o[3], fixed_scale(ps.maxbits[1]));
    const int E2 = fixed_scale(ps.maxbits[2]);
    fixed_add(b + 2, u_p[3 * i], E2);
    fixed_add(b + 4, u_p[3 * i + 1], E2);
    fixed_add(b + 6, u_p[3 * i + 2], E2);
    atomicAdd(reinterpret_cast<unsigned long long*>(b + 8), 1ull);
  }
}

__global__ void k_source_finalize(int64_t E, PartSrc ps, int semi,
                                  const long long* __restrict__ acc64,
                                  double* __restrict__ S_elem, SemiAcc acc,
                                  double* __restrict__ F_elem, double inv_ve) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const long long* a = acc64 + e * kSrcS;
  const int E0 = fixed_scale(ps.maxbits[0]);
  const double s0 = fixed_value(a, E0), s1 = fixed_value(a + 2, E0), s2 = fixed_value(a + 4, E0);
  S_elem[3 * e] = s0;
  S_elem[3 * e + 1] = s1;
  S_elem[3 * e + 2] = s2;
  if (F_elem) {  // as k_fluid_source: F_e = -S_e / V_e
    F_elem[3 * e] = -s0 * inv_ve;
    F_elem[3 * e + 1] = -s1 * inv_ve;
    F_elem[3 * e + 2] = -s2 * inv_ve;
  }
  if (semi) {
    const long long* b = acc64 + E * kSrcS + e * kSrcSemi;
    acc.B[e] = fixed_value(b, fixed_scale(ps.maxbits[1]));
    const int E2 = fixed_scale(ps.maxbits[2]);
    acc.U[3 * e] = fixed_value(b + 2, E2);
    acc.U[3 * e + 1] = fixed_value(b + 4, E2);
    acc.U[3 * e + 2] = fixed_value(b + 6, E2);
    acc.N[e] = (double)b[8];
  }
}

cudaError_t launch_source_sum(const MeshDev& m, int64_t n, PartSrc ps, const double* u_p,
                              int semi, long long* acc64, double* S_elem, SemiAcc acc,
                              double* F_elem, cudaStream_t s) {
  const int64_t words = m.E * (semi ? kSrcS + kSrcSemi : kSrcS);
  cudaError_t e = cudaMemsetAsync(acc64, 0, sizeof(long long) * words, s);
  if (e != cudaSuccess) return e;
  if (n > 0)
    k_source_accumulate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, m.E, ps, u_p, semi,
                                                                    acc64);
  k_source_finalize<<<(unsigned)((m.E + 255) / 256), 256, 0, s>>>(
      m.E, ps, semi, acc64, S_elem, acc, semi ? nullptr : F_elem, 1.0 / m.Ve);
  count_launches(n > 0 ? 2 : 1);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// a7: fluid source F_e = -S_e / V_e, optionally broadcast to the quadrature
// points

__global__ void k_fluid_source(int64_t E, int Q, double inv_ve, const double* __restrict__ S,
                               double* __restrict__ F_e, double* __restrict__ F_q) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double f0 = -S[3 * e] * inv_ve, f1 = -S[3 * e + 1] * inv_ve, f2 = -S[3 * e + 2] * inv_ve;
  if (F_e) {
    F_e[3 * e] = f0;
    F_e[3 * e + 1] = f1;
    F_e[3 * e + 2] = f2;
  }
  if (F_q) {
    double* o = F_q + 3 * e * (int64_t)Q;
    for (int q = 0; q < Q; ++q) {
      o[3 * q] = f0;
      o[3 * q + 1] = f1;
      o[3 * q + 2] = f2;
    }
  }
}

// wide broadcast for F_q: one thread per (element, quadrature point)
__global__ void k_fluid_source_q(int64_t E, int Q, double inv_ve, const double* __restrict__ S,
                                 double* __restrict__ F_q) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= E * Q * 3) return;
  int64_t e = t / (3 * (int64_t)Q);
  int c = (int)(t % 3);
  F_q[t] = -S[3 * e + c] * inv_ve;
}

cudaError_t launch_fluid_source(const MeshDev& m, const double* S_elem, double* F_elem,
                                double* F_q, cudaStream_t s) {
  int bs = 256;
  double inv_ve = 1.0 / m.Ve;
  if (F_elem)
    k_fluid_source<<<(unsigned)((m.E + bs - 1) / bs), bs, 0, s>>>(m.E, m.Q, inv_ve, S_elem,
                                                                  F_elem, nullptr);
  if (F_q) {
    int64_t tot = m.E * m.Q * 3;
    k_fluid_source_q<<<(unsigned)((tot + bs - 1) / bs), bs, 0, s>>>(m.E, m.Q, inv_ve, S_elem,
                                                                    F_q);
  }
  count_launches((F_elem ? 1 : 0) + (F_q ? 1 : 0));
  return cudaGetLastError();
}

// Fluid source with the fluid-side drag (Sec. 2.3.2: the drag written with
// the fluid velocity at the quadrature point and the cell-mean particle
// velocity), one thread per element:
//   F_q = -beta_e (u_f(x_q) - u_p,avg) - S_e / V_e,  beta_e = B_e / V_e,
// u_f at the Gauss points by sum-factorised interpolation of the nodal
// velocity relative to u_p,avg (so that FP32 does not carry the mean),
// S_e the model-B pressure (and shear) part.  F_e is the Gauss average.
template <int K, typename T>
__global__ void __launch_bounds__(128)
k_fluid_source_semi(MeshDev m, Tables tb, const double* __restrict__ S, SemiAcc acc,
                    const double* __restrict__ u_nodal, double* __restrict__ F_e,
                    double* __restrict__ F_q) {
  constexpr int NQ = K + 1, Q = NQ * NQ * NQ;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const double inv_ve = 1.0 / m.Ve;
  const double cnt = acc.N[e];
  const double beta = acc.B[e] * inv_ve;
  double upa[3] = {0.0, 0.0, 0.0};
  if (cnt > 0.0)
    for (int d = 0; d < 3; ++d) upa[d] = acc.U[3 * e + d] / cnt;
  const int e32 = (int)e, exy = m.ne[0] * m.ne[1];  // E < 2^31
  const int ez = e32 / exy;
  const int ey = (e32 - ez * exy) / m.ne[0];
  const int ex = e32 - ez * exy - ey * m.ne[0];
  const int64_t nx = m.nn[0], nxy = (int64_t)m.nn[0] * m.nn[1];
  const int64_t base = (int64_t)ex * K + nx * ((int64_t)ey * K) + nxy * ((int64_t)ez * K);
  T L[NQ][NQ];  // L[q][a] = l_a(g_q)
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T l[NQ];
    lagrange<K, T>(tb.z, tb.lw, (T)tb.g[q], l, (T*)nullptr);
#pragma unroll
    for (int a = 0; a < NQ; ++a) L[q][a] = l[a];
  }
  const T bt = (T)beta;
  double mean[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    T v[NQ][NQ][NQ];  // [c][b][a]: u_j - u_p,avg
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int a = 0; a < NQ; ++a)
          v[c][b][a] = (T)(__ldg(u_nodal + 3 * (base + a + nx * b + nxy * c) + d) - upa[d]);
    T t1[NQ][NQ][NQ];  // [c][b][qx]
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
          T s = 0;
#pragma unroll
          for (int a = 0; a < NQ; ++a) s += L[qx][a] * v[c][b][a];
          t1[c][b][qx] = s;
        }
    T t2[NQ][NQ][NQ];  // [c][qy][qx]
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
          T s = 0;
#pragma unroll
          for (int b = 0; b < NQ; ++b) s += L[qy][b] * t1[c][b][qx];
          t2[c][qy][qx] = s;
        }
    const double sv = -S[3 * e + d] * inv_ve;
#pragma unroll
    for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
      for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) {
          T s = 0;
#pragma unroll
          for (int c = 0; c < NQ; ++c) s += L[qz][c] * t2[c][qy][qx];
          const double F = (double)(-bt * s) + sv;
          const int q = qx + NQ * (qy + NQ * qz);
          if (F_q) F_q[(e * Q + q) * 3 + d] = F;
          mean[d] += tb.w[qx] * tb.w[qy] * tb.w[qz] * F;
        }
  }
  if (F_e)
    for (int d = 0; d < 3; ++d) F_e[3 * e + d] = mean[d];
}

cudaError_t launch_fluid_source_semi(const MeshDev& m, const Tables& t, int precision,
                                     const double* S_elem, SemiAcc acc, const double* u_nodal,
                                     double* F_elem, double* F_q, cudaStream_t s) {
  if (!F_elem && !F_q) return cudaSuccess;
  const unsigned nb = (unsigned)((m.E + 127) / 128);
#define CFDEM_SEMI(KK)                                                                      \
  if (m.k == KK) {                                                                          \
    if (precision == 0)                                                                     \
      k_fluid_source_semi<KK, double><<<nb, 128, 0, s>>>(m, t, S_elem, acc, u_nodal, F_elem, \
                                                         F_q);                              \
    else                                                                                    \
      k_fluid_source_semi<KK, float><<<nb, 128, 0, s>>>(m, t, S_elem, acc, u_nodal, F_elem,  \
                                                        F_q);                               \
    count_launches(1);                                                                      \
    return cudaGetLastError();                                                              \
  }
  CFDEM_SEMI(1)
  CFDEM_SEMI(2)
  CFDEM_SEMI(3)
#undef CFDEM_SEMI
  return cudaErrorInvalidValue;
}

// beta_e = B_e / V_e and u_p,avg,e = U_e / N_e (0 for an empty element)
__global__ void k_drag_coefficients(int64_t E, double inv_ve, SemiAcc acc,
                                    double* __restrict__ beta_e, double* __restrict__ up_avg) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double cnt = acc.N[e];
  if (beta_e) beta_e[e] = acc.B[e] * inv_ve;
  if (up_avg)
    for (int d = 0; d < 3; ++d) up_avg[3 * e + d] = cnt > 0.0 ? acc.U[3 * e + d] / cnt : 0.0;
}

cudaError_t launch_drag_coefficients(const MeshDev& m, SemiAcc acc, double* beta_e,
                                     double* up_avg, cudaStream_t s) {
  k_drag_coefficients<<<(unsigned)((m.E + 255) / 256), 256, 0, s>>>(m.E, 1.0 / m.Ve, acc,
                                                                    beta_e, up_avg);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cfdem
