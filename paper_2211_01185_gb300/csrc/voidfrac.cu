// voidfrac.cu -- void fraction at the quadrature points (step a3).
//
// Quadrature-centred method (QCM): for every Gauss point x_q of every element
//   eps_q = 1 - sum_i V_lens(R, r_i, |x_q - x_i|) / (4/3 pi R^3),
// the sum running over the particles with |x_q - x_i|^2 < (R + r_i)^2, and
// V_lens the volume of the intersection of the averaging sphere (radius R,
// centred at x_q) with particle i.  This is the quadrature-centred reading of
// the void-fraction scheme the paper defers to its VANS companion; Eq.
// (void_fraction) of Sec. 2.1 is its particle-centroid limit, computed by
// k_pcm below.
//
// Kernel design (GB300): one warp per element in both kernels.  The warp
// walks the rows of bins that can hold a neighbour of the element, culls the
// particles against the box of the element's Gauss points, and stages the
// survivors in shared memory.  FP64 path (k_qcm): it then tests
// (quadrature point, candidate) pairs with one candidate per lane, appends
// the hits to a per-warp queue and evaluates the double-float lens volumes
// only on full warps of hits; a segmented warp scan adds up each point's
// share and the last lane of a segment updates that point's sum in shared
// memory, so every sum is accumulated in a fixed order.  Mixed path
// (k_qcm_pts): one Gauss point per lane (see there).
//
// Neighbour predicate.  The FP64 path must reproduce the FP64 definition
// exactly (bit-exact neighbour sets).  It first evaluates the distance in
// FP32 from float-float coordinates; a pair whose squared distance is
// farther than `delta` (relative) from the cutoff is decided by that value
// (delta is chosen on the host above a proven bound on the FP32 error), and
// only pairs inside the band are re-tested in FP64 with the exact
// left-to-right expression.  The mixed path decides every pair in FP32.
#include <cstdint>

#include "internal.h"
#include "df64.cuh"
#include "device_common.cuh"

namespace cfdem {

constexpr int kQcmWarps = 4;      // warps (elements) per block

struct QcmParams {
  double R;            // averaging radius
  float R32;
  float inv_vr32;      // 1 / (4/3 pi R^3)
  double inv_vr;
  float delta;         // relative band of the FP32 predicate
  float hx, hy, hz;    // element size (FP32)
  float hx_hi, hx_lo, hy_hi, hy_lo, hz_hi, hz_lo;  // float-float element size
  float inv_be[3];     // 1 / bin edge
  float qrel[64][3];   // Gauss point minus element centre, FP32
  float g1[3][4];      // per axis: 1D Gauss point minus element centre, FP32
  float gbox[3];       // half extent of the Gauss points' box per axis (a little above)
  double g[4];         // Gauss points on [0,1]
  // double-float constants of the FP64 path's lens volumes
  float g_hi[4], g_lo[4];  // Gauss points on [0,1]
  float R_hi, R_lo;        // averaging radius
  float c43_hi, c43_lo;    // 4 pi / 3
  float c12_hi, c12_lo;    // pi / 12
  const float2* cw;        // volume-conserving weights per sorted particle (hi, lo), or null
  float w3[64], w3_lo[64]; // unit-cube Gauss weights w_qx w_qy w_qz (float pair)
  float vr_ve_hi, vr_ve_lo, vr_ve32;  // V_R / V_e
};

__device__ __forceinline__ float ff_two_prod_sum(float a, float b_hi, float b_lo, float* lo) {
  // a * (b_hi + b_lo) as a float-float; a is an exact small integer + 0.5
  float p = a * b_hi;
  float e = fmaf(a, b_hi, -p);
  *lo = e + a * b_lo;
  return p;
}

__device__ __forceinline__ float lens32(float R, float r, float d2) {
  // d and 1/d from one reciprocal square root (no square root, no division)
  float dm = R - r;
  if (d2 <= dm * dm) {
    float mn = fminf(R, r);
    return (float)(4.0 / 3.0 * kPi) * mn * mn * mn;
  }
  float y = rsqrtf(d2);
  float d = d2 * y;
  float s = (R + r) - d;
  return (float)(kPi / 12.0) * s * s * (d2 + 2.0f * d * (R + r) - 3.0f * dm * dm) * y;
}

// Neumaier compensated accumulation
__device__ __forceinline__ void neumaier(float& s, float& c, float v) {
  float t = s + v;
  if (fabsf(s) >= fabsf(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

template <int K>
struct QcmSmem {
  static constexpr int Q = (K + 1) * (K + 1) * (K + 1);
  float4 qrel[Q];                          // Gauss point minus element centre
  float4 buf[kQcmWarps][64];               // culled candidates not yet tested
  int32_t bslot[kQcmWarps][64];            // their sorted slots
  int32_t gslot[kQcmWarps][32];            // the group under test (one per lane)
  // hits (lane of the group << 6) | q, q-sorted: room for the hits of one
  // layer of Gauss points ((K+1)^2 points x 32 lanes) on top of < 32 pending
  static constexpr int QCAP = 32 * (K + 1) * (K + 1) + 32;
  int32_t queue[kQcmWarps][QCAP];
  df64 accdf[kQcmWarps][Q];                // double-float sums
  int32_t cnt[kQcmWarps][Q];
  long long ids[kQcmWarps][Q];
  double xq[kQcmWarps][Q][3];              // FP64 Gauss points
  P4 g64[kQcmWarps][32];                   // FP64 positions of the group
  // the group's positions relative to the mesh origin and radii as
  // double-float (hi and lo parts), and the Gauss points of the element per
  // axis (x0-relative, hi and lo)
  float4 ghi[kQcmWarps][32], glo[kQcmWarps][32];
  float xqf[kQcmWarps][3][4][2];
};

// lens volume of the FP64 path in double-float arithmetic (relative error
// ~1e-13 on the FP32 pipes): the full smaller sphere for d <= |R - r|, else
// pi (R + r - d)^2 (d^2 + 2 d (R + r) - 3 (R - r)^2) / (12 d)
// (c43 = 4 pi / 3 and c12 = pi / 12 as double-float, split on the host)
__device__ __forceinline__ df64 lens_df(df64 R, df64 r, df64 D, df64 c43, df64 c12) {
  df64 dm = R - r;
  df64 dm2 = dm * dm;
  if (df_le(D, dm2)) {
    df64 mn = df_le(R, r) ? R : r;
    return c43 * (mn * mn * mn);
  }
  df64 d = df_sqrt(D);
  df64 S = R + r;
  df64 sdist = S - d;
  df64 num = D + df64(2.0f) * d * S - df64(3.0f) * dm2;
  return c12 * sdist * sdist * num * df_recip(d);
}

struct QcmWarp {
  int warp, lane;
  unsigned lt_mask;
  double R;
  float R32, band;
  float R_hi, R_lo;
  df64 c43, c12;
  bool want_counts, want_ids;
  const float2* cw;  // per sorted particle scale of its lens volumes, or null
};

// Evaluate the first cnt queued hits (q-sorted) and add each quadrature
// point's share with one segmented warp scan; the last lane of a segment
// updates that point's sum, so every sum is accumulated in a fixed order.
template <int K>
__device__ __forceinline__ void qcm_flush(QcmSmem<K>& sm, const QcmWarp& w, int base, int cnt,
                                          const int32_t* __restrict__ perm) {
  const unsigned FULL = 0xffffffffu;
  const int lane = w.lane, wp = w.warp;
  int q = -1 - lane;  // distinct sentinels for idle lanes
  df64 vdf(0.f, 0.f);
  long long id = 0;
  int one = 0;
  if (lane < cnt) {
    int pk = sm.queue[wp][base + lane];
    q = pk & 63;
    int j = pk >> 6;
    one = 1;
    constexpr int NQ = K + 1;
    const int qx = q % NQ, qy = (q / NQ) % NQ, qz = q / (NQ * NQ);
    float4 H = sm.ghi[wp][j], L = sm.glo[wp][j];
    df64 dx = df64(H.x, L.x) - df64(sm.xqf[wp][0][qx][0], sm.xqf[wp][0][qx][1]);
    df64 dy = df64(H.y, L.y) - df64(sm.xqf[wp][1][qy][0], sm.xqf[wp][1][qy][1]);
    df64 dz = df64(H.z, L.z) - df64(sm.xqf[wp][2][qz][0], sm.xqf[wp][2][qz][1]);
    df64 D = dx * dx + dy * dy + dz * dz;
    vdf = lens_df(df64(w.R_hi, w.R_lo), df64(H.w, L.w), D, w.c43, w.c12);
    if (w.cw) {  // volume-conserving QCM: the particle's lens volumes scaled by c
      const float2 c = __ldg(w.cw + sm.gslot[wp][j]);
      vdf = vdf * df64(c.x, c.y);
    }
    if (w.want_ids) id = perm[sm.gslot[wp][j]];
  }
  if (w.want_counts) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int qu = __shfl_up_sync(FULL, q, off);
      int nu = __shfl_up_sync(FULL, one, off);
      df64 vu(__shfl_up_sync(FULL, vdf.hi, off), __shfl_up_sync(FULL, vdf.lo, off));
      long long iu = w.want_ids ? __shfl_up_sync(FULL, id, off) : 0;
      if (lane >= off && qu == q) {
        one += nu;
        vdf = vdf + vu;
        id += iu;
      }
    }
  } else {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int qu = __shfl_up_sync(FULL, q, off);
      df64 vu(__shfl_up_sync(FULL, vdf.hi, off), __shfl_up_sync(FULL, vdf.lo, off));
      if (lane >= off && qu == q) vdf = vdf + vu;
    }
  }
  int qn = __shfl_down_sync(FULL, q, 1);
  bool last = lane < cnt && (lane == cnt - 1 || qn != q);
  if (last) {
    sm.accdf[wp][q] += vdf;
    if (w.want_counts) {
      sm.cnt[wp][q] += one;
      sm.ids[wp][q] += id;
    }
  }
  __syncwarp();
}

// test the cnt (<= 32) buffered candidates against every quadrature point
template <int K>
__device__ __forceinline__ void qcm_group(QcmSmem<K>& sm, const QcmWarp& w,
                                          const QcmParams& P, int cnt,
                                          const double* __restrict__ xs64,
                                          const float* __restrict__ xs32,
                                          const int32_t* __restrict__ perm) {
  const unsigned FULL = 0xffffffffu;
  const int lane = w.lane, wp = w.warp;
  const bool valid = lane < cnt;
  float4 my = make_float4(0.f, 0.f, 0.f, 0.f);
  int myslot = 0;
  if (valid) {
    my = sm.buf[wp][lane];
    myslot = sm.bslot[wp][lane];
    sm.gslot[wp][lane] = myslot;
    sm.g64[wp][lane] = reinterpret_cast<const P4*>(xs64)[myslot];
    const float4* ff = reinterpret_cast<const float4*>(xs32) + 2 * (int64_t)myslot;
    sm.ghi[wp][lane] = ff[0];
    sm.glo[wp][lane] = ff[1];
  }
  __syncwarp();
  const float c = w.R32 + my.w;
  const float c2 = c * c;
  const float c2_in = c2 / w.band, c2_out = c2 * w.band;
  // squared distance to Gauss point (a, b, c) = sx[a] + (sy[b] + sz[c]):
  // per-axis squares once per candidate, two additions per point
  float sx[K + 1], sy[K + 1];
#pragma unroll
  for (int a = 0; a <= K; ++a) {
    float dx = my.x - P.g1[0][a];
    float dy = my.y - P.g1[1][a];
    sx[a] = dx * dx;
    sy[a] = dy * dy;
  }
  int qn = 0;
  // layers cz = 0..K of Gauss points, then one more pass that only drains
  for (int cz = 0; cz <= K + 1; ++cz) {
    if (cz <= K) {
      // the z offset of Gauss layer cz, from shared memory (a runtime index into
      // the kernel parameters would move them to local memory)
      float dz = my.z - sm.qrel[cz * (K + 1) * (K + 1)].z;
      float sz = dz * dz;
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        float syz = sy[b] + sz;
#pragma unroll
        for (int a = 0; a <= K; ++a) {
          const int q = a + (K + 1) * (b + (K + 1) * cz);
          float d2 = sx[a] + syz;
          bool hit = valid && d2 < c2_in;
          if (valid && d2 >= c2_in && d2 <= c2_out) {  // inside the band: exact FP64 predicate
            P4 pj = sm.g64[wp][lane];
            double ddx = __dsub_rn(pj.x, sm.xq[wp][q][0]);
            double ddy = __dsub_rn(pj.y, sm.xq[wp][q][1]);
            double ddz = __dsub_rn(pj.z, sm.xq[wp][q][2]);
            double dd2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)),
                                   __dmul_rn(ddz, ddz));
            double cc = __dadd_rn(w.R, pj.w);
            hit = dd2 < __dmul_rn(cc, cc);
          }
          unsigned mask = __ballot_sync(FULL, hit);
          if (hit) sm.queue[wp][qn + __popc(mask & w.lt_mask)] = (lane << 6) | q;
          qn += __popc(mask);
        }
      }
    }
    // evaluate the full batches of 32 hits queued so far (after the last
    // layer: all of them) -- the only call of the flush -- and keep the rest
    // at the front of the queue
    const bool last = cz == K + 1;
    if (qn >= 32 || (last && qn > 0)) {
      __syncwarp();
      int base = 0;
      while (qn - base >= 32 || (last && qn > base)) {
        const int c = qn - base < 32 ? qn - base : 32;
        qcm_flush<K>(sm, w, base, c, perm);
        base += c;
      }
      int rest = qn - base;
      int tmp = lane < rest ? sm.queue[wp][base + lane] : 0;
      __syncwarp();
      if (lane < rest) sm.queue[wp][lane] = tmp;
      qn = rest;
    }
  }
  __syncwarp();
}

template <int K>
__global__ void __launch_bounds__(kQcmWarps * 32, 6)
k_qcm(MeshDev m, QcmParams P, BinDev b, const int32_t* __restrict__ bin_start,
      const int32_t* __restrict__ perm, const double* __restrict__ xs64,
      const float* __restrict__ xs32, const DevStatus* __restrict__ st,
      double* __restrict__ eps64, int32_t* __restrict__ nb_count,
      int64_t* __restrict__ nb_idsum) {
  constexpr int NQ = K + 1;
  constexpr int Q = NQ * NQ * NQ;
  __shared__ QcmSmem<K> sm;
  const unsigned FULL = 0xffffffffu;
  QcmWarp w;
  w.warp = threadIdx.x >> 5;
  w.lane = threadIdx.x & 31;
  w.lt_mask = (1u << w.lane) - 1u;
  w.R = P.R;
  w.R32 = P.R32;
  w.band = 1.0f + P.delta;
  w.R_hi = P.R_hi;
  w.R_lo = P.R_lo;
  w.c43 = df64(P.c43_hi, P.c43_lo);
  w.c12 = df64(P.c12_hi, P.c12_lo);
  w.want_ids = nb_idsum != nullptr;
  w.want_counts = nb_count != nullptr || nb_idsum != nullptr;
  w.cw = P.cw;
  const int lane = w.lane, wp = w.warp;
  for (int t = threadIdx.x; t < Q; t += blockDim.x)
    sm.qrel[t] = make_float4(P.qrel[t][0], P.qrel[t][1], P.qrel[t][2], 0.f);
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)kQcmWarps + wp;
  if (e >= m.E) return;  // whole warp leaves together
  // element indices by 32-bit division (E < 2^31; a 64-bit division costs
  // several times as many instructions)
  const int e32 = (int)e, exy = m.ne[0] * m.ne[1];
  const int ez = e32 / exy;
  const int rxy = e32 - ez * exy;
  const int ey = rxy / m.ne[0];
  const int ex = rxy - ey * m.ne[0];

  for (int q = lane; q < Q; q += 32) {
    sm.cnt[wp][q] = 0;
    sm.ids[wp][q] = 0;
    sm.accdf[wp][q] = df64(0.f, 0.f);
    int qx = q % NQ, qy = (q / NQ) % NQ, qz = q / (NQ * NQ);
    // FP64 Gauss point coordinates, rounded exactly as the definition
    sm.xq[wp][q][0] = __dadd_rn(m.x0[0], __dmul_rn(m.h[0], __dadd_rn((double)ex, P.g[qx])));
    sm.xq[wp][q][1] = __dadd_rn(m.x0[1], __dmul_rn(m.h[1], __dadd_rn((double)ey, P.g[qy])));
    sm.xq[wp][q][2] = __dadd_rn(m.x0[2], __dmul_rn(m.h[2], __dadd_rn((double)ez, P.g[qz])));
  }
  if (lane == 0) {
    // Gauss points relative to the origin as double-float, h (e + g), per axis
    const int eax[3] = {ex, ey, ez};
    const float hh[3] = {P.hx_hi, P.hy_hi, P.hz_hi}, hl[3] = {P.hx_lo, P.hy_lo, P.hz_lo};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        df64 t = df64((float)eax[ax]) + df64(P.g_hi[a], P.g_lo[a]);
        df64 G = df64(hh[ax], hl[ax]) * t;
        sm.xqf[wp][ax][a][0] = G.hi;
        sm.xqf[wp][ax][a][1] = G.lo;
      }
  }
  // element centre relative to the mesh origin, float-float
  float chx, clx, chy, cly, chz, clz;
  chx = ff_two_prod_sum((float)ex + 0.5f, P.hx_hi, P.hx_lo, &clx);
  chy = ff_two_prod_sum((float)ey + 0.5f, P.hy_hi, P.hy_lo, &cly);
  chz = ff_two_prod_sum((float)ez + 0.5f, P.hz_hi, P.hz_lo, &clz);
  // half extents of the box spanned by the element's Gauss points (every
  // neighbour of a Gauss point lies within R + r of it)
  const float hhx = P.gbox[0], hhy = P.gbox[1], hhz = P.gbox[2];
  const double rmax = __longlong_as_double((long long)st->rmax_bits);
  const float cut = (float)(P.R + rmax) * (1.0f + 1e-5f);
  // bin range per axis (conservative)
  int bx0, bx1, by0, by1, bz0, bz1;
  {
    int l = (int)floorf((chx - hhx - cut) * P.inv_be[0] - 1e-3f);
    int h = (int)floorf((chx + hhx + cut) * P.inv_be[0] + 1e-3f);
    bx0 = min(max(l, 0), b.nb[0] - 1);
    bx1 = min(max(h, 0), b.nb[0] - 1);
    l = (int)floorf((chy - hhy - cut) * P.inv_be[1] - 1e-3f);
    h = (int)floorf((chy + hhy + cut) * P.inv_be[1] + 1e-3f);
    by0 = min(max(l, 0), b.nb[1] - 1);
    by1 = min(max(h, 0), b.nb[1] - 1);
    l = (int)floorf((chz - hhz - cut) * P.inv_be[2] - 1e-3f);
    h = (int)floorf((chz + hhz + cut) * P.inv_be[2] + 1e-3f);
    bz0 = min(max(l, 0), b.nb[2] - 1);
    bz1 = min(max(h, 0), b.nb[2] - 1);
  }
  __syncwarp();

  // Stream the candidates into the buffer; test each full group of 32 (and
  // the last, partial one).  The bin rows (by, bz) in reach, each spanning
  // bins bx0..bx1, are handled 32 at a time: every lane loads one row's
  // bounds, a warp scan concatenates the rows, and each chunk of 32
  // candidates spans rows (a lane finds its row by binary search over the
  // scanned offsets).  Written as one loop so that the group -- and the flush
  // inside it -- has a single call site in the code.
  int nb = 0;  // buffered culled candidates (warp-uniform)
  const int nrx = by1 - by0 + 1, nrows = nrx * (bz1 - bz0 + 1);
  int rb = -32, base = 0, total = 0;  // row batch, chunk start, candidates in the batch
  int my_s0 = 0, my_excl = 0;         // this lane's row: first slot, offset in the batch
  bool more = true;
  for (;;) {
    while (more && nb < 32) {
      if (base >= total) {  // next batch of rows
        rb += 32;
        if (rb >= nrows) {
          more = false;
          break;
        }
        const int ri = rb + lane;
        int cntr = 0;
        my_s0 = 0;
        if (ri < nrows) {
          int by = by0 + ri % nrx, bz = bz0 + ri / nrx;
          int64_t row = (int64_t)b.nb[0] * (by + (int64_t)b.nb[1] * bz);
          my_s0 = bin_start[row + bx0];
          cntr = bin_start[row + bx1 + 1] - my_s0;
        }
        int incl = cntr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int v = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += v;
        }
        total = __shfl_sync(FULL, incl, 31);
        my_excl = incl - cntr;
        base = 0;
        continue;
      }
      const int kk = base + lane;
      // the row holding candidate kk: the last one whose offset is <= kk
      int lo = 0, hi = 31;
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        int mid = (lo + hi + 1) >> 1;
        int em = __shfl_sync(FULL, my_excl, mid);
        if (em <= kk) lo = mid;
        else hi = mid - 1;
      }
      const int s = __shfl_sync(FULL, my_s0, lo) + (kk - __shfl_sync(FULL, my_excl, lo));
      bool keep = false;
      float4 rel = make_float4(0.f, 0.f, 0.f, 0.f);
      if (kk < total) {
        const float4* p = reinterpret_cast<const float4*>(xs32) + 2 * (int64_t)s;
        float4 hi4 = p[0], lo4 = p[1];
        rel.x = (hi4.x - chx) + (lo4.x - clx);
        rel.y = (hi4.y - chy) + (lo4.y - cly);
        rel.z = (hi4.z - chz) + (lo4.z - clz);
        rel.w = hi4.w;
        float ox = fmaxf(fabsf(rel.x) - hhx, 0.f);
        float oy = fmaxf(fabsf(rel.y) - hhy, 0.f);
        float oz = fmaxf(fabsf(rel.z) - hhz, 0.f);
        float c = (w.R32 + rel.w) * w.band;
        keep = ox * ox + oy * oy + oz * oz < c * c * w.band;
      }
      unsigned mask = __ballot_sync(FULL, keep);
      if (keep) {
        int pos = nb + __popc(mask & w.lt_mask);
        sm.buf[wp][pos] = rel;
        sm.bslot[wp][pos] = s;
      }
      nb += __popc(mask);
      base += 32;
    }
    if (nb == 0) break;
    __syncwarp();
    const int cnt = nb < 32 ? nb : 32;
    qcm_group<K>(sm, w, P, cnt, xs64, xs32, perm);
    int rest = nb - cnt;
    float4 tb = make_float4(0.f, 0.f, 0.f, 0.f);
    int ts = 0;
    if (lane < rest) {
      tb = sm.buf[wp][32 + lane];
      ts = sm.bslot[wp][32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
      sm.buf[wp][lane] = tb;
      sm.bslot[wp][lane] = ts;
    }
    __syncwarp();
    nb = rest;
  }
  __syncwarp();

  // outputs
  const int64_t o = e * Q;
  for (int q = lane; q < Q; q += 32) {
    df64 a = sm.accdf[wp][q];
    if (eps64) eps64[o + q] = 1.0 - ((double)a.hi + (double)a.lo) * P.inv_vr;
    if (nb_count) nb_count[o + q] = sm.cnt[wp][q];
    if (nb_idsum) nb_idsum[o + q] = sm.ids[wp][q];
  }
}

// ----------------------------------------------------------------------------
// Mixed path, lanes = Gauss points.  One warp per element: the candidates
// are fetched and culled against the box of the element's Gauss points as in
// k_qcm, each kept one written to shared memory once with its constants
// (R + r, (R + r)^2, (R - r)^2, the volume of the smaller sphere, the
// volume-conserving weight); then every candidate is broadcast to the lanes,
// each lane tests its own Gauss point (two for Q3; for Q1 four groups of 8
// lanes take every fourth candidate) and adds the lens volume to a
// Neumaier-compensated sum in registers.  No hit queue and no scan: the
// instructions per candidate are a distance, a compare and, for the lanes
// that hit, the lens volume.  Sums run over the candidates in a fixed order
// (the Q1 groups combined by a fixed shuffle tree), so results are
// reproducible.

template <int K>
struct QcmPtsSmem {
  static constexpr int Q = (K + 1) * (K + 1) * (K + 1);
  float4 qrel[Q];                  // Gauss point minus element centre
  float4 cand[kQcmWarps][64];      // culled candidates: position - centre, R + r
  float4 cons[kQcmWarps][64];      // (R + r)^2, (R - r)^2, full-overlap volume, weight
  int32_t slot[kQcmWarps][64];     // their sorted slots
  // per lane, the candidates (of the 32 being tested) that overlap its Gauss
  // point, in candidate order: [warp][hit][lane] (Q <= 32 only)
  uint8_t hits[kQcmWarps][Q > 32 ? 1 : 32][32];
};

template <int K>
__global__ void __launch_bounds__(kQcmWarps * 32, 8)
k_qcm_pts(MeshDev m, QcmParams P, BinDev b, const int32_t* __restrict__ bin_start,
          const int32_t* __restrict__ perm, const float* __restrict__ xs32,
          const DevStatus* __restrict__ st, double* __restrict__ eps64,
          float* __restrict__ eps32, int32_t* __restrict__ nb_count,
          int64_t* __restrict__ nb_idsum) {
  constexpr int NQ = K + 1;
  constexpr int Q = NQ * NQ * NQ;
  constexpr int G = Q <= 8 ? 4 : 1;     // candidate groups of lanes (Q1)
  constexpr int PPL = Q > 32 ? 2 : 1;   // Gauss points per lane (Q3)
  __shared__ QcmPtsSmem<K> sm;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int t = threadIdx.x; t < Q; t += blockDim.x)
    sm.qrel[t] = make_float4(P.qrel[t][0], P.qrel[t][1], P.qrel[t][2], 0.f);
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)kQcmWarps + wp;
  if (e >= m.E) return;  // whole warp leaves together
  const int e32 = (int)e, exy = m.ne[0] * m.ne[1];  // E < 2^31
  const int ez = e32 / exy;
  const int rxy = e32 - ez * exy;
  const int ey = rxy / m.ne[0];
  const int ex = rxy - ey * m.ne[0];
  const bool want_ids = nb_idsum != nullptr;
  const bool want_counts = nb_count != nullptr || want_ids;
  // this lane's Gauss points
  const int grp = G > 1 ? lane / Q : 0;
  float qx[PPL], qy[PPL], qz[PPL], acc[PPL], cmp[PPL];
  int cnt[PPL];
  long long ids[PPL];
  bool qok[PPL];
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    const int q = (G > 1 ? lane % Q : lane) + 32 * p;
    qok[p] = q < Q && grp < G;
    const float4 g = sm.qrel[qok[p] ? q : 0];
    qx[p] = g.x;
    qy[p] = g.y;
    qz[p] = g.z;
    acc[p] = cmp[p] = 0.f;
    cnt[p] = 0;
    ids[p] = 0;
  }
  // element centre relative to the mesh origin, float-float
  float chx, clx, chy, cly, chz, clz;
  // (small integers made floats by the 2^23 trick: no conversion instruction)
  const float fex = __int_as_float(0x4B000000 + ex) - 8388608.0f;
  const float fey = __int_as_float(0x4B000000 + ey) - 8388608.0f;
  const float fez = __int_as_float(0x4B000000 + ez) - 8388608.0f;
  chx = ff_two_prod_sum(fex + 0.5f, P.hx_hi, P.hx_lo, &clx);
  chy = ff_two_prod_sum(fey + 0.5f, P.hy_hi, P.hy_lo, &cly);
  chz = ff_two_prod_sum(fez + 0.5f, P.hz_hi, P.hz_lo, &clz);
  const float hhx = P.gbox[0], hhy = P.gbox[1], hhz = P.gbox[2];
  const df64 rmx = df_from_double_int(__longlong_as_double((long long)st->rmax_bits));
  const float cut = (P.R32 + rmx.hi) * (1.0f + 1e-4f);  // rounded up: conservative
  const float R32 = P.R32;
  const float band = 1.0f + P.delta;
  // bin range per axis (conservative): floors of values clamped to
  // [0, nb - 1] first, taken without conversion instructions
  int bx0, bx1, by0, by1, bz0, bz1;
  {
    auto cellof = [&](float t, int a) {
      int k;
      floor_small(fminf(fmaxf(t, 0.0f), b.nm1f[a]), &k);
      return k;
    };
    bx0 = cellof((chx - hhx - cut) * P.inv_be[0] - 1e-3f, 0);
    bx1 = cellof((chx + hhx + cut) * P.inv_be[0] + 1e-3f, 0);
    by0 = cellof((chy - hhy - cut) * P.inv_be[1] - 1e-3f, 1);
    by1 = cellof((chy + hhy + cut) * P.inv_be[1] + 1e-3f, 1);
    bz0 = cellof((chz - hhz - cut) * P.inv_be[2] - 1e-3f, 2);
    bz1 = cellof((chz + hhz + cut) * P.inv_be[2] + 1e-3f, 2);
  }
  const float c43 = (float)(4.0 / 3.0 * kPi), c12 = (float)(kPi / 12.0);
  // stream the candidates (rows of bins 32 at a time, chunks of 32 candidates
  // across rows, as in k_qcm); every 32 kept ones are tested
  int nb = 0;
  const int nrx = by1 - by0 + 1, nrows = nrx * (bz1 - bz0 + 1);
  int rb = -32, base = 0, total = 0;
  int my_s0 = 0, my_excl = 0;
  bool more = true;
  for (;;) {
    while (more && nb < 32) {
      if (base >= total) {
        rb += 32;
        if (rb >= nrows) {
          more = false;
          break;
        }
        const int ri = rb + lane;
        int cntr = 0;
        my_s0 = 0;
        if (ri < nrows) {
          const int by = by0 + ri % nrx, bz = bz0 + ri / nrx;
          const int64_t row = (int64_t)b.nb[0] * (by + (int64_t)b.nb[1] * bz);
          my_s0 = bin_start[row + bx0];
          cntr = bin_start[row + bx1 + 1] - my_s0;
        }
        int incl = cntr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += v;
        }
        total = __shfl_sync(FULL, incl, 31);
        my_excl = incl - cntr;
        base = 0;
        continue;
      }
      const int kk = base + lane;
      int lo = 0, hi = 31;
#pragma unroll
      for (int stp = 0; stp < 5; ++stp) {
        const int mid = (lo + hi + 1) >> 1;
        const int em = __shfl_sync(FULL, my_excl, mid);
        if (em <= kk) lo = mid;
        else hi = mid - 1;
      }
      const int s = __shfl_sync(FULL, my_s0, lo) + (kk - __shfl_sync(FULL, my_excl, lo));
      bool keep = false;
      float4 rel = make_float4(0.f, 0.f, 0.f, 0.f);
      if (kk < total) {
        const float4* pp = reinterpret_cast<const float4*>(xs32) + 2 * (int64_t)s;
        const float4 hi4 = pp[0], lo4 = pp[1];
        rel.x = (hi4.x - chx) + (lo4.x - clx);
        rel.y = (hi4.y - chy) + (lo4.y - cly);
        rel.z = (hi4.z - chz) + (lo4.z - clz);
        rel.w = hi4.w;
        const float ox = fmaxf(fabsf(rel.x) - hhx, 0.f);
        const float oy = fmaxf(fabsf(rel.y) - hhy, 0.f);
        const float oz = fmaxf(fabsf(rel.z) - hhz, 0.f);
        const float c = (R32 + rel.w) * band;
        keep = ox * ox + oy * oy + oz * oz < c * c * band;
      }
      const unsigned mask = __ballot_sync(FULL, keep);
      if (keep) {
        const int pos = nb + __popc(mask & lt_mask);
        const float r = rel.w, Rr = R32 + r, dm = R32 - r, mn = fminf(R32, r);
        sm.cand[wp][pos] = make_float4(rel.x, rel.y, rel.z, Rr);
        sm.cons[wp][pos] =
            make_float4(Rr * Rr, dm * dm, c43 * mn * mn * mn, P.cw ? __ldg(P.cw + s).x : 1.0f);
        sm.slot[wp][pos] = s;
      }
      nb += __popc(mask);
      base += 32;
    }
    if (nb == 0) break;
    __syncwarp();
    const int cn = nb < 32 ? nb : 32;
    // Q <= 32 (one point per lane, a few hits per point): each lane first
    // lists the candidates that overlap its point, then evaluates the lens
    // volumes of its own list in candidate order (the order of its sum) --
    // the warp runs as many lens rounds as its busiest lane has hits instead
    // of one for every candidate any lane hits.  Q3 (two points per lane,
    // most lanes hit most candidates): test and evaluate in one pass.
    auto lens = [&](int p, int j, float d2, const float4& A, const float4& B) {
      float v;
      if (d2 <= B.y) {
        v = B.z;
      } else {
        const float y = rsqrtf(d2);
        const float d = d2 * y;
        const float sd = A.w - d;
        v = c12 * sd * sd * (d2 + 2.0f * d * A.w - 3.0f * B.y) * y;
      }
      neumaier(acc[p], cmp[p], v * B.w);
      if (want_counts) {
        ++cnt[p];
        if (want_ids) ids[p] += perm[sm.slot[wp][j]];
      }
    };
    if constexpr (PPL == 1) {
      int nh = 0;
      for (int j = grp; j < cn; j += G) {
        const float4 A = sm.cand[wp][j];
        const float rr2 = sm.cons[wp][j].x;
        const float dx = A.x - qx[0], dy = A.y - qy[0], dz = A.z - qz[0];
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (qok[0] && d2 < rr2) sm.hits[wp][nh++][lane] = (uint8_t)j;
      }
      const int mh = (int)__reduce_max_sync(FULL, (unsigned)nh);
      for (int h = 0; h < mh; ++h) {
        if (h < nh) {
          const int j = sm.hits[wp][h][lane];
          const float4 A = sm.cand[wp][j];
          const float4 B = sm.cons[wp][j];
          const float dx = A.x - qx[0], dy = A.y - qy[0], dz = A.z - qz[0];
          lens(0, j, dx * dx + dy * dy + dz * dz, A, B);
        }
      }
    } else {
      for (int j = grp; j < cn; j += G) {
        const float4 A = sm.cand[wp][j];
        const float4 B = sm.cons[wp][j];
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
          const float dx = A.x - qx[p], dy = A.y - qy[p], dz = A.z - qz[p];
          const float d2 = dx * dx + dy * dy + dz * dz;
          if (qok[p] && d2 < B.x) lens(p, j, d2, A, B);
        }
      }
    }
    // keep the candidates past the 32 tested at the front
    const int rest = nb - cn;
    float4 ta = make_float4(0.f, 0.f, 0.f, 0.f), tb = ta;
    int ts = 0;
    if (lane < rest) {
      ta = sm.cand[wp][32 + lane];
      tb = sm.cons[wp][32 + lane];
      ts = sm.slot[wp][32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
      sm.cand[wp][lane] = ta;
      sm.cons[wp][lane] = tb;
      sm.slot[wp][lane] = ts;
    }
    __syncwarp();
    nb = rest;
  }
  // Q1: the groups' sums of the same point, in a fixed tree
  if (G > 1) {
#pragma unroll
    for (int off = 16; off >= Q; off >>= 1) {
      const float oa = __shfl_down_sync(FULL, acc[0], off);
      const float oc = __shfl_down_sync(FULL, cmp[0], off);
      const int on = __shfl_down_sync(FULL, cnt[0], off);
      const long long oi = __shfl_down_sync(FULL, ids[0], off);
      if (lane + off < 32) {
        neumaier(acc[0], cmp[0], oa);
        cmp[0] += oc;
        cnt[0] += on;
        ids[0] += oi;
      }
    }
  }
  const int64_t o = e * Q;
#pragma unroll
  for (int p = 0; p < PPL; ++p) {
    const int q = (G > 1 ? lane % Q : lane) + 32 * p;
    if (!(q < Q && grp == 0)) continue;
    const float v = 1.0f - (acc[p] + cmp[p]) * P.inv_vr32;
    if (eps32) eps32[o + q] = v;
    if (eps64) eps64[o + q] = (double)v;
    if (nb_count) nb_count[o + q] = cnt[p];
    if (nb_idsum) nb_idsum[o + q] = ids[p];
  }
}

static void split_ff(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

// Volume-conserving QCM weights, one thread per sorted particle s:
//   c_s = V_p / S_s,  S_s = sum over the Gauss points within R + r of
//   w_q V_e V(R, r, |x_s - x_q|) / V_R
// (w_q the unit-cube Gauss weights), 1 where S_s = 0.  Distances are taken
// relative to the corner of the particle's own element, so that FP32 keeps
// digits of millimetre-scale offsets in a large box.  FP32 path: FP32
// throughout.  FP64 path: an FP32 prefilter with a margin, then the kept
// pairs' squared distances, lens volumes and the sum in double-float; c is
// stored as a float pair (hi, lo).
template <int K, bool FP64>
__global__ void __launch_bounds__(128)
k_qcm_weights(MeshDev m, QcmParams P, int64_t n, const double* __restrict__ xs64,
              float2* __restrict__ cw) {
  constexpr int NQ = K + 1;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const P4 pt = reinterpret_cast<const P4*>(xs64)[s];
  const double pc[3] = {pt.x, pt.y, pt.z};
  const double r = pt.w;
  const float hf[3] = {P.hx, P.hy, P.hz};
  const df64 hdf[3] = {df64(P.hx_hi, P.hx_lo), df64(P.hy_hi, P.hy_lo), df64(P.hz_hi, P.hz_lo)};
  // particle relative to the corner of its element, FP64 then split
  int ie[3], lo[3], hi[3];
  float xe[3];
  df64 xedf[3];
  const float cut = (float)(P.R + r);
  for (int a = 0; a < 3; ++a) {
    const double rel = pc[a] - m.x0[a];
    int e = (int)floor(rel / m.h[a]);
    e = e < 0 ? 0 : (e > m.ne[a] - 1 ? m.ne[a] - 1 : e);
    ie[a] = e;
    const double off = rel - m.h[a] * (double)e;
    xe[a] = (float)off;
    xedf[a] = df_from_double(off);
    const float cu = cut / hf[a];
    int l = (int)floorf(xe[a] / hf[a] - cu - 1e-3f), h = (int)floorf(xe[a] / hf[a] + cu + 1e-3f);
    lo[a] = ie[a] + l < 0 ? -ie[a] : l;
    hi[a] = ie[a] + h > m.ne[a] - 1 ? m.ne[a] - 1 - ie[a] : h;
  }
  const float cut2 = cut * cut * (FP64 ? 1.0001f : 1.0f);
  const float R32 = P.R32, r32 = (float)r;
  float S32 = 0.f;
  df64 Sdf(0.f, 0.f);
  const df64 Rdf(P.R_hi, P.R_lo), rdf = df_from_double(r);
  const df64 c43(P.c43_hi, P.c43_lo), c12(P.c12_hi, P.c12_lo);
  for (int dz = lo[2]; dz <= hi[2]; ++dz)
    for (int qz = 0; qz < NQ; ++qz) {
      const float Zr = hf[2] * ((float)dz + (float)P.g[qz]);
      const float fz = xe[2] - Zr;
      for (int dy = lo[1]; dy <= hi[1]; ++dy)
        for (int qy = 0; qy < NQ; ++qy) {
          const float Yr = hf[1] * ((float)dy + (float)P.g[qy]);
          const float fy = xe[1] - Yr;
          const float dyz = fy * fy + fz * fz;
          if (!(dyz < cut2)) continue;
          for (int dx = lo[0]; dx <= hi[0]; ++dx)
#pragma unroll
            for (int qx = 0; qx < NQ; ++qx) {
              const float Xr = hf[0] * ((float)dx + (float)P.g[qx]);
              const float fx = xe[0] - Xr;
              const float d2 = fx * fx + dyz;
              if (!(d2 < cut2)) continue;
              const float wq = P.w3[qx + NQ * (qy + NQ * qz)];
              if (FP64) {
                // offsets from the element corner in double-float: h (d + g)
                const df64 X = hdf[0] * (df64((float)dx) + df64(P.g_hi[qx], P.g_lo[qx]));
                const df64 Y = hdf[1] * (df64((float)dy) + df64(P.g_hi[qy], P.g_lo[qy]));
                const df64 Z = hdf[2] * (df64((float)dz) + df64(P.g_hi[qz], P.g_lo[qz]));
                const df64 ddx = xedf[0] - X, ddy = xedf[1] - Y, ddz = xedf[2] - Z;
                const df64 D = ddx * ddx + ddy * ddy + ddz * ddz;
                const df64 Rc = Rdf + rdf;
                if (!df_le(D, Rc * Rc) || (D.hi == (Rc * Rc).hi && D.lo == (Rc * Rc).lo)) continue;
                Sdf += df64(wq, P.w3_lo[qx + NQ * (qy + NQ * qz)]) * lens_df(Rdf, rdf, D, c43, c12);
              } else {
                S32 += wq * lens32(R32, r32, d2);
              }
            }
        }
    }
  // S = V_e / V_R * sum w_q V ; c = V_p / S = (4/3 pi r^3) V_R / (V_e sum)
  float2 out;
  if (FP64) {
    if (Sdf.hi > 0.f) {
      const df64 vp = c43 * (rdf * rdf * rdf);
      const df64 c = vp * df64(P.vr_ve_hi, P.vr_ve_lo) * df_recip(Sdf);
      out = make_float2(c.hi, c.lo);
    } else {
      out = make_float2(1.f, 0.f);
    }
  } else {
    if (S32 > 0.f) {
      const float vp = (float)(4.0 / 3.0 * kPi) * r32 * r32 * r32;
      out = make_float2(vp * P.vr_ve32 / S32, 0.f);
    } else {
      out = make_float2(1.f, 0.f);
    }
  }
  cw[s] = out;
}

cudaError_t launch_qcm(const MeshDev& m, const Tables& t, const BinDev& b, int precision,
                       double R, const int32_t* bin_start, const int32_t* perm,
                       const double* xs64, const float* xs32, const DevStatus* st,
                       double* eps_q64, float* eps_q32, int32_t* nb_count, int64_t* nb_idsum,
                       cudaStream_t s, float2* cw, int64_t n) {
  QcmParams P;
  P.cw = nullptr;
  P.R = R;
  P.R32 = (float)R;
  P.inv_vr = 1.0 / (4.0 / 3.0 * kPi * R * R * R);
  P.inv_vr32 = (float)P.inv_vr;
  P.hx = (float)m.h[0];
  P.hy = (float)m.h[1];
  P.hz = (float)m.h[2];
  split_ff(m.h[0], &P.hx_hi, &P.hx_lo);
  split_ff(m.h[1], &P.hy_hi, &P.hy_lo);
  split_ff(m.h[2], &P.hz_hi, &P.hz_lo);
  for (int a = 0; a < 3; ++a) P.inv_be[a] = (float)(1.0 / b.be[a]);
  int nq = m.k + 1;
  for (int q = 0; q < 64; ++q) {
    int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
    if (q >= nq * nq * nq) qx = qy = qz = 0;
    P.qrel[q][0] = (float)(m.h[0] * (t.g[qx] - 0.5));
    P.qrel[q][1] = (float)(m.h[1] * (t.g[qy] - 0.5));
    P.qrel[q][2] = (float)(m.h[2] * (t.g[qz] - 0.5));
  }
  for (int ax = 0; ax < 3; ++ax)  // rounded up: culling stays conservative
    P.gbox[ax] = (float)(m.h[ax] * (t.g[nq - 1] - 0.5) * (1.0 + 1e-6));
  split_ff(R, &P.R_hi, &P.R_lo);
  split_ff(4.0 / 3.0 * kPi, &P.c43_hi, &P.c43_lo);
  split_ff(kPi / 12.0, &P.c12_hi, &P.c12_lo);
  for (int a = 0; a < 4; ++a) {
    P.g[a] = t.g[a];
    split_ff(t.g[a], &P.g_hi[a], &P.g_lo[a]);
    for (int ax = 0; ax < 3; ++ax)
      P.g1[ax][a] = a < nq ? (float)(m.h[ax] * (t.g[a] - 0.5)) : 0.f;
  }
  // band of the FP32 predicate: above the worst FP32 error of the squared
  // distance, about 2^-22 * 10 * (D / R)^2 relative, with D the largest
  // coordinate offset of a kept candidate (half diagonal + cutoff + bin)
  double hmax = m.h[0] > m.h[1] ? m.h[0] : m.h[1];
  hmax = hmax > m.h[2] ? hmax : m.h[2];
  double bmax = b.be[0] > b.be[1] ? b.be[0] : b.be[1];
  bmax = bmax > b.be[2] ? bmax : b.be[2];
  double D = 2.0 * hmax + 2.0 * R + bmax;
  double bound = 10.0 * (D / R) * (D / R) / 4194304.0;
  double delta = 16.0 * bound;
  if (delta < 1.0 / 4096.0) delta = 1.0 / 4096.0;
  if (delta > 0.25) delta = 0.25;
  P.delta = (float)delta;
  for (int q = 0; q < 64; ++q) {
    int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
    double wq = q < nq * nq * nq ? t.w[qx] * t.w[qy] * t.w[qz] : 0.0;
    split_ff(wq, &P.w3[q], &P.w3_lo[q]);
  }
  const double vr_ve = 4.0 / 3.0 * kPi * R * R * R / m.Ve;
  split_ff(vr_ve, &P.vr_ve_hi, &P.vr_ve_lo);
  P.vr_ve32 = (float)vr_ve;
  if (cw && n > 0) {  // volume-conserving weights first, then the scaled sums
    const unsigned nb = (unsigned)((n + 127) / 128);
#define CFDEM_QW(KK)                                                                \
    if (m.k == KK) {                                                                \
      if (precision == 0)                                                           \
        k_qcm_weights<KK, true><<<nb, 128, 0, s>>>(m, P, n, xs64, cw);             \
      else                                                                          \
        k_qcm_weights<KK, false><<<nb, 128, 0, s>>>(m, P, n, xs64, cw);            \
    }
    CFDEM_QW(1)
    CFDEM_QW(2)
    CFDEM_QW(3)
#undef CFDEM_QW
    count_launches(1);
    P.cw = cw;
  }
  dim3 grid((unsigned)((m.E + kQcmWarps - 1) / kQcmWarps));
  dim3 block(kQcmWarps * 32);
  bool fp64 = precision == 0;
#define CFDEM_QCM(KK)                                                                     \
  if (m.k == KK) {                                                                        \
    if (fp64)                                                                             \
      k_qcm<KK><<<grid, block, 0, s>>>(m, P, b, bin_start, perm, xs64, xs32, st, eps_q64, \
                                       nb_count, nb_idsum);                               \
    else                                                                                  \
      k_qcm_pts<KK><<<grid, block, 0, s>>>(m, P, b, bin_start, perm, xs32, st, eps_q64,   \
                                           eps_q32, nb_count, nb_idsum);                  \
    count_launches(1);                                                                    \
    return cudaGetLastError();                                                            \
  }
  CFDEM_QCM(1)
  CFDEM_QCM(2)
  CFDEM_QCM(3)
#undef CFDEM_QCM
  return cudaErrorInvalidValue;
}

// ----------------------------------------------------------------------------
// Particle-centroid method, Eq. (void_fraction): eps_e = (V_e - sum_{i in e}
// V_p,i) / V_e, copied to every quadrature point of e.

__global__ void k_pcm_accumulate(MeshDev m, int64_t n, const double* __restrict__ x,
                                 const double* __restrict__ r, double* __restrict__ vol,
                                 DevStatus* st) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int ie[3];
  for (int a = 0; a < 3; ++a) {
    double xa = x[3 * i + a];
    double slack = __dmul_rn(1e-12, m.L[a]);
    double lo = __dsub_rn(m.x0[a], slack);
    double hi = __dadd_rn(__dadd_rn(m.x0[a], m.L[a]), slack);
    if (!(xa >= lo && xa <= hi)) {
      atomicMin(&st->first_bad, (unsigned long long)i);
      return;
    }
    double tt = __ddiv_rn(__dsub_rn(xa, m.x0[a]), m.h[a]);
    int v = (int)floor(tt);
    ie[a] = v < 0 ? 0 : (v > m.ne[a] - 1 ? m.ne[a] - 1 : v);
  }
  int64_t e = ie[0] + (int64_t)m.ne[0] * (ie[1] + (int64_t)m.ne[1] * ie[2]);
  double ri = r[i];
  atomicAdd(vol + e, (4.0 / 3.0 * kPi) * ri * ri * ri);
}

__global__ void k_pcm_write(MeshDev m, const double* __restrict__ vol, double* __restrict__ eps64,
                            float* __restrict__ eps32) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m.E * m.Q) return;
  int64_t e = t / m.Q;
  double eps = (m.Ve - vol[e]) / m.Ve;
  if (eps64) eps64[t] = eps;
  if (eps32) eps32[t] = (float)eps;
}

cudaError_t launch_pcm(const MeshDev& m, int64_t n, const double* x, const double* r,
                       double* vol_elem, double* eps_q64, float* eps_q32, DevStatus* st,
                       cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(vol_elem, 0, sizeof(double) * m.E, s);
  if (err != cudaSuccess) return err;
  int bs = 256;
  if (n > 0) k_pcm_accumulate<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(m, n, x, r, vol_elem, st);
  int64_t tot = m.E * m.Q;
  k_pcm_write<<<(unsigned)((tot + bs - 1) / bs), bs, 0, s>>>(m, vol_elem, eps_q64, eps_q32);
  count_launches(n > 0 ? 2 : 1);
  return cudaGetLastError();
}

}  // namespace cfdem
