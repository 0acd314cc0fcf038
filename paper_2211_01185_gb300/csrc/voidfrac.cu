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
// Kernel design (GB300): one warp per element.  The warp walks the rows of
// bins that can hold a neighbour of the element, culls the particles against
// the element box, and stages the survivors in shared memory.  It then tests
// (quadrature point, candidate) pairs 32 at a time, appends the hits to a
// per-warp queue and evaluates the lens volume only on full warps of hits.
// Each lane owns the running sum of one (or two, for Q3) quadrature points;
// the values of a flushed batch reach their owners by warp shuffles, so the
// sums are accumulated in a fixed order.
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

namespace cfdem {

constexpr int kQcmWarps = 4;      // warps (elements) per block
constexpr int kQcmChunk = 128;    // staged candidates per warp

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
  double g[4];         // Gauss points on [0,1]
};

__device__ __forceinline__ float ff_two_prod_sum(float a, float b_hi, float b_lo, float* lo) {
  // a * (b_hi + b_lo) as a float-float; a is an exact small integer + 0.5
  float p = a * b_hi;
  float e = fmaf(a, b_hi, -p);
  *lo = e + a * b_lo;
  return p;
}

__device__ __forceinline__ double lens64(double R, double r, double d2) {
  // intersection volume of spheres of radii R, r at squared distance d2 < (R+r)^2:
  // pi s^2 (d^2 + 2 d (R+r) - 3 (R-r)^2) / (12 d), s = R + r - d, written with
  // y = 1/d from one reciprocal square root (d = d2 y) to spare the FP64
  // square root and division
  double dm = R - r;
  double mn = R < r ? R : r;
  if (d2 <= dm * dm) return (4.0 / 3.0 * kPi) * mn * mn * mn;
  double y = rsqrt(d2);
  double d = d2 * y;
  double s = (R + r) - d;
  return (kPi / 12.0) * s * s * (d + 2.0 * (R + r) - 3.0 * dm * dm * y);
}

__device__ __forceinline__ float lens32(float R, float r, float d2) {
  float dm = R - r;
  float mn = fminf(R, r);
  float d = sqrtf(d2);
  if (d <= fabsf(dm)) return (float)(4.0 / 3.0 * kPi) * mn * mn * mn;
  float s = (R + r) - d;
  return (float)kPi * s * s * (d2 + 2.0f * d * (R + r) - 3.0f * dm * dm) / (12.0f * d);
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

template <int K, bool FP64>
struct QcmSmem {
  float qrel[(K + 1) * (K + 1) * (K + 1)][3];  // Gauss point minus element centre
  float4 cand[kQcmWarps][kQcmChunk];     // rel. position (to element centre), radius
  int32_t cslot[kQcmWarps][kQcmChunk];   // sorted slot
  int32_t queue[kQcmWarps][64];
  double xq[kQcmWarps][FP64 ? (K + 1) * (K + 1) * (K + 1) : 1][3];
};

template <int K, bool FP64>
__global__ void __launch_bounds__(kQcmWarps * 32)
k_qcm(MeshDev m, QcmParams P, BinDev b, const int32_t* __restrict__ bin_start,
      const int32_t* __restrict__ perm, const double* __restrict__ xs64,
      const float* __restrict__ xs32, const DevStatus* __restrict__ st,
      double* __restrict__ eps64, float* __restrict__ eps32, int32_t* __restrict__ nb_count,
      int64_t* __restrict__ nb_idsum) {
  constexpr int NQ = K + 1;
  constexpr int Q = NQ * NQ * NQ;
  __shared__ QcmSmem<K, FP64> sm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-lane quadrature offsets are read with lane-varying indices: keep them
  // in shared memory (the kernel-parameter bank would serialise them)
  for (int t = threadIdx.x; t < Q * 3; t += blockDim.x) sm.qrel[t / 3][t % 3] = P.qrel[t / 3][t % 3];
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)kQcmWarps + warp;
  if (e >= m.E) return;  // whole warp leaves together
  const unsigned FULL = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int ex = (int)(e % m.ne[0]);
  const int ey = (int)((e / m.ne[0]) % m.ne[1]);
  const int ez = (int)(e / ((int64_t)m.ne[0] * m.ne[1]));

  // element centre relative to the mesh origin, float-float
  float c_hi[3], c_lo[3];
  c_hi[0] = ff_two_prod_sum((float)ex + 0.5f, P.hx_hi, P.hx_lo, &c_lo[0]);
  c_hi[1] = ff_two_prod_sum((float)ey + 0.5f, P.hy_hi, P.hy_lo, &c_lo[1]);
  c_hi[2] = ff_two_prod_sum((float)ez + 0.5f, P.hz_hi, P.hz_lo, &c_lo[2]);
  const float hh[3] = {0.5f * P.hx, 0.5f * P.hy, 0.5f * P.hz};

  // FP64 Gauss point coordinates, exactly as the definition rounds them
  if (FP64) {
    for (int q = lane; q < Q; q += 32) {
      int qx = q % NQ, qy = (q / NQ) % NQ, qz = q / (NQ * NQ);
      sm.xq[warp][q][0] = __dadd_rn(m.x0[0], __dmul_rn(m.h[0], __dadd_rn((double)ex, P.g[qx])));
      sm.xq[warp][q][1] = __dadd_rn(m.x0[1], __dmul_rn(m.h[1], __dadd_rn((double)ey, P.g[qy])));
      sm.xq[warp][q][2] = __dadd_rn(m.x0[2], __dmul_rn(m.h[2], __dadd_rn((double)ez, P.g[qz])));
    }
  }

  const double rmax = __longlong_as_double((long long)st->rmax_bits);
  const float cut = (float)(P.R + rmax) * (1.0f + 1e-5f);
  const float R32 = P.R32;
  const float band = 1.0f + P.delta;

  // bin range per axis (conservative)
  int blo[3], bhi[3];
  for (int a = 0; a < 3; ++a) {
    float lo = (c_hi[a] - hh[a] - cut) * P.inv_be[a];
    float hi = (c_hi[a] + hh[a] + cut) * P.inv_be[a];
    int l = (int)floorf(lo - 1e-3f), h = (int)floorf(hi + 1e-3f);
    blo[a] = l < 0 ? 0 : (l > b.nb[a] - 1 ? b.nb[a] - 1 : l);
    bhi[a] = h < 0 ? 0 : (h > b.nb[a] - 1 ? b.nb[a] - 1 : h);
  }

  // per-lane accumulators: quadrature points q0 = lane, q1 = lane + 32
  double acc64_0 = 0.0, acc64_1 = 0.0;
  float acc0 = 0.f, cmp0 = 0.f, acc1 = 0.f, cmp1 = 0.f;
  int cnt0 = 0, cnt1 = 0;
  long long ids0 = 0, ids1 = 0;
  const bool want_ids = nb_idsum != nullptr;
  int qn = 0;  // queue fill (warp-uniform)

  float4* cand = sm.cand[warp];
  int32_t* cslot = sm.cslot[warp];
  int32_t* queue = sm.queue[warp];

  // evaluate the first cnt queued pairs and hand the volumes to their owners
  auto flush = [&](int cnt) {
    double v64 = 0.0;
    float v32 = 0.f;
    int q = 0;
    long long pid = 0;
    if (lane < cnt) {
      int pk = queue[lane];
      q = pk & 63;
      int j = pk >> 6;
      if (FP64) {
        P4 pj = reinterpret_cast<const P4*>(xs64)[cslot[j]];
        double dx = __dsub_rn(pj.x, sm.xq[warp][q][0]);
        double dy = __dsub_rn(pj.y, sm.xq[warp][q][1]);
        double dz = __dsub_rn(pj.z, sm.xq[warp][q][2]);
        double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        v64 = lens64(P.R, pj.w, d2);
      } else {
        float4 cj = cand[j];
        float dx = cj.x - sm.qrel[q][0], dy = cj.y - sm.qrel[q][1], dz = cj.z - sm.qrel[q][2];
        v32 = lens32(R32, cj.w, dx * dx + dy * dy + dz * dz);
      }
      if (want_ids) pid = perm[cslot[j]];
    }
    for (int t = 0; t < cnt; ++t) {
      int qt = __shfl_sync(FULL, q, t);
      long long it = want_ids ? __shfl_sync(FULL, pid, t) : 0;
      if (FP64) {
        double vt = __shfl_sync(FULL, v64, t);
        if (qt == lane) { acc64_0 += vt; ++cnt0; ids0 += it; }
        if (Q > 32 && qt == lane + 32) { acc64_1 += vt; ++cnt1; ids1 += it; }
      } else {
        float vt = __shfl_sync(FULL, v32, t);
        if (qt == lane) { neumaier(acc0, cmp0, vt); ++cnt0; ids0 += it; }
        if (Q > 32 && qt == lane + 32) { neumaier(acc1, cmp1, vt); ++cnt1; ids1 += it; }
      }
    }
    __syncwarp();
  };

  // test all (q, candidate) pairs of the staged chunk
  auto process_chunk = [&](int nc) {
    const int total = nc * Q;
    for (int base = 0; base < total; base += 32) {
      int idx = base + lane;
      bool hit = false;
      int j = 0, q = 0;
      if (idx < total) {
        j = idx / Q;
        q = idx - j * Q;
        float4 cj = cand[j];
        float dx = cj.x - sm.qrel[q][0], dy = cj.y - sm.qrel[q][1], dz = cj.z - sm.qrel[q][2];
        float d2 = dx * dx + dy * dy + dz * dz;
        float c = R32 + cj.w;
        float c2 = c * c;
        if (FP64) {
          if (d2 * band < c2) {
            hit = true;
          } else if (d2 > c2 * band) {
            hit = false;
          } else {  // inside the band: exact FP64 predicate
            P4 pj = reinterpret_cast<const P4*>(xs64)[cslot[j]];
            double ddx = __dsub_rn(pj.x, sm.xq[warp][q][0]);
            double ddy = __dsub_rn(pj.y, sm.xq[warp][q][1]);
            double ddz = __dsub_rn(pj.z, sm.xq[warp][q][2]);
            double dd2 =
                __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
            double cc = __dadd_rn(P.R, pj.w);
            hit = dd2 < __dmul_rn(cc, cc);
          }
        } else {
          hit = d2 < c2;
        }
      }
      unsigned mask = __ballot_sync(FULL, hit);
      if (hit) queue[qn + __popc(mask & lt_mask)] = (j << 6) | q;
      qn += __popc(mask);
      __syncwarp();
      if (qn >= 32) {
        flush(32);
        int rest = qn - 32;
        int tmp = lane < rest ? queue[32 + lane] : 0;
        __syncwarp();
        if (lane < rest) queue[lane] = tmp;
        __syncwarp();
        qn = rest;
      }
    }
    if (qn > 0) {
      flush(qn);
      qn = 0;
    }
  };

  int nc = 0;
  for (int bz = blo[2]; bz <= bhi[2]; ++bz) {
    for (int by = blo[1]; by <= bhi[1]; ++by) {
      int64_t row = (int64_t)b.nb[0] * (by + (int64_t)b.nb[1] * bz);
      int s0 = bin_start[row + blo[0]], s1 = bin_start[row + bhi[0] + 1];
      for (int sb = s0; sb < s1; sb += 32) {
        int s = sb + lane;
        bool keep = false;
        float4 rel = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s < s1) {
          const float4* p = reinterpret_cast<const float4*>(xs32) + 2 * (int64_t)s;
          float4 hi = p[0], lo = p[1];
          rel.x = (hi.x - c_hi[0]) + (lo.x - c_lo[0]);
          rel.y = (hi.y - c_hi[1]) + (lo.y - c_lo[1]);
          rel.z = (hi.z - c_hi[2]) + (lo.z - c_lo[2]);
          rel.w = hi.w;
          float ox = fmaxf(fabsf(rel.x) - hh[0], 0.f);
          float oy = fmaxf(fabsf(rel.y) - hh[1], 0.f);
          float oz = fmaxf(fabsf(rel.z) - hh[2], 0.f);
          float c = (R32 + rel.w) * band;
          keep = ox * ox + oy * oy + oz * oz < c * c * band;
        }
        unsigned mask = __ballot_sync(FULL, keep);
        if (keep) {
          int pos = nc + __popc(mask & lt_mask);
          cand[pos] = rel;
          cslot[pos] = s;
        }
        nc += __popc(mask);
        __syncwarp();
        if (nc > kQcmChunk - 32) {
          process_chunk(nc);
          nc = 0;
        }
      }
    }
  }
  if (nc > 0) process_chunk(nc);

  // outputs
  const int64_t o = e * Q;
  if (lane < Q) {
    double eps;
    if (FP64) {
      eps = 1.0 - acc64_0 * P.inv_vr;
      if (eps64) eps64[o + lane] = eps;
    } else {
      float v = 1.0f - (acc0 + cmp0) * P.inv_vr32;
      if (eps32) eps32[o + lane] = v;
      if (eps64) eps64[o + lane] = (double)v;
    }
    if (nb_count) nb_count[o + lane] = cnt0;
    if (nb_idsum) nb_idsum[o + lane] = ids0;
  }
  if (Q > 32 && lane + 32 < Q) {
    if (FP64) {
      if (eps64) eps64[o + lane + 32] = 1.0 - acc64_1 * P.inv_vr;
    } else {
      float v = 1.0f - (acc1 + cmp1) * P.inv_vr32;
      if (eps32) eps32[o + lane + 32] = v;
      if (eps64) eps64[o + lane + 32] = (double)v;
    }
    if (nb_count) nb_count[o + lane + 32] = cnt1;
    if (nb_idsum) nb_idsum[o + lane + 32] = ids1;
  }
}

static void split_ff(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

cudaError_t launch_qcm(const MeshDev& m, const Tables& t, const BinDev& b, int precision,
                       double R, const int32_t* bin_start, const int32_t* perm,
                       const double* xs64, const float* xs32, const DevStatus* st,
                       double* eps_q64, float* eps_q32, int32_t* nb_count, int64_t* nb_idsum,
                       cudaStream_t s) {
  QcmParams P;
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
  for (int a = 0; a < 4; ++a) P.g[a] = t.g[a];
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
  dim3 grid((unsigned)((m.E + kQcmWarps - 1) / kQcmWarps));
  dim3 block(kQcmWarps * 32);
  bool fp64 = precision == 0;
#define CFDEM_QCM(KK)                                                                     \
  if (m.k == KK) {                                                                        \
    if (fp64)                                                                             \
      k_qcm<KK, true><<<grid, block, 0, s>>>(m, P, b, bin_start, perm, xs64, xs32, st,    \
                                             eps_q64, eps_q32, nb_count, nb_idsum);       \
    else                                                                                  \
      k_qcm<KK, false><<<grid, block, 0, s>>>(m, P, b, bin_start, perm, xs64, xs32, st,   \
                                              eps_q64, eps_q32, nb_count, nb_idsum);      \
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
