// cfdem_api.cu -- host runtime behind the C ABI of include/cfdem.h.
//
// A context owns: the mesh and its 1D reference tables, the resolved
// parameters, the bin grid, the scratch arenas (grown on demand) and the
// device status words.  Every call is ordered on the context's stream.
#include <atomic>
#include <chrono>
#include <mutex>
#include <vector>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/cfdem.h"
#include "internal.h"
#include "context.h"

using namespace cfdem;

// ---------------------------------------------------------------- timers
namespace cfdem {

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

void Timer::create() {
  for (int s = 0; s < kStages; ++s) {
    if (ev[s]) continue;
    ev[s] = new cudaEvent_t[2 * kCap];
    for (int i = 0; i < 2 * kCap; ++i) cudaEventCreate(&ev[s][i]);
  }
}

void Timer::begin(int s, cudaStream_t st) {
  if (!on || !ev[s]) return;
  if (count[s] >= kCap) {
    overflow = true;
    return;
  }
  cudaEventRecord(ev[s][2 * count[s]], st);
}

void Timer::end(int s, cudaStream_t st) {
  if (!on || !ev[s] || count[s] >= kCap) return;
  cudaEventRecord(ev[s][2 * count[s] + 1], st);
  ++count[s];
  ++calls[s];
}

void Timer::collect() {
  for (int s = 0; s < kStages; ++s) {
    for (int i = 0; i < count[s]; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[s][2 * i], ev[s][2 * i + 1]) == cudaSuccess) ms[s] += t;
    }
    count[s] = 0;
  }
}

void Timer::release() {
  for (int s = 0; s < kStages; ++s) {
    if (!ev[s]) continue;
    for (int i = 0; i < 2 * kCap; ++i) cudaEventDestroy(ev[s][i]);
    delete[] ev[s];
    ev[s] = nullptr;
  }
}

}  // namespace cfdem

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cfdem_status fail(cfdem_t c, cfdem_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

cfdem_status cuda_fail(cfdem_t c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(c, CFDEM_ENOMEM, "%s: out of device memory", where);
  return fail(c, CFDEM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// the force kernels' parameters from the context's parameters and mesh
// the integer key of a double whose signed order is the order of the values
// (the same map the device applies to a particle coordinate)
long long order_key(double v) {
  long long b;
  std::memcpy(&b, &v, sizeof b);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

ForceParams force_params(const cfdem_ctx* c) {
  ForceParams fp{};
  fp.rho = c->prm.rho_f;
  fp.mu = c->prm.mu_f;
  for (int a = 0; a < 3; ++a) {
    fp.g[a] = c->prm.g[a];
    fp.inv_h[a] = 1.0 / c->mesh.h[a];
  }
  fp.eps_floor = c->prm.eps_floor;
  fp.drag_model = c->prm.drag_model;
  fp.beta_over_eps = c->prm.beta_over_eps;
  fp.vans_model = c->prm.vans_model;
  fp.shear = c->prm.shear_force;
  fp.fluid_drag = c->prm.fluid_drag;
  fp.rho32 = (float)fp.rho;
  fp.mu32 = (float)fp.mu;
  fp.eps_floor32 = (float)fp.eps_floor;
  double far = 0.0;
  for (int a = 0; a < 3; ++a) {
    const MeshDev& m = c->mesh;
    fp.g32[a] = (float)fp.g[a];
    fp.inv_h32[a] = (float)fp.inv_h[a];
    fp.x0_hi[a] = (float)m.x0[a];
    fp.x0_lo[a] = (float)(m.x0[a] - (double)fp.x0_hi[a]);
    fp.inv_h_hi[a] = (float)fp.inv_h[a];
    fp.inv_h_lo[a] = (float)(fp.inv_h[a] - (double)fp.inv_h_hi[a]);
    fp.nem1f[a] = (float)(m.ne[a] - 1);
    // the bounds of in_box, rounded as the device rounds them
    volatile double slack = 1e-12 * m.L[a];
    volatile double top = m.x0[a] + m.L[a];
    const double lo = m.x0[a] - slack, hi = top + slack;
    fp.box_lo_key[a] = order_key(lo);
    fp.box_hi_key[a] = order_key(hi);
    far = std::fmax(far, (std::fabs(m.x0[a]) + m.L[a]) * fp.inv_h[a]);
  }
  // the double-float location is accurate to ~2^-46 (|x| / h); with its
  // 1e-5 margin around element faces it holds while |x| / h < 2^26
  fp.loc32 = far < 67108864.0 ? 1 : 0;
  return fp;
}

SemiAcc semi_acc(const cfdem_ctx* c) {
  const int64_t E = c->mesh.E;
  return SemiAcc{c->semi, c->semi + E, c->semi + 4 * E};
}

#define CK(expr, where)                                  \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

template <typename T>
cudaError_t grow(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

// ---------------------------------------------------------------- 1D tables
// Gauss-Legendre points and weights on [-1,1] in closed form (n <= 4), GLL
// nodes (roots of P_k' plus end points) in closed form (k <= 3).
void gauss_closed_form(int n, double* s, double* w) {
  switch (n) {
    case 1:
      s[0] = 0.0;
      w[0] = 2.0;
      break;
    case 2: {
      double a = 1.0 / std::sqrt(3.0);
      s[0] = -a;
      s[1] = a;
      w[0] = w[1] = 1.0;
      break;
    }
    case 3: {
      double a = std::sqrt(0.6);
      s[0] = -a;
      s[1] = 0.0;
      s[2] = a;
      w[0] = w[2] = 5.0 / 9.0;
      w[1] = 8.0 / 9.0;
      break;
    }
    default: {  // 4
      double r = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
      double a = std::sqrt(3.0 / 7.0 - r), bb = std::sqrt(3.0 / 7.0 + r);
      double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
      s[0] = -bb;
      s[1] = -a;
      s[2] = a;
      s[3] = bb;
      w[0] = w[3] = wb;
      w[1] = w[2] = wa;
      break;
    }
  }
}

void gll_closed_form(int k, double* z) {
  z[0] = 0.0;
  z[k] = 1.0;
  if (k == 2) z[1] = 0.5;
  if (k == 3) {
    double a = 0.5 / std::sqrt(5.0);
    z[1] = 0.5 - a;
    z[2] = 0.5 + a;
  }
}

void bary_weights(int k, const double* z, double* lw) {
  for (int a = 0; a <= k; ++a) {
    double p = 1.0;
    for (int bb = 0; bb <= k; ++bb)
      if (bb != a) p *= (z[a] - z[bb]);
    lw[a] = 1.0 / p;
  }
}

void lagr(int k, const double* z, const double* lw, double t, double* l, double* dl) {
  for (int a = 0; a <= k; ++a) {
    double v = 1.0, dv = 0.0;
    for (int bb = 0; bb <= k; ++bb) {
      if (bb == a) continue;
      dv = dv * (t - z[bb]) + v;
      v = v * (t - z[bb]);
    }
    l[a] = v * lw[a];
    dl[a] = dv * lw[a];
  }
}

void build_tables(int k, int kp, Tables* t) {
  std::memset(t, 0, sizeof(Tables));
  int nq = k + 1;
  double s[4], w[4];
  gauss_closed_form(nq, s, w);
  for (int q = 0; q < nq; ++q) {
    t->g[q] = 0.5 * (1.0 + s[q]);
    t->w[q] = 0.5 * w[q];
  }
  gll_closed_form(k, t->z);
  gll_closed_form(kp, t->zp);
  bary_weights(k, t->z, t->lw);
  bary_weights(kp, t->zp, t->lwp);
  for (int a = 0; a < 4; ++a) {
    t->zf[a] = (float)t->z[a];
    t->zpf[a] = (float)t->zp[a];
    t->lwf[a] = (float)t->lw[a];
    t->lwpf[a] = (float)t->lwp[a];
    t->z_lo[a] = (float)(t->z[a] - (double)t->zf[a]);
    t->lw_lo[a] = (float)(t->lw[a] - (double)t->lwf[a]);
  }
  double l[4][4], dl[4][4];  // [q][a]
  for (int q = 0; q < nq; ++q) lagr(k, t->z, t->lw, t->g[q], l[q], dl[q]);
  for (int a = 0; a <= k; ++a)
    for (int q = 0; q < nq; ++q) {
      t->Bw[a][q] = l[q][a] * t->w[q];
      t->Bwf[a][q] = (float)t->Bw[a][q];
    }
  // exact with nq = k + 1 Gauss points (degree 2k integrands)
  for (int a = 0; a <= k; ++a)
    for (int bb = 0; bb <= k; ++bb) {
      double m = 0.0, kk = 0.0;
      for (int q = 0; q < nq; ++q) {
        m += t->w[q] * l[q][a] * l[q][bb];
        kk += t->w[q] * dl[q][a] * dl[q][bb];
      }
      t->Mh[a][bb] = m;
      t->Kh[a][bb] = kk;
    }
}

bool is_finite_d(double v) { return std::isfinite(v); }

// the bin grid of edge ~edge over the box: floor(L / edge) bins per axis
// (at least one), coarsened by 1.5 until at most 2^26 bins
BinDev bin_grid(const MeshDev& m, double edge) {
  BinDev b{};
  for (;;) {
    int64_t tot = 1;
    for (int a = 0; a < 3; ++a) {
      double f = std::floor(m.L[a] / edge);
      int nb = f < 1.0 ? 1 : (f > 1e6 ? 1000000 : (int)f);
      b.nb[a] = nb;
      b.be[a] = m.L[a] / nb;
      b.inv_be[a] = 1.0 / b.be[a];
      tot *= nb;
    }
    b.nbins = tot;
    if (tot <= (int64_t)1 << 26) break;
    edge *= 1.5;
  }
  double far = 0.0;
  for (int a = 0; a < 3; ++a) {
    b.x0_hi[a] = (float)m.x0[a];
    b.x0_lo[a] = (float)(m.x0[a] - (double)b.x0_hi[a]);
    b.inv_be_hi[a] = (float)b.inv_be[a];
    b.inv_be_lo[a] = (float)(b.inv_be[a] - (double)b.inv_be_hi[a]);
    volatile double slack = 1e-12 * m.L[a];
    volatile double top = m.x0[a] + m.L[a];
    b.box_lo_key[a] = order_key(m.x0[a] - slack);
    b.box_hi_key[a] = order_key(top + slack);
    b.nm1f[a] = (float)(b.nb[a] - 1);
    far = std::fmax(far, (std::fabs(m.x0[a]) + m.L[a]) * b.inv_be[a]);
  }
  b.loc32 = far < 67108864.0 ? 1 : 0;  // |x| / be < 2^26: see elem_axis_df
  return b;
}

// room for the bin counts and starts of the current grid
cfdem_status ensure_bins(cfdem_t c) {
  if (c->bins.nbins + 1 > c->cap_bins) {
    int64_t nb = c->bins.nbins + 1;
    CK(grow(&c->bin_count, nb), "bins");
    CK(grow(&c->bin_start, nb), "bins");
    CK(grow(&c->scan_tmp, nb / 2048 + 2), "bins");
    c->cap_bins = nb;
  }
  return CFDEM_OK;
}

// resolve R, kp, coefficients and the bin grid once mesh and params exist
cfdem_status resolve(cfdem_t c) {
  if (!c->have_mesh) return CFDEM_OK;
  MeshDev& m = c->mesh;
  cfdem_params& p = c->prm;
  int kp = p.pressure_degree > 0 ? p.pressure_degree : (m.k > 1 ? m.k - 1 : 1);
  if (kp < 1 || kp > 3) return fail(c, CFDEM_EINVAL, "pressure_degree must be 1..3");
  m.kp = kp;
  for (int a = 0; a < 3; ++a) m.np[a] = m.ne[a] * kp + 1;
  m.n_pnodes = (int64_t)m.np[0] * m.np[1] * m.np[2];
  build_tables(m.k, kp, &c->tab);
  c->R = p.qcm_radius > 0 ? p.qcm_radius : std::cbrt(3.0 * m.Ve / (4.0 * kPi));
  double L2 = p.l2_smoothing;
  c->coef[0] = m.h[0] * m.h[1] * m.h[2];
  c->coef[1] = L2 * m.h[1] * m.h[2] / m.h[0];
  c->coef[2] = L2 * m.h[0] * m.h[2] / m.h[1];
  c->coef[3] = L2 * m.h[0] * m.h[1] / m.h[2];
  double edge = p.bin_edge > 0 ? p.bin_edge : c->R + (p.max_radius > 0 ? p.max_radius : c->R);
  c->bins = bin_grid(m, edge);
  c->bin_key_set = false;
  c->shape_key_set = false;
  c->tuned = 0;
  m.shape = pick_shape(m);
  DeviceGuard g(c->device);
  CK(upload_bands(m, c->tab, L2, &c->bands64, &c->bands32, &c->bandsdf), "upload_bands");
  c->cg.bands_df = reinterpret_cast<const df64*>(c->bandsdf);
  if (c->fdm) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    fdm_destroy(c->fdm);
    c->fdm = nullptr;
  }
  c->fdm_note = "";
  if (p.cg_precond == 1) {
    const char* why = nullptr;
    CK(fdm_create(m, c->tab, c->coef, &c->fdm, &why), "fdm_create");
    if (!c->fdm) c->fdm_note = why ? why : "FDM unavailable";
  }
  c->cg.fdm = c->fdm;
  cfdem_status s = ensure_bins(c);
  if (s != CFDEM_OK) return s;
  c->eps_state = 0;
  return CFDEM_OK;
}

cfdem_status ensure_particles(cfdem_t c, int64_t n) {
  if (n <= c->cap_n) return CFDEM_OK;
  int64_t cap = n + n / 4 + 1024;
  CK(grow(&c->bin_of, cap), "particle arena");
  CK(grow(&c->slot, cap), "particle arena");
  CK(grow(&c->perm, cap), "particle arena");
  CK(grow(&c->xs64, 4 * cap), "particle arena");
  CK(grow(&c->xs32, 8 * cap), "particle arena");
  CK(grow(&c->qcm_w, 2 * cap), "particle arena");
  CK(grow(&c->psrc, 4 * cap), "particle arena");
  CK(grow(&c->pelem, cap), "particle arena");
  c->cap_n = cap;
  return CFDEM_OK;
}

void free_mesh_arena(cfdem_t c) {
  void* ps[] = {c->eps64, c->eps32, c->b, c->S, c->vol, c->cg.r, c->cg.z, c->cg.p0,
                c->cg.p1, c->cg.Ap, c->cg.dinv, c->cg.xcor, c->cg.r32, c->cg.z32,
                c->cg.q0, c->cg.q1, c->cg.Aq, c->cg.dinv32, c->cg.d32, c->cg.partials,
                c->cg.sc, c->cg.zn, c->cg.zn32, c->cg.rin32, c->cg.x_df, c->cg.r_df,
                c->cg.Ap_df, c->cg.p0_df, c->cg.p1_df, c->adj_geps,
                c->adj_lam, c->adj_gq, c->rhs_local, c->semi, c->tune_x, c->src_acc,
                c->src_max, c->nodal_df};
  for (void* p : ps)
    if (p) cudaFree(p);
  c->tune_x = nullptr;
  c->shape_key_set = false;
  c->eps64 = nullptr;
  c->eps32 = nullptr;
  c->b = nullptr;
  c->S = nullptr;
  c->vol = nullptr;
  c->adj_geps = c->adj_lam = c->adj_gq = nullptr;
  c->rhs_local = nullptr;
  c->semi = nullptr;
  c->src_acc = nullptr;
  c->src_max = nullptr;
  c->nodal_df = nullptr;
  c->semi_valid = 0;
  FdmPlan* keep = c->cg.fdm;
  const df64* kb = c->cg.bands_df;
  c->cg = CgWork{};
  c->cg.fdm = keep;
  c->cg.bands_df = kb;
}

cfdem_status alloc_mesh_arena(cfdem_t c) {
  const MeshDev& m = c->mesh;
  int64_t eq = m.E * m.Q, nn = m.n_nodes;
  CK(grow(&c->eps64, eq), "mesh arena");
  CK(grow(&c->eps32, eq), "mesh arena");
  CK(grow(&c->b, nn), "mesh arena");
  CK(grow(&c->S, 3 * m.E), "mesh arena");
  CK(grow(&c->vol, m.E), "mesh arena");
  CK(grow(&c->rhs_local, m.E * (int64_t)(m.k + 1) * (m.k + 1) * (m.k + 1)), "mesh arena");
  CK(grow(&c->semi, 5 * m.E), "mesh arena");
  CK(grow(&c->src_acc, 16 * m.E), "mesh arena");
  CK(grow(&c->src_max, 4), "mesh arena");
  c->semi_valid = 0;
  CgWork& w = c->cg;
  CK(grow(&w.r, nn), "cg");
  CK(grow(&w.z, nn), "cg");
  CK(grow(&w.p0, nn), "cg");
  CK(grow(&w.p1, nn), "cg");
  CK(grow(&w.Ap, nn), "cg");
  CK(grow(&w.dinv, nn), "cg");
  CK(grow(&w.r32, nn), "cg");
  CK(grow(&w.z32, nn), "cg");
  CK(grow(&w.q0, nn), "cg");
  CK(grow(&w.q1, nn), "cg");
  CK(grow(&w.Aq, nn), "cg");
  CK(grow(&w.dinv32, nn), "cg");
  CK(grow(&w.d32, nn), "cg");
  CK(grow(&w.zn, nn), "cg");
  CK(grow(&w.zn32, nn), "cg");
  CK(grow(&w.rin32, nn), "cg");
  {
    float* t = nullptr;
    CK(grow(&t, 2 * nn), "cg");
    w.x_df = reinterpret_cast<df64*>(t);
    t = nullptr;
    CK(grow(&t, 2 * nn), "cg");
    w.r_df = reinterpret_cast<df64*>(t);
    t = nullptr;
    CK(grow(&t, 2 * nn), "cg");
    w.Ap_df = reinterpret_cast<df64*>(t);
    t = nullptr;
    CK(grow(&t, 2 * nn), "cg");
    w.p0_df = reinterpret_cast<df64*>(t);
    t = nullptr;
    CK(grow(&t, 2 * nn), "cg");
    w.p1_df = reinterpret_cast<df64*>(t);
  }
  w.nblocks = cg_blocks(m);
  CK(grow(&w.partials, 4 * (size_t)w.nblocks), "cg");
  CK(grow(&w.sc, 1), "cg");
  return CFDEM_OK;
}

// statistics of a solve that ran inside a graph, from the device scalars
// (the stream has been synchronised)
cudaError_t read_pending_stats(cfdem_t c) {
  if (!c->stats_pending || !c->cg.sc) return cudaSuccess;
  CgScalars hs;
  cudaError_t e = cudaMemcpy(&hs, c->cg.sc, sizeof hs, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  double bb = hs.bb > 0 ? hs.bb : 1.0;
  c->last_iters = hs.it;
  c->last_outer = c->prm.precision == 1 ? hs.it : 0;
  c->last_relres = std::sqrt(hs.rr / bb);
  c->last_converged = c->last_relres <= c->prm.cg_rtol;
  if (!c->last_converged) c->pending_not_converged = 1;
  c->stats_pending = false;
  return cudaSuccess;
}

cfdem_status need_mesh(cfdem_t c) {
  if (!c) return CFDEM_EINVAL;
  if (!c->have_mesh) return fail(c, CFDEM_ESTATE, "cfdem_set_mesh has not been called");
  return CFDEM_OK;
}

// bin the particles into the context arena (step a2)
cfdem_status do_bin(cfdem_t c, int64_t n, const double* x, const double* r) {
  cfdem_status s = ensure_particles(c, n);
  if (s != CFDEM_OK) return s;
  c->timer.begin(kStageBin, c->stream);
  CK(cudaMemsetAsync(&c->st->rmax_bits, 0, sizeof(unsigned long long), c->stream), "bin");
  CK(launch_bin(c->mesh, c->bins, n, x, r, c->bin_of, c->slot, c->bin_count, c->bin_start,
                c->perm, c->scan_tmp, c->xs64, c->xs32, c->st, c->stream),
     "bin");
  c->timer.end(kStageBin, c->stream);
  return CFDEM_OK;
}

// (M + L^2 K) x = b by the context's CG (x: start vector in, solution out).
// Inside a stream capture the CG iterates on the device (a conditional node
// of the graph) and its statistics are read at the next synchronise.
cfdem_status solve(cfdem_t c, const double* b, double* x, const char* what) {
  int it = 0, outer = 0, conv = 0;
  double rel = 0.0;
  cudaError_t e;
  const bool captured = stream_capturing(c->stream);
  if (captured && c->timer.on)
    return fail(c, CFDEM_ESTATE, "stage timers must be off while the stream is captured");
  c->cg.loop = captured ? c->loop_stream : nullptr;
  c->cg.timer = c->timer.on ? &c->timer : nullptr;
  c->timer.begin(kStageSolve, c->stream);
  if (c->prm.precision == 1)
    e = run_cg_mixed(c->mesh, c->bands64, c->bands32, c->coef, b, x, c->prm.cg_rtol,
                     c->prm.cg_maxit, c->cg, c->stream, &it, &outer, &rel, &conv);
  else
    e = run_cg64(c->mesh, c->bands64, c->coef, b, x, c->prm.cg_rtol, c->prm.cg_maxit, c->cg,
                 c->stream, &it, &rel, &conv);
  c->cg.loop = nullptr;
  if (e == cudaErrorNotSupported && captured)
    return fail(c, CFDEM_ESTATE,
                "a captured mixed-precision solve needs the fast-diagonalisation preconditioner");
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  c->timer.end(kStageSolve, c->stream);
  if (captured) {
    c->stats_pending = true;
    return CFDEM_OK;
  }
  c->stats_pending = false;
  c->last_iters = it;
  c->last_outer = outer;
  c->last_relres = rel;
  c->last_converged = conv;
  if (!conv) c->pending_not_converged = 1;
  return CFDEM_OK;
}


// ---------------------------------------------------------------- autotuner
// The bin edge of the QCM's particle bins and the tile shape of the
// projection operator decide how much work the void fraction and the solve
// do but not what they compute.  With autotune = 1 the first eager call of a
// new signature times a few candidates on the actual inputs (CUDA events on
// the context's stream, two timed runs after one warm-up, the faster kept)
// and keeps the fastest; the choice is cached per process by signature.

std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, double>> g_bin_choice;  // signature -> bin edge
std::vector<std::pair<TuneKey, int>> g_shape_choice;   // signature -> tile shape

bool same_key(const TuneKey& a, const TuneKey& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

TuneKey base_key(const cfdem_ctx* c) {
  TuneKey k;
  std::memset(&k, 0, sizeof k);
  const MeshDev& m = c->mesh;
  for (int a = 0; a < 3; ++a) {
    k.ne[a] = m.ne[a];
    k.L[a] = m.L[a];
  }
  k.k = m.k;
  k.precision = c->prm.precision;
  return k;
}

double host_ms_since(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// device time of fn() on the stream: one warm-up run, then the faster of two
template <class F>
cudaError_t time_on_stream(cudaStream_t s, F&& fn, float* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = FLT_MAX;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess && rep > 0 && t < best) best = t;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  *ms_out = best;
  return e;
}

// bin edge: candidates R + r_max (the default) and its 1/1.5, 1/2, 1/3, and
// the element edge h and h/2, h/3 (bins nested in elements); each timed on
// binning + QCM of the call's particles
cfdem_status tune_bins(cfdem_t c, int64_t n, const double* x, const double* r) {
  const cfdem_params& p = c->prm;
  if (!p.autotune || p.bin_edge > 0 || p.scheme != 0 || n <= 0) return CFDEM_OK;
  if (stream_capturing(c->stream)) return CFDEM_OK;
  TuneKey key = base_key(c);
  key.variant = p.qcm_conserve;
  key.nbucket = 63 - __builtin_clzll((unsigned long long)n);
  key.R = c->R;
  key.rmax = p.max_radius;
  if (c->bin_key_set && same_key(c->bin_key, key)) return CFDEM_OK;
  const auto t0 = std::chrono::steady_clock::now();
  const MeshDev& m = c->mesh;
  double edge = -1.0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : g_bin_choice)
      if (same_key(kv.first, key)) edge = kv.second;
  }
  cfdem_status s;
  if (edge <= 0) {
    const double cut = c->R + (p.max_radius > 0 ? p.max_radius : c->R);
    const double hmin = std::fmin(m.h[0], std::fmin(m.h[1], m.h[2]));
    const double cand[] = {cut, cut / 1.5, cut / 2.0, cut / 3.0, hmin, hmin / 2.0, hmin / 3.0};
    const bool mixed = p.precision == 1;
    const bool conserve = p.qcm_conserve == 1;
    const bool timer_on = c->timer.on;
    c->timer.on = false;
    std::vector<BinDev> seen;
    float best = FLT_MAX;
    edge = cut;
    for (double ed : cand) {
      const BinDev g = bin_grid(m, ed);
      bool dup = g.nbins > ((int64_t)1 << 24);
      for (const BinDev& o : seen)
        dup = dup || (o.nb[0] == g.nb[0] && o.nb[1] == g.nb[1] && o.nb[2] == g.nb[2]);
      if (dup) continue;
      seen.push_back(g);
      c->bins = g;
      s = ensure_bins(c);
      if (s != CFDEM_OK) {
        c->timer.on = timer_on;
        return s;
      }
      float ms = FLT_MAX;
      cudaError_t e = time_on_stream(c->stream, [&]() -> cudaError_t {
        if (do_bin(c, n, x, r) != CFDEM_OK) return cudaErrorUnknown;
        return launch_qcm(m, c->tab, c->bins, mixed ? 1 : 0, c->R, c->bin_start, c->perm,
                          c->xs64, c->xs32, c->st, mixed ? nullptr : c->eps64,
                          mixed ? c->eps32 : nullptr, nullptr, nullptr, c->stream,
                          conserve ? reinterpret_cast<float2*>(c->qcm_w) : nullptr,
                          conserve ? n : 0);
      }, &ms);
      if (e != cudaSuccess) {
        c->timer.on = timer_on;
        return cuda_fail(c, e, "autotune bins");
      }
      if (ms < best) {
        best = ms;
        edge = ed;
      }
    }
    c->timer.on = timer_on;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_bin_choice.emplace_back(key, edge);
  }
  c->bins = bin_grid(m, edge);
  s = ensure_bins(c);
  if (s != CFDEM_OK) return s;
  c->bin_key = key;
  c->bin_key_set = true;
  c->tuned |= 1;
  c->tune_ms += host_ms_since(t0);
  return CFDEM_OK;
}

// tile shape of the operator: each shape that fits in shared memory timed on
// the solve of the call's right-hand side (from zero, into a scratch vector)
cfdem_status tune_shape(cfdem_t c, const double* b) {
  const cfdem_params& p = c->prm;
  if (!p.autotune || stream_capturing(c->stream)) return CFDEM_OK;
  TuneKey key = base_key(c);
  key.variant = c->fdm ? 1 : 0;
  for (int a = 0; a < 4; ++a) key.coef[a] = c->coef[a];
  if (c->shape_key_set && same_key(c->shape_key, key)) return CFDEM_OK;
  const auto t0 = std::chrono::steady_clock::now();
  MeshDev& m = c->mesh;
  int shape = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : g_shape_choice)
      if (same_key(kv.first, key)) shape = kv.second;
  }
  if (shape < 0) {
    CK(grow(&c->tune_x, m.n_nodes), "autotune scratch");
    Timer* tm = c->cg.timer;
    cudaStream_t loop = c->cg.loop;
    c->cg.timer = nullptr;
    c->cg.loop = nullptr;
    float best = FLT_MAX;
    shape = m.shape;
    for (int sh = 0; sh < 3; ++sh) {
      if (!shape_fits(m, sh)) continue;
      m.shape = sh;
      float ms = FLT_MAX;
      cudaError_t e = time_on_stream(c->stream, [&]() -> cudaError_t {
        cudaError_t ee = cudaMemsetAsync(c->tune_x, 0, sizeof(double) * m.n_nodes, c->stream);
        if (ee != cudaSuccess) return ee;
        int it = 0, outer = 0, conv = 0;
        double rel = 0.0;
        if (p.precision == 1)
          return run_cg_mixed(m, c->bands64, c->bands32, c->coef, b, c->tune_x, p.cg_rtol,
                              p.cg_maxit, c->cg, c->stream, &it, &outer, &rel, &conv);
        return run_cg64(m, c->bands64, c->coef, b, c->tune_x, p.cg_rtol, p.cg_maxit, c->cg,
                        c->stream, &it, &rel, &conv);
      }, &ms);
      if (e != cudaSuccess) {
        c->cg.timer = tm;
        c->cg.loop = loop;
        return cuda_fail(c, e, "autotune tile shape");
      }
      if (ms < best) {
        best = ms;
        shape = sh;
      }
    }
    c->cg.timer = tm;
    c->cg.loop = loop;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_shape_choice.emplace_back(key, shape);
  }
  m.shape = shape;
  c->shape_key = key;
  c->shape_key_set = true;
  c->tuned |= 2;
  c->tune_ms += host_ms_since(t0);
  return CFDEM_OK;
}

}  // namespace

namespace cfdem {
// the 1D reference tables of degree k (and kp) for other translation units
void make_tables(int k, int kp, Tables* t) { build_tables(k, kp, t); }
}  // namespace cfdem

// ============================================================== public API

extern "C" {

const char* cfdem_version(void) { return "cfdem-gb300 0.1 (sm_103a)"; }

void cfdem_params_default(cfdem_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->rho_f = 1.2;
  p->mu_f = 1.8e-5;
  p->g[0] = 0.0;
  p->g[1] = 0.0;
  p->g[2] = -9.81;
  p->scheme = 0;
  p->drag_model = 0;
  p->vans_model = 0;
  p->precision = 0;
  p->cg_rtol = 1e-13;
  p->cg_maxit = 2000;
  p->eps_floor = 0.05;
  p->cg_precond = 1;
  p->shear_force = 0;
  p->fluid_drag = 0;
  p->qcm_conserve = 0;
  p->autotune = 1;
}

cfdem_status cfdem_create(cfdem_t* out, int device, void* stream) {
  if (!out) return CFDEM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return CFDEM_ECUDA;
  cfdem_t c = new cfdem_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cfdem_params_default(&c->prm);
  DeviceGuard g(device);
  if (cudaMalloc((void**)&c->st, sizeof(DevStatus)) != cudaSuccess) {
    delete c;
    return CFDEM_ENOMEM;
  }
  DevStatus init{};
  init.first_bad = ~0ull;
  if (cudaMemcpy(c->st, &init, sizeof init, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->loop_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(c->st);
    delete c;
    return CFDEM_ECUDA;
  }
  *out = c;
  return CFDEM_OK;
}

cfdem_status cfdem_destroy(cfdem_t c) {
  if (!c) return CFDEM_OK;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_mesh_arena(c);
  if (c->fdm) fdm_destroy(c->fdm);
  c->fdm = nullptr;
  c->timer.release();
  void* ps[] = {c->st, c->bands64, c->bands32, c->bandsdf, c->bin_of, c->slot, c->perm, c->xs64,
                c->xs32, c->qcm_w, c->psrc, c->pelem, c->bin_count, c->bin_start,
                c->scan_tmp};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (c->loop_stream) cudaStreamDestroy(c->loop_stream);
  delete c;
  return CFDEM_OK;
}

cfdem_status cfdem_set_mesh(cfdem_t c, const double origin[3], const double extent[3],
                            const int n_el[3], int degree) {
  if (!c || !origin || !extent || !n_el) return fail(c, CFDEM_EINVAL, "null argument");
  if (degree < 1 || degree > 3) return fail(c, CFDEM_EINVAL, "degree must be 1, 2 or 3");
  MeshDev m{};
  for (int a = 0; a < 3; ++a) {
    if (!is_finite_d(origin[a]) || !is_finite_d(extent[a]) || !(extent[a] > 0))
      return fail(c, CFDEM_EINVAL, "origin/extent must be finite, extent > 0");
    if (n_el[a] < 1 || n_el[a] > (1 << 20)) return fail(c, CFDEM_EINVAL, "bad n_el");
    m.x0[a] = origin[a];
    m.L[a] = extent[a];
    m.ne[a] = n_el[a];
    m.h[a] = extent[a] / n_el[a];
    m.nn[a] = n_el[a] * degree + 1;
  }
  m.k = degree;
  m.nq = degree + 1;
  m.Q = m.nq * m.nq * m.nq;
  m.E = (int64_t)m.ne[0] * m.ne[1] * m.ne[2];
  m.n_nodes = (int64_t)m.nn[0] * m.nn[1] * m.nn[2];
  m.Ve = m.h[0] * m.h[1] * m.h[2];
  m.Ve32 = (float)m.Ve;
  if (m.E * m.Q > ((int64_t)1 << 31) || m.n_nodes > ((int64_t)1 << 31))
    return fail(c, CFDEM_EINVAL, "mesh too large");
  m.shape = pick_shape(m);
  ++c->gen;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_mesh_arena(c);
  c->mesh = m;
  c->have_mesh = true;
  cfdem_status s = alloc_mesh_arena(c);
  if (s != CFDEM_OK) {
    c->have_mesh = false;
    return s;
  }
  return resolve(c);
}

cfdem_status cfdem_set_params(cfdem_t c, const cfdem_params* p) {
  if (!c || !p) return fail(c, CFDEM_EINVAL, "null argument");
  if (!(p->rho_f > 0) || !(p->mu_f > 0) || !is_finite_d(p->g[0]) || !is_finite_d(p->g[1]) ||
      !is_finite_d(p->g[2]))
    return fail(c, CFDEM_EINVAL, "rho_f, mu_f must be > 0 and g finite");
  if (p->scheme < 0 || p->scheme > 1) return fail(c, CFDEM_EINVAL, "scheme must be 0 or 1");
  if (p->drag_model < 0 || p->drag_model > 5)
    return fail(c, CFDEM_EINVAL,
                "drag_model must be 0 (Di Felice), 1 (Dallavalle), 2 (Rong), 3 (Koch-Hill), "
                "4 (Gidaspow) or 5 (Beetstra)");
  if (p->vans_model < 0 || p->vans_model > 1) return fail(c, CFDEM_EINVAL, "vans_model 0|1");
  if (p->precision < 0 || p->precision > 1) return fail(c, CFDEM_EINVAL, "precision 0|1");
  if (!(p->qcm_radius >= 0) || !(p->l2_smoothing >= 0) || !(p->cg_rtol > 0) ||
      p->cg_maxit < 1 || !(p->eps_floor > 0 && p->eps_floor <= 1) || !(p->max_radius >= 0) ||
      !(p->bin_edge >= 0))
    return fail(c, CFDEM_EINVAL, "numerical parameter out of range");
  if (p->pressure_degree < 0 || p->pressure_degree > 3)
    return fail(c, CFDEM_EINVAL, "pressure_degree must be 0..3");
  if (p->cg_precond < 0 || p->cg_precond > 1)
    return fail(c, CFDEM_EINVAL, "cg_precond must be 0 (Jacobi) or 1 (FDM)");
  if (p->shear_force < 0 || p->shear_force > 1)
    return fail(c, CFDEM_EINVAL, "shear_force must be 0 or 1");
  if (p->fluid_drag < 0 || p->fluid_drag > 1)
    return fail(c, CFDEM_EINVAL, "fluid_drag must be 0 (explicit) or 1 (fluid-side form)");
  if (p->qcm_conserve < 0 || p->qcm_conserve > 1)
    return fail(c, CFDEM_EINVAL, "qcm_conserve must be 0 or 1");
  if (p->autotune < 0 || p->autotune > 1) return fail(c, CFDEM_EINVAL, "autotune must be 0 or 1");
  c->prm = *p;
  ++c->gen;
  return resolve(c);
}

cfdem_status cfdem_get_params(cfdem_t c, cfdem_params* p) {
  if (!c || !p) return CFDEM_EINVAL;
  *p = c->prm;
  if (c->have_mesh) {
    p->qcm_radius = c->R;
    p->pressure_degree = c->mesh.kp;
    p->bin_edge = c->bins.be[0];
  }
  return CFDEM_OK;
}

cfdem_status cfdem_locate(cfdem_t c, int64_t n, const double* x, int32_t* elem, double* xi) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (n < 0 || (n > 0 && !x)) return fail(c, CFDEM_EINVAL, "bad particle arrays");
  DeviceGuard g(c->device);
  CK(launch_locate(c->mesh, n, x, elem, xi, c->st, c->stream), "locate");
  return CFDEM_OK;
}

cfdem_status cfdem_bin(cfdem_t c, int64_t n, const double* x, int32_t* bin_start,
                       int32_t* perm) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && !x))
    return fail(c, CFDEM_EINVAL, "bad particle arrays");
  DeviceGuard g(c->device);
  s = do_bin(c, n, x, nullptr);  // radii are not needed for the sort itself
  if (s != CFDEM_OK) return s;
  if (bin_start)
    CK(cudaMemcpyAsync(bin_start, c->bin_start, sizeof(int32_t) * (c->bins.nbins + 1),
                       cudaMemcpyDeviceToDevice, c->stream),
       "bin copy");
  if (perm && n > 0)
    CK(cudaMemcpyAsync(perm, c->perm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream),
       "bin copy");
  return CFDEM_OK;
}

cfdem_status cfdem_void_fraction(cfdem_t c, int64_t n, const double* x, const double* r,
                                 double* eps_q, int32_t* nb_count, int64_t* nb_idsum) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!x || !r)))
    return fail(c, CFDEM_EINVAL, "bad particle arrays");
  DeviceGuard g(c->device);
  const MeshDev& m = c->mesh;
  bool mixed = c->prm.precision == 1;
  double* out64 = eps_q ? eps_q : (mixed ? nullptr : c->eps64);
  float* out32 = mixed ? c->eps32 : nullptr;
  if (c->prm.scheme == 1) {
    c->timer.begin(kStageVoid, c->stream);
    CK(launch_pcm(m, n, x, r, c->vol, out64, out32, c->st, c->stream), "pcm");
    c->timer.end(kStageVoid, c->stream);
    if (nb_count) CK(cudaMemsetAsync(nb_count, 0, sizeof(int32_t) * m.E * m.Q, c->stream), "pcm");
    if (nb_idsum) CK(cudaMemsetAsync(nb_idsum, 0, sizeof(int64_t) * m.E * m.Q, c->stream), "pcm");
  } else {
    s = tune_bins(c, n, x, r);
    if (s != CFDEM_OK) return s;
    s = do_bin(c, n, x, r);
    if (s != CFDEM_OK) return s;
    c->timer.begin(kStageVoid, c->stream);
    const bool conserve = c->prm.qcm_conserve == 1;
    CK(launch_qcm(m, c->tab, c->bins, mixed ? 1 : 0, c->R, c->bin_start, c->perm, c->xs64,
                  c->xs32, c->st, out64, out32, nb_count, nb_idsum, c->stream,
                  conserve ? reinterpret_cast<float2*>(c->qcm_w) : nullptr, conserve ? n : 0),
       "qcm");
    c->timer.end(kStageVoid, c->stream);
  }
  if (mixed) {
    c->eps_state = 2;
  } else {
    if (out64 != c->eps64)
      CK(cudaMemcpyAsync(c->eps64, out64, sizeof(double) * m.E * m.Q, cudaMemcpyDeviceToDevice,
                         c->stream),
         "eps copy");
    c->eps_state = 1;
  }
  return CFDEM_OK;
}

cfdem_status cfdem_project_rhs(cfdem_t c, const double* eps_q, double* b) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (!b) return fail(c, CFDEM_EINVAL, "b is NULL");
  DeviceGuard g(c->device);
  if (!eps_q && c->eps_state == 0) return fail(c, CFDEM_ESTATE, "no void fraction computed yet");
  c->timer.begin(kStageRhs, c->stream);
  if (eps_q) {
    CK(launch_rhs(c->mesh, c->tab, eps_q, nullptr, c->rhs_local, b, c->stream), "rhs");
  } else {
    CK(launch_rhs(c->mesh, c->tab, c->eps64, c->eps_state == 2 ? c->eps32 : nullptr,
                  c->rhs_local, b, c->stream),
       "rhs");
  }
  c->timer.end(kStageRhs, c->stream);
  return CFDEM_OK;
}

cfdem_status cfdem_apply(cfdem_t c, const double* x, double* y) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (!x || !y) return fail(c, CFDEM_EINVAL, "null vector");
  DeviceGuard g(c->device);
  CK(launch_apply64(c->mesh, c->bands64, c->coef, x, y, c->stream), "apply");
  return CFDEM_OK;
}

cfdem_status cfdem_project(cfdem_t c, const double* eps_q, double* eps_nodal) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (!eps_nodal) return fail(c, CFDEM_EINVAL, "eps_nodal is NULL");
  s = cfdem_project_rhs(c, eps_q, c->b);
  if (s != CFDEM_OK) return s;
  DeviceGuard g(c->device);
  s = tune_shape(c, c->b);
  if (s != CFDEM_OK) return s;
  return solve(c, c->b, eps_nodal, "project");
}

}  // extern "C"

cfdem_status forces_with_event(cfdem_t c, int64_t n, const double* x, const double* r,
                               const double* u_p, const double* u_nodal, const double* p_nodal,
                               const double* eps_nodal, double* f, double* f_drag,
                               double* F_elem, double* F_q, cudaEvent_t after_kernel) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!x || !r || !u_p || !f)) || !u_nodal ||
      !p_nodal || !eps_nodal)
    return fail(c, CFDEM_EINVAL, "null input");
  DeviceGuard g(c->device);
  const MeshDev& m = c->mesh;
  const bool semi = c->prm.fluid_drag == 1;
  const bool want_src = F_elem || F_q || semi;
  s = ensure_particles(c, n);
  if (s != CFDEM_OK) return s;
  PartSrc ps{want_src ? c->psrc : nullptr, c->pelem, c->src_max};
  if (want_src)
    CK(cudaMemsetAsync(c->src_max, 0, 3 * sizeof(unsigned long long), c->stream), "forces");
  c->timer.begin(kStageForces, c->stream);
  ForceParams fp = force_params(c);
  // mixed path with many particles per node (large elements, dense beds):
  // split the nodal velocity and void fraction into double-float pairs once
  // per node instead of once per particle that reads them (the same split,
  // so the same bits); the buffer is allocated outside a stream capture
  const int64_t nq = (int64_t)(m.k + 1) * (m.k + 1) * (m.k + 1);
  if (c->prm.precision == 1 && n * nq >= 8 * m.n_nodes) {
    if (!c->nodal_df && !stream_capturing(c->stream))
      CK(grow(&c->nodal_df, 2 * (size_t)m.n_nodes), "forces");
    if (c->nodal_df) {
      CK(launch_split_nodal(m.n_nodes, u_nodal, eps_nodal, c->nodal_df, c->stream), "forces");
      fp.nodal_df = c->nodal_df;
    }
  }
  CK(launch_forces(m, c->tab, c->prm.precision, fp, n, x, r, u_p, u_nodal, p_nodal, eps_nodal,
                   f, f_drag, ps, c->st, c->stream),
     "forces");
  c->timer.end(kStageForces, c->stream);
  if (after_kernel) CK(cudaEventRecord(after_kernel, c->stream), "forces");
  if (want_src) {
    c->timer.begin(kStageSource, c->stream);
    // without the fluid-side drag F_e comes out of the same pass as S_e
    CK(launch_source_sum(m, n, ps, u_p, semi ? 1 : 0, c->src_acc, c->S, semi_acc(c), F_elem,
                         c->stream),
       "fluid source");
    if (semi && (F_elem || F_q))
      CK(launch_fluid_source_semi(m, c->tab, c->prm.precision, c->S, semi_acc(c), u_nodal,
                                  F_elem, F_q, c->stream),
         "fluid source");
    else if (F_q)
      CK(launch_fluid_source(m, c->S, nullptr, F_q, c->stream), "fluid source");
    c->timer.end(kStageSource, c->stream);
  }
  c->semi_valid = semi ? 1 : 0;
  return CFDEM_OK;
}

extern "C" {

cfdem_status cfdem_forces(cfdem_t c, int64_t n, const double* x, const double* r,
                          const double* u_p, const double* u_nodal, const double* p_nodal,
                          const double* eps_nodal, double* f, double* f_drag, double* F_elem,
                          double* F_q) {
  return forces_with_event(c, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, f_drag, F_elem, F_q,
                           nullptr);
}

cfdem_status cfdem_fluid_drag_coefficients(cfdem_t c, double* beta_e, double* up_avg) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (!c->semi_valid)
    return fail(c, CFDEM_ESTATE, "no forces call with fluid_drag = 1 since the mesh was set");
  if (!beta_e && !up_avg) return CFDEM_OK;
  DeviceGuard g(c->device);
  CK(launch_drag_coefficients(c->mesh, semi_acc(c), beta_e, up_avg, c->stream),
     "drag coefficients");
  return CFDEM_OK;
}

cfdem_status cfdem_coupling_step(cfdem_t c, int64_t n, const double* x, const double* r,
                                 const double* u_p, const double* u_nodal,
                                 const double* p_nodal, double* eps_nodal, double* f,
                                 double* f_drag, double* F_elem, double* F_q) {
  cfdem_status s = cfdem_void_fraction(c, n, x, r, nullptr, nullptr, nullptr);
  if (s != CFDEM_OK) return s;
  s = cfdem_project(c, nullptr, eps_nodal);
  if (s != CFDEM_OK) return s;
  return cfdem_forces(c, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, f_drag, F_elem, F_q);
}

cfdem_status cfdem_mass_apply(cfdem_t c, const double* x, double* y) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (!x || !y) return fail(c, CFDEM_EINVAL, "null vector");
  DeviceGuard g(c->device);
  const double mass_only[4] = {c->coef[0], 0.0, 0.0, 0.0};
  CK(launch_apply64(c->mesh, c->bands64, mass_only, x, y, c->stream), "mass apply");
  return CFDEM_OK;
}

cfdem_status cfdem_adjoint(cfdem_t c, int64_t n, const double* x, const double* r,
                           const double* u_p, const double* u_nodal, const double* p_nodal,
                           const double* eps_nodal, const double* g_f, const double* g_fdrag,
                           const double* g_eps, double* dJ_dx, double* dJ_du) {
  cfdem_status s = need_mesh(c);
  if (s != CFDEM_OK) return s;
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!x || !r || !u_p || !dJ_dx)) ||
      !u_nodal || !p_nodal || !eps_nodal)
    return fail(c, CFDEM_EINVAL, "null input");
  if (c->prm.scheme == 0 && c->prm.qcm_conserve)
    return fail(c, CFDEM_EINVAL,
                "the adjoint does not differentiate the volume-conserving QCM weights");
  DeviceGuard g(c->device);
  const MeshDev& m = c->mesh;
  if (!c->adj_geps) {  // the mesh arena is released (and these reset) by every set_mesh
    CK(grow(&c->adj_geps, m.n_nodes), "adjoint arena");
    CK(grow(&c->adj_lam, m.n_nodes), "adjoint arena");
    CK(grow(&c->adj_gq, m.E * m.Q), "adjoint arena");
  }
  if (g_eps)
    CK(cudaMemcpyAsync(c->adj_geps, g_eps, sizeof(double) * m.n_nodes, cudaMemcpyDeviceToDevice,
                       c->stream),
       "adjoint");
  else
    CK(cudaMemsetAsync(c->adj_geps, 0, sizeof(double) * m.n_nodes, c->stream), "adjoint");
  if (dJ_du) CK(cudaMemsetAsync(dJ_du, 0, sizeof(double) * 3 * m.n_nodes, c->stream), "adjoint");
  CK(launch_adj_forces(m, c->tab, c->prm.precision, force_params(c), n, x, r, u_p, u_nodal,
                       p_nodal, eps_nodal, g_f, g_fdrag, dJ_dx, dJ_du, c->adj_geps, c->st,
                       c->stream),
     "adjoint forces");
  if (c->prm.scheme == 0) {
    // lambda = A^-1 dJ/deps_h (A symmetric), then through the QCM
    CK(cudaMemsetAsync(c->adj_lam, 0, sizeof(double) * m.n_nodes, c->stream), "adjoint");
    s = solve(c, c->adj_geps, c->adj_lam, "adjoint solve");
    if (s != CFDEM_OK) return s;
    CK(launch_adj_qcm(m, c->tab, c->prm.precision, c->R, c->adj_lam, c->adj_gq, n, x, r,
                      dJ_dx, c->stream),
       "adjoint void fraction");
  }
  return CFDEM_OK;
}

cfdem_status cfdem_synchronize(cfdem_t c) {
  if (!c) return CFDEM_EINVAL;
  DeviceGuard g(c->device);
  cudaError_t e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  CK(read_pending_stats(c), "status");
  DevStatus h;
  CK(cudaMemcpy(&h, c->st, sizeof h, cudaMemcpyDeviceToHost), "status");
  cfdem_status s = CFDEM_OK;
  if (h.first_bad != ~0ull) {
    s = fail(c, CFDEM_OUT_OF_DOMAIN, "particle %llu lies outside the mesh", h.first_bad);
    unsigned long long reset = ~0ull;
    CK(cudaMemcpy(&c->st->first_bad, &reset, sizeof reset, cudaMemcpyHostToDevice), "status");
  } else if (c->pending_not_converged) {
    s = fail(c, CFDEM_NOT_CONVERGED, "CG stopped at %d iterations, relative residual %.3e",
             c->last_iters, c->last_relres);
  }
  c->pending_not_converged = 0;
  return s;
}

cfdem_status cfdem_get_stats(cfdem_t c, cfdem_stats* out) {
  if (!c || !out) return CFDEM_EINVAL;
  std::memset(out, 0, sizeof *out);
  DeviceGuard g(c->device);
  cudaError_t e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "get_stats");
  CK(read_pending_stats(c), "status");
  DevStatus h;
  CK(cudaMemcpy(&h, c->st, sizeof h, cudaMemcpyDeviceToHost), "status");
  out->first_bad_particle = h.first_bad == ~0ull ? -1 : (int64_t)h.first_bad;
  out->cg_iterations = c->last_iters;
  out->cg_outer = c->last_outer;
  out->cg_relres = c->last_relres;
  out->converged = c->last_converged;
  for (int a = 0; a < 3; ++a) {
    out->nb[a] = c->bins.nb[a];
    out->bin_edge[a] = c->bins.be[a];
  }
  out->qcm_radius = c->R;
  out->n_elem = c->mesh.E;
  out->n_qp = c->mesh.E * c->mesh.Q;
  out->n_nodes = c->mesh.n_nodes;
  out->n_pnodes = c->mesh.n_pnodes;
  c->timer.collect();
  for (int s = 0; s < kStages && s < 8; ++s) {
    out->stage_ms[s] = c->timer.ms[s];
    out->stage_calls[s] = c->timer.calls[s];
  }
  out->timer_overflow = c->timer.overflow ? 1 : 0;
  out->kernel_launches = launches_total() - c->launches_at_reset;
  out->precond = c->fdm ? 1 : 0;
  out->tile_shape = c->mesh.shape;
  out->tuned = c->tuned;
  out->tune_ms = c->tune_ms;
  out->fdm_tile = c->fdm ? fdm_tile(c->fdm) : 0;
  return CFDEM_OK;
}

cfdem_status cfdem_set_timing(cfdem_t c, int enable) {
  if (!c) return CFDEM_EINVAL;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  c->timer.collect();
  for (int s = 0; s < kStages; ++s) {
    c->timer.ms[s] = 0.0;
    c->timer.calls[s] = 0;
  }
  c->timer.overflow = false;
  if (enable) c->timer.create();
  c->timer.on = enable != 0;
  ++c->gen;
  c->launches_at_reset = launches_total();
  return CFDEM_OK;
}

const char* cfdem_last_error(cfdem_t c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
