// internal.h -- declarations shared by the CUDA translation units of the
// coupling library.  Nothing here is part of the public C ABI (cfdem.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cfdem {

constexpr double kPi = 3.14159265358979323846;

// One sorted particle in FP64: position and radius (32-byte aligned).
struct __align__(32) P4 {
  double x, y, z, w;
};

// Mesh geometry as the kernels see it.  Axis-aligned box of equal hexahedra.
struct MeshDev {
  double x0[3];      // origin
  double L[3];       // extent
  double h[3];       // element size, L / ne (IEEE division, as the oracle)
  int ne[3];         // elements per axis
  int k;             // Q_k degree of velocity / void fraction
  int kp;            // Q_kp degree of pressure
  int nq;            // Gauss points per axis (k + 1)
  int Q;             // nq^3
  int nn[3];         // Q_k nodes per axis (ne k + 1)
  int np[3];         // Q_kp nodes per axis (ne kp + 1)
  int64_t E;         // elements
  int64_t n_nodes;   // Q_k nodes
  int64_t n_pnodes;  // Q_kp nodes
  double Ve;         // element volume hx hy hz
  float Ve32;        // Ve rounded to FP32 (mixed path)
  int shape;         // tile shape of the projection operator (pick_shape)
};

// 1D reference tables on [0,1] (degree <= 3).  Built on the host from
// closed forms (Gauss-Legendre points, GLL nodes) and exact quadrature.
struct Tables {
  double g[4], w[4];        // Gauss points and weights, nq = k + 1 of them
  double z[4];              // GLL nodes of degree k
  double zp[4];             // GLL nodes of degree kp
  double lw[4], lwp[4];     // 1 / prod_{b != a} (z_a - z_b) for z and zp
  double Bw[4][4];          // Bw[a][q] = l_a(g_q) w_q  (k basis, Gauss weight folded in)
  double Mh[4][4];          // reference mass     int_0^1 l_a l_b
  double Kh[4][4];          // reference stiffness int_0^1 l_a' l_b'
  float zf[4], zpf[4];      // FP32 copies of z, zp, lw, lwp (mixed path)
  float lwf[4], lwpf[4];
  float z_lo[4], lw_lo[4];  // z - zf and lw - lwf: z and lw as double-float
  float Bwf[4][4];          // FP32 copy of Bw
};

// Bin grid over the box.
struct BinDev {
  int nb[3];
  double be[3];      // bin edge per axis, L / nb
  double inv_be[3];  // 1 / be (IEEE division on the host, as on the device)
  int64_t nbins;
  // the same grid for location without FP64 instructions: origin and 1/be
  // as double-float, the in_box bounds as order-preserving integer keys of
  // their bits, and loc32 = 0 where the box is too far from the origin for
  // the double-float margin (then the FP64 rule bins every particle)
  float x0_hi[3], x0_lo[3], inv_be_hi[3], inv_be_lo[3];
  long long box_lo_key[3], box_hi_key[3];
  float nm1f[3];  // nb - 1 as float
  int loc32;
};

// Device-side status words of one context (one allocation).
struct DevStatus {
  unsigned long long first_bad;   // lowest out-of-domain particle index, or ~0ull
  unsigned long long rmax_bits;   // bits of max radius (non-negative double)
  int not_converged;
  int pad;
};

// Scalars of the CG solver kept on the device.
struct CgScalars {
  double rz;        // r . z (current)
  double pAp;
  double alpha, beta;
  double rr;        // r . r
  double bb;        // b . b
  double tol2;      // (rtol)^2 * bb
  int it;           // iterations done
  int done;         // 1 once converged (kernels then return at once)
  unsigned int ticket;  // last-block counter
  int loops;       // bodies of a device-driven CG loop run so far
  float alpha_hi, alpha_lo;  // double-float split of alpha (mixed solve)
  int xnz;          // 1 if the start vector has a nonzero entry (else A x0 = 0 is skipped)
};

// Optional per-stage CUDA-event timers of a context (off by default).  A
// stage is a group of launches on the context's stream; begin/end record an
// event pair, collect() (after a synchronize) adds up the elapsed times.
enum Stage {
  kStageBin = 0,      // a1-a2 locate + counting sort + sorted copies
  kStageVoid = 1,     // a3 void-fraction kernel (QCM or PCM)
  kStageRhs = 2,      // a4 projection right-hand side
  kStageSolve = 3,    // a5 whole solve
  kStageForces = 4,   // a6 forces kernel
  kStageSource = 5,   // a7 fluid source
  kStageOp32 = 6,     // operator launches of the FP32 CG (one per iteration)
  kStageOp64 = 7,     // operator launches in FP64 (FP64 CG or refinement residuals)
  kStages = 8
};

struct Timer {
  static constexpr int kCap = 1024;
  bool on = false;
  cudaEvent_t* ev[kStages] = {};  // 2 * kCap events per stage, created on first use
  int count[kStages] = {};
  long long calls[kStages] = {};
  double ms[kStages] = {};
  bool overflow = false;
  void begin(int s, cudaStream_t st);
  void end(int s, cudaStream_t st);
  void collect();
  void release();
  void create();  // allocate the events (outside any timed region)
};

// the 1D reference tables of degree k and kp (GLL nodes, Gauss rule, ...)
void make_tables(int k, int kp, Tables* t);

// process-wide count of kernel launches made by the library
void count_launches(int n);
long long launches_total();

// Parameters of the per-particle force kernels (from cfdem_params and the
// mesh): fluid density and viscosity, gravity, closure floor, 1/h per axis,
// drag closure, beta_B = beta_A / eps flag, VANS model, shear force flag.
struct ForceParams {
  double rho, mu, g[3], eps_floor;
  double inv_h[3];
  int drag_model, beta_over_eps, vans_model, shear, fluid_drag;
  // mixed path: FP32 copies, and the element location from a double-float
  // split of x (loc32 = 0 where the box is too far from the origin for the
  // FP32 margin, then the FP64 rule locates every particle)
  float rho32, mu32, g32[3], eps_floor32, inv_h32[3];
  float x0_hi[3], x0_lo[3], inv_h_hi[3], inv_h_lo[3];
  float nem1f[3];  // elements per axis - 1, as float
  int loc32;
  // in_box bounds x0 - 1e-12 L and (x0 + L) + 1e-12 L as order-preserving
  // integer keys of their bits (compared without FP64 instructions)
  long long box_lo_key[3], box_hi_key[3];
  // mixed path, optional: the nodal velocity and void fraction already split
  // into double-float pairs, [n_nodes][2] float4 = (u0, u1 | u2, eps), used
  // where many particles read each node (the split is the same either way)
  const float4* nodal_df;
};

// Per-particle fluid-source records written by the forces kernel and summed
// per element by launch_source_sum: S = the particle's share of F_pf (drag,
// and for model B the pressure and shear parts) and its drag coefficient
// [n][4], its element [n] (-1 outside the mesh), and the bits of the largest
// |S| component, |coefficient| and |u_p| component over the particles
// (maxbits[3], reset before the forces kernel).
struct PartSrc {
  double* S;
  int32_t* elem;
  unsigned long long* maxbits;
};

// Per-element accumulators of the fluid-side drag (fluid_drag = 1): sum of
// the particles' drag coefficients, of their velocities [3], and their count.
struct SemiAcc {
  double *B, *U, *N;
};

// ---------------------------------------------------------------- launchers
// particles.cu
cudaError_t launch_locate(const MeshDev& m, int64_t n, const double* x, int32_t* elem,
                          double* xi, DevStatus* st, cudaStream_t s);
cudaError_t launch_bin(const MeshDev& m, const BinDev& b, int64_t n, const double* x,
                       const double* r, int32_t* bin_of, int32_t* slot, int32_t* bin_count,
                       int32_t* bin_start, int32_t* perm, int32_t* scan_tmp, double* xs64,
                       float* xs32, DevStatus* st, cudaStream_t s);
// ps.S / ps.elem receive the per-particle source records (ps.S may be null)
// the nodal velocity and void fraction as double-float pairs for
// ForceParams::nodal_df: out[2 j] = (u0, u1), out[2 j + 1] = (u2, eps) of node j
cudaError_t launch_split_nodal(int64_t n_nodes, const double* u_nodal, const double* eps_nodal,
                               float4* out, cudaStream_t s);
cudaError_t launch_forces(const MeshDev& m, const Tables& t, int precision, const ForceParams& fp,
                          int64_t n, const double* x, const double* r, const double* u_p,
                          const double* u_nodal, const double* p_nodal,
                          const double* eps_nodal, double* f, double* f_drag, PartSrc ps,
                          DevStatus* st, cudaStream_t s);
// per-element sums of the records: S_elem[E][3] and, with semi, the drag
// coefficients, particle velocities and counts into acc.  The sums are exact
// fixed-point sums (acc64: 16 int64 per element of scratch, 6 of them used
// without the fluid-side drag), so their bits
// do not depend on the order of the particles.
// (F_elem, when not null and not semi: also F_e = -S_e / V_e, the fluid
// source of Eq. (fb), written by the same pass)
cudaError_t launch_source_sum(const MeshDev& m, int64_t n, PartSrc ps, const double* u_p,
                              int semi, long long* acc64, double* S_elem, SemiAcc acc,
                              double* F_elem, cudaStream_t s);
cudaError_t launch_fluid_source(const MeshDev& m, const double* S_elem, double* F_elem,
                                double* F_q, cudaStream_t s);
cudaError_t launch_fluid_source_semi(const MeshDev& m, const Tables& t, int precision,
                                     const double* S_elem, SemiAcc acc, const double* u_nodal,
                                     double* F_elem, double* F_q, cudaStream_t s);
cudaError_t launch_drag_coefficients(const MeshDev& m, SemiAcc acc, double* beta_e,
                                     double* up_avg, cudaStream_t s);

// voidfrac.cu
// cw (optional): scratch of n float pairs; when given, the volume-conserving
// weights of the n sorted particles are computed into it first and scale
// every particle's lens volumes
cudaError_t launch_qcm(const MeshDev& m, const Tables& t, const BinDev& b, int precision,
                       double R, const int32_t* bin_start, const int32_t* perm,
                       const double* xs64, const float* xs32, const DevStatus* st,
                       double* eps_q64, float* eps_q32, int32_t* nb_count, int64_t* nb_idsum,
                       cudaStream_t s, float2* cw = nullptr, int64_t n = 0);
cudaError_t launch_pcm(const MeshDev& m, int64_t n, const double* x, const double* r,
                       double* vol_elem, double* eps_q64, float* eps_q32, DevStatus* st,
                       cudaStream_t s);

// projection.cu
// local: scratch of (k+1)^3 E doubles (per-element contributions)
cudaError_t launch_rhs(const MeshDev& m, const Tables& t, const double* eps_q64,
                       const float* eps_q32, double* local, double* b, cudaStream_t s);
cudaError_t upload_bands(const MeshDev& m, const Tables& t, double L2, double** bands64,
                         float** bands32, float** bands_df);
cudaError_t launch_apply64(const MeshDev& m, const double* bands, const double* coef,
                           const double* x, double* y, cudaStream_t s);
cudaError_t launch_adj_forces(const MeshDev& m, const Tables& t, int precision,
                              const ForceParams& fp, int64_t n, const double* x, const double* r,
                              const double* u_p,
                              const double* u_nodal, const double* p_nodal,
                              const double* eps_nodal, const double* gf, const double* gfd,
                              double* dJdx, double* dJdu, double* geps, DevStatus* st,
                              cudaStream_t s);
cudaError_t launch_adj_qcm(const MeshDev& m, const Tables& t, int precision, double R,
                           const double* lam, double* gq, int64_t n, const double* x,
                           const double* r, double* dJdx, cudaStream_t s);
struct FdmPlan;
cudaError_t fdm_create(const MeshDev& m, const Tables& t, const double coef[4], FdmPlan** out,
                       const char** why);
// r . z of the CG formed by the FDM's last pass (slab form only): r the
// residual the FDM was applied to (FP32), the block sums go to partials,
// rz and (unless first) the Fletcher-Reeves beta to sc.
struct FdmDot {
  const float* r = nullptr;
  double* partials = nullptr;
  CgScalars* sc = nullptr;
  int first = 0;
};
// z = P^-1 r; with dot (and the slab form) also r . z into dot->sc, and
// *dot_done = true -- otherwise the caller forms the dot product
cudaError_t fdm_apply(FdmPlan* p, const float* r, float* z, const int* done, cudaStream_t s,
                      const FdmDot* dot = nullptr, bool* dot_done = nullptr);
void fdm_destroy(FdmPlan* p);
// register tile of the plan's slab transforms as 10 rows + columns, 0 for
// the dense form
int fdm_tile(const FdmPlan* p);

struct CgWork {
  // FP64 vectors
  double *r, *z, *p0, *p1, *Ap, *dinv, *xcor, *zn;
  // FP32 vectors (mixed inner solve, FDM conversions)
  float *r32, *z32, *q0, *q1, *Aq, *dinv32, *d32, *zn32, *rin32;
  FdmPlan* fdm;       // fast-diagonalisation preconditioner, or null (Jacobi)
  // double-float vectors of the mixed solve (pairs of floats, hi first)
  struct df64* x_df;
  struct df64* r_df;
  struct df64* Ap_df;
  struct df64* p0_df;
  struct df64* p1_df;
  const struct df64* bands_df;  // operator bands as df64 pairs
  double* partials;   // per-block partial sums
  CgScalars* sc;      // device scalars
  int nblocks;
  Timer* timer;       // may be null
  // non-null while the solve is being captured into a CUDA graph: the stream
  // on which the body of the device-driven CG loop is captured
  cudaStream_t loop;
};
// true when s is a stream under active capture
bool stream_capturing(cudaStream_t s);
int cg_blocks(const MeshDev& m);
// 1 if tile shape `shape` (0..2) fits the operator's shared-memory budget
bool shape_fits(const MeshDev& m, int shape);
int pick_shape(const MeshDev& m);
cudaError_t run_cg64(const MeshDev& m, const double* bands, const double* coef,
                     const double* b, double* x, double rtol, int maxit, CgWork& w,
                     cudaStream_t s, int* iters_host, double* relres_host, int* converged);
cudaError_t run_cg_mixed(const MeshDev& m, const double* bands64, const float* bands32,
                         const double* coef, const double* b, double* x, double rtol,
                         int maxit, CgWork& w, cudaStream_t s, int* iters_host,
                         int* outer_host, double* relres_host, int* converged);

}  // namespace cfdem
