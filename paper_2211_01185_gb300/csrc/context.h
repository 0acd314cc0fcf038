// context.h -- the library context behind the opaque cfdem_t handle (shared
// by the single-bed entry points and the batched ensemble).
#pragma once
#include <string>

#include "../../include/cfdem.h"
#include "internal.h"

using cfdem::BinDev;
using cfdem::CgWork;
using cfdem::DevStatus;
using cfdem::FdmPlan;
using cfdem::MeshDev;
using cfdem::Tables;
using cfdem::Timer;

// The signature a tuned choice is kept for (compared byte by byte: built
// from a zeroed object).
struct TuneKey {
  int ne[3], k, precision, variant;  // variant: QCM conserve flag, or the preconditioner
  int64_t nbucket;                    // particle count bucket (floor(log2 n)), 0 for shapes
  double L[3], R, rmax, coef[4];
};

struct cfdem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool have_mesh = false;
  MeshDev mesh{};
  Tables tab{};
  BinDev bins{};
  cfdem_params prm{};
  double R = 0.0;  // resolved averaging radius
  double coef[4] = {0, 0, 0, 0};
  // device memory
  DevStatus* st = nullptr;
  double* bands64 = nullptr;
  float* bands32 = nullptr;
  float* bandsdf = nullptr;
  // particle arena
  int64_t cap_n = 0;
  int32_t *bin_of = nullptr, *slot = nullptr, *perm = nullptr;
  float4* nodal_df = nullptr;  // mesh arena: double-float nodal u and eps (forces)
  double* xs64 = nullptr;
  float* xs32 = nullptr;
  float* qcm_w = nullptr;      // volume-conserving QCM weights per sorted particle [2 n]
  double* psrc = nullptr;      // per-particle fluid-source records [4 n] (PartSrc::S)
  int32_t* pelem = nullptr;    // element of each particle [n] (PartSrc::elem)
  int64_t cap_bins = 0;
  int32_t *bin_count = nullptr, *bin_start = nullptr, *scan_tmp = nullptr;
  // mesh arena
  double* eps64 = nullptr;     // internal eps_q (FP64 path)
  float* eps32 = nullptr;      // internal eps_q (mixed path)
  double* b = nullptr;
  double* S = nullptr;         // per-element source accumulator [E][3]
  double* vol = nullptr;       // per-element particle volume (PCM)
  double* rhs_local = nullptr; // per-element right-hand-side contributions [(k+1)^3][E]
  double* semi = nullptr;      // fluid-side drag sums: B [E], U [3E], N [E]
  long long* src_acc = nullptr;           // fixed-point source sums [16 E]
  unsigned long long* src_max = nullptr;  // largest |value| bits per class [3] (+1 pad)
  int semi_valid = 0;          // 1 once a forces call with fluid_drag = 1 filled them
  // adjoint arena (grown by the first cfdem_adjoint)
  double* adj_geps = nullptr;  // dJ/deps_h [n_nodes]
  double* adj_lam = nullptr;   // lambda = A^-1 dJ/deps_h [n_nodes]
  double* adj_gq = nullptr;    // dJ/deps_q [E][Q]
  CgWork cg{};
  FdmPlan* fdm = nullptr;
  const char* fdm_note = "";
  int eps_state = 0;           // 0 none, 1 eps64 valid, 2 eps32 valid
  // host-side record
  int last_iters = 0, last_outer = 0, last_converged = 1;
  double last_relres = 0.0;
  int pending_not_converged = 0;
  // set when the last solve ran inside a captured graph: its iteration count
  // and residual are read from the device scalars at the next synchronising
  // call
  bool stats_pending = false;
  cudaStream_t loop_stream = nullptr;  // capture stream of device-driven CG loops
  unsigned gen = 0;                    // bumped by every change of mesh, parameters or timing
  Timer timer;
  long long launches_at_reset = 0;
  // autotuner: the signatures the current bins and tile shape were tuned
  // for, what was tuned (bit 0 bins, bit 1 shape), host time spent, and a
  // scratch vector for the timed solves
  TuneKey bin_key{}, shape_key{};
  bool bin_key_set = false, shape_key_set = false;
  int tuned = 0;
  double tune_ms = 0.0;
  double* tune_x = nullptr;
  std::string err;
};

// cfdem_forces that also records `after_kernel` (when given) on the
// context's stream right after the forces kernel, before the fluid source
// sums: f is final from that point on
cfdem_status forces_with_event(cfdem_t c, int64_t n, const double* x, const double* r,
                               const double* u_p, const double* u_nodal, const double* p_nodal,
                               const double* eps_nodal, double* f, double* f_drag,
                               double* F_elem, double* F_q, cudaEvent_t after_kernel);
