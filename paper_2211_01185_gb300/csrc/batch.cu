// batch.cu -- batched ensemble of independent beds, replayed as one CUDA graph.
//
// Each bed is a full context (mesh, parameters, arenas, FDM plan) with its
// own stream.  A step forks every bed's stream from the batch's capture
// stream, runs cfdem_coupling_step on it and joins it back.  Run eagerly
// this is the same work as stepping the beds one after another, except that
// the GPU may overlap them.  Captured, the whole ensemble becomes one graph:
// every bed is a parallel branch, its CG a conditional while node that
// iterates on the device, so a replay needs one launch and no host round
// trip for any bed.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cfdem.h"
#include "context.h"
#include "internal.h"

struct cfdem_batch {
  int device = 0;
  cudaStream_t user = nullptr;  // the caller's stream
  cudaStream_t cap = nullptr;   // the batch's own stream (graphs are captured and launched here)
  std::vector<cfdem_t> beds;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  std::vector<cudaStream_t> side;   // per bed: uploads of the inputs the forces need
  std::vector<cudaEvent_t> sfork, late;
  cudaEvent_t fork = nullptr, in = nullptr, out = nullptr;
  bool use_graph = true;
  bool replayed = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cfdem_bed_io> key_io;  // arguments the graph was captured with
  std::vector<unsigned> key_gen;     // bed configuration generations at capture
  std::string err;                   // last failure, for cfdem_batch_last_error
};

namespace {

struct BatchDevice {
  int prev = -1;
  explicit BatchDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BatchDevice() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// record a failed CUDA call of the batch itself and return CFDEM_ECUDA
cfdem_status bfail(cfdem_batch_t b, const char* what, cudaError_t e) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  b->err = buf;
  return CFDEM_ECUDA;
}

#define BCK(expr, what)                              \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return bfail(b, what, e_); \
  } while (0)

void drop_graph(cfdem_batch_t b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key_io.clear();
  b->key_gen.clear();
}

// copy `count` doubles if both ends are given
cudaError_t copy_if(const double* src, const double* dst, int64_t count, cudaMemcpyKind kind,
                    cudaStream_t s) {
  if (!src || !dst || count <= 0) return cudaSuccess;
  return cudaMemcpyAsync(const_cast<double*>(dst), src, sizeof(double) * (size_t)count, kind, s);
}

// one bed's coupling step (cfdem_coupling_step: void fraction, projection,
// forces), with the uploads and downloads of its host buffers: x and r on
// the bed's stream ahead of the void fraction, u_p, u_nodal and p_nodal on
// its side stream meanwhile, joined before the forces; f and F_elem back
// after them
cfdem_status step_bed(cfdem_batch_t b, size_t i, const cfdem_bed_io& a) {
  cfdem_t c = b->beds[i];
  cudaStream_t s = b->streams[i], side = b->side[i];
  const MeshDev& m = c->mesh;
  const bool staged = a.host_x || a.host_r || a.host_u_p || a.host_u_nodal || a.host_p_nodal ||
                      a.host_f || a.host_F_elem;
  if (staged && !c->have_mesh) return cfdem_coupling_step(c, a.n, a.x, a.r, a.u_p, a.u_nodal,
                                                          a.p_nodal, a.eps_nodal, a.f, a.f_drag,
                                                          a.F_elem, a.F_q);
  const bool late = a.host_u_p || a.host_u_nodal || a.host_p_nodal;
  if (staged && cfdem::stream_capturing(s)) {
    // a capture takes page-locked host buffers only; with any other the
    // eager step stands and the batch stays eager (CFDEM_ESTATE)
    const void* hs[] = {a.host_x, a.host_r, a.host_u_p, a.host_u_nodal, a.host_p_nodal,
                        a.host_f, a.host_F_elem};
    for (const void* h : hs) {
      if (!h) continue;
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, h) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return CFDEM_ESTATE;
      }
    }
  }
  if (staged) {
    BCK(copy_if(a.host_x, a.x, 3 * a.n, cudaMemcpyHostToDevice, s), "upload x");
    BCK(copy_if(a.host_r, a.r, a.n, cudaMemcpyHostToDevice, s), "upload r");
  }
  if (late) {
    const int64_t npn = (int64_t)m.np[0] * m.np[1] * m.np[2];
    BCK(cudaEventRecord(b->sfork[i], s), "fork uploads");
    BCK(cudaStreamWaitEvent(side, b->sfork[i], 0), "fork uploads");
    BCK(copy_if(a.host_u_p, a.u_p, 3 * a.n, cudaMemcpyHostToDevice, side), "upload u_p");
    BCK(copy_if(a.host_u_nodal, a.u_nodal, 3 * m.n_nodes, cudaMemcpyHostToDevice, side),
        "upload u_nodal");
    BCK(copy_if(a.host_p_nodal, a.p_nodal, npn, cudaMemcpyHostToDevice, side), "upload p_nodal");
    BCK(cudaEventRecord(b->late[i], side), "join uploads");
  }
  cfdem_status st = cfdem_void_fraction(c, a.n, a.x, a.r, nullptr, nullptr, nullptr);
  if (st == CFDEM_OK) st = cfdem_project(c, nullptr, a.eps_nodal);
  // the uploads are joined even after a failure, so that no branch of a
  // capture is left open
  if (late) BCK(cudaStreamWaitEvent(s, b->late[i], 0), "join uploads");
  if (st != CFDEM_OK) return st;
  // f goes down on the side stream as soon as the forces kernel has written
  // it, beside the fluid source sums; F_elem after them
  const bool early_f = staged && a.host_f && a.n > 0;
  st = forces_with_event(c, a.n, a.x, a.r, a.u_p, a.u_nodal, a.p_nodal, a.eps_nodal, a.f,
                         a.f_drag, a.F_elem, a.F_q, early_f ? b->sfork[i] : nullptr);
  if (st != CFDEM_OK) return st;
  if (early_f) {
    BCK(cudaStreamWaitEvent(side, b->sfork[i], 0), "download f");
    BCK(copy_if(a.f, a.host_f, 3 * a.n, cudaMemcpyDeviceToHost, side), "download f");
    BCK(cudaEventRecord(b->late[i], side), "download f");
  }
  if (staged)
    BCK(copy_if(a.F_elem, a.host_F_elem, 3 * m.E, cudaMemcpyDeviceToHost, s),
        "download F_elem");
  if (early_f) BCK(cudaStreamWaitEvent(s, b->late[i], 0), "download f");
  return CFDEM_OK;
}

// fork every bed from b->cap, step it, join it back; *bad = first failing bed
cfdem_status step_all(cfdem_batch_t b, const cfdem_bed_io* io, int* bad) {
  *bad = -1;
  cfdem_status first = CFDEM_OK;
  BCK(cudaEventRecord(b->fork, b->cap), "fork");
  for (size_t i = 0; i < b->beds.size(); ++i) {
    BCK(cudaStreamWaitEvent(b->streams[i], b->fork, 0), "fork");
    const cfdem_bed_io& a = io[i];
    cfdem_status s = step_bed(b, i, a);
    if (s != CFDEM_OK && first == CFDEM_OK) {
      first = s;
      *bad = (int)i;
      char buf[64];
      std::snprintf(buf, sizeof buf, "bed %d: ", (int)i);
      b->err = buf + std::string(cfdem_last_error(b->beds[i]));
    }
    BCK(cudaEventRecord(b->join[i], b->streams[i]), "join");
    BCK(cudaStreamWaitEvent(b->cap, b->join[i], 0), "join");
  }
  return first;
}

bool same_key(cfdem_batch_t b, const cfdem_bed_io* io) {
  if (!b->exec || b->key_io.size() != b->beds.size()) return false;
  if (std::memcmp(b->key_io.data(), io, sizeof(cfdem_bed_io) * b->beds.size()) != 0) return false;
  for (size_t i = 0; i < b->beds.size(); ++i)
    if (b->key_gen[i] != b->beds[i]->gen) return false;
  return true;
}

}  // namespace

extern "C" {

cfdem_status cfdem_batch_create(cfdem_batch_t* out, int device, void* stream, int n_beds) {
  if (!out) return CFDEM_EINVAL;
  *out = nullptr;
  if (n_beds < 1 || n_beds > 4096) return CFDEM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return CFDEM_ECUDA;
  BatchDevice g(device);
  cfdem_batch_t b = new cfdem_batch();
  b->device = device;
  b->user = (cudaStream_t)stream;
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->out, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < n_beds; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->streams.push_back(s);
    ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->join.push_back(ev);
    cudaStream_t ss = nullptr;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    ok = ok && cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->side.push_back(ss);
    ok = ok && cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->sfork.push_back(e1);
    ok = ok && cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->late.push_back(e2);
    cfdem_t c = nullptr;
    ok = ok && cfdem_create(&c, device, s) == CFDEM_OK;
    if (ok) b->beds.push_back(c);
  }
  if (!ok) {
    cfdem_batch_destroy(b);
    return CFDEM_ECUDA;
  }
  *out = b;
  return CFDEM_OK;
}

cfdem_status cfdem_batch_destroy(cfdem_batch_t b) {
  if (!b) return CFDEM_OK;
  BatchDevice g(b->device);
  if (b->cap) cudaStreamSynchronize(b->cap);
  drop_graph(b);
  for (cfdem_t c : b->beds) cfdem_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->sfork) cudaEventDestroy(e);
  for (cudaEvent_t e : b->late) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->in) cudaEventDestroy(b->in);
  if (b->out) cudaEventDestroy(b->out);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return CFDEM_OK;
}

cfdem_t cfdem_batch_bed(cfdem_batch_t b, int i) {
  if (!b || i < 0 || i >= (int)b->beds.size()) return nullptr;
  return b->beds[i];
}

cfdem_status cfdem_batch_set_graph(cfdem_batch_t b, int enable) {
  if (!b) return CFDEM_EINVAL;
  b->use_graph = enable != 0;
  if (!b->use_graph) {
    BatchDevice g(b->device);
    cudaStreamSynchronize(b->cap);
    drop_graph(b);
  }
  return CFDEM_OK;
}

int cfdem_batch_last_replayed(cfdem_batch_t b) { return b && b->replayed ? 1 : 0; }

cfdem_status cfdem_batch_coupling_step(cfdem_batch_t b, const cfdem_bed_io* io) {
  if (!b || !io) return CFDEM_EINVAL;
  BatchDevice g(b->device);
  b->err.clear();
  // order the batch after the caller's work
  BCK(cudaEventRecord(b->in, b->user), "order after the caller's stream");
  BCK(cudaStreamWaitEvent(b->cap, b->in, 0), "order after the caller's stream");
  cfdem_status st = CFDEM_OK;
  b->replayed = false;
  if (b->use_graph && same_key(b, io)) {
    BCK(cudaGraphLaunch(b->exec, b->cap), "graph launch");
    for (cfdem_t c : b->beds) c->stats_pending = true;
    b->replayed = true;
  } else {
    int bad = -1;
    st = step_all(b, io, &bad);
    if (st == CFDEM_OK && b->use_graph) {
      // capture the same step for the next calls; nothing runs here
      drop_graph(b);
      BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed), "begin capture");
      cfdem_status cs = step_all(b, io, &bad);
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->cap, &gr);
      if (cs != CFDEM_OK || e != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();  // the failed capture is not a sticky error
        if (cs == CFDEM_ESTATE) {
          // a bed whose step cannot be captured (stage timers on, a mixed
          // solve without the fast-diagonalisation preconditioner, or host
          // buffers that are not page-locked): the eager results stand and
          // this batch stays eager
          b->use_graph = false;
        } else {
          if (cs == CFDEM_OK) return bfail(b, "end capture", e);
          return cs;
        }
      }
      if (b->use_graph) {
        e = cudaGraphInstantiate(&b->exec, gr, 0);
        if (e != cudaSuccess) {
          cudaGraphDestroy(gr);
          b->exec = nullptr;
          cudaGetLastError();
          return bfail(b, "graph instantiate", e);
        }
        b->graph = gr;
        b->key_io.assign(io, io + b->beds.size());
        b->key_gen.resize(b->beds.size());
        for (size_t i = 0; i < b->beds.size(); ++i) b->key_gen[i] = b->beds[i]->gen;
      }
    }
  }
  BCK(cudaEventRecord(b->out, b->cap), "order the caller's stream after the batch");
  BCK(cudaStreamWaitEvent(b->user, b->out, 0), "order the caller's stream after the batch");
  return st;
}

const char* cfdem_batch_last_error(cfdem_batch_t b) { return b ? b->err.c_str() : "null batch"; }

cfdem_status cfdem_batch_synchronize(cfdem_batch_t b, int* first_failed_bed) {
  if (first_failed_bed) *first_failed_bed = -1;
  if (!b) return CFDEM_EINVAL;
  BatchDevice g(b->device);
  if (cudaStreamSynchronize(b->cap) != cudaSuccess) return CFDEM_ECUDA;
  cfdem_status first = CFDEM_OK;
  for (size_t i = 0; i < b->beds.size(); ++i) {
    cfdem_status s = cfdem_synchronize(b->beds[i]);
    if (s != CFDEM_OK && first == CFDEM_OK) {
      first = s;
      if (first_failed_bed) *first_failed_bed = (int)i;
    }
  }
  return first;
}

}  // extern "C"
