// noalloc.cu -- particle-centroid void fraction without any device allocation.
//
// Some callers cannot create a context, because creating one allocates
// device memory: solvers that hand every byte of the GPU to their own memory
// pool, and loops that must never pay the implicit device synchronisation a
// cudaMalloc can cause.  For them this file offers one entry point,
// cfdem_pcm_void_fraction_static, which needs only the caller's input and
// output buffers.  Its per-element scratch (the
// sum of particle volumes in each element) is the file-scope device array
// g_pcm_volume below, so its size is fixed when the library is loaded.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/cfdem.h"
#include "internal.h"

namespace {

// Scratch shared by every call on a device: the particle volume summed per
// element.  CFDEM_PCM_STATIC_MAX_ELEMS doubles (4 MiB), held by every GPU
// that loads the library until the process exits.
static __device__ __align__(256) double g_pcm_volume[CFDEM_PCM_STATIC_MAX_ELEMS];
// Status word the kernels write when a particle lies outside the mesh (the
// entry point does not read it back; such particles are simply left out).
// first_bad starts at ~0 so that the kernels' atomicMin on it is well formed.
static __device__ __align__(256) cfdem::DevStatus g_pcm_status = {~0ull, 0ull, 0, 0};

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_volume_ptr[kMaxDevices] = {};
cfdem::DevStatus* g_status_ptr[kMaxDevices] = {};

// Device addresses of the two arrays on the current device, looked up once
// per device with that device current.  Their names in host code are only
// host-side handles, so the addresses must come from cudaGetSymbolAddress.
// The cache assumes the device is not reset (cudaDeviceReset) while the
// process runs: a reset reloads the module and would leave stale addresses.
cudaError_t scratch_addresses(int dev, double** vol, cfdem::DevStatus** st) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_volume_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pcm_volume);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_pcm_status);
    if (e != cudaSuccess) return e;
    g_volume_ptr[dev] = static_cast<double*>(p);
    g_status_ptr[dev] = static_cast<cfdem::DevStatus*>(q);
  }
  *vol = g_volume_ptr[dev];
  *st = g_status_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" cfdem_status cfdem_pcm_void_fraction_static(const double origin[3],
                                                       const double extent[3],
                                                       const int n_el[3], int degree, int64_t n,
                                                       const double* x_dev, const double* r_dev,
                                                       double* eps_q_dev, void* stream) {
  using namespace cfdem;
  if (!origin || !extent || !n_el || !eps_q_dev || degree < 1 || degree > 3 || n < 0 ||
      (n > 0 && (!x_dev || !r_dev)))
    return CFDEM_EINVAL;
  MeshDev m{};
  for (int a = 0; a < 3; ++a) {
    // the same checks as cfdem_set_mesh: finite box, 1..2^20 elements per
    // axis (so the element count below cannot overflow)
    if (!std::isfinite(origin[a]) || !std::isfinite(extent[a]) || !(extent[a] > 0))
      return CFDEM_EINVAL;
    if (n_el[a] < 1 || n_el[a] > (1 << 20)) return CFDEM_EINVAL;
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
  m.Ve = m.h[0] * m.h[1] * m.h[2];
  m.Ve32 = (float)m.Ve;
  if (m.E > CFDEM_PCM_STATIC_MAX_ELEMS) return CFDEM_EINVAL;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CFDEM_ECUDA;
  double* vol = nullptr;
  DevStatus* st = nullptr;
  if (scratch_addresses(dev, &vol, &st) != cudaSuccess) return CFDEM_ECUDA;
  // the volumes are cleared on the stream before they are summed, so each
  // call starts from zero whatever the previous call left
  cudaError_t e = launch_pcm(m, n, x_dev, r_dev, vol, eps_q_dev, nullptr, st,
                             (cudaStream_t)stream);
  return e == cudaSuccess ? CFDEM_OK : CFDEM_ECUDA;
}
