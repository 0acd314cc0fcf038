// mapped.cu -- particle location on mapped (curved) Q_k hex meshes.
//
// The paper's beds sit in curved meshes (a subdivided cylinder, Secs. 3.1
// and 3.2; a gmsh mesh, Sec. 3.4) and the particles are located on the fluid
// mesh itself (Sec. 2.3).  Element e maps the reference cube [0,1]^3 by its
// Q_k nodes, X_e(xi) = sum_j P_j l_a(xi_0) l_b(xi_1) l_c(xi_2), and a point x
// lies in e when X_e(xi) = x for a xi in the cube.
//
// Location, one thread per particle: the point's cell of a uniform grid
// lists, in ascending element index, every element whose node box (widened
// by `margin` times its largest edge) overlaps the cell; the elements whose
// widened box contains the point are tried in that order by Newton's method
// on X_e(xi) = x from the cube's centre (FP64; at most 50 steps, converged
// once the largest step component is at most 1e-13, abandoned once xi leaves
// [-3, 4]^3 or the Jacobian is singular), and the first whose xi lies in
// [-1e-10, 1 + 1e-10]^3 is the element (xi clamped to the cube).  The boxes
// are computed on the host with the oracle's arithmetic, so the candidates
// are the same elements in the same order.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/cfdem.h"
#include "internal.h"
#include "device_common.cuh"

struct cfdem_mapped {
  int device = 0;
  int k = 1;
  int64_t E = 0, N = 0;
  cfdem::Tables tab{};
  int32_t* conn = nullptr;   // [E][(k+1)^3]
  double* nodes = nullptr;   // [N][3]
  double* box = nullptr;     // [E][6] widened lo, hi
  int32_t* cell_start = nullptr;
  int32_t* cell_elems = nullptr;
  double g0[3] = {0, 0, 0}, inv_cs[3] = {0, 0, 0};
  int nc[3] = {1, 1, 1};
};

namespace {

using cfdem::Tables;

struct MappedDev {
  int k;
  const int32_t* conn;
  const double* nodes;
  const double* box;
  const int32_t* cell_start;
  const int32_t* cell_elems;
  double g0[3], inv_cs[3];
  int nc[3];
};

// Newton inversion of the map of element e at p (see the file comment);
// returns true with xi in the cube, else false
template <int K>
__device__ bool newton_in(const MappedDev& md, const Tables& tb, int64_t e, const double p[3],
                          double xi_out[3]) {
  constexpr int NQ = K + 1, NL = NQ * NQ * NQ;
  double xi[3] = {0.5, 0.5, 0.5};
  const int32_t* cn = md.conn + e * NL;
  for (int it = 0; it < 50; ++it) {
    double l[3][NQ], dl[3][NQ];
#pragma unroll
    for (int a = 0; a < 3; ++a) cfdem::lagrange<K, double>(tb.z, tb.lw, xi[a], l[a], dl[a]);
    double X[3] = {0.0, 0.0, 0.0}, J[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
          const double* P = md.nodes + 3 * (int64_t)cn[a + NQ * (b + NQ * c)];
          const double w = l[0][a] * l[1][b] * l[2][c];
          const double w0 = dl[0][a] * l[1][b] * l[2][c];
          const double w1 = l[0][a] * dl[1][b] * l[2][c];
          const double w2 = l[0][a] * l[1][b] * dl[2][c];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const double Pi = __ldg(P + i);
            X[i] += w * Pi;
            J[i][0] += w0 * Pi;
            J[i][1] += w1 * Pi;
            J[i][2] += w2 * Pi;
          }
        }
    const double r[3] = {X[0] - p[0], X[1] - p[1], X[2] - p[2]};
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(fabs(det) > 0.0)) return false;
    double d[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {  // Cramer's rule
      double M[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = j == col ? r[i] : J[i][j];
      const double dm = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                        M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                        M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      d[col] = dm / det;
    }
    double big = 0.0;
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xi[a] -= d[a];
      big = fmax(big, fabs(d[a]));
      inside = inside && xi[a] >= -3.0 && xi[a] <= 4.0;
    }
    if (!inside) return false;
    if (big <= 1e-13) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (!(xi[a] >= -1e-10 && xi[a] <= 1.0 + 1e-10)) return false;
#pragma unroll
      for (int a = 0; a < 3; ++a) xi_out[a] = fmin(fmax(xi[a], 0.0), 1.0);
      return true;
    }
  }
  return false;
}

template <int K>
__global__ void __launch_bounds__(128)
k_locate_mapped(MappedDev md, Tables tb, int64_t n, const double* __restrict__ x,
                int32_t* __restrict__ elem, double* __restrict__ xi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
  int32_t found = -1;
  double xo[3] = {0.0, 0.0, 0.0};
  int ci[3];
  bool in_grid = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double t = (p[a] - md.g0[a]) * md.inv_cs[a];
    in_grid = in_grid && t >= 0.0 && t <= (double)md.nc[a];  // false for NaN
    ci[a] = in_grid ? min((int)t, md.nc[a] - 1) : 0;
  }
  if (in_grid) {
    const int64_t cell = ci[0] + (int64_t)md.nc[0] * (ci[1] + (int64_t)md.nc[1] * ci[2]);
    for (int32_t s = md.cell_start[cell]; s < md.cell_start[cell + 1]; ++s) {
      const int32_t e = md.cell_elems[s];
      const double* bx = md.box + 6 * (int64_t)e;
      if (!(p[0] >= bx[0] && p[0] <= bx[3] && p[1] >= bx[1] && p[1] <= bx[4] && p[2] >= bx[2] &&
            p[2] <= bx[5]))
        continue;
      if (newton_in<K>(md, tb, e, p, xo)) {
        found = e;
        break;
      }
    }
  }
  elem[i] = found;
  if (xi) {
    xi[3 * i] = found >= 0 ? xo[0] : 0.0;
    xi[3 * i + 1] = found >= 0 ? xo[1] : 0.0;
    xi[3 * i + 2] = found >= 0 ? xo[2] : 0.0;
  }
}

// out[i][c] = sum_j field[conn[e][j]][c] phi_j(xi_i) (0 where elem < 0)
template <int K>
__global__ void k_interp_mapped(MappedDev md, Tables tb, int64_t n,
                                const int32_t* __restrict__ elem, const double* __restrict__ xi,
                                int ncomp, const double* __restrict__ field,
                                double* __restrict__ out) {
  constexpr int NQ = K + 1, NL = NQ * NQ * NQ;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t e = elem[i];
  if (e < 0) {
    for (int c = 0; c < ncomp; ++c) out[i * ncomp + c] = 0.0;
    return;
  }
  double l[3][NQ];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    cfdem::lagrange<K, double>(tb.z, tb.lw, xi[3 * i + a], l[a], (double*)nullptr);
  const int32_t* cn = md.conn + (int64_t)e * NL;
  for (int c = 0; c < ncomp; ++c) {
    double v = 0.0;
#pragma unroll
    for (int cc = 0; cc < NQ; ++cc)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int a = 0; a < NQ; ++a)
          v += l[0][a] * l[1][b] * l[2][cc] *
               __ldg(field + (int64_t)cn[a + NQ * (b + NQ * cc)] * ncomp + c);
    out[i * ncomp + c] = v;
  }
}

MappedDev dev_view(const cfdem_mapped* m) {
  MappedDev d;
  d.k = m->k;
  d.conn = m->conn;
  d.nodes = m->nodes;
  d.box = m->box;
  d.cell_start = m->cell_start;
  d.cell_elems = m->cell_elems;
  for (int a = 0; a < 3; ++a) {
    d.g0[a] = m->g0[a];
    d.inv_cs[a] = m->inv_cs[a];
    d.nc[a] = m->nc[a];
  }
  return d;
}

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void release(cfdem_mapped* m) {
  void* ps[] = {m->conn, m->nodes, m->box, m->cell_start, m->cell_elems};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
}

template <typename T>
bool upload(T** dst, const T* src, size_t count) {
  if (cudaMalloc((void**)dst, sizeof(T) * (count > 0 ? count : 1)) != cudaSuccess) return false;
  return count == 0 ||
         cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

extern "C" cfdem_status cfdem_mapped_create(cfdem_mapped_t* out, int device, int degree,
                                            int64_t n_elem, const int32_t* conn,
                                            int64_t n_nodes, const double* nodes,
                                            double margin) {
  if (!out) return CFDEM_EINVAL;
  *out = nullptr;
  if (degree < 1 || degree > 3 || n_elem < 1 || n_elem >= ((int64_t)1 << 31) || n_nodes < 1 ||
      n_nodes >= ((int64_t)1 << 31) || !conn || !nodes || !(margin >= 0.0 && margin <= 1.0))
    return CFDEM_EINVAL;
  const int nl = (degree + 1) * (degree + 1) * (degree + 1);
  for (int64_t j = 0; j < n_elem * nl; ++j)
    if (conn[j] < 0 || conn[j] >= n_nodes) return CFDEM_EINVAL;
  for (int64_t j = 0; j < 3 * n_nodes; ++j)
    if (!std::isfinite(nodes[j])) return CFDEM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return CFDEM_ECUDA;
  // widened node boxes, as the oracle computes them
  std::vector<double> box(6 * n_elem);
  double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double vol = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < nl; ++j) {
      const double* P = nodes + 3 * (int64_t)conn[e * nl + j];
      for (int a = 0; a < 3; ++a) {
        if (P[a] < lo[a]) lo[a] = P[a];
        if (P[a] > hi[a]) hi[a] = P[a];
      }
    }
    double side = 0.0;
    for (int a = 0; a < 3; ++a)
      if (hi[a] - lo[a] > side) side = hi[a] - lo[a];
    const double w = margin * side;
    for (int a = 0; a < 3; ++a) {
      lo[a] -= w;
      hi[a] += w;
      box[6 * e + a] = lo[a];
      box[6 * e + 3 + a] = hi[a];
      glo[a] = std::fmin(glo[a], lo[a]);
      ghi[a] = std::fmax(ghi[a], hi[a]);
    }
    vol += (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  }
  cfdem_mapped* m = new cfdem_mapped();
  m->device = device;
  m->k = degree;
  m->E = n_elem;
  m->N = n_nodes;
  cfdem::make_tables(degree, degree, &m->tab);
  // grid of cells about the mean box size, at most 2^22 cells
  double cs = std::cbrt(vol / (double)n_elem);
  for (;;) {
    int64_t tot = 1;
    for (int a = 0; a < 3; ++a) {
      const double ext = ghi[a] - glo[a];
      double f = cs > 0 ? std::ceil(ext / cs) : 1.0;
      m->nc[a] = f < 1.0 ? 1 : (f > 4096.0 ? 4096 : (int)f);
      tot *= m->nc[a];
    }
    if (tot <= ((int64_t)1 << 22)) break;
    cs *= 1.5;
  }
  for (int a = 0; a < 3; ++a) {
    const double ext = ghi[a] - glo[a];
    m->g0[a] = glo[a];
    m->inv_cs[a] = ext > 0 ? (double)m->nc[a] / ext : 0.0;
  }
  const int64_t ncell = (int64_t)m->nc[0] * m->nc[1] * m->nc[2];
  std::vector<int32_t> count(ncell + 1, 0);
  auto cell_range = [&](int64_t e, int a, int* c0, int* c1) {
    const double t0 = (box[6 * e + a] - m->g0[a]) * m->inv_cs[a];
    const double t1 = (box[6 * e + 3 + a] - m->g0[a]) * m->inv_cs[a];
    *c0 = std::max(0, std::min(m->nc[a] - 1, (int)std::floor(t0)));
    *c1 = std::max(0, std::min(m->nc[a] - 1, (int)std::floor(t1)));
  };
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int32_t> fill;
    if (pass == 1) {
      for (int64_t c = 0; c < ncell; ++c) count[c + 1] += count[c];
      fill.assign(count.begin(), count.end() - 1);
    }
    std::vector<int32_t> elems(pass == 1 ? count[ncell] : 0);
    for (int64_t e = 0; e < n_elem; ++e) {  // ascending: each cell's list is sorted
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) cell_range(e, a, &lo[a], &hi[a]);
      for (int cz = lo[2]; cz <= hi[2]; ++cz)
        for (int cy = lo[1]; cy <= hi[1]; ++cy)
          for (int cx = lo[0]; cx <= hi[0]; ++cx) {
            const int64_t c = cx + (int64_t)m->nc[0] * (cy + (int64_t)m->nc[1] * cz);
            if (pass == 0)
              ++count[c + 1];
            else
              elems[fill[c]++] = (int32_t)e;
          }
    }
    if (pass == 1) {
      Guard g(device);
      if (!upload(&m->cell_elems, elems.data(), elems.size()) ||
          !upload(&m->cell_start, count.data(), count.size()) ||
          !upload(&m->conn, conn, (size_t)(n_elem * nl)) ||
          !upload(&m->nodes, nodes, (size_t)(3 * n_nodes)) ||
          !upload(&m->box, box.data(), box.size())) {
        release(m);
        return CFDEM_ENOMEM;
      }
    }
  }
  *out = m;
  return CFDEM_OK;
}

extern "C" cfdem_status cfdem_mapped_destroy(cfdem_mapped_t m) {
  if (!m) return CFDEM_OK;
  Guard g(m->device);
  cudaDeviceSynchronize();
  release(m);
  return CFDEM_OK;
}

extern "C" cfdem_status cfdem_mapped_locate(cfdem_mapped_t m, int64_t n, const double* x,
                                            int32_t* elem, double* xi, void* stream) {
  if (!m || n < 0 || (n > 0 && (!x || !elem))) return CFDEM_EINVAL;
  if (n == 0) return CFDEM_OK;
  Guard g(m->device);
  const MappedDev d = dev_view(m);
  const unsigned nb = (unsigned)((n + 127) / 128);
  cudaStream_t s = (cudaStream_t)stream;
  if (m->k == 1) k_locate_mapped<1><<<nb, 128, 0, s>>>(d, m->tab, n, x, elem, xi);
  if (m->k == 2) k_locate_mapped<2><<<nb, 128, 0, s>>>(d, m->tab, n, x, elem, xi);
  if (m->k == 3) k_locate_mapped<3><<<nb, 128, 0, s>>>(d, m->tab, n, x, elem, xi);
  cfdem::count_launches(1);
  return cudaGetLastError() == cudaSuccess ? CFDEM_OK : CFDEM_ECUDA;
}

extern "C" cfdem_status cfdem_mapped_interpolate(cfdem_mapped_t m, int64_t n, const int32_t* elem,
                                                 const double* xi, int ncomp,
                                                 const double* field, double* out,
                                                 void* stream) {
  if (!m || n < 0 || ncomp < 1 || ncomp > 64 || (n > 0 && (!elem || !xi || !field || !out)))
    return CFDEM_EINVAL;
  if (n == 0) return CFDEM_OK;
  Guard g(m->device);
  const MappedDev d = dev_view(m);
  const unsigned nb = (unsigned)((n + 127) / 128);
  cudaStream_t s = (cudaStream_t)stream;
  if (m->k == 1) k_interp_mapped<1><<<nb, 128, 0, s>>>(d, m->tab, n, elem, xi, ncomp, field, out);
  if (m->k == 2) k_interp_mapped<2><<<nb, 128, 0, s>>>(d, m->tab, n, elem, xi, ncomp, field, out);
  if (m->k == 3) k_interp_mapped<3><<<nb, 128, 0, s>>>(d, m->tab, n, elem, xi, ncomp, field, out);
  cfdem::count_launches(1);
  return cudaGetLastError() == cudaSuccess ? CFDEM_OK : CFDEM_ECUDA;
}
