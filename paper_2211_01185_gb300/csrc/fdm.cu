// fdm.cu -- fast-diagonalisation preconditioner of the projection operator.
//
// On an axis-aligned box of equal elements the operator of the smoothed L2
// projection is the Kronecker sum
//   A = cM Mz(x)My(x)Mx + cKx Mz(x)My(x)Kx + cKy Mz(x)Ky(x)Mx + cKz Kz(x)My(x)Mx.
// With the generalised eigenvectors of each axis, K_a V_a = M_a V_a Lam_a and
// V_a^T M_a V_a = I (Lynch, Rice & Thomas 1964),
//   A^-1 = (Vz(x)Vy(x)Vx) D^-1 (Vz(x)Vy(x)Vx)^T,
//   D = cM + cKx lam_x + cKy lam_y + cKz lam_z   (one value per node).
// Applied in FP32 it is the inverse up to single-precision rounding, so the
// conjugate gradients it preconditions converge in a few iterations.  The six
// 1D transforms are plain dense GEMMs (cuBLAS SGEMM, FP32 math, no TF32).
//
// Host side: the 1D eigenproblems are solved once per mesh/parameter set:
// Cholesky M = L L^T, C = L^-1 K L^-T, symmetric eigen-decomposition of C by
// Householder reduction to tridiagonal form and implicit QR steps with
// Wilkinson shifts (Golub & Van Loan, Sec. 8.3), V = L^-T Q.
#include <cublas_v2.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "internal.h"

namespace cfdem {

namespace {

// symmetric eigen-decomposition: A (n x n, row-major) is replaced by the
// eigenvectors (columns), w receives the eigenvalues.  Returns false if the
// QR iteration did not converge.
bool sym_eig(int n, std::vector<double>& A, std::vector<double>& w) {
  std::vector<double> Q(n * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * (size_t)n + i] = 1.0;
  std::vector<double> v(n), p(n), q(n);
  // Householder reduction: for column k zero A[k+2.., k]
  for (int k = 0; k + 2 < n; ++k) {
    int m = n - k - 1;  // length of the sub-column below the diagonal
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = A[(k + 1 + i) * (size_t)n + k];
      nrm += v[i] * v[i];
    }
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    double alpha = v[0] > 0 ? -nrm : nrm;
    v[0] -= alpha;
    double vn = 0.0;
    for (int i = 0; i < m; ++i) vn += v[i] * v[i];
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = 0; i < m; ++i) v[i] /= vn;
    // trailing block B = A[k+1.., k+1..]: B <- H B H with H = I - 2 v v^T
    double K = 0.0;
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += A[(k + 1 + i) * (size_t)n + (k + 1 + j)] * v[j];
      p[i] = s;
      K += v[i] * s;
    }
    for (int i = 0; i < m; ++i) q[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        A[(k + 1 + i) * (size_t)n + (k + 1 + j)] -= 2.0 * (v[i] * q[j] + q[i] * v[j]);
    A[(k + 1) * (size_t)n + k] = alpha;
    A[k * (size_t)n + (k + 1)] = alpha;
    for (int i = 1; i < m; ++i) {
      A[(k + 1 + i) * (size_t)n + k] = 0.0;
      A[k * (size_t)n + (k + 1 + i)] = 0.0;
    }
    // Q <- Q H on columns k+1..
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += Q[r * (size_t)n + (k + 1 + j)] * v[j];
      for (int j = 0; j < m; ++j) Q[r * (size_t)n + (k + 1 + j)] -= 2.0 * s * v[j];
    }
  }
  std::vector<double> d(n), e(n > 1 ? n - 1 : 1, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A[i * (size_t)n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[(i + 1) * (size_t)n + i];
  // implicit symmetric QR on the tridiagonal (d, e), rotations into Q
  int hi = n - 1;
  long iters = 0;
  const long max_iters = 60L * n + 100;
  while (hi > 0) {
    // deflate converged bottom entries
    if (std::fabs(e[hi - 1]) <= 1e-16 * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 &&
           std::fabs(e[lo - 1]) > 1e-16 * (std::fabs(d[lo - 1]) + std::fabs(d[lo])))
      --lo;
    if (++iters > max_iters) return false;
    // Wilkinson shift from the trailing 2x2 block
    double delta = 0.5 * (d[hi - 1] - d[hi]);
    double eb = e[hi - 1];
    double den = delta + (delta >= 0 ? 1.0 : -1.0) * std::hypot(delta, eb);
    double mu = den != 0.0 ? d[hi] - eb * eb / den : d[hi];
    double x = d[lo] - mu, z = e[lo];
    double bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      double r = std::hypot(x, z);
      double c = r > 0 ? x / r : 1.0, s = r > 0 ? z / r : 0.0;
      if (k > lo) e[k - 1] = r;  // the bulge is folded into the previous off-diagonal
      double a = d[k], bb = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * bb + s * s * cc;
      d[k + 1] = s * s * a - 2.0 * c * s * bb + c * c * cc;
      e[k] = c * s * (cc - a) + (c * c - s * s) * bb;
      if (k + 1 < hi) {
        bulge = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
        z = bulge;
      }
      for (int r2 = 0; r2 < n; ++r2) {
        double vk = Q[r2 * (size_t)n + k], vk1 = Q[r2 * (size_t)n + k + 1];
        Q[r2 * (size_t)n + k] = c * vk + s * vk1;
        Q[r2 * (size_t)n + k + 1] = -s * vk + c * vk1;
      }
    }
  }
  w = d;
  A = Q;
  return true;
}

// assembled 1D matrix of ne elements of degree k from the reference block
void assemble_1d(int ne, int k, const double Mh[4][4], std::vector<double>& out) {
  int n = ne * k + 1;
  out.assign(n * (size_t)n, 0.0);
  for (int el = 0; el < ne; ++el)
    for (int a = 0; a <= k; ++a)
      for (int b = 0; b <= k; ++b) out[(el * k + a) * (size_t)n + (el * k + b)] += Mh[a][b];
}

// generalised eigenproblem K v = lam M v, V^T M V = I; V row-major (columns
// are eigenvectors)
bool gen_eig(int n, const std::vector<double>& M, const std::vector<double>& K,
             std::vector<double>& V, std::vector<double>& lam) {
  std::vector<double> L(M);
  // Cholesky, lower triangle
  for (int j = 0; j < n; ++j) {
    double s = L[j * (size_t)n + j];
    for (int k = 0; k < j; ++k) s -= L[j * (size_t)n + k] * L[j * (size_t)n + k];
    if (!(s > 0)) return false;
    double ljj = std::sqrt(s);
    L[j * (size_t)n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = L[i * (size_t)n + j];
      for (int k = 0; k < j; ++k) t -= L[i * (size_t)n + k] * L[j * (size_t)n + k];
      L[i * (size_t)n + j] = t / ljj;
    }
    for (int i = 0; i < j; ++i) L[i * (size_t)n + j] = 0.0;
  }
  // Y = L^-1 K (forward substitution per column), C = L^-1 Y^T
  std::vector<double> Y(n * (size_t)n), C(n * (size_t)n);
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      double t = K[i * (size_t)n + col];
      for (int k = 0; k < i; ++k) t -= L[i * (size_t)n + k] * Y[k * (size_t)n + col];
      Y[i * (size_t)n + col] = t / L[i * (size_t)n + i];
    }
  for (int col = 0; col < n; ++col)
    for (int i = 0; i < n; ++i) {
      double t = Y[col * (size_t)n + i];  // (Y^T)[i][col]
      for (int k = 0; k < i; ++k) t -= L[i * (size_t)n + k] * C[k * (size_t)n + col];
      C[i * (size_t)n + col] = t / L[i * (size_t)n + i];
    }
  for (int i = 0; i < n; ++i)  // symmetrise rounding
    for (int j = 0; j < i; ++j) {
      double a = 0.5 * (C[i * (size_t)n + j] + C[j * (size_t)n + i]);
      C[i * (size_t)n + j] = C[j * (size_t)n + i] = a;
    }
  if (!sym_eig(n, C, lam)) return false;
  // V = L^-T Q: back substitution L^T V = Q column by column
  V.assign(n * (size_t)n, 0.0);
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      double t = C[i * (size_t)n + col];
      for (int k = i + 1; k < n; ++k) t -= L[k * (size_t)n + i] * V[k * (size_t)n + col];
      V[i * (size_t)n + col] = t / L[i * (size_t)n + i];
    }
  // check V^T M V = I and V^T K V = diag(lam) on a few columns
  double err = 0.0, scale = 0.0;
  for (double l : lam) scale = std::fmax(scale, std::fabs(l));
  int step = n > 40 ? n / 20 : 1;
  for (int a = 0; a < n; a += step)
    for (int b = 0; b < n; b += step) {
      double sm = 0.0, sk = 0.0;
      for (int i = 0; i < n; ++i) {
        double mv = 0.0, kv = 0.0;
        for (int j = (i - 3 > 0 ? i - 3 : 0); j < n && j <= i + 3; ++j) {
          mv += M[i * (size_t)n + j] * V[j * (size_t)n + b];
          kv += K[i * (size_t)n + j] * V[j * (size_t)n + b];
        }
        sm += V[i * (size_t)n + a] * mv;
        sk += V[i * (size_t)n + a] * kv;
      }
      err = std::fmax(err, std::fabs(sm - (a == b ? 1.0 : 0.0)));
      err = std::fmax(err, std::fabs(sk - (a == b ? lam[a] : 0.0)) / (scale > 0 ? scale : 1.0));
    }
  return err < 1e-9;
}

__global__ void k_fdm_dinv(int nx, int ny, int nz, const double* __restrict__ lx,
                           const double* __restrict__ ly, const double* __restrict__ lz,
                           double cM, double cKx, double cKy, double cKz,
                           float* __restrict__ dinv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)nx * ny * nz;
  if (i >= n) return;
  int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((int64_t)nx * ny));
  double d = cM + cKx * lx[ix] + cKy * ly[iy] + cKz * lz[iz];
  dinv[i] = (float)(1.0 / d);
}

__global__ void k_scale(int64_t n, float* __restrict__ v, const float* __restrict__ s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s[i];
}

// row-major C[M x N] = A[M x K] B[K x N] (leading dims = row lengths), batched
cublasStatus_t gemm_rm(cublasHandle_t h, int M, int N, int K, const float* A, long long sA,
                       const float* B, long long sB, float* C, long long sC, int batch) {
  const float one = 1.0f, zero = 0.0f;
  // column-major view: C^T (N x M) = B^T (N x K) A^T (K x M)
  if (batch == 1)
    return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, N, M, K, &one, B, N, A, K, &zero, C, N);
  return cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, N, M, K, &one, B, N, sB, A, K,
                                   sA, &zero, C, N, sC, batch);
}

}  // namespace

struct FdmPlan {
  int n[3] = {0, 0, 0};
  float* V[3] = {nullptr, nullptr, nullptr};   // V_a row-major
  float* VT[3] = {nullptr, nullptr, nullptr};  // V_a^T row-major
  float* dinv = nullptr;                       // 1 / D per node
  float* tmp = nullptr;                        // work vector
  cublasHandle_t blas = nullptr;
};

void fdm_destroy(FdmPlan* p) {
  if (!p) return;
  for (int a = 0; a < 3; ++a) {
    if (p->V[a]) cudaFree(p->V[a]);
    if (p->VT[a]) cudaFree(p->VT[a]);
  }
  if (p->dinv) cudaFree(p->dinv);
  if (p->tmp) cudaFree(p->tmp);
  if (p->blas) cublasDestroy(p->blas);
  delete p;
}

cudaError_t fdm_create(const MeshDev& m, const Tables& t, const double coef[4],
                       FdmPlan** out, const char** why) {
  *out = nullptr;
  *why = nullptr;
  for (int a = 0; a < 3; ++a)
    if (m.nn[a] > 2049) {
      *why = "mesh axis longer than 2049 nodes";
      return cudaSuccess;
    }
  FdmPlan* p = new FdmPlan();
  std::vector<double> lam[3];
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    int n = m.nn[a];
    p->n[a] = n;
    std::vector<double> M, K, V;
    assemble_1d(m.ne[a], m.k, t.Mh, M);
    assemble_1d(m.ne[a], m.k, t.Kh, K);
    if (!gen_eig(n, M, K, V, lam[a])) {
      *why = "1D eigen-decomposition failed its check";
      fdm_destroy(p);
      return cudaSuccess;
    }
    std::vector<float> v32(n * (size_t)n), vt32(n * (size_t)n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        v32[i * (size_t)n + j] = (float)V[i * (size_t)n + j];
        vt32[j * (size_t)n + i] = (float)V[i * (size_t)n + j];
      }
    if ((e = cudaMalloc(&p->V[a], v32.size() * 4)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->VT[a], v32.size() * 4)) != cudaSuccess) break;
    if ((e = cudaMemcpy(p->V[a], v32.data(), v32.size() * 4, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      break;
    e = cudaMemcpy(p->VT[a], vt32.data(), vt32.size() * 4, cudaMemcpyHostToDevice);
  }
  double* dl[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    if ((e = cudaMalloc(&dl[a], lam[a].size() * 8)) != cudaSuccess) break;
    e = cudaMemcpy(dl[a], lam[a].data(), lam[a].size() * 8, cudaMemcpyHostToDevice);
  }
  int64_t nn = m.n_nodes;
  if (e == cudaSuccess) e = cudaMalloc(&p->dinv, nn * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->tmp, nn * 4);
  if (e == cudaSuccess) {
    k_fdm_dinv<<<(unsigned)((nn + 255) / 256), 256>>>(m.nn[0], m.nn[1], m.nn[2], dl[0], dl[1],
                                                       dl[2], coef[0], coef[1], coef[2],
                                                       coef[3], p->dinv);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  for (int a = 0; a < 3; ++a)
    if (dl[a]) cudaFree(dl[a]);
  if (e == cudaSuccess && cublasCreate(&p->blas) != CUBLAS_STATUS_SUCCESS) {
    *why = "cublasCreate failed";
    fdm_destroy(p);
    return cudaSuccess;
  }
  if (e == cudaSuccess) cublasSetMathMode(p->blas, CUBLAS_PEDANTIC_MATH);
  if (e != cudaSuccess) {
    fdm_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

// z = A^-1 r (FP32), r is preserved.  Uses p->tmp.
cudaError_t fdm_apply(FdmPlan* p, const float* r, float* z, cudaStream_t s) {
  cublasSetStream(p->blas, s);
  int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  long long plane = (long long)nx * ny;
  float* t = p->tmp;
  cublasStatus_t st;
  // forward transforms with V^T: x, y, z
  st = gemm_rm(p->blas, nz * ny, nx, nx, r, 0, p->V[0], 0, t, 0, 1);               // t = r Vx
  if (st == CUBLAS_STATUS_SUCCESS)
    st = gemm_rm(p->blas, ny, nx, ny, p->VT[1], 0, t, plane, z, plane, nz);         // z_k = VyT t_k
  if (st == CUBLAS_STATUS_SUCCESS)
    st = gemm_rm(p->blas, nz, (int)plane, nz, p->VT[2], 0, z, 0, t, 0, 1);         // t = VzT z
  if (st != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  int64_t n = plane * nz;
  int vb = (int)((n + 255) / 256);
  vb = vb > 1216 ? 1216 : vb;
  k_scale<<<vb, 256, 0, s>>>(n, t, p->dinv);
  count_launches(1);
  // inverse transforms with V: z, y, x
  st = gemm_rm(p->blas, nz, (int)plane, nz, p->V[2], 0, t, 0, z, 0, 1);            // z = Vz t
  if (st == CUBLAS_STATUS_SUCCESS)
    st = gemm_rm(p->blas, ny, nx, ny, p->V[1], 0, z, plane, t, plane, nz);          // t_k = Vy z_k
  if (st == CUBLAS_STATUS_SUCCESS)
    st = gemm_rm(p->blas, nz * ny, nx, nx, t, 0, p->VT[0], 0, z, 0, 1);             // z = t VxT
  if (st != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  return cudaGetLastError();
}

}  // namespace cfdem
