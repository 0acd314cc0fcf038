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
// conjugate gradients it preconditions converge in a few iterations.
//
// Two device forms:
//  * slab form (default): only x and y are diagonalised.  For a mode (i, j)
//    the z operator is the banded SPD matrix s_ij Mz + cKz Kz with s_ij = cM +
//    cKx lam_x,i + cKy lam_y,j, factorised A = L D L^T on the host.  One
//    kernel transforms each z-slab with Vx, Vy^T in shared memory, one solves
//    the banded systems along z (one lane per mode), one transforms back:
//    about 4 (nx + ny) + 6 k flops per node instead of 4 (nx + ny + nz).
//  * dense form (slabs too large for shared memory): the six 1D transforms as
//    plain dense GEMMs (cuBLAS SGEMM, FP32 math, no TF32).
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

// C[M x N] = A[M x K] B[K x N], row-major in shared memory.  The block is a
// tg x tg grid of threads (tg = ceil(max(M, N) / 5)), each owning the
// strided 5 x 5 outputs (ty + tg a, tx + tg b), so a 65-node slab runs on
// 13 x 13 threads with no idle outputs.
__device__ __forceinline__ void smem_gemm(const float* A, int lda, const float* B, int ldb,
                                          float* C, int ldc, int M, int N, int K, int tg) {
  const int tid = threadIdx.x;
  if (tid >= tg * tg) return;
  const int tx = tid % tg, ty = tid / tg;
  float acc[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) acc[a][b] = 0.f;
  int ra[5], cb[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    ra[a] = min(ty + tg * a, M - 1);
    cb[a] = min(tx + tg * a, N - 1);
  }
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float av[5], bv[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) av[a] = A[ra[a] * lda + k];
#pragma unroll
    for (int b = 0; b < 5; ++b) bv[b] = B[k * ldb + cb[b]];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int b = 0; b < 5; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      int r = ty + tg * a, c = tx + tg * b;
      if (r < M && c < N) C[r * ldc + c] = acc[a][b];
    }
}

// copy n floats global -> shared, 16-byte vectors when both are aligned
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, int n) {
  if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
    int n4 = n >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 4
    for (int t = threadIdx.x; t < n4; t += blockDim.x) d4[t] = s4[t];
    for (int t = (n4 << 2) + threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
  } else {
#pragma unroll 4
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
  }
}

// forward: out_z = Vy^T (in_z Vx); inverse: out_z = Vy (in_z Vx^T), one z-slab
// per block iteration; the two factors stay in shared memory
__global__ void k_fdm_slab(int nx, int ny, int nz, int tg, const float* __restrict__ Bx,
                           const float* __restrict__ Ay, const float* __restrict__ in,
                           int in_stride, float* __restrict__ out, int out_stride,
                           const int* __restrict__ done) {
  if (done && *(volatile const int*)done) return;
  extern __shared__ __align__(16) float fsm[];
  const int plane = nx * ny;
  const int p4 = (plane + 3) & ~3;  // keep every array 16-byte aligned
  float* X = fsm;                   // [ny][nx]
  float* T = X + p4;                // [ny][nx]
  float* MB = T + p4;               // [nx][nx]
  float* MA = MB + ((nx * nx + 3) & ~3);  // [ny][ny]
  stage(MB, Bx, nx * nx);
  stage(MA, Ay, ny * ny);
  for (int z = blockIdx.x; z < nz; z += gridDim.x) {
    stage(X, in + (int64_t)z * in_stride, plane);
    __syncthreads();
    smem_gemm(X, nx, MB, nx, T, nx, ny, nx, nx, tg);      // T = X Bx
    __syncthreads();
    smem_gemm(MA, ny, T, nx, X, nx, ny, nx, ny, tg);      // X = Ay T
    __syncthreads();
    float* dst = out + (int64_t)z * out_stride;
    if (((uintptr_t)dst & 15) == 0) {
      int n4 = plane >> 2;
      float4* d4 = reinterpret_cast<float4*>(dst);
      const float4* x4 = reinterpret_cast<const float4*>(X);
      for (int t = threadIdx.x; t < n4; t += blockDim.x) d4[t] = x4[t];
      for (int t = (n4 << 2) + threadIdx.x; t < plane; t += blockDim.x) dst[t] = X[t];
    } else {
      for (int t = threadIdx.x; t < plane; t += blockDim.x) dst[t] = X[t];
    }
    __syncthreads();
  }
}

// banded solves along z: for every mode m (x-y index of the transformed
// slab) solve L D L^T w = t with the host factors; fac[z][c][mode] = L(z,
// z-1-c) for c < K, fac[z][K][mode] = 1 / D(z).  One lane per mode; 32
// modes per block; lines and factors staged in shared memory by 8 warps with
// 16-byte loads, the recurrences run by warp 0.
template <int K>
__global__ void __launch_bounds__(256)
k_fdm_zsolve(int nmodes, int ms, int nz, const float* __restrict__ fac, float* __restrict__ v,
             const int* __restrict__ done) {
  if (done && *(volatile const int*)done) return;
  extern __shared__ __align__(16) float zsm[];
  float* line = zsm;                  // [nz][32]
  float* f = line + nz * 32;          // [nz][K+1][32]
  const int m0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31;
  // rows have stride ms (a multiple of 4 floats): whole 32-mode rows move as
  // 8 float4
  const bool full = m0 + 32 <= nmodes;
  if (full) {
    // rows of 32 floats = 8 float4 per row
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * 8; t += blockDim.x) {
      int z = t >> 3, q = t & 7;
      reinterpret_cast<float4*>(line)[t] =
          *reinterpret_cast<const float4*>(v + (int64_t)z * ms + m0 + 4 * q);
    }
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * (K + 1) * 8; t += blockDim.x) {
      int zc = t >> 3, q = t & 7;
      reinterpret_cast<float4*>(f)[t] =
          *reinterpret_cast<const float4*>(fac + (int64_t)zc * ms + m0 + 4 * q);
    }
  } else {
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * 32; t += blockDim.x) {
      int z = t >> 5, l = t & 31, mode = m0 + l;
      line[t] = mode < nmodes ? v[(int64_t)z * ms + mode] : 0.f;
    }
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * (K + 1) * 32; t += blockDim.x) {
      int l = t & 31, zc = t >> 5, mode = m0 + l;
      f[t] = mode < nmodes ? fac[(int64_t)zc * ms + mode] : 0.f;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float w[K];  // last K solved values
#pragma unroll
    for (int c = 0; c < K; ++c) w[c] = 0.f;
#pragma unroll 4
    for (int z = 0; z < nz; ++z) {  // L u = t
      float u = line[z * 32 + lane];
#pragma unroll
      for (int c = 0; c < K; ++c) u -= f[(z * (K + 1) + c) * 32 + lane] * w[c];
#pragma unroll
      for (int c = K - 1; c > 0; --c) w[c] = w[c - 1];
      w[0] = u;
      line[z * 32 + lane] = u;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) w[c] = 0.f;
#pragma unroll 4
    for (int z = nz - 1; z >= 0; --z) {  // L^T y = u / D
      float y = line[z * 32 + lane] * f[(z * (K + 1) + K) * 32 + lane];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        int zz = z + 1 + c;
        float lv = zz < nz ? f[(zz * (K + 1) + c) * 32 + lane] : 0.f;
        y -= lv * w[c];
      }
#pragma unroll
      for (int c = K - 1; c > 0; --c) w[c] = w[c - 1];
      w[0] = y;
      line[z * 32 + lane] = y;
    }
  }
  __syncthreads();
  if (full) {
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * 8; t += blockDim.x) {
      int z = t >> 3, q = t & 7;
      *reinterpret_cast<float4*>(v + (int64_t)z * ms + m0 + 4 * q) =
          reinterpret_cast<const float4*>(line)[t];
    }
  } else {
    for (int t = threadIdx.x; t < nz * 32; t += blockDim.x) {
      int z = t >> 5, l = t & 31, mode = m0 + l;
      if (mode < nmodes) v[(int64_t)z * ms + mode] = line[t];
    }
  }
}

// host LDL^T factors of s Mz + cKz Kz (bandwidth k) for every mode
void band_ldlt_factors(int nz, int k, const std::vector<double>& Mz,
                       const std::vector<double>& Kz, double cKz,
                       const std::vector<double>& s_modes, int stride, std::vector<float>& fac) {
  int nm = (int)s_modes.size();
  fac.assign((size_t)nz * (k + 1) * stride, 0.f);
  std::vector<double> L((size_t)nz * (k + 1)), D(nz);
  for (int m = 0; m < nm; ++m) {
    double s = s_modes[m];
    auto A = [&](int i, int j) {
      return s * Mz[(size_t)i * nz + j] + cKz * Kz[(size_t)i * nz + j];
    };
    for (int i = 0; i < nz; ++i) {
      // L(i, i-1-c) for c = k-1 .. 0 (farther first), then D(i)
      for (int c = k - 1; c >= 0; --c) {
        int j = i - 1 - c;
        double val = 0.0;
        if (j >= 0) {
          val = A(i, j);
          for (int p = (i - k > 0 ? i - k : 0); p < j; ++p)
            val -= L[(size_t)i * (k + 1) + (i - 1 - p)] * L[(size_t)j * (k + 1) + (j - 1 - p)] * D[p];
          val /= D[j];
        }
        L[(size_t)i * (k + 1) + c] = val;
      }
      double d = A(i, i);
      for (int p = (i - k > 0 ? i - k : 0); p < i; ++p) {
        double l = L[(size_t)i * (k + 1) + (i - 1 - p)];
        d -= l * l * D[p];
      }
      D[i] = d;
      for (int c = 0; c < k; ++c)
        fac[((size_t)i * (k + 1) + c) * stride + m] = (float)L[(size_t)i * (k + 1) + c];
      fac[((size_t)i * (k + 1) + k) * stride + m] = (float)(1.0 / d);
    }
  }
}

}  // namespace

struct FdmPlan {
  int n[3] = {0, 0, 0};
  int k = 1;
  bool slab = false;          // slab form (x, y diagonalised, banded z solves)
  float* fac = nullptr;       // slab form: LDL^T factors [nz][k+1][nx*ny]
  size_t slab_smem = 0, z_smem = 0;
  int tg = 16, slab_threads = 256;
  int ms = 0;                 // slab form: padded plane stride of tmp and fac
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
  if (p->fac) cudaFree(p->fac);
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
  p->k = m.k;
  for (int a = 0; a < 3; ++a) p->n[a] = m.nn[a];
  const int nx = m.nn[0], ny = m.nn[1], nz = m.nn[2];
  auto r4 = [](size_t v) { return (v + 3) & ~(size_t)3; };
  p->slab_smem = (2 * r4((size_t)nx * ny) + r4((size_t)nx * nx) + r4((size_t)ny * ny)) * sizeof(float);
  int mx = nx > ny ? nx : ny;
  p->tg = (mx + 4) / 5;
  p->slab_threads = ((p->tg * p->tg + 31) / 32) * 32;
  if (p->tg > 32) p->slab_smem = (size_t)1 << 30;   // beyond the thread budget: dense form
  p->z_smem = (size_t)nz * 32 * (m.k + 2) * sizeof(float);
  p->slab = p->slab_smem <= 200 * 1024 && p->z_smem <= 200 * 1024;
  std::vector<double> lam[3];
  cudaError_t e = cudaSuccess;
  const int naxes = p->slab ? 2 : 3;
  for (int a = 0; a < naxes && e == cudaSuccess; ++a) {
    int n = m.nn[a];
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
  int64_t nn = m.n_nodes;
  p->ms = (nx * ny + 3) & ~3;
  if (e == cudaSuccess) e = cudaMalloc(&p->tmp, (size_t)nz * p->ms * 4 + nn * 4);
  if (e == cudaSuccess && p->slab) {
    // banded LDL^T factors of s Mz + cKz Kz for every (x, y) mode
    std::vector<double> Mz, Kz;
    assemble_1d(m.ne[2], m.k, t.Mh, Mz);
    assemble_1d(m.ne[2], m.k, t.Kh, Kz);
    std::vector<double> smodes((size_t)nx * ny);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        smodes[i + (size_t)nx * j] = coef[0] + coef[1] * lam[0][i] + coef[2] * lam[1][j];
    std::vector<float> fac;
    band_ldlt_factors(nz, m.k, Mz, Kz, coef[3], smodes, p->ms, fac);
    if ((e = cudaMalloc(&p->fac, fac.size() * 4)) == cudaSuccess)
      e = cudaMemcpy(p->fac, fac.data(), fac.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_slab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)p->slab_smem);
    if (e == cudaSuccess) {
      if (m.k == 1)
        e = cudaFuncSetAttribute(k_fdm_zsolve<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->z_smem);
      else if (m.k == 2)
        e = cudaFuncSetAttribute(k_fdm_zsolve<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->z_smem);
      else
        e = cudaFuncSetAttribute(k_fdm_zsolve<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->z_smem);
    }
  } else if (e == cudaSuccess) {
    double* dl[3] = {nullptr, nullptr, nullptr};
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
      if ((e = cudaMalloc(&dl[a], lam[a].size() * 8)) != cudaSuccess) break;
      e = cudaMemcpy(dl[a], lam[a].data(), lam[a].size() * 8, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->dinv, nn * 4);
    if (e == cudaSuccess) {
      k_fdm_dinv<<<(unsigned)((nn + 255) / 256), 256>>>(nx, ny, nz, dl[0], dl[1], dl[2],
                                                         coef[0], coef[1], coef[2], coef[3],
                                                         p->dinv);
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
  }
  if (e != cudaSuccess) {
    fdm_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

// z = A^-1 r (FP32), r is preserved.  Uses p->tmp.  The slab-form kernels
// return at once when *done is set (a converged CG), so iterations can be
// queued without host round trips.
cudaError_t fdm_apply(FdmPlan* p, const float* r, float* z, const int* done, cudaStream_t s) {
  int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  if (p->slab) {
    int nblk = nz < 304 ? nz : 304;
    int nm = nx * ny;
    k_fdm_slab<<<nblk, p->slab_threads, p->slab_smem, s>>>(nx, ny, nz, p->tg, p->V[0], p->VT[1],
                                                            r, nm, p->tmp, p->ms, done);
    unsigned zb = (unsigned)((nm + 31) / 32);
    if (p->k == 1)
      k_fdm_zsolve<1><<<zb, 256, p->z_smem, s>>>(nm, p->ms, nz, p->fac, p->tmp, done);
    else if (p->k == 2)
      k_fdm_zsolve<2><<<zb, 256, p->z_smem, s>>>(nm, p->ms, nz, p->fac, p->tmp, done);
    else
      k_fdm_zsolve<3><<<zb, 256, p->z_smem, s>>>(nm, p->ms, nz, p->fac, p->tmp, done);
    k_fdm_slab<<<nblk, p->slab_threads, p->slab_smem, s>>>(nx, ny, nz, p->tg, p->VT[0], p->V[1],
                                                            p->tmp, p->ms, z, nm, done);
    count_launches(3);
    return cudaGetLastError();
  }
  cublasSetStream(p->blas, s);
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
