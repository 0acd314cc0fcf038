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
//    kernel transforms each z-slab in shared memory, one solves the banded
//    systems along z (one lane per mode), one transforms back.  The 1D
//    matrices of a uniform axis are persymmetric, so the eigenvectors are
//    symmetric or antisymmetric and each 1D transform is a butterfly
//    (x_i +- x_(n-1-i)) and two half-size products (see SlabAxis): about
//    2 (nx + ny) + 6 k flops per node instead of 4 (nx + ny + nz).
//  * dense form (slabs too large for shared memory): the six 1D transforms as
//    plain dense GEMMs (cuBLAS SGEMM, FP32 math, no TF32).
//
// Host side: the 1D eigenproblems are solved once per mesh/parameter set:
// Cholesky M = L L^T, C = L^-1 K L^-T, symmetric eigen-decomposition of C by
// Householder reduction to tridiagonal form and implicit QR steps with
// Wilkinson shifts (Golub & Van Loan, Sec. 8.3), V = L^-T Q.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "internal.h"
#include "reduce.cuh"

namespace cfdem {

namespace {

constexpr int kSlabSmemMax = 220 * 1024;  // dynamic shared memory of the slab form, at most

// padded row length of the slab-form transform matrices and tiles: a
// multiple of 8 for the 8 x 8 register tiles, plus 4 against bank conflicts
__host__ __device__ __forceinline__ int slab_pad(int n) { return ((n + 7) & ~7) + 4; }

// Parity split of one axis of n nodes.  On a uniform axis the mass and
// stiffness matrices are persymmetric (unchanged by reversing the node
// order), so their generalised eigenvectors split into symmetric ones (ye of
// them) and antisymmetric ones (yo): with s_i = x_i + x_(n-1-i) and
// d_i = x_i - x_(n-1-i) (i < n/2; s also holds the middle node for odd n),
// the forward transform is y_e = Ce^T s, y_o = Co^T d, and the inverse
// (a = Ce y_e, b = Co y_o) writes x_i = a_i + b_i, x_(n-1-i) = a_i - b_i --
// half the multiply-adds of the full transform.  In shared memory an axis
// is held in "slots": positions (or modes) 0 .. ye-1 in slots 0 .. ye-1,
// the rest from slot oe = ye rounded up to 4, so that both halves start
// 16-byte aligned; d_i sits in the slot of x_(n-1-i).
struct SlabAxis {
  int n, ye, oe, sl;  // nodes, symmetric count, start of the second half, slots
};
__host__ __device__ __forceinline__ SlabAxis slab_axis(int n) {
  SlabAxis a;
  a.n = n;
  a.ye = (n + 1) / 2;
  a.oe = (a.ye + 3) & ~3;
  a.sl = a.oe + n / 2;
  return a;
}
__host__ __device__ __forceinline__ int slot_of(const SlabAxis& a, int p) {
  return p < a.ye ? p : a.oe + (p - a.ye);
}


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

// Generalised eigenpairs of a persymmetric pair (M, K) on its symmetric and
// antisymmetric subspaces (orthonormal bases (e_i +- e_(n-1-i)) / sqrt 2 and
// the middle e_(n/2) for odd n; the antisymmetric vector of slot t pairs
// i = n/2 - 1 - t).  G (sl x sl, row-major, slots of slab_axis(n)) receives
// the folded transforms Ce = D Ve, Co = Vo / sqrt 2 on its diagonal blocks
// (D = 1 / sqrt 2, 1 for the middle node), lam the eigenvalues in mode
// order (symmetric first).  False if (M, K) is not persymmetric to 1e-12 of
// its largest entry, or an eigen-decomposition fails its check.
bool parity_eig(int n, const std::vector<double>& M, const std::vector<double>& K,
                std::vector<double>& G, std::vector<double>& lam) {
  const SlabAxis ax = slab_axis(n);
  const int my = n / 2, ye = ax.ye, yo = n / 2;
  double mm = 0.0, km = 0.0;
  for (size_t i = 0; i < M.size(); ++i) {
    mm = std::fmax(mm, std::fabs(M[i]));
    km = std::fmax(km, std::fabs(K[i]));
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t a = i * (size_t)n + j, b = (n - 1 - i) * (size_t)n + (n - 1 - j);
      if (std::fabs(M[a] - M[b]) > 1e-12 * mm || std::fabs(K[a] - K[b]) > 1e-12 * km)
        return false;
    }
  const double r2 = 1.0 / std::sqrt(2.0);
  // basis vectors: two entries each (index, weight)
  auto sym = [&](int i, int* p, double* w) {
    if (i < my) {
      p[0] = i, p[1] = n - 1 - i, w[0] = w[1] = r2;
    } else {
      p[0] = p[1] = my, w[0] = 1.0, w[1] = 0.0;
    }
  };
  auto anti = [&](int t, int* p, double* w) {
    const int i = my - 1 - t;
    p[0] = i, p[1] = n - 1 - i, w[0] = r2, w[1] = -r2;
  };
  auto reduce = [&](int m, auto basis, const std::vector<double>& A, std::vector<double>& R) {
    R.assign(m * (size_t)m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        int pi[2], pj[2];
        double wi[2], wj[2];
        basis(i, pi, wi);
        basis(j, pj, wj);
        double v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) v += wi[a] * A[pi[a] * (size_t)n + pj[b]] * wj[b];
        R[i * (size_t)m + j] = v;
      }
  };
  std::vector<double> Me, Ke, Mo, Ko, Ve, Vo, le, lo;
  reduce(ye, sym, M, Me);
  reduce(ye, sym, K, Ke);
  reduce(yo, anti, M, Mo);
  reduce(yo, anti, K, Ko);
  if (!gen_eig(ye, Me, Ke, Ve, le)) return false;
  if (yo > 0 && !gen_eig(yo, Mo, Ko, Vo, lo)) return false;
  G.assign(ax.sl * (size_t)ax.sl, 0.0);
  for (int i = 0; i < ye; ++i)
    for (int j = 0; j < ye; ++j)
      G[i * (size_t)ax.sl + j] = (i < my ? r2 : 1.0) * Ve[i * (size_t)ye + j];
  for (int t = 0; t < yo; ++t)
    for (int u = 0; u < yo; ++u)
      G[(ax.oe + t) * (size_t)ax.sl + ax.oe + u] = r2 * Vo[t * (size_t)yo + u];
  lam = le;
  lam.insert(lam.end(), lo.begin(), lo.end());
  return true;
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

// C[M x N] = A[M x K] B[K x N] in shared memory with A stored transposed
// (AT[K][lda]) and B row-major (B[K][ldb]); lda, ldb multiples of 4 floats
// and AT, B, C 16-byte aligned.
// Each thread owns a TR x TC block of C (TR, TC = 4 or 8), so one k step is
// TR/4 + TC/4 128-bit loads and TR TC FMAs; the loads of step k + 1 are
// issued before the FMAs of step k.  Threads form a gm x gn grid (gm =
// ceil(M/TR), gn = ceil(N/TC)); rows and columns past M, N read padding and
// are not stored.  With TRANS_C the block is stored transposed, C[c][r]
// (row length ldc, a multiple of 4), as 128-bit stores.
template <int TR, int TC, bool TRANS_C>
__device__ __forceinline__ void smem_gemm(int tbase, const float* AT, int lda, const float* B,
                                          int ldb, float* C, int ldc, int M, int N, int K) {
  const int gn = (N + TC - 1) / TC, gm = (M + TR - 1) / TR;
  const int tid = (int)threadIdx.x - tbase;  // threads [tbase, tbase + gm gn) take part
  if (tid < 0 || tid >= gm * gn) return;
  const int r0 = (tid / gn) * TR, c0 = (tid % gn) * TC;
  float acc[TR][TC];
#pragma unroll
  for (int a = 0; a < TR; ++a)
#pragma unroll
    for (int b = 0; b < TC; ++b) acc[a][b] = 0.f;
  const float4* ap = reinterpret_cast<const float4*>(AT + r0);
  const float4* bp = reinterpret_cast<const float4*>(B + c0);
  const int la = lda >> 2, lb = ldb >> 2;
  float4 av[TR / 4], bv[TC / 4];
#pragma unroll
  for (int q = 0; q < TR / 4; ++q) av[q] = ap[q];
#pragma unroll
  for (int q = 0; q < TC / 4; ++q) bv[q] = bp[q];
  // the last step also reads row K of A and B (discarded): the caller's
  // shared memory holds a row past every operand
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    ap += la;
    bp += lb;
    float4 an[TR / 4], bn[TC / 4];
#pragma unroll
    for (int q = 0; q < TR / 4; ++q) an[q] = ap[q];
#pragma unroll
    for (int q = 0; q < TC / 4; ++q) bn[q] = bp[q];
    const float* a = reinterpret_cast<const float*>(av);
    const float* b = reinterpret_cast<const float*>(bv);
#pragma unroll
    for (int x = 0; x < TR; ++x)
#pragma unroll
      for (int y = 0; y < TC; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
#pragma unroll
    for (int q = 0; q < TR / 4; ++q) av[q] = an[q];
#pragma unroll
    for (int q = 0; q < TC / 4; ++q) bv[q] = bn[q];
  }
  if (TRANS_C) {
    // 128-bit stores of row groups that hold at least one row < M: the
    // writes stay below M rounded up to 4
#pragma unroll
    for (int y = 0; y < TC; ++y) {
      const int c = c0 + y;
      if (c >= N) continue;
#pragma unroll
      for (int q = 0; q < TR / 4; ++q)
        if (r0 + 4 * q < M)
          *reinterpret_cast<float4*>(C + c * ldc + r0 + 4 * q) =
              make_float4(acc[4 * q][y], acc[4 * q + 1][y], acc[4 * q + 2][y], acc[4 * q + 3][y]);
    }
  } else {
#pragma unroll
    for (int x = 0; x < TR; ++x)
#pragma unroll
      for (int y = 0; y < TC; ++y) {
        int r = r0 + x, c = c0 + y;
        if (r < M && c < N) C[r * ldc + c] = acc[x][y];
      }
  }
}

// asynchronous global -> shared copies (no register round trip, every copy of
// a thread in flight at once); completion by cp.async.wait_all
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// The transform of an axis of n nodes is block diagonal in slots (the two
// parity halves); only its two diagonal blocks are stored, packed: rows
// 0 .. ye-1 the first block, rows ye .. n-1 the second, one more row that
// only the products' last prefetch reads, each row slab_pad(ye) floats
// (slab_packed_floats(n) in all).
__host__ __device__ __forceinline__ int slab_packed_floats(int n) {
  return (n + 1) * slab_pad((n + 1) / 2);
}

struct SlabArgs {
  int nx, ny, nz;
  const float* My;  // y transform, packed blocks
  const float* Mx;  // x transform, packed blocks
};

// Forward (INV = false): out_z = modes of in_z, the y transform then the x
// transform, each as a butterfly (s, d) then two half-size products (My, Mx
// hold Ce and Co on their diagonal blocks).  Inverse (INV = true): the
// products with the transposed blocks, then the butterfly that unfolds
// them.  Mode order in global memory: the symmetric modes of an axis first,
// then the antisymmetric ones (the z solves take their eigenvalues in that
// order).  One block per z-slab; the two halves of each product run side by
// side on two groups of whole warps.
//
// With dot.r set (the inverse transform that writes z), the kernel also
// forms r . z of the CG from the values it stores: one FP32 sum per thread,
// block sums, the last block to finish adds the blocks' sums in block order
// and sets rz and the Fletcher-Reeves beta = rz_new / rz_old (not on the
// first application) -- the dot product kernel that would read r and z
// again is not launched.
template <int TR, int TC, bool INV>
__global__ void k_fdm_slab(SlabArgs sa, const float* __restrict__ in, int in_stride,
                           float* __restrict__ out, int out_stride,
                           const int* __restrict__ done, FdmDot dot) {
  if (done && *(volatile const int*)done) return;
  __shared__ double red[32];
  float rz = 0.f;
  extern __shared__ __align__(16) float fsm[];
  const int nx = sa.nx, ny = sa.ny, nz = sa.nz;
  const SlabAxis ax = slab_axis(nx), ay = slab_axis(ny);
  const int lx = slab_pad(ax.sl), ly = slab_pad(ay.sl);
  const int lpx = slab_pad(ax.ye), lpy = slab_pad(ay.ye);  // packed matrix rows
  float* X = fsm;                   // [sl_y][lx]  slab in slots; also the result Y
  float* PT = X + ay.sl * lx;       // [sl_x][ly]  after the y transform, transposed
  float* MX = PT + ax.sl * ly;      // [nx + 1][lpx]  packed blocks
  float* MY = MX + (nx + 1) * lpx;  // [ny + 1][lpy]  packed blocks
  for (int t = threadIdx.x; t < slab_packed_floats(nx) >> 2; t += blockDim.x)
    cp_async16(MX + 4 * t, sa.Mx + 4 * t);
  for (int t = threadIdx.x; t < slab_packed_floats(ny) >> 2; t += blockDim.x)
    cp_async16(MY + 4 * t, sa.My + 4 * t);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int yo = ny / 2, xo = nx / 2;
  // thread groups of the two halves (whole warps each)
  const int g1 = ((((ay.ye + TR - 1) / TR) * ((ax.sl + TC - 1) / TC)) + 31) & ~31;
  const int g2 = ((((ay.sl + TR - 1) / TR) * ((ax.ye + TC - 1) / TC)) + 31) & ~31;
  for (int z = blockIdx.x; z < nz; z += gridDim.x) {
    const float* src = in + (int64_t)z * in_stride;
    for (int y = wid; y < ny; y += nw) {
      float* row = X + slot_of(ay, y) * lx;
      for (int x = lane; x < nx; x += 32) cp_async4(row + slot_of(ax, x), src + y * nx + x);
    }
    cp_async_wait_all();
    __syncthreads();
    if (!INV) {
      // y butterfly on the rows of X
      for (int t = threadIdx.x; t < yo * ax.sl; t += blockDim.x) {
        const int i = t / ax.sl, c = t - i * ax.sl;
        float* r1 = X + i * lx + c;
        float* r2 = X + slot_of(ay, ny - 1 - i) * lx + c;
        const float a = *r1, b = *r2;
        *r1 = a + b;
        *r2 = a - b;
      }
      __syncthreads();
    }
    // y transform: PT[x slot][y slot] = sum_k MY[k][m] X[k][x], per half
    smem_gemm<TR, TC, true>(0, MY, lpy, X, lx, PT, ly, ay.ye, ax.sl, ay.ye);
    smem_gemm<TR, TC, true>(g1, MY + ay.ye * lpy, lpy, X + ay.oe * lx, lx, PT + ay.oe, ly, yo,
                            ax.sl, yo);
    __syncthreads();
    // x butterfly: forward on the rows of PT (before the x products); the
    // inverse y unfold on the columns of PT (after the y products)
    if (!INV) {
      for (int t = threadIdx.x; t < xo * ay.sl; t += blockDim.x) {
        const int i = t / ay.sl, c = t - i * ay.sl;
        float* r1 = PT + i * ly + c;
        float* r2 = PT + slot_of(ax, nx - 1 - i) * ly + c;
        const float a = *r1, b = *r2;
        *r1 = a + b;
        *r2 = a - b;
      }
    } else {
      for (int t = threadIdx.x; t < ax.sl * yo; t += blockDim.x) {
        const int r = t / yo, i = t - r * yo;
        float* c1 = PT + r * ly + i;
        float* c2 = PT + r * ly + slot_of(ay, ny - 1 - i);
        const float a = *c1, b = *c2;
        *c1 = a + b;
        *c2 = a - b;
      }
    }
    __syncthreads();
    // x transform: Y[y slot][x slot] = sum_k PT[k][y slot] MX[k][m], per half
    smem_gemm<TR, TC, false>(0, PT, ly, MX, lpx, X, lx, ay.sl, ax.ye, ax.ye);
    smem_gemm<TR, TC, false>(g2, PT + ax.oe * ly, ly, MX + ax.ye * lpx, lpx, X + ax.oe, lx,
                             ay.sl, xo, xo);
    __syncthreads();
    if (INV) {
      // x unfold on the columns of Y
      for (int t = threadIdx.x; t < ay.sl * xo; t += blockDim.x) {
        const int r = t / xo, i = t - r * xo;
        float* c1 = X + r * lx + i;
        float* c2 = X + r * lx + slot_of(ax, nx - 1 - i);
        const float a = *c1, b = *c2;
        *c1 = a + b;
        *c2 = a - b;
      }
      __syncthreads();
    }
    float* dst = out + (int64_t)z * out_stride;
    const float* rr = dot.r ? dot.r + (int64_t)z * nx * ny : nullptr;
    for (int y = wid; y < ny; y += nw) {
      const float* row = X + slot_of(ay, y) * lx;
      for (int x = lane; x < nx; x += 32) {
        const float v = row[slot_of(ax, x)];
        dst[y * nx + x] = v;
        if (rr) rz = fmaf(rr[y * nx + x], v, rz);
      }
    }
    __syncthreads();
  }
  if (dot.r) {
    const double sblk = block_sum(rz, red);
    double vals[1] = {sblk};
    double o[1];
    if (last_block_reduce(dot.partials, 1, vals, &dot.sc->ticket, o, red) && threadIdx.x == 0) {
      if (!dot.first) dot.sc->beta = o[0] / dot.sc->rz;
      dot.sc->rz = o[0];
    }
  }
}

// banded solves along z: for every mode m (x-y index of the transformed slab)
// solve L D L^T w = t with the host factors; fac[z][c][mode] = L(z, z-1-c)
// for c < K, fac[z][K][mode] = 1 / D(z) (mode stride ms, a multiple of 4).
// One lane per mode, 32 modes per block; the block's lines and factors are
// copied to shared memory by all its threads with asynchronous copies.
//
// Both recurrences (forward L u = t, backward L^T y = D^-1 u) are split
// into kZSeg (8 or 16) segments of z, one warp each.  A recurrence of order K is
// linear in its K-value carried state, so a segment maps its incoming state
// c_in to its outgoing state as c_out = p + T c_in, with p the result from a
// zero incoming state and T (K x K per mode and segment) fixed by the
// factors alone, tabulated on the host (tr) and staged with the lines.
// Pass 1: every warp runs its segment from a zero state and keeps p; warp 0
// chains the states through the segments with T; pass 2: every warp reruns
// its segment from its true incoming state and writes the result.
// 2 x nz / kZSeg dependent steps per warp instead of nz, all warps busy.

template <int K, int kZSeg>
__global__ void __launch_bounds__(32 * kZSeg)
k_fdm_zsolve(int nmodes, int ms, int nz, const float* __restrict__ fac,
             const float* __restrict__ tr, float* __restrict__ v, const int* __restrict__ done) {
  if (done && *(volatile const int*)done) return;
  extern __shared__ __align__(16) float zsm[];
  float* line = zsm;                          // [nz][32]
  float* f = line + nz * 32;                  // [nz][K+1][32]
  float* car = f + nz * (K + 1) * 32;         // [kZSeg][K][32]  segment results from zero
  float* cin = car + kZSeg * K * 32;          // [kZSeg][K][32]  true incoming states
  float* tm = cin + kZSeg * K * 32;           // [2][kZSeg][K][K][32] transfer matrices
  const int m0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const bool full = m0 + 32 <= nmodes;
  if (full) {
    for (int t = threadIdx.x; t < nz * 8; t += blockDim.x) {
      int z = t >> 3, q = t & 7;
      cp_async16(line + 4 * t, v + (int64_t)z * ms + m0 + 4 * q);
    }
    for (int t = threadIdx.x; t < nz * (K + 1) * 8; t += blockDim.x) {
      int zc = t >> 3, q = t & 7;
      cp_async16(f + 4 * t, fac + (int64_t)zc * ms + m0 + 4 * q);
    }
  } else {
    for (int t = threadIdx.x; t < nz * 32; t += blockDim.x) {
      int z = t >> 5, l = t & 31, mode = m0 + l;
      if (mode < nmodes) cp_async4(line + t, v + (int64_t)z * ms + mode);
      else line[t] = 0.f;
    }
    for (int t = threadIdx.x; t < nz * (K + 1) * 32; t += blockDim.x) {
      int zc = t >> 5, l = t & 31, mode = m0 + l;
      if (mode < nmodes) cp_async4(f + t, fac + (int64_t)zc * ms + mode);
      else f[t] = (zc % (K + 1)) == K ? 1.f : 0.f;
    }
  }
  for (int t = threadIdx.x; t < 2 * kZSeg * K * K * 32; t += blockDim.x) {
    const int row = t >> 5, l = t & 31, md = m0 + l;
    if (md < nmodes) cp_async4(tm + t, tr + (int64_t)row * ms + md);
    else tm[t] = 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  const int zs = seg * nz / kZSeg, ze = (seg + 1) * nz / kZSeg;
  // transfer matrix entry T[dir][s][i][j] of this lane's mode
  auto T = [&](int dir, int s, int i, int j) {
    return tm[(((dir * kZSeg + s) * K + i) * K + j) * 32 + lane];
  };
  // forward step at z: u = t(z) - sum_c L(z, z-1-c) w[c]; w[0] newest
  auto fwd = [&](float* w, bool store) {
#pragma unroll 4
    for (int z = zs; z < ze; ++z) {
      float u = line[z * 32 + lane];
#pragma unroll
      for (int c = K - 1; c >= 0; --c) u -= f[(z * (K + 1) + c) * 32 + lane] * w[c];
#pragma unroll
      for (int c = K - 1; c > 0; --c) w[c] = w[c - 1];
      w[0] = u;
      if (store) line[z * 32 + lane] = u;
    }
  };
  // backward step at z: y = u(z) / D(z) - sum_c L(z+1+c, z) v[c]; v[0] newest
  auto bwd = [&](float* w, bool store) {
#pragma unroll 4
    for (int z = ze - 1; z >= zs; --z) {
      float y = line[z * 32 + lane] * f[(z * (K + 1) + K) * 32 + lane];
#pragma unroll
      for (int c = K - 1; c >= 0; --c) {
        const int zz = z + 1 + c;
        const float l = zz < nz ? f[(zz * (K + 1) + c) * 32 + lane] : 0.f;
        y -= l * w[c];
      }
#pragma unroll
      for (int c = K - 1; c > 0; --c) w[c] = w[c - 1];
      w[0] = y;
      if (store) line[z * 32 + lane] = y;
    }
  };
  float w[K];
  // ---- forward
#pragma unroll
  for (int c = 0; c < K; ++c) w[c] = 0.f;
  fwd(w, false);
#pragma unroll
  for (int c = 0; c < K; ++c) car[(seg * K + c) * 32 + lane] = w[c];
  __syncthreads();
  if (seg == 0) {
    float st[K];
#pragma unroll
    for (int c = 0; c < K; ++c) st[c] = 0.f;
    for (int s = 0; s < kZSeg; ++s) {
#pragma unroll
      for (int c = 0; c < K; ++c) cin[(s * K + c) * 32 + lane] = st[c];
      if (s + 1 == kZSeg) break;
      float nx[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        float a = car[(s * K + i) * 32 + lane];
#pragma unroll
        for (int j = 0; j < K; ++j) a += T(0, s, i, j) * st[j];
        nx[i] = a;
      }
#pragma unroll
      for (int c = 0; c < K; ++c) st[c] = nx[c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) w[c] = cin[(seg * K + c) * 32 + lane];
  fwd(w, true);
  __syncthreads();
  // ---- backward
#pragma unroll
  for (int c = 0; c < K; ++c) w[c] = 0.f;
  bwd(w, false);
#pragma unroll
  for (int c = 0; c < K; ++c) car[(seg * K + c) * 32 + lane] = w[c];
  __syncthreads();
  if (seg == 0) {
    float st[K];
#pragma unroll
    for (int c = 0; c < K; ++c) st[c] = 0.f;
    for (int s = kZSeg - 1; s >= 0; --s) {
#pragma unroll
      for (int c = 0; c < K; ++c) cin[(s * K + c) * 32 + lane] = st[c];
      if (s == 0) break;
      float nx[K];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        float a = car[(s * K + i) * 32 + lane];
#pragma unroll
        for (int j = 0; j < K; ++j) a += T(1, s, i, j) * st[j];
        nx[i] = a;
      }
#pragma unroll
      for (int c = 0; c < K; ++c) st[c] = nx[c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < K; ++c) w[c] = cin[(seg * K + c) * 32 + lane];
  bwd(w, true);
  __syncthreads();
  if (full) {
    for (int t = threadIdx.x; t < nz * 8; t += blockDim.x) {
      int z = t >> 3, q = t & 7;
      *reinterpret_cast<float4*>(v + (int64_t)z * ms + m0 + 4 * q) =
          reinterpret_cast<const float4*>(line)[t];
    }
  } else {
    for (int t = threadIdx.x; t < nz * 32; t += blockDim.x) {
      int z = t >> 5, l = t & 31, md = m0 + l;
      if (md < nmodes) v[(int64_t)z * ms + md] = line[t];
    }
  }
}

// Segment transfer matrices of the two z recurrences (see k_fdm_zsolve),
// from the FP32 factors the device uses: tr[dir][s][i][j][mode] is entry
// (i, j) of the map from a segment's incoming K-value state to its outgoing
// state with zero right-hand side (dir 0 forward, 1 backward).
void zsolve_transfers(int nz, int k, int kZSeg, const std::vector<float>& fac, int stride,
                      int nm, std::vector<float>& tr) {
  tr.assign((size_t)2 * kZSeg * k * k * stride, 0.f);
  auto F = [&](int z, int c, int m) { return (double)fac[((size_t)z * (k + 1) + c) * stride + m]; };
  std::vector<double> w(k), nw(k);
  for (int m = 0; m < nm; ++m)
    for (int s = 0; s < kZSeg; ++s) {
      const int zs = s * nz / kZSeg, ze = (s + 1) * nz / kZSeg;
      for (int j = 0; j < k; ++j) {
        // forward
        std::fill(w.begin(), w.end(), 0.0);
        w[j] = 1.0;
        for (int z = zs; z < ze; ++z) {
          double u = 0.0;
          for (int c = 0; c < k; ++c) u -= F(z, c, m) * w[c];
          for (int c = k - 1; c > 0; --c) w[c] = w[c - 1];
          w[0] = u;
        }
        for (int i = 0; i < k; ++i)
          tr[((size_t)((0 * kZSeg + s) * k + i) * k + j) * stride + m] = (float)w[i];
        // backward
        std::fill(w.begin(), w.end(), 0.0);
        w[j] = 1.0;
        for (int z = ze - 1; z >= zs; --z) {
          double y = 0.0;
          for (int c = 0; c < k; ++c) {
            const int zz = z + 1 + c;
            if (zz < nz) y -= F(zz, c, m) * w[c];
          }
          for (int c = k - 1; c > 0; --c) w[c] = w[c - 1];
          w[0] = y;
        }
        for (int i = 0; i < k; ++i)
          tr[((size_t)((1 * kZSeg + s) * k + i) * k + j) * stride + m] = (float)w[i];
      }
    }
}

// host LDL^T factors of s Mz + cKz Kz (band rows of half-width k) for every
// mode, in FP64, stored in FP32 as fac[z][c][mode] = L(z, z-1-c) (c < k) and
// fac[z][k][mode] = 1 / D(z), mode stride `stride`
void band_ldlt_factors(int nz, int k, const std::vector<double>& Mz,
                       const std::vector<double>& Kz, double cKz,
                       const std::vector<double>& s_modes, int stride, std::vector<float>& fac) {
  const int nm = (int)s_modes.size();
  fac.assign((size_t)nz * (k + 1) * stride, 0.f);
  std::vector<double> L((size_t)nz * k), D(nz);
  auto lw = [&](int i, int j) {  // L(i, j) for i - k <= j < i
    return L[(size_t)i * k + (i - 1 - j)];
  };
  for (int m = 0; m < nm; ++m) {
    const double s = s_modes[m];
    auto A = [&](int i, int j) {
      return s * Mz[(size_t)i * nz + j] + cKz * Kz[(size_t)i * nz + j];
    };
    for (int i = 0; i < nz; ++i) {
      for (int c = k - 1; c >= 0; --c) {  // L(i, i-1-c), farther columns first
        int j = i - 1 - c;
        double val = 0.0;
        if (j >= 0) {
          val = A(i, j);
          for (int p = (i - k > 0 ? i - k : 0); p < j; ++p) val -= lw(i, p) * lw(j, p) * D[p];
          val /= D[j];
        }
        L[(size_t)i * k + c] = val;
      }
      double d = A(i, i);
      for (int p = (i - k > 0 ? i - k : 0); p < i; ++p) d -= lw(i, p) * lw(i, p) * D[p];
      D[i] = d;
      for (int c = 0; c < k; ++c)
        fac[((size_t)i * (k + 1) + c) * stride + m] = (float)L[(size_t)i * k + c];
      fac[((size_t)i * (k + 1) + k) * stride + m] = (float)(1.0 / d);
    }
  }
}

}  // namespace

// threads of k_fdm_slab<tr, tc> for an nx x ny slab: the larger of its two
// products, each run as two halves on groups of whole warps
static int slab_threads_for(int nx, int ny, int tr, int tc) {
  const SlabAxis ax = slab_axis(nx), ay = slab_axis(ny);
  auto cnt = [&](int m, int n) { return ((m + tr - 1) / tr) * ((n + tc - 1) / tc); };
  auto w32 = [](int t) { return (t + 31) & ~31; };
  const int t1 = w32(cnt(ay.ye, ax.sl)) + w32(cnt(ny / 2, ax.sl));
  const int t2 = w32(cnt(ay.sl, ax.ye)) + w32(cnt(ay.sl, nx / 2));
  return t1 > t2 ? t1 : t2;
}

struct FdmPlan {
  int n[3] = {0, 0, 0};
  int k = 1;
  bool slab = false;          // slab form (x, y diagonalised, banded z solves)
  float* fac = nullptr;       // slab form: LDL^T factors [nz][k+1][ms]
  float* tr = nullptr;        // slab form: z-segment transfer matrices [2][zseg][k][k][ms]
  int zseg = 8;               // slab form: z-segments of the banded solves (8 or 16)
  size_t slab_smem = 0, z_smem = 0;
  int slab_threads = 256;
  int slab_tr = 4, slab_tc = 4;  // register tile of the slab transforms (rows x columns)
  int ms = 0;                 // slab form: padded plane stride of tmp and fac
  // dense form: V_a and V_a^T row-major.  Slab form (axes x, y): the two
  // diagonal blocks of the folded parity transforms G_a and G_a^T, packed
  // as SlabArgs describes
  float* V[3] = {nullptr, nullptr, nullptr};
  float* VT[3] = {nullptr, nullptr, nullptr};
  float* dinv = nullptr;                       // dense form: 1 / D per node
  float* tmp = nullptr;                        // work vector
  cublasHandle_t blas = nullptr;
};

static cudaError_t tune_slab(FdmPlan* p);

int fdm_tile(const FdmPlan* p) { return p && p->slab ? 10 * p->slab_tr + p->slab_tc : 0; }

void fdm_destroy(FdmPlan* p) {
  if (!p) return;
  for (int a = 0; a < 3; ++a) {
    if (p->V[a]) cudaFree(p->V[a]);
    if (p->VT[a]) cudaFree(p->VT[a]);
  }
  if (p->dinv) cudaFree(p->dinv);
  if (p->tmp) cudaFree(p->tmp);
  if (p->fac) cudaFree(p->fac);
  if (p->tr) cudaFree(p->tr);
  if (p->blas) cublasDestroy(p->blas);
  delete p;
}

cudaError_t fdm_create(const MeshDev& m, const Tables& t, const double coef[4], FdmPlan** out,
                       const char** why) {
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
  {
    const SlabAxis ax = slab_axis(nx), ay = slab_axis(ny);
    const size_t lx = slab_pad(ax.sl), ly = slab_pad(ay.sl);
    // k_fdm_slab: X / Y [sl_y][lx], PT [sl_x][ly], and the packed blocks of
    // the two transforms (each with the row the products' last prefetch reads)
    p->slab_smem = (ay.sl * lx + ax.sl * ly + (size_t)slab_packed_floats(nx) +
                    (size_t)slab_packed_floats(ny)) * sizeof(float);
    // 4 x 4 register tiles (more warps per slab) where the thread count allows
    // 4 x 4 register tiles where the thread count allows (timed against the
    // other shapes once the plan is built)
    p->slab_tr = p->slab_tc = slab_threads_for(nx, ny, 4, 4) <= 1024 ? 4 : 8;
    p->slab_threads = slab_threads_for(nx, ny, p->slab_tr, p->slab_tc);
    if (p->slab_threads > 1024) p->slab_smem = (size_t)1 << 30;  // dense form instead
  }
  // 16 z-segments where the lines, factors, states and transfer matrices fit
  // in shared memory, else 8
  auto zsmem = [&](int seg) {
    return ((size_t)nz * 32 * (m.k + 2) + (size_t)2 * seg * m.k * 32 +
            (size_t)2 * seg * m.k * m.k * 32) * sizeof(float);
  };
  p->zseg = zsmem(16) <= 220 * 1024 ? 16 : 8;
  p->z_smem = zsmem(p->zseg);
  p->slab = p->slab_smem <= (size_t)kSlabSmemMax && p->z_smem <= 220 * 1024;
  std::vector<double> lam[3];
  cudaError_t e = cudaSuccess;
  const int naxes = p->slab ? 2 : 3;
  for (int a = 0; a < naxes && e == cudaSuccess; ++a) {
    const int n = m.nn[a];
    std::vector<double> M, K, V;
    assemble_1d(m.ne[a], m.k, t.Mh, M);
    assemble_1d(m.ne[a], m.k, t.Kh, K);
    // slab form: the parity-split transforms over the axis' slots; dense
    // form: the full transform
    const int rows = p->slab ? slab_axis(n).sl : n;
    const int ld = p->slab ? slab_pad(rows) : n;
    const bool ok = p->slab ? parity_eig(n, M, K, V, lam[a]) : gen_eig(n, M, K, V, lam[a]);
    if (!ok) {
      *why = "1D eigen-decomposition failed its check";
      fdm_destroy(p);
      return cudaSuccess;
    }
    std::vector<float> v32(rows * (size_t)ld, 0.f), vt32(rows * (size_t)ld, 0.f);
    for (int i = 0; i < rows; ++i)
      for (int j = 0; j < rows; ++j) {
        v32[i * (size_t)ld + j] = (float)V[i * (size_t)rows + j];
        vt32[j * (size_t)ld + i] = (float)V[i * (size_t)rows + j];
      }
    if (p->slab) {  // keep the two diagonal blocks only, packed (SlabArgs)
      const SlabAxis sa = slab_axis(n);
      const int lp = slab_pad(sa.ye);
      auto pack = [&](const std::vector<float>& F) {
        std::vector<float> P((size_t)slab_packed_floats(n), 0.f);
        for (int k = 0; k < sa.ye; ++k)
          for (int c = 0; c < sa.ye; ++c) P[k * (size_t)lp + c] = F[k * (size_t)ld + c];
        for (int k = 0; k < n / 2; ++k)
          for (int c = 0; c < n / 2; ++c)
            P[(sa.ye + k) * (size_t)lp + c] = F[(sa.oe + k) * (size_t)ld + sa.oe + c];
        return P;
      };
      v32 = pack(v32);
      vt32 = pack(vt32);
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
    // banded LDL^T factors of s_m Mz + cKz Kz for every (x, y) mode m, with
    // s_m = cM + cKx lam_x + cKy lam_y
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
    std::vector<float> tr;
    zsolve_transfers(nz, m.k, p->zseg, fac, p->ms, nx * ny, tr);
    if (e == cudaSuccess && (e = cudaMalloc(&p->tr, tr.size() * 4)) == cudaSuccess)
      e = cudaMemcpy(p->tr, tr.data(), tr.size() * 4, cudaMemcpyHostToDevice);
    // the dynamic shared-memory limit is a property of the kernel, shared by
    // every plan (context) of the process: raise it to the device's opt-in
    // maximum rather than to this plan's size, which a later plan with
    // smaller slabs would otherwise lower below what this one launches with
    int dev = 0, optin = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && ((size_t)optin < p->slab_smem || (size_t)optin < p->z_smem))
      e = cudaErrorInvalidValue;
    // the slab kernels also hold a little static shared memory (the dot
    // product's block sums): their dynamic share is capped at the slab
    // form's own limit, which leaves room for it
    const int slab_cap = std::min(optin, kSlabSmemMax);
#define CFDEM_SLAB_ATTR(TR_, TC_, INV_)                                                     \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_fdm_slab<TR_, TC_, INV_>,                                     \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, slab_cap);
    CFDEM_SLAB_ATTR(4, 4, false)
    CFDEM_SLAB_ATTR(4, 4, true)
    CFDEM_SLAB_ATTR(4, 8, false)
    CFDEM_SLAB_ATTR(4, 8, true)
    CFDEM_SLAB_ATTR(8, 4, false)
    CFDEM_SLAB_ATTR(8, 4, true)
    CFDEM_SLAB_ATTR(8, 8, false)
    CFDEM_SLAB_ATTR(8, 8, true)
#undef CFDEM_SLAB_ATTR
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fdm_zsolve<3, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
    if (e == cudaSuccess) e = tune_slab(p);
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

static void launch_slab(const FdmPlan* p, int nblk, cudaStream_t s, bool inv, const float* in,
                        int is, float* out, int os, const int* done, FdmDot dd) {
  SlabArgs sa{p->n[0], p->n[1], p->n[2], inv ? p->VT[1] : p->V[1], inv ? p->VT[0] : p->V[0]};
#define CFDEM_SLAB(TR_, TC_)                                                                  \
  do {                                                                                        \
    if (inv)                                                                                  \
      k_fdm_slab<TR_, TC_, true><<<nblk, p->slab_threads, p->slab_smem, s>>>(sa, in, is, out, \
                                                                             os, done, dd);   \
    else                                                                                      \
      k_fdm_slab<TR_, TC_, false><<<nblk, p->slab_threads, p->slab_smem, s>>>(sa, in, is, out, \
                                                                              os, done, dd);  \
  } while (0)
  if (p->slab_tr == 4 && p->slab_tc == 4) CFDEM_SLAB(4, 4);
  else if (p->slab_tr == 4) CFDEM_SLAB(4, 8);
  else if (p->slab_tc == 4) CFDEM_SLAB(8, 4);
  else CFDEM_SLAB(8, 8);
#undef CFDEM_SLAB
}

// The register tile of the slab transforms: each shape whose thread count
// fits is timed on the plan's own sizes (the forward transform of a zeroed
// work vector, CUDA events, best of five after two warm-up launches) and the
// fastest kept.  Every shape sums each output over the same k order, so the
// choice does not change a bit of the result.
static cudaError_t tune_slab(FdmPlan* p) {
  const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  const int nm = nx * ny;
  const int nblk = nz < 304 ? nz : 304;
  const int shapes[4][2] = {{4, 4}, {4, 8}, {8, 4}, {8, 8}};
  cudaError_t e = cudaMemset(p->tmp, 0, ((size_t)nz * p->ms + (size_t)nm * nz) * sizeof(float));
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  float best = 1e30f;
  int btr = p->slab_tr, btc = p->slab_tc;
  for (const auto& sh : shapes) {
    const int th = slab_threads_for(nx, ny, sh[0], sh[1]);
    if (th > 1024) continue;
    p->slab_tr = sh[0];
    p->slab_tc = sh[1];
    p->slab_threads = th;
    float tmin = 1e30f;
    for (int it = 0; it < 7 && e == cudaSuccess; ++it) {
      e = cudaEventRecord(a, 0);
      if (e == cudaSuccess)
        launch_slab(p, nblk, 0, false, p->tmp, p->ms, p->tmp + (size_t)nz * p->ms, nm, nullptr,
                    FdmDot{});
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(b, 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && it >= 2 && ms < tmin) tmin = ms;
    }
    if (e != cudaSuccess) break;
    if (tmin < best) {
      best = tmin;
      btr = sh[0];
      btc = sh[1];
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->slab_tr = btr;
  p->slab_tc = btc;
  p->slab_threads = slab_threads_for(nx, ny, btr, btc);
  return e;
}

// z = A^-1 r (FP32), r is preserved.  Uses p->tmp.  The slab-form kernels
// return at once when *done is set (a converged CG), so iterations can be
// queued without host round trips.
cudaError_t fdm_apply(FdmPlan* p, const float* r, float* z, const int* done, cudaStream_t s,
                      const FdmDot* dot, bool* dot_done) {
  int nx = p->n[0], ny = p->n[1], nz = p->n[2];
  if (dot_done) *dot_done = false;
  if (p->slab) {
    int nblk = nz < 304 ? nz : 304;
    int nm = nx * ny;
    launch_slab(p, nblk, s, false, r, nm, p->tmp, p->ms, done, FdmDot{});
    unsigned zb = (unsigned)((nm + 31) / 32);
#define CFDEM_ZS(KK, SS)                                                                   \
  k_fdm_zsolve<KK, SS><<<zb, 32 * SS, p->z_smem, s>>>(nm, p->ms, nz, p->fac, p->tr, p->tmp, done)
    if (p->zseg == 16) {
      if (p->k == 1) CFDEM_ZS(1, 16);
      else if (p->k == 2) CFDEM_ZS(2, 16);
      else CFDEM_ZS(3, 16);
    } else {
      if (p->k == 1) CFDEM_ZS(1, 8);
      else if (p->k == 2) CFDEM_ZS(2, 8);
      else CFDEM_ZS(3, 8);
    }
#undef CFDEM_ZS
    launch_slab(p, nblk, s, true, p->tmp, p->ms, z, nm, done, dot ? *dot : FdmDot{});
    if (dot_done) *dot_done = dot != nullptr;
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
