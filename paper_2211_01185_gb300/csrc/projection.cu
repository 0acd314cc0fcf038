// projection.cu -- smoothed L2 projection of the void fraction (steps a4, a5).
//
// The "void fraction smoothing factor L^2" of the paper's parameter tables is
// read as the Helmholtz-smoothed L2 projection: find eps_h in Q_k with
//   int phi_j eps_h + L^2 int grad phi_j . grad eps_h = int phi_j eps_q
// for every nodal basis function phi_j, i.e. (M + L^2 K) eps_h = b.
//
// Matrix-free operator.  On an axis-aligned box of equal elements the
// assembled operator is the Kronecker sum
//   A = cM  Mz(x)My(x)Mx + cKx Mz(x)My(x)Kx + cKy Mz(x)Ky(x)Mx + cKz Kz(x)My(x)Mx
// of assembled 1D reference matrices (bandwidth k) with cM = hx hy hz and
// cKx = L^2 hy hz / hx etc.  k_apply evaluates it node by node with sum
// factorisation over a shared-memory tile with a halo of k nodes:
//   t1 = Mz x, t2 = Kz x          (z pass)
//   s1 = My t1, s2 = Ky t1, s3 = My t2
//   U = cM s1 + cKy s2 + cKz s3, V = cKx s1   (y pass)
//   y = Mx U + Kx V               (x pass)
// seven banded 1D applies per node, no atomics, deterministic.
//
// The right-hand side b_j = sum_e sum_q phi_j(x_q) w_q |J| eps_q is
// assembled element by element with sum factorisation (three 1D contractions)
// and atomic adds into the nodes.
//
// CG: Jacobi-preconditioned conjugate gradients with the scalars on the
// device.  Each kernel reduces its block partial sums in fixed order in the
// last block to finish, so dot products are deterministic, and every kernel
// returns at once after convergence.  The mixed path runs the same CG in FP32
// on the correction equation inside FP64 iterative refinement.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "df64.cuh"
#include "reduce.cuh"

namespace cfdem {

// ---------------------------------------------------------------------------
// right-hand side

// elements (threads) per block of k_rhs: the staged quadrature values fit 40 KB
template <int K, typename T>
constexpr int rhs_block() {
  return ((K + 1) * (K + 1) * (K + 1) * (int)sizeof(T) * 128 <= 40 * 1024) ? 128 : 64;
}

// Per element: its contribution to the right-hand side at each of its
// (k+1)^3 nodes, |J| sum_q phi_j(x_q) w_q eps_q, sum-factorised into three
// 1D contractions (x, then y, then z), one thread per element, in the path's
// precision T.  Written to local[j][e] (no atomics; k_rhs_gather adds the
// slots up per global node), element index fastest so that the stores of a
// warp coalesce.
template <int K, typename T>
__global__ void __launch_bounds__(128)
k_rhs(MeshDev m, Tables tb, const T* __restrict__ eps_q, T* __restrict__ local) {
  constexpr int NQ = K + 1;
  constexpr int Q = NQ * NQ * NQ;
  constexpr int NB = (Q * (int)sizeof(T) * 128 <= 40 * 1024) ? 128 : 64;
  __shared__ T sh[NB * Q];
  const int64_t E = m.E, e0 = blockIdx.x * (int64_t)NB;
  const int64_t tot = E - e0 < NB ? (E - e0) * Q : (int64_t)NB * Q;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) sh[t] = eps_q[e0 * Q + t];
  __syncthreads();
  const int64_t e = e0 + threadIdx.x;
  if (e >= E) return;
  constexpr bool F32 = std::is_same<T, float>::value;
  T B[NQ][NQ];  // B[a][q] = l_a(g_q) w_q (the FP32 path takes the host's FP32 copy)
#pragma unroll
  for (int a = 0; a < NQ; ++a)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if constexpr (F32) B[a][q] = tb.Bwf[a][q];
      else B[a][q] = (T)tb.Bw[a][q];
    }
  const T* ev = sh + threadIdx.x * Q;
  T t1[NQ][NQ][NQ];  // [qz][qy][a]
#pragma unroll
  for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
    for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        T s = 0;
#pragma unroll
        for (int qx = 0; qx < NQ; ++qx) s += B[a][qx] * ev[qx + NQ * (qy + NQ * qz)];
        t1[qz][qy][a] = s;
      }
  T t2[NQ][NQ][NQ];  // [qz][b][a]
#pragma unroll
  for (int qz = 0; qz < NQ; ++qz)
#pragma unroll
    for (int bb = 0; bb < NQ; ++bb)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        T s = 0;
#pragma unroll
        for (int qy = 0; qy < NQ; ++qy) s += B[bb][qy] * t1[qz][qy][a];
        t2[qz][bb][a] = s;
      }
  T detJ;
  if constexpr (F32) detJ = m.Ve32;
  else detJ = (T)m.Ve;
#pragma unroll
  for (int c = 0; c < NQ; ++c)
#pragma unroll
    for (int bb = 0; bb < NQ; ++bb)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        T s = 0;
#pragma unroll
        for (int qz = 0; qz < NQ; ++qz) s += B[c][qz] * t2[qz][bb][a];
        local[(a + NQ * (bb + NQ * c)) * E + e] = s * detJ;
      }
}

// b_j = sum of the element contributions to node j, added in a fixed order
// (elements ascending) in the path's precision T and stored in FP64.  One
// thread per element writes the nodes the element owns: local indices
// 0..k-1 along each axis, and k on the last element of an axis.  A node with
// local index 0 along an axis also takes the contribution of the element
// before it on that axis (local index k there), so a node sums one to eight
// slots.  Grid: x along a row of elements (element index fastest, so that
// for every slot neighbouring threads read neighbouring words of local[j][.]),
// y over e_y, z over e_z (both strided when the mesh exceeds the grid).
template <int K, typename T>
__global__ void __launch_bounds__(32)
k_rhs_gather(MeshDev m, const T* __restrict__ local, double* __restrict__ b) {
  constexpr int NQ = K + 1;
  const int ex = blockIdx.x * 32 + threadIdx.x;
  const int nex = m.ne[0], ney = m.ne[1], nez = m.ne[2];
  if (ex >= nex) return;
  const int64_t E = m.E, sy = nex, sz = (int64_t)nex * ney;
  const int64_t nx = m.nn[0], nxy = (int64_t)m.nn[0] * m.nn[1];
  const bool lastx = ex == nex - 1, px = ex > 0;
  for (int ez = blockIdx.z; ez < nez; ez += gridDim.z) {
    const bool lastz = ez == nez - 1, pz = ez > 0;
    for (int ey = blockIdx.y; ey < ney; ey += gridDim.y) {
      const bool lasty = ey == ney - 1, py = ey > 0;
      const int64_t e = ex + sy * ey + sz * ez;
      const T* pe = local + e;
      double* be = b + (int64_t)ex * K + nx * ((int64_t)ey * K) + nxy * ((int64_t)ez * K);
#pragma unroll
      for (int c = 0; c < NQ; ++c) {
        if (c == K && !lastz) continue;
#pragma unroll
        for (int bb = 0; bb < NQ; ++bb) {
          if (bb == K && !lasty) continue;
#pragma unroll
          for (int a = 0; a < NQ; ++a) {
            if (a == K && !lastx) continue;
            T s = 0;
#pragma unroll
            for (int q = 7; q >= 0; --q) {  // (dz, dy, dx) = bits of q: elements ascending
              const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
              if ((dx && !(a == 0 && px)) || (dy && !(bb == 0 && py)) || (dz && !(c == 0 && pz)))
                continue;
              const int jj = (a + K * dx) + NQ * ((bb + K * dy) + NQ * (c + K * dz));
              s += __ldg(pe + jj * E - (dx + sy * dy + sz * dz));
            }
            if constexpr (std::is_same<T, float>::value)
              be[a + nx * bb + nxy * c] = double_from_float_int(s);  // exact, no conversion
            else
              be[a + nx * bb + nxy * c] = (double)s;
          }
        }
      }
    }
  }
}

cudaError_t launch_rhs(const MeshDev& m, const Tables& t, const double* eps_q64,
                       const float* eps_q32, double* local, double* b, cudaStream_t s) {
  const dim3 g((unsigned)((m.ne[0] + 31) / 32), (unsigned)std::min(m.ne[1], 65535),
               (unsigned)std::min(m.ne[2], 65535));
#define CFDEM_RHS(KK)                                                                       \
  if (m.k == KK) {                                                                          \
    if (eps_q32) {                                                                          \
      constexpr int nb = rhs_block<KK, float>();                                            \
      float* lf = reinterpret_cast<float*>(local);                                          \
      k_rhs<KK, float><<<(unsigned)((m.E + nb - 1) / nb), nb, 0, s>>>(m, t, eps_q32, lf);   \
      k_rhs_gather<KK, float><<<g, 32, 0, s>>>(m, lf, b);                                   \
    } else {                                                                                \
      constexpr int nb = rhs_block<KK, double>();                                           \
      k_rhs<KK, double><<<(unsigned)((m.E + nb - 1) / nb), nb, 0, s>>>(m, t, eps_q64, local); \
      k_rhs_gather<KK, double><<<g, 32, 0, s>>>(m, local, b);                               \
    }                                                                                       \
    count_launches(2);                                                                      \
    return cudaGetLastError();                                                              \
  }
  CFDEM_RHS(1)
  CFDEM_RHS(2)
  CFDEM_RHS(3)
#undef CFDEM_RHS
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// assembled 1D band tables: for axis a and node i, coefficients t = -k..k of
// the reference (unit element length) mass and stiffness rows

static void band_rows(int ne, int k, const double Mh[4][4], double* out /*[n][2k+1]*/) {
  int n = ne * k + 1, w = 2 * k + 1;
  for (int i = 0; i < n * w; ++i) out[i] = 0.0;
  for (int el = 0; el < ne; ++el)
    for (int a = 0; a <= k; ++a)
      for (int bb = 0; bb <= k; ++bb) {
        int i = el * k + a, j = el * k + bb;
        out[i * w + (j - i + k)] += Mh[a][bb];
      }
}

// layout: for axis a: [M rows n_a x w][K rows n_a x w], axes one after another
cudaError_t upload_bands(const MeshDev& m, const Tables& t, double /*L2*/, double** bands64,
                         float** bands32, float** bands_df) {
  int k = m.k, w = 2 * k + 1;
  size_t tot = 0;
  for (int a = 0; a < 3; ++a) tot += 2 * (size_t)m.nn[a] * w;
  std::vector<double> h(tot);
  size_t off = 0;
  for (int a = 0; a < 3; ++a) {
    band_rows(m.ne[a], k, t.Mh, h.data() + off);
    off += (size_t)m.nn[a] * w;
    band_rows(m.ne[a], k, t.Kh, h.data() + off);
    off += (size_t)m.nn[a] * w;
  }
  std::vector<float> hf(tot);
  for (size_t i = 0; i < tot; ++i) hf[i] = (float)h[i];
  std::vector<float> hdf(2 * tot);  // df64 pairs (hi, lo)
  for (size_t i = 0; i < tot; ++i) {
    hdf[2 * i] = (float)h[i];
    hdf[2 * i + 1] = (float)(h[i] - (double)hdf[2 * i]);
  }
  cudaError_t e;
  if (*bands_df) cudaFree(*bands_df);
  *bands_df = nullptr;
  if ((e = cudaMalloc(bands_df, 2 * tot * sizeof(float))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(*bands_df, hdf.data(), 2 * tot * sizeof(float), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  if (*bands64) cudaFree(*bands64);
  if (*bands32) cudaFree(*bands32);
  *bands64 = nullptr;
  *bands32 = nullptr;
  if ((e = cudaMalloc(bands64, tot * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(bands32, tot * sizeof(float))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(*bands64, h.data(), tot * sizeof(double), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  return cudaMemcpy(*bands32, hf.data(), tot * sizeof(float), cudaMemcpyHostToDevice);
}

// ---------------------------------------------------------------------------
// operator

// Node tiles of the operator: X x Y x Z owned nodes plus a halo of k.  The
// shape is picked per mesh (pick_shape) to waste the fewest nodes on partial
// tiles; e.g. 22 x 13 tiles cover a 65 x 65 node plane with 1.5 % waste
// where 16 x 8 tiles waste 27 %.
template <int X_, int Y_, int Z_>
struct Shape {
  static constexpr int X = X_, Y = Y_, Z = Z_;
};
using Shape0 = Shape<16, 8, 8>;
using Shape1 = Shape<22, 13, 4>;
using Shape2 = Shape<25, 15, 4>;
constexpr int kShapes = 3;
constexpr int kApplyThreads = 256;

template <int K, class S>
struct Tile {
  static constexpr int TX = S::X, TY = S::Y, TZ = S::Z;
  static constexpr int H = K, W = 2 * K + 1;
  static constexpr int XW = TX + 2 * H, YW = TY + 2 * H, ZW = TZ + 2 * H;
  static constexpr int NX = ZW * YW * XW;     // input with halo
  static constexpr int NT = TZ * YW * XW;     // after the z pass (each of t1, t2)
  static constexpr int NU = TZ * TY * XW;     // after the y pass (each of U, V)
  static constexpr int NO = TZ * TY * TX;     // owned nodes (their input, for the epilogue)
  // Two layouts: the z pass writes t1, t2 over the input (each thread
  // overwrites only the column it has read), with U, V apart; or t1, t2
  // apart and U, V over the input once the z pass is done.  The smaller one
  // is used.
  static constexpr bool UV_IN_X = 2 * NU <= NX;
  static constexpr int RA = NX > 2 * NT ? NX : 2 * NT;
  static constexpr int SZ_TX = RA + 2 * NU;
  static constexpr int SZ_UX = NX + 2 * NT + (UV_IN_X ? 0 : 2 * NU);
  static constexpr bool T_IN_X = SZ_TX < SZ_UX;
  static constexpr int SZ = T_IN_X ? SZ_TX : SZ_UX;
  // band coefficients of the tile's rows: z (M, K), y (three folded
  // combinations), x (M, K)
  static constexpr int NBZ = 2 * TZ * W, NBY = 3 * TY * W, NBX = 2 * TX * W;
  // with XE: the owned nodes' input kept for the epilogue
  static constexpr int nsm(bool xe) { return SZ + (xe ? NO : 0) + NBZ + NBY + NBX; }
  // y pass: one thread per (chunk of CY rows, z, x) column piece, the number
  // of chunks chosen for the fewest row outputs per thread over whole rounds
  // of the block's threads
  static constexpr int YCOLS = TZ * XW;
  static constexpr int ycost(int nch) {
    return ((YCOLS * nch + 255) / 256) * ((TY + nch - 1) / nch);
  }
  static constexpr int ypick() {
    int best = 1;
    for (int c = 2; c <= TY; ++c)
      if (ycost(c) < ycost(best)) best = c;
    return best;
  }
  static constexpr int YNCH = ypick();
  static constexpr int CY = (TY + YNCH - 1) / YNCH;
};

template <typename T>
struct Coefs {
  T cM, cKx, cKy, cKz;
};

// Sum of products b_k x_k for the banded passes of the tile operator.  In
// FP32/FP64 a plain FMA chain; in double-float the compensated sum DfDotAcc
// (df64.cuh), 12 FP32 instructions per term.
template <typename T>
struct Acc {
  T v;
  __device__ __forceinline__ void zero() { v = (T)0; }
  __device__ __forceinline__ void add(T b, T x) { v += b * x; }
  __device__ __forceinline__ T get() const { return v; }
};

// Double-float ("df64") numbers: an unevaluated sum hi + lo of two floats
// carrying about 48 significant bits, with error-free two-sum and FMA-based
// two-product (Dekker 1971; Knuth, TAOCP vol. 2).  They give the mixed path
// residuals accurate to ~1e-14 on the FP32 pipes, which on this part have 61
// times the FP64 throughput.
template <>
struct Acc<df64> : DfDotAcc {};

// --- load and epilogue policies of the tile operator -----------------------
// Plain: x_eff = x[g]
template <typename T>
struct LoadPlain {
  const T* x;
  __device__ __forceinline__ T operator()(int64_t g, bool) const { return x[g]; }
};
// CG direction: x_eff = z[g] + beta p_old[g], written to p_new for owned nodes
// (first iteration: p = z)
template <typename T>
struct LoadDir {
  const T* z;
  const T* p_old;
  T* p_new;
  T beta;
  bool first;
  __device__ __forceinline__ T operator()(int64_t g, bool own) const {
    T v = first ? z[g] : z[g] + beta * p_old[g];
    if (own) p_new[g] = v;
    return v;
  }
};
// the same for FP32 directions promoted to df64
struct LoadDirF32 {
  const float* z;
  const float* p_old;
  float* p_new;
  float beta;
  bool first;
  __device__ __forceinline__ df64 operator()(int64_t g, bool own) const {
    float v = first ? z[g] : fmaf(beta, p_old[g], z[g]);
    if (own) p_new[g] = v;
    return df64(v);
  }
};
// CG direction in double-float from the FP32 preconditioned residual:
// p = z + beta p_old (first iteration: p = z)
struct LoadDirDf {
  const float* z;
  const df64* p_old;
  df64* p_new;
  df64 beta;
  bool first;
  __device__ __forceinline__ df64 operator()(int64_t g, bool own) const {
    df64 v = first ? df64(z[g]) : df64(z[g]) + beta * p_old[g];
    if (own) p_new[g] = v;
    return v;
  }
};

// y[g] = acc; dot += x_eff * acc (FP64 accumulation)
template <typename T>
struct EpiStore {
  using acc_t = T;
  static constexpr bool kXE = true;
  T* y;
  __device__ __forceinline__ T operator()(int64_t g, T acc, T xe) const {
    y[g] = acc;
    return xe * acc;
  }
};
// df64 image of an FP32 direction: store, dot with the high part
struct EpiStoreDf {
  using acc_t = float;
  static constexpr bool kXE = false;
  df64* y;
  const df64* p;  // the direction, written by this block's load phase
  __device__ __forceinline__ float operator()(int64_t g, df64 acc, df64) const {
    y[g] = acc;
    return __ldcg(reinterpret_cast<const float*>(p + g)) * acc.hi;
  }
};
// residual r = b - A x in df64; r32 = high part (input of the FP32
// preconditioner); returns r.r from the high parts
struct EpiResidualDf {
  using acc_t = float;
  static constexpr bool kXE = false;
  const double* b;  // FP64 right-hand side, split here (bit-field moves)
  df64* r;
  float* r32;
  __device__ __forceinline__ float operator()(int64_t g, df64 acc, df64) const {
    df64 v = df_from_double_int(b[g]) - acc;
    r[g] = v;
    r32[g] = v.hi;
    return v.hi * v.hi;
  }
};

// y = A x on one tile (sum factorisation over the Kronecker sum, see top of
// file).  ld(g, own) gives the input value at node g; ep(g, acc, x_eff)
// consumes the result of an owned node and returns its share of a dot
// product.
//
// The band rows of the tile are staged in shared memory first, the y ones
// folded with the coefficients:
//   U = (cM My + cKy Ky) T1 + (cKz My) T2,  V = (cKx My) T1,  A x = Mx U + Kx V
// with T1 = Mz x, T2 = Kz x.  The z pass runs one thread per haloed (x, y)
// column over all TZ outputs, the y pass one thread per run of CY outputs
// along y (inputs held in registers), the x pass one thread per owned node.
template <int K, class S, typename T, class Load, class Epi>
__device__ __forceinline__ typename Epi::acc_t apply_tile(const MeshDev& m,
                                                          const T* __restrict__ bands,
                                             const Coefs<T>& cf, const Load& ld, const Epi& ep,
                                             T* sm) {
  using TL = Tile<K, S>;
  constexpr int TX = TL::TX, TY = TL::TY, TZ = TL::TZ;
  constexpr int H = TL::H, W = TL::W;
  constexpr int XW = TL::XW, YW = TL::YW, ZW = TL::ZW;
  constexpr int PL = YW * XW;  // one z plane of the haloed input
  const int nx = m.nn[0], ny = m.nn[1], nz = m.nn[2];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int64_t sxy = (int64_t)nx * ny;
  constexpr bool kXE = Epi::kXE;
  T* X = sm;                                         // [ZW][YW][XW]
  T* T1 = TL::T_IN_X ? sm : sm + TL::NX;             // [TZ][YW][XW]
  T* T2 = T1 + TL::NT;
  T* U = TL::T_IN_X ? sm + TL::RA : (TL::UV_IN_X ? X : T2 + TL::NT);  // [TZ][TY][XW]
  T* V = U + TL::NU;
  T* XE = sm + TL::SZ;       // [TZ][TY][TX] input at the owned nodes (kXE)
  T* BZ = XE + (kXE ? TL::NO : 0);  // [TZ][W][2]   Mz, Kz of row z0 + o
  T* BY = BZ + TL::NBZ;      // [TY][W][3]   cM My + cKy Ky, cKz My, cKx My of row y0 + j
  T* BX = BY + TL::NBY;      // [2][W][TX]   Mx, Kx of column x0 + i
  const T* bMx = bands;
  const T* bKx = bMx + (size_t)nx * W;
  const T* bMy = bKx + (size_t)nx * W;
  const T* bKy = bMy + (size_t)ny * W;
  const T* bMz = bKy + (size_t)ny * W;
  const T* bKz = bMz + (size_t)nz * W;

  // band rows of the tile (zero past the mesh)
  for (int t = threadIdx.x; t < TZ * W; t += blockDim.x) {
    const int o = t / W, w = t - o * W, gz = z0 + o;
    T a = T(0), b = T(0);
    if (gz < nz) {
      a = bMz[(size_t)gz * W + w];
      b = bKz[(size_t)gz * W + w];
    }
    BZ[2 * t] = a;
    BZ[2 * t + 1] = b;
  }
  for (int t = threadIdx.x; t < TY * W; t += blockDim.x) {
    const int j = t / W, w = t - j * W, gy = y0 + j;
    T a = T(0), b = T(0), c = T(0);
    if (gy < ny) {
      const T my = bMy[(size_t)gy * W + w], ky = bKy[(size_t)gy * W + w];
      a = cf.cM * my + cf.cKy * ky;
      b = cf.cKz * my;
      c = cf.cKx * my;
    }
    BY[3 * t] = a;
    BY[3 * t + 1] = b;
    BY[3 * t + 2] = c;
  }
  for (int t = threadIdx.x; t < TX * W; t += blockDim.x) {
    const int i = t / W, w = t - i * W, gx = x0 + i;
    T a = T(0), b = T(0);
    if (gx < nx) {
      a = bMx[(size_t)gx * W + w];
      b = bKx[(size_t)gx * W + w];
    }
    BX[w * TX + i] = a;
    BX[(W + w) * TX + i] = b;
  }

  // load with halo: each thread keeps one x column of the haloed tile (its
  // x bounds and ownership worked out once) and walks the (z, y) rows; the
  // owned nodes' input also to XE
  int nonzero = 0;
  {
    constexpr int RT = kApplyThreads / XW;  // rows taken per pass
    const int lx = (int)threadIdx.x % XW, tr = (int)threadIdx.x / XW;
    if (tr < RT) {
      const int gx = x0 + lx - H;
      const bool xin = gx >= 0 && gx < nx, xown = lx >= H && lx < H + TX;
      for (int row = tr; row < ZW * YW; row += RT) {
        const int lz = row / YW, ly = row - lz * YW;
        const int gy = y0 + ly - H, gz = z0 + lz - H;
        T v = T(0);
        if (xin && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
          const bool own = xown && ly >= H && ly < H + TY && lz >= H && lz < H + TZ;
          v = ld(gx + (int64_t)nx * gy + sxy * gz, own);
          if (kXE && own) XE[((lz - H) * TY + (ly - H)) * TX + (lx - H)] = v;
        }
        X[row * XW + lx] = v;
        nonzero |= (v != T(0));
      }
    }
  }
  // a tile whose input (halo included) is zero has a zero image: skip the
  // passes (a cold start of the projection begins with x = 0)
  if (!__syncthreads_or(nonzero)) {
    typename Epi::acc_t dot = 0;
    for (int t = threadIdx.x; t < TX * TY * TZ; t += blockDim.x) {
      int gx = x0 + t % TX, gy = y0 + (t / TX) % TY, gz = z0 + t / (TX * TY);
      if (gx < nx && gy < ny && gz < nz) dot += ep(gx + (int64_t)nx * gy + sxy * gz, T(0), T(0));
    }
    return dot;
  }
  // z pass: column c of the haloed x-y plane, all TZ outputs (with T_IN_X
  // written over the column's input, which this thread has read first)
  for (int c = threadIdx.x; c < PL; c += blockDim.x) {
    T xv[ZW];
#pragma unroll
    for (int q = 0; q < ZW; ++q) xv[q] = X[q * PL + c];
#pragma unroll
    for (int o = 0; o < TZ; ++o) {
      Acc<T> a1, a2;
      a1.zero();
      a2.zero();
#pragma unroll
      for (int w = 0; w < W; ++w) {
        a1.add(BZ[2 * (o * W + w)], xv[o + w]);
        a2.add(BZ[2 * (o * W + w) + 1], xv[o + w]);
      }
      T1[o * PL + c] = a1.get();
      T2[o * PL + c] = a2.get();
    }
  }
  __syncthreads();
  // y pass: rows j0 .. j0 + len - 1 of column (lz, lx)
  constexpr int CY = TL::CY, WIN = CY + 2 * H;
  for (int it = threadIdx.x; it < TL::YCOLS * TL::YNCH; it += blockDim.x) {
    const int ch = it / TL::YCOLS, col = it - ch * TL::YCOLS;
    const int lz = col / XW, lx = col - lz * XW;
    const int j0 = ch * CY;
    const int len = TY - j0 < CY ? TY - j0 : CY;
    const T* s1 = T1 + lz * PL + j0 * XW + lx;
    const T* s2 = T2 + lz * PL + j0 * XW + lx;
    T t1[WIN], t2[WIN];
#pragma unroll
    for (int q = 0; q < WIN; ++q) {
      const bool in = q < len + 2 * H;
      t1[q] = in ? s1[q * XW] : T(0);
      t2[q] = in ? s2[q * XW] : T(0);
    }
    T* du = U + (lz * TY + j0) * XW + lx;
    T* dv = V + (lz * TY + j0) * XW + lx;
#pragma unroll
    for (int j = 0; j < CY; ++j) {
      if (j < len) {
        const T* by = BY + (j0 + j) * (3 * W);
        Acc<T> au, av;
        au.zero();
        av.zero();
#pragma unroll
        for (int w = 0; w < W; ++w) {
          au.add(by[3 * w], t1[j + w]);
          au.add(by[3 * w + 1], t2[j + w]);
          av.add(by[3 * w + 2], t1[j + w]);
        }
        du[j * XW] = au.get();
        dv[j * XW] = av.get();
      }
    }
  }
  __syncthreads();
  // x pass + output (per-thread partial in the epilogue's type, one
  // conversion per thread)
  // (each thread keeps one x column of the owned nodes and walks the rows)
  typename Epi::acc_t dot = 0;
  {
    constexpr int RT = kApplyThreads / TX;
    const int lx = (int)threadIdx.x % TX, tr = (int)threadIdx.x / TX;
    const int gx = x0 + lx;
    if (tr < RT && gx < nx) {
      for (int row = tr; row < TZ * TY; row += RT) {
        const int lz = row / TY, ly = row - lz * TY;
        const int gy = y0 + ly, gz = z0 + lz;
        if (gy >= ny || gz >= nz) continue;
        const T* u = U + row * XW + lx;
        const T* v = V + row * XW + lx;
        Acc<T> ax;
        ax.zero();
#pragma unroll
        for (int w = 0; w < W; ++w) {
          ax.add(BX[w * TX + lx], u[w]);
          ax.add(BX[(W + w) * TX + lx], v[w]);
        }
        dot += ep(gx + (int64_t)nx * gy + sxy * gz, ax.get(),
                  kXE ? XE[row * TX + lx] : T(0));
      }
    }
  }
  return dot;
}

template <int K, class S, typename T>
__global__ void __launch_bounds__(kApplyThreads)
k_apply(MeshDev m, const T* __restrict__ bands, Coefs<T> cf, const T* __restrict__ x,
        T* __restrict__ y, const int* __restrict__ xnz) {
  // a zero start vector (flag cleared by k_flag_nonzero): A x = 0, the
  // consumer reads the flag instead of y
  if (xnz && !*(volatile const int*)xnz) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  LoadPlain<T> ld{x};
  EpiStore<T> ep{y};
  apply_tile<K, S, T>(m, bands, cf, ld, ep, reinterpret_cast<T*>(smraw));
}

// CG step 1: p = z + beta p_old (fused into the load) ; Ap = A p ; alpha =
// rz / (p . Ap)
template <int K, class S, typename T>
__global__ void __launch_bounds__(kApplyThreads)
k_cg_apply(MeshDev m, const T* __restrict__ bands, Coefs<T> cf, const T* __restrict__ z,
           const T* __restrict__ p_old, T* __restrict__ p_new, T* __restrict__ Ap,
           double* partials, CgScalars* sc, int first) {
  if (((volatile CgScalars*)sc)->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  T beta = first ? (T)0 : (T)sc->beta;
  LoadDir<T> ld{z, p_old, p_new, beta, first != 0};
  EpiStore<T> ep{Ap};
  const T d = apply_tile<K, S, T>(m, bands, cf, ld, ep, reinterpret_cast<T*>(smraw));
  double s = block_sum(d, red);
  double vals[1] = {s};
  double out[1];
  if (last_block_reduce(partials, 1, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->pAp = out[0];
    sc->alpha = sc->rz / out[0];
  }
}

// CG step 2: x += alpha p ; r -= alpha Ap ; z = D^-1 r ; beta ; convergence
template <typename T, typename TX_>
__global__ void __launch_bounds__(256)
k_cg_update(int64_t n, TX_* __restrict__ xv, T* __restrict__ r, T* __restrict__ z,
            const T* __restrict__ p, const T* __restrict__ Ap, const T* __restrict__ dinv,
            double* partials, CgScalars* sc, int maxit) {
  if (((volatile CgScalars*)sc)->done) return;
  __shared__ double red[32];
  T alpha = (T)sc->alpha;
  T rz = 0, rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    xv[i] += (TX_)(alpha * p[i]);
    T ri = r[i] - alpha * Ap[i];
    T zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  double s1 = block_sum(rz, red);
  double s2 = block_sum(rr, red);
  double vals[2] = {s1, s2};
  double out[2];
  if (last_block_reduce(partials, 2, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->beta = out[0] / sc->rz;
    sc->rz = out[0];
    sc->rr = out[1];
    sc->it += 1;
    if (out[1] <= sc->tol2 || sc->it >= maxit) sc->done = 1;
  }
}

// start: r = b - Ax ; z = D^-1 r ; rz, rr, bb
template <typename T, typename TB>
__global__ void __launch_bounds__(256)
k_cg_start(int64_t n, const TB* __restrict__ b, const T* __restrict__ Ax, T* __restrict__ r,
           T* __restrict__ z, const T* __restrict__ dinv, double* partials, CgScalars* sc,
           double rtol) {
  __shared__ double red[32];
  T rz = 0, rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T bi = (T)b[i];
    T ri = bi - Ax[i];
    T zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
    bb += bi * bi;
  }
  double s1 = block_sum(rz, red);
  double s2 = block_sum(rr, red);
  double s3 = block_sum(bb, red);
  double vals[3] = {s1, s2, s3};
  double out[3];
  if (last_block_reduce(partials, 3, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->rz = out[0];
    sc->rr = out[1];
    sc->bb = out[2];
    double bbv = out[2] > 0.0 ? out[2] : 1.0;
    sc->tol2 = rtol * rtol * bbv;
    sc->it = 0;
    sc->done = out[1] <= sc->tol2 ? 1 : 0;
    sc->beta = 0.0;
  }
}

// --- preconditioned by the fast diagonalisation (FDM) ---------------------
// update without preconditioning: x += alpha p ; r -= alpha Ap ; rf = (float) r
// for the FDM ; r . r and the convergence flag
template <typename T, typename TX_>
__global__ void __launch_bounds__(256)
k_cg_update_fdm(int64_t n, TX_* __restrict__ xv, T* __restrict__ r, const T* __restrict__ p,
                const T* __restrict__ Ap, float* __restrict__ rf, double* partials,
                CgScalars* sc, int maxit) {
  if (((volatile CgScalars*)sc)->done) return;
  __shared__ double red[32];
  T alpha = (T)sc->alpha;
  T rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    xv[i] += (TX_)(alpha * p[i]);
    T ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    if (rf) rf[i] = (float)ri;
    rr += ri * ri;
  }
  double s = block_sum(rr, red);
  double vals[1] = {s};
  double out[1];
  if (last_block_reduce(partials, 1, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->rr = out[0];
    sc->it += 1;
    if (out[0] <= sc->tol2 || sc->it >= maxit) sc->done = 1;
  }
}

// after z_new = P^-1 r: z_new (from the FP32 FDM output zf) ; rz_new = r . z_new ;
// Polak-Ribiere beta = (rz_new - r . z_old) / rz_old (robust to the rounding
// of the FP32 preconditioner) ; first: plain rz.  With fletcher_reeves the
// plain beta = rz_new / rz_old is used: when the dots are formed from FP32
// products, r . z_old (zero in exact arithmetic, large terms) carries an
// error of order 1e-7 |r||z_old|, which is comparable to rz_new itself once
// the residual has dropped by 1e-6 and would spoil the Polak-Ribiere beta
template <typename T>
__global__ void __launch_bounds__(256)
k_cg_dot_fdm(int64_t n, const T* __restrict__ r, const float* __restrict__ zf,
             const T* __restrict__ z_old, T* __restrict__ z_new, double* partials,
             CgScalars* sc, int first, int ignore_done, int fletcher_reeves = 0) {
  if (!ignore_done && ((volatile CgScalars*)sc)->done) return;
  __shared__ double red[32];
  // per-thread sums in T (a few terms each), one conversion per thread: FP64
  // arithmetic per element would run on the slow FP64 pipe
  T rz = 0, rzo = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T zi = zf ? (T)zf[i] : z_new[i];
    if (zf) z_new[i] = zi;
    T ri = r[i];
    rz += ri * zi;
    if (!first && !fletcher_reeves) rzo += ri * z_old[i];
  }
  double s1 = block_sum(rz, red);
  double s2 = block_sum(rzo, red);
  double vals[2] = {s1, s2};
  double out[2];
  if (last_block_reduce(partials, 2, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    if (!first) sc->beta = (out[0] - out[1]) / sc->rz;
    sc->rz = out[0];
  }
}

// *flag = 1 if x has an entry other than zero (flag cleared beforehand)
template <typename T>
__global__ void __launch_bounds__(256)
k_flag_nonzero(int64_t n, const T* __restrict__ x, int* flag) {
  int nz = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    nz |= x[i] != (T)0;
  if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

// start: r = b - Ax ; rf = (float) r ; rr, bb, tolerance
template <typename T, typename TB>
__global__ void __launch_bounds__(256)
k_cg_start_fdm(int64_t n, const TB* __restrict__ b, const T* __restrict__ Ax,
               T* __restrict__ r, float* __restrict__ rf, double* partials, CgScalars* sc,
               double rtol, int use_flag) {
  __shared__ double red[32];
  T rr = 0, bb = 0;
  // with use_flag, A x was skipped for a zero start vector (sc->xnz == 0)
  const bool ax = !use_flag || ((volatile CgScalars*)sc)->xnz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T bi = (T)b[i];
    T ri = ax ? bi - Ax[i] : bi;
    r[i] = ri;
    if (rf) rf[i] = (float)ri;
    rr += ri * ri;
    bb += bi * bi;
  }
  double s1 = block_sum(rr, red);
  double s2 = block_sum(bb, red);
  double vals[2] = {s1, s2};
  double out[2];
  if (last_block_reduce(partials, 2, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->rr = out[0];
    sc->bb = out[1];
    double bbv = out[1] > 0.0 ? out[1] : 1.0;
    sc->tol2 = rtol * rtol * bbv;
    sc->it = 0;
    sc->done = out[0] <= sc->tol2 ? 1 : 0;
    sc->beta = 0.0;
  }
}

// --- mixed path: outer CG in double-float, FP32 directions and FDM --------
// x (FP64) -> df64 copy, r = b as df64 and r32 = hi(b) (the residual of a
// zero start vector, which k_residual_df leaves in place and overwrites when
// x != 0, splitting b itself), all converted with integer operations; b . b
// from the high parts into sc->bb
__global__ void __launch_bounds__(256)
k_split_df(int64_t n, const double* __restrict__ b,
           const double* __restrict__ x, df64* __restrict__ x_df, df64* __restrict__ r,
           float* __restrict__ r32, double* partials, CgScalars* sc) {
  __shared__ double red[32];
  float bb = 0.f;
  int nz = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const df64 v = df_from_double_int(b[i]);
    r[i] = v;
    r32[i] = v.hi;
    bb = fmaf(v.hi, v.hi, bb);
    const double xi = x[i];
    x_df[i] = df_from_double_int(xi);
    unsigned xl, xh;
    double_halves(xi, &xl, &xh);
    nz |= (xl | (xh << 1)) != 0u;  // x != 0 by integer operations
  }
  if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&sc->xnz, 1);
  double s = block_sum(bb, red);
  double vals[1] = {s};
  double o[1];
  if (last_block_reduce(partials, 1, vals, &sc->ticket, o, red) && threadIdx.x == 0) sc->bb = o[0];
}

__global__ void k_join_df(int64_t n, const df64* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = double_from_df_int(in[i]);
  }
}

// r = b - A x (df64), r32 = hi(r), r . r ; tolerance and convergence flag.
// For a zero start vector (flag from k_split_df) r = b, r32 and r . r = b . b
// are already in place: one thread sets the scalars
template <int K, class S>
__global__ void __launch_bounds__(kApplyThreads)
k_residual_df(MeshDev m, const df64* __restrict__ bands, Coefs<df64> cf,
              const df64* __restrict__ x, const double* __restrict__ b, df64* __restrict__ r,
              float* __restrict__ r32, double* partials, CgScalars* sc, double rtol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  const bool xnz = ((volatile CgScalars*)sc)->xnz;
  double rr;
  if (xnz) {
    LoadPlain<df64> ld{x};
    EpiResidualDf ep{b, r, r32};
    const float d = apply_tile<K, S, df64>(m, bands, cf, ld, ep, reinterpret_cast<df64*>(smraw));
    const double s = block_sum(d, red);
    double vals[1] = {s};
    double out[1];
    if (!last_block_reduce(partials, 1, vals, &sc->ticket, out, red) || threadIdx.x != 0) return;
    rr = out[0];
  } else {
    if (blockIdx.x != 0 || blockIdx.y != 0 || blockIdx.z != 0 || threadIdx.x != 0) return;
    rr = sc->bb;
  }
  sc->rr = rr;
  const double bbv = sc->bb > 0.0 ? sc->bb : 1.0;
  sc->tol2 = rtol * rtol * bbv;
  sc->it = 0;
  sc->done = rr <= sc->tol2 ? 1 : 0;
  sc->beta = 0.0;
}

// p = z + beta p_old (df64) ; Ap = A p in df64 ; alpha = rz / (p . Ap)
template <int K, class S>
__global__ void __launch_bounds__(kApplyThreads)
k_cg_apply_df(MeshDev m, const df64* __restrict__ bands, Coefs<df64> cf,
              const float* __restrict__ z, const df64* __restrict__ p_old,
              df64* __restrict__ p_new, df64* __restrict__ Ap, double* partials, CgScalars* sc,
              int first) {
  if (((volatile CgScalars*)sc)->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  LoadDirDf ld{z, p_old, p_new, first ? df64(0.f) : df_from_double(sc->beta), first != 0};
  EpiStoreDf ep{Ap, p_new};
  const float d = apply_tile<K, S, df64>(m, bands, cf, ld, ep, reinterpret_cast<df64*>(smraw));
  double s = block_sum(d, red);
  double vals[1] = {s};
  double out[1];
  if (last_block_reduce(partials, 1, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->pAp = out[0];
    sc->alpha = sc->rz / out[0];
    sc->alpha_hi = (float)sc->alpha;
    sc->alpha_lo = (float)(sc->alpha - (double)sc->alpha_hi);
  }
}

// x += alpha p ; r -= alpha Ap (df64) ; r32 = hi(r) ; r . r ; convergence
__global__ void __launch_bounds__(256)
k_cg_update_df(int64_t n, df64* __restrict__ x, df64* __restrict__ r, const df64* __restrict__ p,
               const df64* __restrict__ Ap, float* __restrict__ r32, double* partials,
               CgScalars* sc, int maxit) {
  if (((volatile CgScalars*)sc)->done) return;
  __shared__ double red[32];
  const df64 alpha(sc->alpha_hi, sc->alpha_lo);
  float rr = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = x[i] + alpha * p[i];
    df64 v = r[i] - alpha * Ap[i];
    r[i] = v;
    r32[i] = v.hi;
    rr = fmaf(v.hi, v.hi, rr);
  }
  double s = block_sum(rr, red);
  double vals[1] = {s};
  double out[1];
  if (last_block_reduce(partials, 1, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->rr = out[0];
    sc->it += 1;
    if (out[0] <= sc->tol2 || sc->it >= maxit) sc->done = 1;
  }
}

// inverse diagonal of A: cM Mx_ii My_jj Mz_kk + cKx Kx_ii My_jj Mz_kk + ...
template <int K, typename T>
__global__ void k_dinv(MeshDev m, const double* __restrict__ bands, double cM, double cKx,
                       double cKy, double cKz, T* __restrict__ dinv) {
  constexpr int W = 2 * K + 1;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m.n_nodes) return;
  int nx = m.nn[0], ny = m.nn[1], nz = m.nn[2];
  int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((int64_t)nx * ny));
  const double* bMx = bands;
  const double* bKx = bMx + (size_t)nx * W;
  const double* bMy = bKx + (size_t)nx * W;
  const double* bKy = bMy + (size_t)ny * W;
  const double* bMz = bKy + (size_t)ny * W;
  const double* bKz = bMz + (size_t)nz * W;
  double mx = bMx[(size_t)ix * W + K], kx = bKx[(size_t)ix * W + K];
  double my = bMy[(size_t)iy * W + K], ky = bKy[(size_t)iy * W + K];
  double mz = bMz[(size_t)iz * W + K], kz = bKz[(size_t)iz * W + K];
  double d = cM * mx * my * mz + cKx * kx * my * mz + cKy * mx * ky * mz + cKz * mx * my * kz;
  dinv[i] = (T)(1.0 / d);
}

template <typename T>
__global__ void k_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ Ax,
                           double* __restrict__ r, double* partials, CgScalars* sc) {
  __shared__ double red[32];
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ri = b[i] - Ax[i];
    r[i] = ri;
    rr += ri * ri;
    bb += b[i] * b[i];
  }
  double s1 = block_sum(rr, red);
  double s2 = block_sum(bb, red);
  double vals[2] = {s1, s2};
  double out[2];
  if (last_block_reduce(partials, 2, vals, &sc->ticket, out, red) && threadIdx.x == 0) {
    sc->rr = out[0];
    sc->bb = out[1];
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, double scale,
                         float* __restrict__ o, float* __restrict__ zero) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    o[i] = (float)(a[i] * scale);
    zero[i] = 0.0f;
  }
}

__global__ void k_add_scaled(int64_t n, double* __restrict__ x, const float* __restrict__ d,
                             double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i] * scale;
}

// ---------------------------------------------------------------------------
// host side

// the double-float kernels' epilogues keep no copy of the input (kXE false)
template <int K, class S, typename T>
static size_t apply_smem() {
  using TL = Tile<K, S>;
  return (size_t)TL::nsm(!std::is_same<T, df64>::value) * sizeof(T);
}

template <class S>
static dim3 apply_grid_s(const MeshDev& m) {
  return dim3((m.nn[0] + S::X - 1) / S::X, (m.nn[1] + S::Y - 1) / S::Y,
              (m.nn[2] + S::Z - 1) / S::Z);
}

// call f(Shape) with the mesh's tile shape
template <class F>
static auto with_shape(const MeshDev& m, F&& f) {
  if (m.shape == 1) return f(Shape1{});
  if (m.shape == 2) return f(Shape2{});
  return f(Shape0{});
}

// call f(integral_constant<int, k>)
template <class F>
static auto with_k(const MeshDev& m, F&& f) {
  if (m.k == 1) return f(std::integral_constant<int, 1>{});
  if (m.k == 2) return f(std::integral_constant<int, 2>{});
  return f(std::integral_constant<int, 3>{});
}

// work of one tile in 1D taps: z pass on the haloed x-y columns, y pass on
// the x-haloed rows, x pass on the owned nodes
template <int K, class S>
static double tile_cost(const MeshDev& m) {
  using TL = Tile<K, S>;
  dim3 g = apply_grid_s<S>(m);
  double per = 2.0 * TL::TZ * TL::YW * TL::XW + 3.0 * TL::TZ * TL::TY * TL::XW +
               2.0 * TL::TZ * TL::TY * TL::TX;
  return per * g.x * g.y * g.z;
}

int pick_shape(const MeshDev& m) {
  return with_k(m, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    double c[kShapes] = {tile_cost<K, Shape0>(m), tile_cost<K, Shape1>(m), tile_cost<K, Shape2>(m)};
    size_t sm[kShapes] = {apply_smem<K, Shape0, double>(), apply_smem<K, Shape1, double>(),
                          apply_smem<K, Shape2, double>()};
    int best = 0;
    for (int i = 1; i < kShapes; ++i)
      if (sm[i] <= 200 * 1024 && c[i] < 0.97 * c[best]) best = i;
    return best;
  });
}

bool shape_fits(const MeshDev& m, int shape) {
  return with_k(m, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    const size_t sm[kShapes] = {apply_smem<K, Shape0, double>(), apply_smem<K, Shape1, double>(),
                                apply_smem<K, Shape2, double>()};
    return shape >= 0 && shape < kShapes && sm[shape] <= 200 * 1024;
  });
}

int cg_blocks(const MeshDev& m) {
  int na = 0;
  dim3 g0 = apply_grid_s<Shape0>(m), g1 = apply_grid_s<Shape1>(m), g2 = apply_grid_s<Shape2>(m);
  na = (int)(g0.x * g0.y * g0.z);
  na = na > (int)(g1.x * g1.y * g1.z) ? na : (int)(g1.x * g1.y * g1.z);
  na = na > (int)(g2.x * g2.y * g2.z) ? na : (int)(g2.x * g2.y * g2.z);
  return na > 1216 ? na : 1216;
}

template <typename T>
static Coefs<T> make_coefs(const double* c) {
  Coefs<T> cf;
  cf.cM = (T)c[0];
  cf.cKx = (T)c[1];
  cf.cKy = (T)c[2];
  cf.cKz = (T)c[3];
  return cf;
}

template <int K, class S, typename T>
static cudaError_t set_smem() {
  static bool done = false;
  if (done) return cudaSuccess;
  size_t sm = apply_smem<K, S, T>();
  cudaError_t e = cudaFuncSetAttribute(k_apply<K, S, T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cg_apply<K, S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
  if (e == cudaSuccess) done = true;
  return e;
}

template <typename T>
static cudaError_t apply_t(const MeshDev& m, const T* bands, const double* coef, const T* x,
                           T* y, cudaStream_t s, const int* xnz = nullptr) {
  Coefs<T> cf = make_coefs<T>(coef);
  return with_k(m, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    return with_shape(m, [&](auto sh) {
      using S = decltype(sh);
      cudaError_t e = set_smem<K, S, T>();
      if (e != cudaSuccess) return e;
      k_apply<K, S, T><<<apply_grid_s<S>(m), kApplyThreads, apply_smem<K, S, T>(), s>>>(
          m, bands, cf, x, y, xnz);
      count_launches(1);
      return cudaGetLastError();
    });
  });
}

template <typename T>
static cudaError_t cg_apply_t(const MeshDev& m, const T* bands, const double* coef, const T* z,
                              const T* p_old, T* p_new, T* Ap, double* partials, CgScalars* sc,
                              int first, cudaStream_t s) {
  Coefs<T> cf = make_coefs<T>(coef);
  return with_k(m, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    return with_shape(m, [&](auto sh) {
      using S = decltype(sh);
      cudaError_t e = set_smem<K, S, T>();
      if (e != cudaSuccess) return e;
      k_cg_apply<K, S, T><<<apply_grid_s<S>(m), kApplyThreads, apply_smem<K, S, T>(), s>>>(
          m, bands, cf, z, p_old, p_new, Ap, partials, sc, first);
      count_launches(1);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_apply64(const MeshDev& m, const double* bands, const double* coef,
                           const double* x, double* y, cudaStream_t s) {
  return apply_t<double>(m, bands, coef, x, y, s);
}

template <typename T>
static cudaError_t make_dinv(const MeshDev& m, const double* bands64, const double* coef,
                             T* dinv, cudaStream_t s) {
  unsigned g = (unsigned)((m.n_nodes + 255) / 256);
#define CFDEM_DINV(KK)                                                                      \
  if (m.k == KK) {                                                                          \
    k_dinv<KK, T><<<g, 256, 0, s>>>(m, bands64, coef[0], coef[1], coef[2], coef[3], dinv);  \
    count_launches(1);                                                                      \
    return cudaGetLastError();                                                              \
  }
  CFDEM_DINV(1)
  CFDEM_DINV(2)
  CFDEM_DINV(3)
#undef CFDEM_DINV
  return cudaErrorInvalidValue;
}

static int vec_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

// ---------------------------------------------------------------------------
// Device-driven iteration inside a stream capture.  When the stream is being
// captured into a CUDA graph, the CG loops below do not read the device flag
// `done` on the host between chunks; instead they add a conditional WHILE
// node to the graph under construction.  Its body -- captured on a second
// stream `ls` -- holds two CG iterations and ends with k_loop_cond, which sets
// the node's condition from `done`, so the graph iterates on the device until
// the CG has converged or reached its iteration cap.  (Two iterations, so that
// the ping-pong buffers are back in their roles at the end of the body.)  The
// first two iterations are queued before the node, and a k_loop_cond ahead
// of the node decides whether the body runs at all: a solve that converges
// in two iterations -- the mixed cold start -- launches no idle iteration.

// one thread: continue while the CG is not done, and never beyond
// max_bodies - 1 bodies whatever the kernels of the body did (sc->loops is
// cleared with the other scalars at the start of every solve)
__global__ void k_loop_cond(cudaGraphConditionalHandle h, CgScalars* sc, int max_bodies) {
  volatile CgScalars* v = sc;
  int n = v->loops + 1;
  v->loops = n;
  cudaGraphSetConditional(h, (!v->done && n < max_bodies) ? 1u : 0u);
}

// bodies allowed for maxit iterations: two queued ahead, two per body
static int loop_max_bodies(int maxit) { return maxit / 2 + 2; }

static cudaError_t loop_open(cudaStream_t s, cudaStream_t ls, cudaGraphConditionalHandle* h,
                             CgScalars* sc, int maxit) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnmatched;
  if ((e = cudaGraphConditionalHandleCreate(h, g, 0, 0)) != cudaSuccess) return e;
  // the condition for the first body, set upstream of the node
  k_loop_cond<<<1, 1, 0, s>>>(*h, sc, loop_max_bodies(maxit));
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess)
    return e;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return e;
  return cudaStreamBeginCaptureToGraph(ls, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
}

static cudaError_t loop_close(cudaStream_t ls, cudaGraphConditionalHandle h, CgScalars* sc,
                              int maxit, cudaError_t body_status) {
  if (body_status == cudaSuccess) {
    k_loop_cond<<<1, 1, 0, ls>>>(h, sc, loop_max_bodies(maxit));
    count_launches(1);
    body_status = cudaGetLastError();
  }
  cudaGraph_t body = nullptr;
  cudaError_t e = cudaStreamEndCapture(ls, &body);
  return body_status != cudaSuccess ? body_status : e;
}

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!s || cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs == cudaStreamCaptureStatusActive;
}

// one CG solve of A x = b in precision T from the start vector x (in T, or
// FP64 for the outer vector when TX_ = double); iterations run in chunks
// between host checks of the device flag
template <typename T, typename TX_, typename TB>
static cudaError_t cg_solve(const MeshDev& m, const T* bands, const double* coef, const TB* b,
                            TX_* x, const T* x_as_T, double rtol, int maxit, T* r, T* z,
                            T* p0, T* p1, T* Ap, const T* dinv, double* partials,
                            CgScalars* sc, cudaStream_t s, int* iters, double* relres,
                            Timer* tm, cudaStream_t ls) {
  cudaError_t e;
  int64_t n = m.n_nodes;
  int vb = vec_blocks(n);
  const int op_stage = sizeof(T) == 8 ? kStageOp64 : kStageOp32;
  // Ax for the start vector
  if (tm) tm->begin(op_stage, s);
  if ((e = apply_t<T>(m, bands, coef, x_as_T, Ap, s)) != cudaSuccess) return e;
  if (tm) tm->end(op_stage, s);
  k_cg_start<T, TB><<<vb, 256, 0, s>>>(n, b, Ap, r, z, dinv, partials, sc, rtol);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  T* pc = p0;
  T* pn = p1;
  auto iter = [&](int first, cudaStream_t st) -> cudaError_t {
    cudaError_t ee;
    if (tm) tm->begin(op_stage, st);
    if ((ee = cg_apply_t<T>(m, bands, coef, z, pc, pn, Ap, partials, sc, first, st)) !=
        cudaSuccess)
      return ee;
    if (tm) tm->end(op_stage, st);
    k_cg_update<T, TX_><<<vb, 256, 0, st>>>(n, x, r, z, pn, Ap, dinv, partials, sc, maxit);
    count_launches(1);
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    T* t = pc;
    pc = pn;
    pn = t;
    return cudaSuccess;
  };
  if (ls) {  // device-driven loop inside a stream capture
    if ((e = iter(1, s)) != cudaSuccess) return e;
    if ((e = iter(0, s)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = loop_open(s, ls, &h, sc, maxit)) != cudaSuccess) return e;
    e = iter(0, ls);
    if (e == cudaSuccess) e = iter(0, ls);
    if ((e = loop_close(ls, h, sc, maxit, e)) != cudaSuccess) return e;
    *iters = -1;
    *relres = -1.0;
    return cudaSuccess;
  }
  int launched = 0;
  CgScalars hs;
  const int chunk = 16;
  while (launched < maxit) {
    int todo = maxit - launched < chunk ? maxit - launched : chunk;
    for (int it = 0; it < todo; ++it)
      if ((e = iter(launched + it == 0, s)) != cudaSuccess) return e;
    launched += todo;
    if ((e = cudaMemcpyAsync(&hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (hs.done) break;
  }
  if ((e = cudaMemcpyAsync(&hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *iters = hs.it;
  double bb = hs.bb > 0 ? hs.bb : 1.0;
  *relres = std::sqrt(hs.rr / bb);
  return cudaSuccess;
}

// PCG with the FDM preconditioner.  T = vector precision; the preconditioner
// always runs in FP32 (rf: FP32 copy of r when T = double, else r itself).
template <typename T, typename TX_, typename TB>
static cudaError_t cg_solve_fdm(const MeshDev& m, const T* bands, const double* coef,
                                const TB* b, TX_* x, const T* x_as_T, double rtol, int maxit,
                                T* r, T* z, T* zn, T* p0, T* p1, T* Ap, float* rf, float* zf,
                                FdmPlan* fdm, double* partials, CgScalars* sc,
                                cudaStream_t s, int* iters, double* relres, Timer* tm,
                                bool x_is_zero, cudaStream_t ls) {
  cudaError_t e;
  int64_t n = m.n_nodes;
  int vb = vec_blocks(n);
  const int op_stage = sizeof(T) == 8 ? kStageOp64 : kStageOp32;
  const bool conv = sizeof(T) == 8;  // FP32 copies needed for the preconditioner
  float* rin = conv ? rf : reinterpret_cast<float*>(r);
  if (x_is_zero) {
    if ((e = cudaMemsetAsync(Ap, 0, sizeof(T) * n, s)) != cudaSuccess) return e;
  } else {
    // the operator is skipped on the device when x0 has no nonzero entry
    k_flag_nonzero<TX_><<<vb, 256, 0, s>>>(n, x, &sc->xnz);
    count_launches(1);
    if (tm) tm->begin(op_stage, s);
    if ((e = apply_t<T>(m, bands, coef, x_as_T, Ap, s, &sc->xnz)) != cudaSuccess) return e;
    if (tm) tm->end(op_stage, s);
  }
  k_cg_start_fdm<T, TB><<<vb, 256, 0, s>>>(n, b, Ap, r, conv ? rf : nullptr, partials, sc, rtol,
                                          x_is_zero ? 0 : 1);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // z = P^-1 r
  float* zout = conv ? zf : reinterpret_cast<float*>(z);
  if ((e = fdm_apply(fdm, rin, zout, nullptr, s)) != cudaSuccess) return e;
  k_cg_dot_fdm<T><<<vb, 256, 0, s>>>(n, r, conv ? zf : nullptr, z, z, partials, sc, 1, 1);
  count_launches(1);
  T* pc = p0;
  T* pn = p1;
  T* zc = z;   // current preconditioned residual
  T* zo = zn;  // spare buffer
  auto iter = [&](int first, cudaStream_t st) -> cudaError_t {
    cudaError_t ee;
    if (tm) tm->begin(op_stage, st);
    if ((ee = cg_apply_t<T>(m, bands, coef, zc, pc, pn, Ap, partials, sc, first, st)) !=
        cudaSuccess)
      return ee;
    if (tm) tm->end(op_stage, st);
    k_cg_update_fdm<T, TX_><<<vb, 256, 0, st>>>(n, x, r, pn, Ap, conv ? rf : nullptr, partials,
                                                sc, maxit);
    count_launches(1);
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    // z_new = P^-1 r, beta (skipped on the device once converged)
    float* zo_f = conv ? zf : reinterpret_cast<float*>(zo);
    if ((ee = fdm_apply(fdm, rin, zo_f, &sc->done, st)) != cudaSuccess) return ee;
    k_cg_dot_fdm<T><<<vb, 256, 0, st>>>(n, r, conv ? zf : nullptr, zc, zo, partials, sc, 0, 0);
    count_launches(1);
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    T* t = zc;
    zc = zo;
    zo = t;
    t = pc;
    pc = pn;
    pn = t;
    return cudaSuccess;
  };
  if (ls) {  // device-driven loop inside a stream capture
    if ((e = iter(1, s)) != cudaSuccess) return e;
    if ((e = iter(0, s)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = loop_open(s, ls, &h, sc, maxit)) != cudaSuccess) return e;
    e = iter(0, ls);
    if (e == cudaSuccess) e = iter(0, ls);
    if ((e = loop_close(ls, h, sc, maxit, e)) != cudaSuccess) return e;
    *iters = -1;
    *relres = -1.0;
    return cudaSuccess;
  }
  CgScalars hs;
  if ((e = cudaMemcpyAsync(&hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  // iterations are queued in chunks: every kernel of an iteration (operator,
  // update, FDM transforms and solves, dot) returns at once on the device flag
  // `done`, so only one host round trip per chunk is needed; with the FDM
  // (an inverse up to rounding) the FP64 solve converges in about three
  // iterations, so chunks of three leave few launches that return at once
  const int chunk = sizeof(T) == 8 ? 3 : 2;
  int launched = 0;
  while (!hs.done && launched < maxit) {
    int todo = maxit - launched < chunk ? maxit - launched : chunk;
    for (int c = 0; c < todo; ++c)
      if ((e = iter(launched + c == 0, s)) != cudaSuccess) return e;
    launched += todo;
    if ((e = cudaMemcpyAsync(&hs, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  }
  *iters = hs.it;
  double bb = hs.bb > 0 ? hs.bb : 1.0;
  *relres = std::sqrt(hs.rr / bb);
  return cudaSuccess;
}

template <int K, class S>
static cudaError_t set_smem_df() {
  static bool done = false;
  if (done) return cudaSuccess;
  int sm = (int)apply_smem<K, S, df64>();
  cudaError_t e =
      cudaFuncSetAttribute(k_residual_df<K, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cg_apply_df<K, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) done = true;
  return e;
}

static Coefs<df64> split_coefs(const double* c) {
  Coefs<df64> cf;
  auto sp = [](double v) {
    float h = (float)v;
    return df64(h, (float)(v - (double)h));
  };
  cf.cM = sp(c[0]);
  cf.cKx = sp(c[1]);
  cf.cKy = sp(c[2]);
  cf.cKz = sp(c[3]);
  return cf;
}

// Mixed solve: conjugate gradients whose iterate, residual and operator are
// double-float (df64) and whose search directions and FDM preconditioner are
// FP32 -- Krylov-accelerated mixed-precision iterative refinement: the FP32
// preconditioner is the inner solver, the df64 residual keeps the outer
// accuracy at ~1e-14 without the FP64 pipes.
template <int K, class S>
static cudaError_t cg_solve_df(const MeshDev& m, const df64* bands, const double* coef,
                               const double* b, double* x, double rtol, int maxit, CgWork& w,
                               cudaStream_t s, int* iters, double* relres) {
  cudaError_t e;
  int64_t n = m.n_nodes;
  int vb = vec_blocks(n);
  Coefs<df64> cf = split_coefs(coef);
  if ((e = set_smem_df<K, S>()) != cudaSuccess) return e;
  const dim3 g = apply_grid_s<S>(m);
  const size_t sm = apply_smem<K, S, df64>();
  Timer* tm = w.timer;
  if ((e = cudaMemsetAsync(w.sc, 0, sizeof(CgScalars), s)) != cudaSuccess) return e;
  k_split_df<<<vb, 256, 0, s>>>(n, b, x, w.x_df, w.r_df, w.r32, w.partials, w.sc);
  k_residual_df<K, S><<<g, kApplyThreads, sm, s>>>(m, bands, cf, w.x_df, b, w.r_df, w.r32,
                                                w.partials, w.sc, rtol);
  count_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float* zc = w.z32;
  float* zo = w.zn32;
  df64* pc = w.p0_df;
  df64* pn = w.p1_df;
  // z = P^-1 r and r . z (the FDM's last pass forms the dot product where it can)
  const FdmDot dot0{w.r32, w.partials, w.sc, 1};
  bool fused = false;
  if ((e = fdm_apply(w.fdm, w.r32, zc, nullptr, s, &dot0, &fused)) != cudaSuccess) return e;
  if (!fused) {
    k_cg_dot_fdm<float><<<vb, 256, 0, s>>>(n, w.r32, nullptr, zc, zc, w.partials, w.sc, 1, 1);
    count_launches(1);
  }
  auto iter = [&](int first, cudaStream_t st) -> cudaError_t {
    cudaError_t ee;
    if (tm) tm->begin(kStageOp32, st);
    k_cg_apply_df<K, S><<<g, kApplyThreads, sm, st>>>(m, bands, cf, zc, pc, pn, w.Ap_df,
                                                     w.partials, w.sc, first);
    if (tm) tm->end(kStageOp32, st);
    k_cg_update_df<<<vb, 256, 0, st>>>(n, w.x_df, w.r_df, pn, w.Ap_df, w.r32, w.partials, w.sc,
                                      maxit);
    count_launches(2);
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    const FdmDot dot{w.r32, w.partials, w.sc, 0};
    bool fz = false;
    if ((ee = fdm_apply(w.fdm, w.r32, zo, &w.sc->done, st, &dot, &fz)) != cudaSuccess) return ee;
    if (!fz) {  // Fletcher-Reeves beta (see k_cg_dot_fdm)
      k_cg_dot_fdm<float><<<vb, 256, 0, st>>>(n, w.r32, nullptr, zc, zo, w.partials, w.sc, 0, 0,
                                             1);
      count_launches(1);
    }
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    float* t = zc;
    zc = zo;
    zo = t;
    df64* tp = pc;
    pc = pn;
    pn = tp;
    return cudaSuccess;
  };
  if (w.loop) {  // device-driven loop inside a stream capture
    if ((e = iter(1, s)) != cudaSuccess) return e;
    if ((e = iter(0, s)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = loop_open(s, w.loop, &h, w.sc, maxit)) != cudaSuccess) return e;
    e = iter(0, w.loop);
    if (e == cudaSuccess) e = iter(0, w.loop);
    if ((e = loop_close(w.loop, h, w.sc, maxit, e)) != cudaSuccess) return e;
    k_join_df<<<vb, 256, 0, s>>>(n, w.x_df, x);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *iters = -1;
    *relres = -1.0;
    return cudaSuccess;
  }
  CgScalars hs;
  if ((e = cudaMemcpyAsync(&hs, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  // eager: chunks of two iterations (the FDM-preconditioned mixed solve
  // converges in about two), one host round trip per chunk
  const int chunk = 2;
  int launched = 0;
  while (!hs.done && launched < maxit) {
    int todo = maxit - launched < chunk ? maxit - launched : chunk;
    for (int c = 0; c < todo; ++c)
      if ((e = iter(launched + c == 0, s)) != cudaSuccess) return e;
    launched += todo;
    if ((e = cudaMemcpyAsync(&hs, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  }
  k_join_df<<<vb, 256, 0, s>>>(n, w.x_df, x);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *iters = hs.it;
  double bb = hs.bb > 0 ? hs.bb : 1.0;
  *relres = std::sqrt(hs.rr / bb);
  return cudaSuccess;
}

cudaError_t run_cg64(const MeshDev& m, const double* bands, const double* coef,
                     const double* b, double* x, double rtol, int maxit, CgWork& w,
                     cudaStream_t s, int* iters_host, double* relres_host, int* converged) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.sc, 0, sizeof(CgScalars), s)) != cudaSuccess) return e;
  if (w.fdm) {
    e = cg_solve_fdm<double, double, double>(m, bands, coef, b, x, x, rtol, maxit, w.r, w.z,
                                             w.zn, w.p0, w.p1, w.Ap, w.r32, w.z32, w.fdm,
                                             w.partials, w.sc, s, iters_host, relres_host,
                                             w.timer, false, w.loop);
    if (e != cudaSuccess) return e;
    *converged = *relres_host <= rtol;
    return cudaSuccess;
  }
  if ((e = make_dinv<double>(m, bands, coef, w.dinv, s)) != cudaSuccess) return e;
  e = cg_solve<double, double, double>(m, bands, coef, b, x, x, rtol, maxit, w.r, w.z, w.p0,
                                       w.p1, w.Ap, w.dinv, w.partials, w.sc, s, iters_host,
                                       relres_host, w.timer, w.loop);
  if (e != cudaSuccess) return e;
  *converged = *relres_host <= rtol;
  return cudaSuccess;
}

cudaError_t run_cg_mixed(const MeshDev& m, const double* bands64, const float* bands32,
                         const double* coef, const double* b, double* x, double rtol,
                         int maxit, CgWork& w, cudaStream_t s, int* iters_host,
                         int* outer_host, double* relres_host, int* converged) {
  cudaError_t e;
  int64_t n = m.n_nodes;
  int vb = vec_blocks(n);
  if (w.fdm && w.bands_df) {
    int it = 0;
    double rel = 0.0;
    e = with_k(m, [&](auto kc) {
      constexpr int K = decltype(kc)::value;
      return with_shape(m, [&](auto sh) {
        return cg_solve_df<K, decltype(sh)>(m, w.bands_df, coef, b, x, rtol, maxit, w, s, &it,
                                             &rel);
      });
    });
    if (e != cudaSuccess) return e;
    *iters_host = it;
    *outer_host = it;
    *relres_host = rel;
    *converged = rel <= rtol;
    return cudaSuccess;
  }
  // the refinement loop below decides on the host: it cannot run inside a
  // stream capture (the graph form of the mixed solve needs the FDM path)
  if (w.loop) return cudaErrorNotSupported;
  if (!w.fdm && (e = make_dinv<float>(m, bands64, coef, w.dinv32, s)) != cudaSuccess) return e;
  int total_it = 0, outer = 0;
  double relres = 1.0;
  const int max_outer = 8;
  const double inner_rtol = 1e-6;
  CgScalars hs;
  for (;;) {
    // r = b - A x in FP64
    if (w.timer) w.timer->begin(kStageOp64, s);
    if ((e = apply_t<double>(m, bands64, coef, x, w.Ap, s)) != cudaSuccess) return e;
    if (w.timer) w.timer->end(kStageOp64, s);
    if ((e = cudaMemsetAsync(w.sc, 0, sizeof(CgScalars), s)) != cudaSuccess) return e;
    k_residual<double><<<vb, 256, 0, s>>>(n, b, w.Ap, w.r, w.partials, w.sc);
    count_launches(1);
    if ((e = cudaMemcpyAsync(&hs, w.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double bb = hs.bb > 0 ? hs.bb : 1.0;
    relres = std::sqrt(hs.rr / bb);
    if (relres <= rtol || outer >= max_outer || total_it >= maxit) break;
    // FP32 correction solve A d = r / |r|
    double rn = std::sqrt(hs.rr);
    double scale = rn > 0 ? 1.0 / rn : 1.0;
    k_to_f32<<<vb, 256, 0, s>>>(n, w.r, scale, w.rin32, w.d32);
    count_launches(1);
    if ((e = cudaMemsetAsync(w.sc, 0, sizeof(CgScalars), s)) != cudaSuccess) return e;
    int it = 0;
    double rr = 0;
    if (w.fdm)
      e = cg_solve_fdm<float, float, float>(m, bands32, coef, w.rin32, w.d32, w.d32, inner_rtol,
                                            maxit - total_it, w.r32, w.z32, w.zn32, w.q0, w.q1,
                                            w.Aq, nullptr, nullptr, w.fdm, w.partials, w.sc, s,
                                            &it, &rr, w.timer, true, nullptr);
    else
      e = cg_solve<float, float, float>(m, bands32, coef, w.rin32, w.d32, w.d32, inner_rtol,
                                        maxit - total_it, w.r32, w.z32, w.q0, w.q1, w.Aq,
                                        w.dinv32, w.partials, w.sc, s, &it, &rr, w.timer,
                                        nullptr);
    if (e != cudaSuccess) return e;
    total_it += it;
    k_add_scaled<<<vb, 256, 0, s>>>(n, x, w.d32, rn);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++outer;
  }
  *iters_host = total_it;
  *outer_host = outer;
  *relres_host = relres;
  *converged = relres <= rtol;
  return cudaSuccess;
}

}  // namespace cfdem
