// reduce.cuh -- deterministic block and grid reductions of the CG kernels.
#pragma once

#include <cstdint>

#include "df64.cuh"

namespace cfdem {

__device__ __forceinline__ double block_sum(double v, double* red) {
  // red: >= 32 doubles of shared memory
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Block sum of FP32 partials: a fixed shuffle tree in FP32 within each warp,
// then the warps' sums widened exactly (bit moves, no conversion
// instruction) and added in FP64 by warp 0 -- a handful of FP64 additions
// per block instead of a 64-bit shuffle tree per thread (FP64 issues on a
// narrow pipe on this part).  Deterministic; valid in thread 0.
__device__ __forceinline__ double block_sum_f(float v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = double_from_float_int(v);
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 0; w < nw; ++w) s += red[w];
  }
  return s;
}

__device__ __forceinline__ double block_sum(float v, double* red) { return block_sum_f(v, red); }

// last block to finish reduces partials[0..nb) (nvals interleaved values) in
// fixed order; returns true in the last block (results in out[0..nvals))
static __device__ bool last_block_reduce(double* partials, int nvals, const double* vals,
                                         unsigned int* ticket, double* out, double* red) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    const size_t nb = (size_t)gridDim.x * gridDim.y * gridDim.z;
    const size_t blk = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    for (int v = 0; v < nvals; ++v) partials[(size_t)v * nb + blk] = vals[v];
    __threadfence();
    unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    unsigned t = atomicInc(ticket, nblk - 1);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  for (int v = 0; v < nvals; ++v) {
    double s = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x)
      s += ((volatile double*)partials)[(size_t)v * nblk + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[v] = s;
  }
  return true;
}

}  // namespace cfdem
