// alu_peak.cu -- FMA throughput of the device, the denominator of the
// roofline of kernels bound by plain FP32 or FP64 arithmetic.
//
// Every thread runs 8 independent FMA chains (enough to hide the FMA
// latency on every pipe), 152 x 8 blocks of 256 threads; the best of five
// CUDA-event timings of one launch is reported as flops / s with 2 flops per
// FMA.  Built into its own library (libalupeak.so): it is a measurement
// tool, not part of the coupling library.
#include <cuda_runtime.h>

namespace {

template <typename T, int ITER>
__global__ void __launch_bounds__(256) k_fma_chains(T b, T c, T* out) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
#pragma unroll 16
  for (int i = 0; i < ITER; ++i) {
    a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
    a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

template <typename T, int ITER>
cudaError_t measure(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, z = nullptr;
  double best = 0.0;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) == cudaSuccess &&
      (e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&z)) == cudaSuccess) {
    const T b = (T)0.9999, c = (T)1e-4;
    for (int rep = 0; rep < 7 && e == cudaSuccess; ++rep) {
      cudaEventRecord(a, s);
      k_fma_chains<T, ITER><<<blocks, threads, 0, s>>>(b, c, out);
      cudaEventRecord(z, s);
      e = cudaEventSynchronize(z);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
      const double flops = 2.0 * 8.0 * ITER * (double)blocks * threads;
      if (e == cudaSuccess && rep >= 2 && ms > 0.f) {   // two warm-up launches
        const double v = flops / (ms * 1e-3) / 1e12;
        if (v > best) best = v;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  *tflops = best;
  return e;
}

}  // namespace

// FMA throughput of the current device in TFLOP/s: fp64 = 0 for FP32,
// 1 for FP64.  Returns the CUDA error code (0 on success).
extern "C" int alu_fma_peak(int fp64, double* tflops) {
  if (!tflops) return (int)cudaErrorInvalidValue;
  return (int)(fp64 ? measure<double, 512>(tflops) : measure<float, 8192>(tflops));
}
