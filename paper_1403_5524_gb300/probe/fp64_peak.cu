// FP64 pipe peak of the current device, measured: the roofline denominator of the
// FP64-bound kernels (the matching solve, the near-pole window).
//
// Every thread runs eight independent chains of dependent FMAs, x <- x * b + c, so the FP64 pipe
// always has independent work (GB300 saturates its FP64 pipe with four warps per SM and one chain
// each); the grid is eight 256-thread CTAs per SM.  b and c come from memory, so nothing folds at
// compile time, and the chains' sums are stored, so nothing is dropped.  Each FMA counts two
// flops.  The result is the best of `reps` timed launches (CUDA events) after one warm-up.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_kernel(const double* __restrict__ bc, int iters,
                                                         double* __restrict__ out) {
  const double b = bc[0], c = bc[1];
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = (double)(threadIdx.x + q) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// tflops: best measured FP64 rate (10^12 flop/s); ms: that launch's duration.  Returns 0 on
// success, else the CUDA error code.
extern "C" int rm_probe_fp64_peak(int reps, double* tflops, double* ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = sms * 8;
  const int iters = 1 << 14;
  double* bc = nullptr;
  double* out = nullptr;
  cudaEvent_t a = nullptr, z = nullptr;
  e = cudaMalloc(&bc, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads);
  const double hb[2] = {0.999999, 1e-7};
  if (e == cudaSuccess) e = cudaMemcpy(bc, hb, sizeof(hb), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  double best = 1e30;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    cudaEventRecord(a);
    dfma_kernel<<<blocks, kThreads>>>(bc, iters, out);
    cudaEventRecord(z);
    e = cudaEventSynchronize(z);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, z);
    if (r > 0 && e == cudaSuccess && t < best) best = t;  // launch 0 is the warm-up
  }
  if (e == cudaSuccess) {
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *ms = best;
    *tflops = flops / (best * 1e-3) / 1e12;
  }
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (bc) cudaFree(bc);
  if (out) cudaFree(out);
  return (int)e;
}
