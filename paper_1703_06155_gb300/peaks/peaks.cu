// Arithmetic peak probes of the GPU the library runs on: FP64 FMA, FP32 FMA
// and FP64 tensor-core (DMMA, mma.sync m8n8k4) throughput, each measured with
// CUDA events over a grid of 4 CTAs per SM running independent dependency
// chains.  They give the roofline denominators of the FP64- and FP32-pipe
// kernel classes measured rather than derived from unit counts and clocks.
// Separate from libh2 (its own small library, libh2peaks.so).
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int NT = 256;
constexpr int CH = 8;  // independent chains per thread

template <class T>
__global__ void __launch_bounds__(NT) k_fma(T* out, int iters, T b, T c) {
  T a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b, c);
  T s = 0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  if (s == (T)12345.678) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(NT) k_dmma(double* out, int iters) {
  // per warp: 4 independent m8n8k4 FP64 accumulators
  double a = 1e-3 * (threadIdx.x & 31), b = 2e-3;
  double d[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k][0] = d[k][1] = 0.0;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d[k][0]), "+d"(d[k][1])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

// kind 0: FP64 FMA, 1: FP32 FMA, 2: FP64 DMMA.  Writes the measured rate in
// TFLOP/s (FMA = 2 flops; m8n8k4 = 512 flops per warp) to *tflops.
// Returns 0, or a cudaError_t value.
extern "C" int h2_peak_probe(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = 4 * sms;
  void* out = nullptr;
  e = cudaMalloc(&out, blocks * sizeof(double));
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = kind == 2 ? 4096 : kind == 1 ? 131072 : 16384;
  auto launch = [&]() {
    if (kind == 0) k_fma<double><<<blocks, NT>>>((double*)out, iters, 0.999, 1e-7);
    else if (kind == 1) k_fma<float><<<blocks, NT>>>((float*)out, iters, 0.999f, 1e-7f);
    else k_dmma<<<blocks, NT>>>((double*)out, iters);
  };
  launch();  // warm-up
  cudaEventRecord(e0);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return (int)e;
  double flops;
  if (kind == 2) flops = 512.0 * 4 * (double)iters * (blocks * (NT / 32)) * reps;
  else flops = 2.0 * CH * (double)iters * blocks * NT * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return 0;
}
