// FP64 / FP32 FMA and FP64 sqrt / sincos throughput probe (the denominator of the
// FP64 roofline of the pair pipeline).  Bounded loops, no waits.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/peak_probe paper_2608_16208_b300/peak_probe.cu && /tmp/peak_probe
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void dsqrt_k(double* out, int iters) {
  double x = 1.0 + threadIdx.x * 1e-6, acc = 0;
  for (int i = 0; i < iters; ++i) { acc += sqrt(x); x += 1e-9; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}
__global__ void dsincos_k(double* out, int iters) {
  double x = 0.1 + threadIdx.x * 1e-6, acc = 0;
  for (int i = 0; i < iters; ++i) { double s, c; sincos(x, &s, &c); acc += s + c; x += 1e-7; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("SMs %d clock(kHz) %d\n", sms, clk);
  const int threads = 256;
  for (int bps : {4, 8}) {
    int blocks = sms * bps;
    void* buf; cudaMalloc(&buf, (size_t)blocks * threads * 8);
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    for (int rep = 0; rep < 2; ++rep) {
      int it64 = 2000;
      cudaEventRecord(e0);
      fma_chain<double><<<blocks, threads>>>((double*)buf, it64, 0.999, 1e-3);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double flops = 2.0 * 128.0 * it64 * (double)blocks * threads;
      printf("fp64 fma bps=%d: %.3f ms  %.1f GFLOP/s\n", bps, ms, flops / ms / 1e6);
      int it32 = 20000;
      cudaEventRecord(e0);
      fma_chain<float><<<blocks, threads>>>((float*)buf, it32, 0.999f, 1e-3f);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      flops = 2.0 * 128.0 * it32 * (double)blocks * threads;
      printf("fp32 fma bps=%d: %.3f ms  %.1f GFLOP/s\n", bps, ms, flops / ms / 1e6);
      cudaEventRecord(e0);
      dsqrt_k<<<blocks, threads>>>((double*)buf, 2000);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      printf("dsqrt bps=%d: %.3f ms  %.2f Gsqrt/s\n", bps, ms, 2000.0 * blocks * threads / ms / 1e6);
      cudaEventRecord(e0);
      dsincos_k<<<blocks, threads>>>((double*)buf, 500);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      printf("dsincos bps=%d: %.3f ms  %.2f Gsincos/s\n", bps, ms, 500.0 * blocks * threads / ms / 1e6);
    }
    cudaFree(buf);
  }
  cudaError_t err = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
