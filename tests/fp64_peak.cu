// FP64 FMA throughput of this GPU: every thread runs 8 independent FMA chains (enough to
// cover the FP64 unit's latency), one grid of 8 CTAs x 256 threads per SM, timed with CUDA
// events after a warm-up launch.  Prints the rate in TFLOP/s (2 flops per FMA) and the SM
// count; the library's FP64 kernels are judged against this unit's peak.
#include <cstdio>

__global__ void __launch_bounds__(256) fma_chains(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int k = 0; k < iters; ++k) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[0] = s;  // keeps the chains alive; never true for these inputs
}

int main() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return 1;
  const int blocks = sms * 8, threads = 256, iters = 20000;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<<<blocks, threads>>>(out, iters / 10, 0.999999, 1e-6);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  fma_chains<<<blocks, threads>>>(out, iters, 0.999999, 1e-6);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  const cudaError_t err = cudaGetLastError();
  printf("fp64_tflops %.4f sms %d ms %.3f err %s\n", flops / (ms * 1e-3) / 1e12, sms, ms, cudaGetErrorString(err));
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
