// Checks the Newton-Raphson FP64 reciprocal / reciprocal square root of tt_internal.cuh
// against CUDA's correctly rounded 1.0 / x and 1.0 / sqrt(x) on many arguments spanning
// the range the kernels use; prints the largest error in ulps of each.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tt_internal.cuh"

__global__ void eval(const double *x, double *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    out[4 * i + 0] = ttgb::rcp_nr(x[i]);
    out[4 * i + 1] = 1.0 / x[i];
    out[4 * i + 2] = ttgb::rsqrt_nr(fabs(x[i]));
    out[4 * i + 3] = 1.0 / sqrt(fabs(x[i]));
  }
}

static double ulps(double a, double b) {
  int64_t ia, ib;
  memcpy(&ia, &a, 8);
  memcpy(&ib, &b, 8);
  if ((ia < 0) != (ib < 0)) return 1e30;
  return (double)(ia > ib ? ia - ib : ib - ia);
}

int main() {
  const int n = 1 << 20;
  std::vector<double> x(n);
  uint64_t s = 88172645463325252ull;
  for (int i = 0; i < n; ++i) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;  // xorshift64
    const double m = 1.0 + (double)(s >> 11) * (1.0 / 9007199254740992.0);
    const int e = (int)((s >> 3) % 1160) - 580;  // 2^-580 .. 2^579
    x[i] = ldexp(m, e) * ((s & 1) ? -1.0 : 1.0);
  }
  double *dx, *dout;
  cudaMalloc(&dx, n * sizeof(double));
  cudaMalloc(&dout, 4 * n * sizeof(double));
  cudaMemcpy(dx, x.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  eval<<<(n + 255) / 256, 256>>>(dx, dout, n);
  std::vector<double> out(4 * (size_t)n);
  cudaMemcpy(out.data(), dout, 4 * n * sizeof(double), cudaMemcpyDeviceToHost);
  double w_rcp = 0, w_rsq = 0;
  for (int i = 0; i < n; ++i) {
    w_rcp = fmax(w_rcp, ulps(out[4 * i], out[4 * i + 1]));
    w_rsq = fmax(w_rsq, ulps(out[4 * i + 2], out[4 * i + 3]));
  }
  printf("max_ulp_rcp %.0f max_ulp_rsqrt %.0f err %s\n", w_rcp, w_rsq, cudaGetErrorString(cudaGetLastError()));
  return 0;
}
