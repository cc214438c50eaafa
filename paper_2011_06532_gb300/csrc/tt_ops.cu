// tt_ops.cu -- the feeder operations: summation (Sec. 3.2.1), Hadamard product
// (Sec. 3.2.2) and inner product (Sec. 3.2.3).  Summation and Hadamard are pure
// HBM-streaming kernels over the output cores (one thread per output element,
// consecutive threads write consecutive elements).  The inner product runs the
// two-multiplication form of Sec. 3.2.3 per core: each CTA takes a slab of slices,
// forms Z(i) = W_{n-1} X_n(i) and accumulates Y_n(i)^T Z(i); the per-CTA partial sums
// are then added in a fixed order (deterministic) into W_n.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "tt.h"
#include "tt_engine.h"
#include "tt_internal.cuh"

namespace ttgb {

#define TT_CUDA(call)                          \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return TT_ERR_CUDA; \
  } while (0)

// ------------------------------------------------------------------------------------
// summation
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void k_add_core(const T *__restrict__ X, const T *__restrict__ Y, T *__restrict__ Z, int64_t I, int ra0,
                           int ra1, int rb0, int rb1, int rs, int cs, int single) {
  const int r0 = single ? 1 : (rs ? ra0 + rb0 : ra0);  // rows of Z
  const int r1 = single ? 1 : (cs ? ra1 + rb1 : ra1);  // columns of Z
  const int64_t total = (int64_t)r0 * I * r1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (single) {
      Z[e] = X[e] + Y[e];
      continue;
    }
    const int a = (int)(e % r0);
    const int64_t rest = e / r0;
    const int64_t i = rest % I;
    const int c = (int)(rest / I);
    T v = T(0);
    if (a < ra0 && c < ra1) {
      v = X[a + (int64_t)ra0 * (i + I * c)];
    } else {
      const int ya = a - rs, yc = c - cs;
      if (ya >= 0 && ya < rb0 && yc >= 0 && yc < rb1) v = Y[ya + (int64_t)rb0 * (i + I * yc)];
    }
    Z[e] = v;
  }
}

static int grid_for(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

int add_run(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, cudaStream_t st) {
  const int N = a->N;
  out->R[0] = 1;
  out->R[N] = 1;
  for (int n = 1; n < N; ++n) out->R[n] = a->R[n] + b->R[n];
  for (int n = 0; n < N; ++n) {
    const int single = N == 1;
    const int ra0 = (int)a->R[n], ra1 = (int)a->R[n + 1], rb0 = (int)b->R[n], rb1 = (int)b->R[n + 1];
    const int rs = n == 0 ? 0 : ra0;      // row offset of the B block
    const int cs = n == N - 1 ? 0 : ra1;  // column offset of the B block
    const int64_t total = out->R[n] * a->I[n] * out->R[n + 1];
    TraceScope ts_(TT_K_ADD, st);
    if (a->dtype == TT_F64)
      k_add_core<double><<<grid_for(total), 256, 0, st>>>((const double *)a->cores[n], (const double *)b->cores[n],
                                                            (double *)out->cores[n], a->I[n], ra0, ra1, rb0, rb1, rs,
                                                            cs, single);
    else
      k_add_core<float><<<grid_for(total), 256, 0, st>>>((const float *)a->cores[n], (const float *)b->cores[n],
                                                           (float *)out->cores[n], a->I[n], ra0, ra1, rb0, rb1, rs, cs,
                                                           single);
    TT_CUDA(cudaGetLastError());
  }
  return TT_OK;
}

// ------------------------------------------------------------------------------------
// Hadamard product
// ------------------------------------------------------------------------------------

template <typename T>
__global__ void k_hadamard_core(const T *__restrict__ X, const T *__restrict__ Y, T *__restrict__ Z, int64_t I,
                                int ra0, int ra1, int rb0, int rb1) {
  const int r0 = ra0 * rb0, r1 = ra1 * rb1;
  const int64_t total = (int64_t)r0 * I * r1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e % r0);
    const int64_t rest = e / r0;
    const int64_t i = rest % I;
    const int col = (int)(rest / I);
    const int p = row / rb0, q = row - p * rb0, s = col / rb1, t = col - s * rb1;
    Z[e] = X[p + (int64_t)ra0 * (i + I * s)] * Y[q + (int64_t)rb0 * (i + I * t)];
  }
}

int hadamard_run(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, cudaStream_t st) {
  const int N = a->N;
  for (int n = 0; n <= N; ++n) out->R[n] = a->R[n] * b->R[n];
  for (int n = 0; n < N; ++n) {
    const int ra0 = (int)a->R[n], ra1 = (int)a->R[n + 1], rb0 = (int)b->R[n], rb1 = (int)b->R[n + 1];
    const int64_t total = out->R[n] * a->I[n] * out->R[n + 1];
    TraceScope ts_(TT_K_HADAMARD, st);
    if (a->dtype == TT_F64)
      k_hadamard_core<double><<<grid_for(total), 256, 0, st>>>((const double *)a->cores[n],
                                                                 (const double *)b->cores[n], (double *)out->cores[n],
                                                                 a->I[n], ra0, ra1, rb0, rb1);
    else
      k_hadamard_core<float><<<grid_for(total), 256, 0, st>>>((const float *)a->cores[n], (const float *)b->cores[n],
                                                                (float *)out->cores[n], a->I[n], ra0, ra1, rb0, rb1);
    TT_CUDA(cudaGetLastError());
  }
  return TT_OK;
}

// ------------------------------------------------------------------------------------
// inner product
// ------------------------------------------------------------------------------------

constexpr int kDotBlocks = 304;  // CTAs per core (2 per SM); partial sums are reduced in fixed order

// One CTA: slices [s0, s1) of core n.  W (ry0 x rx0, FP64) -> partial (ry1 x rx1, FP64).
// shared: W (ry0*rx0 T), Z (ry0*rx1 T), acc (ry1*rx1 double)
template <typename T>
__global__ void __launch_bounds__(256) k_dot_core(const T *__restrict__ X, const T *__restrict__ Y, int64_t I, int rx0,
                                                  int rx1, int ry0, int ry1, const double *__restrict__ W,
                                                  double *__restrict__ partial, int *E, int big) {
  // big = 0: W (scaled), Z and the accumulator in shared memory; big = 1 (ranks whose three
  // blocks do not fit): only Z in shared memory, W read from global memory and scaled on the
  // fly, the accumulator kept in this block's slice of `partial` (no other block touches it)
  extern __shared__ __align__(16) unsigned char smem[];
  T *Ws = reinterpret_cast<T *>(smem);
  T *Zs = big ? reinterpret_cast<T *>(smem) : Ws + ry0 * rx0;
  double *out = partial + (size_t)blockIdx.x * ry1 * rx1;
  double *acc = big ? out
                    : reinterpret_cast<double *>(smem + ((sizeof(T) * (size_t)(ry0 * rx0 + ry0 * rx1) + 15) / 16) * 16);
  __shared__ double red[8];
  const int t = threadIdx.x;
  // W_{n-1} enters in [2^-32, 2^32] up to an exact power of two, accumulated in E (every
  // block finds the same exponent; block 0 records it)
  const int e = range_exp(block_absmax(W, ry0 * rx0, red));
  const double wsc = ldexp(1.0, -e);
  if (!big)
    for (int idx = t; idx < ry0 * rx0; idx += blockDim.x) Ws[idx] = (T)ldexp(W[idx], -e);
  if (blockIdx.x == 0 && t == 0 && e != 0) *E += e;
  for (int idx = t; idx < ry1 * rx1; idx += blockDim.x) acc[idx] = 0.0;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * I / gridDim.x, s1 = (int64_t)(blockIdx.x + 1) * I / gridDim.x;
  for (int64_t i = s0; i < s1; ++i) {
    // Z = W X(i): Z[p][s] = sum_r W[p][r] X[r, i, s]   (W row-major ry0 x rx0)
    for (int idx = t; idx < ry0 * rx1; idx += blockDim.x) {
      const int p = idx / rx1, s = idx - p * rx1;
      T z = T(0);
      const T *xc = X + (int64_t)rx0 * (i + I * s);
      if (big) {
        for (int r = 0; r < rx0; ++r) z += (T)(W[p * rx0 + r] * wsc) * xc[r];
      } else {
        for (int r = 0; r < rx0; ++r) z += Ws[p * rx0 + r] * xc[r];
      }
      Zs[idx] = z;
    }
    __syncthreads();
    // acc[q][s] += sum_p Y[p, i, q] Z[p][s]
    for (int idx = t; idx < ry1 * rx1; idx += blockDim.x) {
      const int q = idx / rx1, s = idx - q * rx1;
      const T *yc = Y + (int64_t)ry0 * (i + I * q);
      T v = T(0);
      for (int p = 0; p < ry0; ++p) v += yc[p] * Zs[p * rx1 + s];
      acc[idx] += (double)v;
    }
    __syncthreads();
  }
  if (!big)
    for (int idx = t; idx < ry1 * rx1; idx += blockDim.x) out[idx] = acc[idx];
}

__global__ void k_dot_reduce(const double *__restrict__ partial, int nblk, int n, double *__restrict__ W) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += partial[(size_t)k * n + idx];
    W[idx] = s;
  }
}

__global__ void k_dot_init(double *W, int *E) {
  if (threadIdx.x == 0) {
    W[0] = 1.0;
    *E = 0;
  }
}

__global__ void k_dot_finish(double *W, const int *E) {
  if (threadIdx.x == 0) W[0] = ldexp(W[0], *E);
}

static int dot_blocks(int64_t I) { return (int)std::min<int64_t>(I, kDotBlocks); }

int dot_workspace(const tt_tensor *a, const tt_tensor *b, size_t *bytes) {
  int64_t maxw = 1, maxp = 1;
  for (int n = 0; n <= a->N; ++n) maxw = std::max<int64_t>(maxw, a->R[n] * b->R[n]);
  for (int n = 0; n < a->N; ++n) maxp = std::max<int64_t>(maxp, dot_blocks(a->I[n]) * a->R[n + 1] * b->R[n + 1]);
  *bytes = 256 + sizeof(double) * (size_t)(2 * maxw + maxp) + 512;
  return TT_OK;
}

int dot_run(const tt_tensor *a, const tt_tensor *b, double *result, void *ws, size_t ws_bytes, cudaStream_t st) {
  size_t need = 0;
  dot_workspace(a, b, &need);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  int64_t maxw = 1, maxp = 1;
  for (int n = 0; n <= a->N; ++n) maxw = std::max<int64_t>(maxw, a->R[n] * b->R[n]);
  for (int n = 0; n < a->N; ++n) maxp = std::max<int64_t>(maxp, dot_blocks(a->I[n]) * a->R[n + 1] * b->R[n + 1]);
  double *W0 = reinterpret_cast<double *>(ws);
  double *W1 = W0 + maxw;
  double *part = W1 + maxw;
  int *E = reinterpret_cast<int *>(part + maxp);  // exponent of the W rescaling
  {
    TraceScope ts_(TT_K_MISC, st);
    k_dot_init<<<1, 32, 0, st>>>(W0, E);
  }
  TT_CUDA(cudaGetLastError());
  for (int n = 0; n < a->N; ++n) {
    const int rx0 = (int)a->R[n], rx1 = (int)a->R[n + 1], ry0 = (int)b->R[n], ry1 = (int)b->R[n + 1];
    const int nb = dot_blocks(a->I[n]);
    const size_t es = a->dtype == TT_F64 ? 8 : 4;
    size_t smem = ((es * (size_t)(ry0 * rx0 + ry0 * rx1) + 15) / 16) * 16 + sizeof(double) * ry1 * rx1;
    const int big = smem > 220 * 1024 ? 1 : 0;
    if (big) smem = es * (size_t)ry0 * rx1;
    if (smem > 220 * 1024) return TT_ERR_UNSUPPORTED;
    TraceScope ts_(TT_K_DOT, st);
    if (a->dtype == TT_F64) {
      if (smem > 48 * 1024)
        TT_CUDA(cudaFuncSetAttribute(k_dot_core<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_dot_core<double><<<nb, 256, smem, st>>>((const double *)a->cores[n], (const double *)b->cores[n], a->I[n],
                                                  rx0, rx1, ry0, ry1, W0, part, E, big);
    } else {
      if (smem > 48 * 1024)
        TT_CUDA(cudaFuncSetAttribute(k_dot_core<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_dot_core<float><<<nb, 256, smem, st>>>((const float *)a->cores[n], (const float *)b->cores[n], a->I[n], rx0,
                                                 rx1, ry0, ry1, W0, part, E, big);
    }
    TT_CUDA(cudaGetLastError());
    {
      TraceScope ts_(TT_K_DOT, st);
      k_dot_reduce<<<(ry1 * rx1 + 255) / 256, 256, 0, st>>>(part, nb, ry1 * rx1, W1);
    }
    TT_CUDA(cudaGetLastError());
    std::swap(W0, W1);
  }
  {
    TraceScope ts_(TT_K_MISC, st);
    k_dot_finish<<<1, 32, 0, st>>>(W0, E);
  }
  TT_CUDA(cudaGetLastError());
  TT_CUDA(cudaMemcpyAsync(result, W0, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  return TT_OK;
}

// ------------------------------------------------------------------------------------
// inner product without any allocation: scratch in a fixed device array
// ------------------------------------------------------------------------------------

// Scratch of tt_dot_noalloc: every process that loads this library holds this array on
// every device it uses, until exit.  It is shared by all calls (no per-call state).
static __device__ __align__(256) double g_dot_scratch[TT_DOT_NOALLOC_SCRATCH_BYTES / sizeof(double)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of g_dot_scratch for the current device.  The first call on a device
// looks it up (host code cannot use the symbol itself: in host code it names a host-side
// stand-in, not device memory).
static int dot_scratch_ptr(double **out) {
  int dev = 0;
  TT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    TT_CUDA(cudaGetSymbolAddress(&p, g_dot_scratch));
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return TT_OK;
}

int dot_noalloc_run(const tt_tensor *a, const tt_tensor *b, double *result, cudaStream_t st) {
  size_t need = 0;
  dot_workspace(a, b, &need);
  if (need > TT_DOT_NOALLOC_SCRATCH_BYTES) return TT_ERR_UNSUPPORTED;
  double *scratch = nullptr;
  const int r = dot_scratch_ptr(&scratch);
  if (r) return r;
  // W0 is set by the first kernel and every partial sum is written before it is read,
  // so nothing left by an earlier call needs clearing.
  return dot_run(a, b, result, scratch, TT_DOT_NOALLOC_SCRATCH_BYTES, st);
}

}  // namespace ttgb
