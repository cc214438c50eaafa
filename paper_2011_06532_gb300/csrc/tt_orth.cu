// tt_orth.cu -- orthonormalization (Alg. 1 / Alg. 5 and their left-hand mirror) and the
// LRL ordering of TT rounding (Sec. 3.4, Sec. 4.3.2).
//
// Left-hand operations run the right-hand machinery on the mode-reversed tensor.
// Reversing the modes of X gives the TT X' with cores X'_m = X_{N-1-m}^T (the two rank
// indices of each core swapped); its horizontal unfolding transposed, H(X'_m)^T, is the
// vertical unfolding V(X_{N-1-m}) with its rows permuted.  A row permutation leaves the R
// factor of a QR unchanged and permutes the rows of Q, so the right-to-left sweep over X'
// performs, core by core, the left-to-right sweep over X (left-orthonormalization), and
// the truncation from the left over X' is the truncation from the right over X: the LRL
// rounding of X is the reversal of the RLR rounding of X'.  The reversals are two
// memory-bound passes (one over the input, one over the output).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "tt.h"
#include "tt_engine.h"

namespace ttgb {

namespace {

// out (R1 x I x R0) <- in (R0 x I x R1) with the rank indices swapped:
// out[b + R1 (i + I a)] = in[a + R0 (i + I b)].  Tiled through shared memory so that both
// the reads (along a) and the writes (along b) are coalesced.
template <typename S>
__global__ void __launch_bounds__(256) k_reverse_core(const S *in, S *out, int R0, int64_t I, int R1) {
  __shared__ S tile[32][33];
  const int64_t i = blockIdx.z;
  const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int y = ty; y < 32; y += 8) {
    const int a = a0 + tx, b = b0 + y;
    if (a < R0 && b < R1) tile[y][tx] = in[(size_t)a + (size_t)R0 * ((size_t)i + (size_t)I * b)];
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int b = b0 + tx, a = a0 + y;
    if (a < R0 && b < R1) out[(size_t)b + (size_t)R1 * ((size_t)i + (size_t)I * a)] = tile[tx][y];
  }
}

// Queues the reversal of every core of x (shape N, I, R) into the buffers dst (dst[m]
// receives core N-1-m transposed).
int reverse_cores(int N, const int64_t *I, const int64_t *R, int dtype, void *const *src, void *const *dst,
                  cudaStream_t st) {
  for (int n = 0; n < N; ++n) {
    const int R0 = (int)R[n], R1 = (int)R[n + 1];
    // grid.z holds the slices (at most 65535 per launch); longer modes in chunks
    for (int64_t i0 = 0; i0 < I[n]; i0 += 65535) {
      const int64_t ni = std::min<int64_t>(65535, I[n] - i0);
      dim3 grid((R0 + 31) / 32, (R1 + 31) / 32, (unsigned)ni);
      TraceScope ts_(TT_K_MISC, st);
      if (dtype == TT_F64) {
        const double *in = reinterpret_cast<const double *>(src[n]) + (size_t)R0 * i0;
        double *out = reinterpret_cast<double *>(dst[N - 1 - n]) + (size_t)R1 * i0;
        k_reverse_core<double><<<grid, 256, 0, st>>>(in, out, R0, I[n], R1);
      } else {
        const float *in = reinterpret_cast<const float *>(src[n]) + (size_t)R0 * i0;
        float *out = reinterpret_cast<float *>(dst[N - 1 - n]) + (size_t)R1 * i0;
        k_reverse_core<float><<<grid, 256, 0, st>>>(in, out, R0, I[n], R1);
      }
      if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
    }
  }
  return TT_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// The mode-reversed description of x with its cores placed in a region of the workspace.
struct Reversed {
  std::vector<int64_t> I, R;
  std::vector<void *> cores;
  tt_tensor t{};
  size_t bytes = 0;  // total bytes of the cores (each 256-aligned)

  Reversed(const tt_tensor *x, unsigned char *base) {
    const int N = x->N;
    const size_t es = x->dtype == TT_F64 ? 8 : 4;
    I.resize(N);
    R.resize(N + 1);
    cores.resize(N);
    for (int m = 0; m < N; ++m) I[m] = x->I[N - 1 - m];
    for (int m = 0; m <= N; ++m) R[m] = x->R[N - m];
    for (int m = 0; m < N; ++m) {
      cores[m] = base ? base + bytes : nullptr;
      bytes += align256(es * (size_t)R[m] * I[m] * R[m + 1]);
    }
    t.N = N;
    t.dtype = x->dtype;
    t.I = I.data();
    t.R = R.data();
    t.cores = cores.data();
  }
};

// Workspace of the left-hand forms: [reversed input | reversed output | right-hand engine].
}  // namespace

int round_lrl_workspace(const tt_tensor *x, int prec, size_t *bytes) {
  Reversed xr(x, nullptr);
  size_t eng = 0;
  int st = round_workspace(&xr.t, prec, &eng);
  if (st) return st;
  *bytes = 2 * xr.bytes + eng;
  return TT_OK;
}

int round_lrl_run(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                  cudaStream_t st) {
  size_t need = 0;
  int r = round_lrl_workspace(x, prec, &need);
  if (r) return r;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *base = reinterpret_cast<unsigned char *>(ws);
  Reversed xr(x, base);
  Reversed yr(x, base + xr.bytes);  // output buffers of the reversed shapes (ranks never grow)
  r = reverse_cores(x->N, x->I, x->R, x->dtype, x->cores, xr.t.cores, st);
  if (r) return r;
  r = round_run(&xr.t, eps, prec, &yr.t, base + 2 * xr.bytes, ws_bytes - 2 * xr.bytes, st);
  if (r) return r;
  // yr.t.R holds the ranks of the reversed result; reverse it back into out
  const int N = x->N;
  std::vector<int64_t> Ry(N + 1);
  for (int n = 0; n <= N; ++n) Ry[n] = yr.t.R[n];
  r = reverse_cores(N, yr.I.data(), Ry.data(), x->dtype, yr.t.cores, out->cores, st);
  if (r) return r;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TT_ERR_CUDA;
  for (int n = 0; n <= N; ++n) out->R[n] = Ry[N - n];
  return TT_OK;
}

int orth_left_workspace(const tt_tensor *x, int prec, size_t *bytes) {
  Reversed xr(x, nullptr);
  size_t eng = 0;
  int st = orth_workspace(&xr.t, prec, &eng);
  if (st) return st;
  *bytes = 2 * xr.bytes + eng;
  return TT_OK;
}

int orth_left_enqueue(const tt_tensor *x, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st) {
  size_t need = 0;
  int r = orth_left_workspace(x, prec, &need);
  if (r) return r;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return TT_ERR_WORKSPACE;
  unsigned char *base = reinterpret_cast<unsigned char *>(ws);
  Reversed xr(x, base);
  Reversed yr(x, base + xr.bytes);
  r = reverse_cores(x->N, x->I, x->R, x->dtype, x->cores, xr.t.cores, st);
  if (r) return r;
  r = orth_enqueue(&xr.t, prec, &yr.t, base + 2 * xr.bytes, ws_bytes - 2 * xr.bytes, st);
  if (r) return r;
  const int N = x->N;
  std::vector<int64_t> Ry(N + 1);
  for (int n = 0; n <= N; ++n) Ry[n] = yr.t.R[n];
  r = reverse_cores(N, yr.I.data(), Ry.data(), x->dtype, yr.t.cores, out->cores, st);
  if (r) return r;
  for (int n = 0; n <= N; ++n) out->R[n] = Ry[N - n];
  return TT_OK;
}

}  // namespace ttgb
