// tt_engine.h -- host-side entry points shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "tt.h"

namespace ttgb {

int round_workspace(const tt_tensor *x, int prec, size_t *bytes);
int round_run(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);
int round_enqueue(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                  cudaStream_t st, int *ranks_dev, int *status_dev);
int norm_workspace(const tt_tensor *x, size_t *bytes);
int norm_run(const tt_tensor *x, double *result, void *ws, size_t ws_bytes, cudaStream_t st);

int add_run(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, cudaStream_t st);
int hadamard_run(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, cudaStream_t st);
int dot_workspace(const tt_tensor *a, const tt_tensor *b, size_t *bytes);
int dot_run(const tt_tensor *a, const tt_tensor *b, double *result, void *ws, size_t ws_bytes, cudaStream_t st);
int dot_noalloc_run(const tt_tensor *a, const tt_tensor *b, double *result, cudaStream_t st);

// Counts a launch of `kind` and, while tracing is on, brackets it with CUDA events on st.
struct TraceScope {
  TraceScope(int kind, cudaStream_t st);
  ~TraceScope();
  int kind;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

}  // namespace ttgb
