// tt_engine.h -- host-side entry points shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "tt.h"

namespace ttgb {

// Plans are made for a context: a rounding on its own (kCtxSolo) or a member of a batch,
// whose roundings share the GPU with the other members (kCtxBatch).
constexpr int kCtxSolo = 0, kCtxBatch = 1;

int round_workspace(const tt_tensor *x, int prec, size_t *bytes, int ctx = kCtxSolo);
int round_run(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);
int round_enqueue(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                  cudaStream_t st, int *ranks_dev, int *status_dev, int ctx = kCtxSolo);

// ---- tile choices --------------------------------------------------------------------
// A core is planned from its shape class: precision, context, mode size and the ranks
// around it before (R0, R1) and after (K0, K1) the orthogonalization sweep.
struct TileKey {
  int prec = 0, ctx = 0;
  int64_t I = 0;
  int R0 = 0, R1 = 0, K0 = 0, K1 = 0;
  bool operator<(const TileKey &o) const;
  bool operator==(const TileKey &o) const;
};
// P = leaves (CTAs) over the mode, Tt = slices per leaf tile; 0 = the built-in heuristic.
struct TileChoice {
  int P = 0, Tt = 0;
};
// The choice for a key: the calling thread's trial choices while it is tuning, else the
// tuned table; false when neither has one.
bool tile_choice(const TileKey &k, TileChoice *c);
// Every core class of x under precision prec, with the heuristic's choice for each.
int tile_classes(const tt_tensor *x, int prec, int ctx, std::vector<TileKey> *keys,
                 std::vector<TileChoice> *heuristic, std::vector<int64_t> *elems);
int device_sm_count();
int norm_workspace(const tt_tensor *x, size_t *bytes);
int orth_workspace(const tt_tensor *x, int prec, size_t *bytes);
int orth_enqueue(const tt_tensor *x, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);
int orth_left_workspace(const tt_tensor *x, int prec, size_t *bytes);
int orth_left_enqueue(const tt_tensor *x, int prec, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);
int round_lrl_workspace(const tt_tensor *x, int prec, size_t *bytes);
int round_hadamard_run(const tt_tensor *a, const tt_tensor *b, const tt_tensor *z, double eps, int prec,
                       tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);
int round_lrl_run(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                  cudaStream_t st);
int norm_run(const tt_tensor *x, double *result, void *ws, size_t ws_bytes, cudaStream_t st);
int round_sharded_workspace(const tt_tensor *x, int prec, int world, int rank, const int64_t *Ig, size_t *bytes);
int round_sharded_run(const tt_tensor *x, double eps, int prec, const tt_shard *shard, int local_status,
                      uint64_t check, tt_tensor *out, void *ws, size_t ws_bytes, cudaStream_t st);

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
