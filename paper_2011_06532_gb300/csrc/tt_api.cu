// tt_api.cu -- exported C ABI: argument validation and dispatch (see include/tt.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "tt.h"
#include "tt_engine.h"

namespace {

bool valid_tensor(const tt_tensor *x) {
  if (!x || x->N < 1 || !x->I || !x->R || !x->cores) return false;
  if (x->dtype != TT_F64 && x->dtype != TT_F32) return false;
  if (x->R[0] != 1 || x->R[x->N] != 1) return false;
  for (int n = 0; n < x->N; ++n) {
    if (x->I[n] < 1 || x->R[n] < 1 || !x->cores[n]) return false;
  }
  return true;
}

bool ranks_supported(const tt_tensor *x) {
  for (int n = 0; n <= x->N; ++n)
    if (x->R[n] > TT_MAX_RANK) return false;
  return true;
}

// out describes the same modes (N, dtype, I) with host arrays for R and cores
bool valid_out(const tt_tensor *x, const tt_tensor *out) {
  if (!out || out->N != x->N || out->dtype != x->dtype || !out->I || !out->R || !out->cores) return false;
  for (int n = 0; n < x->N; ++n)
    if (out->I[n] != x->I[n] || !out->cores[n]) return false;
  return true;
}

bool same_modes(const tt_tensor *a, const tt_tensor *b) {
  if (a->N != b->N || a->dtype != b->dtype) return false;
  for (int n = 0; n < a->N; ++n)
    if (a->I[n] != b->I[n]) return false;
  return true;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// resolves TT_PREC_DEFAULT and checks that the precision fits the element type; -1 if not
int resolve_prec(const tt_tensor *x, int prec) {
  if (prec == TT_PREC_DEFAULT) return x->dtype == TT_F64 ? TT_PREC_FP64 : TT_PREC_FP32X2;
  if (prec == TT_PREC_FP64) return x->dtype == TT_F64 ? prec : -1;
  if (prec == TT_PREC_FP32X2 || prec == TT_PREC_FP32) return x->dtype == TT_F32 ? prec : -1;
  return -1;
}

}  // namespace

namespace ttgb {

namespace {
struct TraceState {
  std::atomic<int64_t> launches[TT_K_COUNT];
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events[TT_K_COUNT];
};
TraceState &trace_state() {
  static TraceState s;
  return s;
}
}  // namespace

TraceScope::TraceScope(int k, cudaStream_t s) : kind(k), st(s) {
  TraceState &ts = trace_state();
  ts.launches[kind].fetch_add(1);
  if (ts.on.load()) {
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e0, st);
    } else {
      e0 = e1 = nullptr;
    }
  }
}

TraceScope::~TraceScope() {
  if (!e0 || !e1) return;
  cudaEventRecord(e1, st);
  TraceState &ts = trace_state();
  std::lock_guard<std::mutex> g(ts.mu);
  ts.events[kind].emplace_back(e0, e1);
}

}  // namespace ttgb

extern "C" {

int tt_trace(int enable) {
  ttgb::TraceState &ts = ttgb::trace_state();
  std::lock_guard<std::mutex> g(ts.mu);
  if (enable) {
    for (int k = 0; k < TT_K_COUNT; ++k) {
      ts.launches[k].store(0);
      for (auto &p : ts.events[k]) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
      }
      ts.events[k].clear();
    }
  }
  ts.on.store(enable != 0);
  return TT_OK;
}

int tt_trace_read(int kind, int64_t *launches, double *milliseconds) {
  if (kind < 0 || kind >= TT_K_COUNT) return TT_ERR_INVALID_ARG;
  ttgb::TraceState &ts = ttgb::trace_state();
  std::lock_guard<std::mutex> g(ts.mu);
  if (launches) *launches = ts.launches[kind].load();
  if (milliseconds) {
    double sum = 0.0;
    for (auto &p : ts.events[kind]) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.second) != cudaSuccess) return TT_ERR_CUDA;
      if (cudaEventElapsedTime(&ms, p.first, p.second) != cudaSuccess) return TT_ERR_CUDA;
      sum += ms;
    }
    *milliseconds = sum;
  }
  return TT_OK;
}

int tt_round_workspace_size(const tt_tensor *x, int precision, size_t *bytes) {
  if (!valid_tensor(x) || !bytes) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (x->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  return ttgb::round_workspace(x, prec, bytes);
}

int tt_round(const tt_tensor *x, double eps, int precision, tt_tensor *out, void *workspace, size_t workspace_bytes,
             void *stream) {
  if (!valid_tensor(x) || !valid_out(x, out) || !(eps >= 0.0) || !isfinite(eps)) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  return ttgb::round_run(x, eps, prec, out, workspace, workspace_bytes, as_stream(stream));
}

int tt_round_batched(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                     void *workspace, size_t workspace_bytes, void *stream) {
  if (count < 0 || (count > 0 && (!xs || !eps || !outs))) return TT_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k) {
    if (!valid_tensor(&xs[k]) || !valid_out(&xs[k], &outs[k]) || !(eps[k] >= 0.0) || !isfinite(eps[k]))
      return TT_ERR_INVALID_ARG;
    if (resolve_prec(&xs[k], precision) < 0) return TT_ERR_INVALID_ARG;
    if (!ranks_supported(&xs[k])) return TT_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < count; ++k) {
    const int st = ttgb::round_run(&xs[k], eps[k], resolve_prec(&xs[k], precision), &outs[k], workspace,
                                   workspace_bytes, as_stream(stream));
    if (st) return st;
  }
  return TT_OK;
}

int tt_add(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !valid_out(a, out)) return TT_ERR_INVALID_ARG;
  return ttgb::add_run(a, b, out, as_stream(stream));
}

int tt_hadamard(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !valid_out(a, out)) return TT_ERR_INVALID_ARG;
  return ttgb::hadamard_run(a, b, out, as_stream(stream));
}

int tt_dot_workspace_size(const tt_tensor *a, const tt_tensor *b, size_t *bytes) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !bytes) return TT_ERR_INVALID_ARG;
  return ttgb::dot_workspace(a, b, bytes);
}

int tt_dot(const tt_tensor *a, const tt_tensor *b, double *result, void *workspace, size_t workspace_bytes,
           void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !result) return TT_ERR_INVALID_ARG;
  return ttgb::dot_run(a, b, result, workspace, workspace_bytes, as_stream(stream));
}

int tt_dot_noalloc(const tt_tensor *a, const tt_tensor *b, double *result, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !result) return TT_ERR_INVALID_ARG;
  return ttgb::dot_noalloc_run(a, b, result, as_stream(stream));
}

int tt_norm_workspace_size(const tt_tensor *x, size_t *bytes) {
  if (!valid_tensor(x) || !bytes) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  return ttgb::norm_workspace(x, bytes);
}

int tt_norm(const tt_tensor *x, double *result, void *workspace, size_t workspace_bytes, void *stream) {
  if (!valid_tensor(x) || !result) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  return ttgb::norm_run(x, result, workspace, workspace_bytes, as_stream(stream));
}

const char *tt_status_string(int status) {
  switch (status) {
    case TT_OK: return "ok";
    case TT_ERR_INVALID_ARG: return "invalid argument";
    case TT_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case TT_ERR_CUDA: return "CUDA runtime error";
    case TT_ERR_NUMERICAL: return "non-finite values or SVD not converged";
    case TT_ERR_UNSUPPORTED: return "unsupported size (rank above the supported maximum)";
    default: return "unknown status";
  }
}

}  // extern "C"
