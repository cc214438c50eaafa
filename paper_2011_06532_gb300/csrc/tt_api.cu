// tt_api.cu -- exported C ABI: argument validation and dispatch (see include/tt.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
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

// Whether the current device can dereference p at that same address: memory of this
// device, managed memory, or page-locked host memory mapped into the device's address
// space (cudaHostAlloc / cudaHostRegister under unified addressing), which kernels read
// and write over the host link.  Unregistered host memory is refused.
bool device_accessible(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == dev;
    case cudaMemoryTypeManaged: return true;
    case cudaMemoryTypeHost: return at.devicePointer == p;
    default: return false;
  }
}

bool cores_accessible(const tt_tensor *x) {
  for (int n = 0; n < x->N; ++n)
    if (!device_accessible(x->cores[n])) return false;
  return true;
}

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
  if (!cores_accessible(x) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  return ttgb::round_run(x, eps, prec, out, workspace, workspace_bytes, as_stream(stream));
}

int tt_round_ordered_workspace_size(const tt_tensor *x, int precision, int order, size_t *bytes) {
  if (order == TT_ORDER_RLR) return tt_round_workspace_size(x, precision, bytes);
  if (order != TT_ORDER_LRL || !valid_tensor(x) || !bytes) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (x->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  return ttgb::round_lrl_workspace(x, prec, bytes);
}

int tt_round_ordered(const tt_tensor *x, double eps, int precision, int order, tt_tensor *out, void *workspace,
                     size_t workspace_bytes, void *stream) {
  if (order == TT_ORDER_RLR) return tt_round(x, eps, precision, out, workspace, workspace_bytes, stream);
  if (order != TT_ORDER_LRL) return TT_ERR_INVALID_ARG;
  if (!valid_tensor(x) || !valid_out(x, out) || !(eps >= 0.0) || !isfinite(eps)) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (!cores_accessible(x) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  if (x->N == 1) return ttgb::round_run(x, eps, prec, out, workspace, workspace_bytes, as_stream(stream));
  return ttgb::round_lrl_run(x, eps, prec, out, workspace, workspace_bytes, as_stream(stream));
}

namespace {
constexpr int kMaxShards = 1024;

// first slice of shard p of W over a mode of size I (the leaf partition of the kernels)
int64_t shard_begin(int64_t I, int W, int p) { return (int64_t)p * I / W; }
int64_t shard_len(int64_t I, int W, int p) { return shard_begin(I, W, p + 1) - shard_begin(I, W, p); }

bool valid_shard(const tt_shard *s) {
  return s && s->allgather && s->I_global && s->world_size >= 1 && s->world_size <= kMaxShards && s->rank >= 0 &&
         s->rank < s->world_size;
}

// FNV-1a digest of the arguments every shard must share.
struct Digest {
  uint64_t h = 1469598103934665603ull;
  void add(const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  }
};

// This shard's own argument checks (0 if fine) and the digest of the shared ones.
int shard_checks(const tt_tensor *x, double eps, int precision, const tt_shard *s, const tt_tensor *out, int *prec,
                 uint64_t *check) {
  *check = 0;
  *prec = -1;
  if (!valid_tensor(x)) return TT_ERR_INVALID_ARG;
  Digest d;
  d.add(&x->N, sizeof x->N);
  d.add(&x->dtype, sizeof x->dtype);
  d.add(&precision, sizeof precision);
  d.add(&eps, sizeof eps);
  d.add(&s->world_size, sizeof s->world_size);
  d.add(s->I_global, sizeof(int64_t) * x->N);
  d.add(x->R, sizeof(int64_t) * (x->N + 1));
  *check = d.h;
  for (int n = 0; n < x->N; ++n) {
    if (s->I_global[n] < s->world_size) return TT_ERR_INVALID_ARG;
    if (x->I[n] != shard_len(s->I_global[n], s->world_size, s->rank)) return TT_ERR_INVALID_ARG;
  }
  if (!valid_out(x, out) || !(eps >= 0.0) || !isfinite(eps)) return TT_ERR_INVALID_ARG;
  *prec = resolve_prec(x, precision);
  if (*prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (!cores_accessible(x) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  return TT_OK;
}
}  // namespace

int tt_shard_range(int64_t I, int32_t world_size, int32_t rank, int64_t *begin, int64_t *end) {
  if (!begin || !end || world_size < 1 || world_size > kMaxShards || I < world_size || rank < 0 || rank >= world_size)
    return TT_ERR_INVALID_ARG;
  *begin = shard_begin(I, world_size, rank);
  *end = shard_begin(I, world_size, rank + 1);
  return TT_OK;
}

int tt_round_sharded_workspace_size(const tt_tensor *x, int precision, const tt_shard *shard, size_t *bytes) {
  if (!valid_tensor(x) || !bytes || !valid_shard(shard)) return TT_ERR_INVALID_ARG;
  if (shard->world_size == 1) return tt_round_workspace_size(x, precision, bytes);
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  for (int n = 0; n < x->N; ++n)
    if (shard->I_global[n] < shard->world_size ||
        x->I[n] != shard_len(shard->I_global[n], shard->world_size, shard->rank))
      return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  return ttgb::round_sharded_workspace(x, prec, shard->world_size, shard->rank, shard->I_global, bytes);
}

int tt_round_sharded(const tt_tensor *x, double eps, int precision, const tt_shard *shard, tt_tensor *out,
                     void *workspace, size_t workspace_bytes, void *stream) {
  if (!valid_shard(shard)) return TT_ERR_INVALID_ARG;
  if (shard->world_size == 1) {
    if (!valid_tensor(x)) return TT_ERR_INVALID_ARG;
    for (int n = 0; n < x->N; ++n)
      if (shard->I_global[n] != x->I[n]) return TT_ERR_INVALID_ARG;
    return tt_round(x, eps, precision, out, workspace, workspace_bytes, stream);
  }
  int prec = -1;
  uint64_t check = 0;
  const int local = shard_checks(x, eps, precision, shard, out, &prec, &check);
  return ttgb::round_sharded_run(x, eps, prec, shard, local, check, out, workspace, workspace_bytes, as_stream(stream));
}

namespace {
// Shape of the Hadamard product of a and b (ranks multiply), cores unset.
struct ProductShape {
  std::vector<int64_t> R;
  std::vector<void *> cores;
  tt_tensor t{};
  ProductShape(const tt_tensor *a, const tt_tensor *b) {
    R.resize(a->N + 1);
    cores.assign(a->N, nullptr);
    for (int n = 0; n <= a->N; ++n) R[n] = a->R[n] * b->R[n];
    t.N = a->N;
    t.dtype = a->dtype;
    t.I = a->I;
    t.R = R.data();
    t.cores = cores.data();
  }
};
}  // namespace

int tt_round_hadamard_workspace_size(const tt_tensor *a, const tt_tensor *b, int precision, size_t *bytes) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !bytes) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(a, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  ProductShape z(a, b);
  if (!ranks_supported(&z.t)) return TT_ERR_UNSUPPORTED;
  if (a->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  return ttgb::round_workspace(&z.t, prec, bytes);
}

int tt_round_hadamard(const tt_tensor *a, const tt_tensor *b, double eps, int precision, tt_tensor *out,
                      void *workspace, size_t workspace_bytes, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !valid_out(a, out) || !(eps >= 0.0) ||
      !isfinite(eps))
    return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(a, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  ProductShape z(a, b);
  if (!ranks_supported(&z.t)) return TT_ERR_UNSUPPORTED;
  if (!cores_accessible(a) || !cores_accessible(b) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  if (a->N == 1) {
    // a single core: the rounding is a copy of the entrywise product
    int st = ttgb::hadamard_run(a, b, out, as_stream(stream));
    if (st) return st;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return TT_ERR_CUDA;
    out->R[0] = out->R[1] = 1;
    return TT_OK;
  }
  return ttgb::round_hadamard_run(a, b, &z.t, eps, prec, out, workspace, workspace_bytes, as_stream(stream));
}

int tt_orthonormalize_workspace_size(const tt_tensor *x, int precision, int side, size_t *bytes) {
  if (!valid_tensor(x) || !bytes || (side != TT_ORTH_RIGHT && side != TT_ORTH_LEFT)) return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (x->N == 1) {
    *bytes = 0;
    return TT_OK;
  }
  return side == TT_ORTH_RIGHT ? ttgb::orth_workspace(x, prec, bytes) : ttgb::orth_left_workspace(x, prec, bytes);
}

int tt_orthonormalize(const tt_tensor *x, int precision, int side, tt_tensor *out, void *workspace,
                      size_t workspace_bytes, void *stream) {
  if (!valid_tensor(x) || !valid_out(x, out) || (side != TT_ORTH_RIGHT && side != TT_ORTH_LEFT))
    return TT_ERR_INVALID_ARG;
  const int prec = resolve_prec(x, precision);
  if (prec < 0) return TT_ERR_INVALID_ARG;
  if (!ranks_supported(x)) return TT_ERR_UNSUPPORTED;
  if (!cores_accessible(x) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  if (x->N == 1 || side == TT_ORTH_RIGHT)
    return ttgb::orth_enqueue(x, prec, out, workspace, workspace_bytes, as_stream(stream));
  return ttgb::orth_left_enqueue(x, prec, out, workspace, workspace_bytes, as_stream(stream));
}

namespace {

struct BatchStreams {
  bool ready = false;
  cudaStream_t s[TT_BATCH_SLOTS];
  cudaEvent_t fork;
  cudaEvent_t join[TT_BATCH_SLOTS];
};
constexpr int kMaxDevices = 64;
std::mutex g_batch_mu;
BatchStreams g_batch[kMaxDevices];

int batch_streams(BatchStreams **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_batch_mu);
  BatchStreams &b = g_batch[dev];
  if (!b.ready) {
    for (int k = 0; k < TT_BATCH_SLOTS; ++k) {
      if (cudaStreamCreateWithFlags(&b.s[k], cudaStreamNonBlocking) != cudaSuccess) return TT_ERR_CUDA;
      if (cudaEventCreateWithFlags(&b.join[k], cudaEventDisableTiming) != cudaSuccess) return TT_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess) return TT_ERR_CUDA;
    b.ready = true;
  }
  *out = &b;
  return TT_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct BatchLayout {
  int slots = 0;
  size_t slot_bytes = 0, ranks_off = 0, status_off = 0, total = 0;
};

int batch_layout(int32_t count, const tt_tensor *xs, int precision, BatchLayout *lay) {
  size_t mx = 0, nranks = 0;
  for (int k = 0; k < count; ++k) {
    const int prec = resolve_prec(&xs[k], precision);
    if (prec < 0) return TT_ERR_INVALID_ARG;
    size_t b = 0;
    if (xs[k].N > 1) {
      const int st = ttgb::round_workspace(&xs[k], prec, &b, ttgb::kCtxBatch);
      if (st) return st;
    }
    mx = b > mx ? b : mx;
    nranks += (size_t)xs[k].N + 1;
  }
  lay->slots = count < TT_BATCH_SLOTS ? count : TT_BATCH_SLOTS;
  lay->slot_bytes = align256(mx ? mx : 256);
  lay->ranks_off = lay->slot_bytes * lay->slots;
  lay->status_off = lay->ranks_off + align256(sizeof(int32_t) * (nranks ? nranks : 1));
  lay->total = lay->status_off + align256(sizeof(int32_t) * (count ? count : 1));
  return TT_OK;
}

int check_batch(int32_t count, const tt_tensor *xs, const double *eps, tt_tensor *outs, int precision) {
  if (count < 0 || (count > 0 && (!xs || !eps || !outs))) return TT_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k) {
    if (!valid_tensor(&xs[k]) || !valid_out(&xs[k], &outs[k]) || !(eps[k] >= 0.0) || !isfinite(eps[k]))
      return TT_ERR_INVALID_ARG;
    if (resolve_prec(&xs[k], precision) < 0) return TT_ERR_INVALID_ARG;
    if (!ranks_supported(&xs[k])) return TT_ERR_UNSUPPORTED;
    if (!cores_accessible(&xs[k]) || !cores_accessible(&outs[k])) return TT_ERR_INVALID_ARG;
  }
  return TT_OK;
}

int batch_enqueue(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                  int32_t *ranks_dev, int32_t *status_dev, unsigned char *ws, const BatchLayout &lay,
                  cudaStream_t stream) {
  if (count == 0) return TT_OK;
  BatchStreams *bs = nullptr;
  int st = batch_streams(&bs);
  if (st) return st;
  if (cudaEventRecord(bs->fork, stream) != cudaSuccess) return TT_ERR_CUDA;
  for (int s = 0; s < lay.slots; ++s)
    if (cudaStreamWaitEvent(bs->s[s], bs->fork, 0) != cudaSuccess) return TT_ERR_CUDA;
  // Members go to the internal streams largest first, each to the stream with the least
  // work queued so far (longest-processing-time rule), so that one stream does not end
  // up with several of the largest members.  Work ~ sum_n R_{n-1} I_n R_n max(R_{n-1}, R_n).
  std::vector<size_t> roff(count);
  std::vector<double> cost(count);
  std::vector<int> order(count);
  size_t acc = 0;
  for (int k = 0; k < count; ++k) {
    roff[k] = acc;
    acc += (size_t)xs[k].N + 1;
    double c = 0.0;
    for (int n = 0; n < xs[k].N; ++n)
      c += (double)xs[k].R[n] * (double)xs[k].I[n] * (double)xs[k].R[n + 1] *
           (double)std::max(xs[k].R[n], xs[k].R[n + 1]);
    cost[k] = c;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(lay.slots, 0.0);
  for (int k : order) {
    const int slot = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[slot] += cost[k];
    st = ttgb::round_enqueue(&xs[k], eps[k], resolve_prec(&xs[k], precision), &outs[k],
                             ws + (size_t)slot * lay.slot_bytes, lay.slot_bytes, bs->s[slot], ranks_dev + roff[k],
                             status_dev + k, ttgb::kCtxBatch);
    if (st) return st;
  }
  for (int s = 0; s < lay.slots; ++s) {
    if (cudaEventRecord(bs->join[s], bs->s[s]) != cudaSuccess) return TT_ERR_CUDA;
    if (cudaStreamWaitEvent(stream, bs->join[s], 0) != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}

}  // namespace

int tt_round_batched_workspace_size(int32_t count, const tt_tensor *xs, int precision, size_t *bytes) {
  if (count < 0 || (count > 0 && !xs) || !bytes) return TT_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k) {
    if (!valid_tensor(&xs[k])) return TT_ERR_INVALID_ARG;
    if (!ranks_supported(&xs[k])) return TT_ERR_UNSUPPORTED;
  }
  BatchLayout lay;
  const int st = batch_layout(count, xs, precision, &lay);
  if (st) return st;
  *bytes = lay.total;
  return TT_OK;
}

int tt_round_batched_async(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                           int32_t *ranks_dev, int32_t *status_dev, void *workspace, size_t workspace_bytes,
                           void *stream) {
  int st = check_batch(count, xs, eps, outs, precision);
  if (st) return st;
  if (count > 0 && (!ranks_dev || !status_dev)) return TT_ERR_INVALID_ARG;
  BatchLayout lay;
  st = batch_layout(count, xs, precision, &lay);
  if (st) return st;
  if (count > 0 && (!workspace || workspace_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255)))
    return TT_ERR_WORKSPACE;
  return batch_enqueue(count, xs, eps, precision, outs, ranks_dev, status_dev,
                       reinterpret_cast<unsigned char *>(workspace), lay, as_stream(stream));
}

int tt_round_batched(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                     void *workspace, size_t workspace_bytes, void *stream) {
  int st = check_batch(count, xs, eps, outs, precision);
  if (st) return st;
  if (count == 0) return TT_OK;
  BatchLayout lay;
  st = batch_layout(count, xs, precision, &lay);
  if (st) return st;
  if (!workspace || workspace_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return TT_ERR_WORKSPACE;
  unsigned char *ws = reinterpret_cast<unsigned char *>(workspace);
  int32_t *ranks_dev = reinterpret_cast<int32_t *>(ws + lay.ranks_off);
  int32_t *status_dev = reinterpret_cast<int32_t *>(ws + lay.status_off);
  cudaStream_t s = as_stream(stream);
  st = batch_enqueue(count, xs, eps, precision, outs, ranks_dev, status_dev, ws, lay, s);
  if (st) return st;
  size_t nranks = 0;
  for (int k = 0; k < count; ++k) nranks += (size_t)xs[k].N + 1;
  std::vector<int32_t> ranks(nranks), status(count);
  if (cudaMemcpyAsync(ranks.data(), ranks_dev, sizeof(int32_t) * nranks, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TT_ERR_CUDA;
  if (cudaMemcpyAsync(status.data(), status_dev, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TT_ERR_CUDA;
  size_t roff = 0;
  for (int k = 0; k < count; ++k) {
    if (status[k]) return status[k];
    for (int n = 0; n <= xs[k].N; ++n) outs[k].R[n] = ranks[roff + n];
    roff += (size_t)xs[k].N + 1;
  }
  return TT_OK;
}

int tt_add(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !valid_out(a, out)) return TT_ERR_INVALID_ARG;
  if (!cores_accessible(a) || !cores_accessible(b) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  return ttgb::add_run(a, b, out, as_stream(stream));
}

int tt_hadamard(const tt_tensor *a, const tt_tensor *b, tt_tensor *out, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !valid_out(a, out)) return TT_ERR_INVALID_ARG;
  if (!cores_accessible(a) || !cores_accessible(b) || !cores_accessible(out)) return TT_ERR_INVALID_ARG;
  return ttgb::hadamard_run(a, b, out, as_stream(stream));
}

int tt_dot_workspace_size(const tt_tensor *a, const tt_tensor *b, size_t *bytes) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !bytes) return TT_ERR_INVALID_ARG;
  return ttgb::dot_workspace(a, b, bytes);
}

int tt_dot(const tt_tensor *a, const tt_tensor *b, double *result, void *workspace, size_t workspace_bytes,
           void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !result) return TT_ERR_INVALID_ARG;
  if (!cores_accessible(a) || !cores_accessible(b)) return TT_ERR_INVALID_ARG;
  return ttgb::dot_run(a, b, result, workspace, workspace_bytes, as_stream(stream));
}

int tt_dot_noalloc(const tt_tensor *a, const tt_tensor *b, double *result, void *stream) {
  if (!valid_tensor(a) || !valid_tensor(b) || !same_modes(a, b) || !result) return TT_ERR_INVALID_ARG;
  if (!cores_accessible(a) || !cores_accessible(b)) return TT_ERR_INVALID_ARG;
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
  if (!cores_accessible(x)) return TT_ERR_INVALID_ARG;
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
    case TT_ERR_COMM: return "the all-gather of a sharded call failed";
    default: return "unknown status";
  }
}

}  // extern "C"
