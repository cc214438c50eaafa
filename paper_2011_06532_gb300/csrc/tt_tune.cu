// tt_tune.cu -- the tile autotuner.  Each core of a rounding is cut into P leaves (CTAs)
// of consecutive slices, and each leaf walks its slab in tiles of Tt slices (Sec. 4.1:
// the leaves of the TSQR tree; Sec. 5.2 notes that the number of leaves per mode trades
// leaf work against tree depth).  The planner's built-in choice is P = 2 leaves per SM and
// the largest tile that lets two leaves share an SM.  The tuner replaces it, per core
// class (precision, context, I_n, ranks), by the fastest of a set of candidates measured
// with complete roundings on the GPU, and keeps the winners in a process-wide table that
// every later plan consults.  The table can be exported as text and imported again.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "tt.h"
#include "tt_engine.h"

namespace ttgb {

bool TileKey::operator<(const TileKey &o) const {
  return std::tie(prec, ctx, I, R0, R1, K0, K1) < std::tie(o.prec, o.ctx, o.I, o.R0, o.R1, o.K0, o.K1);
}
bool TileKey::operator==(const TileKey &o) const {
  return std::tie(prec, ctx, I, R0, R1, K0, K1) == std::tie(o.prec, o.ctx, o.I, o.R0, o.R1, o.K0, o.K1);
}

namespace {

std::mutex g_mu;
std::map<TileKey, TileChoice> g_table;
std::atomic<uint64_t> g_gen{1};

// While a thread tunes, its plans read only its trial map (keys absent from it take the
// heuristic), never the shared table.
thread_local std::map<TileKey, TileChoice> *t_trial = nullptr;

struct TrialScope {
  explicit TrialScope(std::map<TileKey, TileChoice> *m) { t_trial = m; }
  ~TrialScope() { t_trial = nullptr; }
};

constexpr int kTtFull = 1 << 20;  // "the largest tile that fits" (clamped by the planner)
constexpr float kGain = 0.98f;    // a candidate must beat the incumbent by 2 %

// candidate generators: leaves per core and tile rows
std::vector<int> leaf_options(const TileChoice &h, int64_t I, int nsm) {
  const int64_t cap = std::min<int64_t>(I, 1024);
  std::vector<int> v;
  for (int64_t p : {(int64_t)h.P, (int64_t)nsm / 2, (int64_t)nsm, 2 * (int64_t)nsm, 3 * (int64_t)nsm, 4 * (int64_t)nsm}) {
    const int q = (int)std::max<int64_t>(1, std::min<int64_t>(p, cap));
    if (std::find(v.begin(), v.end(), q) == v.end()) v.push_back(q);
  }
  return v;
}

std::vector<int> tile_options(const TileChoice &h) {
  std::vector<int> v{h.Tt};
  if (h.Tt / 2 >= 1 && h.Tt / 2 != h.Tt) v.push_back(h.Tt / 2);
  v.push_back(kTtFull);
  return v;
}

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Best of `reps` timings (ms) of fn() on st; returns a status through *status.
template <typename F>
float time_best(cudaStream_t st, int reps, F fn, int *status) {
  Events ev;
  float best = 3.4e38f;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(ev.a, st) != cudaSuccess) {
      *status = TT_ERR_CUDA;
      return best;
    }
    const int s = fn();
    if (s) {
      *status = s;
      return best;
    }
    float ms = 0.f;
    if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) {
      *status = TT_ERR_CUDA;
      return best;
    }
    best = std::min(best, ms);
  }
  *status = TT_OK;
  return best;
}

void store(const std::map<TileKey, TileChoice> &m) {
  std::lock_guard<std::mutex> g(g_mu);
  for (const auto &kv : m) g_table[kv.first] = kv.second;
  g_gen++;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

bool tile_choice(const TileKey &k, TileChoice *c) {
  if (t_trial) {
    auto it = t_trial->find(k);
    if (it == t_trial->end()) return false;
    *c = it->second;
    return true;
  }
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_table.find(k);
  if (it == g_table.end()) return false;
  *c = it->second;
  return true;
}

// ---- one rounding: coordinate descent over the core classes ---------------------------

static int solo_classes(const tt_tensor *x, int prec, std::vector<TileKey> *keys, std::vector<TileChoice> *heur,
                        std::vector<int64_t> *elems) {
  std::map<TileKey, TileChoice> none;
  TrialScope ts(&none);
  return tile_classes(x, prec, kCtxSolo, keys, heur, elems);
}

static int solo_workspace(const tt_tensor *x, int prec, size_t *bytes) {
  std::vector<TileKey> keys;
  std::vector<TileChoice> heur;
  std::vector<int64_t> elems;
  int st = solo_classes(x, prec, &keys, &heur, &elems);
  if (st) return st;
  const int nsm = device_sm_count();
  size_t mx = 0;
  // every leaf generator with every tile generator, applied to all classes at once
  for (int pi = 0; pi < 6; ++pi) {
    for (int ti = 0; ti < 3; ++ti) {
      std::map<TileKey, TileChoice> trial;
      for (size_t k = 0; k < keys.size(); ++k) {
        const std::vector<int> ps = leaf_options(heur[k], keys[k].I, nsm);
        const std::vector<int> tts = tile_options(heur[k]);
        trial[keys[k]] = TileChoice{ps[std::min<size_t>(pi, ps.size() - 1)], tts[std::min<size_t>(ti, tts.size() - 1)]};
      }
      TrialScope ts(&trial);
      size_t b = 0;
      st = round_workspace(x, prec, &b);
      if (st) return st;
      mx = std::max(mx, b);
    }
  }
  *bytes = mx;
  return TT_OK;
}

static int autotune_solo(const tt_tensor *x, double eps, int prec, tt_tensor *out, void *ws, size_t ws_bytes,
                         cudaStream_t st) {
  std::vector<TileKey> keys;
  std::vector<TileChoice> heur;
  std::vector<int64_t> elems;
  int r = solo_classes(x, prec, &keys, &heur, &elems);
  if (r) return r;
  if (keys.empty()) return TT_OK;
  const int nsm = device_sm_count();
  std::vector<size_t> order(keys.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return elems[a] > elems[b]; });
  std::map<TileKey, TileChoice> trial;
  for (size_t k = 0; k < keys.size(); ++k) trial[keys[k]] = heur[k];
  TrialScope ts(&trial);
  auto run = [&]() { return round_run(x, eps, prec, out, ws, ws_bytes, st); };
  r = run();  // warm-up (and the heuristic must work)
  if (r) return r;
  float best = time_best(st, 2, run, &r);
  if (r) return r;
  for (size_t k : order) {
    TileChoice keep = trial[keys[k]];
    for (int P : leaf_options(heur[k], keys[k].I, nsm)) {
      for (int Tt : tile_options(heur[k])) {
        const TileChoice cand{P, Tt};
        if (cand.P == keep.P && cand.Tt == keep.Tt) continue;
        trial[keys[k]] = cand;
        size_t need = 0;
        if (round_workspace(x, prec, &need) != TT_OK || need > ws_bytes) continue;
        const float t = time_best(st, 2, run, &r);
        if (r == TT_ERR_CUDA) return r;
        if (r) continue;  // this candidate does not plan or run: keep the incumbent
        if (t < kGain * best) {
          best = t;
          keep = cand;
        }
      }
    }
    trial[keys[k]] = keep;
  }
  store(trial);
  return TT_OK;
}

// ---- a batch: one leaf cap and tile rule for all members ------------------------------

namespace {

struct BatchClasses {
  std::vector<TileKey> keys;
  std::vector<TileChoice> heur;
};

int batch_classes(int32_t count, const tt_tensor *xs, int precision, BatchClasses *bc) {
  std::map<TileKey, TileChoice> none;
  TrialScope ts(&none);
  for (int k = 0; k < count; ++k) {
    const int prec = precision == TT_PREC_DEFAULT ? (xs[k].dtype == TT_F64 ? TT_PREC_FP64 : TT_PREC_FP32X2) : precision;
    std::vector<TileKey> keys;
    std::vector<TileChoice> heur;
    std::vector<int64_t> elems;
    const int st = tile_classes(&xs[k], prec, kCtxBatch, &keys, &heur, &elems);
    if (st) return st;
    for (size_t i = 0; i < keys.size(); ++i) {
      if (std::find(bc->keys.begin(), bc->keys.end(), keys[i]) == bc->keys.end()) {
        bc->keys.push_back(keys[i]);
        bc->heur.push_back(heur[i]);
      }
    }
  }
  return TT_OK;
}

// policy p: leaf cap (4, 2, 1, 1/2, 1/4, 1/8, 1/16 leaves per SM) x tile rule (heuristic, full)
constexpr int kCaps = 7, kTileRules = 2;

std::map<TileKey, TileChoice> batch_policy(const BatchClasses &bc, int cap_i, int tile_i, int nsm) {
  static const double per_sm[kCaps] = {4.0, 2.0, 1.0, 0.5, 0.25, 0.125, 0.0625};
  const int64_t cap = std::max<int64_t>(1, (int64_t)(per_sm[cap_i] * nsm));
  std::map<TileKey, TileChoice> m;
  for (size_t i = 0; i < bc.keys.size(); ++i) {
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>({cap, bc.keys[i].I, 1024}));
    m[bc.keys[i]] = TileChoice{P, tile_i == 0 ? 0 : kTtFull};
  }
  return m;
}

}  // namespace

static int batch_tune_workspace(int32_t count, const tt_tensor *xs, int precision, size_t *bytes) {
  BatchClasses bc;
  int st = batch_classes(count, xs, precision, &bc);
  if (st) return st;
  const int nsm = device_sm_count();
  size_t mx = 0;
  for (int c = 0; c < kCaps; ++c) {
    for (int t = 0; t < kTileRules; ++t) {
      std::map<TileKey, TileChoice> trial = batch_policy(bc, c, t, nsm);
      TrialScope ts(&trial);
      size_t b = 0;
      st = tt_round_batched_workspace_size(count, xs, precision, &b);
      if (st) return st;
      mx = std::max(mx, b);
    }
  }
  *bytes = mx;
  return TT_OK;
}

static int autotune_batch(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                          void *ws, size_t ws_bytes, cudaStream_t st) {
  BatchClasses bc;
  int r = batch_classes(count, xs, precision, &bc);
  if (r) return r;
  if (bc.keys.empty()) return TT_OK;
  const int nsm = device_sm_count();
  // one timed batch per policy (the caller's own run has warmed up the kernels): every
  // leaf cap with the default tile rule, then the other tile rule at the best cap
  auto try_policy = [&](int c, int t, float *ms) -> int {
    std::map<TileKey, TileChoice> trial = batch_policy(bc, c, t, nsm);
    TrialScope ts(&trial);
    size_t need = 0;
    if (tt_round_batched_workspace_size(count, xs, precision, &need) != TT_OK || need > ws_bytes) return TT_ERR_WORKSPACE;
    int s = TT_OK;
    *ms = time_best(st, 1, [&]() { return tt_round_batched(count, xs, eps, precision, outs, ws, ws_bytes, st); }, &s);
    return s;
  };
  float best = 3.4e38f;
  int best_c = -1, best_t = 0;
  for (int c = 0; c < kCaps; ++c) {
    float ms = 0.f;
    r = try_policy(c, 0, &ms);
    if (r == TT_ERR_CUDA) return r;
    if (r == TT_OK && ms < best) {
      best = ms;
      best_c = c;
    }
  }
  if (best_c < 0) return TT_ERR_WORKSPACE;
  for (int t = 1; t < kTileRules; ++t) {
    float ms = 0.f;
    r = try_policy(best_c, t, &ms);
    if (r == TT_ERR_CUDA) return r;
    if (r == TT_OK && ms < kGain * best) {
      best = ms;
      best_t = t;
    }
  }
  store(batch_policy(bc, best_c, best_t, nsm));
  return TT_OK;
}

}  // namespace ttgb

// ---- C ABI ---------------------------------------------------------------------------

extern "C" {

// argument checks shared with tt_api.cu through the public entry points: the tuner calls
// tt_round_workspace_size first, which validates x and the precision
int tt_autotune_workspace_size(const tt_tensor *x, int precision, size_t *bytes) {
  if (!x || !bytes) return TT_ERR_INVALID_ARG;
  size_t b = 0;
  int st = tt_round_workspace_size(x, precision, &b);
  if (st) return st;
  if (x->N < 2) {
    *bytes = b;
    return TT_OK;
  }
  const int prec = precision == TT_PREC_DEFAULT ? (x->dtype == TT_F64 ? TT_PREC_FP64 : TT_PREC_FP32X2) : precision;
  return ttgb::solo_workspace(x, prec, bytes);
}

int tt_autotune(const tt_tensor *x, double eps, int precision, tt_tensor *out, void *workspace,
                size_t workspace_bytes, void *stream) {
  size_t need = 0;
  int st = tt_autotune_workspace_size(x, precision, &need);
  if (st) return st;
  if (workspace && workspace_bytes >= need && !(reinterpret_cast<uintptr_t>(workspace) & 255)) need = 0;
  // one rounding with the current plan validates every argument the way tt_round does
  st = tt_round(x, eps, precision, out, workspace, workspace_bytes, stream);
  if (st) return st;
  if (x->N < 2) return TT_OK;
  if (need) return TT_ERR_WORKSPACE;
  const int prec = precision == TT_PREC_DEFAULT ? (x->dtype == TT_F64 ? TT_PREC_FP64 : TT_PREC_FP32X2) : precision;
  return ttgb::autotune_solo(x, eps, prec, out, workspace, workspace_bytes, ttgb::as_stream(stream));
}

int tt_autotune_batched_workspace_size(int32_t count, const tt_tensor *xs, int precision, size_t *bytes) {
  if (!bytes) return TT_ERR_INVALID_ARG;
  size_t b = 0;
  int st = tt_round_batched_workspace_size(count, xs, precision, &b);
  if (st) return st;
  return ttgb::batch_tune_workspace(count, xs, precision, bytes);
}

int tt_autotune_batched(int32_t count, const tt_tensor *xs, const double *eps, int precision, tt_tensor *outs,
                        void *workspace, size_t workspace_bytes, void *stream) {
  size_t need = 0;
  int st = tt_autotune_batched_workspace_size(count, xs, precision, &need);
  if (st) return st;
  if (count == 0) return TT_OK;
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return TT_ERR_WORKSPACE;
  st = tt_round_batched(count, xs, eps, precision, outs, workspace, workspace_bytes, stream);
  if (st) return st;
  return ttgb::autotune_batch(count, xs, eps, precision, outs, workspace, workspace_bytes, ttgb::as_stream(stream));
}

int tt_tune_export(char *buf, size_t capacity, size_t *length) {
  if (!length) return TT_ERR_INVALID_ARG;
  std::ostringstream os;
  os << "# ttgb tile table v1: prec ctx I R0 R1 K0 K1 P Tt\n";
  {
    std::lock_guard<std::mutex> g(ttgb::g_mu);
    for (const auto &kv : ttgb::g_table) {
      const ttgb::TileKey &k = kv.first;
      os << k.prec << ' ' << k.ctx << ' ' << k.I << ' ' << k.R0 << ' ' << k.R1 << ' ' << k.K0 << ' ' << k.K1 << ' '
         << kv.second.P << ' ' << kv.second.Tt << '\n';
    }
  }
  const std::string s = os.str();
  *length = s.size() + 1;
  if (!buf) return TT_OK;
  if (capacity < s.size() + 1) return TT_ERR_WORKSPACE;
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return TT_OK;
}

int tt_tune_import(const char *text) {
  if (!text) return TT_ERR_INVALID_ARG;
  std::map<ttgb::TileKey, ttgb::TileChoice> m;
  std::istringstream is(text);
  std::string line;
  while (std::getline(is, line)) {
    const size_t first = line.find_first_not_of(" \t\r");
    if (first == std::string::npos || line[first] == '#') continue;
    std::istringstream ls(line);
    long long v[9];
    for (int i = 0; i < 9; ++i)
      if (!(ls >> v[i])) return TT_ERR_INVALID_ARG;
    std::string rest;
    if (ls >> rest) return TT_ERR_INVALID_ARG;
    const bool ok = v[0] >= TT_PREC_FP64 && v[0] <= TT_PREC_FP32 && (v[1] == 0 || v[1] == 1) && v[2] >= 1 &&
                    v[3] >= 1 && v[3] <= TT_MAX_RANK && v[4] >= 1 && v[4] <= TT_MAX_RANK && v[5] >= 1 &&
                    v[5] <= v[3] && v[6] >= 1 && v[6] <= v[4] && v[7] >= 0 && v[7] <= 1024 && v[8] >= 0 &&
                    v[8] <= (1 << 20);
    if (!ok) return TT_ERR_INVALID_ARG;
    ttgb::TileKey k;
    k.prec = (int)v[0];
    k.ctx = (int)v[1];
    k.I = v[2];
    k.R0 = (int)v[3];
    k.R1 = (int)v[4];
    k.K0 = (int)v[5];
    k.K1 = (int)v[6];
    m[k] = ttgb::TileChoice{(int)v[7], (int)v[8]};
  }
  ttgb::store(m);
  return TT_OK;
}

int tt_tune_clear(void) {
  std::lock_guard<std::mutex> g(ttgb::g_mu);
  ttgb::g_table.clear();
  ttgb::g_gen++;
  return TT_OK;
}

uint64_t tt_tune_generation(void) { return ttgb::g_gen.load(); }

}  // extern "C"
