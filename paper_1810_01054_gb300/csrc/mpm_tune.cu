// Launch-shape autotuner of the tile kernels: candidate tables, the process-wide cache (with its
// optional text file), per-scene trials, and the C-ABI entry points; the cache also keeps the tile
// edge that mpm_tune_tile_edge measured fastest for a 2D workload.
//
// A trial step is an ordinary simulation step: the tile kernels process every tile whole inside
// one CTA, so neither the number of CTAs nor (for G2P, whose outputs are per particle) the CTA
// size changes a single bit of the results.  The adjoint gather's group sums are formed per warp
// and then per CTA, so its CTA size would change their rounding: it is fixed per dimension and
// only its CTAs per SM are tuned.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "mpm_scene.h"

#define CK(expr)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA; \
  } while (0)
#define CKS(expr)                \
  do {                           \
    mpm_status s_ = (expr);      \
    if (s_ != MPM_OK) return s_; \
  } while (0)

namespace gbmpm {
namespace {

constexpr int kReps = 2;  // timed launches per candidate; the faster one counts

// P2G and the adjoint scatter take 128-thread CTAs in 2D only (a 3D work item is 9 nodes)
const TileLaunch kCandP2G3[] = {{2, 256}, {3, 256}, {4, 256}, {6, 256}, {8, 256}};
const TileLaunch kCandP2G2[] = {{2, 256}, {3, 256}, {4, 256}, {6, 256}, {8, 256}, {4, 128}, {6, 128}};
const TileLaunch kCandG2P[] = {{2, 256}, {3, 256}, {4, 256}, {8, 256}, {16, 256}, {6, 128}, {8, 128}, {16, 128}};
const TileLaunch kCandAdj[] = {{2, 256}, {3, 256}, {4, 256}, {6, 256}, {8, 256}};

struct CandList {
  const TileLaunch* c;
  int n;
};

CandList cands(int k, int dim) {
  switch (k) {
    case TK_P2G:
    case TK_P2G_ADJ:
      if (dim == 2) return {kCandP2G2, int(sizeof(kCandP2G2) / sizeof(kCandP2G2[0]))};
      return {kCandP2G3, int(sizeof(kCandP2G3) / sizeof(kCandP2G3[0]))};
    case TK_G2P:
      return {kCandG2P, int(sizeof(kCandG2P) / sizeof(kCandG2P[0]))};
    default:
      return {kCandAdj, int(sizeof(kCandAdj) / sizeof(kCandAdj[0]))};
  }
}

bool is_candidate(int k, int dim, TileLaunch t) {
  const CandList l = cands(k, dim);
  for (int i = 0; i < l.n; ++i)
    if (l.c[i].ctas_per_sm == t.ctas_per_sm && l.c[i].threads == t.threads) return true;
  return false;
}

int log2_bucket(long long v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

using Key = std::tuple<int, int, int, int>;  // dim, log2 particles, log2 grid tiles, SMs
struct Entry {
  TileLaunch l[TK_COUNT];
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;
// keys whose entry came from batch trials that tuned only some kernels: bit k = kernel k tuned
// (absent: every kernel of the entry is tuned)
std::map<Key, unsigned> g_partial;
bool g_env_loaded = false;
// tile edge per workload key (dim, log2 particles, log2 grid nodes, SMs), from mpm_tune_tile_edge
std::map<Key, int> g_edge;

Key make_key(int dim, long long particles, long long tiles, int sms) {
  return Key(dim, log2_bucket(particles < 1 ? 1 : particles), log2_bucket(tiles < 1 ? 1 : tiles), sms);
}

// Caller holds g_mu.
mpm_status load_locked(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return MPM_ERR_ARG;
  char head[512] = {0};
  if (!std::fgets(head, sizeof(head), f) || std::string(head).rfind("gbmpm-tune 1", 0) != 0 ||
      std::string(head).find('\n') == std::string::npos) {
    std::fclose(f);
    return MPM_ERR_ARG;
  }
  std::map<Key, Entry> add;
  std::map<Key, int> add_edge;
  char line[512];
  bool bad = false;
  while (!bad && std::fgets(line, sizeof(line), f)) {
    int v[4 + 2 * TK_COUNT], used = 0, n = 0;
    const char* q = line;
    if (std::string(line).rfind("edge ", 0) == 0) {  // edge dim log2_particles log2_nodes sms tile_edge
      int e[5], u = 0, m = 0;
      q = line + 5;
      while (m < 5 && std::sscanf(q, "%d%n", &e[m], &u) == 1) {
        q += u;
        ++m;
      }
      for (const char* c = q; *c; ++c) bad = bad || !(*c == ' ' || *c == '\t' || *c == '\n' || *c == '\r');
      bad = bad || m != 5 || !(e[0] == 2 || e[0] == 3) || e[1] < 0 || e[2] < 0 || e[3] < 1 ||
            !(e[4] == 4 || (e[4] == 8 && e[0] == 2));
      if (!bad) add_edge[Key(e[0], e[1], e[2], e[3])] = e[4];
      continue;
    }
    while (n < 4 + 2 * TK_COUNT && std::sscanf(q, "%d%n", &v[n], &used) == 1) {
      q += used;
      ++n;
    }
    for (const char* c = q; *c; ++c) bad = bad || !(*c == ' ' || *c == '\t' || *c == '\n' || *c == '\r');
    if (n == 0 || bad) continue;  // blank line, or refused below
    if (n != 4 + 2 * TK_COUNT || (v[0] != 2 && v[0] != 3) || v[1] < 0 || v[2] < 0 || v[3] < 1) {
      bad = true;
      break;
    }
    Entry e;
    for (int k = 0; k < TK_COUNT; ++k) {
      e.l[k] = TileLaunch{v[4 + 2 * k], v[5 + 2 * k]};
      bad = bad || !is_candidate(k, v[0], e.l[k]);
    }
    add[Key(v[0], v[1], v[2], v[3])] = e;
  }
  if (bad) {
    std::fclose(f);
    return MPM_ERR_ARG;
  }
  std::fclose(f);
  for (auto& kv : add) g_cache[kv.first] = kv.second;
  for (auto& kv : add_edge) g_edge[kv.first] = kv.second;
  return MPM_OK;
}

// Caller holds g_mu.
mpm_status save_locked(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return MPM_ERR_ARG;
  std::fprintf(f, "gbmpm-tune 1 (dim log2_particles log2_tiles sms, then ctas_per_sm threads of p2g g2p p2g_adj "
                 "adj_gather; threads are chosen for g2p, and in 2D for p2g and p2g_adj)\n");
  for (auto& kv : g_cache) {
    if (g_partial.count(kv.first)) continue;  // some kernels of this key not tuned yet
    std::fprintf(f, "%d %d %d %d", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 std::get<3>(kv.first));
    for (int k = 0; k < TK_COUNT; ++k) std::fprintf(f, " %d %d", kv.second.l[k].ctas_per_sm, kv.second.l[k].threads);
    std::fprintf(f, "\n");
  }
  for (auto& kv : g_edge)
    std::fprintf(f, "edge %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 std::get<3>(kv.first), kv.second);
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) return MPM_ERR_ARG;
  return MPM_OK;
}

// Caller holds g_mu.
void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* p = std::getenv("GBMPM_TUNE_CACHE");
  if (p && *p) load_locked(p);  // a missing or unreadable file starts an empty cache
}

bool lookup(const Key& key, Entry* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end() || g_partial.count(key)) return false;
  *out = it->second;
  return true;
}

void store(const Key& key, const Entry& e) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  g_cache[key] = e;
  g_partial.erase(key);
  const char* p = std::getenv("GBMPM_TUNE_CACHE");
  if (p && *p) save_locked(p);
}

Key scene_key(const mpm_scene* s) { return make_key(s->dim, s->N, s->hp.n_tiles, s->ctx->sm_count); }

}  // namespace

bool tune_edge_lookup(int dim, long long particles, long long nodes, int sms, int* edge) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  auto it = g_edge.find(make_key(dim, particles, nodes, sms));
  if (it == g_edge.end()) return false;
  *edge = it->second;
  return true;
}

void tune_edge_store(int dim, long long particles, long long nodes, int sms, int edge) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  g_edge[make_key(dim, particles, nodes, sms)] = edge;
  const char* p = std::getenv("GBMPM_TUNE_CACHE");
  if (p && *p) save_locked(p);
}

namespace {

bool phase_runs(int ph, int k) {
  if (ph == PH_REV) return k == TK_P2G_ADJ || k == TK_ADJ_GATHER;
  if (ph == PH_STEP || ph == PH_ROLL || ph == PH_RCM) return k == TK_P2G || k == TK_G2P;
  return false;
}

void destroy_events(mpm_scene* s) {
  for (int k = 0; k < TK_COUNT; ++k)
    for (int j = 0; j < 2; ++j)
      if (s->tune.ev[k][j]) {
        cudaEventDestroy(s->tune.ev[k][j]);
        s->tune.ev[k][j] = nullptr;
      }
}

}  // namespace

mpm_status tune_init(mpm_scene* s) {
  TuneState& t = s->tune;
  for (int k = 0; k < TK_COUNT; ++k) {
    t.pending[k] = t.tuned[k] = false;
    t.cand[k] = t.rep[k] = t.best[k] = 0;
  }
  default_launch(s->b, s->ctx->sm_count);
  if (s->impl != MPM_IMPL_TILED || t.mode == MPM_TUNE_OFF) return MPM_OK;
  Entry e;
  if (t.mode == MPM_TUNE_AUTO && lookup(scene_key(s), &e)) {
    for (int k = 0; k < TK_COUNT; ++k) {
      s->b.launch[k] = e.l[k];
      t.tuned[k] = true;
    }
    return MPM_OK;
  }
  for (int k = 0; k < TK_COUNT; ++k)
    for (int j = 0; j < 2; ++j)
      if (!t.ev[k][j]) CK(cudaEventCreate(&t.ev[k][j]));
  for (int k = 0; k < TK_COUNT; ++k) t.pending[k] = true;
  return MPM_OK;
}

void tune_release(mpm_scene* s) { destroy_events(s); }

bool tune_wants(const mpm_scene* s, int ph) {
  for (int k = 0; k < TK_COUNT; ++k)
    if (s->tune.pending[k] && phase_runs(ph, k)) return true;
  return false;
}

namespace {

// Shapes under trial into b (kernels pending and, with ph >= 0, run by phase ph).
void trial_begin(TuneState& t, BatchDev& b, int dim, int ph) {
  for (int k = 0; k < TK_COUNT; ++k)
    if (t.pending[k] && (ph < 0 || phase_runs(ph, k))) b.launch[k] = cands(k, dim).c[t.cand[k]];
}

// After a timed step: each pending kernel's time, next candidate, and when a kernel has tried
// them all its fastest shape into b.  *finished = some kernel finished in this step.
// One timed launch of kernel k's current candidate; true when k has now tried every candidate
// (its fastest shape is then in b).
bool record_time(TuneState& t, BatchDev& b, int dim, int k, float ms) {
  t.cur_ms[k] = t.rep[k] == 0 ? ms : std::fmin(t.cur_ms[k], ms);
  if (++t.rep[k] < kReps) return false;
  if (t.cand[k] == 0 || t.cur_ms[k] < t.best_ms[k]) {
    t.best[k] = t.cand[k];
    t.best_ms[k] = t.cur_ms[k];
  }
  t.rep[k] = 0;
  if (++t.cand[k] < cands(k, dim).n) return false;
  t.pending[k] = false;
  t.tuned[k] = true;
  b.launch[k] = cands(k, dim).c[t.best[k]];
  return true;
}

mpm_status trial_end(TuneState& t, BatchDev& b, int dim, int ph, bool* finished) {
  *finished = false;
  for (int k = 0; k < TK_COUNT; ++k) {
    if (!(t.pending[k] && (ph < 0 || phase_runs(ph, k)))) continue;
    CK(cudaEventSynchronize(t.ev[k][1]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, t.ev[k][0], t.ev[k][1]));
    *finished = record_time(t, b, dim, k, ms) || *finished;
  }
  return MPM_OK;
}

mpm_status create_batch_events(TuneState& t) {
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < TK_COUNT; ++k) {
      t.timed[s][k] = -1;
      for (int j = 0; j < 2; ++j)
        if (!t.evs[s][k][j]) CK(cudaEventCreate(&t.evs[s][k][j]));
    }
  t.set = 0;
  return MPM_OK;
}

void destroy_batch_events(TuneState& t) {
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < TK_COUNT; ++k)
      for (int j = 0; j < 2; ++j)
        if (t.evs[s][k][j]) {
          cudaEventDestroy(t.evs[s][k][j]);
          t.evs[s][k][j] = nullptr;
        }
  for (int k = 0; k < TK_COUNT; ++k) t.ev[k][0] = t.ev[k][1] = nullptr;
}

}  // namespace

mpm_status tune_step(mpm_scene* s, int ph) {
  TuneState& t = s->tune;
  trial_begin(t, s->b, s->dim, ph);
  t.timing = true;
  const mpm_status st = enqueue_step(s, ph, s->ctx->stream);
  t.timing = false;
  CKS(st);
  bool finished = false;
  CKS(trial_end(t, s->b, s->dim, ph, &finished));
  if (finished) {
    bool all = true;
    for (int k = 0; k < TK_COUNT; ++k) all = all && t.tuned[k];
    if (all) {
      Entry e;
      for (int k = 0; k < TK_COUNT; ++k) e.l[k] = s->b.launch[k];
      store(scene_key(s), e);
      destroy_events(s);
    }
  }
  return MPM_OK;
}

mpm_status batch_tune_init(TuneState& t, BatchDev& b, int dim, unsigned kernels) {
  for (int k = 0; k < TK_COUNT; ++k) {
    t.pending[k] = t.tuned[k] = false;
    t.cand[k] = t.rep[k] = t.best[k] = 0;
  }
  t.timing = false;
  const Key key = make_key(dim, b.total_particles, b.total_tiles, b.sm_count);
  Entry e;
  bool have;
  unsigned mask = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    env_load_locked();
    auto it = g_cache.find(key);
    have = it != g_cache.end();
    if (have) e = it->second;
    auto m = g_partial.find(key);
    mask = have ? (m == g_partial.end() ? ~0u : m->second) : 0u;
  }
  for (int k = 0; k < TK_COUNT; ++k) {
    if (have) b.launch[k] = e.l[k];
    if (!(kernels & (1u << k))) continue;
    if (mask & (1u << k)) {
      t.tuned[k] = true;
    } else {
      t.pending[k] = true;
    }
  }
  bool any = false;
  for (int k = 0; k < TK_COUNT; ++k) any = any || t.pending[k];
  if (any) CKS(create_batch_events(t));
  return MPM_OK;
}

bool batch_tune_cached(BatchDev& b, int dim, unsigned kernels) {
  const Key key = make_key(dim, b.total_particles, b.total_tiles, b.sm_count);
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  auto m = g_partial.find(key);
  const unsigned mask = m == g_partial.end() ? ~0u : m->second;
  if ((mask & kernels) != kernels) return false;
  for (int k = 0; k < TK_COUNT; ++k) b.launch[k] = it->second.l[k];
  return true;
}

void batch_tune_begin(TuneState& t, BatchDev& b, int dim) {
  bool any = false;
  for (int k = 0; k < TK_COUNT; ++k) any = any || t.pending[k];
  if (!any) return;
  trial_begin(t, b, dim, -1);
  for (int k = 0; k < TK_COUNT; ++k) {  // this step records into the current event set
    t.ev[k][0] = t.evs[t.set][k][0];
    t.ev[k][1] = t.evs[t.set][k][1];
    t.timed[t.set][k] = t.pending[k] ? t.cand[k] : -1;
  }
  t.timing = true;
}

// The times of the previous timed step (whose events are done by now or soon: this step is
// already queued behind it) count for the candidate they timed, if it is still the current one.
mpm_status batch_tune_end(TuneState& t, BatchDev& b, int dim) {
  if (!t.timing) return MPM_OK;
  t.timing = false;
  const int prev = t.set ^ 1;
  bool finished = false;
  for (int k = 0; k < TK_COUNT; ++k) {
    const int c = t.timed[prev][k];
    t.timed[prev][k] = -1;
    if (c < 0 || !t.pending[k] || c != t.cand[k]) continue;
    CK(cudaEventSynchronize(t.evs[prev][k][1]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, t.evs[prev][k][0], t.evs[prev][k][1]));
    finished = record_time(t, b, dim, k, ms) || finished;
  }
  t.set = prev;
  bool left = false;
  for (int k = 0; k < TK_COUNT; ++k) left = left || t.pending[k];
  if (finished && !left) {
    // merge this composition's kernels into the key's entry; a key whose four kernels are not all
    // tuned yet stays out of the cache file
    const Key key = make_key(dim, b.total_particles, b.total_tiles, b.sm_count);
    std::lock_guard<std::mutex> lk(g_mu);
    env_load_locked();
    auto it = g_cache.find(key);
    Entry e;
    unsigned mask = 0;
    if (it != g_cache.end()) {
      e = it->second;
      auto m = g_partial.find(key);
      mask = m == g_partial.end() ? ~0u : m->second;
    } else {
      for (int k = 0; k < TK_COUNT; ++k) e.l[k] = kDefaultLaunch;
    }
    for (int k = 0; k < TK_COUNT; ++k)
      if (t.tuned[k]) {
        e.l[k] = b.launch[k];
        mask |= 1u << k;
      }
    g_cache[key] = e;
    if ((mask & ((1u << TK_COUNT) - 1)) == (1u << TK_COUNT) - 1) {
      g_partial.erase(key);
      const char* p = std::getenv("GBMPM_TUNE_CACHE");
      if (p && *p) save_locked(p);
    } else {
      g_partial[key] = mask;
    }
    destroy_batch_events(t);
  }
  return MPM_OK;
}

void batch_tune_release(TuneState& t) { destroy_batch_events(t); }

}  // namespace gbmpm

using namespace gbmpm;

extern "C" {

mpm_status mpm_scene_set_tuning(mpm_scene* s, int mode) {
  if (!s || mode < MPM_TUNE_OFF || mode > MPM_TUNE_FORCE) return MPM_ERR_ARG;
  if (s->batch_refs > 0) return MPM_ERR_STATE;
  CK(cudaStreamSynchronize(s->ctx->stream));
  s->tune.mode = mode;
  invalidate_graphs(s);  // graphs hold the launch shapes they were captured with
  return tune_init(s);
}

mpm_status mpm_scene_launch(const mpm_scene* s, int kernel, int* ctas_per_sm, int* threads, int* tuned) {
  if (!s || kernel < 0 || kernel >= TK_COUNT) return MPM_ERR_ARG;
  if (ctas_per_sm) *ctas_per_sm = s->b.launch[kernel].ctas_per_sm;
  if (threads) *threads = kernel == TK_ADJ_GATHER ? (s->dim == 3 ? 128 : 256) : s->b.launch[kernel].threads;
  if (tuned) *tuned = s->tune.tuned[kernel] ? 1 : 0;
  return MPM_OK;
}

mpm_status mpm_tune_cache_lookup(int dim, long long particles, long long grid_tiles, int sm_count, int* shape,
                                 int* found) {
  if ((dim != 2 && dim != 3) || sm_count < 1 || !shape || !found) return MPM_ERR_ARG;
  Entry e;
  *found = lookup(make_key(dim, particles, grid_tiles, sm_count), &e) ? 1 : 0;
  if (*found)
    for (int k = 0; k < TK_COUNT; ++k) {
      shape[2 * k] = e.l[k].ctas_per_sm;
      shape[2 * k + 1] = e.l[k].threads;
    }
  return MPM_OK;
}

mpm_status mpm_tune_cache_store(int dim, long long particles, long long grid_tiles, int sm_count, const int* shape) {
  if ((dim != 2 && dim != 3) || sm_count < 1 || !shape) return MPM_ERR_ARG;
  Entry e;
  for (int k = 0; k < TK_COUNT; ++k) {
    e.l[k] = TileLaunch{shape[2 * k], shape[2 * k + 1]};
    if (!is_candidate(k, dim, e.l[k])) return MPM_ERR_ARG;
  }
  store(make_key(dim, particles, grid_tiles, sm_count), e);
  return MPM_OK;
}

mpm_status mpm_tune_cache_save(const char* path) {
  if (!path) return MPM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  return save_locked(path);
}

mpm_status mpm_tune_cache_load(const char* path) {
  if (!path) return MPM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  return load_locked(path);
}

}  // extern "C"
