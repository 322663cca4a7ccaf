// Batched execution of many scenes (include/mpm.h, mpm_batch_*).
//
// Scenes of one dimension advance together: every launch of a batched step covers all scenes of
// a sub-batch through one scene table (one record per scene, selected on the device from that
// scene's own tables and step counter, with the scene's tile and particle offsets in the batch).
// Scenes whose next work is a forward step (rollout or segment recompute) form the forward
// sub-batch; scenes in their reverse pass form the reverse sub-batch.  Both run every tick, the
// reverse one on the context's second stream beside the forward one (disjoint scenes, each with
// its own tile arrays and node blocks), joined before the tick's bookkeeping.  Tiles
// never span scenes and every sum inside a tile has a fixed order, so a scene's results are the
// same bits alone or in any mix.
//
// Per-scene life cycle of a request: rollout of n_steps (checkpoint every ceil(sqrt(n_steps))
// steps); with want_grad, the reverse pass seeded by loss = mean of the final x_0, segment by
// segment (recompute, then reverse steps).  Results stay in the scene (mpm_get_state,
// mpm_get_gradients).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "mpm_scene.h"

using namespace gbmpm;

namespace {

enum SlotState { S_FREE = 0, S_FWD, S_RCM, S_REV, S_DONE };

struct Slot {
  mpm_scene* s = nullptr;
  int state = S_FREE;
  int T = 0, want_grad = 0, done_steps = 0, seg = 0, left = 0;
  size_t mem = 0;
  mpm_status status = MPM_OK;
};

struct SubBatch {
  std::vector<int> members;  // slot indices
  BatchDev b{};
  SelectPar* dsel = nullptr;
  ScenePar* cur = nullptr;
  CtrlPar* dctrl = nullptr;
  int* pbase = nullptr;
  int cap_scenes = 0, cap_tiles = 0, cap_particles = 0;
  bool need_keys = true;  // composition changed: bin keys and histogram from the selected states
  // launch shapes: the cache entry of the composition's key, else trials during its steps
  TuneState tune;
  long long key_particles = -1, key_tiles = -1;
  int trial_wait = 0;  // steps of this key left before its trials start (0: none pending)
  float4 *partial = nullptr, *partial_b = nullptr;  // node blocks (each half its own: they run at once)
  int cap_edge = 0;  // tile edge the node-block arrays are sized for
};

// Steps a composition key must run before its launch-shape trials start: a serving mix changes
// composition every few ticks, and trials that never finish would only cost time.
constexpr int kTrialWait = 32;

#define CK(expr)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA; \
  } while (0)
#define CKS(expr)                \
  do {                           \
    mpm_status s_ = (expr);      \
    if (s_ != MPM_OK) return s_; \
  } while (0)

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_sub(SubBatch& sb) {
  batch_tune_release(sb.tune);
  sb.key_particles = sb.key_tiles = -1;
  dfree(sb.dsel);
  dfree(sb.cur);
  dfree(sb.dctrl);
  dfree(sb.pbase);
  dfree(sb.b.tile_scene);
  dfree(sb.b.tile_count);
  dfree(sb.b.tile_fill);
  dfree(sb.b.tile_start);
  dfree(sb.b.tile_slot);
  dfree(sb.b.active);
  dfree(sb.b.n_active);
  dfree(sb.b.block_sums);
  dfree(sb.b.work);
  dfree(sb.b.sorted);
  dfree(sb.b.gpartial);
  dfree(sb.partial);
  dfree(sb.partial_b);
  sb.cap_scenes = sb.cap_tiles = sb.cap_particles = 0;
}

// Nodes of a tile's node block ((edge + 2)^dim).
int block_nodes(int dim, int edge) {
  const int bn = edge + 2;
  return dim == 2 ? bn * bn : bn * bn * bn;
}

}  // namespace

struct mpm_batch {
  mpm_ctx* ctx = nullptr;
  int dim = 0;
  int edge = 0;  // tile edge of the admitted scenes (set by the first admission into an empty batch)
  size_t budget = 0, used = 0;
  std::vector<Slot> slots;
  SubBatch fwd, rev;
  bool dirty = true;
  cudaEvent_t fork = nullptr, join = nullptr;  // the reverse half runs on the second stream
  // per-tick bookkeeping: counter writes of the scenes changing phase (one launch), the slots whose
  // request finished (one status gather), device array of the gathered status words
  std::vector<std::pair<int*, int>> pend_ctr;
  std::vector<int> finishing;
  int* d_status = nullptr;
  int status_cap = 0;
};

namespace {

mpm_status grow(mpm_batch* B, SubBatch& sb, int n_scenes, int tiles, int particles) {
  const int sc = std::max(1, n_scenes), tl = std::max(1, tiles), pc = std::max(64, particles);
  if (sc <= sb.cap_scenes && tl <= sb.cap_tiles && pc <= sb.cap_particles && sb.cap_edge == B->edge)
    return MPM_OK;
  CK(cudaStreamSynchronize(B->ctx->stream));
  free_sub(sb);
  CK(cudaMalloc(&sb.dsel, sizeof(SelectPar) * sc));
  CK(cudaMalloc(&sb.cur, sizeof(ScenePar) * sc));
  CK(cudaMalloc(&sb.dctrl, sizeof(CtrlPar) * sc));
  CK(cudaMalloc(&sb.pbase, sizeof(int) * (sc + 1)));
  CK(cudaMalloc(&sb.b.tile_scene, sizeof(int) * tl));
  CK(cudaMalloc(&sb.b.tile_count, sizeof(uint32_t) * tl));
  CK(cudaMalloc(&sb.b.tile_fill, sizeof(uint32_t) * tl));
  CK(cudaMalloc(&sb.b.tile_start, sizeof(uint32_t) * (tl + 1)));
  CK(cudaMalloc(&sb.b.tile_slot, sizeof(int) * tl));
  CK(cudaMalloc(&sb.b.active, sizeof(int) * tl));
  CK(cudaMalloc(&sb.b.n_active, sizeof(int)));
  CK(cudaMalloc(&sb.b.block_sums, sizeof(uint32_t) * (2 * ((tl + 2047) / 2048) + 2)));
  CK(cudaMalloc(&sb.b.work, sizeof(uint32_t) * 4));
  CK(cudaMemsetAsync(sb.b.work, 0, sizeof(uint32_t) * 4, B->ctx->stream));
  CK(cudaMalloc(&sb.b.sorted, sizeof(uint32_t) * pc));
  CK(cudaMalloc(&sb.b.gpartial, sizeof(float) * size_t(tl) * MAX_GROUPS));
  CK(cudaMemsetAsync(sb.b.tile_count, 0, sizeof(uint32_t) * tl, B->ctx->stream));
  CK(cudaMemsetAsync(sb.b.tile_fill, 0, sizeof(uint32_t) * tl, B->ctx->stream));
  sb.cap_scenes = sc;
  sb.cap_tiles = tl;
  sb.cap_particles = pc;
  CK(cudaMalloc(&sb.partial, sizeof(float4) * size_t(tl) * block_nodes(B->dim, B->edge)));
  CK(cudaMalloc(&sb.partial_b, sizeof(float4) * size_t(tl) * block_nodes(B->dim, B->edge)));
  sb.cap_edge = B->edge;
  return MPM_OK;
}

// Tile kernels a half of the batch runs: forward steps P2G and G2P, reverse steps the adjoint
// scatter and gather.
unsigned half_kernels(const mpm_batch* B, const SubBatch& sb) {
  return &sb == &B->fwd ? (1u << TK_P2G) | (1u << TK_G2P) : (1u << TK_P2G_ADJ) | (1u << TK_ADJ_GATHER);
}

int phase_of(int state) { return state == S_FWD ? PH_ROLL : state == S_RCM ? PH_RCM : PH_REV; }

// Lays the members of a sub-batch out in the batch's tile and particle spaces and uploads the
// scene table sources (selections, controllers, offsets).
mpm_status compose(mpm_batch* B, SubBatch& sb) {
  int tiles = 0, particles = 0;
  for (int i : sb.members) {
    tiles += B->slots[i].s->hp.n_tiles;
    particles += B->slots[i].s->N;
  }
  CKS(grow(B, sb, int(sb.members.size()), tiles, particles));
  sb.b.partial = sb.partial;
  sb.b.partial_b = sb.partial_b;
  std::vector<SelectPar> sel;
  std::vector<CtrlPar> ctl;
  std::vector<int> pb(1, 0), tscene(std::max(1, tiles), 0);
  int tb = 0, p0 = 0;
  for (size_t m = 0; m < sb.members.size(); ++m) {
    mpm_scene* s = B->slots[sb.members[m]].s;
    SelectPar q = s->hsel[phase_of(B->slots[sb.members[m]].state)];
    q.tile_base = tb;
    q.pbase = p0;
    sel.push_back(q);
    CtrlPar c = s->ctrl;
    c.gpart = sb.b.gpartial;
    c.active = sb.b.active;
    c.n_active = sb.b.n_active;
    c.whole = sb.members.size() == 1 ? 1 : 0;  // others' tiles share the active list otherwise
    ctl.push_back(c);
    for (int t = 0; t < s->hp.n_tiles; ++t) tscene[tb + t] = int(m);
    tb += s->hp.n_tiles;
    p0 += s->N;
    pb.push_back(p0);
  }
  cudaStream_t st = B->ctx->stream;
  CK(cudaStreamSynchronize(st));
  if (!sel.empty()) {
    CK(cudaMemcpy(sb.dsel, sel.data(), sizeof(SelectPar) * sel.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sb.dctrl, ctl.data(), sizeof(CtrlPar) * ctl.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(sb.pbase, pb.data(), sizeof(int) * pb.size(), cudaMemcpyHostToDevice));
  if (tiles > 0) CK(cudaMemcpy(sb.b.tile_scene, tscene.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice));
  sb.b.scenes = sb.cur;
  sb.b.tile_edge = B->edge;
  sb.b.n_scenes = int(sb.members.size());
  sb.b.scene_pbase = sb.pbase;
  sb.b.total_particles = particles;
  sb.b.total_tiles = tiles;
  // a new workload key takes its shapes anew; an empty composition keeps the last key's shapes
  // and trials (a lockstep batch alternates each half between its members and nothing)
  if (!sb.members.empty() && (particles != sb.key_particles || tiles != sb.key_tiles)) {
    default_launch(sb.b, B->ctx->sm_count);
    CKS(batch_tune_init(sb.tune, sb.b, B->dim, 0u));  // cached shapes, no trials yet
    sb.trial_wait = batch_tune_cached(sb.b, B->dim, half_kernels(B, sb)) ? 0 : kTrialWait;
    sb.key_particles = particles;
    sb.key_tiles = tiles;
  }
  sb.b.has_material = 0;
  for (int m : sb.members) sb.b.has_material |= B->slots[m].s->hp.gmat ? 1 : 0;
  sb.need_keys = true;
  return MPM_OK;
}

// Counts a step of the half's key; its trials start once the key has run kTrialWait steps.
mpm_status trial_clock(mpm_batch* B, SubBatch& sb) {
  if (sb.trial_wait > 0 && --sb.trial_wait == 0) CKS(batch_tune_init(sb.tune, sb.b, B->dim, half_kernels(B, sb)));
  return MPM_OK;
}

mpm_status recompose(mpm_batch* B) {
  B->fwd.members.clear();
  B->rev.members.clear();
  for (int i = 0; i < int(B->slots.size()); ++i) {
    const int st = B->slots[i].state;
    if (st == S_FWD || st == S_RCM) B->fwd.members.push_back(i);
    if (st == S_REV) B->rev.members.push_back(i);
  }
  CKS(compose(B, B->fwd));
  CKS(compose(B, B->rev));
  B->dirty = false;
  return MPM_OK;
}

template <int D>
mpm_status forward_step(mpm_batch* B, cudaStream_t st) {
  SubBatch& sb = B->fwd;
  const int n = int(sb.members.size());
  if (n == 0) return MPM_OK;
  CK(launch_select(sb.dsel, n, sb.cur, st));
  for (int m = 0; m < n; ++m) {
    mpm_scene* s = B->slots[sb.members[m]].s;
    if (ctrl_reads_state(s->ctrl)) CK(ctrl_step_forward(s->hp, sb.cur + m, s->ctrl, st));
  }
  if (sb.need_keys) {
    CK(launch_keys<D>(sb.b, st));
    sb.need_keys = false;
  }
  CK(launch_sort<D>(sb.b, st));
  CKS(trial_clock(B, sb));
  batch_tune_begin(sb.tune, sb.b, D);
  {
    TuneScope ts(sb.tune, TK_P2G, st);
    CK(launch_p2g<D>(sb.b, false, st));
  }
  {
    TuneScope ts(sb.tune, TK_G2P, st);
    CK(launch_g2p<D>(sb.b, st));  // advances every member's forward counter, bins state n+1
  }
  return batch_tune_end(sb.tune, sb.b, D);
}

template <int D>
mpm_status reverse_step(mpm_batch* B, cudaStream_t st) {
  SubBatch& sb = B->rev;
  const int n = int(sb.members.size());
  if (n == 0) return MPM_OK;
  CK(launch_select(sb.dsel, n, sb.cur, st));
  CK(launch_keys<D>(sb.b, st));
  for (int m = 0; m < n; ++m) {
    mpm_scene* s = B->slots[sb.members[m]].s;
    if (ctrl_reads_state(s->ctrl)) CK(ctrl_step_forward(s->hp, sb.cur + m, s->ctrl, st));
  }
  CK(launch_sort<D>(sb.b, st));
  CKS(trial_clock(B, sb));
  batch_tune_begin(sb.tune, sb.b, D);
  {
    TuneScope ts(sb.tune, TK_P2G_ADJ, st);
    CK(launch_p2g<D>(sb.b, true, st));
  }
  {
    TuneScope ts(sb.tune, TK_ADJ_GATHER, st);
    CK(launch_adj_gather<D>(sb.b, st));
  }
  CKS(batch_tune_end(sb.tune, sb.b, D));
  CK(ctrl_backward_batched(sb.cur, sb.dctrl, n, st));  // rewinds every member's reverse counter
  for (int m = 0; m < n; ++m) {
    mpm_scene* s = B->slots[sb.members[m]].s;
    if (ctrl_reads_state(s->ctrl)) CK(ctrl_scatter_x(s->hp, sb.cur + m, s->ctrl, st));
  }
  return MPM_OK;
}

// Start of the reverse work of segment sg (recompute from its checkpoint, then reverse steps).
mpm_status begin_segment(mpm_batch* B, Slot& sl) {
  mpm_scene* s = sl.s;
  const int L = std::min(s->roll_k, s->roll_T - sl.seg * s->roll_k);
  if (L > 1) {
    CKS(set_counter(s, s->d_step, s->roll_start + sl.seg * s->roll_k));
    sl.state = S_RCM;
    sl.left = L - 1;
  } else {
    sl.state = S_REV;
    sl.left = L;
  }
  B->dirty = true;
  return MPM_OK;
}

// Writes the counters the scenes' phase changes asked for (set_counter through the sink), in
// order, with as few launches as the list needs.
mpm_status flush_counters(mpm_batch* B) {
  cudaStream_t st = B->ctx->stream;
  for (size_t i0 = 0; i0 < B->pend_ctr.size(); i0 += INT_LIST_MAX) {
    IntPtrList l;
    l.n = int(std::min<size_t>(INT_LIST_MAX, B->pend_ctr.size() - i0));
    for (int i = 0; i < l.n; ++i) {
      l.ptr[i] = B->pend_ctr[i0 + i].first;
      l.val[i] = B->pend_ctr[i0 + i].second;
    }
    CK(launch_set_int_list(l, st));
  }
  B->pend_ctr.clear();
  return MPM_OK;
}

// Finished requests: the reverse passes' scenes get the bin keys of their current state back, then
// one gather and one copy read every finished scene's status word.
mpm_status finish_requests(mpm_batch* B) {
  if (B->finishing.empty()) return MPM_OK;
  cudaStream_t st = B->ctx->stream;
  for (int idx : B->finishing)
    if (B->slots[idx].want_grad) CKS(restore_keys(B->slots[idx].s));
  const int n = int(B->finishing.size());
  if (n > B->status_cap) {
    CK(cudaStreamSynchronize(st));
    dfree(B->d_status);
    B->status_cap = 0;
    CK(cudaMalloc(&B->d_status, sizeof(int) * n));
    B->status_cap = n;
  }
  for (int i0 = 0; i0 < n; i0 += INT_LIST_MAX) {
    IntPtrList l;
    l.n = std::min(INT_LIST_MAX, n - i0);
    for (int i = 0; i < l.n; ++i) l.ptr[i] = B->slots[B->finishing[i0 + i]].s->d_status;
    CK(launch_gather_ints(l, B->d_status + i0, st));
  }
  std::vector<int> h(n);
  CK(cudaMemcpyAsync(h.data(), B->d_status, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) {
    Slot& sl = B->slots[B->finishing[i]];
    sl.status = mpm_status(h[i]);
    sl.state = S_DONE;
  }
  B->finishing.clear();
  B->dirty = true;
  return MPM_OK;
}

// Slot bookkeeping after one batched step.  Counter writes are collected (one launch for all
// scenes), finished requests are closed together.
mpm_status advance(mpm_batch* B) {
  for (int idx = 0; idx < int(B->slots.size()); ++idx) {
    Slot& sl = B->slots[idx];
    if (sl.state != S_FWD && sl.state != S_RCM && sl.state != S_REV) continue;
    mpm_scene* s = sl.s;
    s->ctr_sink = &B->pend_ctr;
    mpm_status st = MPM_OK;
    if (sl.state == S_FWD) {
      if (++sl.done_steps >= sl.T) {
        s->step += sl.T;
        s->have_rollout = true;
        if (sl.want_grad) {
          st = seed_mean_x0(s);
          sl.seg = s->roll_nseg - 1;
          if (st == MPM_OK) st = begin_segment(B, sl);
        } else {
          sl.state = S_DONE;  // status read in finish_requests
          B->finishing.push_back(idx);
        }
      }
    } else if (sl.state == S_RCM) {
      if (--sl.left <= 0) {
        const int L = std::min(s->roll_k, s->roll_T - sl.seg * s->roll_k);
        sl.state = S_REV;
        sl.left = L;
        B->dirty = true;
      }
    } else if (--sl.left <= 0) {  // S_REV
      if (--sl.seg >= 0) {
        st = begin_segment(B, sl);
      } else {
        finish_backward_quiet(s);
        sl.state = S_DONE;
        B->finishing.push_back(idx);
      }
    }
    s->ctr_sink = nullptr;
    if (st != MPM_OK) return st;
  }
  CKS(flush_counters(B));
  return finish_requests(B);
}

size_t request_bytes(const mpm_scene* s, int T) {
  const int k = T <= 16 ? 1 : int(std::ceil(std::sqrt(double(T))));
  const int nseg = (T + k - 1) / k;
  return (size_t(nseg) + size_t(k - 1)) * s->state_bytes;
}

}  // namespace

extern "C" {

mpm_status mpm_batch_create(mpm_ctx* ctx, int dim, size_t mem_budget, mpm_batch** out) {
  if (!ctx || !out || (dim != 2 && dim != 3)) return MPM_ERR_ARG;
  mpm_batch* B = new (std::nothrow) mpm_batch();
  if (!B) return MPM_ERR_OOM;
  B->ctx = ctx;
  B->dim = dim;
  B->budget = mem_budget;
  if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) != cudaSuccess) {
    if (B->fork) cudaEventDestroy(B->fork);
    delete B;
    return MPM_ERR_CUDA;
  }
  ctx->live.fetch_add(1);
  *out = B;
  return MPM_OK;
}

mpm_status mpm_batch_destroy(mpm_batch* B) {
  if (!B) return MPM_ERR_ARG;
  cudaStreamSynchronize(B->ctx->stream);
  cudaStreamSynchronize(B->ctx->aux);
  for (Slot& sl : B->slots)  // the scenes of unreleased slots are the caller's again
    if (sl.state != S_FREE && sl.s) sl.s->batch_refs -= 1;
  free_sub(B->fwd);
  free_sub(B->rev);
  dfree(B->d_status);
  cudaEventDestroy(B->fork);
  cudaEventDestroy(B->join);
  B->ctx->live.fetch_sub(1);
  delete B;
  return MPM_OK;
}

mpm_status mpm_batch_admit(mpm_batch* B, mpm_scene* s, int n_steps, int want_grad, int* slot) {
  if (!B || !s || !slot || n_steps < 1) return MPM_ERR_ARG;
  *slot = -1;
  if (s->dim != B->dim || s->impl != MPM_IMPL_TILED || s->ctx != B->ctx) return MPM_ERR_ARG;
  bool empty = true;
  for (const Slot& sl : B->slots) {
    if (sl.s == s && sl.state != S_FREE) return MPM_ERR_STATE;  // a scene runs in one slot at a time
    empty = empty && sl.state == S_FREE;
  }
  // one tile edge per batch: the tile kernels of a launch are instantiated for one edge
  if (!empty && s->b.tile_edge != B->edge) return MPM_ERR_ARG;
  const size_t need = request_bytes(s, n_steps);
  if (B->budget != 0 && B->used + need > B->budget) return MPM_OK;  // no room now: *slot stays -1
  int idx = -1;
  for (int i = 0; i < int(B->slots.size()); ++i)
    if (B->slots[i].state == S_FREE) {
      idx = i;
      break;
    }
  if (idx < 0) {
    B->slots.push_back(Slot());
    idx = int(B->slots.size()) - 1;
  }
  const int k = n_steps <= 16 ? 1 : int(std::ceil(std::sqrt(double(n_steps))));
  mpm_status st = prepare_rollout(s, n_steps, k, 0);
  if (st != MPM_OK) return st;
  Slot& sl = B->slots[idx];
  sl = Slot();
  if (empty) B->edge = s->b.tile_edge;
  sl.s = s;
  sl.state = S_FWD;
  sl.T = n_steps;
  sl.want_grad = want_grad;
  sl.mem = need;
  B->used += need;
  B->dirty = true;
  s->batch_refs += 1;
  *slot = idx;
  return MPM_OK;
}

mpm_status mpm_batch_tick(mpm_batch* B, int max_steps) {
  if (!B || max_steps < 1) return MPM_ERR_ARG;
  for (int it = 0; it < max_steps; ++it) {
    bool busy = false;
    for (const Slot& sl : B->slots) busy = busy || sl.state == S_FWD || sl.state == S_RCM || sl.state == S_REV;
    if (!busy) break;
    if (B->dirty) CKS(recompose(B));
    // the two halves touch disjoint scenes and buffers: the reverse half runs on the second
    // stream beside the forward half, joined before the bookkeeping
    cudaStream_t ms = B->ctx->stream, as = B->ctx->aux;
    CK(cudaEventRecord(B->fork, ms));
    CK(cudaStreamWaitEvent(as, B->fork, 0));
    if (B->dim == 2) {
      CKS(forward_step<2>(B, ms));
      CKS(reverse_step<2>(B, as));
    } else {
      CKS(forward_step<3>(B, ms));
      CKS(reverse_step<3>(B, as));
    }
    CK(cudaEventRecord(B->join, as));
    CK(cudaStreamWaitEvent(ms, B->join, 0));
    CKS(advance(B));
  }
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_batch_poll(mpm_batch* B, int slot, int* done) {
  if (!B || !done || slot < 0 || slot >= int(B->slots.size()) || B->slots[slot].state == S_FREE) return MPM_ERR_ARG;
  const Slot& sl = B->slots[slot];
  *done = sl.state == S_DONE ? 1 : 0;
  if (sl.state == S_DONE && sl.status != MPM_OK) return sl.status;
  return MPM_OK;
}

mpm_status mpm_batch_release(mpm_batch* B, int slot) {
  if (!B || slot < 0 || slot >= int(B->slots.size()) || B->slots[slot].state == S_FREE) return MPM_ERR_ARG;
  Slot& sl = B->slots[slot];
  if (sl.state != S_DONE) return MPM_ERR_STATE;
  B->used -= sl.mem;
  sl.s->batch_refs -= 1;
  sl = Slot();
  B->dirty = true;
  return MPM_OK;
}

}  // extern "C"
