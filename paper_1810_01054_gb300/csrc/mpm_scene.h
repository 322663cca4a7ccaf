// Internal definitions of the C ABI objects (contexts, scenes) shared by the API and the batch
// scheduler translation units.
#pragma once

#include <atomic>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"

namespace gbmpm {
constexpr int GRAPH_STEPS = 8;  // steps per replayed graph
enum Phase { PH_STEP = 0, PH_ROLL = 1, PH_RCM = 2, PH_REV = 3, PH_PREP = 4, PH_COUNT = 5 };
// Selections beyond the phases': the reverse sort loads on a graph branch, into buffer set A (the
// scene's own) and set B (mpm_scene::bB), stepping back from the graph's first reverse step.
enum BranchSel { SEL_LOAD_A = PH_COUNT, SEL_LOAD_B = PH_COUNT + 1, SEL_COUNT = PH_COUNT + 2 };
// One choice of the multi-level store's planner for a range (mpm_api.cu).
struct MLChoice {
  long long cost = 1LL << 60;  // forward steps; 2^60 = infeasible
  int d = 0;                   // -k: single-level with interval k; j > 0: split at j
  int peak = 0;                // most slots beyond the range's start in use at once
};
}  // namespace gbmpm

using gbmpm::BatchDev;
using gbmpm::CtrlPar;
using gbmpm::ScenePar;
using gbmpm::SelectPar;

struct mpm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t capture = nullptr;  // private stream graphs are captured on
  cudaStream_t aux = nullptr;      // second stream: a reverse pass's segment recompute runs here
  cudaStream_t capture2 = nullptr; // branch of a capture: an open-loop controller's reverse
  cudaStream_t capture3 = nullptr; // branch of a capture: the reverse steps' sort loads
  int sm_count = 1;
  // launch timing (mpm_profile_*): event pairs around launches of the selected kinds; while a
  // mask is set, steps are launched directly (not from graphs) so every launch can be bracketed
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;
  int prof_used = 0;
  std::atomic<int> live{0};  // scenes and batches created on this context and not yet destroyed
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
};

// Autotuner state of a scene (mpm_tune.cu): which tile kernels are still trying candidate launch
// shapes, the candidate under trial, and the best time seen per kernel.
struct TuneState {
  int mode = 1;                         // MPM_TUNE_*
  bool pending[gbmpm::TK_COUNT] = {};   // kernel still being tried
  bool tuned[gbmpm::TK_COUNT] = {};     // shape came from the cache or from trials
  int cand[gbmpm::TK_COUNT] = {};       // candidate under trial
  int rep[gbmpm::TK_COUNT] = {};        // timed launches of it so far
  int best[gbmpm::TK_COUNT] = {};
  float cur_ms[gbmpm::TK_COUNT] = {};
  float best_ms[gbmpm::TK_COUNT] = {};
  bool timing = false;                  // the step being enqueued records the events below
  cudaEvent_t ev[gbmpm::TK_COUNT][2] = {};
  // batches read a step's trial times one step later, so the host never waits for the GPU: two
  // event sets in turn (ev points at the one being recorded) and the candidate each set timed
  cudaEvent_t evs[2][gbmpm::TK_COUNT][2] = {};
  int timed[2][gbmpm::TK_COUNT] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}};
  int set = 0;
};

struct mpm_scene {
  mpm_ctx* ctx = nullptr;
  int dim = 0, N = 0, npad = 0, G = 0, nparams = 0, impl = 0, n_nodes = 0;
  size_t state_bytes = 0;
  ScenePar hp{};             // host template of the scene record
  CtrlPar ctrl{};
  BatchDev b{};              // private batch of one scene; b.scenes = cur
  std::vector<void*> allocs; // everything allocated at creation
  // storage order: slot p of every per-particle array holds the caller's particle order[p]
  // (fixed at creation from the initial positions; every entry point maps through it)
  int* d_order = nullptr;
  std::vector<int> h_order;
  float4* state = nullptr;   // current state planes
  float4* adj[2] = {nullptr, nullptr};
  int* d_step = nullptr;     // forward step counter (controller time)
  int* d_bstep = nullptr;    // reverse step counter
  int* d_status = nullptr;
  // per-particle material (mpm_scene_set_material): E_p, m_p and the (gE, gm) accumulator
  float* d_pE = nullptr;
  float* d_pmass = nullptr;
  float* d_gmat = nullptr;
  ScenePar* cur = nullptr;   // device: the record of the running step
  SelectPar* dsel = nullptr; // device: one selection per phase, then the branch loads'
  SelectPar hsel[gbmpm::SEL_COUNT]{};
  int step = 0;              // host mirror of the current step
  // device record tables, one per phase family (uploaded only when their content changes)
  struct Table {
    ScenePar* dev = nullptr;
    int cap = 0;
    std::vector<ScenePar> host;
  } tables[3];               // 0 = in-place step, 1 = rollout, 2 = recompute + reverse
  struct Map {
    int* dev = nullptr;
    int cap = 0;
    std::vector<int> host;
  } maps[3];                 // record index per step: rollout, recompute, reverse
  Graph graphs[gbmpm::PH_COUNT][gbmpm::GRAPH_STEPS + 1];  // [phase][steps in the graph, 1..GRAPH_STEPS]
  // rollout record
  bool have_rollout = false;
  bool have_grad = false;    // adjoint buffers hold a finished reverse pass
  int roll_T = 0, roll_k = 0, roll_start = 0, roll_nseg = 0;
  std::vector<float4*> ckpt;
  std::vector<float4*> seg;  // k - 1 recompute buffers
  std::vector<void*> roll_allocs;
  // Multi-level store (a rollout whose budget is below the single-level store): state slots, the
  // free ones, and the spine of split ranges the forward stored on its way to the last range.
  // ckpt/seg then point into the slots (pool_backed) instead of roll_allocs.
  struct MLFrame {
    int a, L, start, slots, j, child;  // range [a, a + L) from slot start, split at j into slot child
  };
  bool roll_multi = false;
  bool pool_backed = false;
  std::vector<float4*> ml_pool;
  std::vector<void*> ml_allocs;
  std::vector<int> ml_free;
  std::vector<int> ml_base_slots;  // slots the running single-level range took from ml_free
  std::vector<MLFrame> ml_spine;
  int ml_T = 0, ml_start = 0, ml_first = -1, ml_final = -1, ml_top_slots = 0;
  long long ml_fwd_steps = 0;  // forward steps the schedule runs (rollout and reverse pass)
  std::unordered_map<long long, gbmpm::MLChoice> ml_memo;  // planner choices by (length, slots)
  // staging scratch
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  TuneState tune;
  int batch_refs = 0;  // batch slots holding the scene (admitted, not yet released)
  // The segment recompute's own workspace (tile arrays, selected record, bin keys, actuation,
  // grid), so that mpm_backward can run it on the context's second stream beside the reverse
  // steps; odd segments recompute into seg2 while the reverse steps still read seg.
  BatchDev b2{};
  CtrlPar ctrl2{};  // the controller with its own reduction scratch (state-reading forms)
  ScenePar* cur2 = nullptr;
  uint32_t* key2 = nullptr;
  float* act2 = nullptr;
  float4* grid2 = nullptr;
  std::vector<void*> ws2_allocs;
  std::vector<float4*> seg2;
  uint32_t* sort_store = nullptr;  // 2 x k slots (segment parity, state in segment) of sorts
  float* ctrl_store = nullptr;     // the same slots of controller inputs and actuations (controllers
                                   // that read the state)
  bool rcm_ws2 = false;     // the reverse tables send the recompute to workspace 2
  bool graphs_ws2 = false;  // workspace the recompute graphs were captured with
  size_t roll_budget = 0;
  cudaEvent_t ev_rcm[2] = {}, ev_rev[2] = {}, ev_fork = nullptr;
  // Reverse graphs of a tiled scene whose controller reads no state: each step's controller
  // reverse is captured on a branch (ctx->capture2) that the next step's adjoint gather joins, so it
  // runs beside that step's sort and adjoint scatter (BatchDev::rewind_ctr).
  // With it, and the sorts kept by the recompute, the reverse graphs load the sort of step j + 2
  // on a second branch (ctx->capture3) while steps j and j + 1 run: odd steps of a graph use the
  // buffer set B below (tile arrays, bin keys, actuation, published record), even steps the scene's.
  BatchDev bB{};
  ScenePar* curB = nullptr;
  uint32_t* keyB = nullptr;
  float* actB = nullptr;
  int* d_gstep = nullptr;          // first reverse step of the running graph
  cudaEvent_t ev_load[3] = {};     // fork after the first load; loads of even and odd steps done
  cudaEvent_t ev_gather = nullptr; // a step's adjoint gather done (its buffer set is free)
  bool ctrl_branch = false;
  bool ctrl_join = false;          // a branch is captured and not yet joined
  int* d_rows = nullptr;           // active-slot count of the last adjoint gather
  cudaEvent_t ev_ctrl[2] = {};     // fork, join
  // while set, set_counter appends (counter, value) here instead of launching a write: the batch
  // scheduler writes the counters of all its scenes with one launch
  std::vector<std::pair<int*, int>>* ctr_sink = nullptr;
};


namespace gbmpm {
// Helpers the batch scheduler shares with the single-scene entry points (mpm_api.cu).
mpm_status prepare_rollout(mpm_scene* s, int T, int k, size_t budget);
// flags of prepare_backward used by the multi-level store for its later ranges
enum BackwardFlags {
  BW_KEEP_SEED = 1,   // the adjoint of the range's last state is already in adj[0]
  BW_ACCUMULATE = 2,  // controller-parameter and material gradients keep what earlier ranges added
  BW_NO_OVERLAP = 4,  // the recompute runs in line (no second workspace)
};
mpm_status prepare_backward(mpm_scene* s, const float* gxT, const float* gvT, const float* gCT, const float* gFT,
                            int mem_space, bool mean_x0_seed = false, int flags = 0);
mpm_status seed_mean_x0(mpm_scene* s);
mpm_status finish_backward(mpm_scene* s, float* gx0, float* gv0, float* gC0, float* gF0, float* gctrl,
                           int mem_space);
// The part of finish_backward a batch needs when nothing is read out: the gradient is marked
// available and the forward counter restored (through the counter sink); the caller then restores
// the bin keys (restore_keys, after the counter is written) and reads the status.
void finish_backward_quiet(mpm_scene* s);
// Bin keys and tile histogram of the scene's current state (after a reverse pass left those of
// the rollout's first state).
mpm_status restore_keys(mpm_scene* s);
mpm_status set_counter(mpm_scene* s, int* dctr, int value);
mpm_status read_status(mpm_scene* s);
mpm_status scene_sync_status(mpm_scene* s);

// One step of phase ph enqueued on st (mpm_api.cu); graphs are not used.
mpm_status enqueue_step(mpm_scene* s, int ph, cudaStream_t st);
// Drops the scene's captured graphs (they are captured again with the current launch shapes).
void invalidate_graphs(mpm_scene* s);
// Records rebuilt after the scene template changed (mpm_scene_set_material / _set_walls).
mpm_status refresh_records(mpm_scene* s);

// Event pair around one launch of kind k (no-op unless k is being timed).
struct ProfScope {
  mpm_ctx* c;
  cudaStream_t st;
  int slot = -1;
  ProfScope(mpm_ctx* ctx, cudaStream_t stream, int kind) : c(ctx), st(stream) {
    if (!(c->prof_mask & (1u << kind))) return;
    if (2 * (c->prof_used + 1) > int(c->prof_ev.size())) return;
    slot = c->prof_used++;
    c->prof_kind[slot] = kind;
    cudaEventRecord(c->prof_ev[2 * slot], st);
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], st);
  }
};

// Autotuner (mpm_tune.cu).
// Looks the scene's workload up in the cache, or arms trials for its tile kernels (mode AUTO/FORCE).
mpm_status tune_init(mpm_scene* s);
void tune_release(mpm_scene* s);
// True while a tile kernel that phase ph launches is still being tried.
bool tune_wants(const mpm_scene* s, int ph);
// One directly-launched step of phase ph with the candidate shapes under trial, timed.
mpm_status tune_step(mpm_scene* s, int ph);
// Tile edge that mpm_tune_tile_edge chose for a workload (dim, particles, grid nodes, SMs), and
// storing one (rewrites the cache file named by GBMPM_TUNE_CACHE, if any).
bool tune_edge_lookup(int dim, long long particles, long long nodes, int sms, int* edge);
void tune_edge_store(int dim, long long particles, long long nodes, int sms, int edge);
// Batches (mpm_batch.cu): a sub-batch composition's shapes come from the cache; on a miss the
// kernels it runs are tried the way a scene's are, during its ordinary steps.
//  batch_tune_init   cache shapes of the composition's key, or trials armed for `kernels` (mask)
//  batch_tune_begin  candidate shapes of the kernels under trial into b (before a step)
//  batch_tune_end    times of that step's trials; when the last finishes, the key's cache entry
//                    takes the chosen shapes of these kernels
mpm_status batch_tune_init(TuneState& t, BatchDev& b, int dim, unsigned kernels);
// True when the cache entry of b's key has every kernel of the mask tuned (shapes then in b).
bool batch_tune_cached(BatchDev& b, int dim, unsigned kernels);
void batch_tune_begin(TuneState& t, BatchDev& b, int dim);
mpm_status batch_tune_end(TuneState& t, BatchDev& b, int dim);
void batch_tune_release(TuneState& t);
// Records CUDA events around one launch of tile kernel k while its shape is being tried.
struct TuneScope {
  TuneState& t;
  int k;
  cudaStream_t st;
  bool on;
  TuneScope(TuneState& state, int kernel, cudaStream_t stream)
      : t(state), k(kernel), st(stream), on(state.timing && state.pending[kernel]) {
    if (on) cudaEventRecord(t.ev[k][0], st);
  }
  ~TuneScope() {
    if (on) cudaEventRecord(t.ev[k][1], st);
  }
};
}  // namespace gbmpm
