// Internal structures shared by the kernel and C-ABI translation units of libgbmpm.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mpm_device.cuh"

namespace gbmpm {

// Kernels launched by this library (process-wide tally, read by mpm_launch_count).  While a
// thread captures a CUDA graph its launches go to the capture's tally instead; the graph's kernels
// are counted each time it is launched.
void count_launches(int n);

long long launch_total();
void capture_tally(long long* tally);  // non-null: this thread is capturing

// Scheduling priority given to the kernels this thread launches (0: the stream's).  Reverse-pass
// graphs are captured with the device's highest priority, so their kernels' CTAs go ahead of the
// recompute running beside them on the second stream.
extern thread_local int g_launch_priority;

// Launches kernel k with programmatic stream serialization (its CTAs may be scheduled while the
// previous kernel on s finishes).  k must begin with pdl_enter().
template <class... P, class... A>
cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = g_launch_priority;
  cfg.attrs = at;
  cfg.numAttrs = g_launch_priority ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

constexpr uint32_t KEY_INVALID = 0xffffffffu;
constexpr int MAX_GROUPS = 64;  // actuation groups per scene
constexpr int MAX_HIDDEN = 128; // controller MLP width

// Per-scene parameters and device pointers, as the kernels see them (one entry per scene of
// a launch).  Particle state stays in the caller's particle order for the scene's lifetime.
struct ScenePar {
  int dim;
  int n[3];
  float dx, inv_dx, dt;
  float gravity[3];
  Material mat;
  float mass, vol;
  // optional per-particle Young's modulus and mass (NULL: mat and mass above for every particle);
  // mat = E x (mu_per_E, la_per_E), the Lame parameters of E = 1 at the scene's nu.  With them
  // the reverse step adds this step's dL/dE_p, dL/dm_p into gmat[p] = (gE, gm).
  const float* pE;
  const float* pmass;
  float mu_per_E, la_per_E;
  float2* gmat;
  BCPar bc;
  int N, npad;      // particles, plane stride (N rounded up)
  int G;            // actuation groups
  int nt[3];        // tiles per axis
  int n_tiles;      // product of nt
  int tile_base;    // first batch-global tile id of this scene
  int pbase;        // first batch-global particle slot of this scene
  int step;         // global step index of the state being advanced (t_n = step*dt)
  float4* planes;   // state planes [PLANES][npad] read by the step
  float4* planes_out;  // where G2P writes state n+1 (== planes for an in-place step)
  const float4* adj_in;   // adjoint planes of state n+1 (reverse step)
  float4* adj_out;        // adjoint planes of state n  (reverse step)
  uint32_t* key;          // [N] tile << 6 | cell-in-tile, KEY_INVALID if the stencil left the grid
  float4* grid;           // [nodes] (v*, m) after the boundary condition
  float4* grid_b;         // [nodes] reverse: (pbar, mbar)
  const int32_t* group;   // [N]
  const float* act_dir;   // [G][dim]
  float* act;             // [G] actuation of the current step
  float* act_grad;        // [G] dL/da of the current reverse step
  float* sig_contrib;     // [N] per-particle part of dL/da (S4 (K))
  int* status;            // first-error status word
  int* step_ctr;          // step counter the step advances (G2P) or rewinds (controller adjoint)
  // sort store (reverse pass with the recompute beside it): a recompute step stores the sort of
  // the state it reads here, a reverse step loads the sort of its state from here (NULL: none)
  uint32_t* sort_slot;
  // controllers that read the state, same reverse pass: the forward of a recompute step writes its
  // controller input z (and, through act, its actuation) into this state's slot; the reverse step
  // reads both from there instead of evaluating the controller again (NULL: the controller's own
  // scratch)
  float* ctrl_z;
};

// Floats of one controller slot: input z (at most 3 (1 + 2 MAX_GROUPS)), then the actuation.
constexpr int CTRL_Z_CAP = 3 * (1 + 2 * 64);
constexpr int CTRL_SLOT_FLOATS = CTRL_Z_CAP + 64 + 1;

// Words of one sort-store slot: sorted ids [npad] | bin keys [npad] | tile_start [nt + 1] |
// tile_slot [nt] | active [nt] | n_active [1].
inline size_t sort_slot_words(int npad, int nt) { return 2 * size_t(npad) + 3 * size_t(nt) + 2; }

// Where a scene's record for the current step comes from (see k_select).
struct SelectPar {
  const ScenePar* table;  // the scene's record table for the running phase
  const int* map;         // record index of step n at map[n - base]; NULL = record 0
  int base;
  const int* ctr;         // step counter n
  int tile_base, pbase;   // batch offsets of the scene
  int ctrl_type, G;       // sinusoid and table controllers are evaluated by the selection
  int ctrl_len;           // table controller: steps in the table
  float freq, dt;
  const float* params;
  float* act;
  // non-NULL: the published record's bin keys and actuation are these instead of the table's (a
  // second set of reverse-step buffers, so the next step's sort can be loaded beside this one)
  uint32_t* key_rec;
  float* act_rec;
};

// Tile kernels whose launch shape (CTAs per SM of the persistent grid, threads per CTA) is
// chosen per workload by the autotuner (mpm_tune.cu).
enum TileKernel { TK_P2G = 0, TK_G2P = 1, TK_P2G_ADJ = 2, TK_ADJ_GATHER = 3, TK_COUNT = 4 };
struct TileLaunch {
  int ctas_per_sm;
  int threads;
};
// Launch shapes used when nothing was tuned: four CTAs per SM of 256 threads.
constexpr TileLaunch kDefaultLaunch{4, 256};

// One batch of scenes of equal dimension that advance together.
struct BatchDev {
  ScenePar* scenes;     // device [n_scenes]
  int n_scenes;
  int* scene_pbase;     // device [n_scenes + 1] prefix of particle counts
  int* tile_scene;      // device [total_tiles] owning scene of every batch tile
  int total_particles;
  int total_tiles;
  uint32_t* tile_count; // [total_tiles], zero between steps
  uint32_t* tile_fill;  // [total_tiles], zero between steps
  uint32_t* tile_start; // [total_tiles + 1]
  int* tile_slot;       // [total_tiles] active-slot of the tile or -1
  int* active;          // [total_tiles] batch tile id of every active slot
  int* n_active;        // [1]
  uint32_t* block_sums; // scan scratch
  uint32_t* work;       // [4] tile counters of the dynamically scheduled P2G and adjoint gather and
                        // their CTAs-done tickets; zero between launches
  uint32_t* sorted;     // [total_particles] scene-local particle ids, tile-major, canonical
  float4* partial;      // [total_tiles * BLOCK_NODES] node blocks of P2G
  float4* partial_b;    // [total_tiles * BLOCK_NODES] node blocks of the adjoint scatter
  float* gpartial;      // [total_tiles * MAX_GROUPS] per active tile group sums of dL/da
  int tile_edge;                // cells per tile edge of every scene in the batch (0 or 4; 8: 2D)
  int has_material;             // some scene has per-particle material (gmat): material gradients
  int sm_count;                 // SMs of the device
  TileLaunch launch[TK_COUNT];  // launch shape of each tile kernel
  // A scene alone whose controller reads no state: CTA 0 of the adjoint gather rewinds its reverse
  // step counter (instead of the controller reverse) and keeps the step's active-slot count in
  // rewind_rows, so the controller reverse can run beside the next reverse step (null: off).
  int* rewind_ctr;
  int* rewind_rows;
};

// Sets every tile kernel of b to the default launch shape.
inline void default_launch(BatchDev& b, int sm_count) {
  b.sm_count = sm_count;
  for (int k = 0; k < TK_COUNT; ++k) b.launch[k] = kDefaultLaunch;
}

// ---------------------------------------------------------------------------- launchers
// Sets the kernels' launch attributes (large dynamic shared memory); once per process/device.
cudaError_t configure_kernels();
// Tiled (sorted, deterministic) form.
// sel non-null (a single scene): the first kernel also makes the step's record selection (what
// launch_select does), publishing it to b.scenes[0].
template <int D>
cudaError_t launch_keys(const BatchDev& b, cudaStream_t s, const SelectPar* sel = nullptr);
template <int D>
cudaError_t launch_sort(const BatchDev& b, cudaStream_t s, const SelectPar* sel = nullptr);
template <int D>
cudaError_t launch_p2g(const BatchDev& b, bool with_adjoint, cudaStream_t s);
// G2P (Eqs. 7-10) including the grid update of its node block (Eq. 6, gravity, boundary).
template <int D>
cudaError_t launch_g2p(const BatchDev& b, cudaStream_t s);
// Adjoint gather (S4 (F)-(K), (J)) including the grid adjoint of its node block (S3, S5) and
// the per-tile group sums of dL/da into gpartial.
template <int D>
cudaError_t launch_adj_gather(const BatchDev& b, cudaStream_t s);

// Plain form (one scene, global atomics, dense grid): the baseline the tiled form is measured against.
template <int D>
cudaError_t launch_plain_step(const ScenePar* dev_scene, const ScenePar& host_scene, cudaStream_t s);
template <int D>
cudaError_t launch_plain_adjoint(const ScenePar* dev_scene, const ScenePar& host_scene, float* gpart, cudaStream_t s);

// Controllers.  ctrl_* describe one scene's controller.
struct CtrlPar {
  int type;        // 0 sinusoid amplitude, 1 sinusoid basis, 2 MLP on group centroids, 3 per-step table
  int G, dim, hidden;
  float freq, scale;
  const float* params;   // device
  float* gparams;        // device, accumulated by the reverse pass
  const float* inv_count;  // device [G] 1/|g| (0 for empty groups)
  float inv_n;            // 1/N
  float* centroid;        // device [G*dim + dim] scratch: group centroids then body centroid
  float* gz;              // device [G*dim] scratch: dL/dz of the MLP input
  float* partials;        // device scratch for the deterministic group reductions
  int n_partials;         // number of reduction partial rows available
  // state-reading forms: the particles in group order (stable, ungrouped first) and the group of
  // each entry (-1: none), for the group reductions of x and v
  const int* perm;
  const int* pgroup;
  // rows of per-tile (tiled form) or per-block (plain form) group sums of dL/da, MAX_GROUPS each:
  // the tiled rows of the scene are the active slots whose tile lies in the scene's tile range
  const float* gpart;
  const int* active;      // tiled form: batch active tile list (NULL: plain form)
  const int* n_active;
  int plain_rows;
  int whole;              // tiled form, scene alone in its batch: its rows are all active slots
};

// Controllers whose input is the state (MLP on centroids, closed loop on group means of x and v):
// they need group reductions each step and add an input adjoint to dL/dx (and dL/dv).
inline bool ctrl_reads_state(const CtrlPar& c) { return (c.type == 2 || c.type == 4) && c.G > 0; }
int reduction_rows(int N);                  // partial rows of the group reductions (per reduced quantity)
constexpr int RED_ROW_FLOATS = MAX_GROUPS * 3 + 3;  // floats per partial row
// Controller forward (MLP form; the sinusoid forms are evaluated by k_select) and the reverse of
// the step *sp.step_ctr, which it then decrements.
cudaError_t ctrl_step_forward(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s);
cudaError_t ctrl_step_backward(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s);
// Reverse of a controller that reads no state (sinusoid and table forms) for the step after the
// one *ctr names, whose group sums are rows [0, *rows) of c.gpart: the counter was already rewound
// by the adjoint gather (BatchDev::rewind_ctr), so the launch depends on nothing but that kernel.
cudaError_t ctrl_backward_open(const CtrlPar& c, const int* ctr, const int* rows, float dt, float* act_grad,
                               cudaStream_t s);
// Batched form: one block per scene; records and controllers are device arrays of n entries.
cudaError_t ctrl_backward_batched(const ScenePar* cur, const CtrlPar* cs, int n, cudaStream_t s);
cudaError_t ctrl_scatter_x(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s);

// Copies every scene's record for the current step into cur[] (one block per scene).
cudaError_t launch_select(const SelectPar* sel, int n_scenes, ScenePar* cur, cudaStream_t s);
// Sort store of a single scene: the sort just made in b (raw tile lists, tile arrays, keys) into
// slot `dst` (NULL: the slot named by the published record b.scenes[0]), and the sort of the
// state the reverse selection `sel` names back into b (publishing the record, like launch_keys).
// The load selects step *sel->ctr - back; with `snap` it also writes that step number there.
template <int D>
cudaError_t launch_store_sort(const BatchDev& b, uint32_t* dst, cudaStream_t s);
template <int D>
cudaError_t launch_load_sort(const BatchDev& b, const SelectPar* sel, cudaStream_t s, int back = 0,
                             int* snap = nullptr);
// Adjoint planes of the seed dL/dx_T = e_0 / N (the batched gradient requests' loss).
cudaError_t launch_seed_mean_x0(int dim, int N, int npad, float4* planes, cudaStream_t s);
// A list of device ints passed by value (kernel parameters hold up to INT_LIST_MAX entries).
constexpr int INT_LIST_MAX = 1024;
struct IntPtrList {
  int n;
  int* ptr[INT_LIST_MAX];
  int val[INT_LIST_MAX];
};
// *ptr[i] = val[i] in list order.
cudaError_t launch_set_int_list(const IntPtrList& l, cudaStream_t s);
// out[i] = *ptr[i].
cudaError_t launch_gather_ints(const IntPtrList& l, int* out, cudaStream_t s);
// *p = v on the stream (kernel argument, so no host buffer outlives the call).
cudaError_t launch_set_int(int* p, int v, cudaStream_t s);

// Layout conversions between row-major [N][d], [N][d][d] arrays in the caller's particle order and
// the state planes in storage order: storage slot p holds caller particle order[p] (NULL: p).
cudaError_t launch_pack(int dim, int N, int npad, const float* x, const float* v, const float* C, const float* F,
                        float4* planes, int* status, const int* order, cudaStream_t s);
cudaError_t launch_unpack(int dim, int N, int npad, const float4* planes, float* x, float* v, float* C, float* F,
                          const int* order, cudaStream_t s);

}  // namespace gbmpm
