// C ABI of libgbmpm (include/mpm.h): contexts, scenes, stepping, checkpointed rollouts and the
// rollout-level reverse pass (Section III "memo"; Supplement S2-S5 per step).
//
// Checkpointing: a rollout of T steps stores the state every k steps.  The stored states are
// written by the step itself (G2P writes out of place at segment boundaries), so storing costs no
// extra copy.  The reverse pass walks the segments from last to first, recomputes the states of
// a segment out of place from its checkpoint, then runs the reverse steps of that segment.
// Memory: ceil(T/k) + (k - 1) + 2 states.  k = 1 keeps every state (the paper's memo) and
// recomputes nothing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"

using namespace gbmpm;

struct mpm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 1;
  // launch timing (mpm_profile_*): event pairs around launches of the selected kinds
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;
  int prof_used = 0;
};

struct mpm_scene {
  mpm_ctx* ctx = nullptr;
  int dim = 0, N = 0, npad = 0, G = 0, nparams = 0, impl = 0, n_nodes = 0;
  size_t state_bytes = 0;
  ScenePar hp{};             // host template of the device scene record
  CtrlPar ctrl{};
  BatchDev b{};              // private batch of one scene (tiled form)
  std::vector<void*> allocs; // everything allocated at creation
  float4* state = nullptr;   // current state planes
  float4* adj[2] = {nullptr, nullptr};
  int* d_step = nullptr;     // forward step counter (controller time)
  int* d_bstep = nullptr;    // reverse step counter
  int* d_status = nullptr;
  int step = 0;              // host mirror of the current step
  // device scene records, one cached table per purpose (uploaded only when its content changes):
  // table 0 = in-place forward on `state`, 1 = rollout, 2 = reverse pass
  ScenePar* dconf = nullptr;  // == tables[0].dev
  struct Table {
    ScenePar* dev = nullptr;
    int cap = 0;
    std::vector<ScenePar> host;
  } tables[3];
  // rollout record
  bool have_rollout = false;
  int roll_T = 0, roll_k = 0, roll_start = 0, roll_nseg = 0;
  std::vector<float4*> ckpt;
  std::vector<float4*> seg;  // k - 1 recompute buffers
  std::vector<void*> roll_allocs;
  // staging scratch
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
};

namespace {

mpm_status cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return MPM_OK;
  if (e == cudaErrorMemoryAllocation) return MPM_ERR_OOM;
  return MPM_ERR_CUDA;
}

#define CK(expr)                                 \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

#define CKS(expr)                   \
  do {                              \
    mpm_status s_ = (expr);         \
    if (s_ != MPM_OK) return s_;    \
  } while (0)

template <class T>
mpm_status dalloc(mpm_scene* s, T** p, size_t count, std::vector<void*>& list) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  CK(cudaMalloc(&q, bytes));
  list.push_back(q);
  *p = reinterpret_cast<T*>(q);
  (void)s;
  return MPM_OK;
}

int planes_of(int dim) { return dim == 2 ? Cfg<2>::PLANES : Cfg<3>::PLANES; }
int tile_edge(int dim) { return dim == 2 ? Cfg<2>::B : Cfg<3>::B; }
int block_nodes(int dim) { return dim == 2 ? Cfg<2>::BLOCK_NODES : Cfg<3>::BLOCK_NODES; }

int ctrl_param_count(int type, int G, int dim, int H) {
  if (type == MPM_CTRL_SIN) return G;
  if (type == MPM_CTRL_BASIS) return 4 * G;
  if (type == MPM_CTRL_MLP) {
    int Z = G * dim;
    return H * Z + H + H * H + H + G * H + G;
  }
  return -1;
}

// Device pointer of caller data: copies host data into the scene scratch (offset bytes in).
mpm_status stage(mpm_scene* s, const void* src, size_t bytes, int mem_space, size_t offset, const void** out) {
  if (!src) {
    *out = nullptr;
    return MPM_OK;
  }
  if (mem_space == 1) {
    *out = src;
    return MPM_OK;
  }
  char* dst = reinterpret_cast<char*>(s->scratch) + offset;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->ctx->stream));
  *out = dst;
  return MPM_OK;
}

mpm_status ensure_scratch(mpm_scene* s, size_t bytes) {
  if (bytes <= s->scratch_bytes) return MPM_OK;
  CK(cudaStreamSynchronize(s->ctx->stream));
  if (s->scratch) cudaFree(s->scratch);
  s->scratch = nullptr;
  s->scratch_bytes = 0;
  CK(cudaMalloc(&s->scratch, bytes));
  s->scratch_bytes = bytes;
  return MPM_OK;
}


// Upload a table of scene records unless the device already holds exactly this table
// (synchronously: work enqueued afterwards reads it, and work in flight may read the old one).
mpm_status upload_conf(mpm_scene* s, int which, const std::vector<ScenePar>& confs, ScenePar** dev) {
  auto& t = s->tables[which];
  const bool same = t.host.size() == confs.size() &&
                    std::memcmp(t.host.data(), confs.data(), sizeof(ScenePar) * confs.size()) == 0;
  if (!same) {
    CK(cudaStreamSynchronize(s->ctx->stream));
    if (int(confs.size()) > t.cap) {
      if (t.dev) cudaFree(t.dev);
      t.dev = nullptr;
      t.cap = 0;
      CK(cudaMalloc(&t.dev, sizeof(ScenePar) * confs.size()));
      t.cap = int(confs.size());
    }
    CK(cudaMemcpy(t.dev, confs.data(), sizeof(ScenePar) * confs.size(), cudaMemcpyHostToDevice));
    t.host = confs;
  }
  if (dev) *dev = t.dev;
  if (which == 0) s->dconf = t.dev;
  return MPM_OK;
}

ScenePar conf_fwd(const mpm_scene* s, float4* in, float4* out) {
  ScenePar p = s->hp;
  p.planes = in;
  p.planes_out = out;
  return p;
}

ScenePar conf_bwd(const mpm_scene* s, float4* st, const float4* ain, float4* aout) {
  ScenePar p = s->hp;
  p.planes = st;
  p.planes_out = st;
  p.adj_in = ain;
  p.adj_out = aout;
  return p;
}

mpm_status set_counter(mpm_scene* s, int* dctr, int value) {
  CK(launch_set_int(dctr, value, s->ctx->stream));
  return MPM_OK;
}

// Event pair around one launch of kind k (no-op unless k is being timed).
struct ProfScope {
  mpm_ctx* c;
  int slot = -1;
  ProfScope(mpm_ctx* ctx, int kind) : c(ctx) {
    if (!(c->prof_mask & (1u << kind))) return;
    if (2 * (c->prof_used + 1) > int(c->prof_ev.size())) return;
    slot = c->prof_used++;
    c->prof_kind[slot] = kind;
    cudaEventRecord(c->prof_ev[2 * slot], c->stream);
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
  }
};

// One forward step with device record `dsp` (host copy `hsp`).
mpm_status forward_step(mpm_scene* s, const ScenePar* dsp, const ScenePar& hsp, int* ctr) {
  cudaStream_t st = s->ctx->stream;
  mpm_ctx* c = s->ctx;
  {
    ProfScope p(c, MPM_K_CTRL);
    CK(ctrl_step_forward(hsp, dsp, s->ctrl, ctr, 1, st));
  }
  if (s->impl == MPM_IMPL_PLAIN) {
    ProfScope p(c, MPM_K_PLAIN);
    CK(s->dim == 2 ? launch_plain_step<2>(dsp, hsp, st) : launch_plain_step<3>(dsp, hsp, st));
    return MPM_OK;
  }
  BatchDev bb = s->b;
  bb.scenes = const_cast<ScenePar*>(dsp);
  const bool two = s->dim == 2;
  {
    ProfScope p(c, MPM_K_SORT);
    CK(two ? launch_sort<2>(bb, st) : launch_sort<3>(bb, st));
  }
  {
    ProfScope p(c, MPM_K_P2G);
    CK(two ? launch_p2g<2>(bb, false, st) : launch_p2g<3>(bb, false, st));
  }
  {
    ProfScope p(c, MPM_K_GRID);
    CK(two ? launch_grid<2>(bb, false, st) : launch_grid<3>(bb, false, st));
  }
  {
    ProfScope p(c, MPM_K_G2P);
    CK(two ? launch_g2p<2>(bb, st) : launch_g2p<3>(bb, st));
  }
  return MPM_OK;
}

// One reverse step on record `dsp` (state n, adjoint n+1 in, adjoint n out).
mpm_status reverse_step(mpm_scene* s, const ScenePar* dsp, const ScenePar& hsp) {
  cudaStream_t st = s->ctx->stream;
  mpm_ctx* c = s->ctx;
  BatchDev bb = s->b;
  bb.scenes = const_cast<ScenePar*>(dsp);
  const bool two = s->dim == 2;
  if (s->impl != MPM_IMPL_PLAIN) {
    ProfScope p(c, MPM_K_SORT);
    CK(two ? launch_keys<2>(bb, st) : launch_keys<3>(bb, st));
  }
  {
    ProfScope p(c, MPM_K_CTRL);
    CK(ctrl_step_forward(hsp, dsp, s->ctrl, s->d_bstep, 0, st));
  }
  if (s->impl == MPM_IMPL_PLAIN) {
    ProfScope p(c, MPM_K_PLAIN);
    CK(two ? launch_plain_adjoint<2>(dsp, hsp, st) : launch_plain_adjoint<3>(dsp, hsp, st));
  } else {
    {
      ProfScope p(c, MPM_K_SORT);
      CK(two ? launch_sort<2>(bb, st) : launch_sort<3>(bb, st));
    }
    {
      ProfScope p(c, MPM_K_P2G_ADJ);
      CK(two ? launch_p2g<2>(bb, true, st) : launch_p2g<3>(bb, true, st));
    }
    {
      ProfScope p(c, MPM_K_GRID_ADJ);
      CK(two ? launch_grid<2>(bb, true, st) : launch_grid<3>(bb, true, st));
    }
    {
      ProfScope p(c, MPM_K_ADJ_GATHER);
      CK(two ? launch_adj_gather<2>(bb, st) : launch_adj_gather<3>(bb, st));
    }
  }
  {
    ProfScope p(c, MPM_K_CTRL);
    CK(ctrl_step_backward(hsp, dsp, s->ctrl, s->d_bstep, st));
  }
  return MPM_OK;
}

mpm_status read_status(mpm_scene* s) {
  int v = 0;
  CK(cudaStreamSynchronize(s->ctx->stream));
  CK(cudaMemcpy(&v, s->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return mpm_status(v);
}

mpm_status refresh_keys(mpm_scene* s) {
  if (s->impl == MPM_IMPL_PLAIN) return MPM_OK;
  BatchDev bb = s->b;
  bb.scenes = s->dconf;
  CK(s->dim == 2 ? launch_keys<2>(bb, s->ctx->stream) : launch_keys<3>(bb, s->ctx->stream));
  return MPM_OK;
}

void free_rollout(mpm_scene* s) {
  if (!s->roll_allocs.empty()) cudaStreamSynchronize(s->ctx->stream);
  for (void* p : s->roll_allocs) cudaFree(p);
  s->roll_allocs.clear();
  s->ckpt.clear();
  s->seg.clear();
  s->have_rollout = false;
}

}  // namespace

extern "C" {

const char* mpm_status_str(mpm_status s) {
  switch (s) {
    case MPM_OK: return "ok";
    case MPM_ERR_ARG: return "invalid argument";
    case MPM_ERR_OOM: return "out of device memory or memory budget";
    case MPM_ERR_DOMAIN: return "a particle stencil left the grid";
    case MPM_ERR_INVERTED: return "det F <= 0";
    case MPM_ERR_TIMEOUT: return "bounded device wait expired";
    case MPM_ERR_CUDA: return "CUDA error";
    case MPM_ERR_STATE: return "call out of order";
    case MPM_ERR_DENSITY: return "too many particles in one tile";
    case MPM_ERR_INTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

mpm_status mpm_ctx_create(mpm_ctx** out, int device, void* cuda_stream) {
  if (!out) return MPM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return MPM_ERR_ARG;
  CK(cudaSetDevice(device));
  mpm_ctx* c = new (std::nothrow) mpm_ctx();
  if (!c) return MPM_ERR_OOM;
  c->device = device;
  if (cuda_stream) {
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e);
    }
    c->own_stream = true;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return MPM_OK;
}

mpm_status mpm_ctx_destroy(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return MPM_OK;
}

mpm_status mpm_sync(mpm_ctx* c) {
  if (!c) return MPM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_scene_destroy(mpm_scene* s) {
  if (!s) return MPM_ERR_ARG;
  cudaStreamSynchronize(s->ctx->stream);
  free_rollout(s);
  for (void* p : s->allocs) cudaFree(p);
  for (auto& t : s->tables)
    if (t.dev) cudaFree(t.dev);
  if (s->scratch) cudaFree(s->scratch);
  delete s;
  return MPM_OK;
}

mpm_status mpm_scene_create(mpm_ctx* c, const mpm_scene_desc* d, mpm_scene** out) {
  if (!c || !d || !out) return MPM_ERR_ARG;
  *out = nullptr;
  const int dim = d->dim;
  if (dim != 2 && dim != 3) return MPM_ERR_ARG;
  for (int a = 0; a < dim; ++a)
    if (d->n_grid[a] < 5) return MPM_ERR_ARG;
  if (!(d->dx > 0.f) || !(d->dt > 0.f) || !(d->E > 0.f) || !(d->nu > -1.f && d->nu < 0.5f)) return MPM_ERR_ARG;
  if (!(d->p_mass > 0.f) || !(d->p_vol > 0.f)) return MPM_ERR_ARG;
  if (d->bc_type != MPM_BC_STICKY && d->bc_type != MPM_BC_SLIP) return MPM_ERR_ARG;
  if (d->bc_width < 0 || !(d->friction_c >= 0.f)) return MPM_ERR_ARG;
  if (d->n_particles < 0 || d->n_particles >= (1 << 26)) return MPM_ERR_ARG;
  if (d->n_particles > 0 && !d->x0) return MPM_ERR_ARG;
  if (d->n_groups < 0 || d->n_groups > MAX_GROUPS) return MPM_ERR_ARG;
  if (d->n_groups > 0 && !d->act_dir) return MPM_ERR_ARG;
  if (d->impl != MPM_IMPL_TILED && d->impl != MPM_IMPL_PLAIN) return MPM_ERR_ARG;
  if (d->mem_space != 0 && d->mem_space != 1) return MPM_ERR_ARG;
  if (d->ctrl_type == MPM_CTRL_MLP &&
      (d->ctrl_hidden < 1 || d->ctrl_hidden > MAX_HIDDEN || d->n_groups * dim > MAX_GROUPS * 3))
    return MPM_ERR_ARG;
  const int np = ctrl_param_count(d->ctrl_type, d->n_groups, dim, d->ctrl_hidden);
  if (np < 0 || np != d->n_ctrl_params || (np > 0 && !d->ctrl_params)) return MPM_ERR_ARG;
  // explicit-integration limit dt <= C dx sqrt(rho / E) with C = 1 (Section VI)
  const double rho = double(d->p_mass) / double(d->p_vol);
  if (double(d->dt) > double(d->dx) * std::sqrt(rho / double(d->E)) * (1.0 + 1e-6)) return MPM_ERR_ARG;

  CK(cudaSetDevice(c->device));
  mpm_scene* s = new (std::nothrow) mpm_scene();
  if (!s) return MPM_ERR_OOM;
  s->ctx = c;
  s->dim = dim;
  s->N = d->n_particles;
  s->npad = std::max(64, (s->N + 63) / 64 * 64);
  s->G = d->n_groups;
  s->nparams = np;
  s->impl = d->impl;
  s->n_nodes = 1;
  for (int a = 0; a < dim; ++a) s->n_nodes *= d->n_grid[a];
  const int PL = planes_of(dim);
  s->state_bytes = sizeof(float4) * size_t(PL) * size_t(s->npad);

  ScenePar& p = s->hp;
  std::memset(&p, 0, sizeof(p));
  p.dim = dim;
  const int B = tile_edge(dim);
  p.n_tiles = 1;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = a < dim ? d->n_grid[a] : 1;
    p.gravity[a] = a < dim ? d->gravity[a] : 0.f;
    p.nt[a] = a < dim ? (p.n[a] + B - 1) / B : 1;
    p.n_tiles *= p.nt[a];
  }
  p.dx = d->dx;
  p.inv_dx = 1.0f / d->dx;
  p.dt = d->dt;
  p.mat.mu = float(double(d->E) / (2.0 * (1.0 + double(d->nu))));
  p.mat.la = float(double(d->E) * double(d->nu) / ((1.0 + double(d->nu)) * (1.0 - 2.0 * double(d->nu))));
  p.mass = d->p_mass;
  p.vol = d->p_vol;
  p.bc.type = d->bc_type;
  p.bc.width = d->bc_width;
  p.bc.c = d->friction_c;
  p.N = s->N;
  p.npad = s->npad;
  p.G = s->G;
  p.tile_base = 0;
  p.pbase = 0;

  auto fail = [&](mpm_status st) {
    mpm_scene_destroy(s);
    return st;
  };
  mpm_status st = MPM_OK;
#define ALLOC(ptr, n)                                       \
  do {                                                      \
    st = dalloc(s, &(ptr), size_t(n), s->allocs);           \
    if (st != MPM_OK) return fail(st);                      \
  } while (0)
  ALLOC(s->state, size_t(PL) * s->npad);
  ALLOC(s->adj[0], size_t(PL) * s->npad);
  ALLOC(s->adj[1], size_t(PL) * s->npad);
  uint32_t* key;
  ALLOC(key, s->npad);
  float4 *grid, *grid_b;
  ALLOC(grid, s->n_nodes);
  ALLOC(grid_b, s->n_nodes);
  int32_t* group;
  ALLOC(group, s->npad);
  float *act_dir, *act, *act_grad, *sig;
  ALLOC(act_dir, std::max(1, s->G * dim));
  ALLOC(act, std::max(1, s->G));
  ALLOC(act_grad, std::max(1, s->G));
  ALLOC(sig, s->npad);
  ALLOC(s->d_step, 1);
  ALLOC(s->d_bstep, 1);
  ALLOC(s->d_status, 1);
  p.planes = p.planes_out = s->state;
  p.key = key;
  p.grid = grid;
  p.grid_b = grid_b;
  p.group = group;
  p.act_dir = act_dir;
  p.act = act;
  p.act_grad = act_grad;
  p.sig_contrib = sig;
  p.status = s->d_status;
  // controller
  CtrlPar& cp = s->ctrl;
  cp.type = d->ctrl_type;
  cp.G = s->G;
  cp.dim = dim;
  cp.hidden = d->ctrl_hidden;
  cp.freq = d->ctrl_freq;
  cp.scale = d->ctrl_scale;
  cp.inv_n = s->N > 0 ? 1.0f / float(s->N) : 0.0f;
  float *params, *gparams, *inv_count, *centroid, *gz, *partials;
  ALLOC(params, std::max(1, np));
  ALLOC(gparams, std::max(1, np));
  ALLOC(inv_count, std::max(1, s->G));
  ALLOC(centroid, MAX_GROUPS * 3 + 3);
  ALLOC(gz, MAX_GROUPS * 3);
  const int rows = std::max(1, reduction_rows(s->N));
  ALLOC(partials, size_t(rows) * RED_ROW_FLOATS);
  cp.params = params;
  cp.gparams = gparams;
  cp.inv_count = inv_count;
  cp.centroid = centroid;
  cp.gz = gz;
  cp.partials = partials;
  cp.n_partials = rows;
  // batch of one
  BatchDev& b = s->b;
  b.n_scenes = 1;
  b.total_particles = s->N;
  b.total_tiles = p.n_tiles;
  const int NB = block_nodes(dim);
  int* pbase;
  ALLOC(pbase, 2);
  int* tile_scene;
  ALLOC(tile_scene, p.n_tiles);
  ALLOC(b.tile_count, p.n_tiles);
  ALLOC(b.tile_fill, p.n_tiles);
  ALLOC(b.tile_start, p.n_tiles + 1);
  ALLOC(b.tile_slot, p.n_tiles);
  ALLOC(b.active, p.n_tiles);
  ALLOC(b.n_active, 1);
  ALLOC(b.block_sums, 2 * ((p.n_tiles + 8191) / 8192) + 2);
  ALLOC(b.sorted, s->npad);
  if (s->impl == MPM_IMPL_TILED) {
    ALLOC(b.partial, size_t(p.n_tiles) * NB);
    ALLOC(b.partial_b, size_t(p.n_tiles) * NB);
  }
#undef ALLOC
  b.scene_pbase = pbase;
  b.tile_scene = tile_scene;
  b.max_ctas = c->sm_count * 4;
  b.p2g_block = 256;
  cudaStream_t stream = c->stream;
  // zero-initialised counters and scene tables
  if ((st = cuda_fail(cudaMemsetAsync(b.tile_count, 0, sizeof(uint32_t) * p.n_tiles, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(b.tile_fill, 0, sizeof(uint32_t) * p.n_tiles, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(tile_scene, 0, sizeof(int) * p.n_tiles, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(s->d_status, 0, sizeof(int), stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(s->d_step, 0, sizeof(int), stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(grid, 0, sizeof(float4) * s->n_nodes, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(grid_b, 0, sizeof(float4) * s->n_nodes, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(group, 0xff, sizeof(int32_t) * s->npad, stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemsetAsync(sig, 0, sizeof(float) * s->npad, stream))) != MPM_OK) return fail(st);
  {
    int hb[2] = {0, s->N};
    if ((st = cuda_fail(cudaMemcpy(pbase, hb, sizeof(hb), cudaMemcpyHostToDevice))) != MPM_OK) return fail(st);
  }
  // inputs
  const size_t xb = sizeof(float) * size_t(s->N) * dim, mb = xb * dim;
  if ((st = ensure_scratch(s, 2 * xb + 2 * mb + sizeof(int32_t) * s->N + 64 * 4)) != MPM_OK) return fail(st);
  const void *x0, *v0, *C0, *F0, *grp;
  if ((st = stage(s, d->x0, xb, d->mem_space, 0, &x0)) != MPM_OK) return fail(st);
  if ((st = stage(s, d->v0, xb, d->mem_space, xb, &v0)) != MPM_OK) return fail(st);
  if ((st = stage(s, d->C0, mb, d->mem_space, 2 * xb, &C0)) != MPM_OK) return fail(st);
  if ((st = stage(s, d->F0, mb, d->mem_space, 2 * xb + mb, &F0)) != MPM_OK) return fail(st);
  if ((st = stage(s, d->group, sizeof(int32_t) * s->N, d->mem_space, 2 * xb + 2 * mb, &grp)) != MPM_OK) return fail(st);
  if ((st = cuda_fail(launch_pack(dim, s->N, s->npad, (const float*)x0, (const float*)v0, (const float*)C0,
                                  (const float*)F0, s->state, s->d_status, stream))) != MPM_OK)
    return fail(st);
  if (grp && s->N > 0) {
    if ((st = cuda_fail(cudaMemcpyAsync(group, grp, sizeof(int32_t) * s->N, cudaMemcpyDeviceToDevice, stream))) != MPM_OK)
      return fail(st);
  }
  if ((st = cuda_fail(cudaStreamSynchronize(stream))) != MPM_OK) return fail(st);
  // small per-group arrays go through the host so group sizes can be counted there
  std::vector<float> hdir(std::max(1, s->G * dim), 0.f), hparams(std::max(1, np), 0.f), hinv(std::max(1, s->G), 0.f);
  std::vector<int32_t> hgroup(s->N, -1);
  {
    cudaMemcpyKind k = d->mem_space == 1 ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    if (s->G > 0 && (st = cuda_fail(cudaMemcpy(hdir.data(), d->act_dir, sizeof(float) * s->G * dim, k))) != MPM_OK)
      return fail(st);
    if (np > 0 && (st = cuda_fail(cudaMemcpy(hparams.data(), d->ctrl_params, sizeof(float) * np, k))) != MPM_OK)
      return fail(st);
    if (d->group && s->N > 0 &&
        (st = cuda_fail(cudaMemcpy(hgroup.data(), d->group, sizeof(int32_t) * s->N, k))) != MPM_OK)
      return fail(st);
  }
  std::vector<int> count(std::max(1, s->G), 0);
  for (int i = 0; i < s->N; ++i)
    if (hgroup[i] >= 0 && hgroup[i] < s->G) count[hgroup[i]]++;
  for (int g = 0; g < s->G; ++g) hinv[g] = count[g] > 0 ? 1.0f / float(count[g]) : 0.0f;
  if ((st = cuda_fail(cudaMemcpy(act_dir, hdir.data(), sizeof(float) * hdir.size(), cudaMemcpyHostToDevice))) != MPM_OK)
    return fail(st);
  if ((st = cuda_fail(cudaMemcpy(params, hparams.data(), sizeof(float) * hparams.size(), cudaMemcpyHostToDevice))) != MPM_OK)
    return fail(st);
  if ((st = cuda_fail(cudaMemcpy(inv_count, hinv.data(), sizeof(float) * hinv.size(), cudaMemcpyHostToDevice))) != MPM_OK)
    return fail(st);
  std::vector<ScenePar> confs(1, conf_fwd(s, s->state, s->state));
  if ((st = upload_conf(s, 0, confs, nullptr)) != MPM_OK) return fail(st);
  if ((st = refresh_keys(s)) != MPM_OK) return fail(st);
  int v = 0;
  if ((st = cuda_fail(cudaStreamSynchronize(stream))) != MPM_OK) return fail(st);
  if ((st = cuda_fail(cudaMemcpy(&v, s->d_status, sizeof(int), cudaMemcpyDeviceToHost))) != MPM_OK) return fail(st);
  if (v != 0) return fail(mpm_status(v));
  *out = s;
  return MPM_OK;
}

mpm_status mpm_scene_info(const mpm_scene* s, int* n_particles, int* n_groups, int* n_ctrl_params, int* step,
                          size_t* state_bytes) {
  if (!s) return MPM_ERR_ARG;
  if (n_particles) *n_particles = s->N;
  if (n_groups) *n_groups = s->G;
  if (n_ctrl_params) *n_ctrl_params = s->nparams;
  if (step) *step = s->step;
  if (state_bytes) *state_bytes = s->state_bytes;
  return MPM_OK;
}

mpm_status mpm_step(mpm_scene* s, int n_steps) {
  if (!s || n_steps < 0) return MPM_ERR_ARG;
  s->have_rollout = false;
  for (int i = 0; i < n_steps; ++i) CKS(forward_step(s, s->dconf, s->hp, s->d_step));
  s->step += n_steps;
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_rollout(mpm_scene* s, int T, int k, size_t budget) {
  if (!s || T < 1 || k < 0) return MPM_ERR_ARG;
  s->have_rollout = false;
  const size_t S = s->state_bytes;
  if (k == 0) {
    if (budget == 0 || size_t(T) * S <= budget) {
      k = 1;
    } else {
      k = int(std::ceil(std::sqrt(double(T))));
    }
  }
  k = std::min(k, T);
  const int nseg = (T + k - 1) / k;
  const size_t need = (size_t(nseg) + size_t(k - 1)) * S;
  if (budget != 0 && need > budget) return MPM_ERR_OOM;
  if (int(s->ckpt.size()) != nseg || int(s->seg.size()) != k - 1) {
    free_rollout(s);  // buffers of another shape
    s->ckpt.assign(nseg, nullptr);
    for (int i = 0; i < nseg; ++i) {
      mpm_status st = dalloc(s, &s->ckpt[i], S / sizeof(float4), s->roll_allocs);
      if (st != MPM_OK) {
        free_rollout(s);
        return st;
      }
    }
    s->seg.assign(std::max(0, k - 1), nullptr);
    for (int i = 0; i < k - 1; ++i) {
      mpm_status st = dalloc(s, &s->seg[i], S / sizeof(float4), s->roll_allocs);
      if (st != MPM_OK) {
        free_rollout(s);
        return st;
      }
    }
  }
  // records: [0] state->state, [1 + 2j] state->ckpt[j], [2 + 2j] ckpt[j]->state, then (k = 1)
  // ckpt[n] -> ckpt[n+1]; every stored state is written by the step that produces it.
  std::vector<ScenePar> confs;
  confs.push_back(conf_fwd(s, s->state, s->state));
  for (int j = 0; j < nseg; ++j) {
    confs.push_back(conf_fwd(s, s->state, s->ckpt[j]));
    confs.push_back(conf_fwd(s, s->ckpt[j], s->state));
  }
  std::vector<int> cidx(T);
  for (int n = 0; n < T; ++n) {
    const bool from_ck = (n % k) == 0;
    const bool to_ck = ((n + 1) % k) == 0 && (n + 1) / k < nseg;
    if (from_ck && to_ck) {
      cidx[n] = int(confs.size());
      confs.push_back(conf_fwd(s, s->ckpt[n / k], s->ckpt[(n + 1) / k]));
    } else if (from_ck) {
      cidx[n] = 2 + 2 * (n / k);
    } else if (to_ck) {
      cidx[n] = 1 + 2 * ((n + 1) / k);
    } else {
      cidx[n] = 0;
    }
  }
  ScenePar* table = nullptr;
  CKS(upload_conf(s, 1, confs, &table));
  cudaStream_t st = s->ctx->stream;
  CK(cudaMemcpyAsync(s->ckpt[0], s->state, S, cudaMemcpyDeviceToDevice, st));
  for (int n = 0; n < T; ++n) CKS(forward_step(s, table + cidx[n], confs[cidx[n]], s->d_step));
  s->roll_T = T;
  s->roll_k = k;
  s->roll_nseg = nseg;
  s->roll_start = s->step;
  s->step += T;
  s->have_rollout = true;
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_backward(mpm_scene* s, const float* gxT, const float* gvT, const float* gCT, const float* gFT,
                        float* gx0, float* gv0, float* gC0, float* gF0, float* gctrl, int mem_space) {
  if (!s || (mem_space != 0 && mem_space != 1)) return MPM_ERR_ARG;
  if (!s->have_rollout) return MPM_ERR_STATE;
  cudaStream_t st = s->ctx->stream;
  const int dim = s->dim, N = s->N, T = s->roll_T, k = s->roll_k, nseg = s->roll_nseg;
  const size_t xb = sizeof(float) * size_t(N) * dim, mb = xb * dim;
  CKS(ensure_scratch(s, 2 * xb + 2 * mb + 64));
  const void *a, *bv, *c, *f;
  CKS(stage(s, gxT, xb, mem_space, 0, &a));
  CKS(stage(s, gvT, xb, mem_space, xb, &bv));
  CKS(stage(s, gCT, mb, mem_space, 2 * xb, &c));
  CKS(stage(s, gFT, mb, mem_space, 2 * xb + mb, &f));
  // seed: F seed defaults to 0 (not identity) for adjoints
  CK(cudaMemsetAsync(s->adj[0], 0, s->state_bytes, st));
  {
    // pack with F = 0 when absent: pack writes identity for a NULL F, so pass zeros explicitly
    if (!f && N > 0) {
      CK(cudaMemsetAsync(reinterpret_cast<char*>(s->scratch) + 2 * xb + mb, 0, mb, st));
      f = reinterpret_cast<char*>(s->scratch) + 2 * xb + mb;
    }
    const float* xs = a ? (const float*)a : nullptr;
    if (!xs && N > 0) {
      CK(cudaMemsetAsync(s->scratch, 0, xb, st));
      xs = (const float*)s->scratch;
    }
    CK(launch_pack(dim, N, s->npad, xs, (const float*)bv, (const float*)c, (const float*)f, s->adj[0], s->d_status,
                   st));
  }
  CK(cudaMemsetAsync(s->ctrl.gparams, 0, sizeof(float) * std::max(1, s->nparams), st));
  // records for every segment: recompute F_{s,j} then reverse B_{s,n,parity}
  std::vector<ScenePar> confs;
  std::vector<int> seg_c0(nseg);
  for (int sg = 0; sg < nseg; ++sg) {
    const int L = std::min(k, T - sg * k);
    seg_c0[sg] = int(confs.size());
    auto segp = [&](int j) { return j == 0 ? s->ckpt[sg] : s->seg[j - 1]; };
    for (int j = 0; j + 1 < L; ++j) confs.push_back(conf_fwd(s, segp(j), segp(j + 1)));
    for (int n = 0; n < L; ++n) {
      confs.push_back(conf_bwd(s, segp(n), s->adj[0], s->adj[1]));
      confs.push_back(conf_bwd(s, segp(n), s->adj[1], s->adj[0]));
    }
  }
  ScenePar* table = nullptr;
  CKS(upload_conf(s, 2, confs, &table));
  CKS(set_counter(s, s->d_bstep, s->roll_start + T - 1));
  int cur = 0;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int L = std::min(k, T - sg * k);
    const int c0 = seg_c0[sg];
    if (L > 1) {
      // bin keys of the checkpoint the recompute starts from
      if (s->impl != MPM_IMPL_PLAIN) {
        BatchDev bb = s->b;
        bb.scenes = table + c0;
        CK(s->dim == 2 ? launch_keys<2>(bb, st) : launch_keys<3>(bb, st));
      }
      CKS(set_counter(s, s->d_step, s->roll_start + sg * k));
      for (int j = 0; j + 1 < L; ++j) CKS(forward_step(s, table + c0 + j, confs[c0 + j], s->d_step));
    }
    for (int n = L - 1; n >= 0; --n) {
      const int ci = c0 + (L - 1) + 2 * n + cur;
      CKS(reverse_step(s, table + ci, confs[ci]));
      cur ^= 1;
    }
  }
  // outputs
  const float4* res = s->adj[cur];
  if (mem_space == 1) {
    CK(launch_unpack(dim, N, s->npad, res, gx0, gv0, gC0, gF0, st));
    if (gctrl && s->nparams > 0)
      CK(cudaMemcpyAsync(gctrl, s->ctrl.gparams, sizeof(float) * s->nparams, cudaMemcpyDeviceToDevice, st));
  } else {
    CKS(ensure_scratch(s, 2 * xb + 2 * mb + 64));
    char* sc = reinterpret_cast<char*>(s->scratch);
    float* dx_ = (float*)sc;
    float* dv_ = (float*)(sc + xb);
    float* dC_ = (float*)(sc + 2 * xb);
    float* dF_ = (float*)(sc + 2 * xb + mb);
    CK(launch_unpack(dim, N, s->npad, res, dx_, dv_, dC_, dF_, st));
    if (gx0) CK(cudaMemcpyAsync(gx0, dx_, xb, cudaMemcpyDeviceToHost, st));
    if (gv0) CK(cudaMemcpyAsync(gv0, dv_, xb, cudaMemcpyDeviceToHost, st));
    if (gC0) CK(cudaMemcpyAsync(gC0, dC_, mb, cudaMemcpyDeviceToHost, st));
    if (gF0) CK(cudaMemcpyAsync(gF0, dF_, mb, cudaMemcpyDeviceToHost, st));
    if (gctrl && s->nparams > 0)
      CK(cudaMemcpyAsync(gctrl, s->ctrl.gparams, sizeof(float) * s->nparams, cudaMemcpyDeviceToHost, st));
  }
  // the keys now describe state 0 of the rollout; restore those of the current state
  CKS(refresh_keys(s));
  return read_status(s);
}

mpm_status mpm_get_state(mpm_scene* s, int step, float* x, float* v, float* C, float* F, int mem_space) {
  if (!s || (mem_space != 0 && mem_space != 1)) return MPM_ERR_ARG;
  const float4* src = s->state;
  if (step >= 0) {
    if (!s->have_rollout) return MPM_ERR_STATE;
    const int local = step - s->roll_start;
    if (local < 0 || local % s->roll_k != 0 || local / s->roll_k >= s->roll_nseg) return MPM_ERR_ARG;
    src = s->ckpt[local / s->roll_k];
  }
  cudaStream_t st = s->ctx->stream;
  const int dim = s->dim, N = s->N;
  const size_t xb = sizeof(float) * size_t(N) * dim, mb = xb * dim;
  if (mem_space == 1) {
    CK(launch_unpack(dim, N, s->npad, src, x, v, C, F, st));
  } else {
    CKS(ensure_scratch(s, 2 * xb + 2 * mb + 64));
    char* sc = reinterpret_cast<char*>(s->scratch);
    CK(launch_unpack(dim, N, s->npad, src, (float*)sc, (float*)(sc + xb), (float*)(sc + 2 * xb),
                     (float*)(sc + 2 * xb + mb), st));
    if (x) CK(cudaMemcpyAsync(x, sc, xb, cudaMemcpyDeviceToHost, st));
    if (v) CK(cudaMemcpyAsync(v, sc + xb, xb, cudaMemcpyDeviceToHost, st));
    if (C) CK(cudaMemcpyAsync(C, sc + 2 * xb, mb, cudaMemcpyDeviceToHost, st));
    if (F) CK(cudaMemcpyAsync(F, sc + 2 * xb + mb, mb, cudaMemcpyDeviceToHost, st));
  }
  return read_status(s);
}

mpm_status mpm_set_state(mpm_scene* s, const float* x, const float* v, const float* C, const float* F, int step,
                         int mem_space) {
  if (!s || (mem_space != 0 && mem_space != 1) || (s->N > 0 && !x)) return MPM_ERR_ARG;
  s->have_rollout = false;
  cudaStream_t st = s->ctx->stream;
  const int dim = s->dim, N = s->N;
  const size_t xb = sizeof(float) * size_t(N) * dim, mb = xb * dim;
  CKS(ensure_scratch(s, 2 * xb + 2 * mb + 64));
  const void *a, *b, *c, *f;
  CKS(stage(s, x, xb, mem_space, 0, &a));
  CKS(stage(s, v, xb, mem_space, xb, &b));
  CKS(stage(s, C, mb, mem_space, 2 * xb, &c));
  CKS(stage(s, F, mb, mem_space, 2 * xb + mb, &f));
  CK(cudaMemsetAsync(s->d_status, 0, sizeof(int), st));
  CK(launch_pack(dim, N, s->npad, (const float*)a, (const float*)b, (const float*)c, (const float*)f, s->state,
                 s->d_status, st));
  if (step >= 0) {
    CKS(set_counter(s, s->d_step, step));
    s->step = step;
  }
  CKS(refresh_keys(s));
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_set_ctrl_params(mpm_scene* s, const float* params, int n, int mem_space) {
  if (!s || n != s->nparams || (n > 0 && !params)) return MPM_ERR_ARG;
  if (n == 0) return MPM_OK;
  CK(cudaStreamSynchronize(s->ctx->stream));
  CK(cudaMemcpy(const_cast<float*>(s->ctrl.params), params, sizeof(float) * n,
                mem_space == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  return MPM_OK;
}

mpm_status mpm_get_grid(mpm_scene* s, float* m, float* v, int mem_space) {
  if (!s || (mem_space != 0 && mem_space != 1)) return MPM_ERR_ARG;
  CK(cudaStreamSynchronize(s->ctx->stream));
  std::vector<float4> h(s->n_nodes);
  CK(cudaMemcpy(h.data(), s->hp.grid, sizeof(float4) * s->n_nodes, cudaMemcpyDeviceToHost));
  const int dim = s->dim;
  std::vector<float> hm(s->n_nodes), hv(size_t(s->n_nodes) * dim);
  for (int i = 0; i < s->n_nodes; ++i) {
    const float c[4] = {h[i].x, h[i].y, h[i].z, h[i].w};
    hm[i] = c[dim];
    for (int a = 0; a < dim; ++a) hv[size_t(i) * dim + a] = c[a];
  }
  cudaMemcpyKind kk = mem_space == 1 ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  if (m) CK(cudaMemcpy(m, hm.data(), sizeof(float) * hm.size(), kk));
  if (v) CK(cudaMemcpy(v, hv.data(), sizeof(float) * hv.size(), kk));
  return read_status(s);
}

mpm_status mpm_profile_start(mpm_ctx* c, unsigned mask, int max_launches) {
  if (!c || max_launches < 0) return MPM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  const size_t need = 2 * size_t(max_launches);
  while (c->prof_ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    c->prof_ev.push_back(e);
  }
  c->prof_kind.assign(max_launches, -1);
  c->prof_used = 0;
  c->prof_mask = mask;
  return MPM_OK;
}

mpm_status mpm_profile_read(mpm_ctx* c, int kind, int* count, double* total_ms) {
  if (!c || kind < 0 || kind >= MPM_K_COUNT) return MPM_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  int n = 0;
  double t = 0.0;
  for (int i = 0; i < c->prof_used; ++i) {
    if (c->prof_kind[i] != kind) continue;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    t += ms;
    ++n;
  }
  if (count) *count = n;
  if (total_ms) *total_ms = t;
  return MPM_OK;
}

mpm_status mpm_launch_count(long long* count) {
  if (!count) return MPM_ERR_ARG;
  *count = launch_total();
  return MPM_OK;
}

}  // extern "C"
