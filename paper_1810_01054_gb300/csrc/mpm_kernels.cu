// sm_103a kernels of the differentiable MLS-MPM step (ChainQueen, arXiv 1810.01054).
//
// Forward step (Section III, Eqs. 3-10), tiled form:
//   k_hist / scan / k_scatter : bin particles by the tile of their stencil base cell
//   k_p2g                     : per tile, canonical (cell, id) order, per-particle stress and
//                               MLS matrix G (Eq. 4), per-cell register accumulation of the
//                               3^d stencil (Eqs. 3, 5), fixed-order reduction into the tile's
//                               (B+2)^d node block -- no atomics on floating point anywhere
//   k_grid                    : sums the <= 2^d node blocks covering each node in a fixed order,
//                               Eq. 6, gravity, boundary (S5)
//   k_g2p                     : per tile, node block staged in shared memory, Eqs. 7-10 and the
//                               next step's bin key
// Reverse step (Supplement S2-S5): k_p2g also scatters (C) from (A), (B) in the same pass; k_grid
// applies (L), (D), (E); k_adj_gather evaluates (F)-(K), (J).
//
// Every floating-point sum has a fixed order, so results are bitwise reproducible run to run and
// independent of which other scenes share the launch.
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "mpm_internal.h"

namespace gbmpm {

static std::atomic<long long> g_launches{0};
static thread_local long long* t_capture = nullptr;
void capture_tally(long long* tally) { t_capture = tally; }
void count_launches(int n) {
  if (t_capture)
    *t_capture += n;
  else
    g_launches.fetch_add(n, std::memory_order_relaxed);
}
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }

// ============================================================================ helpers
__device__ __forceinline__ int find_scene(const int* __restrict__ pbase, int n_scenes, int gp) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(pbase + mid) <= gp)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ctr[t] += 1 for every active lane's t (t < 0: nothing); returns the old value plus the lane's rank
// among the lanes with the same t -- one atomic per distinct t in the warp.
__device__ __forceinline__ uint32_t warp_aggregated_inc(uint32_t* ctr, int t) {
  const unsigned mask = __activemask();
  const unsigned peers = __match_any_sync(mask, t);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader && t >= 0) base = atomicAdd(ctr + t, uint32_t(__popc(peers)));
  base = __shfl_sync(peers, base, leader);
  return base + uint32_t(__popc(peers & ((1u << lane) - 1u)));
}

template <int D>
__device__ __forceinline__ int lin3(const int* c, const int* n) {
  int l = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) l = l * n[a] + c[a];
  return l;
}

template <int D>
__device__ __forceinline__ void unlin(int l, const int* n, int* c) {
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    c[a] = l % n[a];
    l /= n[a];
  }
}

template <int D, int TB>
__device__ __forceinline__ int cell_lin(const int* c) {
  constexpr int B = Tile<D, TB>::B;
  int l = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) l = l * B + c[a];
  return l;
}

// Bin key of a particle at x: (scene-local tile << 6) | cell within the tile (TB^D-cell tiles).
template <int D, int TB>
__device__ __forceinline__ uint32_t bin_key(const float* x, const ScenePar& sp) {
  constexpr int B = Tile<D, TB>::B;
  int base[D];
  float f[D];
  if (!stencil_base<D>(x, sp.inv_dx, sp.n, base, f)) {
    set_status(sp.status, ST_DOMAIN);
    return KEY_INVALID;
  }
  int t[D], c[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    t[a] = base[a] / B;
    c[a] = base[a] - t[a] * B;
  }
  return (uint32_t(lin3<D>(t, sp.nt)) << 6) | uint32_t(cell_lin<D, TB>(c));
}

// Actuation group of particle id (-1: none).
__device__ __forceinline__ int group_of(const ScenePar& sp, int id) {
  const int g = sp.group ? __ldg(sp.group + id) : -1;
  return g < sp.G ? g : -1;
}

// Actuation stress diagonal of a particle of group g: sigma_a = a_g Diag(dir_g) (Section III).
template <int D>
__device__ __forceinline__ void actuation(const ScenePar& sp, int g, float* sig) {
  float a = g >= 0 ? __ldg(sp.act + g) : 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) sig[k] = g >= 0 ? a * __ldg(sp.act_dir + g * D + k) : 0.0f;
}

// Material of particle id: the scene's, or its own Young's modulus and mass when the scene has
// per-particle arrays (Lame parameters E_p x the scene's per-unit-E factors).
struct PMat {
  Material mat;
  float mass;
};
__device__ __forceinline__ PMat pmat_of(const ScenePar& sp, int id) {
  PMat r{sp.mat, sp.mass};
  if (sp.pE) {
    const float E = __ldg(sp.pE + id);
    r.mat.mu = E * sp.mu_per_E;
    r.mat.la = E * sp.la_per_E;
  }
  if (sp.pmass) r.mass = __ldg(sp.pmass + id);
  return r;
}

// Per-particle quantities of P2G for a particle of group g and material pm: stress with
// actuation and G of Eq. 4.  Returns J.
template <int D>
__device__ __forceinline__ float particle_G(const Part<D>& q, const ScenePar& sp, int g, const PMat& pm,
                                            float (&P)[D][D], float (&A)[D][D], float (&G)[D][D], float* sig) {
  actuation<D>(sp, g, sig);
  float J = stress<D>(q.F, pm.mat, sig, P, A);
  float kG = -4.0f * sp.inv_dx * sp.inv_dx * sp.dt * sp.vol;
  mls_G<D>(P, q.F, q.C, kG, pm.mass, G);
  return J;
}

// ============================================================================ record selection
// Scene record of step n = *ctr: table[map[n - base]] (map NULL: table[0]) with the batch offsets
// patched in, copied to dst by the calling CTA's threads (no barrier: each thread writes its own
// words, the offsets in place of the copied ones).
__device__ __forceinline__ int selected_index(const SelectPar& q, int n) { return q.map ? q.map[n - q.base] : 0; }

// Word i of pointer v (little-endian halves).
__device__ __forceinline__ int ptr_word(const void* v, int i) {
  const unsigned long long u = reinterpret_cast<unsigned long long>(v);
  return int(uint32_t(i ? u >> 32 : u));
}

__device__ __forceinline__ void select_copy(const SelectPar& q, int n, ScenePar* dst) {
  const int* src = reinterpret_cast<const int*>(q.table + selected_index(q, n));
  int* d = reinterpret_cast<int*>(dst);
  constexpr int W = int(sizeof(ScenePar) / sizeof(int));
  constexpr int TB = int(offsetof(ScenePar, tile_base) / sizeof(int));
  constexpr int PB = int(offsetof(ScenePar, pbase) / sizeof(int));
  constexpr int KO = int(offsetof(ScenePar, key) / sizeof(int));
  constexpr int AO = int(offsetof(ScenePar, act) / sizeof(int));
  static_assert(offsetof(ScenePar, key) % 8 == 0 && offsetof(ScenePar, act) % 8 == 0, "pointer words");
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    int v = i == TB ? q.tile_base : (i == PB ? q.pbase : src[i]);
    if (q.key_rec && (i == KO || i == KO + 1)) v = ptr_word(q.key_rec, i - KO);
    if (q.act_rec && (i == AO || i == AO + 1)) v = ptr_word(q.act_rec, i - AO);
    d[i] = v;
  }
}

// The selection of step n for one scene: its record into cur, and the sinusoid and table
// controllers' actuation a_g(t_n) into q.act.
__device__ __forceinline__ void select_publish_at(const SelectPar& q, int n, ScenePar* cur) {
  select_copy(q, n, cur);
  const float tt = float(n) * q.dt;
  const int g = threadIdx.x;
  if (g < q.G && q.ctrl_type == 0) {
    q.act[g] = q.params[g] * sinf(6.283185307179586f * q.freq * tt);
  } else if (g < q.G && q.ctrl_type == 1) {
    const float w = 6.283185307179586f * q.freq * tt;
    q.act[g] = q.params[g * 4] * sinf(w) + q.params[g * 4 + 1] * cosf(w) + q.params[g * 4 + 2] * sinf(2.0f * w) +
               q.params[g * 4 + 3] * cosf(2.0f * w);
  } else if (g < q.G && q.ctrl_type == 3) {
    q.act[g] = (n >= 0 && n < q.ctrl_len) ? q.params[size_t(n) * q.G + g] : 0.0f;
  }
}

// The selection of the step the counter names.
__device__ __forceinline__ void select_publish(const SelectPar& q, ScenePar* cur) { select_publish_at(q, *q.ctr, cur); }

// ============================================================================ keys / sort
// Bin keys of the state being read, and the tile histogram (tile_count must be zero on entry).
// With SEL (a single scene) the kernel also makes the step's selection: every CTA copies the
// selected record to shared memory for its own use and CTA 0 publishes it (and the actuation) for
// the kernels that follow, which replaces the selection launch.
template <int D, int TB, bool SEL>
__global__ void k_keys(BatchDev b, const SelectPar* __restrict__ sel) {
  pdl_enter();
  __shared__ __align__(16) ScenePar srec[1];
  if constexpr (SEL) {
    const int n = *sel->ctr;
    select_copy(*sel, n, srec);
    if (blockIdx.x == 0) select_publish(*sel, b.scenes);
    __syncthreads();
  }
  int gp = blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= b.total_particles) return;
  const ScenePar& sp = SEL ? srec[0] : b.scenes[find_scene(b.scene_pbase, b.n_scenes, gp)];
  int p = gp - sp.pbase;
  float4 q = sp.planes[p];
  float x[3] = {q.x, q.y, q.z};
  const uint32_t k = bin_key<D, TB>(x, sp);
  sp.key[p] = k;
  warp_aggregated_inc(b.tile_count, k != KEY_INVALID ? int(sp.tile_base + (k >> 6)) : -1);
}

// Exclusive block scan of (sum, count) pairs over blockDim.x <= 1024 threads.
__device__ __forceinline__ void block_scan2(uint32_t& a, uint32_t& c, uint32_t& tot_a, uint32_t& tot_c) {
  __shared__ uint32_t wa[32], wc[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t ia = a, ic = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t ta = __shfl_up_sync(0xffffffffu, ia, o), tc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      ia += ta;
      ic += tc;
    }
  }
  if (lane == 31) {
    wa[w] = ia;
    wc[w] = ic;
  }
  __syncthreads();
  if (w == 0) {
    uint32_t xa = lane < nw ? wa[lane] : 0u, xc = lane < nw ? wc[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t ta = __shfl_up_sync(0xffffffffu, xa, o), tc = __shfl_up_sync(0xffffffffu, xc, o);
      if (lane >= o) {
        xa += ta;
        xc += tc;
      }
    }
    wa[lane] = xa;
    wc[lane] = xc;
  }
  __syncthreads();
  uint32_t pa = w > 0 ? wa[w - 1] : 0u, pc = w > 0 ? wc[w - 1] : 0u;
  tot_a = wa[nw - 1];
  tot_c = wc[nw - 1];
  a = pa + ia - a;
  c = pc + ic - c;
  __syncthreads();
}

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 2;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;
// Small batches scan the tile histogram inside the scatter kernel (k_scatter<D, true>); the P2G
// that follows every scatter clears the counters.
__host__ __device__ __forceinline__ bool fused_scan(const BatchDev& b) { return b.total_tiles <= SCAN_TILE; }

// Phase 1 of the tile scan: per-block totals of particle counts and of active tiles.
template <bool SEL>
__global__ void k_scan_reduce(BatchDev b, const SelectPar* __restrict__ sel) {
  pdl_enter();
  if (SEL && blockIdx.x == gridDim.x - 1) {  // an extra CTA makes the step's selection (k_scatter)
    select_publish(*sel, b.scenes);
    return;
  }
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
  uint32_t s = 0, c = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    int t = base + i;
    if (t < b.total_tiles) {
      uint32_t v = b.tile_count[t];
      s += v;
      c += v > 0;
    }
  }
  uint32_t ta, tc;
  block_scan2(s, c, ta, tc);
  if (threadIdx.x == 0) {
    b.block_sums[2 * blockIdx.x] = ta;
    b.block_sums[2 * blockIdx.x + 1] = tc;
  }
}

// Phase 2: tile_start, tile_slot, active list, n_active; resets the per-step counters for the
// next step.
__global__ void k_scan_down(BatchDev b) {
  pdl_enter();
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
  uint32_t cnt[SCAN_PER_THREAD];
  uint32_t s = 0, c = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    int t = base + i;
    cnt[i] = t < b.total_tiles ? b.tile_count[t] : 0u;
    s += cnt[i];
    c += cnt[i] > 0;
  }
  // this block's offsets: the totals of the blocks before it (one warp; a few dozen at most)
  __shared__ uint32_t boff[2];
  if (threadIdx.x < 32) {
    uint32_t a = 0, n = 0;
    for (int i = threadIdx.x; i < int(blockIdx.x); i += 32) {
      a += b.block_sums[2 * i];
      n += b.block_sums[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if (threadIdx.x == 0) {
      boff[0] = a;
      boff[1] = n;
    }
  }
  uint32_t ts, tc;
  block_scan2(s, c, ts, tc);  // its barriers publish boff
  s += boff[0];
  c += boff[1];
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; ++i) {
    int t = base + i;
    if (t < b.total_tiles) {
      b.tile_start[t] = s;
      if (cnt[i] > 0) {
        b.tile_slot[t] = int(c);
        b.active[c] = t;
        ++c;
      } else {
        b.tile_slot[t] = -1;
      }
      s += cnt[i];
      b.tile_count[t] = 0u;
      b.tile_fill[t] = 0u;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
    b.tile_start[b.total_tiles] = s;
    *b.n_active = int(c);
  }
}

// Scatter of the particles into their tiles' ranges of `sorted`.  With FUSED (total_tiles <=
// SCAN_TILE) the tile scan is done here instead of by the scan kernels: every CTA scans the whole
// histogram in shared memory (it is small), CTA 0 publishes tile_start, tile_slot, the active list
// and n_active; the P2G that follows clears the per-step counters.
// With SEL (a single scene, fused scan) one extra CTA, launched after the scatter's own, makes the
// step's selection (see k_keys) alongside them; the scatter reads only the record's step-invariant
// fields (keys, offsets, status), which it takes from the phase's first record instead of the
// one being published.
template <int D, bool FUSED, bool SEL>
__global__ void __launch_bounds__(256) k_scatter(BatchDev b, const SelectPar* __restrict__ sel) {
  pdl_enter();
  if (SEL && blockIdx.x == gridDim.x - 1) {
    select_publish(*sel, b.scenes);
    return;
  }
  constexpr int PER = FUSED ? SCAN_TILE / 256 : 1;
  __shared__ uint32_t sstart[FUSED ? SCAN_TILE + 1 : 1];
  if constexpr (FUSED) {
    const int nt = b.total_tiles, t0 = threadIdx.x * PER;
    uint32_t cnt[PER], s = 0, c = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      cnt[i] = t0 + i < nt ? b.tile_count[t0 + i] : 0u;
      s += cnt[i];
      c += cnt[i] > 0;
    }
    uint32_t ts, tc;
    block_scan2(s, c, ts, tc);
    const bool pub = blockIdx.x == 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int t = t0 + i;
      if (t < nt) {
        sstart[t] = s;
        if (pub) {
          b.tile_start[t] = s;
          if (cnt[i] > 0) {
            b.tile_slot[t] = int(c);
            b.active[c] = t;
          } else {
            b.tile_slot[t] = -1;
          }
        }
        s += cnt[i];
        c += cnt[i] > 0;
      }
    }
    if (threadIdx.x == 0) {
      sstart[nt] = ts;
      if (pub) {
        b.tile_start[nt] = ts;
        *b.n_active = int(tc);
      }
    }
    __syncthreads();
  }
  int gp = blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= b.total_particles) return;
  const ScenePar& sp = SEL ? sel->table[0] : b.scenes[find_scene(b.scene_pbase, b.n_scenes, gp)];
  const int pbase = SEL ? sel->pbase : sp.pbase, tbase = SEL ? sel->tile_base : sp.tile_base;
  int p = gp - pbase;
  const uint32_t k = sp.key[p];
  const int t = k != KEY_INVALID ? int(tbase + (k >> 6)) : -1;
  const uint32_t rank = warp_aggregated_inc(b.tile_fill, t);
  if (t < 0) return;
  const uint32_t start = FUSED ? sstart[t] : b.tile_start[t];
  const uint32_t end = FUSED ? sstart[t + 1] : b.tile_start[t + 1];
  if (start + rank >= end) {  // a key the histogram did not count: record it, write nothing
    set_status(sp.status, ST_BINNING);
    return;
  }
  b.sorted[start + rank] = ((k & 63u) << 26) | uint32_t(p);  // cell in tile, particle id
}

// ============================================================================ sort store
// A reverse pass whose recompute runs beside it keeps the sort of every recomputed state: the
// recompute copies it out right after its scatter, the reverse step copies it back instead of
// binning and scattering again.  Single scene; slot layout of sort_slot_words.
// The pieces of one sort: raw tile lists and bin keys (N each), tile_start (nt + 1), tile_slot,
// active (nt each), n_active; copied from the src pointers to the dst pointers.
struct SortRefs {
  uint32_t *sorted, *key, *tstart;
  int *tslot, *active, *n_active;
};

__device__ __forceinline__ SortRefs slot_refs(uint32_t* o, int np, int nt) {
  return {o, o + np, o + 2 * np, reinterpret_cast<int*>(o + 2 * np + nt + 1),
          reinterpret_cast<int*>(o + 2 * np + 2 * nt + 1), reinterpret_cast<int*>(o + 2 * np + 3 * nt + 1)};
}

__device__ __forceinline__ void sort_copy(const SortRefs& src, const SortRefs& dst, int N, int nt) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    dst.sorted[i] = src.sorted[i];
    dst.key[i] = src.key[i];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nt; i += stride) {
    dst.tstart[i] = src.tstart[i];
    if (i < nt) {
      dst.tslot[i] = src.tslot[i];
      dst.active[i] = src.active[i];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst.n_active = *src.n_active;
}

template <int D>
__global__ void __launch_bounds__(256) k_store_sort(BatchDev b, uint32_t* dst) {
  pdl_enter();
  const ScenePar& sp = b.scenes[0];
  uint32_t* slot = dst ? dst : sp.sort_slot;
  if (!slot) return;
  const int nt = b.total_tiles;
  const SortRefs from{b.sorted, sp.key, b.tile_start, b.tile_slot, b.active, b.n_active};
  sort_copy(from, slot_refs(slot, sp.npad, nt), b.total_particles, nt);
}

// Every CTA reads the selected record's slot itself; CTA 0 publishes the record and actuation
// (and, with snap, the selected step number).
template <int D>
__global__ void __launch_bounds__(256) k_load_sort(BatchDev b, const SelectPar* __restrict__ sel, int back,
                                                   int* snap) {
  pdl_enter();
  __shared__ uint32_t* src;
  __shared__ uint32_t* key;
  __shared__ int np;
  const int n = *sel->ctr - back;
  if (threadIdx.x == 0) {
    const ScenePar& r = sel->table[selected_index(*sel, n)];
    src = r.sort_slot;
    key = sel->key_rec ? sel->key_rec : r.key;
    np = r.npad;
  }
  if (blockIdx.x == 0) {
    select_publish_at(*sel, n, b.scenes);
    if (snap && threadIdx.x == 0) *snap = n;
  }
  __syncthreads();
  if (!src) return;  // uniform across the CTA
  const int nt = b.total_tiles;
  const SortRefs to{b.sorted, key, b.tile_start, b.tile_slot, b.active, b.n_active};
  sort_copy(slot_refs(src, np, nt), to, b.total_particles, nt);
}

template <int D>
cudaError_t launch_store_sort(const BatchDev& b, uint32_t* dst, cudaStream_t s) {
  const int n = std::max(b.total_particles, b.total_tiles + 1);
  const int grid = std::max(1, std::min((n + 255) / 256, 4 * b.sm_count));
  launch_pdl(k_store_sort<D>, dim3(grid), dim3(256), 0, s, b, dst);
  count_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_load_sort(const BatchDev& b, const SelectPar* sel, cudaStream_t s, int back, int* snap) {
  const int n = std::max(b.total_particles, b.total_tiles + 1);
  const int grid = std::max(1, std::min((n + 255) / 256, 4 * b.sm_count));
  launch_pdl(k_load_sort<D>, dim3(grid), dim3(256), 0, s, b, sel, back, snap);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_store_sort<2>(const BatchDev&, uint32_t*, cudaStream_t);
template cudaError_t launch_store_sort<3>(const BatchDev&, uint32_t*, cudaStream_t);
template cudaError_t launch_load_sort<2>(const BatchDev&, const SelectPar*, cudaStream_t, int, int*);
template cudaError_t launch_load_sort<3>(const BatchDev&, const SelectPar*, cudaStream_t, int, int*);

// Dynamic tile scheduling (the forward P2G and the adjoint gather, when a launch has more than two
// active tiles per CTA; fewer, and the other tile kernels, measured faster with the fixed stride):
// a CTA takes its first active slot by its index and every later one from the kernel's counter
// work[w], so CTAs that finish early take more tiles.  Which CTA computes a tile changes no bit of
// it.  The last CTA to finish (its ticket in work[w + 2]) puts both words back to zero for the next
// launch.
__device__ __forceinline__ void claim_next(const BatchDev& b, int w, int* s_next, int it) {
  if (threadIdx.x == 0) s_next[it & 1] = int(gridDim.x) + int(atomicAdd(b.work + w, 1u));
}
__device__ __forceinline__ int take_next(const int* s_next, int it) {
  __syncthreads();  // the claim of this iteration is visible (and the one before it consumed)
  return s_next[it & 1];
}
__device__ __forceinline__ void release_work(const BatchDev& b, int w) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(b.work + w + 2, 1u) == gridDim.x - 1) {
      b.work[w] = 0u;
      b.work[w + 2] = 0u;
    }
  }
}

// ============================================================================ P2G (tiled)
// Phase A  canonical order of the tile's particles: by cell, then by particle id (counting sort
//          over the tile's cells, insertion sort inside each cell) -- fixes every later sum order.
// Phase B  one record per particle (fraction f, momentum part a, MLS matrix M = dx G, mass; plus
//          the adjoint-scatter record (C) in the reverse pass), all staged in shared memory.
// Phase C  work item = (cell, part): 2D one stencil node, 3D one x-slab of 9 nodes; a thread
//          accumulates its item over the cell's particles in registers (fixed particle order).
// Phase D  node block = fixed-order sum of the cell stencils covering each node -> global.
template <int D, int TB, bool ADJ, int T = 256>
struct P2GCfg {
  static constexpr int RF = 2 * D + D * D + 1;             // f, a, M, mass
  static constexpr int RA = ADJ ? D + D * D : 0;           // a', M'
  static constexpr int RW = ((RF + RA) % 2 == 0) ? RF + RA + 1 : RF + RA;  // odd stride: no bank conflicts
  static constexpr int CHF = D + 1;                        // momentum + mass
  static constexpr int CHA = ADJ ? D : 0;                  // vbar*
  static constexpr int CH = CHF + CHA;
  // floats per accumulator entry in shared memory: 3D entries are whole float4s (4, or 8 in the
  // reverse pass), read and summed as float4 in phase D
  static constexpr int CHS = D == 3 ? (CH + 3) / 4 * 4 : CH;
  static constexpr int PARTS = D == 2 ? 9 : 3;             // work items per cell
  static constexpr int NK = D == 2 ? 1 : 9;                // stencil nodes per work item
  static constexpr int THREADS = T;
  static constexpr int ITEMS = Tile<D, TB>::CELLS * PARTS;  // 2D 144 (576 with 8 x 8 tiles), 3D 192
  static constexpr int IPT = (ITEMS + T - 1) / T;          // work items per thread
  static constexpr int REC_CAP = D == 2 ? 1024 : 512;      // records staged at once
  static constexpr int CAP = Tile<D, TB>::SORT_CAP;
  static constexpr size_t REC_BYTES = size_t(REC_CAP) * RW * 4;
  static constexpr size_t ACC_BYTES = size_t(Tile<D, TB>::CELLS) * Cfg<D>::STENCIL * CHS * 4;
  static constexpr size_t IDS_BYTES = size_t(CAP) * 4;
  static constexpr size_t U1 = REC_BYTES > ACC_BYTES ? REC_BYTES : ACC_BYTES;
  static constexpr size_t U_BYTES = U1 > IDS_BYTES ? U1 : IDS_BYTES;
  static constexpr size_t SMEM = IDS_BYTES + U_BYTES;
  static_assert(D == 2 || IPT == 1, "a 3D work item holds 9 nodes: one item per thread");
  static_assert(Tile<D, TB>::BLOCK_NODES <= THREADS, "one node per thread in phase D");
};

// T threads per CTA (256; 128 in 2D, where a thread then owns up to two of the 144 work items):
// the work items and every sum keep their order, so T changes no bit of the results.
// Resident CTAs: the 3D forward P2G keeps 3 of 256 threads per SM (85 registers, a few spills in
// its record phase; 4 % faster on the 1M-particle cluster than 2 at 126 registers); the adjoint
// scatter holds 63 accumulators and keeps 2.
template <int D, int TB, bool ADJ, int T>
__global__ void __launch_bounds__(T, T == 256 ? (D == 3 && !ADJ ? 3 : 2) : 4) k_p2g(BatchDev b) {
  pdl_enter();
  using K = P2GCfg<D, TB, ADJ, T>;
  constexpr int B = Tile<D, TB>::B, CELLS = Tile<D, TB>::CELLS, NB = Tile<D, TB>::BLOCK_NODES,
                BN = Tile<D, TB>::BN;
  constexpr int ST = Cfg<D>::STENCIL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* ids = reinterpret_cast<uint32_t*>(smem_raw);
  float* U = reinterpret_cast<float*>(smem_raw + K::IDS_BYTES);
  __shared__ int cstart[CELLS + 1], cfill[CELLS];
  const int tid = threadIdx.x;
  // the CTA's first active tile is requested together with the count (the entry is in bounds
  // whatever the count; it is used only when the slot is below it)
  const int first_gt = b.total_tiles > 0 ? b.active[int(blockIdx.x) < b.total_tiles ? blockIdx.x : 0] : 0;
  const int n_active = *b.n_active;
  // the per-step counters are cleared here whichever scan ran (the fused one leaves them set, the
  // separate one leaves the scatter's fill counts): every step then starts from zero, also when a
  // batch's composition moves it between the two scans
  for (int i = blockIdx.x * blockDim.x + tid; i < b.total_tiles; i += gridDim.x * blockDim.x) {
    b.tile_count[i] = 0u;
    b.tile_fill[i] = 0u;
  }

  __shared__ int s_next[2];
  // the per-cell counters are zero whenever a tile starts: here, and again at the end of every tile
  if (tid < CELLS) cfill[tid] = 0;
  __syncthreads();
  const bool dyn = !ADJ && n_active > 2 * int(gridDim.x);  // uniform across the grid
  int it = 0;
  for (int slot = blockIdx.x; slot < n_active; slot = dyn ? take_next(s_next, it++) : slot + int(gridDim.x)) {
    if (dyn) claim_next(b, 0, s_next, it);
    const int gt = slot == int(blockIdx.x) ? first_gt : b.active[slot];
    const ScenePar& sp = b.scenes[b.n_scenes == 1 ? 0 : b.tile_scene[gt]];
    const uint32_t st = b.tile_start[gt];
    const int cnt = int(b.tile_start[gt + 1] - st);
    if (cnt > K::CAP) {  // the step fails (status); the tile adds nothing to the grid
      if (tid == 0) set_status(sp.status, ST_DENSITY);
      for (int i = tid; i < NB; i += blockDim.x) {
        b.partial[size_t(slot) * NB + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (ADJ) b.partial_b[size_t(slot) * NB + i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;  // uniform across the CTA
    }
    int t[D];
    unlin<D>(gt - sp.tile_base, sp.nt, t);
    // this thread's work items tid + j T: (cell, stencil part)
    bool item_thread[K::IPT];
    int my_cell[K::IPT], my_part[K::IPT], ikx[K::IPT], iky[K::IPT];
    float acc[K::IPT][K::NK][K::CH];  // 2D
    // 3D (one item per thread): the channels in pairs for the packed FP32 FMA, whose halves round
    // exactly as two fmaf: (p_x, p_y), (p_z, m), and in the reverse pass (vbar*_x, vbar*_y), vbar*_z
    float2 aP01[K::NK], aP2m[K::NK], aQ01[K::NK];
    float aQ2[K::NK];
#pragma unroll
    for (int k = 0; k < K::NK; ++k) {
      aP01[k] = aP2m[k] = aQ01[k] = make_float2(0.0f, 0.0f);
      aQ2[k] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < K::IPT; ++j) {
      const int it = tid + j * T;
      item_thread[j] = it < K::ITEMS;
      my_cell[j] = it / K::PARTS;
      my_part[j] = it - K::PARTS * my_cell[j];
      ikx[j] = D == 2 ? my_part[j] / 3 : my_part[j];  // stencil x offset of the item
      iky[j] = D == 2 ? my_part[j] % 3 : 0;           // 2D: stencil y offset of the item
#pragma unroll
      for (int k = 0; k < K::NK; ++k)
#pragma unroll
        for (int c = 0; c < K::CH; ++c) acc[j][k][c] = 0.0f;
    }
    const float dx = sp.dx, dt = sp.dt;
    const float Dx4 = 4.0f * sp.inv_dx;  // (4/dx^2) * dx

    // Phase B for one particle: record of particle `id` (state in r[], bin cell `kc` of its key,
    // actuation group g) at staging row `row`.
    auto make_record = [&](int id, uint32_t kc, int g, float* r, int row) {
      Part<D> q;
      unpack<D>(r, q);
      int base[D];
      float f[D];
      stencil_base<D>(q.x, sp.inv_dx, sp.n, base, f);
      const PMat pm = pmat_of(sp, id);
      // the particle must sit in the cell its key names; otherwise it contributes nothing
      float wm = pm.mass;
      {
        int c[D];
        const int bn[3] = {B, B, B};
        unlin<D>(int(kc), bn, c);
        bool ok = true;
#pragma unroll
        for (int a = 0; a < D; ++a) ok = ok && base[a] == t[a] * B + c[a];
        if (!ok) {
          set_status(sp.status, ST_BINNING);
          wm = 0.0f;
        }
      }
      float P[D][D], A[D][D], G[D][D], sig[D];
      const float J = particle_G<D>(q, sp, g, pm, P, A, G, sig);
      if (!(J > 0.0f)) set_status(sp.status, ST_INVERTED);
      const float keep = wm > 0.0f ? 1.0f : 0.0f;
      float* rec = U + size_t(row) * K::RW;
      int o = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) rec[o++] = f[a];
      // a = m v - dx G f ; M = dx G, since G (x_i - x_p) = dx G (k - f)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < D; ++c) s += G[a][c] * f[c];
        rec[o++] = keep * (pm.mass * q.v[a] - dx * s);
      }
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c) rec[o++] = keep * dx * G[a][c];
      rec[o++] = wm;
      if constexpr (ADJ) {
        // (A) vbar' = gv1 + dt gx1 ; (B) Cbar' = gC1 + dt gF1 F^T ; record of (C):
        // vbar' + (4/dx^2) Cbar' (x_i - x_p) = [vbar' - (4/dx) Cbar' f] + (4/dx) Cbar' k
        float ra[Cfg<D>::S];
        load_planes<D, Cfg<D>::PLANES>(sp.adj_in, sp.npad, id, ra);
        Part<D> g1;
        unpack<D>(ra, g1);
        float vb[D], Cb[D][D];
#pragma unroll
        for (int a = 0; a < D; ++a) vb[a] = g1.v[a] + dt * g1.x[a];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) s += g1.F[a][k] * q.F[c][k];
            Cb[a][c] = g1.C[a][c] + dt * s;
          }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float s = 0.0f;
#pragma unroll
          for (int c = 0; c < D; ++c) s += Cb[a][c] * f[c];
          rec[o++] = keep * (vb[a] - Dx4 * s);
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) rec[o++] = keep * Dx4 * Cb[a][c];
      }
    };

    // Phase C over staged rows [lo, hi) (row = canonical position - c0): this thread's work item j
    // accumulates its stencil nodes over the cell's particles in canonical order.
    auto accumulate = [&](int j, int lo, int hi, int c0) {
      for (int ei = lo; ei < hi; ++ei) {
        const float* rec = U + size_t(ei - c0) * K::RW;
        const float mass = rec[K::RF - 1];
        float w[D][3], dwd[3];
#pragma unroll
        for (int a = 0; a < D; ++a) bspline(rec[a], 1.0f, w[a], dwd);
        const float* av = rec + D;      // a
        const float* Mv = rec + 2 * D;  // M, row-major
        // the item's own offsets select weights by value: a runtime index would put w in local memory
        const float wx = ikx[j] == 0 ? w[0][0] : (ikx[j] == 1 ? w[0][1] : w[0][2]);
        if constexpr (D == 2) {
          const float N = wx * (iky[j] == 0 ? w[1][0] : (iky[j] == 1 ? w[1][1] : w[1][2]));
#pragma unroll
          for (int a = 0; a < D; ++a) acc[j][0][a] += N * (av[a] + Mv[a * D] * float(ikx[j]) + Mv[a * D + 1] * float(iky[j]));
          acc[j][0][D] += N * mass;
          if constexpr (ADJ) {
            const float* aa = rec + K::RF;
            const float* Ma = aa + D;
#pragma unroll
            for (int a = 0; a < D; ++a)
              acc[j][0][K::CHF + a] += N * (aa[a] + Ma[a * D] * float(ikx[j]) + Ma[a * D + 1] * float(iky[j]));
          }
        } else {
          // u = a + M[:,0] kx, then per row + M[:,1] ky and per node + M[:,2] kz (M row-major)
          const float kxf = float(ikx[j]);
          const float2 u01 = __ffma2_rn(make_float2(Mv[0], Mv[3]), make_float2(kxf, kxf), make_float2(av[0], av[1]));
          const float u2s = fmaf(Mv[6], kxf, av[2]);
          float2 q01 = make_float2(0.0f, 0.0f);
          float q2s = 0.0f;
          if constexpr (ADJ) {
            const float* aa = rec + K::RF;
            const float* Ma = aa + D;
            q01 = __ffma2_rn(make_float2(Ma[0], Ma[3]), make_float2(kxf, kxf), make_float2(aa[0], aa[1]));
            q2s = fmaf(Ma[6], kxf, aa[2]);
          }
#pragma unroll
          for (int ky = 0; ky < 3; ++ky) {
            const float wxy = wx * w[1][ky];
            const float kyf = float(ky);
            const float2 v01 = __ffma2_rn(make_float2(Mv[1], Mv[4]), make_float2(kyf, kyf), u01);
            const float v2 = fmaf(Mv[7], kyf, u2s);
            float2 r01 = make_float2(0.0f, 0.0f);
            float r2 = 0.0f;
            if constexpr (ADJ) {
              const float* Ma = rec + K::RF + D;
              r01 = __ffma2_rn(make_float2(Ma[1], Ma[4]), make_float2(kyf, kyf), q01);
              r2 = fmaf(Ma[7], kyf, q2s);
            }
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
              const float N = wxy * w[2][kz];
              const float kzf = float(kz);
              const int k = ky * 3 + kz;
              const float2 NN = make_float2(N, N);
              const float2 t01 = __ffma2_rn(make_float2(Mv[2], Mv[5]), make_float2(kzf, kzf), v01);
              const float t2 = fmaf(Mv[8], kzf, v2);
              aP01[k] = __ffma2_rn(NN, t01, aP01[k]);
              aP2m[k] = __ffma2_rn(NN, make_float2(t2, mass), aP2m[k]);
              if constexpr (ADJ) {
                const float* Ma = rec + K::RF + D;
                const float2 s01 = __ffma2_rn(make_float2(Ma[2], Ma[5]), make_float2(kzf, kzf), r01);
                const float s2 = fmaf(Ma[8], kzf, r2);
                aQ01[k] = __ffma2_rn(NN, s01, aQ01[k]);
                aQ2[k] = fmaf(N, s2, aQ2[k]);
              }
            }
          }
        }
      }
    };

    // Exclusive starts of cells lane and lane + 32 from the counts in cfill, formed by every warp
    // that calls it (all 32 lanes); warp 0 also writes them, and the total, to cstart.
    auto warp_scan_cells = [&](int& e0, int& e1) {
      const int lane = tid & 31;
      const int v0 = lane < CELLS ? cfill[lane] : 0, v1 = lane + 32 < CELLS ? cfill[lane + 32] : 0;
      int i0 = v0, i1 = v1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int a0 = __shfl_up_sync(0xffffffffu, i0, o), a1 = __shfl_up_sync(0xffffffffu, i1, o);
        if (lane >= o) {
          i0 += a0;
          i1 += a1;
        }
      }
      const int tot0 = __shfl_sync(0xffffffffu, i0, 31);
      e0 = i0 - v0;
      e1 = tot0 + i1 - v1;
      if (tid < 32) {
        if (lane < CELLS) cstart[lane] = e0;
        if (lane + 32 < CELLS) cstart[lane + 32] = e1;
        if (lane == 31) cstart[CELLS] = tot0 + (CELLS > 32 ? i1 : 0);
      }
    };
    // start of cell c from the lane-held starts of warp_scan_cells (all 32 lanes call it)
    auto cell_start_of = [&](int e0, int e1, int c) {
      const int lo = __shfl_sync(0xffffffffu, e0, c & 31), hi = __shfl_sync(0xffffffffu, e1, c & 31);
      return c < 32 ? lo : hi;
    };

    // scan of the per-cell counts in cfill into cstart (one warp; CELLS <= 64)
    auto scan_cells = [&]() {
      if (tid < 32) {
        const int lane = tid;
        int v0 = lane < CELLS ? cfill[lane] : 0, v1 = lane + 32 < CELLS ? cfill[lane + 32] : 0;
        int i0 = v0, i1 = v1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int a0 = __shfl_up_sync(0xffffffffu, i0, o), a1 = __shfl_up_sync(0xffffffffu, i1, o);
          if (lane >= o) {
            i0 += a0;
            i1 += a1;
          }
        }
        const int tot0 = __shfl_sync(0xffffffffu, i0, 31);
        if (lane < CELLS) cstart[lane] = i0 - v0;
        if (lane + 32 < CELLS) cstart[lane + 32] = tot0 + i1 - v1;
        if (lane == 31) cstart[CELLS] = tot0 + (CELLS > 32 ? i1 : 0);
      }
    };

    if (cnt <= 2 * K::THREADS && cnt <= K::REC_CAP) {
      // ---- fast path: every thread owns raw entries tid and tid + THREADS of the tile list.
      // Its first particle's state is requested at once and arrives while the tile is being
      // bucketed; its canonical position is the cell start plus the number of smaller ids in its
      // cell (order: cell, then particle id), and its record is written straight there.
      const uint32_t r0 = tid < cnt ? b.sorted[st + tid] : 0xffffffffu;
      const uint32_t r1 = tid + K::THREADS < cnt ? b.sorted[st + tid + K::THREADS] : 0xffffffffu;
      float pre[Cfg<D>::S];
      int g0 = -1, g1 = -1;
      if (r0 != 0xffffffffu) {
        load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, int(r0 & 0x3ffffffu), pre);
        g0 = group_of(sp, int(r0 & 0x3ffffffu));
      }
      if (r1 != 0xffffffffu) g1 = group_of(sp, int(r1 & 0x3ffffffu));
      // the counting atomics also give each entry its place among its cell's entries
      const int k0 = r0 != 0xffffffffu ? atomicAdd(&cfill[r0 >> 26], 1) : 0;
      const int k1 = r1 != 0xffffffffu ? atomicAdd(&cfill[r1 >> 26], 1) : 0;
      __syncthreads();
      {
        // every warp scans the cell counts itself (warp 0 also publishes cstart for the phases
        // below), so the entries are placed without another barrier
        int e0, e1;
        warp_scan_cells(e0, e1);
        const uint32_t c0 = r0 != 0xffffffffu ? r0 >> 26 : 0u, c1 = r1 != 0xffffffffu ? r1 >> 26 : 0u;
        const int s0 = cell_start_of(e0, e1, int(c0)), s1 = cell_start_of(e0, e1, int(c1));
        if (r0 != 0xffffffffu) ids[s0 + k0] = r0 & 0x3ffffffu;
        if (r1 != 0xffffffffu) ids[s1 + k1] = r1 & 0x3ffffffu;
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t rr = h == 0 ? r0 : r1;
        if (rr == 0xffffffffu) continue;
        const uint32_t id = rr & 0x3ffffffu, c = rr >> 26;
        int pos = cstart[c];
        for (int j = cstart[c]; j < cstart[c + 1]; ++j) pos += ids[j] < id;
        b.sorted[st + pos] = id;  // canonical order for the gathers of this step
        if (h == 0) {
          make_record(int(id), c, g0, pre, pos);
        } else {
          float r[Cfg<D>::S];
          load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, int(id), r);
          make_record(int(id), c, g1, r, pos);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < K::IPT; ++j)
        if (item_thread[j]) accumulate(j, cstart[my_cell[j]], cstart[my_cell[j] + 1], 0);
    } else {
      // ---- general path: bucket, insertion-sort each cell's ids, stage records in chunks
      uint32_t* raw = reinterpret_cast<uint32_t*>(U);
      if (tid < CELLS) cfill[tid] = 0;
      __syncthreads();
      for (int i = tid; i < cnt; i += blockDim.x) {
        const uint32_t r = b.sorted[st + i];  // (cell << 26) | id, written by the scatter
        raw[i] = r;
        atomicAdd(&cfill[r >> 26], 1);
      }
      __syncthreads();
      scan_cells();
      __syncthreads();
      if (tid < CELLS) cfill[tid] = 0;
      __syncthreads();
      for (int i = tid; i < cnt; i += blockDim.x) {
        const uint32_t r = raw[i];
        const uint32_t c = r >> 26;
        ids[cstart[c] + atomicAdd(&cfill[c], 1)] = r & 0x3ffffffu;
      }
      __syncthreads();
      if (tid < CELLS) {  // insertion sort of each cell's ids
        const int s0 = cstart[tid], s1 = cstart[tid + 1];
        for (int i = s0 + 1; i < s1; ++i) {
          const uint32_t v = ids[i];
          int j = i - 1;
          while (j >= s0 && ids[j] > v) {
            ids[j + 1] = ids[j];
            --j;
          }
          ids[j + 1] = v;
        }
      }
      __syncthreads();
      for (int i = tid; i < cnt; i += blockDim.x) b.sorted[st + i] = ids[i];
      int cs[K::IPT], ce[K::IPT];
#pragma unroll
      for (int j = 0; j < K::IPT; ++j) {
        cs[j] = item_thread[j] ? cstart[my_cell[j]] : 0;
        ce[j] = item_thread[j] ? cstart[my_cell[j] + 1] : 0;
      }
      for (int c0 = 0; c0 < cnt; c0 += K::REC_CAP) {
        __syncthreads();  // previous records consumed (and phase A's scratch released)
        const int c1 = cnt < c0 + K::REC_CAP ? cnt : c0 + K::REC_CAP;
        for (int e = c0 + tid; e < c1; e += K::THREADS) {
          const int id = int(ids[e]);
          float r[Cfg<D>::S];
          load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, id, r);
          make_record(id, sp.key[id] & 63u, group_of(sp, id), r, e - c0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K::IPT; ++j)
          if (item_thread[j]) accumulate(j, cs[j] > c0 ? cs[j] : c0, ce[j] < c1 ? ce[j] : c1, c0);
      }
    }
    __syncthreads();  // records done; U becomes the per-cell stencil accumulator array
#pragma unroll
    for (int j = 0; j < K::IPT; ++j) {
      if (!item_thread[j]) continue;
      float* ca = U + size_t(my_cell[j]) * ST * K::CHS;
#pragma unroll
      for (int k = 0; k < K::NK; ++k) {
        float* e = ca + (my_part[j] * K::NK + k) * K::CHS;
        if constexpr (D == 3) {
          float4* e4 = reinterpret_cast<float4*>(e);
          e4[0] = make_float4(aP01[k].x, aP01[k].y, aP2m[k].x, aP2m[k].y);
          if constexpr (ADJ) e4[1] = make_float4(aQ01[k].x, aQ01[k].y, aQ2[k], 0.0f);
        } else {
#pragma unroll
          for (int c = 0; c < K::CH; ++c) e[c] = acc[j][k][c];
        }
      }
    }
    __syncthreads();
    // ---- phase D: node block = fixed-order sum over the cells whose stencil covers it -----
    if (tid < NB) {
      int nl[D];
      {
        int l = tid;
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
          nl[a] = l % BN;
          l /= BN;
        }
      }
      float s[K::CH];
#pragma unroll
      for (int c = 0; c < K::CH; ++c) s[c] = 0.0f;
      float2 s01 = make_float2(0.0f, 0.0f), s23 = s01, s45 = s01;  // 3D
      float s6 = 0.0f;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int cx = nl[0] - kx;
        if (cx < 0 || cx >= B) continue;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const int cy = nl[1] - ky;
          if (cy < 0 || cy >= B) continue;
          if constexpr (D == 2) {
            const int cell = cx * B + cy;
            const float* ca = U + (size_t(cell) * ST + kx * 3 + ky) * K::CH;
#pragma unroll
            for (int c = 0; c < K::CH; ++c) s[c] += ca[c];
          } else {
#pragma unroll
            for (int kz = 0; kz < 3; ++kz) {
              const int cz = nl[2] - kz;
              if (cz < 0 || cz >= B) continue;
              const int cell = (cx * B + cy) * B + cz;
              const float4* ca = reinterpret_cast<const float4*>(U + (size_t(cell) * ST + kx * 9 + ky * 3 + kz) * K::CHS);
              // the same per-channel sums in the same order, two channels per packed add
              const float4 e = ca[0];
              s01 = __fadd2_rn(s01, make_float2(e.x, e.y));
              s23 = __fadd2_rn(s23, make_float2(e.z, e.w));
              if constexpr (ADJ) {
                const float4 e2 = ca[1];
                s45 = __fadd2_rn(s45, make_float2(e2.x, e2.y));
                s6 += e2.z;
              }
            }
          }
        }
      }
      float4 o;
      if constexpr (D == 2)
        o = make_float4(s[0], s[1], s[2], 0.0f);
      else
        o = make_float4(s01.x, s01.y, s23.x, s23.y);
      b.partial[size_t(slot) * NB + tid] = o;
      if constexpr (ADJ) {
        float4 oa;
        if constexpr (D == 2)
          oa = make_float4(s[K::CHF], s[K::CHF + 1], 0.0f, 0.0f);
        else
          oa = make_float4(s45.x, s45.y, s6, 0.0f);
        b.partial_b[size_t(slot) * NB + tid] = oa;
      }
    }
    if (tid < CELLS) cfill[tid] = 0;  // for the next tile (nothing reads the counts after placement)
    __syncthreads();
  }
  if (dyn) release_work(b, 0);
}

// ============================================================================ grid
// The grid update of Eq. 6 with gravity and the boundary condition, evaluated by every CTA that
// gathers from a node block: node i of tile t's (B+2)^D block sums, in a fixed order, the P2G node
// blocks of the <= 2^D tiles whose blocks contain it.  With ADJ the adjoint-scatter blocks give
// vbar*, and (L), (D), (E) give pbar and mbar.  Nodes a tile owns (its B^D corner) are also
// written to the dense grid for inspection.
template <int D, int TB, bool ADJ>
__device__ __forceinline__ void build_node_block(const BatchDev& b, const ScenePar& sp, const int* t, float4* sv,
                                                 float4* sb) {
  constexpr int B = Tile<D, TB>::B, NB = Tile<D, TB>::BLOCK_NODES, BN = Tile<D, TB>::BN;
  constexpr int NN = D == 2 ? 9 : 27;  // tiles t + o, o in {-1, 0, 1}^D
  __shared__ int nslot[NN];
  if (threadIdx.x < NN) {
    int o[3] = {int(threadIdx.x) / (D == 2 ? 3 : 9) - 1, (int(threadIdx.x) / (D == 2 ? 1 : 3)) % 3 - 1,
                int(threadIdx.x) % 3 - 1};
    int u[D];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = t[a] + o[a];
      ok = ok && u[a] >= 0 && u[a] < sp.nt[a];
    }
    nslot[threadIdx.x] = ok ? b.tile_slot[sp.tile_base + lin3<D>(u, sp.nt)] : -1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NB; i += blockDim.x) {
    int nl[D], nd[D], r[D], qo[D];
    bool in_grid = true, owned = true;
    {
      int l = i;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        nl[a] = l % BN;
        l /= BN;
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      nd[a] = t[a] * B + nl[a];
      in_grid = in_grid && nd[a] < sp.n[a];
      owned = owned && nl[a] < B;
      qo[a] = nl[a] / B;  // the node's tile is t + qo
      r[a] = nl[a] - qo[a] * B;
    }
    if (!in_grid) {
      sv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (ADJ) sb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    // sources: tiles t + qo - e with e in {0,1}^D and r + e*B inside the block; independent loads
    float4 pv[1 << D], pa[1 << D];
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {
      int so = 0, l = 0;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int ea = (e >> (D - 1 - a)) & 1;
        const int loc = r[a] + ea * B;
        ok = ok && loc < BN;
        so = so * 3 + (qo[a] - ea + 1);
        l = l * BN + loc;
      }
      const int slot = ok ? nslot[so] : -1;
      pv[e] = slot >= 0 ? b.partial[size_t(slot) * NB + l] : make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (ADJ) pa[e] = slot >= 0 ? b.partial_b[size_t(slot) * NB + l] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sa[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < (1 << D); ++e) {  // fixed order
      s[0] += pv[e].x;
      s[1] += pv[e].y;
      s[2] += pv[e].z;
      s[3] += pv[e].w;
      if constexpr (ADJ) {
        sa[0] += pa[e].x;
        sa[1] += pa[e].y;
        sa[2] += pa[e].z;
      }
    }
    const float m = s[D];
    float vraw[D], v[D];
    if (m > 0.0f) {
      const float rm = 1.0f / m;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        vraw[a] = s[a] * rm;
        v[a] = vraw[a] + sp.dt * sp.gravity[a];
      }
      bc_apply<D>(nd, sp.n, sp.bc, v);
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = vraw[a] = 0.0f;
    }
    float4 o;
    if constexpr (D == 2)
      o = make_float4(v[0], v[1], m, 0.0f);
    else
      o = make_float4(v[0], v[1], v[2], m);
    sv[i] = o;
    if (owned) sp.grid[lin3<D>(nd, sp.n)] = o;
    if constexpr (ADJ) {
      float g[D], pb[D], mb = 0.0f;
      if (m > 0.0f) {
        float vg[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          g[a] = sa[a];
          vg[a] = vraw[a] + sp.dt * sp.gravity[a];
        }
        bc_adjoint<D>(nd, sp.n, sp.bc, vg, g);  // (L); gravity passes the adjoint through
        const float rm = 1.0f / m;
        float dot = 0.0f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          pb[a] = g[a] * rm;        // (D)
          dot += vraw[a] * g[a];
        }
        mb = -dot * rm;             // (E)
      } else {
#pragma unroll
        for (int a = 0; a < D; ++a) pb[a] = 0.0f;
      }
      float4 ob;
      if constexpr (D == 2)
        ob = make_float4(pb[0], pb[1], mb, 0.0f);
      else
        ob = make_float4(pb[0], pb[1], pb[2], mb);
      sb[i] = ob;
      if (owned) sp.grid_b[lin3<D>(nd, sp.n)] = ob;
    }
  }
}

// Deterministic per-warp group sums: lanes hold (group g, value c); the sum of every group present
// in the warp is formed by a fixed butterfly and added to the register of the lane that owns the
// group (lane g % 32, slot g / 32).  All 32 lanes must call it.
__device__ __forceinline__ void warp_group_add(int g, float c, float& lo, float& hi) {
  const int lane = threadIdx.x & 31;
  unsigned todo = __ballot_sync(0xffffffffu, g >= 0);
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int gs = __shfl_sync(0xffffffffu, g, leader);
    float v = g == gs ? c : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == (gs & 31)) {
      if (gs >> 5)
        hi += v;
      else
        lo += v;
    }
    todo &= ~__ballot_sync(0xffffffffu, g == gs);
  }
}

// ============================================================================ G2P core
// Gathers v* over the stencil (Eqs. 7, 8) and updates F and x (Eqs. 9, 10).
template <int D, class Fetch>
__device__ __forceinline__ void g2p_core(Part<D>& q, const float* f, const float (&w)[D][3], float dt, float inv_dx,
                                         Fetch fetch) {
  // sum_i N v and sum_i N v k^T (k the integer node offset; the f part is taken once below),
  // formed as nested weighted sums: over z within a row, over y within an x-slab, then over x
  float vn[D], Cn[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vn[a] = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) Cn[a][c] = 0.0f;
  }
#pragma unroll
  for (int kx = 0; kx < 3; ++kx) {
    float sv[D], sy[D], sz[D];  // slab sums of wy wz v, ky wy wz v, kz wy wz v
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      float r[D], rz[D];  // row sums of wz v and kz wz v (2D: the node's v)
      if constexpr (D == 3) {
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const float4 g = fetch(kx, ky, kz);
          const float vv[3] = {g.x, g.y, g.z};
          const float wz = w[D == 3 ? 2 : 0][kz];
#pragma unroll
          for (int a = 0; a < D; ++a) {
            r[a] = kz == 0 ? wz * vv[a] : r[a] + wz * vv[a];
            if (kz == 1) rz[a] = wz * vv[a];
            if (kz == 2) rz[a] += (2.0f * wz) * vv[a];
          }
        }
      } else {
        const float4 g = fetch(kx, ky, 0);
        r[0] = g.x;
        r[1] = g.y;
      }
      const float wy = w[1][ky];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        sv[a] = ky == 0 ? wy * r[a] : sv[a] + wy * r[a];
        if (ky == 1) sy[a] = wy * r[a];
        if (ky == 2) sy[a] += (2.0f * wy) * r[a];
        if constexpr (D == 3) sz[a] = ky == 0 ? wy * rz[a] : sz[a] + wy * rz[a];
      }
    }
    const float wx = w[0][kx];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vn[a] += wx * sv[a];
      if (kx > 0) Cn[a][0] += (float(kx) * wx) * sv[a];
      Cn[a][1] += wx * sy[a];
      if constexpr (D == 3) Cn[a][D - 1] += wx * sz[a];
    }
  }
  const float s = 4.0f * inv_dx;  // (4/dx^2) * dx, since x_i - x_p = dx (k - f)
  float Fo[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Cn[a][c] = s * (Cn[a][c] - f[c] * vn[a]);
      Fo[a][c] = q.F[a][c];
    }
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float acc = Fo[a][c];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += dt * Cn[a][k] * Fo[k][c];
      q.F[a][c] = acc;
      q.C[a][c] = Cn[a][c];
    }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    q.v[a] = vn[a];
    q.x[a] += dt * vn[a];
  }
}

// Particles of a tile staged in shared memory by asynchronous copies (first STAGE of them).
template <int D>
struct G2PCfg {
  static constexpr int STAGE = 512;
  static constexpr int NP = Cfg<D>::XF_PLANES;
};

template <int D, int TB, int T>
__global__ void __launch_bounds__(T, 768 / T) k_g2p(BatchDev b) {
  pdl_enter();
  using K = G2PCfg<D>;
  constexpr int B = Tile<D, TB>::B, NB = Tile<D, TB>::BLOCK_NODES, BN = Tile<D, TB>::BN;
  __shared__ float4 sv[NB];
  __shared__ float4 stage[K::NP][K::STAGE];
  const int tid = threadIdx.x;
  // the CTA's first active tile is requested together with the count (the entry is in bounds
  // whatever the count; it is used only when the slot is below it)
  const int first_gt = b.total_tiles > 0 ? b.active[int(blockIdx.x) < b.total_tiles ? blockIdx.x : 0] : 0;
  const int n_active = *b.n_active;
  if (blockIdx.x == 0)  // this step's counters move on (every reader of them ran before)
    for (int s = tid; s < b.n_scenes; s += blockDim.x)
      if (b.scenes[s].step_ctr) *b.scenes[s].step_ctr += 1;
  for (int slot = blockIdx.x; slot < n_active; slot += gridDim.x) {
    const int gt = slot == int(blockIdx.x) ? first_gt : b.active[slot];
    const ScenePar& sp = b.scenes[b.n_scenes == 1 ? 0 : b.tile_scene[gt]];
    int t[D];
    unlin<D>(gt - sp.tile_base, sp.nt, t);
    const uint32_t st = b.tile_start[gt];
    const int cnt = int(b.tile_start[gt + 1] - st);
    // a tile over P2G's capacity was skipped there (the step reports it): its list still holds
    // the scatter's cell-tagged entries, so it is skipped here too
    if (cnt > Tile<D, TB>::SORT_CAP) {  // uniform across the CTA
      // its particles are not advanced: their keys go invalid so the next step's histogram and
      // scatter (which count keys) stay consistent; the step has already reported the error
      for (int e = tid; e < cnt; e += blockDim.x) sp.key[b.sorted[st + e] & 0x3ffffffu] = KEY_INVALID;
      continue;
    }
    const int staged = cnt < K::STAGE ? cnt : K::STAGE;
    // request the x, F planes of the tile's particles; they arrive while the node block is built
    // (the thread's list entries are read first, all at once, then the copies are issued)
    {
      constexpr int SPT = (K::STAGE + T - 1) / T;
      uint32_t ent[SPT];
#pragma unroll
      for (int u = 0; u < SPT; ++u) ent[u] = tid + u * T < staged ? b.sorted[st + tid + u * T] : 0u;
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int e = tid + u * T;
        if (e >= staged) break;
        const int id = int(ent[u] & 0x3ffffffu);
#pragma unroll
        for (int j = 0; j < K::NP; ++j) cp_async16(&stage[j][e], sp.planes + size_t(j) * sp.npad + id);
      }
    }
    cp_async_commit();
    build_node_block<D, TB, false>(b, sp, t, sv, nullptr);
    cp_async_wait_all();
    __syncthreads();
    for (int e = tid; e < cnt; e += blockDim.x) {
      const int id = int(b.sorted[st + e] & 0x3ffffffu);
      float r[Cfg<D>::S];
      if (e < K::STAGE) {
#pragma unroll
        for (int j = 0; j < K::NP; ++j) {
          const float4 q = stage[j][e];
          r[4 * j] = q.x;
          r[4 * j + 1] = q.y;
          r[4 * j + 2] = q.z;
          r[4 * j + 3] = q.w;
        }
      } else {
        load_planes<D, K::NP>(sp.planes, sp.npad, id, r);
      }
      Part<D> q;
      unpack<D>(r, q);
      int base[D];
      float f[D], w[D][3], dw[3];
      stencil_base<D>(q.x, sp.inv_dx, sp.n, base, f);
      bool inside = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        bspline(f[a], sp.inv_dx, w[a], dw);
        base[a] -= t[a] * B;  // local stencil origin inside the node block
        inside = inside && base[a] >= 0 && base[a] < B;
      }
      if (!inside) {  // bin key disagrees with the position: never index outside the block
        set_status(sp.status, ST_BINNING);
        sp.key[id] = KEY_INVALID;  // not advanced, not counted: the next scatter stays in bounds
        continue;
      }
      g2p_core<D>(q, f, w, sp.dt, sp.inv_dx, [&](int kx, int ky, int kz) {
        int l = (base[0] + kx) * BN + base[1] + ky;
        if constexpr (D == 3) l = l * BN + base[2] + kz;
        return sv[l];
      });
      float ro[Cfg<D>::S];
      pack<D>(q, ro);
      store_planes<D, Cfg<D>::PLANES>(sp.planes_out, sp.npad, id, ro);
      const uint32_t nk = bin_key<D, TB>(q.x, sp);  // bin of state n+1 and its histogram
      sp.key[id] = nk;
      warp_aggregated_inc(b.tile_count, nk != KEY_INVALID ? int(sp.tile_base + (nk >> 6)) : -1);
    }
    __syncthreads();
  }
}

// ============================================================================ adjoint gather
// Supplement S4: (F) vbar, (I) Cbar, (G) Pbar, (H) Fbar, (J) xbar, (K) sigma-bar -> dL/da.
// `fetch(kx,ky,kz, v, pb)` returns (v*, m) in v and (pbar, mbar) in pb.  With MAT and per-particle
// material (sp.gmat) this step's dL/dE_p = (F - F^{-T}):Pbar dmu/dE + ln J (F^{-T}:Pbar) dlambda/dE
// and dL/dm_p = sum_i N (mbar_i + pbar_i . (v_p + C_p (x_i - x_p))) are added into gmat[id].
// A load the compiler keeps where it is written (not merged with an earlier load of the same
// address), so that values needed only after a long loop need not stay in registers through it.
__device__ __forceinline__ float4 ldg_fresh(const float4* p) {
  float4 r;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p)
               : "memory");
  return r;
}

template <int D, bool MAT, class Fetch, class Reload>
__device__ __forceinline__ float adj_core(Part<D>& q, Part<D>& g1, const float* f, const float (&w)[D][3],
                                          const float (&dw)[D][3], const ScenePar& sp, int id, int g, Fetch fetch,
                                          Reload reload, Part<D>& g0) {
  const PMat pm = pmat_of(sp, id);
  const float dt = sp.dt, dx = sp.dx, mass = pm.mass;
  const float Dinv = 4.0f * sp.inv_dx * sp.inv_dx;
  const float kG = -Dinv * dt * sp.vol;
  float G[D][D], sig[D];
  {
    float P[D][D], A[D][D];  // recomputed after the stencil loop: not kept live across it
    particle_G<D>(q, sp, g, pm, P, A, G, sig);
  }
  // s_i = vbar'.v* + Dinv v*^T Cbar' d + pbar.(m v + G d) + m mbar with d = (k - f) dx is affine in
  // the integer node offset k: alpha(k) = vbar' + Dinv Cbar' d and beta(k) = m v + G d are kept as
  // their value at the slab/row start plus one column per axis (Ac[c] = Dinv dx Cbar'[:, c],
  // Bc[c] = dx G[:, c]), so a node costs additions instead of two matrix-vector products
  float Ac[D][D], Bc[D][D], al[D], be[D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) s += g1.F[a][k] * q.F[c][k];
      Ac[c][a] = Dinv * dx * (g1.C[a][c] + dt * s);  // Cbar' = C' + dt F' F^T
      Bc[c][a] = dx * G[a][c];
    }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float sa = g1.v[a] + dt * g1.x[a], sb = mass * q.v[a];  // vbar' and m v
#pragma unroll
    for (int c = 0; c < D; ++c) {
      sa -= Ac[c][a] * f[c];
      sb -= Bc[c][a] * f[c];
    }
    al[a] = sa;
    be[a] = sb;
  }
  // accumulators: gxs = sum dN s_i; sv = sum N v*, spb = sum N pbar; Tv/Tp = the same sums weighted
  // by the y (and z) node offset; Rv/Rp = running totals of sv/spb at each x-slab end, from which the
  // x-offset-weighted sums follow (sum kx S_kx = 3 S - R for kx = 0, 1, 2)
  float gxs[D], sv[D], spb[D], Tv[D][D - 1], Tp[D][D - 1], Rv[D], Rp[D], smb = 0.0f;  // smb = sum N mbar
  if constexpr (D == 3) {
    // the x and y components of every 3-vector in pairs for the packed FP32 operations (each half
    // rounds as its own fmaf / fmul / fadd), the z component alone: the same operations in the same
    // order as the loop below
    float2 A01[3], B01[3];
    float A2[3], B2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A01[c] = make_float2(Ac[c][0], Ac[c][1]);
      A2[c] = Ac[c][2];
      B01[c] = make_float2(Bc[c][0], Bc[c][1]);
      B2[c] = Bc[c][2];
    }
    float2 al01 = make_float2(al[0], al[1]), be01 = make_float2(be[0], be[1]);
    float al2 = al[2], be2 = be[2];
    const float2 z2 = make_float2(0.0f, 0.0f);
    float2 gx01 = z2, sv01 = z2, sp01 = z2, tvy01 = z2, tvz01 = z2, tpy01 = z2, tpz01 = z2, rv01 = z2, rp01 = z2;
    float gx2 = 0.0f, sv2 = 0.0f, sp2 = 0.0f, tvy2 = 0.0f, tvz2 = 0.0f, tpy2 = 0.0f, tpz2 = 0.0f, rv2 = 0.0f,
          rp2 = 0.0f;
#pragma unroll 1
    for (int kx = 0; kx < 3; ++kx) {
      const float wx = kx == 0 ? w[0][0] : (kx == 1 ? w[0][1] : w[0][2]);
      const float dwx = kx == 0 ? dw[0][0] : (kx == 1 ? dw[0][1] : dw[0][2]);
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const float wxy = wx * w[1][ky], dwxy = dwx * w[1][ky], wxdy = wx * dw[1][ky];
        const float kyf = float(ky);
        const float2 ky2 = make_float2(kyf, kyf);
        float2 ar01 = al01, br01 = be01;
        float ar2 = al2, br2 = be2;
        if (ky > 0) {
          ar01 = __ffma2_rn(ky2, A01[1], al01);
          ar2 = fmaf(kyf, A2[1], al2);
          br01 = __ffma2_rn(ky2, B01[1], be01);
          br2 = fmaf(kyf, B2[1], be2);
        }
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const float wz = w[2][kz];
          const float N = wxy * wz;
          const float2 dN01 = __fmul2_rn(make_float2(dwxy, wxdy), make_float2(wz, wz));
          const float dN2 = wxy * dw[2][kz];
          const float kzf = float(kz);
          const float2 kz2 = make_float2(kzf, kzf);
          float2 alpha01 = ar01, beta01 = br01;
          float alpha2 = ar2, beta2 = br2;
          if (kz > 0) {
            alpha01 = __ffma2_rn(kz2, A01[2], ar01);
            alpha2 = fmaf(kzf, A2[2], ar2);
            beta01 = __ffma2_rn(kz2, B01[2], br01);
            beta2 = fmaf(kzf, B2[2], br2);
          }
          float4 v4, p4;
          fetch(kx, ky, kz, v4, p4);
          const float mb = p4.w;
          float si = mass * mb;
          if constexpr (MAT) smb += N * mb;
          si += v4.x * alpha01.x + p4.x * beta01.x;
          si += v4.y * alpha01.y + p4.y * beta01.y;
          si += v4.z * alpha2 + p4.z * beta2;
          gx01 = __ffma2_rn(dN01, make_float2(si, si), gx01);
          gx2 = fmaf(dN2, si, gx2);
          const float2 NN = make_float2(N, N);
          const float2 qv01 = __fmul2_rn(NN, make_float2(v4.x, v4.y)), qp01 = __fmul2_rn(NN, make_float2(p4.x, p4.y));
          const float qv2 = N * v4.z, qp2 = N * p4.z;
          sv01 = __fadd2_rn(sv01, qv01);
          sv2 += qv2;
          sp01 = __fadd2_rn(sp01, qp01);
          sp2 += qp2;
          if (ky > 0) {
            tvy01 = __ffma2_rn(ky2, qv01, tvy01);
            tvy2 = fmaf(kyf, qv2, tvy2);
            tpy01 = __ffma2_rn(ky2, qp01, tpy01);
            tpy2 = fmaf(kyf, qp2, tpy2);
          }
          if (kz > 0) {
            tvz01 = __ffma2_rn(kz2, qv01, tvz01);
            tvz2 = fmaf(kzf, qv2, tvz2);
            tpz01 = __ffma2_rn(kz2, qp01, tpz01);
            tpz2 = fmaf(kzf, qp2, tpz2);
          }
        }
      }
      rv01 = __fadd2_rn(rv01, sv01);
      rv2 += sv2;
      rp01 = __fadd2_rn(rp01, sp01);
      rp2 += sp2;
      al01 = __fadd2_rn(al01, A01[0]);
      al2 += A2[0];
      be01 = __fadd2_rn(be01, B01[0]);
      be2 += B2[0];
    }
    gxs[0] = gx01.x;
    gxs[1] = gx01.y;
    gxs[2] = gx2;
    sv[0] = sv01.x;
    sv[1] = sv01.y;
    sv[2] = sv2;
    spb[0] = sp01.x;
    spb[1] = sp01.y;
    spb[2] = sp2;
    Tv[0][0] = tvy01.x;
    Tv[1][0] = tvy01.y;
    Tv[2][0] = tvy2;
    Tv[0][D - 2] = tvz01.x;
    Tv[1][D - 2] = tvz01.y;
    Tv[2][D - 2] = tvz2;
    Tp[0][0] = tpy01.x;
    Tp[1][0] = tpy01.y;
    Tp[2][0] = tpy2;
    Tp[0][D - 2] = tpz01.x;
    Tp[1][D - 2] = tpz01.y;
    Tp[2][D - 2] = tpz2;
    Rv[0] = rv01.x;
    Rv[1] = rv01.y;
    Rv[2] = rv2;
    Rp[0] = rp01.x;
    Rp[1] = rp01.y;
    Rp[2] = rp2;
  } else {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    gxs[a] = sv[a] = spb[a] = Rv[a] = Rp[a] = 0.0f;
#pragma unroll
    for (int c = 0; c < D - 1; ++c) Tv[a][c] = Tp[a][c] = 0.0f;
  }
#pragma unroll 1
  for (int kx = 0; kx < 3; ++kx) {
    // weights of this x-slab as scalars (a loop index must not index the weight arrays)
    const float wx = kx == 0 ? w[0][0] : (kx == 1 ? w[0][1] : w[0][2]);
    const float dwx = kx == 0 ? dw[0][0] : (kx == 1 ? dw[0][1] : dw[0][2]);
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const float wxy = wx * w[1][ky], dwxy = dwx * w[1][ky], wxdy = wx * dw[1][ky];
      float ar[D], br[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        ar[a] = ky == 0 ? al[a] : al[a] + float(ky) * Ac[1][a];
        br[a] = ky == 0 ? be[a] : be[a] + float(ky) * Bc[1][a];
      }
#pragma unroll
      for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz) {
        constexpr int Z = D == 3 ? 2 : 0;
        float N, dN[D], alpha[D], beta[D];
        if constexpr (D == 3) {
          N = wxy * w[Z][kz];
          dN[0] = dwxy * w[Z][kz];
          dN[1] = wxdy * w[Z][kz];
          dN[Z] = wxy * dw[Z][kz];
#pragma unroll
          for (int a = 0; a < D; ++a) {
            alpha[a] = kz == 0 ? ar[a] : ar[a] + float(kz) * Ac[Z][a];
            beta[a] = kz == 0 ? br[a] : br[a] + float(kz) * Bc[Z][a];
          }
        } else {
          N = wxy;
          dN[0] = dwxy;
          dN[1] = wxdy;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            alpha[a] = ar[a];
            beta[a] = br[a];
          }
        }
        float4 v4, p4;
        fetch(kx, ky, kz, v4, p4);
        const float vs[3] = {v4.x, v4.y, v4.z};
        const float pb[3] = {p4.x, p4.y, p4.z};
        const float mb = D == 2 ? p4.z : p4.w;
        float si = mass * mb;
        if constexpr (MAT) smb += N * mb;
#pragma unroll
        for (int a = 0; a < D; ++a) si += vs[a] * alpha[a] + pb[a] * beta[a];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          gxs[a] += dN[a] * si;
          const float qv = N * vs[a], qp = N * pb[a];
          sv[a] += qv;
          spb[a] += qp;
          if (ky > 0) {
            Tv[a][0] += float(ky) * qv;
            Tp[a][0] += float(ky) * qp;
          }
          if constexpr (D == 3) {
            if (kz > 0) {
              Tv[a][D - 2] += float(kz) * qv;
              Tp[a][D - 2] += float(kz) * qp;
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      Rv[a] += sv[a];
      Rp[a] += spb[a];
      al[a] += Ac[0][a];
      be[a] += Bc[0][a];
    }
  }
  }
  // the epilogue's inputs read again (same bits): not kept in registers through the stencil loop
  reload(q, g1);
  // Gbar = sum N pbar d^T (= dx (sum N pbar k^T - spb f^T)), Cn = sum N v* (k - f)^T
  float Gbar[D][D], Cn[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float tv[D], tp[D];
    tv[0] = 3.0f * sv[a] - Rv[a];
    tp[0] = 3.0f * spb[a] - Rp[a];
#pragma unroll
    for (int c = 1; c < D; ++c) {
      tv[c] = Tv[a][c - 1];
      tp[c] = Tp[a][c - 1];
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Cn[a][c] = tv[c] - f[c] * sv[a];
      Gbar[a][c] = dx * (tp[c] - f[c] * spb[a]);
    }
  }
  // (J): gx = gx' + sum dN s_i - Dinv Cbar'^T sum N v* - G^T sum N pbar
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < D; ++c) t += Ac[a][c] * sv[c] + Bc[a][c] * spb[c];
    g0.x[a] = g1.x[a] + gxs[a] - sp.inv_dx * t;
    g0.v[a] = mass * spb[a];  // (F)
  }
  const float sC = 4.0f * sp.inv_dx;
  float Pb[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Cn[a][c] *= sC;
      g0.C[a][c] = mass * Gbar[a][c];  // (I)
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) s += Gbar[a][k] * q.F[k][c];
      Pb[a][c] = kG * s;  // (G)
    }
  float P[D][D], A[D][D];
  const float J = stress<D>(q.F, pm.mat, sig, P, A);
  float H[D][D];
  nh_hessian_apply<D>(A, J, pm.mat, Pb, H);
  if (MAT && sp.gmat) {  // material gradients of this step (P2G is where E_p and m_p enter)
    float gmu = 0.0f, gla = 0.0f, gm = smb;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      gm += q.v[a] * spb[a];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        gmu += (q.F[a][c] - A[a][c]) * Pb[a][c];
        gla += A[a][c] * Pb[a][c];
        gm += q.C[a][c] * Gbar[a][c];
      }
    }
    const float gE = gmu * sp.mu_per_E + logf(J > 0.0f ? J : 1.0f) * gla * sp.la_per_E;
    float2 acc = sp.gmat[id];
    acc.x += gE;
    acc.y += gm;
    sp.gmat[id] = acc;
  }
  // (H) Fbar = (I + dt C^{n+1})^T Fbar' + H[Pbar] + Pbar sigma^T + kG Gbar^T P
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float s = g1.F[a][c];
      float t = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        s += dt * Cn[k][a] * g1.F[k][c];
        t += Gbar[k][a] * P[k][c];
      }
      g0.F[a][c] = s + H[a][c] + Pb[a][c] * sig[c] + kG * t;
    }
  // (K) sigma-bar = F^T Pbar, contracted with the group's direction
  float contrib = 0.0f;
  if (g >= 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) s += q.F[k][a] * Pb[k][a];
      contrib += __ldg(sp.act_dir + g * D + a) * s;
    }
  }
  return contrib;
}

// CTA size of the adjoint gather: fixed per dimension (its group sums are formed per warp, then
// per CTA, so the size sets their rounding; batches never mix dimensions).  128 threads measured
// faster in 3D, 256 in 2D.
template <int D>
constexpr int kAdjThreads = D == 3 ? 128 : 256;

template <int D, int TB, bool MAT>
__global__ void __launch_bounds__(kAdjThreads<D>, 512 / kAdjThreads<D>) k_adj_gather(BatchDev b) {
  pdl_enter();
  constexpr int B = Tile<D, TB>::B, NB = Tile<D, TB>::BLOCK_NODES, BN = Tile<D, TB>::BN;
  __shared__ float4 sv[NB], sb[NB];
  __shared__ float wpart[8][MAX_GROUPS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the CTA's first active tile is requested together with the count (the entry is in bounds
  // whatever the count; it is used only when the slot is below it)
  const int first_gt = b.total_tiles > 0 ? b.active[int(blockIdx.x) < b.total_tiles ? blockIdx.x : 0] : 0;
  const int n_active = *b.n_active;
  if (b.rewind_ctr && blockIdx.x == 0 && tid == 0) {
    *b.rewind_rows = n_active;
    *b.rewind_ctr -= 1;
  }
  __shared__ int s_next[2];
  const bool dyn = n_active > 2 * int(gridDim.x);  // uniform across the grid
  int it = 0;
  for (int slot = blockIdx.x; slot < n_active; slot = dyn ? take_next(s_next, it++) : slot + int(gridDim.x)) {
    if (dyn) claim_next(b, 1, s_next, it);
    const int gt = slot == int(blockIdx.x) ? first_gt : b.active[slot];
    const ScenePar& sp = b.scenes[b.n_scenes == 1 ? 0 : b.tile_scene[gt]];
    int t[D];
    unlin<D>(gt - sp.tile_base, sp.nt, t);
    const uint32_t st = b.tile_start[gt];
    const int cnt = int(b.tile_start[gt + 1] - st);
    if (cnt > Tile<D, TB>::SORT_CAP) {  // skipped by the adjoint scatter (the step reports it)
      if (tid < MAX_GROUPS) b.gpartial[size_t(slot) * MAX_GROUPS + tid] = 0.0f;
      continue;  // uniform across the CTA
    }
    // the first particle's state is requested before the node block is built, so the two overlap
    // (requesting its adjoint too, or staging the second particle in shared memory, measured slower)
    float r[Cfg<D>::S];
    if (tid < cnt) load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, int(b.sorted[st + tid] & 0x3ffffffu), r);
    build_node_block<D, TB, true>(b, sp, t, sv, sb);
    __syncthreads();
    float lo = 0.0f, hi = 0.0f;  // per-warp group sums of (K), lane-owned
    for (int e0 = 0; e0 < cnt; e0 += blockDim.x) {
      const int e = e0 + tid;
      int g = -1;
      float contrib = 0.0f;
      if (e < cnt) {
        const int id = int(b.sorted[st + e] & 0x3ffffffu);
        if (e0 > 0) load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, id, r);
        Part<D> q, g1, g0;
        unpack<D>(r, q);
        load_planes<D, Cfg<D>::PLANES>(sp.adj_in, sp.npad, id, r);
        unpack<D>(r, g1);
        const int gq = group_of(sp, id);
        int base[D];
        float f[D], w[D][3], dw[D][3];
        stencil_base<D>(q.x, sp.inv_dx, sp.n, base, f);
        bool inside = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          bspline(f[a], sp.inv_dx, w[a], dw[a]);
          base[a] -= t[a] * B;
          inside = inside && base[a] >= 0 && base[a] < B;
        }
        if (inside) {
          auto fetch = [&](int kx, int ky, int kz, float4& v, float4& p) {
            int l = (base[0] + kx) * BN + base[1] + ky;
            if constexpr (D == 3) l = l * BN + base[2] + kz;
            v = sv[l];
            p = sb[l];
          };
          auto reload = [&](Part<D>& qq, Part<D>& gg) {
            float rq[Cfg<D>::S], rg[Cfg<D>::S];
            constexpr int NP = MAT ? Cfg<D>::PLANES : Cfg<D>::XF_PLANES;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
              const float4 a = ldg_fresh(sp.planes + size_t(j) * sp.npad + id);
              rq[4 * j] = a.x;
              rq[4 * j + 1] = a.y;
              rq[4 * j + 2] = a.z;
              rq[4 * j + 3] = a.w;
            }
#pragma unroll
            for (int j = 0; j < Cfg<D>::XF_PLANES; ++j) {
              const float4 a = ldg_fresh(sp.adj_in + size_t(j) * sp.npad + id);
              rg[4 * j] = a.x;
              rg[4 * j + 1] = a.y;
              rg[4 * j + 2] = a.z;
              rg[4 * j + 3] = a.w;
            }
            // planes 0..XF_PLANES-1 hold x and F; with MAT also v and C
#pragma unroll
            for (int i = 0; i < D; ++i) {
              qq.x[i] = rq[i];
              gg.x[i] = rg[i];
#pragma unroll
              for (int c = 0; c < D; ++c) {
                qq.F[i][c] = rq[D + i * D + c];
                gg.F[i][c] = rg[D + i * D + c];
              }
            }
            if constexpr (MAT) {
#pragma unroll
              for (int i = 0; i < D; ++i) {
                qq.v[i] = rq[D + D * D + i];
#pragma unroll
                for (int c = 0; c < D; ++c) qq.C[i][c] = rq[2 * D + D * D + i * D + c];
              }
            }
          };
          contrib = adj_core<D, MAT>(q, g1, f, w, dw, sp, id, gq, fetch, reload, g0);
          pack<D>(g0, r);
          store_planes<D, Cfg<D>::PLANES>(sp.adj_out, sp.npad, id, r);
          g = gq;
        } else {
          set_status(sp.status, ST_BINNING);
        }
      }
      warp_group_add(g, contrib, lo, hi);
    }
    wpart[warp][lane] = lo;
    wpart[warp][lane + 32] = hi;
    __syncthreads();
    if (tid < MAX_GROUPS) {
      float s = 0.0f;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) s += wpart[w][tid];
      b.gpartial[size_t(slot) * MAX_GROUPS + tid] = s;
    }
    __syncthreads();
  }
  if (dyn) release_work(b, 1);
}

// ============================================================================ launchers (tiled)
// Every tiled launcher picks the instantiation of the batch's tile edge: 4, or 8 for 2D scenes
// created with 8 x 8-cell tiles.
template <int D>
static bool wide_tiles(const BatchDev& b) {
  return D == 2 && b.tile_edge == 8;
}

template <int D, int TB>
static cudaError_t keys_impl(const BatchDev& b, cudaStream_t s, const SelectPar* sel) {
  if (sel) {  // at least one CTA: the selection is published even without particles
    const int nblk = b.total_particles > 0 ? (b.total_particles + 255) / 256 : 1;
    launch_pdl(k_keys<D, TB, true>, dim3(nblk), dim3(256), 0, s, b, sel);
    count_launches(1);
    return cudaGetLastError();
  }
  if (b.total_particles == 0) return cudaSuccess;
  launch_pdl(k_keys<D, TB, false>, dim3((b.total_particles + 255) / 256), dim3(256), 0, s, b, sel);
  count_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_keys(const BatchDev& b, cudaStream_t s, const SelectPar* sel) {
  cudaError_t e = cudaMemsetAsync(b.tile_count, 0, sizeof(uint32_t) * size_t(b.total_tiles), s);
  if (e != cudaSuccess) return e;
  if constexpr (D == 2)
    if (wide_tiles<D>(b)) return keys_impl<D, 8>(b, s, sel);
  return keys_impl<D, 4>(b, s, sel);
}

template <int D>
cudaError_t launch_sort(const BatchDev& b, cudaStream_t s, const SelectPar* sel) {
  if (fused_scan(b)) {  // scan inside the scatter; at least one CTA so the scan results are written
    const int nblk = b.total_particles > 0 ? (b.total_particles + 255) / 256 : 1;
    if (sel)
      launch_pdl(k_scatter<D, true, true>, dim3(nblk + 1), dim3(256), 0, s, b, sel);
    else
      launch_pdl(k_scatter<D, true, false>, dim3(nblk), dim3(256), 0, s, b, sel);
    count_launches(1);
    return cudaGetLastError();
  }
  const int nblk = (b.total_tiles + SCAN_TILE - 1) / SCAN_TILE;
  if (sel)
    launch_pdl(k_scan_reduce<true>, dim3(nblk + 1), dim3(SCAN_THREADS), 0, s, b, sel);
  else
    launch_pdl(k_scan_reduce<false>, dim3(nblk), dim3(SCAN_THREADS), 0, s, b, sel);
  launch_pdl(k_scan_down, dim3(nblk), dim3(SCAN_THREADS), 0, s, b);
  if (b.total_particles > 0)
    launch_pdl(k_scatter<D, false, false>, dim3((b.total_particles + 255) / 256), dim3(256), 0, s, b,
               static_cast<const SelectPar*>(nullptr));
  count_launches((b.total_particles > 0 ? 1 : 0) + 2);
  return cudaGetLastError();
}

template <int D, int TB, bool ADJ>
static cudaError_t p2g_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_p2g<D, TB, ADJ, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(P2GCfg<D, TB, ADJ, 256>::SMEM));
  if constexpr (D == 2) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_p2g<D, TB, ADJ, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(P2GCfg<D, TB, ADJ, 128>::SMEM));
  }
  return e;
}

cudaError_t configure_kernels() {
  cudaError_t e;
  if ((e = p2g_configure<2, 4, false>()) != cudaSuccess) return e;
  if ((e = p2g_configure<2, 4, true>()) != cudaSuccess) return e;
  if ((e = p2g_configure<2, 8, false>()) != cudaSuccess) return e;
  if ((e = p2g_configure<2, 8, true>()) != cudaSuccess) return e;
  if ((e = p2g_configure<3, 4, false>()) != cudaSuccess) return e;
  return p2g_configure<3, 4, true>();
}

// Persistent-grid size of tile kernel k: its CTAs per SM times the SMs, at most one per tile.
static int tile_grid(const BatchDev& b, int k) {
  const int g = b.launch[k].ctas_per_sm * b.sm_count;
  const int grid = g < b.total_tiles ? g : b.total_tiles;
  return grid < 1 ? 1 : grid;
}

template <int D, int TB, bool ADJ>
static cudaError_t p2g_impl(const BatchDev& b, cudaStream_t s) {
  const int k = ADJ ? TK_P2G_ADJ : TK_P2G;
  const int grid = tile_grid(b, k);
  bool small = false;  // 128-thread CTAs (2D only)
  if constexpr (D == 2) small = b.launch[k].threads == 128;
  if constexpr (D == 2) {
    if (small)
      launch_pdl(k_p2g<D, TB, ADJ, 128>, dim3(grid), dim3(128), P2GCfg<D, TB, ADJ, 128>::SMEM, s, b);
  }
  if (!small) launch_pdl(k_p2g<D, TB, ADJ, 256>, dim3(grid), dim3(256), P2GCfg<D, TB, ADJ, 256>::SMEM, s, b);
  count_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_p2g(const BatchDev& b, bool with_adjoint, cudaStream_t s) {
  if constexpr (D == 2)
    if (wide_tiles<D>(b)) return with_adjoint ? p2g_impl<D, 8, true>(b, s) : p2g_impl<D, 8, false>(b, s);
  return with_adjoint ? p2g_impl<D, 4, true>(b, s) : p2g_impl<D, 4, false>(b, s);
}

template <int D, int TB>
static cudaError_t g2p_impl(const BatchDev& b, cudaStream_t s) {
  const int grid = tile_grid(b, TK_G2P);
  if (b.launch[TK_G2P].threads == 128)
    launch_pdl(k_g2p<D, TB, 128>, dim3(grid), dim3(128), 0, s, b);
  else
    launch_pdl(k_g2p<D, TB, 256>, dim3(grid), dim3(256), 0, s, b);
  count_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_g2p(const BatchDev& b, cudaStream_t s) {
  if constexpr (D == 2)
    if (wide_tiles<D>(b)) return g2p_impl<D, 8>(b, s);
  return g2p_impl<D, 4>(b, s);
}

template <int D, int TB>
static cudaError_t adj_gather_impl(const BatchDev& b, cudaStream_t s) {
  const int grid = tile_grid(b, TK_ADJ_GATHER);
  if (b.has_material)
    launch_pdl(k_adj_gather<D, TB, true>, dim3(grid), dim3(kAdjThreads<D>), 0, s, b);
  else
    launch_pdl(k_adj_gather<D, TB, false>, dim3(grid), dim3(kAdjThreads<D>), 0, s, b);
  count_launches(1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_adj_gather(const BatchDev& b, cudaStream_t s) {
  if constexpr (D == 2)
    if (wide_tiles<D>(b)) return adj_gather_impl<D, 8>(b, s);
  return adj_gather_impl<D, 4>(b, s);
}

template cudaError_t launch_keys<2>(const BatchDev&, cudaStream_t, const SelectPar*);
template cudaError_t launch_keys<3>(const BatchDev&, cudaStream_t, const SelectPar*);
template cudaError_t launch_sort<2>(const BatchDev&, cudaStream_t, const SelectPar*);
template cudaError_t launch_sort<3>(const BatchDev&, cudaStream_t, const SelectPar*);
template cudaError_t launch_p2g<2>(const BatchDev&, bool, cudaStream_t);
template cudaError_t launch_p2g<3>(const BatchDev&, bool, cudaStream_t);
template cudaError_t launch_g2p<2>(const BatchDev&, cudaStream_t);
template cudaError_t launch_g2p<3>(const BatchDev&, cudaStream_t);
template cudaError_t launch_adj_gather<2>(const BatchDev&, cudaStream_t);
template cudaError_t launch_adj_gather<3>(const BatchDev&, cudaStream_t);

// ============================================================================ plain form
// One scene; P2G and the adjoint scatter add into a zeroed dense grid with global float atomics;
// the grid kernels visit every node.  Same per-particle math as the tiled form.
template <int D, bool ADJ>
__global__ void k_plain_scatter(const ScenePar* __restrict__ dsp) {
  const ScenePar& sp = *dsp;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= sp.N) return;
  float r[Cfg<D>::S];
  load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, id, r);
  Part<D> q;
  unpack<D>(r, q);
  Sten<D> stn;
  if (!make_stencil<D>(q.x, sp.inv_dx, sp.n, stn)) {
    set_status(sp.status, ST_DOMAIN);
    return;
  }
  float P[D][D], A[D][D], G[D][D], sig[D];
  const PMat pm = pmat_of(sp, id);
  const float J = particle_G<D>(q, sp, group_of(sp, id), pm, P, A, G, sig);
  if (!(J > 0.0f)) set_status(sp.status, ST_INVERTED);
  float vb[D], Cb[D][D];
  if constexpr (ADJ) {
    Part<D> g1;
    load_planes<D, Cfg<D>::PLANES>(sp.adj_in, sp.npad, id, r);
    unpack<D>(r, g1);
#pragma unroll
    for (int a = 0; a < D; ++a) vb[a] = g1.v[a] + sp.dt * g1.x[a];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) s += g1.F[a][k] * q.F[c][k];
        Cb[a][c] = g1.C[a][c] + sp.dt * s;
      }
  }
  const float Dinv = 4.0f * sp.inv_dx * sp.inv_dx;
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz) {
        const int k[3] = {kx, ky, kz};
        float N = 1.0f;
        int nd[D];
        float dp[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          N *= stn.w[a][k[a]];
          nd[a] = stn.base[a] + k[a];
          dp[a] = (float(k[a]) - stn.f[a]) * sp.dx;
        }
        const int nl = lin3<D>(nd, sp.n);
        float* gp = reinterpret_cast<float*>(sp.grid + nl);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float s = pm.mass * q.v[a];
#pragma unroll
          for (int c = 0; c < D; ++c) s += G[a][c] * dp[c];
          atomicAdd(gp + a, N * s);
        }
        atomicAdd(gp + (D == 2 ? 2 : 3), N * pm.mass);
        if constexpr (ADJ) {
          float* gb = reinterpret_cast<float*>(sp.grid_b + nl);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            float s = vb[a];
#pragma unroll
            for (int c = 0; c < D; ++c) s += Dinv * Cb[a][c] * dp[c];
            atomicAdd(gb + a, N * s);
          }
        }
      }
}

template <int D, bool ADJ>
__global__ void k_plain_grid(const ScenePar* __restrict__ dsp, int n_nodes) {
  const ScenePar& sp = *dsp;
  const int nl = blockIdx.x * blockDim.x + threadIdx.x;
  if (nl >= n_nodes) return;
  int node[D];
  unlin<D>(nl, sp.n, node);
  const float4 s4 = sp.grid[nl];
  const float s[4] = {s4.x, s4.y, s4.z, s4.w};
  const float m = D == 2 ? s[2] : s[3];
  float vraw[D], v[D];
  if (m > 0.0f) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vraw[a] = s[a] / m;
      v[a] = vraw[a] + sp.dt * sp.gravity[a];
    }
    bc_apply<D>(node, sp.n, sp.bc, v);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = vraw[a] = 0.0f;
  }
  if constexpr (D == 2)
    sp.grid[nl] = make_float4(v[0], v[1], m, 0.0f);
  else
    sp.grid[nl] = make_float4(v[0], v[1], v[2], m);
  if constexpr (ADJ) {
    const float4 b4 = sp.grid_b[nl];
    float g[D] = {};
    float pb[D], mb = 0.0f;
    g[0] = b4.x;
    g[1] = b4.y;
    if constexpr (D == 3) g[D == 3 ? 2 : 0] = b4.z;
    if (m > 0.0f) {
      float vg[D];
#pragma unroll
      for (int a = 0; a < D; ++a) vg[a] = vraw[a] + sp.dt * sp.gravity[a];
      bc_adjoint<D>(node, sp.n, sp.bc, vg, g);
      float dot = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        pb[a] = g[a] / m;
        dot += vraw[a] * g[a];
      }
      mb = -dot / m;
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) pb[a] = 0.0f;
    }
    if constexpr (D == 2)
      sp.grid_b[nl] = make_float4(pb[0], pb[1], mb, 0.0f);
    else
      sp.grid_b[nl] = make_float4(pb[0], pb[1], pb[2], mb);
  }
}

template <int D>
__global__ void k_plain_g2p(const ScenePar* __restrict__ dsp) {
  const ScenePar& sp = *dsp;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id == 0 && sp.step_ctr) *sp.step_ctr += 1;
  if (id >= sp.N) return;
  float r[Cfg<D>::S];
  load_planes<D, Cfg<D>::XF_PLANES>(sp.planes, sp.npad, id, r);
  Part<D> q;
  unpack<D>(r, q);
  Sten<D> stn;
  if (!make_stencil<D>(q.x, sp.inv_dx, sp.n, stn)) return;  // status already set by the scatter
  g2p_core<D>(q, stn.f, stn.w, sp.dt, sp.inv_dx, [&](int kx, int ky, int kz) {
    int nd[D];
    nd[0] = stn.base[0] + kx;
    nd[1] = stn.base[1] + ky;
    if constexpr (D == 3) nd[D == 3 ? 2 : 0] = stn.base[D == 3 ? 2 : 0] + kz;
    return sp.grid[lin3<D>(nd, sp.n)];
  });
  pack<D>(q, r);
  store_planes<D, Cfg<D>::PLANES>(sp.planes_out, sp.npad, id, r);
}

template <int D>
__global__ void k_plain_gather(const ScenePar* __restrict__ dsp) {
  const ScenePar& sp = *dsp;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= sp.N) return;
  float r[Cfg<D>::S];
  load_planes<D, Cfg<D>::PLANES>(sp.planes, sp.npad, id, r);
  Part<D> q, g1, g0;
  unpack<D>(r, q);
  load_planes<D, Cfg<D>::PLANES>(sp.adj_in, sp.npad, id, r);
  unpack<D>(r, g1);
  Sten<D> stn;
  if (!make_stencil<D>(q.x, sp.inv_dx, sp.n, stn)) return;
  const float c = adj_core<D, true>(q, g1, stn.f, stn.w, stn.dw, sp, id, group_of(sp, id), [&](int kx, int ky, int kz, float4& v, float4& p) {
    int nd[D];
    nd[0] = stn.base[0] + kx;
    nd[1] = stn.base[1] + ky;
    if constexpr (D == 3) nd[D == 3 ? 2 : 0] = stn.base[D == 3 ? 2 : 0] + kz;
    const int nl = lin3<D>(nd, sp.n);
    v = sp.grid[nl];
    p = sp.grid_b[nl];
  }, [](Part<D>&, Part<D>&) {}, g0);
  pack<D>(g0, r);
  store_planes<D, Cfg<D>::PLANES>(sp.adj_out, sp.npad, id, r);
  sp.sig_contrib[id] = c;
}

// Per-block (256 particles) group sums of the (K) contributions of the plain form.
__global__ void k_plain_group_partials(const ScenePar* __restrict__ dsp, float* __restrict__ gpart) {
  const ScenePar& sp = *dsp;
  __shared__ float wpart[8][MAX_GROUPS];
  const int id = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int g = -1;
  float c = 0.0f;
  if (id < sp.N) {
    g = sp.group ? sp.group[id] : -1;
    if (g >= sp.G) g = -1;
    c = sp.sig_contrib[id];
  }
  float lo = 0.0f, hi = 0.0f;
  warp_group_add(g, c, lo, hi);
  wpart[warp][lane] = lo;
  wpart[warp][lane + 32] = hi;
  __syncthreads();
  if (threadIdx.x < MAX_GROUPS) {
    float s = 0.0f;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += wpart[w][threadIdx.x];
    gpart[size_t(blockIdx.x) * MAX_GROUPS + threadIdx.x] = s;
  }
}

static int host_nodes(const ScenePar& sp) {
  int c = 1;
  for (int a = 0; a < sp.dim; ++a) c *= sp.n[a];
  return c;
}

template <int D>
cudaError_t launch_plain_step(const ScenePar* dsp, const ScenePar& sp, cudaStream_t s) {
  const int nn = host_nodes(sp);
  cudaError_t e = cudaMemsetAsync(sp.grid, 0, sizeof(float4) * size_t(nn), s);
  if (e != cudaSuccess) return e;
  if (sp.N > 0) k_plain_scatter<D, false><<<(sp.N + 255) / 256, 256, 0, s>>>(dsp);
  k_plain_grid<D, false><<<(nn + 255) / 256, 256, 0, s>>>(dsp, nn);
  k_plain_g2p<D><<<(sp.N + 255) / 256 + (sp.N == 0), 256, 0, s>>>(dsp);
  count_launches(sp.N > 0 ? 3 : 2);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_plain_adjoint(const ScenePar* dsp, const ScenePar& sp, float* gpart, cudaStream_t s) {
  const int nn = host_nodes(sp);
  cudaError_t e = cudaMemsetAsync(sp.grid, 0, sizeof(float4) * size_t(nn), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sp.grid_b, 0, sizeof(float4) * size_t(nn), s);
  if (e != cudaSuccess) return e;
  if (sp.N > 0) k_plain_scatter<D, true><<<(sp.N + 255) / 256, 256, 0, s>>>(dsp);
  k_plain_grid<D, true><<<(nn + 255) / 256, 256, 0, s>>>(dsp, nn);
  if (sp.N > 0) k_plain_gather<D><<<(sp.N + 255) / 256, 256, 0, s>>>(dsp);
  if (sp.N > 0) k_plain_group_partials<<<(sp.N + 255) / 256, 256, 0, s>>>(dsp, gpart);
  count_launches(sp.N > 0 ? 4 : 1);
  return cudaGetLastError();
}

template cudaError_t launch_plain_step<2>(const ScenePar*, const ScenePar&, cudaStream_t);
template cudaError_t launch_plain_step<3>(const ScenePar*, const ScenePar&, cudaStream_t);
template cudaError_t launch_plain_adjoint<2>(const ScenePar*, const ScenePar&, float*, cudaStream_t);
template cudaError_t launch_plain_adjoint<3>(const ScenePar*, const ScenePar&, float*, cudaStream_t);

// ============================================================================ pack / unpack
// Storage slot p takes caller particle q = order[p] (q = p without an order).
__global__ void k_pack(int dim, int N, int npad, const float* x, const float* v, const float* C, const float* F,
                       float4* planes, int* status, const int* __restrict__ order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npad) return;
  const int S = dim == 2 ? 12 : 24, d2 = dim * dim;
  float r[24];
  if (p < N) {
    const size_t q = order ? size_t(order[p]) : size_t(p);
    int o = 0;
    for (int a = 0; a < dim; ++a) r[o++] = x[q * dim + a];
    for (int a = 0; a < d2; ++a) r[o++] = F ? F[q * d2 + a] : ((a % (dim + 1)) == 0 ? 1.0f : 0.0f);
    for (int a = 0; a < dim; ++a) r[o++] = v ? v[q * dim + a] : 0.0f;
    for (int a = 0; a < d2; ++a) r[o++] = C ? C[q * d2 + a] : 0.0f;
    for (int a = 0; a < S; ++a)
      if (!(r[a] == r[a]) || fabsf(r[a]) > 3.0e38f) set_status(status, -1);
  } else {
    for (int a = 0; a < S; ++a) r[a] = 0.0f;
  }
  for (int j = 0; j < S / 4; ++j) planes[size_t(j) * npad + p] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
}

// Storage slot p goes to caller particle q = order[p] (q = p without an order).
__global__ void k_unpack(int dim, int N, int npad, const float4* planes, float* x, float* v, float* C, float* F,
                         const int* __restrict__ order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const size_t qo = order ? size_t(order[p]) : size_t(p);
  const int S = dim == 2 ? 12 : 24, d2 = dim * dim;
  float r[24];
  for (int j = 0; j < S / 4; ++j) {
    float4 q = planes[size_t(j) * npad + p];
    r[4 * j] = q.x;
    r[4 * j + 1] = q.y;
    r[4 * j + 2] = q.z;
    r[4 * j + 3] = q.w;
  }
  int o = 0;
  for (int a = 0; a < dim; ++a, ++o)
    if (x) x[qo * dim + a] = r[o];
  for (int a = 0; a < d2; ++a, ++o)
    if (F) F[qo * d2 + a] = r[o];
  for (int a = 0; a < dim; ++a, ++o)
    if (v) v[qo * dim + a] = r[o];
  for (int a = 0; a < d2; ++a, ++o)
    if (C) C[qo * d2 + a] = r[o];
}

// Device-side choice of this step's scene records: scene s of the launch uses
// table[map[*ctr - base]] (map NULL: table[0]), with the batch offsets patched in; the
// sinusoid controllers' actuation a_g(t_n) is evaluated here too.  Every step of a rollout is
// then the same launch sequence, which CUDA graphs replay.  (A single tiled scene makes this
// selection inside the first kernel of its step instead: k_keys, k_scatter, k_scan_reduce.)
__global__ void k_select(const SelectPar* __restrict__ sel, ScenePar* __restrict__ cur) {
  pdl_enter();
  select_publish(sel[blockIdx.x], cur + blockIdx.x);
}

cudaError_t launch_select(const SelectPar* sel, int n_scenes, ScenePar* cur, cudaStream_t s) {
  if (n_scenes <= 0) return cudaSuccess;
  launch_pdl(k_select, dim3(n_scenes), dim3(64), 0, s, sel, cur);
  count_launches(1);
  return cudaGetLastError();
}

// Adjoint planes of the seed dL/dx_T = e_0 / N (loss = mean final x_0), zero elsewhere and in the
// padding: what k_pack writes for that seed with zero v, C and F seeds.
__global__ void k_seed_mean_x0(int dim, int N, int npad, float4* planes) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npad) return;
  const int S = dim == 2 ? 12 : 24;
  const float s0 = p < N ? 1.0f / float(N) : 0.0f;
  for (int j = 0; j < S / 4; ++j) planes[size_t(j) * npad + p] = make_float4(j == 0 ? s0 : 0.0f, 0.0f, 0.0f, 0.0f);
}

cudaError_t launch_seed_mean_x0(int dim, int N, int npad, float4* planes, cudaStream_t s) {
  if (npad == 0) return cudaSuccess;
  k_seed_mean_x0<<<(npad + 255) / 256, 256, 0, s>>>(dim, N, npad, planes);
  count_launches(1);
  return cudaGetLastError();
}

// Writes of many counters in one launch, in list order (one thread: the list may name a counter
// twice), and the gather of many status words into one array.
__global__ void k_set_int_list(IntPtrList l) {
  if (threadIdx.x == 0)
    for (int i = 0; i < l.n; ++i) *l.ptr[i] = l.val[i];
}

__global__ void k_gather_ints(IntPtrList l, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < l.n) out[i] = *l.ptr[i];
}

cudaError_t launch_set_int_list(const IntPtrList& l, cudaStream_t s) {
  if (l.n <= 0) return cudaSuccess;
  k_set_int_list<<<1, 32, 0, s>>>(l);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_ints(const IntPtrList& l, int* out, cudaStream_t s) {
  if (l.n <= 0) return cudaSuccess;
  k_gather_ints<<<(l.n + 255) / 256, 256, 0, s>>>(l, out);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_set_int(int* p, int v) { *p = v; }

cudaError_t launch_set_int(int* p, int v, cudaStream_t s) {
  k_set_int<<<1, 1, 0, s>>>(p, v);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack(int dim, int N, int npad, const float* x, const float* v, const float* C, const float* F,
                        float4* planes, int* status, const int* order, cudaStream_t s) {
  if (npad == 0) return cudaSuccess;
  k_pack<<<(npad + 255) / 256, 256, 0, s>>>(dim, N, npad, x, v, C, F, planes, status, order);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int dim, int N, int npad, const float4* planes, float* x, float* v, float* C, float* F,
                          const int* order, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  k_unpack<<<(N + 255) / 256, 256, 0, s>>>(dim, N, npad, planes, x, v, C, F, order);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace gbmpm
