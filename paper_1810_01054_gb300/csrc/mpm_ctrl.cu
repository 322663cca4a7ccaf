// Actuation controllers and their adjoints (Section V-B: a = tanh(W z + b) generating the
// actuation of every group at every step), plus the deterministic per-group reductions they
// need: group centroids of x (controller input) and per-group sums of dL/da (Supplement S4 (K)).
//
// Reductions are two-level with a fixed order at both levels (group sums of x and v: segmented
// scans over the particles in group order, warps combine in warp order, rows in row order; dL/da:
// per-tile rows in row order), so they are bitwise reproducible.  The MLP's dot products give each
// output 16 threads and a fixed butterfly.
#include "mpm_internal.h"

namespace gbmpm {

constexpr float kTwoPi = 6.283185307179586f;
constexpr int RED_WARPS = 8;
constexpr int RED_WR = 64;                        // particles per warp
constexpr int RED_ROW = RED_WARPS * RED_WR;       // particles per partial row
constexpr int RED_STRIDE = MAX_GROUPS * 3 + 3;    // floats per row: [64 groups][3] + body[3]

int reduction_rows(int N) { return (N + RED_ROW - 1) / RED_ROW; }

// Group sums of x (mode 0) or v (mode 2), dim channels, and the body sum, over the particles in
// group order: perm lists the particles by group (stable; ungrouped first) and pgroup[i] is the
// group of perm[i] (-1: none), both fixed at scene creation.  A warp takes 32 consecutive entries
// at a time, where every group is one run of lanes: a segmented scan over the lanes gives each
// run's sum at its last lane, which adds it to the warp's accumulator of that group (one writer
// per group and chunk, chunks in order).  Warps then combine in warp order into the block's row.
template <int CH>
__global__ void __launch_bounds__(256) k_group_rows(const ScenePar* __restrict__ dsp, float* __restrict__ rows,
                                                    int mode, const int* __restrict__ perm,
                                                    const int* __restrict__ pgroup) {
  pdl_enter();
  const ScenePar& sp = *dsp;
  __shared__ float wacc[RED_WARPS][MAX_GROUPS][CH];
  __shared__ float wbody[RED_WARPS][CH];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int start = blockIdx.x * RED_ROW + w * RED_WR;
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);  // lanes 0..lane
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    wacc[w][lane][c] = 0.0f;
    wacc[w][lane + 32][c] = 0.0f;
  }
  __syncwarp();
  float body[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) body[c] = 0.0f;
  // every chunk's loads are issued first (K chunks per warp), then the chunks are summed in order
  constexpr int K = RED_WR / 32;
  int gk[K];
  float vk[K][CH];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = start + 32 * k + lane;
    gk[k] = -2;  // past the end
#pragma unroll
    for (int c = 0; c < CH; ++c) vk[k][c] = 0.0f;
    if (i < sp.N) {
      const int p = perm[i];
      gk[k] = pgroup[i];
      if (mode == 0) {
        const float4 q = sp.planes[p];
        const float xv[3] = {q.x, q.y, q.z};
#pragma unroll
        for (int c = 0; c < CH; ++c) vk[k][c] = xv[c];
      } else {  // v: floats D + D*D .. of the state, inside one plane for D = 2, 3
        constexpr int O = CH + CH * CH;
        const float4 q = sp.planes[size_t(O / 4) * sp.npad + p];
        const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int c = 0; c < CH; ++c) vk[k][c] = qv[O % 4 + c];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int g = gk[k];
    float val[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) val[c] = vk[k][c];
#pragma unroll
    for (int c = 0; c < CH; ++c) body[c] += val[c];
    const int gp = __shfl_up_sync(0xffffffffu, g, 1);
    const int gn = __shfl_down_sync(0xffffffffu, g, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || gp != g);
    const int first = 31 - __clz(heads & upto);  // first lane of this lane's run
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float t = __shfl_up_sync(0xffffffffu, val[c], o);
        if (lane - o >= first) val[c] += t;
      }
    }
    if (g >= 0 && (lane == 31 || gn != g)) {
#pragma unroll
      for (int c = 0; c < CH; ++c) wacc[w][g][c] += val[c];
    }
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    float b = body[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (lane == 0) wbody[w][c] = b;
  }
  __syncthreads();
  float* row = rows + size_t(blockIdx.x) * RED_STRIDE;
  for (int i = threadIdx.x; i < MAX_GROUPS * CH; i += blockDim.x) {
    const int g = i / CH, c = i - g * CH;
    float s = 0.0f;
    for (int ww = 0; ww < RED_WARPS; ++ww) s += wacc[ww][g][c];
    row[g * 3 + c] = s;
  }
  if (threadIdx.x < CH) {
    float s = 0.0f;
    for (int ww = 0; ww < RED_WARPS; ++ww) s += wbody[ww][threadIdx.x];
    row[MAX_GROUPS * 3 + threadIdx.x] = s;
  }
}

// Sum rows in a fixed order into out[g*3+c] (groups) and out[192+c] (body); 1024-thread CTA.  Only
// the U = (G + 1) CH outputs in use are summed, each by S = 1024 / U interleaved splits combined
// in split order; the other outputs are set to zero.
__device__ void reduce_rows(const float* __restrict__ rows, int n_rows, int G, int CH, float* out) {
  __shared__ float part[1024];
  const int O = MAX_GROUPS * 3 + 3;  // outputs
  const int U = (G + 1) * CH;        // outputs in use
  const int S = blockDim.x / U;      // splits per output in use
  const int u = threadIdx.x % U, s = threadIdx.x / U;
  auto out_index = [&](int v) { return v < G * CH ? (v / CH) * 3 + v % CH : MAX_GROUPS * 3 + (v - G * CH); };
  float acc = 0.0f;
  if (s < S) {
    const int o = out_index(u);
    for (int r = s; r < n_rows; r += S) acc += rows[size_t(r) * RED_STRIDE + o];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < U) {
    float t = 0.0f;
    for (int k = 0; k < S; ++k) t += part[k * U + threadIdx.x];
    out[out_index(threadIdx.x)] = t;
  }
  if (threadIdx.x < O) {
    const int o = threadIdx.x;
    const bool used = o < MAX_GROUPS * 3 ? (o / 3 < G && o % 3 < CH) : (o - MAX_GROUPS * 3 < CH);
    if (!used) out[o] = 0.0f;
  }
  __syncthreads();
}

// out_o = sum_j A[o * so + j * sj] x[j] for o < n_out, j < n_in, in a 1024-thread CTA: 16 threads
// per output (thread t sums j = t, t + 16, ... in order, then a fixed butterfly over the 16), 64
// outputs per pass; fin(o, sum) runs on the first thread of each output.  Every thread calls it.
template <class F>
__device__ __forceinline__ void dot_rows(const float* A, int so, int sj, const float* x, int n_in, int n_out, F fin) {
  const int t = threadIdx.x & 15;
  for (int o0 = 0; o0 < n_out; o0 += 64) {
    const int o = o0 + (threadIdx.x >> 4);
    float u = 0.0f;
    if (o < n_out)
      for (int j = t; j < n_in; j += 16) u += A[size_t(o) * so + size_t(j) * sj] * x[j];
#pragma unroll
    for (int m = 8; m > 0; m >>= 1) u += __shfl_xor_sync(0xffffffffu, u, m);
    if (o < n_out && t == 0) fin(o, u);
  }
}

// The MLP's parameters (W1, b1, W2, b2, W3, b3, contiguous) copied to shared memory in one pass
// when they fit (the soft body's 48-64-64-16 network: 8336 floats), so the layers read no global
// memory; else the global copy.  Every thread calls it; it ends with a barrier either way.
constexpr int MLP_STAGE = 8704;
__device__ const float* mlp_params(const CtrlPar& c) {
  __shared__ float stage[MLP_STAGE];
  const int G = c.G, Z = G * c.dim, H = c.hidden;
  const int n = H * Z + H + H * H + H + G * H + G;
  const bool fits = n <= MLP_STAGE;  // uniform
  if (fits)
    for (int i = threadIdx.x; i < n; i += blockDim.x) stage[i] = c.params[i];
  __syncthreads();
  return fits ? stage : c.params;
}

// The MLP's three layers from its input z (shared): h1, h2 (shared) and fin3(g, u3), u3 the last
// layer's pre-activation, with parameters P (mlp_params).  The forward and the reverse step's
// replay share it, so they agree bit for bit.
template <class F>
__device__ __forceinline__ void mlp_layers(const CtrlPar& c, const float* P, const float* z, float* h1, float* h2,
                                           F fin3) {
  const int G = c.G, Z = G * c.dim, H = c.hidden;
  const float* W1 = P;
  const float* b1 = W1 + H * Z;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + G * H;
  dot_rows(W1, Z, 1, z, Z, H, [&](int o, float u) { h1[o] = tanhf(u + b1[o]); });
  __syncthreads();
  dot_rows(W2, H, 1, h1, H, H, [&](int o, float u) { h2[o] = tanhf(u + b2[o]); });
  __syncthreads();
  dot_rows(W3, H, 1, h2, H, G, [&](int o, float u) { fin3(o, u + b3[o]); });
}

// ----------------------------------------------------------------------------- forward
// MLP controller of step n = *step_ctr (the sinusoid forms are evaluated by the record
// selection): group centroids from the partial rows, then the three tanh layers -> sp.act.
__global__ void __launch_bounds__(1024) k_ctrl_forward(const ScenePar* __restrict__ dsp, CtrlPar c, const float* rows,
                                                       int n_rows) {
  pdl_enter();
  const ScenePar& sp = *dsp;
  __shared__ float red[MAX_GROUPS * 3 + 3];
  __shared__ float z[MAX_GROUPS * 3], h1[MAX_HIDDEN], h2[MAX_HIDDEN];
  const int G = c.G, tid = threadIdx.x;
  const int dim = c.dim, Z = G * dim;
  reduce_rows(rows, n_rows, G, dim, red);
  if (tid < Z) {
    const int g = tid / dim, a = tid - g * dim;
    const float cg = red[g * 3 + a] * c.inv_count[g];
    const float cb = red[MAX_GROUPS * 3 + a] * c.inv_n;
    z[tid] = cg - cb;
    float* cen = sp.ctrl_z ? sp.ctrl_z : c.centroid;
    cen[tid] = cg;
    if (tid < dim) cen[Z + tid] = cb;
  }
  const float* P = mlp_params(c);  // its barrier also publishes z
  mlp_layers(c, P, z, h1, h2, [&](int g, float u) { sp.act[g] = c.scale * tanhf(u); });
}

// Closed-loop controller of step n (type 4, Section V-B): z = [target, c_g, u_g] with c_g, u_g the
// group means of x and v (partial rows of x, then of v), a = scale * tanh(W z + b) -> sp.act; z is
// kept for the reverse step (in the record's controller slot, else in c.centroid).
__global__ void __launch_bounds__(1024) k_ctrl_forward_com(const ScenePar* __restrict__ dsp, CtrlPar c,
                                                           const float* rows, int n_rows) {
  pdl_enter();
  const ScenePar& sp = *dsp;
  __shared__ float rx[MAX_GROUPS * 3 + 3], rv[MAX_GROUPS * 3 + 3];
  __shared__ float z[3 * (1 + 2 * MAX_GROUPS)];
  const int G = c.G, dim = c.dim, tid = threadIdx.x, Z = dim * (1 + 2 * G);
  reduce_rows(rows, n_rows, G, dim, rx);
  reduce_rows(rows + size_t(n_rows) * (MAX_GROUPS * 3 + 3), n_rows, G, dim, rv);
  if (tid < Z) {
    float val;
    if (tid < dim) {
      val = c.params[tid];
    } else if (tid < dim + G * dim) {
      const int i = tid - dim;
      val = rx[(i / dim) * 3 + i % dim] * c.inv_count[i / dim];
    } else {
      const int i = tid - dim - G * dim;
      val = rv[(i / dim) * 3 + i % dim] * c.inv_count[i / dim];
    }
    z[tid] = val;
    (sp.ctrl_z ? sp.ctrl_z : c.centroid)[tid] = val;
  }
  __syncthreads();
  const float* b = c.params + dim + size_t(G) * Z;
  dot_rows(c.params + dim, Z, 1, z, Z, G, [&](int g, float u) { sp.act[g] = c.scale * tanhf(u + b[g]); });
}

// ----------------------------------------------------------------------------- backward
// dL/da_g = sum over the group of the (K) contributions; accumulate dL/dparams for step n;
// for the MLP also dL/dz, turned into per-group coefficients for the x adjoint.
// First index i in [0, n) with a[i] >= key (a ascending), found by one warp in 32-way steps: each
// round probes 32 evenly spaced entries and keeps the interval between the last probe below key and
// the first probe at or above it.  All 32 lanes call it and get the same result.
__device__ __forceinline__ int first_at_least(const int* a, int n, int key) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int step = (hi - lo + 31) / 32;
    const int p = lo + lane * step;
    const bool ge = p < hi && a[p] >= key;
    const unsigned m = __ballot_sync(0xffffffffu, ge) | __ballot_sync(0xffffffffu, p >= hi);
    const int f = m ? __ffs(m) - 1 : 32;  // first probe at/above key (or past the end)
    if (f == 0) return lo;
    const int nlo = lo + (f - 1) * step + 1;
    const int nhi = f < 32 ? lo + f * step : hi;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
  }
  return lo;
}

// dL/da_g of one step = sum of rows [lo, hi) of the per-tile (per-block) partials, 16 fixed
// interleaved splits per group combined in split order; into ga (shared) and act_grad.
__device__ void ctrl_group_sums(const CtrlPar& c, int lo, int hi, float* ga, float* act_grad) {
  __shared__ float part[16][MAX_GROUPS];
  const int G = c.G, tid = threadIdx.x;
  const int g = tid & (MAX_GROUPS - 1), split = tid >> 6;
  float acc = 0.0f;
  if (g < G)
    for (int r = lo + split; r < hi; r += 16) acc += c.gpart[size_t(r) * MAX_GROUPS + g];
  part[split][g] = acc;
  __syncthreads();
  if (tid < G) {
    float t = 0.0f;
    for (int k = 0; k < 16; ++k) t += part[k][tid];
    ga[tid] = t;
    act_grad[tid] = t;
  }
  __syncthreads();
}

// Parameter adjoint of the forms that read no state, step n at time t: sinusoid amplitude (type 0),
// sinusoid basis (type 1), per-step table (type 3).
__device__ void ctrl_open_params(const CtrlPar& c, int n, float t, const float* ga) {
  const int G = c.G, tid = threadIdx.x;
  if (c.type == 0) {
    if (tid < G) c.gparams[tid] += ga[tid] * sinf(kTwoPi * c.freq * t);
  } else if (c.type == 3) {  // table: dL/dU[n][g] = dL/da_g(t_n)
    if (tid < G && n >= 0 && n < c.hidden) c.gparams[size_t(n) * G + tid] += ga[tid];
  } else if (c.type == 1) {
    if (tid < G * 4) {
      const int g = tid / 4, j = tid - 4 * g;
      const float w = kTwoPi * c.freq * t;
      const float bs[4] = {sinf(w), cosf(w), sinf(2.0f * w), cosf(2.0f * w)};
      c.gparams[tid] += ga[g] * bs[j];
    }
  }
}

// STATE: the forms that read the state (closed loop, MLP) are compiled in; without it the kernel
// handles only the open-loop forms and needs no room for the MLP's parameters.
template <bool STATE>
__device__ void ctrl_backward_body(const ScenePar& sp, const CtrlPar& c) {
  __shared__ float ga[MAX_GROUPS], z[MAX_GROUPS * 3], h1[MAX_HIDDEN], h2[MAX_HIDDEN], o3[MAX_GROUPS];
  __shared__ float gu3[MAX_GROUPS], gu2[MAX_HIDDEN], gu1[MAX_HIDDEN];
  int* step_ctr = sp.step_ctr;
  const int n = *step_ctr;
  const float t = float(n) * sp.dt;
  const int G = c.G, tid = threadIdx.x;
  {
    __shared__ int range[2];  // this scene's rows
    if (tid < 32) {
      int lo = 0, hi = c.plain_rows;
      if (c.active) {
        const int na = *c.n_active;
        if (c.whole) {
          hi = na;
        } else {
          lo = first_at_least(c.active, na, sp.tile_base);
          hi = first_at_least(c.active, na, sp.tile_base + sp.n_tiles);
        }
      }
      if (tid == 0) {
        range[0] = lo;
        range[1] = hi;
      }
    }
    __syncthreads();
    ctrl_group_sums(c, range[0], range[1], ga, sp.act_grad);
  }
  if (!STATE || c.type == 0 || c.type == 1 || c.type == 3) {
    ctrl_open_params(c, n, t, ga);
  } else if (c.type == 4) {  // closed loop: z of this step as its forward kept it
    const int dim = c.dim, Z = dim * (1 + 2 * G);
    const float* cen = sp.ctrl_z ? sp.ctrl_z : c.centroid;
    __shared__ float gu4[MAX_GROUPS];
    const float* b = c.params + dim + size_t(G) * Z;
    dot_rows(c.params + dim, Z, 1, cen, Z, G, [&](int g, float u) {
      const float th = tanhf(u + b[g]);
      gu4[g] = ga[g] * c.scale * (1.0f - th * th);
      c.gparams[dim + size_t(G) * Z + g] += gu4[g];  // b
    });
    __syncthreads();
    for (int i = tid; i < G * Z; i += blockDim.x) c.gparams[dim + i] += gu4[i / Z] * cen[i % Z];  // W
    // dL/dz: the target's part goes to its parameters, the group means' to gz
    dot_rows(c.params + dim, 1, Z, gu4, G, Z, [&](int j, float u) {
      if (j < dim)
        c.gparams[j] += u;
      else
        c.gz[j - dim] = u;  // [c_g part (G*dim)][u_g part (G*dim)]
    });
  } else {
    const int dim = c.dim, Z = G * dim, H = c.hidden;
    const float* P = mlp_params(c);
    const float* W1 = P;
    const float* b1 = W1 + H * Z;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    float* gW1 = c.gparams;
    float* gb1 = gW1 + H * Z;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + G * H;
    // forward replay from the centroids of this step (kept by k_ctrl_forward)
    const float* cen = sp.ctrl_z ? sp.ctrl_z : c.centroid;
    if (tid < Z) z[tid] = cen[tid] - cen[Z + tid % dim];
    __syncthreads();
    mlp_layers(c, P, z, h1, h2, [&](int g, float u) {
      o3[g] = tanhf(u);
      gu3[g] = ga[g] * c.scale * (1.0f - o3[g] * o3[g]);
      gb3[g] += gu3[g];
    });
    __syncthreads();
    for (int i = tid; i < G * H; i += blockDim.x) gW3[i] += gu3[i / H] * h2[i % H];
    dot_rows(W3, 1, H, gu3, G, H, [&](int i, float u) {
      gu2[i] = u * (1.0f - h2[i] * h2[i]);
      gb2[i] += gu2[i];
    });
    __syncthreads();
    for (int i = tid; i < H * H; i += blockDim.x) gW2[i] += gu2[i / H] * h1[i % H];
    dot_rows(W2, 1, H, gu2, H, H, [&](int i, float u) {
      gu1[i] = u * (1.0f - h1[i] * h1[i]);
      gb1[i] += gu1[i];
    });
    __syncthreads();
    for (int i = tid; i < H * Z; i += blockDim.x) gW1[i] += gu1[i / Z] * z[i % Z];
    dot_rows(W1, 1, Z, gu1, H, Z, [&](int j, float u) { c.gz[j] = u; });
  }
  __syncthreads();
  if (tid == 0) *step_ctr = n - 1;
}

template <bool STATE>
__global__ void __launch_bounds__(1024) k_ctrl_backward(const ScenePar* __restrict__ dsp, CtrlPar c) {
  pdl_enter();
  ctrl_backward_body<STATE>(*dsp, c);
}

// Reverse of a form that reads no state for one step of a scene alone: the adjoint gather of the
// step rewound the counter to n - 1 and kept the step's active-slot count in *rows.  Reads no scene
// record, so it may run while the next reverse step selects and publishes its own.
__global__ void __launch_bounds__(1024) k_ctrl_backward_open(CtrlPar c, const int* __restrict__ ctr,
                                                             const int* __restrict__ rows, float dt,
                                                             float* act_grad) {
  pdl_enter();
  __shared__ float ga[MAX_GROUPS];
  const int n = *ctr + 1;
  ctrl_group_sums(c, 0, *rows, ga, act_grad);
  ctrl_open_params(c, n, float(n) * dt, ga);
}

// One block per scene of a batch: scene i uses cur[i] and cs[i].
__global__ void __launch_bounds__(1024) k_ctrl_backward_multi(const ScenePar* __restrict__ cur,
                                                              const CtrlPar* __restrict__ cs) {
  pdl_enter();
  ctrl_backward_body<true>(cur[blockIdx.x], cs[blockIdx.x]);
}

// x (and, for the closed-loop form, v) adjoint of the controller input: the MLP's centroids
// (z_g = c_g - c_body, so the body term), or the closed-loop form's group means of x and v.
template <int D>
__global__ void k_ctrl_scatter_x(const ScenePar* __restrict__ dsp, CtrlPar c) {
  pdl_enter();
  const ScenePar& sp = *dsp;
  __shared__ float coef[MAX_GROUPS * 3], coefv[MAX_GROUPS * 3], body[3];
  const int G = c.G;
  const bool com = c.type == 4;
  for (int i = threadIdx.x; i < G * D; i += blockDim.x) {
    coef[i] = c.gz[i] * c.inv_count[i / D];
    coefv[i] = com ? c.gz[G * D + i] * c.inv_count[i / D] : 0.0f;
  }
  if (threadIdx.x < D) {
    float s = 0.0f;
    for (int g = 0; g < G; ++g) s += c.gz[g * D + threadIdx.x];
    body[threadIdx.x] = com ? 0.0f : -s * c.inv_n;
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= sp.N) return;
  const int g = sp.group ? sp.group[p] : -1;
  float4 q = sp.adj_out[p];
  float add[3] = {body[0], body[1], D == 3 ? body[D == 3 ? 2 : 0] : 0.0f};
  if (g >= 0 && g < G) {
#pragma unroll
    for (int a = 0; a < D; ++a) add[a] += coef[g * D + a];
  }
  q.x += add[0];
  q.y += add[1];
  if (D == 3) q.z += add[2];
  sp.adj_out[p] = q;
  if (com && g >= 0 && g < G) {  // v: floats D + D*D .. of the adjoint state, inside one plane
    constexpr int O = D + D * D;
    float4* pv = sp.adj_out + size_t(O / 4) * sp.npad + p;
    float4 w = *pv;
    float* wc = reinterpret_cast<float*>(&w);
#pragma unroll
    for (int a = 0; a < D; ++a) wc[O % 4 + a] += coefv[g * D + a];
    *pv = w;
  }
}

// Controller forward for one step: the forms that read the state (MLP on centroids, closed loop on
// group means of x and v): group rows, then the controller.
cudaError_t ctrl_step_forward(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s) {
  if (!ctrl_reads_state(c)) return cudaSuccess;
  const int rows = reduction_rows(sp.N);
  const bool com = c.type == 4;
  int n = 0;
  if (rows > 0) {
    float* vrows = c.partials + size_t(rows) * RED_STRIDE;
    if (sp.dim == 2) {
      launch_pdl(k_group_rows<2>, dim3(rows), dim3(256), 0, s, dsp, c.partials, 0, c.perm, c.pgroup);
      if (com) launch_pdl(k_group_rows<2>, dim3(rows), dim3(256), 0, s, dsp, vrows, 2, c.perm, c.pgroup);
    } else {
      launch_pdl(k_group_rows<3>, dim3(rows), dim3(256), 0, s, dsp, c.partials, 0, c.perm, c.pgroup);
      if (com) launch_pdl(k_group_rows<3>, dim3(rows), dim3(256), 0, s, dsp, vrows, 2, c.perm, c.pgroup);
    }
    n += com ? 2 : 1;
  }
  if (com)
    launch_pdl(k_ctrl_forward_com, dim3(1), dim3(1024), 0, s, dsp, c, c.partials, rows);
  else
    launch_pdl(k_ctrl_forward, dim3(1), dim3(1024), 0, s, dsp, c, c.partials, rows);
  count_launches(n + 1);
  return cudaGetLastError();
}

cudaError_t ctrl_backward_open(const CtrlPar& c, const int* ctr, const int* rows, float dt, float* act_grad,
                               cudaStream_t s) {
  launch_pdl(k_ctrl_backward_open, dim3(1), dim3(1024), 0, s, c, ctr, rows, dt, act_grad);
  count_launches(1);
  return cudaGetLastError();
}

// Reverse of the controllers of n scenes (records cur[i], controllers cs[i], both on the device);
// the MLP scenes' centroid adjoint is added to their dL/dx separately (ctrl_scatter_x).
cudaError_t ctrl_backward_batched(const ScenePar* cur, const CtrlPar* cs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  launch_pdl(k_ctrl_backward_multi, dim3(n), dim3(1024), 0, s, cur, cs);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t ctrl_scatter_x(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s) {
  if (!ctrl_reads_state(c) || sp.N == 0) return cudaSuccess;
  if (sp.dim == 2)
    launch_pdl(k_ctrl_scatter_x<2>, dim3((sp.N + 255) / 256), dim3(256), 0, s, dsp, c);
  else
    launch_pdl(k_ctrl_scatter_x<3>, dim3((sp.N + 255) / 256), dim3(256), 0, s, dsp, c);
  count_launches(1);
  return cudaGetLastError();
}

// Controller backward for one reverse step: group sums of (K), parameter adjoint, and (MLP) the
// centroid adjoint added to dL/dx of state n.  Rewinds the scene's step counter.
cudaError_t ctrl_step_backward(const ScenePar& sp, const ScenePar* dsp, const CtrlPar& c, cudaStream_t s) {
  if (ctrl_reads_state(c))
    launch_pdl(k_ctrl_backward<true>, dim3(1), dim3(1024), 0, s, dsp, c);
  else
    launch_pdl(k_ctrl_backward<false>, dim3(1), dim3(1024), 0, s, dsp, c);
  if (ctrl_reads_state(c) && sp.N > 0) {
    if (sp.dim == 2)
      launch_pdl(k_ctrl_scatter_x<2>, dim3((sp.N + 255) / 256), dim3(256), 0, s, dsp, c);
    else
      launch_pdl(k_ctrl_scatter_x<3>, dim3((sp.N + 255) / 256), dim3(256), 0, s, dsp, c);
  }
  count_launches(1 + ((ctrl_reads_state(c) && sp.N > 0) ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace gbmpm
