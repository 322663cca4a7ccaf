// Actuation controllers and their adjoints (Section V-B: a = tanh(W z + b) generating the
// actuation of every group at every step), plus the deterministic per-group reductions they
// need: group centroids of x (controller input) and per-group sums of dL/da (Supplement S4 (K)).
//
// Reductions are two-level with a fixed order at both levels (lanes own groups, warps combine in
// warp order, rows combine in row order), so they are bitwise reproducible.
#include "mpm_internal.h"

namespace gbmpm {

constexpr float kTwoPi = 6.283185307179586f;
constexpr int RED_WARPS = 8;
constexpr int RED_WR = 256;                       // particles per warp
constexpr int RED_ROW = RED_WARPS * RED_WR;       // particles per partial row
constexpr int RED_STRIDE = MAX_GROUPS * 3 + 3;    // floats per row: [64 groups][3] + body[3]

int reduction_rows(int N) { return (N + RED_ROW - 1) / RED_ROW; }

// Group sums of x (dim channels) and the body sum, for the MLP controller's centroids.
template <int CH>
__global__ void __launch_bounds__(256) k_group_rows(const ScenePar* __restrict__ dsp, float* __restrict__ rows,
                                                    int mode) {
  pdl_enter();
  const ScenePar& sp = *dsp;
  __shared__ float wacc[RED_WARPS][MAX_GROUPS][CH];
  __shared__ float wbody[RED_WARPS][CH];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int start = blockIdx.x * RED_ROW + w * RED_WR;
  float lo[CH], hi[CH], body[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) lo[c] = hi[c] = body[c] = 0.0f;
  for (int k = 0; k < RED_WR; k += 32) {
    const int p = start + k + lane;
    int g = -1;
    float val[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) val[c] = 0.0f;
    if (p < sp.N) {
      g = sp.group ? sp.group[p] : -1;
      if (g >= sp.G) g = -1;
      if (mode == 0) {
        const float4 q = sp.planes[p];
        const float xv[3] = {q.x, q.y, q.z};
#pragma unroll
        for (int c = 0; c < CH; ++c) val[c] = xv[c];
      } else if (mode == 2) {  // v: floats D + D*D .. of the state, inside one plane for D = 2, 3
        constexpr int O = CH + CH * CH;
        const float4 q = sp.planes[size_t(O / 4) * sp.npad + p];
        const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int c = 0; c < CH; ++c) val[c] = qv[O % 4 + c];
      } else {
        val[0] = sp.sig_contrib[p];
      }
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) body[c] += val[c];
    for (int j = 0; j < 32; ++j) {
      const int gj = __shfl_sync(0xffffffffu, g, j);
      float vj[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) vj[c] = __shfl_sync(0xffffffffu, val[c], j);
      if (gj >= 0 && (gj & 31) == lane) {
        if (gj >> 5) {
#pragma unroll
          for (int c = 0; c < CH; ++c) hi[c] += vj[c];
        } else {
#pragma unroll
          for (int c = 0; c < CH; ++c) lo[c] += vj[c];
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    wacc[w][lane][c] = lo[c];
    wacc[w][lane + 32][c] = hi[c];
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

// Sum rows in a fixed order into out[g*3+c] (groups) and out[192+c] (body); 1024-thread CTA.
__device__ void reduce_rows(const float* __restrict__ rows, int n_rows, int G, int CH, float* out) {
  __shared__ float part[1024];
  const int O = MAX_GROUPS * 3 + 3;  // outputs, some unused
  const int S = blockDim.x / O;      // splits per output (5 with 1024 threads)
  const int o = threadIdx.x % O, s = threadIdx.x / O;
  float acc = 0.0f;
  const bool used = s < S && ((o < MAX_GROUPS * 3 && (o / 3) < G && (o % 3) < CH) || (o >= MAX_GROUPS * 3 && (o - MAX_GROUPS * 3) < CH));
  if (used)
    for (int r = s; r < n_rows; r += S) acc += rows[size_t(r) * RED_STRIDE + o];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < O) {
    float t = 0.0f;
    for (int k = 0; k < S; ++k) t += part[k * O + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
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
  const int dim = c.dim, Z = G * dim, H = c.hidden;
  reduce_rows(rows, n_rows, G, dim, red);
  if (tid < Z) {
    const int g = tid / dim, a = tid - g * dim;
    const float cg = red[g * 3 + a] * c.inv_count[g];
    const float cb = red[MAX_GROUPS * 3 + a] * c.inv_n;
    z[tid] = cg - cb;
    c.centroid[tid] = cg;
    if (tid < dim) c.centroid[Z + tid] = cb;
  }
  __syncthreads();
  const float* W1 = c.params;
  const float* b1 = W1 + H * Z;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + G * H;
  if (tid < H) {
    float u = b1[tid];
    for (int j = 0; j < Z; ++j) u += W1[tid * Z + j] * z[j];
    h1[tid] = tanhf(u);
  }
  __syncthreads();
  if (tid < H) {
    float u = b2[tid];
    for (int j = 0; j < H; ++j) u += W2[tid * H + j] * h1[j];
    h2[tid] = tanhf(u);
  }
  __syncthreads();
  if (tid < G) {
    float u = b3[tid];
    for (int j = 0; j < H; ++j) u += W3[tid * H + j] * h2[j];
    sp.act[tid] = c.scale * tanhf(u);
  }
}

// Closed-loop controller of step n (type 4, Section V-B): z = [target, c_g, u_g] with c_g, u_g the
// group means of x and v (partial rows of x, then of v), a = scale * tanh(W z + b) -> sp.act; z is
// kept in c.centroid for the reverse step.
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
    c.centroid[tid] = val;
  }
  __syncthreads();
  if (tid < G) {
    const float* W = c.params + dim + size_t(tid) * Z;
    float u = c.params[dim + size_t(G) * Z + tid];
    for (int j = 0; j < Z; ++j) u += W[j] * z[j];
    sp.act[tid] = c.scale * tanhf(u);
  }
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
  if (c.type == 0 || c.type == 1 || c.type == 3) {
    ctrl_open_params(c, n, t, ga);
  } else if (c.type == 4) {  // closed loop: z of this step from the forward replay in c.centroid
    const int dim = c.dim, Z = dim * (1 + 2 * G);
    __shared__ float gu4[MAX_GROUPS];
    if (tid < G) {
      const float* W = c.params + dim + size_t(tid) * Z;
      float u = c.params[dim + size_t(G) * Z + tid];
      for (int j = 0; j < Z; ++j) u += W[j] * c.centroid[j];
      const float th = tanhf(u);
      gu4[tid] = ga[tid] * c.scale * (1.0f - th * th);
      c.gparams[dim + size_t(G) * Z + tid] += gu4[tid];  // b
    }
    __syncthreads();
    for (int i = tid; i < G * Z; i += blockDim.x) c.gparams[dim + i] += gu4[i / Z] * c.centroid[i % Z];  // W
    if (tid < Z) {  // dL/dz: the target's part goes to its parameters, the group means' to gz
      float sacc = 0.0f;
      for (int g = 0; g < G; ++g) sacc += c.params[dim + size_t(g) * Z + tid] * gu4[g];
      if (tid < dim)
        c.gparams[tid] += sacc;
      else
        c.gz[tid - dim] = sacc;  // [c_g part (G*dim)][u_g part (G*dim)]
    }
  } else {
    const int dim = c.dim, Z = G * dim, H = c.hidden;
    const float* W1 = c.params;
    const float* b1 = W1 + H * Z;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + G * H;
    float* gW1 = c.gparams;
    float* gb1 = gW1 + H * Z;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + G * H;
    // forward replay from the centroids of this step (written by k_ctrl_forward)
    if (tid < Z) z[tid] = c.centroid[tid] - c.centroid[Z + tid % dim];
    __syncthreads();
    if (tid < H) {
      float u = b1[tid];
      for (int j = 0; j < Z; ++j) u += W1[tid * Z + j] * z[j];
      h1[tid] = tanhf(u);
    }
    __syncthreads();
    if (tid < H) {
      float u = b2[tid];
      for (int j = 0; j < H; ++j) u += W2[tid * H + j] * h1[j];
      h2[tid] = tanhf(u);
    }
    __syncthreads();
    if (tid < G) {
      float u = b3[tid];
      for (int j = 0; j < H; ++j) u += W3[tid * H + j] * h2[j];
      o3[tid] = tanhf(u);
      gu3[tid] = ga[tid] * c.scale * (1.0f - o3[tid] * o3[tid]);
      gb3[tid] += gu3[tid];
    }
    __syncthreads();
    for (int i = tid; i < G * H; i += blockDim.x) gW3[i] += gu3[i / H] * h2[i % H];
    if (tid < H) {
      float s = 0.0f;
      for (int g = 0; g < G; ++g) s += gu3[g] * W3[g * H + tid];
      gu2[tid] = s * (1.0f - h2[tid] * h2[tid]);
      gb2[tid] += gu2[tid];
    }
    __syncthreads();
    for (int i = tid; i < H * H; i += blockDim.x) gW2[i] += gu2[i / H] * h1[i % H];
    if (tid < H) {
      float s = 0.0f;
      for (int i = 0; i < H; ++i) s += gu2[i] * W2[i * H + tid];
      gu1[tid] = s * (1.0f - h1[tid] * h1[tid]);
      gb1[tid] += gu1[tid];
    }
    __syncthreads();
    for (int i = tid; i < H * Z; i += blockDim.x) gW1[i] += gu1[i / Z] * z[i % Z];
    if (tid < Z) {
      float s = 0.0f;
      for (int i = 0; i < H; ++i) s += gu1[i] * W1[i * Z + tid];
      c.gz[tid] = s;
    }
  }
  __syncthreads();
  if (tid == 0) *step_ctr = n - 1;
}

__global__ void __launch_bounds__(1024) k_ctrl_backward(const ScenePar* __restrict__ dsp, CtrlPar c) {
  pdl_enter();
  ctrl_backward_body(*dsp, c);
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
  ctrl_backward_body(cur[blockIdx.x], cs[blockIdx.x]);
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
      launch_pdl(k_group_rows<2>, dim3(rows), dim3(256), 0, s, dsp, c.partials, 0);
      if (com) launch_pdl(k_group_rows<2>, dim3(rows), dim3(256), 0, s, dsp, vrows, 2);
    } else {
      launch_pdl(k_group_rows<3>, dim3(rows), dim3(256), 0, s, dsp, c.partials, 0);
      if (com) launch_pdl(k_group_rows<3>, dim3(rows), dim3(256), 0, s, dsp, vrows, 2);
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
  launch_pdl(k_ctrl_backward, dim3(1), dim3(1024), 0, s, dsp, c);
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
