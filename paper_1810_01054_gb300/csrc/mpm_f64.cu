// Double-precision plain form of the differentiable MLS-MPM step (mpm64_* in include/mpm.h).
//
// Section VI measures gradient accuracy on float64 runs (case B: colliding elastic bodies, the
// adjoint against central finite differences).  This file is that precision on the GPU: the step
// of Section III (Eqs. 3-10) and its reverse pass (Supplement S2-S5, (A)-(L)) in FP64, using the
// scalar-generic math of mpm_device.cuh (stencil, neo-Hookean stress and Hessian product, MLS G,
// per-wall boundary projection and its adjoint) instantiated for double.
//
// Form: one thread per particle, scatter by global double atomics into a zeroed dense grid, one
// thread per node for the grid update, gathers per particle.  The order of the atomic sums is not
// fixed, so runs agree to rounding (not bit for bit); the tile path stays the deterministic one.
// A rollout keeps every state on the device (the accuracy study's scenes are small), so the
// reverse pass recomputes nothing.
//
// Layout: a state is S = 2 dim + 2 dim^2 component planes of N doubles, component c of particle p
// at [c * N + p], components in the record order x, F, v, C (row-major matrices); the grid is
// [nodes][4] doubles, (p or v*, m) in the forward sums and (vbar or pbar, mbar) in the reverse.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"
#include "mpm_scene.h"

namespace gbmpm {
namespace {

constexpr int F64_THREADS = 256;

// Everything one FP64 launch reads: scene constants and the buffers of the step being run.
struct Par64 {
  int N, G;
  int n[3];
  double dx, inv_dx, dt, mass, kG, Dinv;
  MaterialT<double> mat;
  double gravity[3];
  BCParT<double> bc;
  const int32_t* group;    // [N], -1 = unactuated
  const double* act_dir;   // [G][dim]
  const double* act;       // [G] actuation of this step, nullptr = none
  const double* st;        // state n
  double* st_out;          // state n + 1 (forward)
  const double* adj_in;    // adjoint of state n + 1 (reverse)
  double* adj_out;         // adjoint of state n (reverse)
  double* grid;            // [nodes][4]
  double* grid_b;          // [nodes][4]
  double* g_act;           // [G] dL/da of this step (reverse), nullptr = not wanted
  int* status;
};

template <int D>
__device__ __forceinline__ void load64(const double* __restrict__ st, int N, int p, Part<D, double>& q) {
  int c = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) q.x[a] = st[size_t(c++) * N + p];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) q.F[a][b] = st[size_t(c++) * N + p];
#pragma unroll
  for (int a = 0; a < D; ++a) q.v[a] = st[size_t(c++) * N + p];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) q.C[a][b] = st[size_t(c++) * N + p];
}

template <int D>
__device__ __forceinline__ void store64(double* __restrict__ st, int N, int p, const Part<D, double>& q) {
  int c = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) st[size_t(c++) * N + p] = q.x[a];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) st[size_t(c++) * N + p] = q.F[a][b];
#pragma unroll
  for (int a = 0; a < D; ++a) st[size_t(c++) * N + p] = q.v[a];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) st[size_t(c++) * N + p] = q.C[a][b];
}

template <int D>
__device__ __forceinline__ int node_lin(const int* nd, const int* n) {
  return D == 2 ? nd[0] * n[1] + nd[1] : (nd[0] * n[1] + nd[1]) * n[2] + nd[D == 3 ? 2 : 0];
}

// Group of particle p (-1: none) and its actuation stress diagonal sigma_a = a_g dir_g.
template <int D>
__device__ __forceinline__ int actuation64(const Par64& p, int id, double* sig) {
  int g = p.group ? p.group[id] : -1;
  if (g >= p.G) g = -1;
#pragma unroll
  for (int a = 0; a < D; ++a) sig[a] = (g >= 0 && p.act) ? p.act[g] * p.act_dir[g * D + a] : 0.0;
  return g;
}

// Stress P (elastic + F sigma_a), F^{-T}, J and the MLS momentum matrix G of Eq. 4.
template <int D>
__device__ __forceinline__ double stress_G64(const Par64& p, const Part<D, double>& q, const double* sig,
                                             double (&P)[D][D], double (&A)[D][D], double (&G)[D][D]) {
  const double J = stress<D>(q.F, p.mat, sig, P, A);
  mls_G<D>(P, q.F, q.C, p.kG, p.mass, G);
  return J;
}

// Visits the stencil nodes of a particle: f(node linear index, N, dN/dx_p, d = x_i - x_p).
template <int D, class Fn>
__device__ __forceinline__ void for_stencil(const Sten<D, double>& s, const int* n, double dx, Fn fn) {
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz) {
        const int k[3] = {kx, ky, kz};
        int nd[D];
        double N = 1.0, dN[D], d[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          nd[a] = s.base[a] + k[a];
          N *= s.w[a][k[a]];
          d[a] = (double(k[a]) - s.f[a]) * dx;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double t = 1.0;
#pragma unroll
          for (int b = 0; b < D; ++b) t *= (a == b) ? s.dw[b][k[b]] : s.w[b][k[b]];
          dN[a] = t;
        }
        fn(node_lin<D>(nd, n), N, dN, d);
      }
}

// P2G (Eqs. 3-5): m_i += N m_p, p_i += N (m_p v_p + G_p d).  With ADJ also the reverse step's
// (A)-(C) scatter of state n+1's adjoint: vbar_i += N (vbar_p + (4/dx^2) Cbar_p d) with
// vbar_p = vbar' + dt xbar' (A) and Cbar_p = Cbar' + dt Fbar' F^T (B).
template <int D, bool ADJ>
__global__ void __launch_bounds__(F64_THREADS) k64_p2g(Par64 p) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= p.N) return;
  Part<D, double> q;
  load64<D>(p.st, p.N, id, q);
  Sten<D, double> stn;
  if (!make_stencil<D>(q.x, p.inv_dx, p.n, stn)) {
    set_status(p.status, ST_DOMAIN);
    return;
  }
  double sig[D], P[D][D], A[D][D], G[D][D];
  actuation64<D>(p, id, sig);
  const double J = stress_G64<D>(p, q, sig, P, A, G);
  if (!(J > 0.0)) set_status(p.status, ST_INVERTED);
  double vb[D] = {}, Cb[D][D] = {};
  if constexpr (ADJ) {
    Part<D, double> g1;
    load64<D>(p.adj_in, p.N, id, g1);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vb[a] = g1.v[a] + p.dt * g1.x[a];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += g1.F[a][k] * q.F[c][k];
        Cb[a][c] = g1.C[a][c] + p.dt * s;
      }
    }
  }
  for_stencil<D>(stn, p.n, p.dx, [&](int nl, double N, const double*, const double* d) {
    double* gp = p.grid + size_t(nl) * 4;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double s = p.mass * q.v[a];
#pragma unroll
      for (int c = 0; c < D; ++c) s += G[a][c] * d[c];
      atomicAdd(gp + a, N * s);
    }
    atomicAdd(gp + 3, N * p.mass);
    if constexpr (ADJ) {
      double* gb = p.grid_b + size_t(nl) * 4;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double s = vb[a];
#pragma unroll
        for (int c = 0; c < D; ++c) s += p.Dinv * Cb[a][c] * d[c];
        atomicAdd(gb + a, N * s);
      }
    }
  });
}

// Grid update: v* = BC(p / m + dt g) (Section III, Supplement S5).  With ADJ the reverse of it:
// (L) through the boundary, then (D) pbar = vbar / m and (E) mbar = -v . vbar / m.
template <int D, bool ADJ>
__global__ void __launch_bounds__(F64_THREADS) k64_grid(Par64 p, int n_nodes) {
  const int nl = blockIdx.x * blockDim.x + threadIdx.x;
  if (nl >= n_nodes) return;
  int node[D];
  {
    int r = nl;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      node[a] = r % p.n[a];
      r /= p.n[a];
    }
  }
  double* gp = p.grid + size_t(nl) * 4;
  const double m = gp[3];
  double vraw[D], v[D];
  const double rm = m > 0.0 ? 1.0 / m : 0.0;  // one division per node (FP64 divides are long chains)
  if (m > 0.0) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vraw[a] = gp[a] * rm;
      v[a] = vraw[a] + p.dt * p.gravity[a];
    }
    bc_apply<D>(node, p.n, p.bc, v);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = vraw[a] = 0.0;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) gp[a] = v[a];
  if constexpr (ADJ) {
    double* gb = p.grid_b + size_t(nl) * 4;
    double g[D], pb[D], mb = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) g[a] = gb[a];
    if (m > 0.0) {
      double vg[D];
#pragma unroll
      for (int a = 0; a < D; ++a) vg[a] = vraw[a] + p.dt * p.gravity[a];
      bc_adjoint<D>(node, p.n, p.bc, vg, g);
      double dot = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        pb[a] = g[a] * rm;
        dot += vraw[a] * g[a];
      }
      mb = -dot * rm;
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) pb[a] = 0.0;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) gb[a] = pb[a];
    gb[3] = mb;
  }
}

// G2P (Eqs. 7-10): v = sum N v*, C = (4/dx^2) sum N v* d^T, F <- (I + dt C) F, x <- x + dt v.
template <int D>
__global__ void __launch_bounds__(F64_THREADS) k64_g2p(Par64 p) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= p.N) return;
  Part<D, double> q;
  load64<D>(p.st, p.N, id, q);
  Sten<D, double> stn;
  if (!make_stencil<D>(q.x, p.inv_dx, p.n, stn)) {  // status already set by P2G: carry the particle over
    store64<D>(p.st_out, p.N, id, q);
    return;
  }
  double vn[D] = {}, Cn[D][D] = {};
  for_stencil<D>(stn, p.n, p.dx, [&](int nl, double N, const double*, const double* d) {
    const double* gp = p.grid + size_t(nl) * 4;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double Nv = N * gp[a];
      vn[a] += Nv;
#pragma unroll
      for (int c = 0; c < D; ++c) Cn[a][c] += Nv * d[c];
    }
  });
  Part<D, double> o;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) o.C[a][c] = p.Dinv * Cn[a][c];
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double s = q.F[a][c];
#pragma unroll
      for (int k = 0; k < D; ++k) s += p.dt * o.C[a][k] * q.F[k][c];
      o.F[a][c] = s;
    }
    o.v[a] = vn[a];
    o.x[a] = q.x[a] + p.dt * vn[a];
  }
  store64<D>(p.st_out, p.N, id, o);
}

// Reverse G2P per particle, Supplement S4 (F)-(K) in their direct form:
//   (F) vbar = m sum N pbar_i                (I) Cbar = m sum N pbar_i d^T
//   (G) Pbar = kG Gbar F, Gbar = sum N pbar_i d^T, kG = -(4/dx^2) dt V0
//   (H) Fbar = (I + dt C^{n+1})^T Fbar' + d2Psi[Pbar] + Pbar sigma_a + kG Gbar^T P
//   (J) xbar = xbar' + sum dN s_i - (4/dx^2) Cbar_p^T sum N v*_i - G^T sum N pbar_i,
//       s_i = vbar_p . v*_i + (4/dx^2) v*_i . Cbar_p d + pbar_i . (m v + G d) + m mbar_i
//   (K) dL/da_g += dir_g . diag(F^T Pbar)
// with vbar_p, Cbar_p the (A), (B) totals of state n+1's adjoint.  Block-level group sums of (K)
// go to g_act with one atomic per group and block.
template <int D>
__global__ void __launch_bounds__(F64_THREADS) k64_adjoint(Par64 p) {
  __shared__ double gsum[MAX_GROUPS];
  const bool want_act = p.g_act != nullptr && p.G > 0;
  if (want_act) {
    for (int g = threadIdx.x; g < p.G; g += blockDim.x) gsum[g] = 0.0;
    __syncthreads();
  }
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  Sten<D, double> stn;
  Part<D, double> q;
  const bool live = id < p.N && (load64<D>(p.st, p.N, id, q), make_stencil<D>(q.x, p.inv_dx, p.n, stn));
  if (live) {
    Part<D, double> g1, g0;
    load64<D>(p.adj_in, p.N, id, g1);
    double sig[D], P[D][D], A[D][D], G[D][D];
    const int grp = actuation64<D>(p, id, sig);
    const double J = stress_G64<D>(p, q, sig, P, A, G);
    double vb[D], Cb[D][D], mv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vb[a] = g1.v[a] + p.dt * g1.x[a];
      mv[a] = p.mass * q.v[a];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += g1.F[a][k] * q.F[c][k];
        Cb[a][c] = g1.C[a][c] + p.dt * s;
      }
    }
    double gxs[D] = {}, sv[D] = {}, spb[D] = {}, Cn[D][D] = {}, Gb[D][D] = {};
    for_stencil<D>(stn, p.n, p.dx, [&](int nl, double N, const double* dN, const double* d) {
      const double* gv = p.grid + size_t(nl) * 4;
      const double* gb = p.grid_b + size_t(nl) * 4;
      double si = p.mass * gb[3];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double cd = 0.0, gd = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          cd += Cb[a][c] * d[c];
          gd += G[a][c] * d[c];
        }
        si += gv[a] * (vb[a] + p.Dinv * cd) + gb[a] * (mv[a] + gd);
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        gxs[a] += dN[a] * si;
        sv[a] += N * gv[a];
        spb[a] += N * gb[a];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          Cn[a][c] += N * gv[a] * d[c];
          Gb[a][c] += N * gb[a] * d[c];
        }
      }
    });
    double Pb[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double t = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) t += p.Dinv * Cb[c][a] * sv[c] + G[c][a] * spb[c];
      g0.x[a] = g1.x[a] + gxs[a] - t;   // (J)
      g0.v[a] = p.mass * spb[a];         // (F)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        Cn[a][c] *= p.Dinv;
        g0.C[a][c] = p.mass * Gb[a][c];  // (I)
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += Gb[a][k] * q.F[k][c];
        Pb[a][c] = p.kG * s;             // (G)
      }
    }
    double H[D][D];
    nh_hessian_apply<D>(A, J, p.mat, Pb, H);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double s = g1.F[a][c], t = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          s += p.dt * Cn[k][a] * g1.F[k][c];
          t += Gb[k][a] * P[k][c];
        }
        g0.F[a][c] = s + H[a][c] + Pb[a][c] * sig[c] + p.kG * t;  // (H)
      }
    store64<D>(p.adj_out, p.N, id, g0);
    if (want_act && grp >= 0) {  // (K)
      double contrib = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) s += q.F[k][a] * Pb[k][a];
        contrib += p.act_dir[grp * D + a] * s;
      }
      atomicAdd(&gsum[grp], contrib);
    }
  }
  if (want_act) {
    __syncthreads();
    for (int g = threadIdx.x; g < p.G; g += blockDim.x)
      if (gsum[g] != 0.0) atomicAdd(p.g_act + g, gsum[g]);
  }
}

// Launch shape of a kernel over n items.  FP64 arithmetic issues at a small fraction of the FP32
// rate on this GPU, so a kernel is bound by the FP64 pipes of the SMs it occupies: blocks shrink
// (down to one warp) until the grid covers every SM, and only large launches use full blocks.
struct Shape {
  int blocks, threads;
};
Shape shape_for(int n, int sms) {
  int t = (n + sms - 1) / sms;
  t = std::min(F64_THREADS, std::max(32, (t + 31) / 32 * 32));
  return {std::max(1, (n + t - 1) / t), t};
}

template <int D>
cudaError_t launch_step64(const Par64& p, int n_nodes, mpm_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.grid, 0, sizeof(double) * 4 * size_t(n_nodes), s);
  if (e != cudaSuccess) return e;
  if (p.N > 0) {
    ProfScope ps(c, s, MPM_K_F64_P2G);
    const Shape sh = shape_for(p.N, c->sm_count);
    k64_p2g<D, false><<<sh.blocks, sh.threads, 0, s>>>(p);
  }
  {
    ProfScope ps(c, s, MPM_K_F64_GRID);
    const Shape sh = shape_for(n_nodes, c->sm_count);
    k64_grid<D, false><<<sh.blocks, sh.threads, 0, s>>>(p, n_nodes);
  }
  if (p.N > 0) {
    ProfScope ps(c, s, MPM_K_F64_G2P);
    const Shape sh = shape_for(p.N, c->sm_count);
    k64_g2p<D><<<sh.blocks, sh.threads, 0, s>>>(p);
  }
  count_launches(p.N > 0 ? 3 : 1);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_reverse64(const Par64& p, int n_nodes, mpm_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.grid, 0, sizeof(double) * 4 * size_t(n_nodes), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.grid_b, 0, sizeof(double) * 4 * size_t(n_nodes), s);
  if (e != cudaSuccess) return e;
  if (p.N > 0) {
    ProfScope ps(c, s, MPM_K_F64_P2G_ADJ);
    const Shape sh = shape_for(p.N, c->sm_count);
    k64_p2g<D, true><<<sh.blocks, sh.threads, 0, s>>>(p);
  }
  {
    ProfScope ps(c, s, MPM_K_F64_GRID);
    const Shape sh = shape_for(n_nodes, c->sm_count);
    k64_grid<D, true><<<sh.blocks, sh.threads, 0, s>>>(p, n_nodes);
  }
  if (p.N > 0) {
    ProfScope ps(c, s, MPM_K_F64_ADJ);
    const Shape sh = shape_for(p.N, c->sm_count);
    k64_adjoint<D><<<sh.blocks, sh.threads, 0, s>>>(p);
  }
  count_launches(p.N > 0 ? 3 : 1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace gbmpm

using gbmpm::Par64;

struct mpm_scene64 {
  mpm_ctx* ctx = nullptr;
  int dim = 0, N = 0, G = 0, n_nodes = 0, S = 0;
  Par64 hp{};                  // scene constants; buffer pointers are filled per launch
  double* init = nullptr;      // [S][N] initial state of the next rollout
  double* adj[2] = {nullptr, nullptr};
  double* act = nullptr;       // [L][G] actuation table
  double* g_act = nullptr;     // [L][G] dL/dU of the last reverse pass
  int L = 0;
  double* hist = nullptr;      // [T + 1][S][N] states of the last rollout
  int T = -1;                  // steps of the last rollout (-1: none)
  size_t hist_cap = 0;         // states hist can hold
  std::vector<void*> allocs;
  // whole rollouts and reverse passes replayed as CUDA graphs (one launch instead of ~4 per step);
  // captured for a rollout length T and dropped when a buffer they name is reallocated
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int T = -1;
    long long kernels = 0;
  } gfwd, grev;
};

namespace {

mpm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MPM_OK;
  return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
}

#define CK64(expr)                                    \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_status(e_);    \
  } while (0)

template <class T>
mpm_status alloc64(mpm_scene64* s, T** p, size_t count) {
  void* q = nullptr;
  CK64(cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16)));
  s->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return MPM_OK;
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// Writes x, v, C, F (host, particle-major; NULL v, C = 0, NULL F = I) as component planes.
mpm_status upload_state(mpm_scene64* s, double* dst, const double* x, const double* v, const double* C,
                        const double* F) {
  const int D = s->dim, N = s->N;
  if (N == 0) return MPM_OK;
  if (!x) return MPM_ERR_ARG;
  std::vector<double> h(size_t(s->S) * N);
  for (int p = 0; p < N; ++p) {
    int c = 0;
    for (int a = 0; a < D; ++a) h[size_t(c++) * N + p] = x[size_t(p) * D + a];
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) h[size_t(c++) * N + p] = F ? F[(size_t(p) * D + a) * D + b] : (a == b ? 1.0 : 0.0);
    for (int a = 0; a < D; ++a) h[size_t(c++) * N + p] = v ? v[size_t(p) * D + a] : 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) h[size_t(c++) * N + p] = C ? C[(size_t(p) * D + a) * D + b] : 0.0;
  }
  if (!finite_all(h.data(), h.size())) return MPM_ERR_ARG;
  CK64(cudaMemcpyAsync(dst, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s->ctx->stream));
  CK64(cudaStreamSynchronize(s->ctx->stream));
  return MPM_OK;
}

// Reads component planes back as x, v, C, F (host, particle-major; NULL skips one).
mpm_status download_state(mpm_scene64* s, const double* src, double* x, double* v, double* C, double* F) {
  const int D = s->dim, N = s->N;
  if (N == 0) return MPM_OK;
  std::vector<double> h(size_t(s->S) * N);
  CK64(cudaMemcpyAsync(h.data(), src, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->ctx->stream));
  CK64(cudaStreamSynchronize(s->ctx->stream));
  for (int p = 0; p < N; ++p) {
    int c = 0;
    for (int a = 0; a < D; ++a, ++c)
      if (x) x[size_t(p) * D + a] = h[size_t(c) * N + p];
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b, ++c)
        if (F) F[(size_t(p) * D + a) * D + b] = h[size_t(c) * N + p];
    for (int a = 0; a < D; ++a, ++c)
      if (v) v[size_t(p) * D + a] = h[size_t(c) * N + p];
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b, ++c)
        if (C) C[(size_t(p) * D + a) * D + b] = h[size_t(c) * N + p];
  }
  return MPM_OK;
}

mpm_status read_status64(mpm_scene64* s) {
  int v = 0;
  CK64(cudaStreamSynchronize(s->ctx->stream));
  CK64(cudaMemcpy(&v, s->hp.status, sizeof(int), cudaMemcpyDeviceToHost));
  return mpm_status(v);
}

const double* step_act(const mpm_scene64* s, int t) {
  return (s->G > 0 && t < s->L) ? s->act + size_t(t) * s->G : nullptr;
}

void drop_graphs(mpm_scene64* s) {
  for (mpm_scene64::Graph* g : {&s->gfwd, &s->grev}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    *g = mpm_scene64::Graph();
  }
}

// The T steps of a rollout from the initial state (status cleared first).
mpm_status enqueue_rollout(mpm_scene64* s, int T, cudaStream_t str) {
  const size_t stride = size_t(s->S) * std::max(1, s->N);
  CK64(cudaMemsetAsync(s->hp.status, 0, sizeof(int), str));
  CK64(cudaMemcpyAsync(s->hist, s->init, sizeof(double) * stride, cudaMemcpyDeviceToDevice, str));
  for (int t = 0; t < T; ++t) {
    Par64 p = s->hp;
    p.st = s->hist + size_t(t) * stride;
    p.st_out = s->hist + size_t(t + 1) * stride;
    p.act = step_act(s, t);
    CK64(s->dim == 2 ? gbmpm::launch_step64<2>(p, s->n_nodes, s->ctx, str)
                     : gbmpm::launch_step64<3>(p, s->n_nodes, s->ctx, str));
  }
  return MPM_OK;
}

// The reverse steps T-1 .. 0 (adjoint of state T in adj[0]; that of state 0 ends in adj[T & 1]).
mpm_status enqueue_reverse(mpm_scene64* s, int T, cudaStream_t str) {
  const size_t stride = size_t(s->S) * std::max(1, s->N);
  if (size_t(s->L) * s->G > 0) CK64(cudaMemsetAsync(s->g_act, 0, sizeof(double) * size_t(s->L) * s->G, str));
  int cur = 0;
  for (int t = T - 1; t >= 0; --t) {
    Par64 p = s->hp;
    p.st = s->hist + size_t(t) * stride;
    p.adj_in = s->adj[cur];
    p.adj_out = s->adj[cur ^ 1];
    p.act = step_act(s, t);
    p.g_act = p.act ? s->g_act + size_t(t) * s->G : nullptr;
    CK64(s->dim == 2 ? gbmpm::launch_reverse64<2>(p, s->n_nodes, s->ctx, str)
                     : gbmpm::launch_reverse64<3>(p, s->n_nodes, s->ctx, str));
    cur ^= 1;
  }
  return MPM_OK;
}

// Runs the rollout (reverse = false) or reverse pass of length T on the context stream: directly
// while launch timing is on, else as a graph, captured on first use for this T.
mpm_status run64(mpm_scene64* s, bool reverse, int T) {
  mpm_ctx* c = s->ctx;
  if (c->prof_mask) return reverse ? enqueue_reverse(s, T, c->stream) : enqueue_rollout(s, T, c->stream);
  mpm_scene64::Graph& g = reverse ? s->grev : s->gfwd;
  if (!g.exec || g.T != T) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = mpm_scene64::Graph();
    long long tally = 0;
    CK64(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
    gbmpm::capture_tally(&tally);
    mpm_status st = reverse ? enqueue_reverse(s, T, c->capture) : enqueue_rollout(s, T, c->capture);
    gbmpm::capture_tally(nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture, &graph);
    if (st != MPM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    CK64(e);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK64(e);
    g.T = T;
    g.kernels = tally;
  }
  CK64(cudaGraphLaunch(g.exec, c->stream));
  gbmpm::count_launches(int(g.kernels));
  return MPM_OK;
}

}  // namespace

extern "C" {

mpm_status mpm64_destroy(mpm_scene64* s) {
  if (!s) return MPM_ERR_ARG;
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->ctx->stream);
  drop_graphs(s);
  for (void* p : s->allocs) cudaFree(p);
  if (s->hist) cudaFree(s->hist);
  s->ctx->live.fetch_sub(1);
  delete s;
  return MPM_OK;
}

mpm_status mpm64_create(mpm_ctx* c, const mpm_scene64_desc* d, mpm_scene64** out) {
  if (!c || !d || !out) return MPM_ERR_ARG;
  *out = nullptr;
  const int dim = d->dim;
  if (dim != 2 && dim != 3) return MPM_ERR_ARG;
  for (int a = 0; a < dim; ++a)
    if (d->n_grid[a] < 5) return MPM_ERR_ARG;
  if (!(d->dx > 0) || !(d->dt > 0) || !(d->E > 0) || !(d->nu > -1 && d->nu < 0.5)) return MPM_ERR_ARG;
  if (!(d->p_mass > 0) || !(d->p_vol > 0) || d->bc_width < 0) return MPM_ERR_ARG;
  if (!std::isfinite(d->dx) || !std::isfinite(d->dt) || !std::isfinite(d->E) || !std::isfinite(d->p_mass) ||
      !std::isfinite(d->p_vol))
    return MPM_ERR_ARG;
  for (int w = 0; w < 2 * dim; ++w) {
    if (d->wall_kind[w] != MPM_BC_STICKY && d->wall_kind[w] != MPM_BC_SLIP && d->wall_kind[w] != MPM_BC_OPEN)
      return MPM_ERR_ARG;
    if (!(d->wall_c[w] >= 0) || !std::isfinite(d->wall_c[w])) return MPM_ERR_ARG;
  }
  for (int a = 0; a < dim; ++a)
    if (!std::isfinite(d->gravity[a])) return MPM_ERR_ARG;
  if (d->n_particles < 0 || d->n_particles >= (1 << 26)) return MPM_ERR_ARG;
  if (d->n_particles > 0 && !d->x0) return MPM_ERR_ARG;
  if (d->n_groups < 0 || d->n_groups > gbmpm::MAX_GROUPS) return MPM_ERR_ARG;
  if (d->n_groups > 0 && (!d->act_dir || !finite_all(d->act_dir, size_t(d->n_groups) * dim))) return MPM_ERR_ARG;
  if (d->group)
    for (int p = 0; p < d->n_particles; ++p)
      if (d->group[p] < -1 || d->group[p] >= d->n_groups) return MPM_ERR_ARG;
  if (d->n_act_steps < 0 || (d->n_act_steps > 0 && d->n_groups > 0 && !d->act)) return MPM_ERR_ARG;
  // explicit-integration limit dt <= C dx sqrt(rho / E) with C = 1 (Section VI)
  if (d->dt > d->dx * std::sqrt((d->p_mass / d->p_vol) / d->E) * (1.0 + 1e-12)) return MPM_ERR_ARG;

  CK64(cudaSetDevice(c->device));
  mpm_scene64* s = new (std::nothrow) mpm_scene64();
  if (!s) return MPM_ERR_OOM;
  s->ctx = c;
  c->live.fetch_add(1);
  s->dim = dim;
  s->N = d->n_particles;
  s->G = d->n_groups;
  s->S = 2 * dim + 2 * dim * dim;
  s->n_nodes = 1;
  for (int a = 0; a < dim; ++a) s->n_nodes *= d->n_grid[a];
  Par64& p = s->hp;
  std::memset(&p, 0, sizeof(p));
  p.N = s->N;
  p.G = s->G;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = a < dim ? d->n_grid[a] : 1;
    p.gravity[a] = a < dim ? d->gravity[a] : 0.0;
  }
  p.dx = d->dx;
  p.inv_dx = 1.0 / d->dx;
  p.dt = d->dt;
  p.mass = d->p_mass;
  p.Dinv = 4.0 * p.inv_dx * p.inv_dx;
  p.kG = -p.Dinv * d->dt * d->p_vol;
  // Lame parameters by the textbook map from (E, nu)
  p.mat.mu = d->E / (2.0 * (1.0 + d->nu));
  p.mat.la = d->E * d->nu / ((1.0 + d->nu) * (1.0 - 2.0 * d->nu));
  p.bc.width = d->bc_width;
  for (int w = 0; w < 6; ++w) {
    p.bc.kind[w] = w < 2 * dim ? d->wall_kind[w] : MPM_BC_OPEN;
    p.bc.c[w] = w < 2 * dim ? d->wall_c[w] : 0.0;
  }
  auto fail = [&](mpm_status st) {
    mpm64_destroy(s);
    return st;
  };
  mpm_status st = MPM_OK;
  const size_t SN = size_t(s->S) * std::max(1, s->N);
  int32_t* group = nullptr;
  double* act_dir = nullptr;
  if ((st = alloc64(s, &s->init, SN)) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &s->adj[0], SN)) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &s->adj[1], SN)) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &p.grid, size_t(4) * s->n_nodes)) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &p.grid_b, size_t(4) * s->n_nodes)) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &group, std::max(1, s->N))) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &act_dir, std::max(1, s->G * dim))) != MPM_OK) return fail(st);
  if ((st = alloc64(s, &p.status, 1)) != MPM_OK) return fail(st);
  p.group = group;
  p.act_dir = act_dir;
  cudaStream_t str = c->stream;
  if (s->N > 0) {
    std::vector<int32_t> gh(s->N, -1);
    if (d->group) std::copy(d->group, d->group + s->N, gh.begin());
    if (cudaMemcpyAsync(group, gh.data(), sizeof(int32_t) * s->N, cudaMemcpyHostToDevice, str) != cudaSuccess ||
        cudaStreamSynchronize(str) != cudaSuccess)
      return fail(MPM_ERR_CUDA);
  }
  if (s->G > 0 && (cudaMemcpyAsync(act_dir, d->act_dir, sizeof(double) * s->G * dim, cudaMemcpyHostToDevice, str) !=
                       cudaSuccess ||
                   cudaStreamSynchronize(str) != cudaSuccess))
    return fail(MPM_ERR_CUDA);
  if (cudaMemsetAsync(p.status, 0, sizeof(int), str) != cudaSuccess) return fail(MPM_ERR_CUDA);
  if ((st = upload_state(s, s->init, d->x0, d->v0, d->C0, d->F0)) != MPM_OK) return fail(st);
  if ((st = mpm64_set_actuation(s, d->act, d->n_act_steps)) != MPM_OK) return fail(st);
  *out = s;
  return MPM_OK;
}

mpm_status mpm64_set_state(mpm_scene64* s, const double* x, const double* v, const double* C, const double* F) {
  if (!s) return MPM_ERR_ARG;
  CK64(cudaSetDevice(s->ctx->device));
  mpm_status st = upload_state(s, s->init, x, v, C, F);
  if (st != MPM_OK) return st;
  s->T = -1;  // the stored rollout no longer starts from this state
  return MPM_OK;
}

mpm_status mpm64_set_actuation(mpm_scene64* s, const double* U, int L) {
  if (!s || L < 0 || (L > 0 && s->G > 0 && !U)) return MPM_ERR_ARG;
  const size_t n = size_t(L) * s->G;
  if (n > 0 && !finite_all(U, n)) return MPM_ERR_ARG;
  CK64(cudaSetDevice(s->ctx->device));
  CK64(cudaStreamSynchronize(s->ctx->stream));
  drop_graphs(s);  // they name the old table buffers
  for (double* q : {s->act, s->g_act}) {
    if (!q) continue;
    s->allocs.erase(std::find(s->allocs.begin(), s->allocs.end(), static_cast<void*>(q)));
    cudaFree(q);
  }
  s->act = s->g_act = nullptr;
  s->L = L;
  mpm_status st = alloc64(s, &s->act, std::max<size_t>(1, n));
  if (st == MPM_OK) st = alloc64(s, &s->g_act, std::max<size_t>(1, n));
  if (st != MPM_OK) {
    s->L = 0;
    return st;
  }
  if (n > 0) CK64(cudaMemcpyAsync(s->act, U, sizeof(double) * n, cudaMemcpyHostToDevice, s->ctx->stream));
  CK64(cudaStreamSynchronize(s->ctx->stream));
  s->T = -1;
  return MPM_OK;
}

mpm_status mpm64_rollout(mpm_scene64* s, int T) {
  if (!s || T < 0) return MPM_ERR_ARG;
  CK64(cudaSetDevice(s->ctx->device));
  const size_t state = sizeof(double) * size_t(s->S) * std::max(1, s->N);
  if (size_t(T) + 1 > s->hist_cap) {
    CK64(cudaStreamSynchronize(s->ctx->stream));
    drop_graphs(s);  // they name the old history buffer
    if (s->hist) cudaFree(s->hist);
    s->hist = nullptr;
    s->hist_cap = 0;
    s->T = -1;
    void* q = nullptr;
    CK64(cudaMalloc(&q, state * (size_t(T) + 1)));
    s->hist = static_cast<double*>(q);
    s->hist_cap = size_t(T) + 1;
  }
  mpm_status st = run64(s, false, T);
  if (st != MPM_OK) return st;
  s->T = T;
  return MPM_OK;
}

mpm_status mpm64_get_state(mpm_scene64* s, int step, double* x, double* v, double* C, double* F) {
  if (!s) return MPM_ERR_ARG;
  if (s->T < 0) return MPM_ERR_STATE;
  if (step == -1) step = s->T;
  if (step < 0 || step > s->T) return MPM_ERR_ARG;
  CK64(cudaSetDevice(s->ctx->device));
  mpm_status st = read_status64(s);
  if (st != MPM_OK) return st;
  return download_state(s, s->hist + size_t(step) * s->S * std::max(1, s->N), x, v, C, F);
}

mpm_status mpm64_backward(mpm_scene64* s, const double* gx_T, const double* gv_T, const double* gC_T,
                          const double* gF_T, double* gx0, double* gv0, double* gC0, double* gF0, double* g_act) {
  if (!s) return MPM_ERR_ARG;
  if (s->T < 0) return MPM_ERR_STATE;
  CK64(cudaSetDevice(s->ctx->device));
  mpm_status st = read_status64(s);
  if (st != MPM_OK) return st;
  const int D = s->dim, N = s->N;
  // seeds: NULL = 0 (upload_state takes NULL F as I, so F's seed is passed through zeros)
  std::vector<double> zx(size_t(N) * D, 0.0), zF(size_t(N) * D * D, 0.0);
  st = upload_state(s, s->adj[0], gx_T ? gx_T : zx.data(), gv_T, gC_T, gF_T ? gF_T : zF.data());
  if (st != MPM_OK) return st;
  cudaStream_t str = s->ctx->stream;
  st = run64(s, true, s->T);
  if (st != MPM_OK) return st;
  st = read_status64(s);
  if (st != MPM_OK) return st;
  st = download_state(s, s->adj[s->T & 1], gx0, gv0, gC0, gF0);
  if (st != MPM_OK) return st;
  const size_t n = size_t(s->L) * s->G;
  if (g_act && n > 0) {
    CK64(cudaMemcpyAsync(g_act, s->g_act, sizeof(double) * n, cudaMemcpyDeviceToHost, str));
    CK64(cudaStreamSynchronize(str));
  }
  return MPM_OK;
}

mpm_status mpm64_info(const mpm_scene64* s, int* n_particles, int* n_groups, int* n_act_steps, int* rollout_steps) {
  if (!s) return MPM_ERR_ARG;
  if (n_particles) *n_particles = s->N;
  if (n_groups) *n_groups = s->G;
  if (n_act_steps) *n_act_steps = s->L;
  if (rollout_steps) *rollout_steps = s->T;
  return MPM_OK;
}

}  // extern "C"
