// mpm_step_noalloc: one forward MLS-MPM step that allocates nothing.
//
// Some callers cannot call cudaMalloc: a control loop with a hard latency budget (cudaMalloc may
// block and synchronise the device), or a host process whose device memory is owned entirely by
// another allocator, such as a framework's caching pool.  This entry point takes the caller's
// input and output arrays and keeps its only scratch -- the dense node grid of the step -- in a
// file-scope __device__ array of fixed size, which every GPU that loads this library holds until
// the process exits.
//
// The step is the plain form of the library (P2G with float atomics into a dense grid, grid
// update, G2P), so it matches mpm_step on an MPM_IMPL_PLAIN scene up to the order of the atomic
// additions.
#include <cmath>
#include <mutex>

#include "../../include/mpm.h"
#include "mpm_device.cuh"

namespace {

using namespace gbmpm;

// Largest grid the fixed scratch holds: 2^18 nodes (512^2 in 2D, 64^3 in 3D), one float4 each.
constexpr int kNoAllocMaxNodes = 1 << 18;
static __device__ __align__(256) float4 g_noalloc_grid[kNoAllocMaxNodes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float4* g_grid_ptr[kMaxDevices] = {};  // device address of g_noalloc_grid, per device

struct NAPar {
  int n[3];
  float dx, inv_dx, dt;
  float gravity[3];
  Material mat;
  float mass, vol;
  BCPar bc;
  int N, G, n_nodes;
  const float *x, *v, *C, *F;
  const int32_t* group;
  const float* act_dir;
  const float* act;
  float *xo, *vo, *Co, *Fo;
  int* status;
};

template <int D>
__device__ __forceinline__ int node_lin(const int* c, const int* n) {
  int l = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) l = l * n[a] + c[a];
  return l;
}

__global__ void k_na_clear(float4* grid, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) grid[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int D>
__device__ __forceinline__ void na_load(const NAPar& p, int i, float* x, float (&F)[D][D], float* v, float (&C)[D][D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    x[a] = p.x[size_t(i) * D + a];
    v[a] = p.v ? p.v[size_t(i) * D + a] : 0.f;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      F[a][b] = p.F ? p.F[(size_t(i) * D + a) * D + b] : (a == b ? 1.f : 0.f);
      C[a][b] = p.C ? p.C[(size_t(i) * D + a) * D + b] : 0.f;
    }
  }
}

template <int D>
__global__ void k_na_p2g(NAPar p, float4* __restrict__ grid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  float x[D], v[D], F[D][D], C[D][D];
  na_load<D>(p, i, x, F, v, C);
  Sten<D> st;
  if (!make_stencil<D>(x, p.inv_dx, p.n, st)) {
    set_status(p.status, ST_DOMAIN);
    return;
  }
  float sig[D];
  const int g = p.group ? p.group[i] : -1;
#pragma unroll
  for (int a = 0; a < D; ++a) sig[a] = (g >= 0 && g < p.G) ? p.act[g] * p.act_dir[g * D + a] : 0.f;
  float P[D][D], A[D][D], G[D][D];
  const float J = stress<D>(F, p.mat, sig, P, A);
  if (!(J > 0.f)) set_status(p.status, ST_INVERTED);
  mls_G<D>(P, F, C, -4.f * p.inv_dx * p.inv_dx * p.dt * p.vol, p.mass, G);
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz) {
        const int k[3] = {kx, ky, kz};
        float N = 1.f, dp[D];
        int nd[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          N *= st.w[a][k[a]];
          nd[a] = st.base[a] + k[a];
          dp[a] = (float(k[a]) - st.f[a]) * p.dx;
        }
        float* gp = reinterpret_cast<float*>(grid + node_lin<D>(nd, p.n));
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float s = p.mass * v[a];
#pragma unroll
          for (int c = 0; c < D; ++c) s += G[a][c] * dp[c];
          atomicAdd(gp + a, N * s);
        }
        atomicAdd(gp + D, N * p.mass);
      }
}

template <int D>
__global__ void k_na_grid(NAPar p, float4* __restrict__ grid) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= p.n_nodes) return;
  int nd[D];
  int r = l;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    nd[a] = r % p.n[a];
    r /= p.n[a];
  }
  const float4 s4 = grid[l];
  const float s[4] = {s4.x, s4.y, s4.z, s4.w};
  const float m = s[D];
  float v[D];
  if (m > 0.f) {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = s[a] / m + p.dt * p.gravity[a];
    bc_apply<D>(nd, p.n, p.bc, v);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = 0.f;
  }
  float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < D; ++a) o[a] = v[a];
  o[D] = m;
  grid[l] = make_float4(o[0], o[1], o[2], o[3]);
}

template <int D>
__global__ void k_na_g2p(NAPar p, const float4* __restrict__ grid) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  float x[D], v[D], F[D][D], C[D][D];
  na_load<D>(p, i, x, F, v, C);
  Sten<D> st;
  if (!make_stencil<D>(x, p.inv_dx, p.n, st)) return;  // reported by the scatter
  float vn[D], Cn[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vn[a] = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) Cn[a][c] = 0.f;
  }
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kz = 0; kz < (D == 3 ? 3 : 1); ++kz) {
        const int k[3] = {kx, ky, kz};
        float N = 1.f, dk[D];
        int nd[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          N *= st.w[a][k[a]];
          nd[a] = st.base[a] + k[a];
          dk[a] = float(k[a]) - st.f[a];
        }
        const float4 g4 = grid[node_lin<D>(nd, p.n)];
        const float gv[3] = {g4.x, g4.y, g4.z};
#pragma unroll
        for (int a = 0; a < D; ++a) {
          vn[a] += N * gv[a];
#pragma unroll
          for (int c = 0; c < D; ++c) Cn[a][c] += N * gv[a] * dk[c];
        }
      }
  const float s = 4.f * p.inv_dx;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) Cn[a][c] *= s;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    p.vo[size_t(i) * D + a] = vn[a];
    p.xo[size_t(i) * D + a] = x[a] + p.dt * vn[a];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float f = F[a][c];
#pragma unroll
      for (int k = 0; k < D; ++k) f += p.dt * Cn[a][k] * F[k][c];
      p.Fo[(size_t(i) * D + a) * D + c] = f;
      p.Co[(size_t(i) * D + a) * D + c] = Cn[a][c];
    }
  }
}

// Device address of the fixed scratch on the current device, looked up once per device.
mpm_status scratch_for_current_device(float4** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_grid_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_grid) != cudaSuccess || !ptr) return MPM_ERR_CUDA;
    g_grid_ptr[dev] = static_cast<float4*>(ptr);
  }
  *out = g_grid_ptr[dev];
  return MPM_OK;
}

// Launches one kernel and returns that launch's own error (cudaLaunchKernel reports it directly,
// so an error left pending by the caller's earlier work is neither read nor cleared here).
template <class... Args>
cudaError_t na_launch(void (*kernel)(Args...), int blocks, cudaStream_t s, Args... args) {
  void* argv[] = {static_cast<void*>(&args)...};
  return cudaLaunchKernel(reinterpret_cast<const void*>(kernel), dim3(blocks), dim3(256), argv, 0, s);
}

// Restores the caller's current device when the entry point switched it.
struct DeviceGuard {
  int saved = -1;
  ~DeviceGuard() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

template <int D>
mpm_status na_enqueue(const NAPar& p, float4* grid, cudaStream_t s) {
  const int nb = (p.n_nodes + 255) / 256, pb = (p.N + 255) / 256;
  // the previous call's grid is still in the array
  if (na_launch(k_na_clear, nb, s, grid, p.n_nodes) != cudaSuccess) return MPM_ERR_CUDA;
  if (p.N > 0 && na_launch(k_na_p2g<D>, pb, s, p, grid) != cudaSuccess) return MPM_ERR_CUDA;
  if (na_launch(k_na_grid<D>, nb, s, p, grid) != cudaSuccess) return MPM_ERR_CUDA;
  if (p.N > 0 && na_launch(k_na_g2p<D>, pb, s, p, static_cast<const float4*>(grid)) != cudaSuccess)
    return MPM_ERR_CUDA;
  return MPM_OK;
}

}  // namespace

extern "C" mpm_status mpm_step_noalloc(const mpm_noalloc_step* a, void* cuda_stream) {
  if (!a) return MPM_ERR_ARG;
  const int D = a->dim;
  if (D != 2 && D != 3) return MPM_ERR_ARG;
  long long nodes = 1;
  for (int k = 0; k < D; ++k) {
    // each side is bounded before it multiplies, so the product cannot wrap
    if (a->n_grid[k] < 5 || a->n_grid[k] > kNoAllocMaxNodes) return MPM_ERR_ARG;
    nodes *= a->n_grid[k];
    if (nodes > kNoAllocMaxNodes) return MPM_ERR_ARG;  // beyond the fixed scratch
  }
  if (a->n_particles < 0 || a->n_particles >= (1 << 26)) return MPM_ERR_ARG;
  if (a->n_particles > 0 && (!a->x || !a->x_out || !a->v_out || !a->C_out || !a->F_out)) return MPM_ERR_ARG;
  if (a->n_groups < 0 || (a->n_groups > 0 && (!a->act || !a->act_dir))) return MPM_ERR_ARG;
  // the same checks as mpm_scene_create, whose plain form this step reproduces
  if (!(a->dx > 0.f) || !(a->dt > 0.f) || !(a->E > 0.f) || !(a->nu > -1.f && a->nu < 0.5f)) return MPM_ERR_ARG;
  if (!(a->p_mass > 0.f) || !(a->p_vol > 0.f)) return MPM_ERR_ARG;
  if (a->bc_type != MPM_BC_STICKY && a->bc_type != MPM_BC_SLIP) return MPM_ERR_ARG;
  if (a->bc_width < 0 || !(a->friction_c >= 0.f) || !std::isfinite(a->friction_c)) return MPM_ERR_ARG;
  for (int k = 0; k < D; ++k)
    if (!std::isfinite(a->gravity[k])) return MPM_ERR_ARG;
  const double rho = double(a->p_mass) / double(a->p_vol);
  if (double(a->dt) > double(a->dx) * std::sqrt(rho / double(a->E)) * (1.0 + 1e-6)) return MPM_ERR_ARG;
  DeviceGuard guard;
  if (a->device >= 0) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return MPM_ERR_CUDA;
    if (cur != a->device) {
      if (cudaSetDevice(a->device) != cudaSuccess) return MPM_ERR_CUDA;
      guard.saved = cur;
    }
  }
  float4* grid = nullptr;
  mpm_status st = scratch_for_current_device(&grid);
  if (st != MPM_OK) return st;
  NAPar p{};
  for (int k = 0; k < 3; ++k) {
    p.n[k] = k < D ? a->n_grid[k] : 1;
    p.gravity[k] = k < D ? a->gravity[k] : 0.f;
  }
  p.dx = a->dx;
  p.inv_dx = 1.f / a->dx;
  p.dt = a->dt;
  p.mat.mu = float(double(a->E) / (2.0 * (1.0 + double(a->nu))));
  p.mat.la = float(double(a->E) * double(a->nu) / ((1.0 + double(a->nu)) * (1.0 - 2.0 * double(a->nu))));
  p.mass = a->p_mass;
  p.vol = a->p_vol;
  p.bc.width = a->bc_width;
  for (int w = 0; w < 6; ++w) {  // the same kind and friction on every wall
    p.bc.kind[w] = a->bc_type;
    p.bc.c[w] = a->friction_c;
  }
  p.N = a->n_particles;
  p.G = a->n_groups;
  p.n_nodes = int(nodes);
  p.x = a->x;
  p.v = a->v;
  p.C = a->C;
  p.F = a->F;
  p.group = a->group;
  p.act_dir = a->act_dir;
  p.act = a->act;
  p.xo = a->x_out;
  p.vo = a->v_out;
  p.Co = a->C_out;
  p.Fo = a->F_out;
  p.status = a->status;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  return D == 2 ? na_enqueue<2>(p, grid, s) : na_enqueue<3>(p, grid, s);
}
