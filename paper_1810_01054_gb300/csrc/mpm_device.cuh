// Device-side math of the differentiable MLS-MPM step (ChainQueen, arXiv 1810.01054).
//
// Per-particle pieces used by every kernel of the library: the quadratic B-spline stencil and
// its gradient, the neo-Hookean stress and its Hessian product (Section III and Supplement S4
// (H)), the MLS momentum matrix G of Eq. 4, the boundary projection of Supplement S5 (L) and its
// adjoint.  These are templates on the scalar type R: the tile and plain kernels run them in FP32,
// the double-precision plain form (mpm_f64.cu) in FP64.  Layout helpers for the SoA float4 state
// planes live here too.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbmpm {

// --------------------------------------------------------------------------- configuration
// Tiles: a CTA owns a block of B^D cells ("tile"); particles are binned by the cell of their
// stencil base, and a tile's particles touch the (B+2)^D node block starting at the tile origin.
template <int D>
struct Cfg;
template <>
struct Cfg<2> {
  static constexpr int B = 4;             // tile edge in cells
  static constexpr int CELLS = 16;        // cells per tile
  static constexpr int BN = 6;            // node-block edge (B + 2)
  static constexpr int BLOCK_NODES = 36;  // nodes per block
  static constexpr int SORT_CAP = 2048;   // most particles one tile may hold
  static constexpr int S = 12;            // floats per particle state: x(2) F(4) v(2) C(4)
  static constexpr int PLANES = 3;        // float4 planes per particle
  static constexpr int XF_PLANES = 2;     // planes holding x and F (what G2P reads)
  static constexpr int STENCIL = 9;
};
template <>
struct Cfg<3> {
  static constexpr int B = 4;
  static constexpr int CELLS = 64;
  static constexpr int BN = 6;
  static constexpr int BLOCK_NODES = 216;
  static constexpr int SORT_CAP = 4096;
  static constexpr int S = 24;            // x(3) F(9) v(3) C(9)
  static constexpr int PLANES = 6;
  static constexpr int XF_PLANES = 3;
  static constexpr int STENCIL = 27;
};

// Tile shape of the tiled form: TB^D cells per tile (TB = 4; 2D also 8 for sparse scenes, where a
// tile then holds four times the particles of a 4 x 4 tile), its node block (TB + 2)^D, and the
// most particles a tile's kernels stage.  The bin key holds the cell within the tile in 6 bits.
template <int D, int TB>
struct Tile {
  static constexpr int B = TB;
  static constexpr int CELLS = D == 2 ? TB * TB : TB * TB * TB;
  static constexpr int BN = TB + 2;
  static constexpr int BLOCK_NODES = D == 2 ? BN * BN : BN * BN * BN;
  static constexpr int SORT_CAP = D == 2 && TB == 4 ? 2048 : 4096;
  static_assert(CELLS <= 64, "the bin key holds the cell in 6 bits");
  static_assert(TB == 4 || (D == 2 && TB == 8), "tile edges: 4, and 8 in 2D");
};

// Status codes written to the per-scene device status word (first error wins).
enum : int {
  ST_OK = 0,
  ST_DOMAIN = -3,    // a stencil left the grid
  ST_INVERTED = -4,  // det F <= 0
  ST_TIMEOUT = -5,   // a bounded device wait ran out
  ST_DENSITY = -8,   // more particles in one tile than the tile kernels stage
  ST_BINNING = -9,   // a particle's bin key disagrees with its position (access skipped)
};

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// --------------------------------------------------------------------------- particle record
// One particle's state in the order x, F, v, C (row-major matrices).  The four-float planes of
// the state arrays are consecutive chunks of this record, so the first XF_PLANES planes hold
// exactly the inputs of G2P (x and F).
template <int D, class R = float>
struct Part {
  R x[D];
  R F[D][D];
  R v[D];
  R C[D][D];
};

template <int D>
__device__ __forceinline__ void unpack(const float* r, Part<D>& q) {
  int o = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) q.x[a] = r[o++];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) q.F[a][b] = r[o++];
#pragma unroll
  for (int a = 0; a < D; ++a) q.v[a] = r[o++];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) q.C[a][b] = r[o++];
}

template <int D>
__device__ __forceinline__ void pack(const Part<D>& q, float* r) {
  int o = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) r[o++] = q.x[a];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) r[o++] = q.F[a][b];
#pragma unroll
  for (int a = 0; a < D; ++a) r[o++] = q.v[a];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) r[o++] = q.C[a][b];
}

// Load the first `np` planes of particle p (plane j of the array starts at planes + j*npad).
template <int D, int NP>
__device__ __forceinline__ void load_planes(const float4* __restrict__ planes, int npad, int p, float* r) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float4 q = __ldg(planes + size_t(j) * npad + p);
    r[4 * j + 0] = q.x;
    r[4 * j + 1] = q.y;
    r[4 * j + 2] = q.z;
    r[4 * j + 3] = q.w;
  }
}

template <int D, int NP>
__device__ __forceinline__ void store_planes(float4* __restrict__ planes, int npad, int p, const float* r) {
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    planes[size_t(j) * npad + p] = make_float4(r[4 * j + 0], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
  }
}

// --------------------------------------------------------------------------- async staging
// 16-byte global -> shared copies that complete in the background (cp.async, L2 only), so a
// CTA can request a tile's particle records and do other work while they arrive.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Programmatic dependent launch.  A kernel launched with launch_pdl may be scheduled while the
// kernel before it on the stream is still running; pdl_wait() blocks until that kernel has
// completed and its writes are visible.  Every CTA of such a kernel calls pdl_wait() first, before
// any access to memory and before it can exit: the kernel then cannot complete ahead of its
// predecessor, so completion stays ordered along the whole stream.  pdl_trigger() lets the next
// kernel be scheduled; its CTAs then wait in pdl_wait() for this one to finish.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

// --------------------------------------------------------------------------- scalar functions
// One name per function for both precisions (the float overloads are the FP32 library calls).
__device__ __forceinline__ float s_log(float a) { return logf(a); }
__device__ __forceinline__ double s_log(double a) { return log(a); }
__device__ __forceinline__ float s_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double s_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float s_floor(float a) { return floorf(a); }
__device__ __forceinline__ double s_floor(double a) { return floor(a); }
__device__ __forceinline__ float s_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double s_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float s_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double s_max(double a, double b) { return fmax(a, b); }

// --------------------------------------------------------------------------- small matrices
template <int D, class R>
__device__ __forceinline__ R det(const R (&F)[D][D]) {
  if constexpr (D == 2) {
    return F[0][0] * F[1][1] - F[0][1] * F[1][0];
  } else {
    return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
           F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
  }
}

// F^{-T} from the cofactor matrix: (F^{-T})_{ij} = cof(F)_{ij} / det F.
template <int D, class R>
__device__ __forceinline__ void inv_transpose(const R (&F)[D][D], R J, R (&A)[D][D]) {
  R rJ = R(1) / J;
  if constexpr (D == 2) {
    A[0][0] = F[1][1] * rJ;
    A[0][1] = -F[1][0] * rJ;
    A[1][0] = -F[0][1] * rJ;
    A[1][1] = F[0][0] * rJ;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        A[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) * rJ;
      }
  }
}

// --------------------------------------------------------------------------- stencil
// Quadratic B-spline: per axis base = floor(x/dx - 0.5), f = x/dx - base in [0.5, 1.5); node
// base+k has weight w_k(f) and dw_k = d w_k / d x_p.
template <int D, class R = float>
struct Sten {
  int base[D];
  R f[D];
  R w[D][3];
  R dw[D][3];
};

template <int D, class R>
__device__ __forceinline__ bool stencil_base(const R* x, R inv_dx, const int* n, int* base, R* f) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    R xs = x[a] * inv_dx;
    R b = s_floor(xs - R(0.5));
    ok = ok && (b >= R(0)) && (b <= R(n[a] - 3));
    base[a] = ok ? int(b) : 0;
    f[a] = xs - b;
  }
  return ok;
}

template <class R>
__device__ __forceinline__ void bspline(R f, R inv_dx, R* w, R* dw) {
  R t0 = R(1.5) - f, t1 = f - R(1), t2 = f - R(0.5);
  w[0] = R(0.5) * t0 * t0;
  w[1] = R(0.75) - t1 * t1;
  w[2] = R(0.5) * t2 * t2;
  dw[0] = -t0 * inv_dx;
  dw[1] = R(-2) * t1 * inv_dx;
  dw[2] = t2 * inv_dx;
}

template <int D, class R>
__device__ __forceinline__ bool make_stencil(const R* x, R inv_dx, const int* n, Sten<D, R>& s) {
  bool ok = stencil_base<D>(x, inv_dx, n, s.base, s.f);
#pragma unroll
  for (int a = 0; a < D; ++a) bspline(s.f[a], inv_dx, s.w[a], s.dw[a]);
  return ok;
}

// --------------------------------------------------------------------------- constitutive
template <class R>
struct MaterialT {
  R mu, la;
};
using Material = MaterialT<float>;

// P = mu (F - F^{-T}) + lambda ln J F^{-T} + F sigma_a, sigma_a = a Diag(dir).
// Returns J (caller checks J > 0 before trusting P).
template <int D, class R>
__device__ __forceinline__ R stress(const R (&F)[D][D], MaterialT<R> m, const R* sig_diag, R (&P)[D][D],
                                    R (&A)[D][D]) {
  R J = det<D>(F);
  R Js = J > R(0) ? J : R(1);
  inv_transpose<D>(F, Js, A);
  R lJ = s_log(Js);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) P[i][j] = m.mu * (F[i][j] - A[i][j]) + m.la * lJ * A[i][j] + F[i][j] * sig_diag[j];
  return J;
}

// G = -(4/dx^2) dt V0 P F^T + m C  (Eq. 4)
template <int D, class R>
__device__ __forceinline__ void mls_G(const R (&P)[D][D], const R (&F)[D][D], const R (&C)[D][D], R kG, R mass,
                                      R (&G)[D][D]) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) s += P[i][k] * F[j][k];
      G[i][j] = kG * s + mass * C[i][j];
    }
}

// mu Pbar + (mu - lambda ln J) F^{-T} Pbar^T F^{-T} + lambda (F^{-T}:Pbar) F^{-T}
template <int D, class R>
__device__ __forceinline__ void nh_hessian_apply(const R (&A)[D][D], R J, MaterialT<R> m, const R (&Pb)[D][D],
                                                 R (&H)[D][D]) {
  R lJ = s_log(J > R(0) ? J : R(1));
  R AP = R(0);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) AP += A[i][j] * Pb[i][j];
  R T[D][D];  // A Pb^T
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) s += A[i][k] * Pb[j][k];
      T[i][j] = s;
    }
  R c = m.mu - m.la * lJ;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R s = R(0);
#pragma unroll
      for (int k = 0; k < D; ++k) s += T[i][k] * A[k][j];
      H[i][j] = m.mu * Pb[i][j] + c * s + m.la * AP * A[i][j];
    }
}

// --------------------------------------------------------------------------- boundary (S5)
// Boundary of the grid: a band `width` nodes deep along each of the 2 dim walls; wall w = 2a + side
// (axis a, low side 0) is sticky (kind 0), slip with Coulomb friction c[w] (kind 1, S5) or open
// (kind 2).
template <class R>
struct BCParT {
  int width;
  int kind[6];
  R c[6];
};
using BCPar = BCParT<float>;

// Regulariser of the tangential norm (keeps the projection differentiable at v_t = 0).
template <class R>
__device__ __forceinline__ R bc_eps() {
  return R(1e-20);
}
template <>
__device__ __forceinline__ float bc_eps<float>() {
  return 1e-20f;
}

// Whether node idx lies in wall w's band.
__device__ __forceinline__ bool wall_hit(const int* idx, const int* n, int width, int w) {
  const int a = w >> 1;
  return (w & 1) ? idx[a] >= n[a] - width : idx[a] < width;
}

// One wall: v <- l_t* v_t / l_t + max(l_n, 0) n, l_t* = max(l_t + c min(l_n, 0), 0).
template <int D, class R>
__device__ __forceinline__ void project(R* v, int axis, R sgn, R c) {
  R ln = v[axis] * sgn;
  R vt[D];
  R lt2 = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vt[a] = v[a] - (a == axis ? ln * sgn : R(0));
    lt2 += vt[a] * vt[a];
  }
  R lt = s_sqrt(lt2 + bc_eps<R>());
  R Rt = lt + c * s_min(ln, R(0));
  R lts = s_max(Rt, R(0));
  R s = lts / lt;
#pragma unroll
  for (int a = 0; a < D; ++a) v[a] = s * vt[a] + (a == axis ? s_max(ln, R(0)) * sgn : R(0));
}

// Adjoint of `project` at input v (forward value recomputed here), g in/out.
template <int D, class R>
__device__ __forceinline__ void project_adj(const R* v, int axis, R sgn, R c, R* g) {
  R ln = v[axis] * sgn;
  R vt[D];
  R lt2 = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vt[a] = v[a] - (a == axis ? ln * sgn : R(0));
    lt2 += vt[a] * vt[a];
  }
  R lt = s_sqrt(lt2 + bc_eps<R>());
  R Rt = lt + c * s_min(ln, R(0));
  R lts = s_max(Rt, R(0));
  R rlt = R(1) / lt;
  R g_lts = R(0), s = R(0), gn = g[axis] * sgn;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    g_lts += g[a] * vt[a] * rlt;
    s += vt[a] * g[a] * lts;  // v_t . vhat_bar with vhat_bar = g l_t*
  }
  R HR = Rt >= R(0) ? R(1) : R(0);
  R g_lt = -s * rlt * rlt + g_lts * HR;
  R gvt[D];
  R vtn = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    gvt[a] = (g_lt * vt[a] + g[a] * lts) * rlt;
    vtn += (a == axis ? gvt[a] * sgn : R(0));
  }
  R g_ln = -vtn + g_lts * HR * c * (ln <= R(0) ? R(1) : R(0)) + (ln >= R(0) ? R(1) : R(0)) * gn;
#pragma unroll
  for (int a = 0; a < D; ++a) g[a] = gvt[a] + (a == axis ? g_ln * sgn : R(0));
}

// Boundary condition on the node velocity (gravity already added).  A node in a sticky wall's
// band is fixed; otherwise the slip walls whose band contains it are applied in sequence: axis
// 0, 1, 2, low side before high side, each with its own friction; open walls do nothing.
template <int D, class R>
__device__ __forceinline__ void bc_apply(const int* idx, const int* n, const BCParT<R>& bc, R* v) {
  bool hit[2 * D], any = false, sticky = false;
#pragma unroll
  for (int w = 0; w < 2 * D; ++w) {
    hit[w] = wall_hit(idx, n, bc.width, w);
    any = any || hit[w];
    sticky = sticky || (hit[w] && bc.kind[w] == 0);
  }
  if (!any) return;
  if (sticky) {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = R(0);
    return;
  }
#pragma unroll
  for (int w = 0; w < 2 * D; ++w)
    if (hit[w] && bc.kind[w] == 1) project<D>(v, w >> 1, (w & 1) ? R(-1) : R(1), bc.c[w]);
}

// Adjoint of bc_apply: g holds dL/dv* on entry and dL/dv_g on exit; vg = velocity before BC.
template <int D, class R>
__device__ __forceinline__ void bc_adjoint(const int* idx, const int* n, const BCParT<R>& bc, const R* vg, R* g) {
  bool hit[2 * D], any = false, sticky = false;
#pragma unroll
  for (int w = 0; w < 2 * D; ++w) {
    hit[w] = wall_hit(idx, n, bc.width, w) && bc.kind[w] != 2;
    any = any || hit[w];
    sticky = sticky || (hit[w] && bc.kind[w] == 0);
  }
  if (!any) return;
  if (sticky) {
#pragma unroll
    for (int a = 0; a < D; ++a) g[a] = R(0);
    return;
  }
  // replay the wall sequence (wall w: axis w / 2, low side for even w) to get every wall's input,
  // then walk it backwards; the loops are unrolled so the inputs stay in registers
  R vin[2 * D][D];
  R v[D];
#pragma unroll
  for (int a = 0; a < D; ++a) v[a] = vg[a];
#pragma unroll
  for (int w = 0; w < 2 * D; ++w) {
#pragma unroll
    for (int b = 0; b < D; ++b) vin[w][b] = v[b];
    if (hit[w]) project<D>(v, w >> 1, (w & 1) ? R(-1) : R(1), bc.c[w]);
  }
#pragma unroll
  for (int w = 2 * D - 1; w >= 0; --w)
    if (hit[w]) project_adj<D>(vin[w], w >> 1, (w & 1) ? R(-1) : R(1), bc.c[w], g);
}

}  // namespace gbmpm
