// FP64 CPU oracle for the differentiable MLS-MPM time step (ChainQueen, arXiv 1810.01054).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
// (and its `--impl reference` arm) may load this code.  It shares no code, header, table or
// helper with the CUDA library; it is a plain, slow, single-threaded restatement of the method:
//
//   forward  - Section III, Eqs. 3-10 (P2G, grid normalisation, G2P, F and x update), with the
//              actuation model P = P(F) + F sigma_a of Section III; the constitutive model is the
//              compressible neo-Hookean solid, psi = mu/2 (tr F^T F - d) - mu ln J + lambda/2 (ln J)^2.
//   reverse  - Supplement S2 (A)-(C), S3 (D)-(E), S4 (F)-(K) and S5 (L), evaluated in that order.
//   control  - the tanh controller of Section V-B in the three forms used by the workloads.
//
// Loops run particle -> stencil node with no sorting, tiling or fusion; every quantity is
// recomputed from its definition.  Readings of passages the paper leaves open (weights'
// base, grid geometry, empty nodes, gravity placement, boundary set, epsilon of S5, typos of
// S1/S4) are restated where they are used below.
//
// Status codes: 0 ok, -1 bad argument, -3 a stencil left the grid, -4 det F <= 0.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

typedef struct {
  int dim;            // 2 or 3
  int n_grid[3];      // nodes per axis; node i sits at i*dx, i in [0, n)
  double dx, dt;
  double gravity[3];
  double E, nu;       // Young's modulus, Poisson ratio (Lame parameters by the textbook map)
  double p_mass, p_vol;  // m_p (unless p_m below is given) and V_p^0 (uniform within a scene)
  int bc_type;        // 0 sticky, 1 slip with Coulomb friction c (S5)
  int bc_width;       // boundary band width in nodes
  double friction_c;
  int n_particles;
  int n_groups;
  const int32_t* group;   // [N], -1 = unactuated
  const double* act_dir;  // [G][dim]
  int ctrl_type;          // 0 sinusoid amplitude, 1 sinusoid basis, 2 MLP on centroids
  int ctrl_hidden;
  double ctrl_freq;
  double ctrl_scale;
  const double* p_E;      // [N] per-particle Young's modulus, NULL = E for every particle
  const double* p_m;      // [N] per-particle mass, NULL = p_mass for every particle
  const int* wall_kind;   // [2 dim] per wall (axis a, low side 2a, high side 2a+1): 0 sticky,
                          // 1 slip with friction wall_c, 2 open; NULL = bc_type on every wall
  const double* wall_c;   // [2 dim] friction of each wall, NULL = friction_c
} oracle_scene;

}  // extern "C"

namespace {

const double kPi = 3.14159265358979323846;
const double kEps = 1e-20;  // epsilon of the tangential length in S5 (unspecified there)

struct M3 {
  double a[3][3];
};

M3 zero3() {
  M3 m;
  std::memset(m.a, 0, sizeof(m.a));
  return m;
}

M3 load_mat(const double* p, int d) {
  M3 m = zero3();
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) m.a[i][j] = p[i * d + j];
  return m;
}

void store_mat(double* p, const M3& m, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) p[i * d + j] = m.a[i][j];
}

M3 matmul(const M3& A, const M3& B, int d) {
  M3 C = zero3();
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      for (int k = 0; k < d; ++k) C.a[i][j] += A.a[i][k] * B.a[k][j];
  return C;
}

M3 transpose(const M3& A, int d) {
  M3 T = zero3();
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) T.a[i][j] = A.a[j][i];
  return T;
}

double det(const M3& F, int d) {
  if (d == 2) return F.a[0][0] * F.a[1][1] - F.a[0][1] * F.a[1][0];
  return F.a[0][0] * (F.a[1][1] * F.a[2][2] - F.a[1][2] * F.a[2][1]) -
         F.a[0][1] * (F.a[1][0] * F.a[2][2] - F.a[1][2] * F.a[2][0]) +
         F.a[0][2] * (F.a[1][0] * F.a[2][1] - F.a[1][1] * F.a[2][0]);
}

// Inverse by the adjugate: F^{-1} = adj(F) / det F.
M3 inverse(const M3& F, int d) {
  M3 R = zero3();
  double J = det(F, d);
  if (d == 2) {
    R.a[0][0] = F.a[1][1] / J;
    R.a[0][1] = -F.a[0][1] / J;
    R.a[1][0] = -F.a[1][0] / J;
    R.a[1][1] = F.a[0][0] / J;
    return R;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // cofactor of F[j][i]
      int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
      R.a[i][j] = (F.a[r0][c0] * F.a[r1][c1] - F.a[r0][c1] * F.a[r1][c0]) / J;
    }
  return R;
}

// Lame parameters from (E, nu) by the textbook map; per particle when the scene carries E_p.
// dmu/dE and dlambda/dE are the same map at E = 1.
void lame_E(double E, double nu, double* mu, double* la) {
  *mu = E / (2.0 * (1.0 + nu));
  *la = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}
void lame(const oracle_scene* s, double* mu, double* la) { lame_E(s->E, s->nu, mu, la); }
void lame_of(const oracle_scene* s, int p, double* mu, double* la) {
  lame_E(s->p_E ? s->p_E[p] : s->E, s->nu, mu, la);
}
double mass_of(const oracle_scene* s, int p) { return s->p_m ? s->p_m[p] : s->p_mass; }

// Neo-Hookean first Piola-Kirchhoff stress P = d psi / dF = mu (F - F^{-T}) + lambda ln J F^{-T}.
M3 neohookean_P(const M3& F, int d, double mu, double la) {
  double J = det(F, d);
  M3 FinvT = transpose(inverse(F, d), d);
  M3 P = zero3();
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      P.a[i][j] = mu * (F.a[i][j] - FinvT.a[i][j]) + la * std::log(J) * FinvT.a[i][j];
  return P;
}

// Second derivative of psi contracted with Pbar: the term sum_{gamma,eta} Pbar_{gamma eta}
// d^2 psi / dF_{gamma eta} dF_{alpha beta} of S4 (H), for the neo-Hookean psi:
//   mu Pbar + (mu - lambda ln J) F^{-T} Pbar^T F^{-T} + lambda (F^{-T} : Pbar) F^{-T}.
M3 neohookean_hessian_apply(const M3& F, const M3& Pbar, int d, double mu, double la) {
  double J = det(F, d);
  M3 A = transpose(inverse(F, d), d);
  M3 APtA = matmul(matmul(A, transpose(Pbar, d), d), A, d);
  double AdotP = 0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) AdotP += A.a[i][j] * Pbar.a[i][j];
  M3 R = zero3();
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      R.a[i][j] = mu * Pbar.a[i][j] + (mu - la * std::log(J)) * APtA.a[i][j] + la * AdotP * A.a[i][j];
  return R;
}

// Quadratic B-spline stencil of one particle.  Reading of the paper (it names N only): per
// axis, base = floor(x/dx - 0.5), f = x/dx - base in [0.5, 1.5), and the weights of nodes
// base+0, base+1, base+2 are 1/2 (1.5-f)^2, 3/4 - (f-1)^2, 1/2 (f-0.5)^2.  dw holds the
// derivatives of these weights with respect to the particle position x_p.
struct Stencil {
  int base[3];
  double w[3][3];
  double dw[3][3];
};

bool make_stencil(const oracle_scene* s, const double* x, Stencil* st) {
  int d = s->dim;
  for (int a = 0; a < d; ++a) {
    double xs = x[a] / s->dx;
    double b = std::floor(xs - 0.5);
    double f = xs - b;
    if (!(b >= 0.0) || b + 2.0 > double(s->n_grid[a] - 1)) return false;
    st->base[a] = int(b);
    st->w[a][0] = 0.5 * (1.5 - f) * (1.5 - f);
    st->w[a][1] = 0.75 - (f - 1.0) * (f - 1.0);
    st->w[a][2] = 0.5 * (f - 0.5) * (f - 0.5);
    st->dw[a][0] = -(1.5 - f) / s->dx;
    st->dw[a][1] = -2.0 * (f - 1.0) / s->dx;
    st->dw[a][2] = (f - 0.5) / s->dx;
  }
  return true;
}

int n_nodes(const oracle_scene* s) {
  int c = 1;
  for (int a = 0; a < s->dim; ++a) c *= s->n_grid[a];
  return c;
}

int n_stencil(int d) { return d == 2 ? 9 : 27; }

// Offsets k of stencil entry q (last axis fastest).
void stencil_offset(int q, int d, int* k) {
  if (d == 2) {
    k[0] = q / 3;
    k[1] = q % 3;
    k[2] = 0;
  } else {
    k[0] = q / 9;
    k[1] = (q / 3) % 3;
    k[2] = q % 3;
  }
}

int node_index(const oracle_scene* s, const int* idx) {
  int lin = 0;
  for (int a = 0; a < s->dim; ++a) lin = lin * s->n_grid[a] + idx[a];
  return lin;
}

void node_coords(const oracle_scene* s, int lin, int* idx) {
  for (int a = s->dim - 1; a >= 0; --a) {
    idx[a] = lin % s->n_grid[a];
    lin /= s->n_grid[a];
  }
}

// N_ip and dN_ip/dx_p for stencil entry q.
void weight(const Stencil& st, int d, int q, double* N, double* dN) {
  int k[3];
  stencil_offset(q, d, k);
  double n = 1.0;
  for (int a = 0; a < d; ++a) n *= st.w[a][k[a]];
  *N = n;
  for (int a = 0; a < d; ++a) {
    double g = st.dw[a][k[a]];
    for (int b = 0; b < d; ++b)
      if (b != a) g *= st.w[b][k[b]];
    dN[a] = g;
  }
}

// Boundary nodes: those with an axis index < bc_width or >= n - bc_width.
bool in_band(const oracle_scene* s, const int* idx) {
  for (int a = 0; a < s->dim; ++a)
    if (idx[a] < s->bc_width || idx[a] >= s->n_grid[a] - s->bc_width) return true;
  return false;
}

// One wall of S5 (L): project v against inward normal n with friction c.
struct ProjTape {
  double v[3], n[3], vt[3], ln, lt, lts, R;
};

void project_forward(const double* v, const double* nrm, double c, int d, double* out, ProjTape* t) {
  double ln = 0;
  for (int a = 0; a < d; ++a) ln += v[a] * nrm[a];
  double vt[3], lt2 = 0;
  for (int a = 0; a < d; ++a) {
    vt[a] = v[a] - ln * nrm[a];
    lt2 += vt[a] * vt[a];
  }
  double lt = std::sqrt(lt2 + kEps);
  double R = lt + c * std::min(ln, 0.0);
  double lts = std::max(R, 0.0);
  for (int a = 0; a < d; ++a) out[a] = lts * (vt[a] / lt) + std::max(ln, 0.0) * nrm[a];
  if (t) {
    for (int a = 0; a < 3; ++a) {
      t->v[a] = a < d ? v[a] : 0;
      t->n[a] = a < d ? nrm[a] : 0;
      t->vt[a] = a < d ? vt[a] : 0;
    }
    t->ln = ln;
    t->lt = lt;
    t->lts = lts;
    t->R = R;
  }
}

inline double H(double x) { return x >= 0.0 ? 1.0 : 0.0; }  // H(x) = [x >= 0] as in S5

// Adjoint of project_forward, following S5 (L) term by term.
void project_adjoint(const ProjTape& t, double c, int d, const double* gout, double* gv) {
  double vhat[3];
  for (int a = 0; a < d; ++a) vhat[a] = t.vt[a] / t.lt;
  double g_lts = 0;
  for (int a = 0; a < d; ++a) g_lts += gout[a] * vhat[a];
  double g_vhat[3];
  for (int a = 0; a < d; ++a) g_vhat[a] = gout[a] * t.lts;
  double s = 0;
  for (int a = 0; a < d; ++a) s += t.vt[a] * g_vhat[a];
  double g_lt = -s / (t.lt * t.lt) + g_lts * H(t.R);
  double g_vt[3];
  for (int a = 0; a < d; ++a) g_vt[a] = (g_lt * t.vt[a] + g_vhat[a]) / t.lt;
  double vtn = 0, gn = 0;
  for (int a = 0; a < d; ++a) {
    vtn += g_vt[a] * t.n[a];
    gn += t.n[a] * gout[a];
  }
  double g_ln = -vtn + g_lts * H(t.R) * c * H(-t.ln) + H(t.ln) * gn;
  for (int a = 0; a < d; ++a) gv[a] = g_ln * t.n[a] + g_vt[a];
}

// Boundary condition applied to a node velocity.  Wall w = 2a + side (axis a, low side first) is
// sticky, slip with its own friction c (S5) or open; its band holds the nodes with idx[a] < width
// (low) or idx[a] >= n_a - width (high).  A node in the band of a sticky wall is fixed (v* = 0);
// otherwise the slip walls whose band contains it are applied one after another, axis 0,1,2, low
// side before high side, with inward normal +e_a (low) or -e_a (high); open walls do nothing.
// With one kind and c for every wall this is the uniform sticky or slip boundary.
struct BCTape {
  int n_walls;
  ProjTape walls[6];
  double c[6];
};

int wall_kind(const oracle_scene* s, int w) { return s->wall_kind ? s->wall_kind[w] : s->bc_type; }
double wall_c(const oracle_scene* s, int w) { return s->wall_c ? s->wall_c[w] : s->friction_c; }
bool wall_hit(const oracle_scene* s, const int* idx, int w) {
  const int a = w >> 1;
  return (w & 1) ? idx[a] >= s->n_grid[a] - s->bc_width : idx[a] < s->bc_width;
}
bool sticky_node(const oracle_scene* s, const int* idx) {
  for (int w = 0; w < 2 * s->dim; ++w)
    if (wall_hit(s, idx, w) && wall_kind(s, w) == 0) return true;
  return false;
}

void bc_forward(const oracle_scene* s, const int* idx, const double* vin, double* vout, BCTape* tape) {
  int d = s->dim;
  if (tape) tape->n_walls = 0;
  if (!in_band(s, idx)) {
    for (int a = 0; a < d; ++a) vout[a] = vin[a];
    return;
  }
  if (sticky_node(s, idx)) {
    for (int a = 0; a < d; ++a) vout[a] = 0;
    return;
  }
  double v[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) v[a] = vin[a];
  for (int w = 0; w < 2 * d; ++w) {
    if (!wall_hit(s, idx, w) || wall_kind(s, w) != 1) continue;
    double nrm[3] = {0, 0, 0};
    nrm[w >> 1] = (w & 1) ? -1.0 : 1.0;
    double out[3];
    if (tape) tape->c[tape->n_walls] = wall_c(s, w);
    ProjTape* t = tape ? &tape->walls[tape->n_walls++] : nullptr;
    project_forward(v, nrm, wall_c(s, w), d, out, t);
    for (int b = 0; b < d; ++b) v[b] = out[b];
  }
  for (int a = 0; a < d; ++a) vout[a] = v[a];
}

void bc_adjoint(const oracle_scene* s, const int* idx, const BCTape& tape, const double* gout, double* gin) {
  int d = s->dim;
  if (!in_band(s, idx)) {
    for (int a = 0; a < d; ++a) gin[a] = gout[a];
    return;
  }
  if (sticky_node(s, idx)) {
    for (int a = 0; a < d; ++a) gin[a] = 0;
    return;
  }
  double g[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) g[a] = gout[a];
  for (int w = tape.n_walls - 1; w >= 0; --w) {
    double gi[3];
    project_adjoint(tape.walls[w], tape.c[w], d, g, gi);
    for (int a = 0; a < d; ++a) g[a] = gi[a];
  }
  for (int a = 0; a < d; ++a) gin[a] = g[a];
}

// Per-particle quantities of P2G (Section III, Eq. 4 and the actuation model).
struct ParticleP2G {
  M3 F, P, G, sig;
  double J;
};

bool particle_stress(const oracle_scene* s, const double* act, int p, const double* F_in,
                     const double* C_in, ParticleP2G* q) {
  int d = s->dim;
  double mu, la;
  lame_of(s, p, &mu, &la);
  q->F = load_mat(F_in, d);
  q->J = det(q->F, d);
  if (!(q->J > 0.0)) return false;
  q->sig = zero3();
  int g = s->group ? s->group[p] : -1;
  if (g >= 0 && g < s->n_groups) {
    for (int a = 0; a < d; ++a) q->sig.a[a][a] = act[g] * s->act_dir[g * d + a];
  }
  // P = P(F) + F sigma_a
  M3 P = neohookean_P(q->F, d, mu, la);
  M3 Fs = matmul(q->F, q->sig, d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) P.a[i][j] += Fs.a[i][j];
  q->P = P;
  // G = -(4/dx^2) dt V0 P F^T + m C
  double k = -4.0 / (s->dx * s->dx) * s->dt * s->p_vol;
  M3 PFt = matmul(P, transpose(q->F, d), d);
  M3 C = load_mat(C_in, d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) q->G.a[i][j] = k * PFt.a[i][j] + mass_of(s, p) * C.a[i][j];
  return true;
}

// Grid quantities of one step.
struct Grid {
  std::vector<double> m, p, vraw, vg, vstar;  // p, vraw, vg, vstar: [nodes][d]
  std::vector<BCTape> tape;
};

int forward_grid(const oracle_scene* s, const double* act, const double* x, const double* v,
                 const double* C, const double* F, Grid* g, bool keep_tape) {
  int d = s->dim, N = s->n_particles, nn = n_nodes(s), ns = n_stencil(d);
  g->m.assign(nn, 0.0);
  g->p.assign(size_t(nn) * d, 0.0);
  g->vraw.assign(size_t(nn) * d, 0.0);
  g->vg.assign(size_t(nn) * d, 0.0);
  g->vstar.assign(size_t(nn) * d, 0.0);
  if (keep_tape) g->tape.assign(nn, BCTape());
  // P2G (Eqs. 3-5)
  for (int p = 0; p < N; ++p) {
    Stencil st;
    if (!make_stencil(s, x + p * d, &st)) return -3;
    ParticleP2G q;
    if (!particle_stress(s, act, p, F + p * d * d, C + p * d * d, &q)) return -4;
    for (int e = 0; e < ns; ++e) {
      int k[3], idx[3];
      stencil_offset(e, d, k);
      for (int a = 0; a < d; ++a) idx[a] = st.base[a] + k[a];
      double N_, dN[3];
      weight(st, d, e, &N_, dN);
      int lin = node_index(s, idx);
      double dpos[3];
      for (int a = 0; a < d; ++a) dpos[a] = idx[a] * s->dx - x[p * d + a];
      g->m[lin] += N_ * mass_of(s, p);
      for (int a = 0; a < d; ++a) {
        double Gd = 0;
        for (int b = 0; b < d; ++b) Gd += q.G.a[a][b] * dpos[b];
        g->p[size_t(lin) * d + a] += N_ * (mass_of(s, p) * v[p * d + a] + Gd);
      }
    }
  }
  // Grid operations: Eq. 6, then gravity and the boundary condition (readings: gravity is
  // added after normalisation; a node is active iff m_i > 0 exactly, else v* = 0).
  for (int lin = 0; lin < nn; ++lin) {
    if (!(g->m[lin] > 0.0)) continue;
    int idx[3];
    node_coords(s, lin, idx);
    double vg[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      g->vraw[size_t(lin) * d + a] = g->p[size_t(lin) * d + a] / g->m[lin];
      vg[a] = g->vraw[size_t(lin) * d + a] + s->dt * s->gravity[a];
      g->vg[size_t(lin) * d + a] = vg[a];
    }
    double vs[3];
    bc_forward(s, idx, vg, vs, keep_tape ? &g->tape[lin] : nullptr);
    for (int a = 0; a < d; ++a) g->vstar[size_t(lin) * d + a] = vs[a];
  }
  return 0;
}

// Input of the closed-loop controller (type 4): z = [target (d), c_g (d per group), u_g (d per
// group)] with c_g, u_g the unweighted means of x and v over group g (0 for an empty group); the
// group sizes go to cnt when given.
void com_input(const oracle_scene* s, const double* params, const double* x, const double* v,
               std::vector<double>* z, std::vector<double>* cnt_out) {
  const int G = s->n_groups, d = s->dim, N = s->n_particles;
  std::vector<double> cnt(G, 0.0), cx(size_t(G) * d, 0.0), cv(size_t(G) * d, 0.0);
  for (int p = 0; p < N; ++p) {
    const int g = s->group ? s->group[p] : -1;
    if (g < 0 || g >= G) continue;
    cnt[g] += 1.0;
    for (int a = 0; a < d; ++a) {
      cx[g * d + a] += x[p * d + a];
      cv[g * d + a] += v[p * d + a];
    }
  }
  z->assign(size_t(d) * (1 + 2 * G), 0.0);
  for (int a = 0; a < d; ++a) (*z)[a] = params[a];
  for (int g = 0; g < G; ++g)
    for (int a = 0; a < d; ++a) {
      (*z)[d + g * d + a] = cnt[g] > 0 ? cx[g * d + a] / cnt[g] : 0.0;
      (*z)[d + G * d + g * d + a] = cnt[g] > 0 ? cv[g * d + a] / cnt[g] : 0.0;
    }
  if (cnt_out) *cnt_out = cnt;
}

}  // namespace

extern "C" {

int oracle_version() { return 1; }

// Actuation a_g(t_n), t_n = step * dt, for every group (Section V-B controller forms).
//   type 0: a_g = A_g sin(2 pi f t)                      params [G]
//   type 1: a_g = sum_j W_gj b_j(t),
//           b = [sin 2pi f t, cos 2pi f t, sin 4pi f t, cos 4pi f t]   params [G][4]
//   type 2: z = (c_g - c_body) for every group (G*d), c = unweighted centroids of x;
//           h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), a = scale * tanh(W3 h2 + b3)
//   type 3: the actuation of every step is a decision variable (the per-step actuation of the
//           trajectory-optimisation examples, Section V-C): a_g(t_n) = U[n][g] for 0 <= n < L,
//           L = ctrl_hidden steps, and 0 after the table      params [L][G]
//   type 4: the closed-loop controller of Section V-B, a = scale * tanh(W z + b) with z = target
//           position, centre of mass and velocity of every component (group):
//           z = [target, c_1..c_G, u_1..u_G], c_g, u_g the means of x, v over group g
//                                                  params [target (d), W [G][d(1+2G)], b [G]]
int oracle_controller_xv(const oracle_scene* s, const double* params, int step, const double* x, const double* v,
                         double* act) {
  int G = s->n_groups, d = s->dim, N = s->n_particles;
  double t = step * s->dt;
  if (s->ctrl_type == 0) {
    for (int g = 0; g < G; ++g) act[g] = params[g] * std::sin(2.0 * kPi * s->ctrl_freq * t);
    return 0;
  }
  if (s->ctrl_type == 1) {
    double w = 2.0 * kPi * s->ctrl_freq * t;
    double b[4] = {std::sin(w), std::cos(w), std::sin(2.0 * w), std::cos(2.0 * w)};
    for (int g = 0; g < G; ++g) {
      double a = 0;
      for (int j = 0; j < 4; ++j) a += params[g * 4 + j] * b[j];
      act[g] = a;
    }
    return 0;
  }
  if (s->ctrl_type == 2) {
    int H_ = s->ctrl_hidden, Z = G * d;
    std::vector<double> cg(size_t(G) * d, 0.0), cnt(G, 0.0), cb(d, 0.0);
    for (int p = 0; p < N; ++p) {
      for (int a = 0; a < d; ++a) cb[a] += x[p * d + a];
      int g = s->group[p];
      if (g < 0 || g >= G) continue;
      cnt[g] += 1.0;
      for (int a = 0; a < d; ++a) cg[g * d + a] += x[p * d + a];
    }
    std::vector<double> z(Z);
    for (int g = 0; g < G; ++g)
      for (int a = 0; a < d; ++a)
        z[g * d + a] = (cnt[g] > 0 ? cg[g * d + a] / cnt[g] : 0.0) - cb[a] / N;
    const double* W1 = params;
    const double* b1 = W1 + H_ * Z;
    const double* W2 = b1 + H_;
    const double* b2 = W2 + H_ * H_;
    const double* W3 = b2 + H_;
    const double* b3 = W3 + G * H_;
    std::vector<double> h1(H_), h2(H_);
    for (int i = 0; i < H_; ++i) {
      double u = b1[i];
      for (int j = 0; j < Z; ++j) u += W1[i * Z + j] * z[j];
      h1[i] = std::tanh(u);
    }
    for (int i = 0; i < H_; ++i) {
      double u = b2[i];
      for (int j = 0; j < H_; ++j) u += W2[i * H_ + j] * h1[j];
      h2[i] = std::tanh(u);
    }
    for (int g = 0; g < G; ++g) {
      double u = b3[g];
      for (int j = 0; j < H_; ++j) u += W3[g * H_ + j] * h2[j];
      act[g] = s->ctrl_scale * std::tanh(u);
    }
    return 0;
  }
  if (s->ctrl_type == 3) {
    for (int g = 0; g < G; ++g) act[g] = (step >= 0 && step < s->ctrl_hidden) ? params[size_t(step) * G + g] : 0.0;
    return 0;
  }
  if (s->ctrl_type == 4) {
    if (!v) return -1;
    std::vector<double> z;
    com_input(s, params, x, v, &z, nullptr);
    const int Z = int(z.size());
    const double* W = params + d;
    const double* b = W + size_t(G) * Z;
    for (int g = 0; g < G; ++g) {
      double u = b[g];
      for (int j = 0; j < Z; ++j) u += W[size_t(g) * Z + j] * z[j];
      act[g] = s->ctrl_scale * std::tanh(u);
    }
    return 0;
  }
  return -1;
}

int oracle_controller(const oracle_scene* s, const double* params, int step, const double* x, double* act) {
  return oracle_controller_xv(s, params, step, x, nullptr, act);
}

// Reverse of oracle_controller: gparams += (da/dparams)^T gact; gx += (da/dx)^T gact (type 2).
int oracle_controller_adjoint_xv(const oracle_scene* s, const double* params, int step, const double* x,
                                 const double* v, const double* gact, double* gparams, double* gx, double* gv) {
  int G = s->n_groups, d = s->dim, N = s->n_particles;
  double t = step * s->dt;
  if (s->ctrl_type == 0) {
    for (int g = 0; g < G; ++g) gparams[g] += gact[g] * std::sin(2.0 * kPi * s->ctrl_freq * t);
    return 0;
  }
  if (s->ctrl_type == 1) {
    double w = 2.0 * kPi * s->ctrl_freq * t;
    double b[4] = {std::sin(w), std::cos(w), std::sin(2.0 * w), std::cos(2.0 * w)};
    for (int g = 0; g < G; ++g)
      for (int j = 0; j < 4; ++j) gparams[g * 4 + j] += gact[g] * b[j];
    return 0;
  }
  if (s->ctrl_type == 2) {
    int H_ = s->ctrl_hidden, Z = G * d;
    std::vector<double> cg(size_t(G) * d, 0.0), cnt(G, 0.0), cb(d, 0.0);
    for (int p = 0; p < N; ++p) {
      for (int a = 0; a < d; ++a) cb[a] += x[p * d + a];
      int g = s->group[p];
      if (g < 0 || g >= G) continue;
      cnt[g] += 1.0;
      for (int a = 0; a < d; ++a) cg[g * d + a] += x[p * d + a];
    }
    std::vector<double> z(Z);
    for (int g = 0; g < G; ++g)
      for (int a = 0; a < d; ++a)
        z[g * d + a] = (cnt[g] > 0 ? cg[g * d + a] / cnt[g] : 0.0) - cb[a] / N;
    const double* W1 = params;
    const double* b1 = W1 + H_ * Z;
    const double* W2 = b1 + H_;
    const double* b2 = W2 + H_ * H_;
    const double* W3 = b2 + H_;
    const double* b3 = W3 + G * H_;
    double* gW1 = gparams;
    double* gb1 = gW1 + H_ * Z;
    double* gW2 = gb1 + H_;
    double* gb2 = gW2 + H_ * H_;
    double* gW3 = gb2 + H_;
    double* gb3 = gW3 + G * H_;
    std::vector<double> h1(H_), h2(H_), o(G);
    for (int i = 0; i < H_; ++i) {
      double u = b1[i];
      for (int j = 0; j < Z; ++j) u += W1[i * Z + j] * z[j];
      h1[i] = std::tanh(u);
    }
    for (int i = 0; i < H_; ++i) {
      double u = b2[i];
      for (int j = 0; j < H_; ++j) u += W2[i * H_ + j] * h1[j];
      h2[i] = std::tanh(u);
    }
    for (int g = 0; g < G; ++g) {
      double u = b3[g];
      for (int j = 0; j < H_; ++j) u += W3[g * H_ + j] * h2[j];
      o[g] = std::tanh(u);
    }
    // a = scale * o, o = tanh(u3)
    std::vector<double> gu3(G), gh2(H_, 0.0), gu2(H_), gh1(H_, 0.0), gu1(H_), gz(Z, 0.0);
    for (int g = 0; g < G; ++g) gu3[g] = gact[g] * s->ctrl_scale * (1.0 - o[g] * o[g]);
    for (int g = 0; g < G; ++g) {
      gb3[g] += gu3[g];
      for (int j = 0; j < H_; ++j) {
        gW3[g * H_ + j] += gu3[g] * h2[j];
        gh2[j] += gu3[g] * W3[g * H_ + j];
      }
    }
    for (int i = 0; i < H_; ++i) gu2[i] = gh2[i] * (1.0 - h2[i] * h2[i]);
    for (int i = 0; i < H_; ++i) {
      gb2[i] += gu2[i];
      for (int j = 0; j < H_; ++j) {
        gW2[i * H_ + j] += gu2[i] * h1[j];
        gh1[j] += gu2[i] * W2[i * H_ + j];
      }
    }
    for (int i = 0; i < H_; ++i) gu1[i] = gh1[i] * (1.0 - h1[i] * h1[i]);
    for (int i = 0; i < H_; ++i) {
      gb1[i] += gu1[i];
      for (int j = 0; j < Z; ++j) {
        gW1[i * Z + j] += gu1[i] * z[j];
        gz[j] += gu1[i] * W1[i * Z + j];
      }
    }
    if (gx) {
      // z_g = c_g - c_body: dc_g/dx_p = 1/|g| for p in g, dc_body/dx_p = 1/N.
      std::vector<double> gcb(d, 0.0);
      for (int g = 0; g < G; ++g)
        for (int a = 0; a < d; ++a) gcb[a] -= gz[g * d + a];
      for (int p = 0; p < N; ++p) {
        int g = s->group[p];
        for (int a = 0; a < d; ++a) {
          double acc = gcb[a] / N;
          if (g >= 0 && g < G && cnt[g] > 0) acc += gz[g * d + a] / cnt[g];
          gx[p * d + a] += acc;
        }
      }
    }
    return 0;
  }
  if (s->ctrl_type == 3) {
    if (step >= 0 && step < s->ctrl_hidden)
      for (int g = 0; g < G; ++g) gparams[size_t(step) * G + g] += gact[g];
    return 0;
  }
  if (s->ctrl_type == 4) {
    if (!v) return -1;
    std::vector<double> z, cnt;
    com_input(s, params, x, v, &z, &cnt);
    const int Z = int(z.size());
    const double* W = params + d;
    const double* b = W + size_t(G) * Z;
    double* gW = gparams + d;
    double* gb = gW + size_t(G) * Z;
    std::vector<double> gz(Z, 0.0);
    for (int g = 0; g < G; ++g) {
      double u = b[g];
      for (int j = 0; j < Z; ++j) u += W[size_t(g) * Z + j] * z[j];
      const double th = std::tanh(u);
      const double gu = gact[g] * s->ctrl_scale * (1.0 - th * th);
      gb[g] += gu;
      for (int j = 0; j < Z; ++j) {
        gW[size_t(g) * Z + j] += gu * z[j];
        gz[j] += W[size_t(g) * Z + j] * gu;
      }
    }
    for (int a = 0; a < d; ++a) gparams[a] += gz[a];  // the target is an input held in params
    for (int p = 0; p < N; ++p) {
      const int g = s->group ? s->group[p] : -1;
      if (g < 0 || g >= G || !(cnt[g] > 0)) continue;
      for (int a = 0; a < d; ++a) {
        gx[p * d + a] += gz[d + g * d + a] / cnt[g];
        if (gv) gv[p * d + a] += gz[d + G * d + g * d + a] / cnt[g];
      }
    }
    return 0;
  }
  return -1;
}

int oracle_controller_adjoint(const oracle_scene* s, const double* params, int step, const double* x,
                              const double* gact, double* gparams, double* gx) {
  return oracle_controller_adjoint_xv(s, params, step, x, nullptr, gact, gparams, gx, nullptr);
}

// One forward step n -> n+1 (Section III Eqs. 3-10 with gravity and boundary).  Optional
// outputs: grid mass [nodes] and grid velocity v* [nodes][d] after the boundary condition.
int oracle_step(const oracle_scene* s, const double* act, const double* x, const double* v, const double* C,
                const double* F, double* x1, double* v1, double* C1, double* F1, double* grid_m,
                double* grid_v) {
  int d = s->dim, N = s->n_particles, ns = n_stencil(d);
  if (d != 2 && d != 3) return -1;
  Grid g;
  int rc = forward_grid(s, act, x, v, C, F, &g, false);
  if (rc) return rc;
  if (grid_m) std::memcpy(grid_m, g.m.data(), sizeof(double) * g.m.size());
  if (grid_v) std::memcpy(grid_v, g.vstar.data(), sizeof(double) * g.vstar.size());
  double Dinv = 4.0 / (s->dx * s->dx);
  // G2P (Eqs. 7-10)
  for (int p = 0; p < N; ++p) {
    Stencil st;
    make_stencil(s, x + p * d, &st);
    double vn[3] = {0, 0, 0};
    M3 Cn = zero3();
    for (int e = 0; e < ns; ++e) {
      int k[3], idx[3];
      stencil_offset(e, d, k);
      for (int a = 0; a < d; ++a) idx[a] = st.base[a] + k[a];
      double N_, dN[3];
      weight(st, d, e, &N_, dN);
      int lin = node_index(s, idx);
      double dpos[3];
      for (int a = 0; a < d; ++a) dpos[a] = idx[a] * s->dx - x[p * d + a];
      for (int a = 0; a < d; ++a) {
        double vi = g.vstar[size_t(lin) * d + a];
        vn[a] += N_ * vi;
        for (int b = 0; b < d; ++b) Cn.a[a][b] += Dinv * N_ * vi * dpos[b];
      }
    }
    M3 Fo = load_mat(F + p * d * d, d);
    M3 A = zero3();
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) A.a[i][j] = (i == j ? 1.0 : 0.0) + s->dt * Cn.a[i][j];
    M3 Fn = matmul(A, Fo, d);
    for (int a = 0; a < d; ++a) {
      v1[p * d + a] = vn[a];
      x1[p * d + a] = x[p * d + a] + s->dt * vn[a];
    }
    store_mat(C1 + p * d * d, Cn, d);
    store_mat(F1 + p * d * d, Fn, d);
  }
  return 0;
}

// One reverse step.  Given state n and the adjoints of state n+1 (gx1, gv1, gC1, gF1: total
// derivatives of the loss with respect to x, v, C, F of step n+1), writes the adjoints of
// state n and gact[g] = dL/da_g(t_n).  Letters refer to the supplement.
//
// Material gradients (optional gE, gm, per particle, this step's contribution): E_p enters only P
// through mu_p and lambda_p, so dL/dE_p = (F - F^{-T}) : Pbar dmu/dE + ln J (F^{-T} : Pbar)
// dlambda/dE with Pbar of (G); m_p enters only P2G (Eqs. 3, 4: m_i, and p_i through m v_p and
// the m C_p term of G), so dL/dm_p = sum_i N_ip (mbar_i + pbar_i . (v_p + C_p (x_i - x_p))).
int oracle_step_adjoint_mat(const oracle_scene* s, const double* act, const double* x, const double* v,
                            const double* C, const double* F, const double* gx1, const double* gv1,
                            const double* gC1, const double* gF1, double* gx0, double* gv0, double* gC0,
                            double* gF0, double* gact, double* gE, double* gm_p) {
  int d = s->dim, N = s->n_particles, nn = n_nodes(s), ns = n_stencil(d);
  if (d != 2 && d != 3) return -1;
  double dmu_dE, dla_dE;
  lame_E(1.0, s->nu, &dmu_dE, &dla_dE);
  Grid g;
  int rc = forward_grid(s, act, x, v, C, F, &g, true);
  if (rc) return rc;
  double Dinv = 4.0 / (s->dx * s->dx);
  double kG = -Dinv * s->dt * s->p_vol;
  // (A) vbar' = dL/dv^{n+1} + dt dL/dx^{n+1};  (B) Cbar' = dL/dC^{n+1} + dt dL/dF^{n+1} F^{nT}
  std::vector<double> vb(size_t(N) * d);
  std::vector<M3> Cb(N);
  for (int p = 0; p < N; ++p) {
    for (int a = 0; a < d; ++a) vb[p * d + a] = gv1[p * d + a] + s->dt * gx1[p * d + a];
    M3 Fo = load_mat(F + p * d * d, d);
    M3 gF = load_mat(gF1 + p * d * d, d);
    M3 gFFt = matmul(gF, transpose(Fo, d), d);
    M3 gC = load_mat(gC1 + p * d * d, d);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) Cb[p].a[i][j] = gC.a[i][j] + s->dt * gFFt.a[i][j];
  }
  // (C) vbar*_i = sum_p N [vbar'_p + Dinv Cbar'_p (x_i - x_p)]
  std::vector<double> gvs(size_t(nn) * d, 0.0);
  for (int p = 0; p < N; ++p) {
    Stencil st;
    make_stencil(s, x + p * d, &st);
    for (int e = 0; e < ns; ++e) {
      int k[3], idx[3];
      stencil_offset(e, d, k);
      for (int a = 0; a < d; ++a) idx[a] = st.base[a] + k[a];
      double N_, dN[3];
      weight(st, d, e, &N_, dN);
      int lin = node_index(s, idx);
      double dpos[3];
      for (int a = 0; a < d; ++a) dpos[a] = idx[a] * s->dx - x[p * d + a];
      for (int a = 0; a < d; ++a) {
        double t = vb[p * d + a];
        for (int b = 0; b < d; ++b) t += Dinv * Cb[p].a[a][b] * dpos[b];
        gvs[size_t(lin) * d + a] += N_ * t;
      }
    }
  }
  // (L) boundary adjoint, gravity is additive so vbar_raw = vbar_g; (D) pbar = vbar_raw / m;
  // (E) mbar = -(v_raw . vbar_raw) / m; all zero on inactive nodes (m_i = 0).
  std::vector<double> gp(size_t(nn) * d, 0.0), gm(nn, 0.0);
  for (int lin = 0; lin < nn; ++lin) {
    if (!(g.m[lin] > 0.0)) continue;
    int idx[3];
    node_coords(s, lin, idx);
    double gin[3];
    bc_adjoint(s, idx, g.tape[lin], &gvs[size_t(lin) * d], gin);
    double dotv = 0;
    for (int a = 0; a < d; ++a) {
      gp[size_t(lin) * d + a] = gin[a] / g.m[lin];
      dotv += g.vraw[size_t(lin) * d + a] * gin[a];
    }
    gm[lin] = -dotv / g.m[lin];
  }
  for (int gi = 0; gi < s->n_groups; ++gi) gact[gi] = 0.0;
  // Backward G2P: (F) (G) (H) (I) (J) (K)
  for (int p = 0; p < N; ++p) {
    Stencil st;
    make_stencil(s, x + p * d, &st);
    ParticleP2G q;
    particle_stress(s, act, p, F + p * d * d, C + p * d * d, &q);
    const double mp = mass_of(s, p);
    double mu, la;
    lame_of(s, p, &mu, &la);
    const M3 Cp = load_mat(C + p * d * d, d);
    double gmass = 0.0;  // dL/dm_p of this step
    double gvp[3] = {0, 0, 0}, gxp[3] = {0, 0, 0};
    M3 Gbar = zero3();
    M3 Cn = zero3();  // C^{n+1}, recomputed for (H)
    for (int e = 0; e < ns; ++e) {
      int k[3], idx[3];
      stencil_offset(e, d, k);
      for (int a = 0; a < d; ++a) idx[a] = st.base[a] + k[a];
      double N_, dN[3];
      weight(st, d, e, &N_, dN);
      int lin = node_index(s, idx);
      double dpos[3];
      for (int a = 0; a < d; ++a) dpos[a] = idx[a] * s->dx - x[p * d + a];
      const double* vs = &g.vstar[size_t(lin) * d];
      const double* pb = &gp[size_t(lin) * d];
      double mb = gm[lin];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Cn.a[a][b] += Dinv * N_ * vs[a] * dpos[b];
      // (F)
      for (int a = 0; a < d; ++a) gvp[a] += N_ * mp * pb[a];
      // m_p in m_i and in p_i = N (m_p v_p + m_p C_p (x_i - x_p) + stress term)
      double pvc = 0;
      for (int a = 0; a < d; ++a) {
        double Cd = 0;
        for (int b = 0; b < d; ++b) Cd += Cp.a[a][b] * dpos[b];
        pvc += pb[a] * (v[p * d + a] + Cd);
      }
      gmass += N_ * (mb + pvc);
      // Gbar = sum_i N pbar_i (x_i - x_p)^T, shared by (G), (H), (I)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Gbar.a[a][b] += N_ * pb[a] * dpos[b];
      // (J) with dN = dN/dx_p
      double vbv = 0;  // vbar' . v*_i
      for (int a = 0; a < d; ++a) vbv += vb[p * d + a] * vs[a];
      double vCd = 0;  // v*_i^T Cbar' (x_i - x_p)
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) vCd += vs[a] * Cb[p].a[a][b] * dpos[b];
      double pmom = 0;  // pbar_i . (m v_p + G (x_i - x_p))
      for (int a = 0; a < d; ++a) {
        double Gd = 0;
        for (int b = 0; b < d; ++b) Gd += q.G.a[a][b] * dpos[b];
        pmom += pb[a] * (mp * v[p * d + a] + Gd);
      }
      for (int al = 0; al < d; ++al) {
        double CtV = 0, GtP = 0;
        for (int b = 0; b < d; ++b) {
          CtV += Cb[p].a[b][al] * vs[b];
          GtP += q.G.a[b][al] * pb[b];
        }
        gxp[al] += dN[al] * vbv + Dinv * (-N_ * CtV + dN[al] * vCd) + dN[al] * pmom - N_ * GtP +
                   mp * mb * dN[al];
      }
    }
    // (I) Cbar = m Gbar
    M3 gCp = zero3();
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) gCp.a[a][b] = mp * Gbar.a[a][b];
    // (G) Pbar = -Dinv dt V0 Gbar F
    M3 GF = matmul(Gbar, q.F, d);
    M3 Pbar = zero3();
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) Pbar.a[a][b] = kG * GF.a[a][b];
    // (H) Fbar = (I + dt C^{n+1})^T Fbar' + H_psi[Pbar] + Pbar sigma^T + kG Gbar^T P
    M3 A = zero3();
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) A.a[i][j] = (i == j ? 1.0 : 0.0) + s->dt * Cn.a[i][j];
    M3 gFn = load_mat(gF1 + p * d * d, d);
    M3 t1 = matmul(transpose(A, d), gFn, d);
    M3 t2 = neohookean_hessian_apply(q.F, Pbar, d, mu, la);
    if (gE) {  // dP/dmu = F - F^{-T}, dP/dlambda = ln J F^{-T}
      M3 FinvT = transpose(inverse(q.F, d), d);
      double gmu = 0, gla = 0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          gmu += (q.F.a[a][b] - FinvT.a[a][b]) * Pbar.a[a][b];
          gla += FinvT.a[a][b] * Pbar.a[a][b];
        }
      gla *= std::log(q.J);
      gE[p] = gmu * dmu_dE + gla * dla_dE;
    }
    if (gm_p) gm_p[p] = gmass;
    M3 t3 = matmul(Pbar, transpose(q.sig, d), d);
    M3 t4 = matmul(transpose(Gbar, d), q.P, d);
    M3 gFp = zero3();
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) gFp.a[a][b] = t1.a[a][b] + t2.a[a][b] + t3.a[a][b] + kG * t4.a[a][b];
    // (K) sigbar = F^T Pbar; a_g enters sigma as a_g * Diag(dir_g)
    int gi = s->group ? s->group[p] : -1;
    if (gi >= 0 && gi < s->n_groups) {
      M3 sb = matmul(transpose(q.F, d), Pbar, d);
      double acc = 0;
      for (int a = 0; a < d; ++a) acc += s->act_dir[gi * d + a] * sb.a[a][a];
      gact[gi] += acc;
    }
    for (int a = 0; a < d; ++a) {
      gv0[p * d + a] = gvp[a];
      gx0[p * d + a] = gx1[p * d + a] + gxp[a];
    }
    store_mat(gC0 + p * d * d, gCp, d);
    store_mat(gF0 + p * d * d, gFp, d);
  }
  return 0;
}

int oracle_step_adjoint(const oracle_scene* s, const double* act, const double* x, const double* v,
                        const double* C, const double* F, const double* gx1, const double* gv1,
                        const double* gC1, const double* gF1, double* gx0, double* gv0, double* gC0,
                        double* gF0, double* gact) {
  return oracle_step_adjoint_mat(s, act, x, v, C, F, gx1, gv1, gC1, gF1, gx0, gv0, gC0, gF0, gact, nullptr,
                                 nullptr);
}

// Forward rollout storing every state (the paper's "memo" of Section III): xs [(T+1)][N][d],
// vs, Cs, Fs likewise, acts [T][G].  Step n uses a(t_n) from the controller evaluated on x_n.
int oracle_rollout(const oracle_scene* s, const double* params, int n_steps, const double* x0,
                   const double* v0, const double* C0, const double* F0, double* xs, double* vs,
                   double* Cs, double* Fs, double* acts) {
  int d = s->dim, N = s->n_particles, G = s->n_groups;
  size_t sx = size_t(N) * d, sm = size_t(N) * d * d;
  std::memcpy(xs, x0, sizeof(double) * sx);
  std::memcpy(vs, v0, sizeof(double) * sx);
  std::memcpy(Cs, C0, sizeof(double) * sm);
  std::memcpy(Fs, F0, sizeof(double) * sm);
  std::vector<double> act(G > 0 ? G : 1, 0.0);
  for (int n = 0; n < n_steps; ++n) {
    int rc = oracle_controller_xv(s, params, n, xs + n * sx, vs + n * sx, act.data());
    if (rc) return rc;
    for (int g = 0; g < G; ++g) acts[size_t(n) * G + g] = act[g];
    rc = oracle_step(s, act.data(), xs + n * sx, vs + n * sx, Cs + n * sm, Fs + n * sm, xs + (n + 1) * sx,
                     vs + (n + 1) * sx, Cs + (n + 1) * sm, Fs + (n + 1) * sm, nullptr, nullptr);
    if (rc) return rc;
  }
  return 0;
}

// Rollout-level chain rule (Section III): from seeds on the final state to the adjoints of the
// initial state and of the controller parameters, which are used at every step.
// With gE, gm: dL/dE_p and dL/dm_p summed over every step (the material is the same at all steps).
int oracle_backward_mat(const oracle_scene* s, const double* params, int n_params, int n_steps,
                        const double* xs, const double* vs, const double* Cs, const double* Fs,
                        const double* acts, const double* gxT, const double* gvT, const double* gCT,
                        const double* gFT, double* gx0, double* gv0, double* gC0, double* gF0,
                        double* gparams, double* gE, double* gm) {
  int d = s->dim, N = s->n_particles, G = s->n_groups;
  size_t sx = size_t(N) * d, sm = size_t(N) * d * d;
  std::vector<double> ax(sx, 0.0), av(sx, 0.0), aC(sm, 0.0), aF(sm, 0.0);
  if (gxT) std::memcpy(ax.data(), gxT, sizeof(double) * sx);
  if (gvT) std::memcpy(av.data(), gvT, sizeof(double) * sx);
  if (gCT) std::memcpy(aC.data(), gCT, sizeof(double) * sm);
  if (gFT) std::memcpy(aF.data(), gFT, sizeof(double) * sm);
  for (int i = 0; i < n_params; ++i) gparams[i] = 0.0;
  for (int p = 0; p < N && gE; ++p) gE[p] = 0.0;
  for (int p = 0; p < N && gm; ++p) gm[p] = 0.0;
  std::vector<double> bx(sx), bv(sx), bC(sm), bF(sm), gact(G > 0 ? G : 1), sE(gE ? N : 0), sm_(gm ? N : 0);
  for (int n = n_steps - 1; n >= 0; --n) {
    int rc = oracle_step_adjoint_mat(s, acts + size_t(n) * G, xs + n * sx, vs + n * sx, Cs + n * sm,
                                     Fs + n * sm, ax.data(), av.data(), aC.data(), aF.data(), bx.data(),
                                     bv.data(), bC.data(), bF.data(), gact.data(), gE ? sE.data() : nullptr,
                                     gm ? sm_.data() : nullptr);
    if (rc) return rc;
    for (int p = 0; p < N && gE; ++p) gE[p] += sE[p];
    for (int p = 0; p < N && gm; ++p) gm[p] += sm_[p];
    rc = oracle_controller_adjoint_xv(s, params, n, xs + n * sx, vs + n * sx, gact.data(), gparams, bx.data(),
                                      bv.data());
    if (rc) return rc;
    ax.swap(bx);
    av.swap(bv);
    aC.swap(bC);
    aF.swap(bF);
  }
  std::memcpy(gx0, ax.data(), sizeof(double) * sx);
  std::memcpy(gv0, av.data(), sizeof(double) * sx);
  std::memcpy(gC0, aC.data(), sizeof(double) * sm);
  std::memcpy(gF0, aF.data(), sizeof(double) * sm);
  return 0;
}

int oracle_backward(const oracle_scene* s, const double* params, int n_params, int n_steps,
                    const double* xs, const double* vs, const double* Cs, const double* Fs,
                    const double* acts, const double* gxT, const double* gvT, const double* gCT,
                    const double* gFT, double* gx0, double* gv0, double* gC0, double* gF0,
                    double* gparams) {
  return oracle_backward_mat(s, params, n_params, n_steps, xs, vs, Cs, Fs, acts, gxT, gvT, gCT, gFT, gx0, gv0,
                             gC0, gF0, gparams, nullptr, nullptr);
}

// Constitutive helpers exposed for the constitutive pins: P(F) and H_psi[Pbar].
int oracle_neohookean(int d, double E, double nu, const double* F, const double* Pbar, double* P,
                      double* HP) {
  oracle_scene s;
  std::memset(&s, 0, sizeof(s));
  s.dim = d;
  s.E = E;
  s.nu = nu;
  double mu, la;
  lame(&s, &mu, &la);
  M3 Fm = load_mat(F, d);
  if (!(det(Fm, d) > 0)) return -4;
  if (P) store_mat(P, neohookean_P(Fm, d, mu, la), d);
  if (HP && Pbar) store_mat(HP, neohookean_hessian_apply(Fm, load_mat(Pbar, d), d, mu, la), d);
  return 0;
}

// Boundary projection of one node velocity and its adjoint (for the S5 pins).
int oracle_bc(const oracle_scene* s, const int* idx, const double* vin, double* vout, const double* gout,
              double* gin) {
  BCTape tape;
  bc_forward(s, idx, vin, vout, &tape);
  if (gout && gin) bc_adjoint(s, idx, tape, gout, gin);
  return 0;
}

}  // extern "C"
