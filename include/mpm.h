/*
 * mpm.h - C ABI of libgbmpm: the differentiable MLS-MPM time step of ChainQueen
 * (Hu et al., arXiv 1810.01054) on hand-written sm_103a CUDA kernels.
 *
 * One explicit step n -> n+1 (Section III, Eqs. 3-10):
 *   P2G    m_i = sum_p N_ip m_p,  p_i = sum_p N_ip [m_p v_p + G_p (x_i - x_p)],
 *          G_p = -(4/dx^2) dt V_p^0 P_p F_p^T + m_p C_p,  P_p = P(F_p) + F_p sigma_a
 *   grid   v_i = p_i / m_i, then gravity and the boundary condition (sticky or slip, Supplement S5)
 *   G2P    v_p = sum_i N_ip v_i,  C_p = (4/dx^2) sum_i N_ip v_i (x_i - x_p)^T,
 *          F_p <- (I + dt C_p) F_p,  x_p <- x_p + dt v_p
 * with N the quadratic B-spline, P(F) the compressible neo-Hookean stress and sigma_a the
 * actuation stress a_g(t) Diag(dir_g) of the particle's group g.  The reverse pass implements
 * Supplement S2-S5, (A)-(L), chained over a whole rollout (Section III, "memo").
 *
 * Conventions for every entry point:
 *  - Every function returns mpm_status (0 = OK, < 0 = error); nothing throws or aborts across
 *    the ABI.  Work is enqueued on the context's stream (a reverse pass's segment recompute and a
 *    batch's reverse half run on a private second stream, always joined back into the context's
 *    stream before the call returns; the CUDA graphs a scene replays may branch inside, but each
 *    completes as one unit in the context stream's order); device-side errors (a stencil leaving
 *    the grid, det F <= 0, a tile over capacity) are recorded in the scene's status word, first
 *    error wins, and reported by the next synchronising call (mpm_sync, mpm_get_state,
 *    mpm_backward).  A scene with a recorded error keeps it until mpm_set_state.
 *  - Arrays are row-major and FP32: positions and velocities [N][dim], C and F [N][dim][dim],
 *    particle order as given at creation (results come back in the same order).
 *  - mem_space 0 = host pointers, 1 = device pointers (e.g. torch tensors' data_ptr()).  Inputs
 *    are copied; the caller keeps ownership of everything it passes in and of every output buffer.
 *  - Node i of the grid sits at i*dx, i in [0, n) per axis.  A particle whose quadratic stencil
 *    would leave [0, n) is an error, never clamped.
 */
#ifndef GBMPM_MPM_H_
#define GBMPM_MPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPM_OK = 0,
  MPM_ERR_ARG = -1,      /* invalid argument or descriptor */
  MPM_ERR_OOM = -2,      /* device allocation failed or memory budget too small */
  MPM_ERR_DOMAIN = -3,   /* a particle's stencil left the grid */
  MPM_ERR_INVERTED = -4, /* det F <= 0 (neo-Hookean undefined) */
  MPM_ERR_TIMEOUT = -5,  /* a bounded device wait ran out */
  MPM_ERR_CUDA = -6,     /* a CUDA call failed */
  MPM_ERR_STATE = -7,    /* call out of order (e.g. backward without a rollout) */
  MPM_ERR_DENSITY = -8,  /* more particles in one cell tile than the tile kernels stage: 2048 in a
                            4x4 tile (2D), 4096 in a 4x4x4 tile (3D) */
  MPM_ERR_INTERNAL = -9  /* a kernel's own consistency check failed (a particle binned to the wrong
                            tile); the offending access was skipped */
} mpm_status;

typedef struct mpm_ctx mpm_ctx;
typedef struct mpm_scene mpm_scene;
typedef struct mpm_batch mpm_batch;

/* Creates a context on CUDA device `device`, enqueuing on `cuda_stream` (a cudaStream_t; NULL
 * creates a private non-blocking stream). */
mpm_status mpm_ctx_create(mpm_ctx** out, int device, void* cuda_stream);
/* Destroys the context.  Every scene and batch created on it must be destroyed first:
 * MPM_ERR_STATE (and nothing freed) while any is alive. */
mpm_status mpm_ctx_destroy(mpm_ctx* ctx);
/* Waits for the context's stream; returns the first CUDA error seen. */
mpm_status mpm_sync(mpm_ctx* ctx);
const char* mpm_status_str(mpm_status s);

/* Controller families (Section V-B uses a = tanh(W z + b); these are its forms here):
 *  MPM_CTRL_SIN   a_g(t) = A_g sin(2 pi f t)                               params [G]
 *  MPM_CTRL_BASIS a_g(t) = sum_j W_gj b_j(t), b = [sin 2pi f t, cos 2pi f t, sin 4pi f t, cos 4pi f t]
 *                                                                          params [G][4]
 *  MPM_CTRL_MLP   z = centroid_g(x) - centroid_all(x) for every group (G*dim inputs),
 *                 a = scale * tanh(W3 tanh(W2 tanh(W1 z + b1) + b2) + b3)  params W1[H][G*dim], b1[H],
 *                                                                          W2[H][H], b2[H], W3[G][H], b3[G]
 *  MPM_CTRL_TABLE every step's actuation is a decision variable (the trajectory-optimisation
 *                 examples, Section V-C): a_g(t_n) = U[n][g] for steps 0 <= n < L, 0 after
 *                                                                          params U[L][G], L = ctrl_hidden
 *  MPM_CTRL_COM   the closed-loop controller of Section V-B: a = scale * tanh(W z + b) with
 *                 z = [target, c_1..c_G, u_1..u_G], c_g and u_g the means of x and v over group g
 *                 (0 for an empty group)                                  params target[dim],
 *                                                                          W[G][dim (1 + 2G)], b[G]
 *                 (the gradient includes dL/dtarget; the reverse pass adds dL/dx and dL/dv through
 *                 the group means)
 * with t = n * dt at the start of step n (n the scene's step counter). */
enum { MPM_CTRL_SIN = 0, MPM_CTRL_BASIS = 1, MPM_CTRL_MLP = 2, MPM_CTRL_TABLE = 3, MPM_CTRL_COM = 4 };
enum { MPM_BC_STICKY = 0, MPM_BC_SLIP = 1, MPM_BC_OPEN = 2 /* per wall only (mpm_scene_set_walls) */ };
enum { MPM_IMPL_TILED = 0, MPM_IMPL_PLAIN = 1 };

typedef struct {
  int dim;             /* 2 or 3 */
  int n_grid[3];       /* nodes per axis (only the first dim used), each >= 5 */
  float dx, dt;        /* cell size, time step; dt <= dx sqrt(rho/E) is required (Section VI) */
  float gravity[3];
  float E, nu;         /* Young's modulus > 0, Poisson ratio in (-1, 0.5) */
  float p_mass, p_vol; /* m_p and V_p^0 of every particle (> 0) */
  int bc_type;         /* MPM_BC_STICKY: v* = 0 on band nodes; MPM_BC_SLIP: S5 projection, friction c */
  int bc_width;        /* band = nodes with an axis index < bc_width or >= n - bc_width */
  float friction_c;    /* Coulomb coefficient c of S5 (slip only) */
  int n_particles;     /* 0 <= N < 2^26 */
  const float* x0;     /* [N][dim] */
  const float* v0;     /* [N][dim], NULL = 0 */
  const float* C0;     /* [N][dim][dim], NULL = 0 */
  const float* F0;     /* [N][dim][dim], NULL = identity */
  const int32_t* group;/* [N] actuation group of every particle, -1 = none; NULL = all -1 */
  int n_groups;        /* 0 <= G <= 64 */
  const float* act_dir;/* [G][dim] actuation direction: sigma_a = a_g Diag(dir_g) */
  int ctrl_type;       /* MPM_CTRL_* */
  int ctrl_hidden;     /* MLP width H <= 128 (MLP; G*dim <= 192); table length L >= 0 (TABLE) */
  float ctrl_freq;     /* f of the sinusoid forms */
  float ctrl_scale;    /* output scale of the MLP */
  int n_ctrl_params;   /* must equal the family's parameter count above */
  const float* ctrl_params;
  int impl;            /* MPM_IMPL_TILED (sorted, deterministic) or MPM_IMPL_PLAIN (atomics baseline) */
  int mem_space;       /* where every pointer of this descriptor lives */
  int tile_edge;       /* cells per tile edge of the tiled form: 4; 8 (2D only: sparse scenes, a tile
                          then holds the particles of four 4 x 4 tiles); 0 = chosen at creation
                          (2D: the edge mpm_tune_tile_edge cached for the workload, else 8 x 8 for
                          a scene averaging under 96 particles per occupied 4 x 4 tile, else
                          4 x 4) */
} mpm_scene_desc;

/* Creates a scene (Section III state: x, v, C, F per particle; grid per desc) at step 0.  Copies
 * every input; the library owns the scene's device buffers until mpm_scene_destroy.
 * The tiled form stores the particles in an order of its own (by tile, cell and position of the
 * initial state), so its kernels read neighbouring memory whatever order the caller's arrays
 * have, and the same particles given in another order give the same result bits.  Every
 * per-particle array passed to or returned by any entry point is in the caller's order. */
mpm_status mpm_scene_create(mpm_ctx* ctx, const mpm_scene_desc* desc, mpm_scene** out);
mpm_status mpm_scene_destroy(mpm_scene* scene);
/* Cells per tile edge the scene was created with (4 or 8). */
mpm_status mpm_scene_tile_edge(const mpm_scene* scene, int* edge);

/* Advances the current state by n_steps steps (Eqs. 3-10 with the controller's actuation),
 * asynchronously on the context stream.  Keeps no history. */
mpm_status mpm_step(mpm_scene* scene, int n_steps);

/* Rollout for differentiation (Section III "memo"): n_steps steps from the current state,
 * asynchronously; the checkpoint buffers are kept for the next rollout of the same shape.
 * storing the state every ckpt_interval steps (0 = choose from mem_budget_bytes: every step if
 * all states fit; else, in the tiled form, the smallest interval whose checkpoints, two sets of
 * recompute buffers and the sorts an overlapped reverse pass keeps all fit, so that the fewest
 * steps are recomputed and the recompute runs beside the reverse steps; else about sqrt(n_steps);
 * mpm_scene_plan_rollout reports the choice); the states in between are recomputed by
 * mpm_backward.  mem_budget_bytes = 0 means no
 * limit.
 * With ckpt_interval = 0 and a budget below that single-level store ((ceil(T/k) + k - 1) states),
 * the rollout keeps a multi-level store instead: a recursive schedule (store a state, reverse the
 * later part, release it, reverse the earlier part) planned for the fewest recomputed steps within
 * floor(budget / state size) states, at least 3 (the first and final states and one more), for
 * rollouts of up to 8192 steps; mpm_plan_checkpoints reports its cost.  Its gradients are the same
 * bits as the single-level store's.  Such a rollout supports one mpm_backward, and mpm_get_state
 * of a stored step returns MPM_ERR_STATE.  MPM_ERR_OOM when neither store fits the budget. */
mpm_status mpm_rollout(mpm_scene* scene, int n_steps, int ckpt_interval, size_t mem_budget_bytes);

/* The schedule of a budget counted in whole states only (budget_states = budget / state size; 0 =
 * no limit): every state when they fit, else the single-level store at about sqrt(n_steps), else
 * the multi-level store.  Reports the forward steps run over the rollout and its reverse pass
 * together (n_steps when every state is kept; the reverse steps themselves are n_steps in every
 * schedule), the number of states stored at most, and whether the multi-level store is used (NULL
 * outputs are skipped).  MPM_ERR_OOM when no schedule fits.  Host only.  This is the schedule of
 * mpm_rollout with ckpt_interval 0 for the multi-level store and for the plain form; a tiled
 * scene's single-level interval also counts the overlap's stores: mpm_scene_plan_rollout. */
mpm_status mpm_plan_checkpoints(int n_steps, long long budget_states, long long* forward_steps, int* states_used,
                                int* multi_level);
/* What mpm_rollout(scene, n_steps, ckpt_interval, mem_budget_bytes) would do: *k_out the interval
 * of its single-level store (0 with the multi-level store), *forward_steps the forward steps of
 * the rollout and its reverse pass together, *multi_level 1 for the multi-level store (NULL
 * outputs are skipped).  MPM_ERR_OOM when the given interval's store, or every store, exceeds
 * the budget; MPM_ERR_ARG for n_steps < 1 or ckpt_interval < 0.  Host only (no GPU work). */
mpm_status mpm_scene_plan_rollout(const mpm_scene* scene, int n_steps, int ckpt_interval, size_t mem_budget_bytes,
                                  int* k_out, long long* forward_steps, int* multi_level);

/* Reverse pass of the last rollout (Supplement S2-S5 at every step, chained to the first state
 * and to the controller parameters used at every step).  Seeds are dL/d(final x, v, C, F)
 * (NULL = 0); outputs are dL/d(initial x, v, C, F) and dL/d(controller params) (NULL = not
 * wanted).  Synchronises; returns the scene's first device error. */
mpm_status mpm_backward(mpm_scene* scene, const float* gx_T, const float* gv_T, const float* gC_T,
                        const float* gF_T, float* gx0, float* gv0, float* gC0, float* gF0,
                        float* g_ctrl_params, int mem_space);

/* Result of the last finished reverse pass (mpm_backward, or a batched gradient request): dL/d
 * of the rollout's first x, v, C, F and of the controller parameters (NULL = not wanted).
 * Synchronises; MPM_ERR_STATE if no reverse pass has finished since the last rollout. */
mpm_status mpm_get_gradients(mpm_scene* scene, float* gx0, float* gv0, float* gC0, float* gF0, float* g_ctrl_params,
                             int mem_space);
/* Copies the state out (step -1 = current, else a checkpointed step of the last rollout).
 * Synchronises; returns the scene's first device error. */
mpm_status mpm_get_state(mpm_scene* scene, int step, float* x, float* v, float* C, float* F, int mem_space);
/* Replaces the current state (NULL C = 0, NULL F = I, NULL v = 0) and clears the error status;
 * optionally sets the step counter (step >= 0) that drives the controller's time.  Asynchronous:
 * non-finite inputs are reported (MPM_ERR_ARG) by the next synchronising call. */
mpm_status mpm_set_state(mpm_scene* scene, const float* x, const float* v, const float* C, const float* F,
                         int step, int mem_space);
/* Replaces the controller parameters (n must equal the scene's parameter count). */
mpm_status mpm_set_ctrl_params(mpm_scene* scene, const float* params, int n, int mem_space);
/* Per-particle material (an extension: the paper's co-design and inference examples treat
 * material parameters as optimisation variables, Sections V-A and V-C).  E [N] Young's modulus and
 * mass [N] per particle replace the descriptor's E and p_mass (NULL keeps the scene's value for
 * every particle; both NULL returns to the uniform scene); nu and V^0 stay per scene.  Values must
 * be finite and positive, and dt must satisfy dt <= dx sqrt(rho_p / E_p) for every particle
 * (rho_p = m_p / V^0), else MPM_ERR_ARG and nothing changes.  Synchronises.  Invalidates an
 * earlier rollout (run mpm_rollout again).  While per-particle material is set, mpm_backward also
 * accumulates dL/dE_p and dL/dm_p over every reverse step:
 *   dL/dE_p  = sum_n (F - F^-T) : Pbar dmu/dE + ln J (F^-T : Pbar) dlambda/dE   (Pbar of S4 (G))
 *   dL/dm_p  = sum_n sum_i N_ip (mbar_i + pbar_i . (v_p + C_p (x_i - x_p)))   (S3 (D), (E))
 * read with mpm_get_material_gradients (MPM_ERR_STATE without material or without a finished
 * reverse pass; outputs on the host or the device per mem_space; NULL skips one). */
mpm_status mpm_scene_set_material(mpm_scene* scene, const float* E, const float* mass, int mem_space);
mpm_status mpm_get_material_gradients(mpm_scene* scene, float* gE, float* gm, int mem_space);
/* Per-wall boundary (Supplement S5's friction projection on selected walls).  Wall w = 2a + side
 * (axis a, side 0 = low) gets kind[w] (MPM_BC_STICKY, MPM_BC_SLIP with Coulomb friction c[w] >= 0,
 * or MPM_BC_OPEN) for w < 2 dim; the band depth stays bc_width.  A node in a sticky wall's band is
 * fixed; otherwise the slip walls whose band contains it are applied in sequence (axis 0, 1, 2, low
 * side first), each with its own c; open walls constrain nothing (a particle whose stencil then
 * leaves the grid is MPM_ERR_DOMAIN as always).  NULL kind or c keeps the current values.
 * Synchronises; invalidates an earlier rollout.  MPM_ERR_ARG (and nothing changes) for an unknown
 * kind or a negative or non-finite c. */
mpm_status mpm_scene_set_walls(mpm_scene* scene, const int* kind, const float* c);
/* Grid of the last forward step: mass m_i [nodes] and velocity v*_i [nodes][dim] after the
 * boundary condition (nodes never touched by a particle hold stale values for the tiled form). */
mpm_status mpm_get_grid(mpm_scene* scene, float* m, float* v, int mem_space);
/* Sizes: particles, groups, controller parameters, current step; bytes of one stored state. */
mpm_status mpm_scene_info(const mpm_scene* scene, int* n_particles, int* n_groups, int* n_ctrl_params,
                          int* step, size_t* state_bytes);

/* Batched execution: scenes of one dimension advanced together by the same persistent launches
 * (one scene table, per-scene offsets).  A batch holds references to scenes it does not own.
 *  mpm_batch_create   empty batch of dimension dim on ctx, admitting scenes while their device
 *                     memory fits mem_budget (0 = no limit)
 *  mpm_batch_admit    adds a scene that will run n_steps more steps (and, with want_grad, its
 *                     reverse pass, seeded by loss = mean of final x_0); *slot = -1 if full.
 *                     The scenes of a batch share one tile edge: the first admitted scene sets
 *                     it until the batch is empty again; a scene of another edge is refused
 *                     with MPM_ERR_ARG (keep a batch per dimension and tile edge)
 *  mpm_batch_tick     advances every admitted scene by up to max_steps steps
 *  mpm_batch_poll     *done = 1 when the slot's work is finished (results stay in the scene);
 *                     a request that stopped on a device error (a particle left the grid, a
 *                     tile over capacity) is finished too: *done = 1 and the return value is
 *                     that error, which the scene's own calls also report.  Only that slot
 *                     stops; the other scenes of the batch go on unaffected.  MPM_ERR_ARG for
 *                     a free or out-of-range slot (then *done is left unchanged)
 *  mpm_batch_release  frees a finished slot for the next admission
 * From admission until its slot is released (or the batch destroyed) a scene is driven by the
 * batch: calls that would change it (step, rollout, backward, set_state, set_ctrl_params,
 * set_material, set_walls, set_tuning, destroy) return MPM_ERR_STATE; reading its results is
 * allowed once mpm_batch_poll reports the slot done. */
mpm_status mpm_batch_create(mpm_ctx* ctx, int dim, size_t mem_budget, mpm_batch** out);
mpm_status mpm_batch_destroy(mpm_batch* batch);
mpm_status mpm_batch_admit(mpm_batch* batch, mpm_scene* scene, int n_steps, int want_grad, int* slot);
mpm_status mpm_batch_tick(mpm_batch* batch, int max_steps);
mpm_status mpm_batch_poll(mpm_batch* batch, int slot, int* done);
mpm_status mpm_batch_release(mpm_batch* batch, int slot);

/* Double-precision plain form (an extension for the accuracy study of Section VI, whose case B
 * runs colliding elastic bodies in float64 and checks the adjoint against central finite
 * differences).  The same step (Eqs. 3-10) and reverse pass (Supplement S2-S5, (A)-(L)) in FP64,
 * one thread per particle with atomic scatter: run-to-run results agree to rounding, not bit for
 * bit (the tile form above is the deterministic one).  Scope: uniform material, per-wall boundary,
 * and actuation given per step as a table (the MPM_CTRL_TABLE form: a_g(t_n) = U[n][g] for
 * n < L, 0 after); other controller families and per-particle material stay FP32-only.
 * A rollout always starts from the scene's initial state at step 0 and keeps every state on the
 * device ((T + 1) (2 dim + 2 dim^2) N doubles).  All pointers are host pointers; arrays are
 * row-major and particle-major as in the FP32 API ([N][dim], [N][dim][dim]). */
typedef struct mpm_scene64 mpm_scene64;
typedef struct {
  int dim;               /* 2 or 3 */
  int n_grid[3];         /* nodes per axis, each >= 5 */
  double dx, dt;         /* dt <= dx sqrt(rho / E) (Section VI) */
  double gravity[3];
  double E, nu;          /* Young's modulus > 0, Poisson ratio in (-1, 0.5) */
  double p_mass, p_vol;  /* m_p and V_p^0 of every particle (> 0) */
  int bc_width;          /* band depth of every wall */
  int wall_kind[6];      /* wall w = 2 axis + side: MPM_BC_STICKY, MPM_BC_SLIP or MPM_BC_OPEN */
  double wall_c[6];      /* Coulomb coefficient of each slip wall (>= 0, Supplement S5) */
  int n_particles;       /* 0 <= N < 2^26 */
  const double* x0;      /* [N][dim] */
  const double* v0;      /* [N][dim], NULL = 0 */
  const double* C0;      /* [N][dim][dim], NULL = 0 */
  const double* F0;      /* [N][dim][dim], NULL = identity */
  const int32_t* group;  /* [N] actuation group in [-1, G), NULL = all -1 */
  int n_groups;          /* 0 <= G <= 64 */
  const double* act_dir; /* [G][dim]: sigma_a = a_g Diag(dir_g) */
  int n_act_steps;       /* L >= 0 */
  const double* act;     /* [L][G] actuation table U (may be NULL when L G = 0) */
} mpm_scene64_desc;

/* Creates the scene (copies every input).  MPM_ERR_ARG for an invalid or non-finite input. */
mpm_status mpm64_create(mpm_ctx* ctx, const mpm_scene64_desc* desc, mpm_scene64** out);
mpm_status mpm64_destroy(mpm_scene64* scene);
/* Replaces the initial state (NULL v, C = 0, NULL F = I); drops the stored rollout. */
mpm_status mpm64_set_state(mpm_scene64* scene, const double* x, const double* v, const double* C, const double* F);
/* Replaces the actuation table U [L][G]; drops the stored rollout. */
mpm_status mpm64_set_actuation(mpm_scene64* scene, const double* U, int L);
/* T steps from the initial state, every state kept (asynchronous; MPM_ERR_OOM if they do not
 * fit).  Device errors (a stencil leaving the grid, det F <= 0) are reported by the next
 * mpm64_get_state or mpm64_backward. */
mpm_status mpm64_rollout(mpm_scene64* scene, int n_steps);
/* State at step 0..T of the last rollout (-1 = T); NULL skips an output.  Synchronises. */
mpm_status mpm64_get_state(mpm_scene64* scene, int step, double* x, double* v, double* C, double* F);
/* Reverse pass of the last rollout seeded by dL/d(x_T, v_T, C_T, F_T) (NULL = 0): dL/d of the
 * initial x, v, C, F and dL/dU [L][G] (NULL skips one).  Synchronises. */
mpm_status mpm64_backward(mpm_scene64* scene, const double* gx_T, const double* gv_T, const double* gC_T,
                          const double* gF_T, double* gx0, double* gv0, double* gC0, double* gF0, double* g_act);
/* Sizes: particles, groups, actuation steps L, steps of the stored rollout (-1: none). */
mpm_status mpm64_info(const mpm_scene64* scene, int* n_particles, int* n_groups, int* n_act_steps,
                      int* rollout_steps);

/* Instrumentation.  Kernel kinds for timing: */
enum {
  MPM_K_SORT = 0,       /* bin keys, tile histogram, scan, scatter */
  MPM_K_P2G = 1,        /* tiled P2G (forward) */
  MPM_K_GRID = 2,       /* grid normalisation, gravity, boundary */
  MPM_K_G2P = 3,        /* tiled G2P + F, x update */
  MPM_K_P2G_ADJ = 4,    /* P2G recompute fused with the adjoint scatter (A)-(C) */
  MPM_K_GRID_ADJ = 5,   /* grid recompute with (L), (D), (E) */
  MPM_K_ADJ_GATHER = 6, /* adjoint gather (F)-(K), (J) */
  MPM_K_CTRL = 7,       /* controller forward/backward and group reductions */
  MPM_K_PLAIN = 8,      /* the plain (atomic) form's step or reverse step */
  MPM_K_F64_P2G = 9,    /* FP64 form: P2G scatter (forward) */
  MPM_K_F64_GRID = 10,  /* FP64 form: grid update, forward or reverse */
  MPM_K_F64_G2P = 11,   /* FP64 form: G2P */
  MPM_K_F64_P2G_ADJ = 12, /* FP64 form: P2G recompute + adjoint scatter (A)-(C) */
  MPM_K_F64_ADJ = 13,   /* FP64 form: per-particle adjoint (F)-(K), (J) */
  MPM_K_COUNT = 14
};
/* Starts timing every launch of the kinds in `mask` (bit k = kind k) with CUDA events on the
 * context stream, for at most max_launches launches; restarts the tally. */
mpm_status mpm_profile_start(mpm_ctx* ctx, unsigned mask, int max_launches);
/* Synchronises and returns the number of timed launches of `kind` and their summed duration. */
mpm_status mpm_profile_read(mpm_ctx* ctx, int kind, int* count, double* total_ms);
/* Total number of kernels this library has launched in the process (all contexts). */
mpm_status mpm_launch_count(long long* count);

/* Launch-shape autotuning (no counterpart in the paper, whose kernels were launched with fixed
 * shapes on its own GPU).  The four tile kernels -- P2G, G2P, the adjoint scatter and the
 * adjoint gather -- run as persistent grids; how many CTAs per SM each gets (and, for G2P and in 2D
 * for P2G and the adjoint scatter, 128 or 256 threads per CTA) is chosen per workload.  Under MPM_TUNE_AUTO (the default) a scene looks
 * its workload key -- dimension, log2 buckets of its particle and grid-tile counts, SM count -- up
 * in a process-wide cache; on a miss its next steps try every candidate shape of each kernel in
 * turn (two timed launches each, CUDA events, launched directly instead of from graphs), keep
 * the fastest and store it in the cache.  Every tile is processed whole by one CTA, so results
 * are bitwise the same under every shape and the trial steps are ordinary steps.  A batch keys
 * each of its two compositions (scenes in forward steps, scenes in reverse steps) the same way:
 * it takes the cache entry when there is one, else its own steps try the candidates of the kernels
 * that composition runs (the key's entry is complete, and saved, once both halves are tuned).
 * MPM_TUNE_FORCE re-tunes ignoring the cache; MPM_TUNE_OFF uses the default shapes (4 CTAs of
 * 256 threads per SM). */
enum { MPM_TUNE_OFF = 0, MPM_TUNE_AUTO = 1, MPM_TUNE_FORCE = 2 };
/* Tile kernels, for mpm_scene_launch and the cache arrays below (in this order). */
enum { MPM_TK_P2G = 0, MPM_TK_G2P = 1, MPM_TK_P2G_ADJ = 2, MPM_TK_ADJ_GATHER = 3, MPM_TK_COUNT = 4 };
mpm_status mpm_scene_set_tuning(mpm_scene* scene, int mode);
/* Launch shape of tile kernel `kernel` for this scene; *tuned = 1 once it came from the cache or
 * from trials, 0 while it is the default or still being tried. */
mpm_status mpm_scene_launch(const mpm_scene* scene, int kernel, int* ctas_per_sm, int* threads, int* tuned);
/* The process-wide cache.  shape[2k], shape[2k+1] = CTAs per SM and threads of tile kernel k.
 *  mpm_tune_cache_lookup  *found = 1 and shape filled when the key of (dim, particles, grid
 *                         tiles, sm_count) has an entry
 *  mpm_tune_cache_store   sets the entry of that key (shapes are checked against the candidates)
 *  mpm_tune_cache_save    writes every entry to a text file (one line per key)
 *  mpm_tune_cache_load    adds the entries of such a file (MPM_ERR_ARG if it is malformed)
 * None of them touches the GPU.  When the environment variable GBMPM_TUNE_CACHE names a file,
 * it is loaded at the first lookup and rewritten after every tuning that finishes. */
mpm_status mpm_tune_cache_lookup(int dim, long long particles, long long grid_tiles, int sm_count, int* shape,
                                 int* found);
mpm_status mpm_tune_cache_store(int dim, long long particles, long long grid_tiles, int sm_count, const int* shape);
mpm_status mpm_tune_cache_save(const char* path);
mpm_status mpm_tune_cache_load(const char* path);
/* Tile-edge autotuning (particles per tile; no counterpart in the paper).  For a 2D tiled scene
 * described by `desc` it creates the scene with 4 x 4-cell and with 8 x 8-cell tiles in turn, runs
 * each through two untimed and one timed pass of `steps` forward steps (every state kept) and
 * their reverse pass, destroys it, and returns the edge whose pass took less GPU time in *edge and
 * the two passes' milliseconds per step in ms[0] (4 x 4) and ms[1] (8 x 8) (ms may be NULL).  The
 * choice goes into the process-wide cache under the workload's key (dimension, log2 buckets of its
 * particle and grid-node counts, SM count; saved with the launch shapes, as lines
 * "edge dim log2_particles log2_nodes sms tile_edge"), and mpm_scene_create with tile_edge = 0 takes
 * the cached edge for that key before the density rule.  3D scenes and the plain form have one
 * tile shape: *edge = 4 and nothing runs.  The descriptor's pointers are read as for
 * mpm_scene_create; the context stream is used and synchronised.  Errors: MPM_ERR_ARG for a NULL
 * argument, steps < 1 or a descriptor mpm_scene_create refuses; whatever creating, stepping or
 * reversing the trial scenes returns (the cache is then unchanged). */
mpm_status mpm_tune_tile_edge(mpm_ctx* ctx, const mpm_scene_desc* desc, int steps, int* edge, float* ms);

/* Allocation-free forward step (no counterpart in the paper; an addition for callers that must
 * not allocate device memory: a control loop with a hard latency budget, where cudaMalloc may
 * block and synchronise the device, or a process whose device memory is owned entirely by
 * another allocator).
 *
 * One step of the plain form (Eqs. 3-10 with gravity and the boundary condition) from the
 * caller's state arrays to the caller's output arrays, all device pointers, row-major FP32 as
 * everywhere in this header; act[g] is the actuation a_g of this step.  The only scratch, the
 * dense node grid, lives in a fixed array of 2^18 float4 nodes (4 MiB: 512^2 in 2D, 64^3 in 3D)
 * that every GPU loading this library holds until the process exits; larger grids are rejected
 * with MPM_ERR_ARG.  No cudaMalloc, cudaFree or allocating library call is made.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *  - Every call shares the array and clears the part it uses before use; calls whose work
 *    overlaps on the GPU (e.g. on two streams) race on it.
 *  - device < 0 keeps the current device; device >= 0 is made current for the call and the
 *    caller's current device is restored before it returns.  status (device int, may be NULL)
 *    receives the first device-side error as in the rest of this header.
 *  - Arguments are checked as mpm_scene_create checks them (each grid side and the node count
 *    bounded before anything is multiplied or launched; bc_width >= 0, friction_c finite and
 *    >= 0, p_mass > 0, p_vol > 0, the explicit-integration limit on dt): MPM_ERR_ARG.
 *  - MPM_ERR_CUDA when one of its own launches fails; an error left pending by the caller's
 *    earlier work is neither read nor cleared.
 * Asynchronous on cuda_stream (a cudaStream_t, NULL = the legacy default stream). */
typedef struct {
  int device;
  int dim;
  int n_grid[3];
  float dx, dt;
  float gravity[3];
  float E, nu;
  float p_mass, p_vol;
  int bc_type, bc_width;
  float friction_c;
  int n_particles;
  const float* x;        /* [N][dim] */
  const float* v;        /* [N][dim], NULL = 0 */
  const float* C;        /* [N][dim][dim], NULL = 0 */
  const float* F;        /* [N][dim][dim], NULL = identity */
  const int32_t* group;  /* [N], NULL = all -1 */
  int n_groups;
  const float* act_dir;  /* [G][dim] */
  const float* act;      /* [G] */
  float* x_out;
  float* v_out;
  float* C_out;
  float* F_out;
  int* status;
} mpm_noalloc_step;
mpm_status mpm_step_noalloc(const mpm_noalloc_step* args, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GBMPM_MPM_H_ */
