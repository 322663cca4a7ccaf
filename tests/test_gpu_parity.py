"""GPU path (libgbmpm through its C ABI) against the FP64 oracle on the same seeded inputs.

Forward: one step on small 2D/3D scenes (sticky, slip, friction, every controller form, several
tiles, a ragged tail of particles), 10-step re-synced windows over the whole 100-step 64^2 square
workload, and one full-size step of each larger workload.  Reverse: full-horizon gradients of
the 64^2 square workload, gradients of every controller form, and one full-size reverse step.
Both kernel forms (tiled/sorted and plain/atomic) are checked.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import (FWD_TOL, assert_grad_close, assert_state_close, mean_x0_seed, oracle_step_from,
                                rel_l2)

pytestmark = pytest.mark.gpu

IMPLS = [0, 1]  # tiled, plain


@pytest.fixture(scope="module")
def M():
    from paper_1810_01054_gb300 import mpm
    mpm.lib()
    return mpm


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def small_scenes():
    return {
        "2d_sticky": S.blob(2, 32, 300, 1, v_scale=0.5, c_scale=2.0, f_scale=0.05, radius_cells=5.0,
                            center=(0.5, 6.5 / 32), bc_width=3, amp=2.0),
        "3d_sticky": S.blob(3, 24, 700, 2, v_scale=0.5, c_scale=2.0, f_scale=0.05, radius_cells=4.0,
                            center=(0.5, 5.0 / 24, 0.45), bc_width=3, amp=2.0),
        "2d_slip_friction": S.blob(2, 32, 257, 3, v_scale=0.8, bc_type=S.BC_SLIP, friction_c=0.4, bc_width=3,
                                   radius_cells=4.0, center=(0.4, 4.8 / 32), amp=1.0),
        "3d_slip": S.blob(3, 24, 333, 4, v_scale=0.8, bc_type=S.BC_SLIP, friction_c=0.0, bc_width=3,
                          radius_cells=3.5, center=(0.5, 4.5 / 24, 5.0 / 24), amp=1.0),
        "2d_basis": S.blob(2, 32, 200, 5, ctrl_type=S.CTRL_BASIS, n_groups=4, freq=4.0, radius_cells=4.0,
                           v_scale=0.3),
        "3d_mlp": S.blob(3, 16, 400, 6, ctrl_type=S.CTRL_MLP, n_groups=4, hidden=16, scale=5.0, radius_cells=3.5,
                         v_scale=0.3),
        # per-step actuation table (30 rows, longer than the 25-step rollouts below)
        "2d_table": S.blob(2, 32, 300, 7, ctrl_type=S.CTRL_TABLE, n_groups=4, hidden=30, radius_cells=4.5,
                           v_scale=0.3, amp=3.0),
        "3d_table": S.blob(3, 20, 500, 8, ctrl_type=S.CTRL_TABLE, n_groups=3, hidden=30, radius_cells=3.5,
                           v_scale=0.3, amp=3.0),
        # the closed-loop controller on group centres of mass and velocities (some particles in no group)
        "2d_com": _ungroup(S.blob(2, 32, 300, 9, ctrl_type=S.CTRL_COM, n_groups=4, scale=5.0, radius_cells=4.5,
                                  v_scale=0.5)),
        "3d_com": _ungroup(S.blob(3, 20, 500, 10, ctrl_type=S.CTRL_COM, n_groups=3, scale=5.0, radius_cells=3.5,
                                  v_scale=0.5)),
    }


def _ungroup(spec, every=9):
    spec.group[::every] = -1
    return spec


@pytest.mark.parametrize("impl", IMPLS, ids=["tiled", "plain"])
@pytest.mark.parametrize("name", list(small_scenes().keys()))
def test_one_step_forward(M, ctx, name, impl):
    spec = small_scenes()[name]
    gpu = M.Scene(ctx, spec, impl=impl)
    st0 = O.Scene(spec).initial_state()
    # start at step 3 so the sinusoid controllers are non-zero
    gpu.set_state(*st0, step=3)
    gpu.step(1)
    got = gpu.get_state()
    ref = oracle_step_from(spec, st0, 3)
    assert_state_close(got, ref)


@pytest.mark.parametrize("impl", IMPLS, ids=["tiled", "plain"])
def test_walker_square_windows(M, ctx, impl):
    """64^2 grid, 1024 particles, 100 steps: every 10-step window re-synced to the oracle."""
    spec = S.walker_square_2d(0)
    osc = O.Scene(spec)
    xs, vs, Cs, Fs, acts = osc.rollout(100)
    gpu = M.Scene(ctx, spec, impl=impl)
    for w in range(10):
        n0 = 10 * w
        gpu.set_state(xs[n0], vs[n0], Cs[n0], Fs[n0], step=n0)
        gpu.step(10)
        x, v, Cm, F = gpu.get_state()
        n1 = n0 + 10
        assert_state_close((x, v), (xs[n1], vs[n1]), names=("x", "v"))


@pytest.mark.parametrize("impl", IMPLS, ids=["tiled", "plain"])
def test_walker_square_full_horizon_gradient(M, ctx, impl):
    """dL/dv0 and dL/dA over the full 100 steps, L = mean final x_0, against the oracle."""
    spec = S.walker_square_2d(0)
    osc = O.Scene(spec)
    traj = osc.rollout(100)
    seed = mean_x0_seed(osc.N, 2)
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (seed, None, None, None))
    gpu = M.Scene(ctx, spec, impl=impl)
    gpu.rollout(100, 10)
    x, v, _, _ = gpu.get_state()
    assert rel_l2(x, traj[0][100]) < 1e-3
    gx, gv, gC, gF, gp = gpu.backward(seed)
    assert_grad_close(gv, ogv, "dL/dv0")
    assert_grad_close(gp, ogp, "dL/dA")
    assert_grad_close(gx, ogx, "dL/dx0")
    assert_grad_close(gF, ogF, "dL/dF0")


@pytest.mark.parametrize("name", ["2d_basis", "3d_mlp", "2d_slip_friction", "3d_sticky", "2d_table", "3d_table",
                                  "2d_com", "3d_com"])
def test_controller_and_state_gradients(M, ctx, name):
    spec = small_scenes()[name]
    T = 25
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    rng = np.random.default_rng(7)
    wx = rng.normal(size=traj[0][T].shape) / osc.N
    wv = rng.normal(size=traj[1][T].shape) / osc.N
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (wx, wv, None, None))
    gpu = M.Scene(ctx, spec)
    gpu.rollout(T, 4)
    gx, gv, gC, gF, gp = gpu.backward(wx, wv)
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF), ("params", gp, ogp)):
        assert_grad_close(a, b, f"{name} dL/d{nm}")
    if spec.ctrl_type == S.CTRL_TABLE:  # rows past the rollout stay exactly zero
        assert np.all(gp.reshape(spec.ctrl_hidden, -1)[T:] == 0)


def test_tiled_is_bitwise_deterministic_and_checkpoint_invariant(M, ctx):
    """The tiled form sums in a fixed order everywhere: two runs agree bit for bit, and the
    recomputed states of any checkpoint interval equal the stored ones, so gradients too."""
    spec = S.walker_square_2d(0)
    seed = mean_x0_seed(spec.n_particles, 2)
    outs = []
    for k in (1, 7, 64, 100, 7):
        gpu = M.Scene(ctx, spec)
        gpu.rollout(100, k)
        outs.append(gpu.backward(seed))
        gpu.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_recompute_beside_reverse_steps_is_bitwise_the_sequential_pass(M, ctx):
    """The reverse pass recomputes the next segment on a second stream (own workspace, odd
    segments in a second buffer set) unless the memory budget leaves no room for those buffers;
    both schedules, and repeated passes reusing the captured graphs, give the same bits.  The
    walker-size scene with the sinusoid-basis controller and uneven last segment (T = 150, k = 16)."""
    spec = S.walker_2d(1, n_steps=150)
    seed = mean_x0_seed(spec.n_particles, 2)
    sc = M.Scene(ctx, spec)
    S_bytes = sc.info()["state_bytes"]
    k = 16
    for T in (150, 145):  # last segment of 6 states, and of a single state
        nseg = (T + k - 1) // k
        outs = []
        for budget in (0, (nseg + k - 1) * S_bytes, 0):  # overlapped, sequential (tight budget), overlapped
            sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)
            sc.rollout(T, k, budget)
            outs.append(sc.get_state() + sc.backward(seed))
        for o in outs[1:]:
            for a, b in zip(o, outs[0]):
                assert np.array_equal(a, b), T
    sc.close()


@pytest.mark.parametrize("ctrl", ["basis_2d", "table_3d"])
def test_controller_reverse_beside_next_step_is_bitwise_the_serial_pass(M, ctx, ctrl):
    """Controllers that read no state (sinusoid basis, per-step table) have their reverse captured
    on a branch of the reverse graphs, beside the next step's sort and adjoint scatter, and the
    sorts of a graph's later steps load on a second branch into two alternating buffer sets; with
    launch timing on, the same steps are launched one after another on one stream and one buffer
    set.  Both give the same bits (T = 50, k = 16: segments replayed as 8-step and single-step
    graphs)."""
    if ctrl == "basis_2d":
        spec = S.walker_2d(1, n_steps=50)
    else:
        spec = S.blob(3, 16, 1200, 73, ctrl_type=S.CTRL_TABLE, n_groups=3, hidden=40, amp=3.0,
                      radius_cells=3.0, v_scale=0.3)
    seed = mean_x0_seed(spec.n_particles, spec.dim)
    T, k = 50, 16
    sc = M.Scene(ctx, spec)
    outs = []
    for direct in (False, True, False):
        if direct:
            ctx.profile_start([M.K_CTRL])
        sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)
        sc.rollout(T, k)
        outs.append(sc.get_state() + sc.backward(seed))
        if direct:
            assert ctx.profile_read(M.K_CTRL)[0] >= T  # the steps were launched directly
            ctx.profile_start([])
    sc.close()
    assert np.abs(outs[0][-1]).max() > 0
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("ctrl", ["mlp_3d", "com_2d"])
def test_recompute_beside_reverse_steps_with_state_reading_controllers(M, ctx, ctrl):
    """Controllers that read the state (MLP on group centroids, closed loop on group means) run
    their forward in the recompute with scratch of their own: overlapped and sequential reverse
    passes give the same bits."""
    if ctrl == "mlp_3d":
        spec = S.blob(3, 20, 1500, 71, ctrl_type=S.CTRL_MLP, n_groups=4, hidden=16, scale=5.0,
                      radius_cells=3.5, v_scale=0.3)
    else:
        spec = S.blob(2, 32, 800, 72, ctrl_type=S.CTRL_COM, n_groups=3, radius_cells=5.0, v_scale=0.3)
    seed = mean_x0_seed(spec.n_particles, spec.dim)
    sc = M.Scene(ctx, spec)
    S_bytes = sc.info()["state_bytes"]
    T, k = 40, 7
    nseg = (T + k - 1) // k
    outs = []
    for budget in (0, (nseg + k - 1) * S_bytes):
        sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)
        sc.rollout(T, k, budget)
        outs.append(sc.get_state() + sc.backward(seed))
    sc.close()
    for a, b in zip(outs[1], outs[0]):
        assert np.array_equal(a, b)


def test_plain_and_tiled_agree(M, ctx):
    spec = S.walker_square_2d(0)
    res = []
    for impl in IMPLS:
        gpu = M.Scene(ctx, spec, impl=impl)
        gpu.step(50)
        res.append(gpu.get_state())
    assert_state_close(res[0], res[1], tol=1e-5)


def test_domain_and_inversion_errors(M, ctx):
    spec = S.blob(2, 16, 20, 0)
    spec.x0[0] = [2.6 / 16, 0.5]
    spec.v0[0] = [-400.0, 0.0]  # leaves the grid within one step
    spec = spec.copy(bc_width=0)
    g = M.Scene(ctx, spec)
    g.step(2)
    with pytest.raises(M.MPMError) as e:
        g.get_state()
    assert e.value.status == -3
    spec2 = S.blob(2, 16, 20, 0)
    spec2.F0[3] = np.diag([1.0, -0.5])
    g2 = M.Scene(ctx, spec2)
    g2.step(1)
    with pytest.raises(M.MPMError) as e:
        g2.get_state()
    assert e.value.status == -4
    # set_state clears the error
    g2.set_state(*O.Scene(S.blob(2, 16, 20, 0)).initial_state())
    g2.step(1)
    g2.get_state()


def test_empty_scene(M, ctx):
    spec = S.blob(2, 16, 1, 0)
    spec = spec.copy(x0=np.zeros((0, 2)), v0=np.zeros((0, 2)), C0=np.zeros((0, 2, 2)), F0=np.zeros((0, 2, 2)),
                     group=np.zeros(0, np.int32))
    g = M.Scene(ctx, spec)
    g.rollout(3, 1)
    out = g.backward(np.zeros((0, 2)))
    assert out[0].shape == (0, 2)


# ----------------------------------------------------------------------------- full sizes
FULL = {
    "walker_2d": lambda: S.walker_2d(1),
    "soft_body_3d": lambda: S.soft_body_3d(2),
    "box_cluster_3d": lambda: S.box_cluster_3d(3),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_one_step_forward_and_reverse(M, ctx, name):
    """At the full workload sizes, in the launch configuration the benchmark times: one forward
    step and one reverse step against the oracle (a step touches every particle and node)."""
    spec = FULL[name]()
    osc = O.Scene(spec)
    st0 = osc.initial_state()
    step0 = 5
    gpu = M.Scene(ctx, spec)
    gpu.set_state(*st0, step=step0)
    gpu.step(1)
    ref = oracle_step_from(spec, st0, step0)
    assert_state_close(gpu.get_state(), ref)
    # one reverse step: L = <w, x_1> + <u, v_1>
    rng = np.random.default_rng(3)
    wx = rng.normal(size=st0[0].shape) / osc.N
    wv = rng.normal(size=st0[1].shape) / osc.N
    gpu.set_state(*st0, step=step0)
    gpu.rollout(1)
    act = osc.controller(step0, st0[0])
    (ogx, ogv, ogC, ogF), ogact = osc.step_adjoint(act, st0, (wx, wv, np.zeros_like(st0[2]), np.zeros_like(st0[3])))
    gx, gv, gC, gF, gp = gpu.backward(wx, wv)
    ogp, ogx_ctrl = osc.controller_adjoint(step0, st0[0], ogact)
    for nm, a, b in (("x", gx, ogx + ogx_ctrl), ("v", gv, ogv), ("C", gC, ogC), ("F", gF, ogF)):
        assert_grad_close(a, b, f"{name} one-step dL/d{nm}")
    assert_grad_close(gp, ogp, f"{name} one-step dL/dparams")


def _dense(dim):
    """Dense blobs: tiles above P2G's one-pass capacity (512 particles in 3D, 2 x 256 in 2D) take
    the bucket-and-sort path with records staged in chunks, and G2P's gather reads the particles
    past its 512-particle staging directly."""
    if dim == 3:
        return S.blob(3, 16, 3000, 81, radius_cells=2.0, v_scale=0.3, c_scale=1.0, f_scale=0.03,
                      center=(6.0 / 16, 7.0 / 16, 6.0 / 16), amp=2.0)
    return S.blob(2, 16, 3000, 82, radius_cells=3.0, v_scale=0.3, c_scale=1.0, f_scale=0.03,
                  center=(6.0 / 16, 7.0 / 16), amp=2.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_dense_tiles_match_oracle(M, ctx, dim):
    spec = _dense(dim)
    n = spec.n_grid[0]
    base = np.floor(spec.x0 * n - 0.5).astype(int) // 4  # tile of every particle (4-cell tiles)
    _, counts = np.unique(base, axis=0, return_counts=True)
    assert counts.max() > (512 if dim == 3 else 1024)  # the general path really runs
    osc = O.Scene(spec)
    st0 = osc.initial_state()
    ref = oracle_step_from(spec, st0, 0)
    for impl in IMPLS:
        g = M.Scene(ctx, spec, impl=impl)
        g.step(1)
        assert_state_close(g.get_state(), ref)
        g.close()
    T = 10
    traj = osc.rollout(T)
    rng = np.random.default_rng(3)
    wx = rng.normal(size=traj[0][T].shape) / osc.N
    wv = rng.normal(size=traj[1][T].shape) / osc.N
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (wx, wv, None, None))
    g = M.Scene(ctx, spec)
    g.rollout(T, 4)
    gx, gv, gC, gF, gp = g.backward(wx, wv)
    g.close()
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF), ("params", gp, ogp)):
        assert_grad_close(a, b, f"dense {dim}d dL/d{nm}")


@pytest.mark.parametrize("dim", [2, 3])
def test_tile_over_capacity_is_reported(M, ctx, dim):
    """More particles in one tile than the tile kernels stage (2048 in 2D, 4096 in 3D): the step
    reports MPM_ERR_DENSITY instead of dropping or overrunning anything."""
    N = 2500 if dim == 2 else 5000
    spec = S.blob(dim, 16, N, 83, radius_cells=1.2, center=np.full(dim, 6.0 / 16))
    g = M.Scene(ctx, spec)
    g.step(1)
    with pytest.raises(M.MPMError) as e:
        g.get_state()
    assert e.value.status == -8
    # stepping on is safe: the tile's particles drop out of the binning, nothing is overrun
    g.step(3)
    with pytest.raises(M.MPMError) as e:
        g.get_state()
    assert e.value.status == -8
    g.close()


# ----------------------------------------------------------------------------- multi-level store
def _ml_case(case):
    if case == "2d_sin":
        return S.walker_square_2d(0, n_steps=40), 0, 40
    if case == "2d_plain":
        return S.walker_square_2d(0, n_steps=30), 1, 30
    if case == "2d_table":  # per-step actuation: every range must resume at its own global step
        return S.blob(2, 32, 300, 7, ctrl_type=S.CTRL_TABLE, n_groups=4, hidden=40, radius_cells=4.5,
                      v_scale=0.3, amp=3.0), 0, 33
    if case == "3d_mlp":  # a controller that reads the state
        return S.blob(3, 16, 400, 6, ctrl_type=S.CTRL_MLP, n_groups=4, hidden=16, scale=5.0, radius_cells=3.5,
                      v_scale=0.3), 0, 27
    if case == "2d_material":
        return S.with_material(S.walker_square_2d(0, n_steps=25), 5), 0, 25
    raise ValueError(case)


@pytest.mark.parametrize("case", ["2d_sin", "2d_plain", "2d_table", "3d_mlp", "2d_material"])
def test_multi_level_store_is_bitwise_the_store_all(M, ctx, case):
    """Budgets below the single-level store ((ceil(T/k) + k - 1) states) take the multi-level
    store; it recomputes more but runs the same reverse steps on the same states, so the final
    state and every gradient are the bits of a rollout that keeps every state (the tiled form; the
    plain form's atomic sums agree to rounding)."""
    spec, impl, T = _ml_case(case)
    sc = M.Scene(ctx, spec, impl=impl)
    S_bytes = sc.info()["state_bytes"]
    rng = np.random.default_rng(11)
    wx = rng.normal(size=(spec.n_particles, spec.dim)) / spec.n_particles
    wv = rng.normal(size=(spec.n_particles, spec.dim)) / spec.n_particles
    material = getattr(spec, "E_arr", None) is not None
    outs = []
    for states in (0, 5, 3):  # every state; 5 and 3 states (the least the store accepts)
        if states:
            assert M.plan_checkpoints(T, states)[2]  # the multi-level store is planned
        sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0, step=0)
        sc.rollout(T, 0, states * S_bytes)
        res = list(sc.get_state()) + list(sc.backward(wx, wv))
        if material:
            res += list(sc.material_gradients())
        if states:  # the spine is spent: one reverse pass per multi-level rollout
            with pytest.raises(M.MPMError) as e:
                sc.backward(wx, wv)
            assert e.value.status == -7
            assert sc.info()["step"] == T  # the scene is back at the rollout's final state
        outs.append(res)
    sc.close()
    assert np.abs(outs[0][5]).max() > 0
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            if impl == 0:
                assert np.array_equal(a, b)
            else:  # the plain form adds with float atomics: the same sums in another order
                assert rel_l2(a, b) < 1e-5


def test_multi_level_store_below_three_states_is_refused(M, ctx):
    spec = S.walker_square_2d(0, n_steps=20)
    sc = M.Scene(ctx, spec)
    with pytest.raises(M.MPMError) as e:
        sc.rollout(20, 0, 2 * sc.info()["state_bytes"])
    assert e.value.status == -2
    sc.close()


# ----------------------------------------------------------------------------- storage order
def _permuted(spec, pr):
    ch = dict(x0=spec.x0[pr], v0=spec.v0[pr], C0=spec.C0[pr], F0=spec.F0[pr], group=spec.group[pr])
    for nm in ("E_arr", "mass_arr"):
        if getattr(spec, nm, None) is not None:
            ch[nm] = getattr(spec, nm)[pr]
    return spec.copy(**ch)


@pytest.mark.parametrize("case", ["2d_sin", "3d_mlp", "2d_material", "2d_com"])
def test_caller_particle_order_changes_no_bit(M, ctx, case):
    """The library keeps particles in its own storage order (by tile, cell and position of the
    initial state), so the same particles handed over in a random order give the same bits, in
    the caller's order: final state, every gradient, the material gradients."""
    if case == "2d_com":
        spec, T = small_scenes()["2d_com"], 20
    else:
        spec, _, T = _ml_case(case)
    N, d = spec.n_particles, spec.dim
    pr = np.random.default_rng(5).permutation(N)
    rng = np.random.default_rng(6)
    wx = rng.normal(size=(N, d)) / N
    wv = rng.normal(size=(N, d)) / N
    res = []
    for sp, perm in ((spec, np.arange(N)), (_permuted(spec, pr), pr)):
        sc = M.Scene(ctx, sp)
        sc.rollout(T, 7)
        out = list(sc.get_state()) + list(sc.backward(wx[perm], wv[perm]))
        if getattr(sp, "E_arr", None) is not None:
            out += list(sc.material_gradients())
        sc.close()
        res.append(out)
    for i, (a, b) in enumerate(zip(res[0], res[1])):
        if i == 8:  # controller parameters: not per particle
            assert np.array_equal(a, b)
        else:
            assert np.array_equal(a[pr], b), i


# ----------------------------------------------------------------------------- tile edge
@pytest.mark.parametrize("edge", [4, 8])
@pytest.mark.parametrize("name", ["2d_sticky", "2d_slip_friction", "2d_com"])
def test_both_tile_edges_match_oracle(M, ctx, name, edge):
    """2D scenes run with 4 x 4- or 8 x 8-cell tiles (the binning, the node blocks and every tile
    kernel follow the scene's edge): one step and a 12-step rollout's gradients against the
    oracle for each."""
    spec = small_scenes()[name].copy(tile_edge=edge)
    gpu = M.Scene(ctx, spec)
    assert gpu.tile_edge == edge
    st0 = O.Scene(spec).initial_state()
    gpu.set_state(*st0, step=3)
    gpu.step(1)
    assert_state_close(gpu.get_state(), oracle_step_from(spec, st0, 3))
    T = 12
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    rng = np.random.default_rng(4)
    wx = rng.normal(size=traj[0][T].shape) / osc.N
    wv = rng.normal(size=traj[1][T].shape) / osc.N
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (wx, wv, None, None))
    gpu.set_state(*st0, step=0)
    gpu.rollout(T, 5)
    gx, gv, gC, gF, gp = gpu.backward(wx, wv)
    gpu.close()
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF), ("params", gp, ogp)):
        assert_grad_close(a, b, f"{name} edge {edge} dL/d{nm}")


def test_tile_edge_chosen_from_particle_density(M, ctx):
    """0 lets the library choose: 8 x 8 tiles for a sparse 2D scene (the 1,024-particle square:
    ~50 particles per occupied 4 x 4 tile), 4 x 4 for a dense one (the walker at 16 per cell) and
    for 3D; 8 is refused in 3D."""
    assert M.Scene(ctx, S.walker_square_2d(0)).tile_edge == 8
    assert M.Scene(ctx, S.walker_2d(1, n_steps=10)).tile_edge == 4
    assert M.Scene(ctx, small_scenes()["3d_sticky"]).tile_edge == 4
    assert M.Scene(ctx, S.walker_square_2d(0).copy(tile_edge=4)).tile_edge == 4
    with pytest.raises(M.MPMError) as e:
        M.Scene(ctx, small_scenes()["3d_sticky"].copy(tile_edge=8))
    assert e.value.status == -1


@pytest.mark.parametrize("dim,side", [(3, 20), (2, 80)])
def test_falling_cube_matches_oracle(M, ctx, dim, side):
    """The paper's speed-comparison scene (a falling elastic cube at Table II's particle counts):
    10-step windows of a 30-step fall onto the sticky floor, and the gradient of a 30-step rollout
    keeping every state, as the bench times it."""
    spec = S.falling_cube(dim, side, n_steps=30)
    osc = O.Scene(spec)
    traj = osc.rollout(30)
    gpu = M.Scene(ctx, spec)
    for w in range(3):
        n0 = 10 * w
        gpu.set_state(traj[0][n0], traj[1][n0], traj[2][n0], traj[3][n0], step=n0)
        gpu.step(10)
        x, v, Cm, F = gpu.get_state()
        ref = tuple(t[n0 + 10] for t in traj[:4])
        assert_state_close((x, v, F), (ref[0], ref[1], ref[3]), names=("x", "v", "F"))
        # C is exactly zero while the cube falls as a rigid body (the oracle's is ~1e-16): its error
        # is measured against its natural size |v| / dx
        scale = max(np.linalg.norm(ref[2]), np.linalg.norm(ref[1]) / spec.dx)
        assert np.linalg.norm(Cm - ref[2]) / scale <= FWD_TOL
    rng = np.random.default_rng(8)
    wx = rng.normal(size=traj[0][30].shape) / osc.N
    wv = rng.normal(size=traj[1][30].shape) / osc.N
    ogx, ogv, ogC, ogF, _ = osc.backward(traj, (wx, wv, None, None))
    gpu.set_state(*osc.initial_state(), step=0)
    gpu.rollout(30, 1)
    gx, gv, gC, gF, _ = gpu.backward(wx, wv)
    gpu.close()
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF)):
        assert_grad_close(a, b, f"cube {dim}d dL/d{nm}")
