"""The double-precision plain form on the GPU (mpm64_*) against the FP64 oracle on the same
seeded inputs, and the Section VI accuracy study (case B, colliding elastic discs in float64):
the GPU adjoint against GPU central finite differences at 1, 10, 100 and 1000 steps.

Tolerance (FP64 on both sides, different summation orders): every stencil sum of 9 or 27 terms
and every per-particle product is exact to a few units of 2^-53 ~ 1.1e-16; over a rollout of T
steps these differences add up and are carried along by the dynamics.  For the rollouts here
(<= 100 steps, mild contact) the bound 1e-9 relative (whole-array L2 and element-wise over the
array's max) leaves several orders of magnitude for amplification while still catching any
dropped or wrong term, which moves results by >= 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


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


def _close(a, b, what, tol=TOL64, scale=0.0):
    """Relative L2 and element-wise error of a against b, each over max(size of b, scale): the
    scale floors arrays that are zero up to rounding (C of a rigid translation)."""
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    e = a - b
    r = np.linalg.norm(e) / max(np.linalg.norm(b), scale * np.sqrt(b.size), 1e-300)
    m = np.abs(e).max() / max(np.abs(b).max(), scale, 1e-300)
    assert r <= tol and m <= 10 * tol, f"{what}: relative L2 {r:.3e}, max scaled {m:.3e} (tol {tol:.0e})"


def _cases():
    bil = S.billiards_2d()
    # 2D: per-step actuation table on two groups, slip floor with friction, open ceiling
    a = S.blob(2, 32, 300, 61, v_scale=0.3, radius_cells=4.0, center=(0.5, 5.5 / 32), bc_width=3,
               ctrl_type=S.CTRL_TABLE, hidden=40, amp=3.0, c_scale=0.5, f_scale=0.02)
    a = a.copy(wall_kind=np.array([S.BC_STICKY, S.BC_SLIP, S.BC_SLIP, S.BC_OPEN], np.int32),
               wall_c=np.array([0.0, 0.0, 0.4, 0.0]))
    # 3D: three groups with a table shorter than the rollout (zero actuation after it)
    b = S.blob(3, 16, 400, 62, v_scale=0.3, radius_cells=3.0, center=(0.5, 4.5 / 16, 0.5), bc_width=3,
               n_groups=3, ctrl_type=S.CTRL_TABLE, hidden=12, amp=3.0, c_scale=0.5, f_scale=0.02)
    b = b.copy(bc_type=S.BC_SLIP, friction_c=0.3)
    return {"billiards_2d": (bil, 100), "2d_table_walls": (a, 40), "3d_table_slip": (b, 20)}


@pytest.mark.parametrize("name", list(_cases()))
def test_fp64_rollout_and_gradients_match_oracle(M, ctx, name):
    spec, T = _cases()[name]
    rng = np.random.default_rng(3)
    N, d = spec.n_particles, spec.dim
    wx, wv = rng.normal(size=(N, d)) / N, rng.normal(size=(N, d)) / N
    wC, wF = rng.normal(size=(N, d, d)) / N, rng.normal(size=(N, d, d)) / N
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (wx, wv, wC, wF))
    sc = M.Scene64(ctx, spec)
    sc.rollout(T)
    # natural sizes: positions and F of order 1, velocities of order 1, C of order |v| / dx
    scales = (1.0, 1.0, 1.0 / spec.dx, 1.0)
    for t in (1, T // 2, T):
        for nm, a, b, sc_ in zip("xvCF", sc.get_state(t), (traj[0][t], traj[1][t], traj[2][t], traj[3][t]), scales):
            _close(a, b, f"{name} {nm}_{t}", scale=sc_)
    gx, gv, gC, gF, gU = sc.backward(wx, wv, wC, wF)
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF)):
        _close(a, b, f"{name} dL/d{nm}")
    if spec.n_groups:
        _close(gU.ravel(), np.asarray(ogp).ravel(), f"{name} dL/dU")
        assert np.abs(gU).max() > 0
    sc.close()


def test_runs_agree_to_rounding_and_state_resets(M, ctx):
    spec, T = _cases()["2d_table_walls"]
    sc = M.Scene64(ctx, spec)
    sc.rollout(T)
    a = sc.get_state()
    # another initial state, then the original again: the rollout restarts from step 0
    sc.set_state(spec.x0 + 1e-3, spec.v0, spec.C0, spec.F0)
    sc.rollout(T)
    moved = sc.get_state()
    sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0)
    sc.rollout(T)
    b = sc.get_state()
    sc.close()
    for u, w in zip(a, b):
        _close(u, w, "repeat", tol=1e-13)
    assert rel_l2(moved[0], a[0]) > 1e-5


def _b_centroid_grad(M, ctx, spec, T, h):
    """L = x centroid of ball B at step T: dL/d(vx of A, one direction) by the adjoint and by
    central differences, both on the GPU in FP64."""
    a = S.billiards_ball_a(spec)
    w = np.zeros_like(spec.x0)
    w[~a, 0] = 1.0 / (~a).sum()
    sc = M.Scene64(ctx, spec)
    sc.rollout(T)
    g = sc.backward(w)[1][a, 0].sum()
    L = []
    for sgn in (1, -1):
        v0 = spec.v0.copy()
        v0[a, 0] += sgn * h
        sc.set_state(spec.x0, v0, spec.C0, spec.F0)
        sc.rollout(T)
        L.append(np.sum(w * sc.get_state()[0]))
    sc.close()
    return g, (L[0] - L[1]) / (2 * h)


def test_accuracy_study_colliding_discs(M, ctx):
    """Section VI case B (paper: relative error 2.39e-8 at 100 steps, 2.83e-8 at 1000; no value at
    1 and 10 steps, where no collision has happened yet)."""
    spec = S.billiards_2d()
    for T in (1, 10):
        g, fd = _b_centroid_grad(M, ctx, spec, T, 1e-6)
        # no shared node yet: the adjoint is exactly zero; the two FD runs differ only by the
        # order of atomic sums inside ball B
        assert g == 0.0 and abs(fd) <= 1e-9
    for T in (100, 1000):
        g, fd = _b_centroid_grad(M, ctx, spec, T, 1e-6)
        assert abs(g) > 1e-2
        assert abs(g - fd) <= 1e-7 * abs(fd), (T, g, fd, abs(g - fd) / abs(fd))


def test_fp64_errors_are_reported(M, ctx):
    spec = S.blob(2, 32, 50, 63, radius_cells=3.0)
    bad = spec.copy(bc_width=0)
    bad.x0[0] = [2.6 / 32, 0.5]
    bad.v0[0] = [-800.0, 0.0]
    sc = M.Scene64(ctx, bad, act=np.zeros((0, bad.n_groups)))
    sc.rollout(5)
    with pytest.raises(M.MPMError) as e:
        sc.get_state()
    assert e.value.status == -3
    # the next rollout from a valid state clears it
    sc.set_state(spec.x0, spec.v0, spec.C0, spec.F0)
    sc.rollout(5)
    sc.get_state()
    with pytest.raises(M.MPMError):
        sc.set_state(np.full_like(spec.x0, np.nan))
    sc.close()
    with pytest.raises(ValueError):
        M.Scene64(ctx, spec)  # sinusoid controller: the FP64 form wants a table
    with pytest.raises(M.MPMError):
        M.Scene64(ctx, spec.copy(dt=1.0), act=np.zeros((0, spec.n_groups)))  # explicit limit
    sc = M.Scene64(ctx, spec, act=np.zeros((0, spec.n_groups)))
    with pytest.raises(M.MPMError) as e:
        sc.backward()  # no rollout yet
    assert e.value.status == -7
    sc.close()


def test_fp64_empty_scene_and_table_replacement(M, ctx):
    empty = S.blob(2, 16, 0, 64, radius_cells=1.0)
    sc = M.Scene64(ctx, empty, act=np.zeros((0, empty.n_groups)))
    sc.rollout(5)
    assert all(a.size == 0 for a in sc.get_state())
    assert all(a.size == 0 for a in sc.backward()[:4])
    sc.close()
    # a new actuation table replaces the old one: the rollout and dL/dU follow the oracle
    spec, T = _cases()["2d_table_walls"]
    U2 = 0.5 * np.asarray(spec.ctrl_params).reshape(spec.ctrl_hidden, spec.n_groups)[:30]
    sc = M.Scene64(ctx, spec)
    sc.set_actuation(U2)
    sc.rollout(T)
    N, d = spec.n_particles, spec.dim
    w = np.random.default_rng(9).normal(size=(N, d)) / N
    gU = sc.backward(w)[4]
    x = sc.get_state()[0]
    sc.close()
    ospec = spec.copy(ctrl_params=U2.ravel(), ctrl_hidden=U2.shape[0])
    osc = O.Scene(ospec)
    traj = osc.rollout(T)
    ogp = osc.backward(traj, (w, None, None, None))[4]
    _close(x, traj[0][T], "x after a new table", scale=1.0)
    assert gU.shape == U2.shape
    _close(gU.ravel(), np.asarray(ogp).ravel(), "dL/dU of the new table")
