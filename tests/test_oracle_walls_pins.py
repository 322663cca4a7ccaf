"""Pins of per-wall boundary conditions in the oracle (CPU): each wall sticky, slip with its own
Coulomb friction c (Supplement S5) or open.

  - one kind and one c on every wall reproduce the uniform sticky / slip scenes bit for bit;
  - at edge and corner nodes of mixed walls the (L) adjoint matches central differences of the
    forward projection, an open wall leaves velocity and adjoint untouched, a sticky wall wins;
  - rollout gradients against central differences for a body touching a frictional floor, a
    sticky wall and an open ceiling.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S

STICKY, SLIP, OPEN = S.BC_STICKY, S.BC_SLIP, S.BC_OPEN


@pytest.mark.parametrize("bc", [STICKY, SLIP])
def test_uniform_walls_reproduce_the_uniform_boundary_bitwise(bc):
    spec = S.blob(2, 16, 40, 41, v_scale=0.8, bc_type=bc, friction_c=0.3, radius_cells=2.5,
                  center=(0.3, 3.2 / 16), bc_width=2, amp=2.0, dt=1e-3)
    walls = spec.copy(wall_kind=np.full(4, bc, np.int32), wall_c=np.full(4, 0.3))
    T = 12
    a, b = O.Scene(spec), O.Scene(walls)
    ta, tb = a.rollout(T), b.rollout(T)
    for u, w in zip(ta, tb):
        assert np.array_equal(u, w)
    rng = np.random.default_rng(1)
    seeds = (rng.normal(size=ta[0][T].shape), rng.normal(size=ta[1][T].shape), None, None)
    for u, w in zip(a.backward(ta, seeds), b.backward(tb, seeds)):
        assert np.array_equal(u, w)


def _wall_scene(dim, kinds, cs, n=12, width=2):
    spec = S.blob(dim, n, 4, 3, radius_cells=1.0, bc_width=width)
    return O.Scene(spec.copy(wall_kind=np.asarray(kinds, np.int32), wall_c=np.asarray(cs, float)))


def _fd_check(sc, idx, rng, dim):
    for _ in range(6):
        vin = rng.normal(size=dim)
        gout = rng.normal(size=dim)
        vout, gin = O.bc(sc, idx, vin, gout)
        dv = rng.normal(size=dim)
        h = 1e-7
        fd = gout @ (O.bc(sc, idx, vin + h * dv) - O.bc(sc, idx, vin - h * dv)) / (2 * h)
        assert abs(fd - gin @ dv) <= 1e-6 * max(1.0, abs(fd)), (idx, vin, fd, gin @ dv)


def test_mixed_walls_2d_adjoint_and_semantics():
    # x-low slip c=0.5, x-high sticky, y-low (floor) slip c=0.2, y-high open
    n = 12
    sc = _wall_scene(2, [SLIP, STICKY, SLIP, OPEN], [0.5, 0.0, 0.2, 0.0], n=n)
    rng = np.random.default_rng(0)
    for idx in ([0, 0], [1, 5], [5, 0], [0, n - 1], [6, 6]):  # slip corner, slip edges, slip+open corner, interior
        _fd_check(sc, idx, rng, 2)
    v = np.array([0.3, -0.7])
    g = np.array([1.1, -0.4])
    # open wall: identity forward and reverse
    vo, gi = O.bc(sc, [5, n - 1], v, g)
    assert np.array_equal(vo, v) and np.array_equal(gi, g)
    # a sticky wall wins at its corners (with the floor, and with the open ceiling)
    for idx in ([n - 1, 0], [n - 1, n - 1], [n - 2, 6]):
        vo, gi = O.bc(sc, idx, v, g)
        assert np.all(vo == 0) and np.all(gi == 0)
    # the corner of two slip walls equals applying the x wall, then the floor
    only_x = _wall_scene(2, [SLIP, OPEN, OPEN, OPEN], [0.5, 0, 0, 0], n=n)
    only_y = _wall_scene(2, [OPEN, OPEN, SLIP, OPEN], [0, 0, 0.2, 0], n=n)
    v1 = O.bc(only_x, [0, 0], v)
    assert np.array_equal(O.bc(sc, [0, 0], v), O.bc(only_y, [0, 0], v1))


def _project(v, nrm, c):
    """S5 one-wall projection restated: normal part kept when it leaves the wall, tangential part
    shrunk by c times the compression (to zero at most)."""
    ln = v @ nrm
    vt = v - ln * nrm
    lt = np.sqrt(vt @ vt + 1e-20)
    return max(lt + c * min(ln, 0.0), 0.0) / lt * vt + max(ln, 0.0) * nrm


@pytest.mark.parametrize("dim", [2, 3])
def test_each_wall_projects_with_its_own_friction(dim):
    n = 12
    cs = [0.1, 0.5, 0.9, 0.3, 0.7, 0.2][: 2 * dim]
    sc = _wall_scene(dim, [SLIP] * (2 * dim), cs, n=n)
    rng = np.random.default_rng(dim)
    for w in range(2 * dim):
        a, side = w // 2, w % 2
        idx = [n // 2] * dim
        idx[a] = n - 1 if side else 0
        nrm = np.zeros(dim)
        nrm[a] = -1.0 if side else 1.0
        for _ in range(4):
            v = rng.normal(size=dim)
            v -= (abs(v @ nrm) + 0.5) * nrm  # pressing into the wall: friction acts
            assert np.allclose(O.bc(sc, idx, v), _project(v, nrm, cs[w]), rtol=1e-14, atol=1e-15)


def test_mixed_walls_3d_adjoint():
    n = 10
    sc = _wall_scene(3, [SLIP, SLIP, SLIP, OPEN, STICKY, SLIP], [0.4, 0.1, 0.7, 0, 0, 0.25], n=n)
    rng = np.random.default_rng(2)
    for idx in ([0, 0, 5], [0, 0, n - 1], [n - 1, 0, n - 1], [5, 0, 5], [0, 5, 5], [5, n - 1, n - 1]):
        _fd_check(sc, idx, rng, 3)
    for idx in ([5, 5, 0], [0, 5, 0], [0, 0, 0], [n - 1, 0, 0]):  # z-low is sticky, also after slip walls
        vo, gi = O.bc(sc, idx, np.ones(3), np.ones(3))
        assert np.all(vo == 0) and np.all(gi == 0)


def test_rollout_gradient_fd_with_mixed_walls():
    """A blob dropped into the corner of a frictional floor (slip c = 0.4) and a sticky left wall,
    with an open ceiling and a frictionless right wall; the chain rule over the rollout against
    FP64 central differences (the paper's method)."""
    n = 16
    spec = S.blob(2, n, 30, 44, v_scale=0.5, radius_cells=2.2, center=(3.6 / n, 3.6 / n), bc_width=2, amp=2.0,
                  dt=2e-3, gravity=(0.0, -9.8))
    spec = spec.copy(wall_kind=np.array([STICKY, SLIP, SLIP, OPEN], np.int32), wall_c=np.array([0, 0.0, 0.4, 0]))
    sc = O.Scene(spec)
    T = 15
    traj = sc.rollout(T)
    rng = np.random.default_rng(11)
    w, wv = rng.normal(size=traj[0][T].shape), rng.normal(size=traj[1][T].shape)
    loss = lambda tr: np.sum(w * tr[0][T]) + np.sum(wv * tr[1][T])
    gx0, gv0, gC0, gF0, gp = sc.backward(traj, (w, wv, None, None))
    x0, v0, C0, F0 = sc.initial_state()
    h = 1e-6
    dv = rng.normal(size=v0.shape)
    fd = (loss(sc.rollout(T, (x0, v0 + h * dv, C0, F0))) - loss(sc.rollout(T, (x0, v0 - h * dv, C0, F0)))) / (2 * h)
    assert abs(fd - np.sum(gv0 * dv)) <= 1e-6 * max(1, abs(fd))
    dx = rng.normal(size=x0.shape) * 0.1
    fd = (loss(sc.rollout(T, (x0 + h * dx, v0, C0, F0))) - loss(sc.rollout(T, (x0 - h * dx, v0, C0, F0)))) / (2 * h)
    assert abs(fd - np.sum(gx0 * dx)) <= 1e-6 * max(1, abs(fd))
    # the scene does touch the walls: the same loss with uniform sticky walls differs
    stick = O.Scene(spec.copy(wall_kind=np.zeros(4, np.int32)))
    assert abs(loss(stick.rollout(T)) - loss(traj)) > 1e-6
