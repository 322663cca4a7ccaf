"""Per-wall boundary conditions on the GPU (sticky, slip with its own friction, open) against the
FP64 oracle: state and every gradient of checkpointed rollouts of bodies pressed into mixed
corners, both kernel forms; uniform per-wall settings bitwise equal to the uniform scene."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import assert_grad_close, assert_state_close

pytestmark = pytest.mark.gpu

STICKY, SLIP, OPEN = S.BC_STICKY, S.BC_SLIP, S.BC_OPEN


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


def _cases():
    # 2D: sticky left wall, frictionless right wall, floor with c = 0.5, open ceiling; thrown
    # into the lower-left corner
    a = S.blob(2, 32, 400, 51, v_scale=0.3, radius_cells=4.0, center=(5.5 / 32, 5.5 / 32), bc_width=3, amp=2.0)
    a.v0 += np.array([-0.8, -0.6])
    a = a.copy(wall_kind=np.array([STICKY, SLIP, SLIP, OPEN], np.int32), wall_c=np.array([0.0, 0.0, 0.5, 0.0]))
    # 3D: slip walls with different friction on x and z, sticky floor, open ceiling
    b = S.blob(3, 20, 600, 52, v_scale=0.3, radius_cells=3.0, center=(4.5 / 20, 5.0 / 20, 4.5 / 20), bc_width=3,
               amp=2.0)
    b.v0 += np.array([-0.6, -0.5, -0.6])
    b = b.copy(wall_kind=np.array([SLIP, SLIP, STICKY, OPEN, SLIP, SLIP], np.int32),
               wall_c=np.array([0.3, 0.0, 0.0, 0.0, 0.8, 0.1]))
    return {"2d_corner": (a, 30), "3d_corner": (b, 20)}


@pytest.mark.parametrize("impl", [0, 1], ids=["tiled", "plain"])
@pytest.mark.parametrize("name", list(_cases()))
def test_mixed_walls_match_oracle(M, ctx, name, impl):
    spec, T = _cases()[name]
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    rng = np.random.default_rng(5)
    wx = rng.normal(size=traj[0][T].shape) / osc.N
    wv = rng.normal(size=traj[1][T].shape) / osc.N
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (wx, wv, None, None))
    sc = M.Scene(ctx, spec, impl=impl)
    sc.rollout(T, 6)
    assert_state_close(sc.get_state(), tuple(a[T] for a in traj[:4]))
    gx, gv, gC, gF, gp = sc.backward(wx, wv)
    sc.close()
    for nm, a, b in (("x0", gx, ogx), ("v0", gv, ogv), ("C0", gC, ogC), ("F0", gF, ogF), ("params", gp, ogp)):
        assert_grad_close(a, b, f"{name} dL/d{nm}")


@pytest.mark.parametrize("bc", [STICKY, SLIP])
def test_uniform_walls_are_bitwise_the_uniform_boundary(M, ctx, bc):
    spec = S.blob(2, 32, 300, 53, v_scale=0.8, bc_type=bc, friction_c=0.3, radius_cells=4.0,
                  center=(0.3, 5.0 / 32), bc_width=3, amp=2.0)
    walls = spec.copy(wall_kind=np.full(4, bc, np.int32), wall_c=np.full(4, 0.3))
    out = []
    for sp in (spec, walls):
        sc = M.Scene(ctx, sp)
        sc.rollout(20, 5)
        out.append(sc.get_state() + sc.backward(np.ones((sp.n_particles, 2)) / sp.n_particles))
        sc.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_wall_arguments_are_checked(M, ctx):
    sc = M.Scene(ctx, S.walker_square_2d(0, n_steps=5))
    with pytest.raises(M.MPMError):
        sc.set_walls(kind=[0, 1, 3, 0])
    with pytest.raises(M.MPMError):
        sc.set_walls(c=[0.1, -0.2, 0.0, 0.0])
    with pytest.raises(ValueError):
        sc.set_walls(kind=[0, 1, 2])
    sc.set_walls(kind=[OPEN, OPEN, STICKY, OPEN], c=[0.0, 0.0, 0.0, 0.0])
    sc.step(3)
    sc.close()
