"""Per-particle Young's modulus and mass and their gradients on the GPU, against the FP64 oracle
(same seeded inputs): forward states and every gradient of a rollout, one full-size step, the
uniform-array case bitwise equal to the uniform scene, batching, and argument checks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import assert_grad_close, assert_state_close, mean_x0_seed

pytestmark = pytest.mark.gpu


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
    return {
        "2d_walker_square": (S.with_material(S.walker_square_2d(0, n_steps=40), 11), 40, 8),
        "3d_mlp": (S.with_material(S.blob(3, 16, 400, 6, ctrl_type=S.CTRL_MLP, n_groups=4, hidden=16, scale=5.0,
                                          radius_cells=3.5, v_scale=0.3), 12), 15, 5),
        "2d_slip_friction": (S.with_material(S.blob(2, 32, 257, 3, v_scale=0.8, bc_type=S.BC_SLIP, friction_c=0.4,
                                                    bc_width=3, radius_cells=4.0, center=(0.4, 4.8 / 32), amp=1.0),
                                             13), 20, 4),
    }


@pytest.mark.parametrize("impl", [0, 1], ids=["tiled", "plain"])
@pytest.mark.parametrize("name", list(_cases()))
def test_material_rollout_and_gradients_match_oracle(M, ctx, name, impl):
    spec, T, k = _cases()[name]
    sc = M.Scene(ctx, spec, impl=impl)
    sc.rollout(T, k)
    st = sc.get_state()
    grads = sc.backward(mean_x0_seed(sc.N, sc.dim))
    gE, gm = sc.material_gradients()
    sc.close()
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    assert_state_close(st, tuple(a[T] for a in traj[:4]))
    ogx, ogv, ogC, ogF, ogp, ogE, ogm = osc.backward(traj, (mean_x0_seed(osc.N, osc.dim), None, None, None),
                                                     material=True)
    for nm, a, b in (("x", grads[0], ogx), ("v", grads[1], ogv), ("F", grads[3], ogF), ("params", grads[4], ogp)):
        assert_grad_close(a, b, f"{name} dL/d{nm}")
    assert_grad_close(gE, ogE, f"{name} dL/dE_p")
    assert_grad_close(gm, ogm, f"{name} dL/dm_p")


def test_full_size_one_step_material_gradients(M, ctx):
    """walker_2d (31k particles) at full size in the benchmark's launch configuration: one reverse
    step's dL/dE_p and dL/dm_p against the oracle, L = <w, x_1> + <u, v_1>."""
    spec = S.with_material(S.walker_2d(1), 21)
    osc = O.Scene(spec)
    x0, v0, C0, F0 = osc.initial_state()
    rng0 = np.random.default_rng(4)  # a deformed state: at F = I the stress and dP/dE vanish
    F0 = F0 + 0.03 * rng0.normal(size=F0.shape)
    C0 = C0 + 0.5 * rng0.normal(size=C0.shape)
    st0 = (x0, v0, C0, F0)
    step0 = 3
    gpu = M.Scene(ctx, spec)
    gpu.set_state(*st0, step=step0)
    gpu.rollout(1)
    rng = np.random.default_rng(8)
    wx = rng.normal(size=st0[0].shape) / osc.N
    wv = rng.normal(size=st0[1].shape) / osc.N
    gpu.backward(wx, wv)
    gE, gm = gpu.material_gradients()
    gpu.close()
    act = osc.controller(step0, st0[0])
    _, _, (ogE, ogm) = osc.step_adjoint(act, st0, (wx, wv, np.zeros_like(st0[2]), np.zeros_like(st0[3])),
                                        material=True)
    assert_grad_close(gE, ogE, "walker_2d one-step dL/dE_p")
    assert_grad_close(gm, ogm, "walker_2d one-step dL/dm_p")


def test_uniform_arrays_are_bitwise_the_uniform_scene(M, ctx):
    spec = S.walker_square_2d(0, n_steps=30)
    uni = spec.copy(E_arr=np.full(spec.n_particles, spec.E), mass_arr=np.full(spec.n_particles, spec.p_mass))
    out = []
    for sp in (spec, uni):
        sc = M.Scene(ctx, sp)
        sc.rollout(30, 6)
        out.append((sc.get_state(), sc.backward(mean_x0_seed(sc.N, 2))))
        sc.close()
    for a, b in zip(out[0][0] + out[0][1], out[1][0] + out[1][1]):
        assert np.array_equal(a, b)


def test_material_scene_in_a_batch_equals_alone(M, ctx):
    reqs = [(S.with_material(S.blob(2, 32, 300, 1, v_scale=0.3, radius_cells=5.0, center=(0.5, 7.0 / 32),
                                    bc_width=3, amp=2.0), 5), 23),
            (S.walker_square_2d(0), 30)]
    alone = []
    for spec, T in reqs:
        sc = M.Scene(ctx, spec)
        sc.rollout(T, 1 if T <= 16 else int(np.ceil(np.sqrt(T))))
        g = sc.backward(mean_x0_seed(sc.N, 2))
        alone.append((sc.get_state(), g, sc.material_gradients() if spec.E_arr is not None else None))
        sc.close()
    batch = M.Batch(ctx, 2)
    scenes = [M.Scene(ctx, spec) for spec, _ in reqs]
    slots = [batch.admit(sc, T, True) for sc, (_, T) in zip(scenes, reqs)]
    while not all(batch.poll(s) for s in slots):
        batch.tick(4)
    for sc, (st, g, mg) in zip(scenes, alone):
        for a, b in zip(sc.get_state() + sc.gradients(), st + g):
            assert np.array_equal(a, b)
        if mg is not None:
            for a, b in zip(sc.material_gradients(), mg):
                assert np.array_equal(a, b)
    batch.close()


def test_material_arguments_are_checked(M, ctx):
    spec = S.walker_square_2d(0, n_steps=10)
    sc = M.Scene(ctx, spec)
    N = spec.n_particles
    with pytest.raises(M.MPMError):
        sc.material_gradients()  # no per-particle material
    with pytest.raises(M.MPMError):
        sc.set_material(E=np.full(N, -1.0))
    with pytest.raises(M.MPMError):
        sc.set_material(mass=np.where(np.arange(N) == 3, np.nan, spec.p_mass))
    # 100x stiffer particles break dt <= dx sqrt(rho / E)
    with pytest.raises(M.MPMError):
        sc.set_material(E=np.full(N, 100.0 * spec.E))
    sc.set_material(E=np.full(N, spec.E))
    with pytest.raises(M.MPMError):
        sc.material_gradients()  # no reverse pass yet
    sc.close()
