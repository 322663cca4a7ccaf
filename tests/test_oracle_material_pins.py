"""Pins of the oracle's material gradients (CPU): dL/dE_p and dL/dm_p for per-particle Young's
modulus and mass.

E_p enters the step only through P (Eq. 4, neo-Hookean with the textbook Lame map), m_p only
through P2G (m_i and p_i of Eqs. 3-5).  The checks are independent of that derivation:
  - per-particle arrays equal to the scene's constants reproduce the uniform scene bit for bit;
  - central finite differences of a full rollout's loss (FP64, the paper's own FD method);
  - scaling every mass and every E_p by one factor leaves the motion unchanged when no actuation
    is applied (stress and momentum scale together, v = p / m does not), so
    sum_p (m_p dL/dm_p + E_p dL/dE_p) = 0;
  - a particle alone at F = I feels no stress and its mass cancels in v = p / m: both are zero.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S

T_2D, T_3D = 8, 5


def _scenes():
    a = S.blob(2, 16, 40, 11, v_scale=0.4, c_scale=1.0, f_scale=0.05, radius_cells=2.5,
               center=(0.5, 3.6 / 16), bc_width=2, amp=3.0, dt=1e-3)
    b = S.blob(3, 10, 30, 12, v_scale=0.4, c_scale=1.0, f_scale=0.05, radius_cells=1.8,
               center=(0.5, 3.2 / 10, 0.45), bc_width=2, amp=3.0, dt=1e-3)
    c = S.blob(2, 16, 40, 13, v_scale=0.4, bc_type=S.BC_SLIP, friction_c=0.3, radius_cells=2.5,
               center=(0.45, 3.4 / 16), bc_width=2, amp=3.0, dt=1e-3)
    return {"2d_sticky": (S.with_material(a, 1), T_2D), "3d_sticky": (S.with_material(b, 2), T_3D),
            "2d_slip_friction": (S.with_material(c, 3), T_2D)}


def _weights(spec, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(spec.n_particles, spec.dim)), rng.normal(size=(spec.n_particles, spec.dim))


def _loss(spec, T, wx, wv):
    xs, vs, _, _, _ = O.Scene(spec).rollout(T)
    return float(np.sum(wx * xs[T]) + np.sum(wv * vs[T]))


def _grads(spec, T, wx, wv):
    sc = O.Scene(spec)
    traj = sc.rollout(T)
    return sc.backward(traj, (wx, wv, None, None), material=True)


def test_uniform_arrays_reproduce_the_uniform_scene_bitwise():
    spec = _scenes()["2d_sticky"][0].copy(E_arr=None, mass_arr=None)
    uni = spec.copy(E_arr=np.full(spec.n_particles, spec.E), mass_arr=np.full(spec.n_particles, spec.p_mass))
    wx, wv = _weights(spec, 0)
    ta, tb = O.Scene(spec).rollout(T_2D), O.Scene(uni).rollout(T_2D)
    for a, b in zip(ta, tb):
        assert np.array_equal(a, b)
    ga = O.Scene(spec).backward(ta, (wx, wv, None, None))
    gb = O.Scene(uni).backward(tb, (wx, wv, None, None), material=True)
    for a, b in zip(ga, gb[:5]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", list(_scenes()))
def test_material_gradients_match_central_differences(name):
    spec, T = _scenes()[name]
    wx, wv = _weights(spec, 7)
    *_, gE, gm = _grads(spec, T, wx, wv)
    rng = np.random.default_rng(5)
    for p in rng.choice(spec.n_particles, 4, replace=False):
        for arr_name, g, rel_h in (("E_arr", gE, 1e-6), ("mass_arr", gm, 1e-6)):
            base = getattr(spec, arr_name)
            h = rel_h * base[p]
            up, dn = base.copy(), base.copy()
            up[p] += h
            dn[p] -= h
            fd = (_loss(spec.copy(**{arr_name: up}), T, wx, wv) - _loss(spec.copy(**{arr_name: dn}), T, wx, wv)) / (2 * h)
            scale = max(abs(fd), 1e-3 * np.max(np.abs(g)))
            assert abs(g[p] - fd) <= 2e-5 * scale, f"{name} {arr_name}[{p}]: adjoint {g[p]:.9e} vs FD {fd:.9e}"


@pytest.mark.parametrize("name", list(_scenes()))
def test_joint_scaling_of_mass_and_modulus_is_a_symmetry_without_actuation(name):
    spec, T = _scenes()[name]
    spec = spec.copy(ctrl_params=np.zeros_like(spec.ctrl_params))  # a_g = 0 at every step
    wx, wv = _weights(spec, 9)
    *_, gE, gm = _grads(spec, T, wx, wv)
    terms = spec.mass_arr * gm + spec.E_arr * gE
    assert abs(terms.sum()) <= 1e-9 * np.abs(terms).sum()
    assert np.abs(terms).sum() > 0  # both gradients are non-trivial here
    # with actuation the symmetry is broken (the actuation stress does not scale with E)
    spec_a, _ = _scenes()[name]
    *_, gEa, gma = _grads(spec_a, T, wx, wv)
    ta = spec_a.mass_arr * gma + spec_a.E_arr * gEa
    assert abs(ta.sum()) > 1e-6 * np.abs(ta).sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_isolated_particle_at_rest_shape_has_zero_material_gradient(dim):
    spec = S.blob(dim, 12, 1, 21, v_scale=0.5, c_scale=2.0, radius_cells=0.0, n_groups=0, dt=1e-3)
    spec = S.with_material(spec, 4)
    sc = O.Scene(spec)
    st = sc.initial_state()
    assert np.allclose(st[3], np.eye(dim))
    rng = np.random.default_rng(1)
    adj = (rng.normal(size=(1, dim)), rng.normal(size=(1, dim)), rng.normal(size=(1, dim, dim)),
           rng.normal(size=(1, dim, dim)))
    (gx, gv, gC, gF), _, (gE, gm) = sc.step_adjoint(np.zeros(0), st, adj, material=True)
    assert gE[0] == 0.0
    # the terms that cancel in dL/dm_p are of size |adjoint| / m_p (pbar = vbar* / m_i)
    term = max(np.abs(a).max() for a in adj) / spec.mass_arr[0]
    assert abs(gm[0]) <= 1e-13 * term
