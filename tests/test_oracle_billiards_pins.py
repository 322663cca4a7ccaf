"""Pins of the oracle on the float64 accuracy scene of Section VI (two colliding elastic discs,
no gravity, no wall contact), from facts the method fixes independently of its code:

  - P2G and G2P of MLS-MPM with APIC transfer linear momentum exactly (Eqs. 3-8: sum_i N_ip = 1,
    sum_i N_ip (x_i - x_p) = 0), so with no external force total momentum sum m v stays at its
    initial value through the collision, and the centre of mass moves on a straight line,
    sum m x_T = sum m x_0 + T dt sum m v_0 (x_{n+1} = x_n + dt v_{n+1});
  - before the discs share a grid node, ball B sits exactly still and ball A translates rigidly;
  - the collision transfers momentum (B moves after it) and the adjoint of "B's final x
    centroid" with respect to A's initial velocity matches FP64 central differences (the
    paper's accuracy method), and is exactly zero while no collision has happened.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S


@pytest.fixture(scope="module")
def scene():
    spec = S.billiards_2d()
    sc = O.Scene(spec)
    return spec, sc, sc.rollout(300), S.billiards_ball_a(spec)


def test_momentum_and_centre_of_mass_are_conserved_through_the_collision(scene):
    spec, sc, tr, a = scene
    m = spec.p_mass
    P0 = m * spec.v0.sum(0)
    X0 = m * spec.x0.sum(0)
    for T in (10, 50, 100, 300):
        P = m * tr[1][T].sum(0)
        assert np.allclose(P, P0, rtol=0, atol=1e-12 * np.abs(P0).max()), (T, P, P0)
        X = m * tr[0][T].sum(0)
        assert np.allclose(X, X0 + T * spec.dt * P0, rtol=0, atol=1e-12 * np.abs(X0).max()), T
    # the collision happened: B carries a good part of the momentum at the end
    assert m * tr[1][300][~a].sum(0)[0] > 0.5 * P0[0]


def test_before_contact_b_is_still_and_a_translates(scene):
    spec, sc, tr, a = scene
    for T in (1, 10):
        assert np.array_equal(tr[0][T][~a], spec.x0[~a])
        assert np.allclose(tr[0][T][a], spec.x0[a] + T * spec.dt * spec.v0[a], rtol=0, atol=1e-14)
        assert np.allclose(tr[1][T][a], spec.v0[a], rtol=0, atol=1e-12)


def _loss_and_grad(spec, T, h=None):
    """L = x centroid of ball B at step T; dL/d(vx of every A particle) summed (one direction)."""
    a = S.billiards_ball_a(spec)
    sc = O.Scene(spec)
    tr = sc.rollout(T)
    w = np.zeros_like(spec.x0)
    w[~a, 0] = 1.0 / (~a).sum()
    gv0 = sc.backward(tr, (w, None, None, None))[1]
    g = gv0[a, 0].sum()
    if h is None:
        return g
    L = []
    for sgn in (1, -1):
        v0 = spec.v0.copy()
        v0[a, 0] += sgn * h
        L.append(np.sum(w * O.Scene(spec.copy(v0=v0)).rollout(T)[0][T]))
    return g, (L[0] - L[1]) / (2 * h)


def test_gradient_is_zero_before_the_collision():
    spec = S.billiards_2d()
    for T in (1, 10):
        assert _loss_and_grad(spec, T) == 0.0


def test_collision_gradient_matches_central_differences():
    spec = S.billiards_2d()
    g, fd = _loss_and_grad(spec, 100, h=1e-6)
    assert abs(g) > 1e-2  # B's final position does depend on A's speed
    assert abs(g - fd) <= 1e-6 * abs(fd), (g, fd)
