"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: conservation laws of
Eqs. 1-2, the exact affine reproduction of APIC/MLS transfers, the discrete free-fall
trajectory, closed-form gradients (the analogues of Table III's A1/A2 cases), the energy
whose derivative the stress is, frame indifference, and central finite differences of every
reverse formula of the supplement (the paper's own FP64 FD methodology, Section IV-B).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S


def _blob(dim, **kw):
    n = kw.pop("n", 16 if dim == 2 else 12)
    npart = kw.pop("npart", 24)
    seed = kw.pop("seed", 0)
    return S.blob(dim, n, npart, seed, **kw)


# ----------------------------------------------------------------------------- I1, I2
@pytest.mark.parametrize("dim", [2, 3])
def test_grid_mass_and_momentum_conservation(dim):
    """I1/I2: sum_i m_i = sum_p m_p and sum_i p_i = sum_p m_p v_p (Eqs. 3-5): the B-spline
    weights are a partition of unity and sum_i N (x_i - x_p) = 0 cancels the stress and APIC
    terms.  Gravity 0 and no boundary contact, so m_i v*_i = p_i."""
    sp = _blob(dim, gravity=(0.0,) * dim, v_scale=0.7, c_scale=3.0, f_scale=0.1, npart=40, seed=3)
    sc = O.Scene(sp)
    x, v, Cm, F = sc.initial_state()
    act = np.array([2.0, -3.0])
    _, (gm, gv) = sc.step(act, x, v, Cm, F, want_grid=True)
    M = sp.p_mass * sc.N
    assert abs(gm.sum() - M) <= 1e-12 * M
    mom_grid = (gm[:, None] * gv).sum(axis=0)
    mom_part = sp.p_mass * v.sum(axis=0)
    assert np.allclose(mom_grid, mom_part, rtol=0, atol=1e-12 * np.abs(mom_part).max())


# ----------------------------------------------------------------------------- I3
@pytest.mark.parametrize("dim", [2, 3])
def test_affine_field_reproduced_exactly(dim):
    """I3: F = I (so P = 0), no actuation, no gravity, v_p = b + A x_p, C_p = A gives grid
    velocities b + A x_i and G2P returns v_p = b + A x_p, C_p = A (APIC with the quadratic
    B-spline, whose second moment is dx^2/4, i.e. D^{-1} = 4/dx^2)."""
    rng = np.random.default_rng(7)
    sp = _blob(dim, gravity=(0.0,) * dim, n_groups=0, npart=50, seed=5)
    sc = O.Scene(sp)
    x, _, _, F = sc.initial_state()
    b = rng.normal(size=dim)
    A = rng.normal(size=(dim, dim))
    v = b + x @ A.T
    Cm = np.broadcast_to(A, (sc.N, dim, dim)).copy()
    (x1, v1, C1, F1), (gm, gv) = sc.step(np.zeros(0), x, v, Cm, F, want_grid=True)
    act_nodes = np.nonzero(gm > 0)[0]
    idx = np.stack(np.unravel_index(act_nodes, sp.n_grid), axis=1)
    xi = idx * sp.dx
    assert np.allclose(gv[act_nodes], b + xi @ A.T, rtol=0, atol=1e-12)
    assert np.allclose(v1, v, rtol=0, atol=1e-12)
    assert np.allclose(C1, Cm, rtol=0, atol=1e-10)
    assert np.allclose(x1, x + sp.dt * v, rtol=0, atol=1e-14)
    assert np.allclose(F1, np.eye(dim) + sp.dt * A, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- I4
@pytest.mark.parametrize("dim", [2, 3])
def test_free_fall_centre_of_mass(dim):
    """I4: without boundary contact total momentum changes only by M dt g per step, so for any
    stress and actuation the centre of mass follows x_T = x_0 + T dt v_0 + dt^2 g T(T+1)/2."""
    g = np.array([0.0, -9.8, 0.0][:dim])
    n = 32 if dim == 2 else 24
    sp = S.blob(dim, n, 60, 11, v_scale=0.2, c_scale=1.0, f_scale=0.05, radius_cells=3.0, amp=3.0)
    sc = O.Scene(sp)
    T = 20
    xs, vs, Cs, Fs, acts = sc.rollout(T)
    dt = sp.dt
    xc0, vc0 = xs[0].mean(axis=0), vs[0].mean(axis=0)
    expect = xc0 + T * dt * vc0 + dt * dt * g * T * (T + 1) / 2
    assert np.allclose(xs[T].mean(axis=0), expect, rtol=0, atol=1e-12)
    assert np.abs(acts).max() > 0.1  # the actuation really was active


# ----------------------------------------------------------------------------- I5
@pytest.mark.parametrize("dim", [2, 3])
def test_closed_form_gradient_no_contact(dim):
    """I5 (Table III A1 analogue): L = mean_p x_{p,0}(T) with no contact is
    mean(x0_0) + T dt mean(v0_0) + const, so dL/dv0 = T dt / N e_0, dL/dx0 = e_0 / N and
    dL/dC0 = dL/dF0 = dL/dA = 0 exactly, whatever the stress and actuation do."""
    n = 32 if dim == 2 else 24
    sp = S.blob(dim, n, 40, 2, v_scale=0.2, c_scale=1.0, f_scale=0.05, radius_cells=3.0, amp=3.0)
    sc = O.Scene(sp)
    T = 12
    traj = sc.rollout(T)
    N = sc.N
    gxT = np.zeros((N, dim))
    gxT[:, 0] = 1.0 / N
    gx0, gv0, gC0, gF0, gp = sc.backward(traj, (gxT, None, None, None))
    e0 = np.zeros(dim)
    e0[0] = 1.0
    assert np.allclose(gv0, T * sp.dt / N * e0, rtol=0, atol=1e-13)
    assert np.allclose(gx0, e0 / N, rtol=0, atol=1e-12)
    assert np.abs(gC0).max() < 1e-13 and np.abs(gF0).max() < 1e-11
    assert np.abs(gp).max() < 1e-12


def test_closed_form_gradient_slip_floor():
    """I5 (Table III A2 analogue): a block sliding along a frictionless (slip, c = 0) floor keeps
    its tangential momentum, so dL/dv0_{p,0} = T dt / N for L = mean_p x_{p,0}(T), although the
    floor removes normal momentum at every step of contact."""
    sp = S.walker_square_2d(0, n_steps=30)
    sp = sp.copy(bc_type=S.BC_SLIP, friction_c=0.0)
    sp.v0[:, 0] = 0.5
    sc = O.Scene(sp)
    T = 30
    traj = sc.rollout(T)
    N = sc.N
    # the floor was really hit: vertical momentum is not the free-fall value
    vy = traj[1][T][:, 1].mean()
    assert abs(vy - (-9.8 * T * sp.dt)) > 1e-3
    gxT = np.zeros((N, 2))
    gxT[:, 0] = 1.0 / N
    gx0, gv0, *_ = sc.backward(traj, (gxT, None, None, None))
    assert np.allclose(gv0[:, 0], T * sp.dt / N, rtol=1e-9, atol=0)


# ----------------------------------------------------------------------------- I6
def _psi(F, mu, la):
    d = F.shape[0]
    J = np.linalg.det(F)
    return mu / 2 * (np.trace(F.T @ F) - d) - mu * np.log(J) + la / 2 * np.log(J) ** 2


@pytest.mark.parametrize("dim", [2, 3])
def test_neohookean_stress_is_energy_gradient(dim):
    """I6: P(I) = 0, P = dpsi/dF by central differences of the energy, frame indifference
    P(RF) = R P(F), and the Hessian product of S4 (H) equals the directional FD of P."""
    rng = np.random.default_rng(1)
    E, nu = 20.0, 0.3
    mu, la = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    P0, _ = O.neohookean(np.eye(dim), E, nu)
    assert np.abs(P0).max() < 1e-14
    for _ in range(5):
        F = np.eye(dim) + 0.3 * rng.normal(size=(dim, dim))
        if np.linalg.det(F) <= 0.2:
            continue
        P, _ = O.neohookean(F, E, nu)
        h = 1e-6
        Pfd = np.zeros((dim, dim))
        for i in range(dim):
            for j in range(dim):
                dF = np.zeros((dim, dim))
                dF[i, j] = h
                Pfd[i, j] = (_psi(F + dF, mu, la) - _psi(F - dF, mu, la)) / (2 * h)
        assert np.allclose(P, Pfd, rtol=1e-7, atol=1e-7)
        Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        PR, _ = O.neohookean(Q @ F, E, nu)
        assert np.allclose(PR, Q @ P, rtol=0, atol=1e-12)
        Pbar = rng.normal(size=(dim, dim))
        dF = rng.normal(size=(dim, dim))
        _, HP = O.neohookean(F, E, nu, Pbar)
        Pp, _ = O.neohookean(F + h * dF, E, nu)
        Pm, _ = O.neohookean(F - h * dF, E, nu)
        lhs = np.sum(HP * dF)
        rhs = np.sum(Pbar * (Pp - Pm) / (2 * h))
        assert abs(lhs - rhs) <= 1e-7 * max(1.0, abs(rhs))


# ----------------------------------------------------------------------------- I8
def test_sticky_band_zero_velocity():
    """I8: nodes in the sticky band have v* = 0, and a particle whose whole stencil lies in the
    band leaves G2P with v = 0 and C = 0."""
    sp = _blob(2, n=16, npart=30, seed=4, v_scale=1.0, bc_width=2)
    sp.x0[0] = [1.2 / 16, 1.1 / 16]  # base (0, 0): nodes 0..2 on both axes; band nodes 0,1
    sp.x0[1] = [0.9 / 16, 0.9 / 16]  # base (0, 0) as well
    sp = sp.copy(bc_width=3)  # now nodes 0..2 are all in the band
    sc = O.Scene(sp)
    x, v, Cm, F = sc.initial_state()
    (x1, v1, C1, F1), (gm, gv) = sc.step(np.zeros(2), x, v, Cm, F, want_grid=True)
    idx = np.stack(np.unravel_index(np.arange(gm.size), sp.n_grid), axis=1)
    band = ((idx < 3) | (idx >= 16 - 3)).any(axis=1)
    assert np.all(gv[band] == 0.0)
    assert np.all(v1[:2] == 0.0) and np.all(C1[:2] == 0.0)
    assert np.abs(gv[~band & (gm > 0)]).max() > 0


# ----------------------------------------------------------------------------- S5
def test_friction_projection_forward_cases():
    """S5 (L) forward: separating motion (l_n >= 0) is untouched, approaching motion loses its
    normal part, and with c > 0 the tangential speed drops by c |l_n| (clamped at 0)."""
    sp = _blob(2, n=16, npart=4, seed=1, bc_type=S.BC_SLIP, friction_c=0.5, bc_width=2)
    sc = O.Scene(sp)
    idx = (8, 1)  # floor band only: inward normal +e_1
    assert np.allclose(O.bc(sc, idx, [0.3, 0.2]), [0.3, 0.2], atol=1e-12)
    assert np.allclose(O.bc(sc, idx, [0.3, -0.2]), [0.3 - 0.5 * 0.2, 0.0], atol=1e-12)
    assert np.allclose(O.bc(sc, idx, [0.05, -0.2]), [0.0, 0.0], atol=1e-12)
    sc0 = O.Scene(sp.copy(friction_c=0.0))
    assert np.allclose(O.bc(sc0, idx, [0.3, -0.2]), [0.3, 0.0], atol=1e-12)
    sticky = O.Scene(sp.copy(bc_type=S.BC_STICKY))
    assert np.all(O.bc(sticky, idx, [0.3, -0.2]) == 0.0)


@pytest.mark.parametrize("dim,c", [(2, 0.0), (2, 0.7), (3, 0.0), (3, 0.4)])
def test_friction_projection_adjoint_fd(dim, c):
    """S5 (L) reverse against central differences, on single walls and on corners (walls applied
    in sequence), away from the kinks l_n = 0 and R = 0."""
    rng = np.random.default_rng(int(10 * c) + dim)
    n = 12
    sp = S.blob(dim, n, 4, 0, bc_type=S.BC_SLIP, friction_c=c, bc_width=2)
    sc = O.Scene(sp)
    cases = [(1,) + (5,) * (dim - 1), (5,) * (dim - 1) + (n - 1,), (0,) * dim, (n - 1,) + (0,) * (dim - 1)]
    h = 1e-6
    for idx in cases:
        for _ in range(6):
            v = rng.normal(size=dim)
            go = rng.normal(size=dim)
            _, gin = O.bc(sc, idx, v, go)
            fd = np.zeros(dim)
            for a in range(dim):
                e = np.zeros(dim)
                e[a] = h
                fd[a] = go @ (O.bc(sc, idx, v + e) - O.bc(sc, idx, v - e)) / (2 * h)
            assert np.allclose(gin, fd, rtol=1e-6, atol=1e-8), (idx, v)


# ----------------------------------------------------------------------------- I7
def _flat(t):
    return np.concatenate([np.ravel(a) for a in t])


def _unflat(vec, like):
    out, o = [], 0
    for a in like:
        out.append(vec[o:o + a.size].reshape(a.shape))
        o += a.size
    return out


CASES_STEP = [
    dict(dim=2, bc_type=S.BC_STICKY, seed=0),
    dict(dim=3, bc_type=S.BC_STICKY, seed=1),
    dict(dim=2, bc_type=S.BC_SLIP, friction_c=0.0, seed=2),
    dict(dim=2, bc_type=S.BC_SLIP, friction_c=0.6, seed=3),
    dict(dim=3, bc_type=S.BC_SLIP, friction_c=0.3, seed=4),
]


@pytest.mark.parametrize("case", CASES_STEP, ids=lambda c: f"{c['dim']}d-bc{c['bc_type']}-c{c.get('friction_c', 0)}")
def test_step_adjoint_dot_product(case):
    """I7: <ybar, J xdot> = <J^T ybar, xdot> for one step, J xdot by FP64 central differences;
    scenes touch the boundary band so (L) and the sticky zeroing are exercised, and every
    state component (x, v, C, F) and the actuation are perturbed."""
    dim = case["dim"]
    n = 12
    rng = np.random.default_rng(100 + case["seed"])
    sp = S.blob(dim, n, 30, case["seed"], bc_type=case["bc_type"], friction_c=case.get("friction_c", 0.0),
                bc_width=2, v_scale=0.5, c_scale=2.0, f_scale=0.1, radius_cells=2.0,
                center=np.full(dim, 3.6 / n), dt=2e-3, amp=2.0)
    sc = O.Scene(sp)
    st = sc.initial_state()
    act = rng.normal(size=sc.G)
    out = sc.step(act, *st)
    ybar = [rng.normal(size=a.shape) for a in out]
    adj, gact = sc.step_adjoint(act, st, ybar)
    xdot = [rng.normal(size=a.shape) for a in st]
    adot = rng.normal(size=sc.G)
    h = 1e-6
    sp_ = [a + h * b for a, b in zip(st, xdot)]
    sm_ = [a - h * b for a, b in zip(st, xdot)]
    op = sc.step(act + h * adot, *sp_)
    om = sc.step(act - h * adot, *sm_)
    jvp = (_flat(op) - _flat(om)) / (2 * h)
    lhs = _flat(ybar) @ jvp
    rhs = _flat(adj) @ _flat(xdot) + gact @ adot
    assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(lhs)), (lhs, rhs)
    # and component-wise on the position block alone (the (J) term of the supplement)
    xd = [xdot[0], np.zeros_like(st[1]), np.zeros_like(st[2]), np.zeros_like(st[3])]
    op = sc.step(act, *[a + h * b for a, b in zip(st, xd)])
    om = sc.step(act, *[a - h * b for a, b in zip(st, xd)])
    lhs = _flat(ybar) @ ((_flat(op) - _flat(om)) / (2 * h))
    rhs = np.sum(adj[0] * xdot[0])
    assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("ctrl", [S.CTRL_SIN, S.CTRL_BASIS, S.CTRL_MLP, S.CTRL_TABLE])
def test_controller_adjoint_fd(ctrl):
    """The controller forms' reverse (parameters and, for the MLP, positions through the group
    centroids) against central differences."""
    rng = np.random.default_rng(ctrl)
    sp = S.blob(3, 12, 40, 9, n_groups=4, ctrl_type=ctrl, hidden=10 if ctrl == S.CTRL_TABLE else 6, freq=4.0,
                scale=3.0)
    sc = O.Scene(sp)
    x = sc.initial_state()[0]
    step = 7
    ga = rng.normal(size=sc.G)
    gp, gx = sc.controller_adjoint(step, x, ga)
    h = 1e-6
    pd = rng.normal(size=sc.params.shape)
    fd = ga @ (sc.controller(step, x, sc.params + h * pd) - sc.controller(step, x, sc.params - h * pd)) / (2 * h)
    assert abs(fd - gp @ pd) <= 1e-7 * max(1, abs(fd))
    xd = rng.normal(size=x.shape)
    fdx = ga @ (sc.controller(step, x + h * xd) - sc.controller(step, x - h * xd)) / (2 * h)
    assert abs(fdx - np.sum(gx * xd)) <= 1e-7 * max(1, abs(fdx))
    if ctrl != S.CTRL_MLP:
        assert np.all(gx == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_closed_loop_controller_adjoint_fd(dim):
    """The closed-loop form a = scale tanh(W z + b), z = [target, group centres of mass, group
    velocities]: its reverse for the parameters (target included), x and v against central
    differences; particles of no group get no x or v adjoint."""
    rng = np.random.default_rng(50 + dim)
    sp = S.blob(dim, 12, 40, 19, n_groups=3, ctrl_type=S.CTRL_COM, scale=3.0, v_scale=0.5)
    sp.group[::7] = -1  # some particles in no group
    sc = O.Scene(sp)
    x, v = sc.initial_state()[:2]
    step, h = 5, 1e-6
    ga = rng.normal(size=sc.G)
    gp, gx, gv = sc.controller_adjoint(step, x, ga, v=v)
    a = lambda **k: sc.controller(step, k.get("x", x), params=k.get("p"), v=k.get("v", v))
    pd = rng.normal(size=sc.params.shape)
    fd = ga @ (a(p=sc.params + h * pd) - a(p=sc.params - h * pd)) / (2 * h)
    assert abs(fd - gp @ pd) <= 1e-7 * max(1, abs(fd))
    xd = rng.normal(size=x.shape)
    fd = ga @ (a(x=x + h * xd) - a(x=x - h * xd)) / (2 * h)
    assert abs(fd - np.sum(gx * xd)) <= 1e-7 * max(1, abs(fd))
    vd = rng.normal(size=v.shape)
    fd = ga @ (a(v=v + h * vd) - a(v=v - h * vd)) / (2 * h)
    assert abs(fd - np.sum(gv * vd)) <= 1e-7 * max(1, abs(fd))
    assert np.all(gx[::7] == 0) and np.all(gv[::7] == 0)
    assert np.any(gv != 0)


@pytest.mark.parametrize("ctrl,dim", [(S.CTRL_SIN, 2), (S.CTRL_BASIS, 2), (S.CTRL_MLP, 3), (S.CTRL_TABLE, 2),
                                      (S.CTRL_COM, 2), (S.CTRL_COM, 3)])
def test_rollout_gradient_fd(ctrl, dim):
    """I7 over a rollout: the chain rule of Section III from a loss on the final state back to the
    initial v0, x0 and the controller parameters used at every step, against FP64 central FD
    (the paper's Table III B/C methodology) on a tiny scene touching the sticky floor."""
    rng = np.random.default_rng(40 + ctrl)
    n = 16 if dim == 2 else 12
    T = 15
    sp = S.blob(dim, n, 24, 20 + ctrl, n_groups=3, ctrl_type=ctrl, hidden=T + 3 if ctrl == S.CTRL_TABLE else 5,
                freq=4.0, scale=2.0, v_scale=0.3, radius_cells=2.0, center=np.full(dim, 3.8 / n), amp=2.0,
                bc_width=2, dt=2e-3)
    sc = O.Scene(sp)
    traj = sc.rollout(T)
    w = rng.normal(size=traj[0][T].shape)
    wv = rng.normal(size=traj[1][T].shape)
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
    dF = rng.normal(size=F0.shape) * 0.1
    fd = (loss(sc.rollout(T, (x0, v0, C0, F0 + h * dF))) - loss(sc.rollout(T, (x0, v0, C0, F0 - h * dF)))) / (2 * h)
    assert abs(fd - np.sum(gF0 * dF)) <= 1e-6 * max(1, abs(fd))
    dp = rng.normal(size=sc.params.shape)
    fd = (loss(sc.rollout(T, params=sc.params + h * dp)) - loss(sc.rollout(T, params=sc.params - h * dp))) / (2 * h)
    assert abs(fd - gp @ dp) <= 1e-6 * max(1, abs(fd))
    if ctrl == S.CTRL_TABLE:  # rows of steps the rollout never reaches have no effect
        assert np.all(gp.reshape(T + 3, 3)[T:] == 0) and np.any(gp.reshape(T + 3, 3)[:T] != 0)


def test_table_controller_filled_with_a_sinusoid_is_that_sinusoid():
    """A table whose rows are the sinusoid controller's outputs reproduces its rollout exactly, and
    the chain rule between the two forms holds: dL/dA_g = sum_n dL/dU[n][g] sin(2 pi f t_n)."""
    T = 12
    sin = S.blob(2, 16, 30, 31, n_groups=3, ctrl_type=S.CTRL_SIN, freq=4.0, v_scale=0.3, radius_cells=2.0,
                 center=(0.5, 3.8 / 16), amp=3.0, bc_width=2, dt=2e-3)
    ss = O.Scene(sin)
    x0 = ss.initial_state()[0]
    U = np.stack([ss.controller(n, x0) for n in range(T)])            # a_g(t_n) with A
    basis = np.stack([ss.controller(n, x0, params=np.ones(3)) for n in range(T)])  # sin(2 pi f t_n)
    tab = sin.copy(ctrl_type=S.CTRL_TABLE, ctrl_hidden=T, ctrl_params=U.ravel())
    ts = O.Scene(tab)
    ra, rb = ss.rollout(T), ts.rollout(T)
    for a, b in zip(ra, rb):
        assert np.array_equal(a, b)
    rng = np.random.default_rng(3)
    w = rng.normal(size=ra[0][T].shape)
    gA = ss.backward(ra, (w, None, None, None))[4]
    gU = ts.backward(rb, (w, None, None, None))[4].reshape(T, 3)
    assert np.allclose(gA, np.sum(gU * basis, axis=0), rtol=1e-12, atol=1e-14 * np.abs(gU).max())


def test_domain_and_inversion_errors():
    """Readings of the grid geometry and constitutive domain: a stencil that leaves [0, n) and a
    deformation gradient with det F <= 0 are errors, never clamped."""
    sp = _blob(2, npart=5, seed=0)
    sp.x0[0] = [0.2 / 16, 0.5]
    with pytest.raises(O.OracleError, match="-3"):
        O.Scene(sp).step(np.zeros(2), *O.Scene(sp).initial_state())
    sp = _blob(2, npart=5, seed=0)
    sp.F0[1] = np.diag([1.0, -1.0])
    with pytest.raises(O.OracleError, match="-4"):
        O.Scene(sp).step(np.zeros(2), *O.Scene(sp).initial_state())
