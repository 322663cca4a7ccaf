"""Pin of the MLS stress term of Eq. 4 (CPU only): P2G's stress impulse is the grid gradient of a
discrete elastic plus actuation energy.

With v = C = 0 and no gravity, the grid momentum of Eqs. 3-5 is p_i = sum_p N_ip G_p (x_i - x_p)
with G_p = -D^{-1} dt V0 P_p F_p^T (Eq. 4) and P_p = P(F_p) + F_p sigma_a (Section III's actuation
model).  MLS-MPM obtains exactly this force from an energy: move every grid node by a virtual
displacement u_i, deform each particle's F by the MLS gradient of that displacement,

    F_p(u) = (I + sum_i u_i w_ip^T) F_p,   w_ip = D_p^{-1} N_ip (x_i - x_p),
    D_p    = sum_i N_ip (x_i - x_p)(x_i - x_p)^T,

and p_i = -dt dE/du_i at u = 0, where E(u) = sum_p V0 [psi(F_p(u)) + 1/2 a_g sum_d dir_gd (F^T F)_dd].
The last term is the energy whose F-derivative is F sigma_a with sigma_a = a_g Diag(dir_g).

The test evaluates dE/du_i by a fourth-order central difference of psi, written here. The weights
come from scipy's B-spline basis element, and D_p from its own definition, so nothing is shared
with the oracle. What it rules out, each of which every other pin misses: a wrong factor in
-D^{-1} dt V0, a transposed P F^T, sigma_a F in place of F sigma_a, and a wrong sign.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S

_BSPLINE = BSpline.basis_element([-1.5, -0.5, 0.5, 1.5], extrapolate=False)


def _psi(F, mu, la):
    """Compressible neo-Hookean energy density (the constitutive reading of Section III)."""
    d = F.shape[0]
    J = np.linalg.det(F)
    lnJ = np.log(J)
    return 0.5 * mu * (np.sum(F * F) - d) - mu * lnJ + 0.5 * la * lnJ * lnJ


def _energy(F, mu, la, a, direction):
    """psi plus the actuation energy 1/2 a sum_d dir_d (F^T F)_dd, per unit reference volume."""
    FtF_diag = np.sum(F * F, axis=0)
    return _psi(F, mu, la) + 0.5 * a * float(direction @ FtF_diag)


def _stencil(xp, dx, dim):
    """Grid nodes i with |x_i - x_p| < 1.5 dx per axis, and their weights N_ip (library B-spline)."""
    lo = np.ceil(xp / dx - 1.5).astype(int)
    nodes, weights = [], []
    for k in np.ndindex(*([3] * dim)):
        idx = lo + np.array(k)
        t = (idx * dx - xp) / dx
        if np.any(np.abs(t) >= 1.5):
            continue
        w = float(np.prod(_BSPLINE(t)))
        nodes.append(idx)
        weights.append(w)
    return np.array(nodes), np.array(weights)


def _impulse_from_energy(spec, act, x, F):
    """p_i = -dt dE/du_i by a five-point central difference in each node displacement."""
    dim, dx, dt = spec.dim, spec.dx, spec.dt
    nu = spec.nu
    E_arr = getattr(spec, "E_arr", None)
    p = {}
    for q in range(x.shape[0]):
        E = float(E_arr[q]) if E_arr is not None else spec.E
        mu = E / (2.0 * (1.0 + nu))
        la = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        g = int(spec.group[q])
        a = float(act[g]) if g >= 0 else 0.0
        direction = np.asarray(spec.act_dir[g], np.float64) if g >= 0 else np.zeros(dim)
        nodes, N = _stencil(x[q], dx, dim)
        r = nodes * dx - x[q]                          # x_i - x_p
        D = (N[:, None, None] * r[:, :, None] * r[:, None, :]).sum(axis=0)
        Dinv = np.linalg.inv(D)
        for i, idx in enumerate(nodes):
            w = Dinv @ (N[i] * r[i])
            key = tuple(idx)
            acc = p.setdefault(key, np.zeros(dim))
            for ax in range(dim):
                dF = np.outer(np.eye(dim)[ax], w) @ F[q]  # d F_p(u) / d u_{i,ax}
                h = 1e-4 / np.abs(dF).max()
                e = [_energy(F[q] + s * h * dF, mu, la, a, direction) for s in (2, 1, -1, -2)]
                dE = (-e[0] + 8 * e[1] - 8 * e[2] + e[3]) / (12 * h)
                acc[ax] += -dt * spec.p_vol * dE
    return p


def _scene(dim, seed, material):
    n = 16 if dim == 2 else 12
    spec = S.blob(dim, n, 30 if dim == 2 else 24, seed, gravity=(0.0,) * dim, f_scale=0.2 if dim == 3 else 0.25, radius_cells=2.0,
                  n_groups=3, bc_width=2, dt=1e-3, E=30.0, nu=0.3)
    dets = np.linalg.det(spec.F0)
    assert dets.min() > 0.3
    if material:
        spec = S.with_material(spec, seed + 100, spread=0.4)
    return spec


@pytest.mark.parametrize("material", [False, True], ids=["uniform", "per_particle_E"])
@pytest.mark.parametrize("dim", [2, 3])
def test_p2g_stress_impulse_is_minus_dt_energy_gradient(dim, material):
    spec = _scene(dim, 40 + dim, material)
    sc = O.Scene(spec)
    x, _, _, F = sc.initial_state()
    N = sc.N
    rng = np.random.default_rng(dim)
    act = rng.uniform(-5.0, 5.0, size=sc.G)
    zeros_v, zeros_C = np.zeros((N, dim)), np.zeros((N, dim, dim))
    _, (gm, gv) = sc.step(act, x, zeros_v, zeros_C, F, want_grid=True)
    # every stencil stays clear of the boundary band, so m_i v*_i = p_i on every active node
    band = spec.bc_width
    lo = np.floor(x / spec.dx - 0.5).astype(int)
    assert lo.min() >= band and (lo + 2).max() < spec.n_grid[0] - band
    expect = _impulse_from_energy(spec, act, x, F)
    got = np.zeros((len(expect), dim))
    want = np.zeros_like(got)
    for j, (key, val) in enumerate(sorted(expect.items())):
        lin = int(np.ravel_multi_index(key, tuple(spec.n_grid[:dim])))
        got[j] = gm[lin] * gv[lin]
        want[j] = val
    assert np.count_nonzero(gm) == len(expect)
    scale = np.abs(want).max()
    assert scale > 0
    err = np.abs(got - want).max() / scale
    assert err < 1e-8, f"stress impulse differs from -dt dE/du by {err:.3e} (relative to max)"


def test_actuation_energy_picks_F_sigma_not_sigma_F():
    """The actuation energy's F-derivative is F sigma_a (Section III), which differs from sigma_a F
    for a general F: the test above would fail for the other orientation."""
    rng = np.random.default_rng(0)
    F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    d = np.array([0.2, 0.9, -0.4])
    a = 2.5
    sig = a * np.diag(d)
    grad = np.zeros((3, 3))
    h = 1e-5
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            grad[i, j] = (_energy(F + E, 0.0, 0.0, a, d) - _energy(F - E, 0.0, 0.0, a, d)) / (2 * h)
    assert np.allclose(grad, F @ sig, rtol=0, atol=1e-8)
    assert not np.allclose(grad, sig @ F, rtol=0, atol=1e-2)
