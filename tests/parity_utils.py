"""Shared helpers of the GPU parity tests: comparison metrics and oracle drivers."""
import numpy as np

from oracle import oracle as O

# Tolerances stated for this method: forward within relative 1e-4 of the FP64 oracle on
# positions and velocities over 10-step windows; gradients within relative 1e-3 with cosine
# similarity >= 0.999 over full horizons.  Relative error = ||a - b||_2 / ||b||_2 over the whole
# array (the paper leaves "relative error" undefined; this is the reading used throughout).
FWD_TOL = 1e-4
GRAD_TOL = 1e-3
GRAD_COS = 0.999


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cosine(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-300))


def max_scaled(a, b):
    """max |a - b| over max |b|: an element-wise bound that a localised error cannot hide in."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def assert_state_close(gpu, ref, tol=FWD_TOL, names=("x", "v", "C", "F"), elem_tol=None):
    elem_tol = 10 * tol if elem_tol is None else elem_tol
    for name, a, b in zip(names, gpu, ref):
        r = rel_l2(a, b)
        m = max_scaled(a, b)
        assert r <= tol, f"{name}: relative L2 {r:.3e} > {tol:.1e}"
        assert m <= elem_tol, f"{name}: max scaled error {m:.3e} > {elem_tol:.1e}"


def assert_grad_close(gpu, ref, name, tol=GRAD_TOL, cos=GRAD_COS, elem_tol=None):
    """Whole-array relative L2 and cosine, plus an element-wise bound (max |a - b| over max |b|,
    10x the relative tolerance) that a wrong gradient on a few particles cannot hide under."""
    elem_tol = 10 * tol if elem_tol is None else elem_tol
    r = rel_l2(gpu, ref)
    c = cosine(gpu, ref)
    m = max_scaled(gpu, ref) if np.size(ref) else 0.0
    assert r <= tol and c >= cos and m <= elem_tol, (
        f"{name}: relative L2 {r:.3e} (tol {tol:.0e}), cosine {c:.6f} (min {cos}), "
        f"max scaled {m:.3e} (tol {elem_tol:.0e})")


def oracle_step_from(spec, state, step):
    sc = O.Scene(spec)
    act = sc.controller(step, state[0], v=state[1])
    return sc.step(act, *state)


def mean_x0_seed(N, dim):
    g = np.zeros((N, dim))
    g[:, 0] = 1.0 / N
    return g
