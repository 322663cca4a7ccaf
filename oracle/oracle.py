"""ctypes wrapper around the FP64 MLS-MPM oracle (``mpm_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference arm may use this module; the library never does.  It reads scene descriptions by
attribute (dim, n_grid, dx, dt, ...; see ``paper_1810_01054_gb300.scenes.SceneSpec``) and
imports nothing from the CUDA library.

Array conventions: x, v are [N, d]; C, F are [N, d, d] (row-major); all float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmpm_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_DOMAIN, ERR_INVERTED = 0, -1, -3, -4


class OracleError(RuntimeError):
    pass


class _Scene(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n_grid", C.c_int * 3),
        ("dx", C.c_double),
        ("dt", C.c_double),
        ("gravity", C.c_double * 3),
        ("E", C.c_double),
        ("nu", C.c_double),
        ("p_mass", C.c_double),
        ("p_vol", C.c_double),
        ("bc_type", C.c_int),
        ("bc_width", C.c_int),
        ("friction_c", C.c_double),
        ("n_particles", C.c_int),
        ("n_groups", C.c_int),
        ("group", C.c_void_p),
        ("act_dir", C.c_void_p),
        ("ctrl_type", C.c_int),
        ("ctrl_hidden", C.c_int),
        ("ctrl_freq", C.c_double),
        ("ctrl_scale", C.c_double),
        ("p_E", C.c_void_p),
        ("p_m", C.c_void_p),
        ("wall_kind", C.c_void_p),
        ("wall_c", C.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no fast-math, single-threaded)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            for name in ("oracle_step", "oracle_step_adjoint", "oracle_step_adjoint_mat", "oracle_controller",
                         "oracle_controller_xv", "oracle_controller_adjoint", "oracle_controller_adjoint_xv",
                         "oracle_rollout", "oracle_backward",
                         "oracle_backward_mat", "oracle_neohookean", "oracle_bc"):
                getattr(_lib, name).restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Scene:
    """Holds a packed scene struct plus the arrays it points to (kept alive here)."""

    def __init__(self, spec):
        self.spec = spec
        d = int(spec.dim)
        self.dim = d
        self.N = int(np.asarray(spec.x0).shape[0])
        self.G = int(np.asarray(spec.act_dir).shape[0])
        self._group = np.ascontiguousarray(np.asarray(spec.group, dtype=np.int32))
        self._dir = _f64(spec.act_dir, (max(self.G, 0), d)) if self.G else np.zeros((1, d))
        s = _Scene()
        s.dim = d
        ng = list(spec.n_grid) + [1] * (3 - len(spec.n_grid))
        for a in range(3):
            s.n_grid[a] = int(ng[a])
        s.dx, s.dt = float(spec.dx), float(spec.dt)
        g = list(spec.gravity) + [0.0] * (3 - len(spec.gravity))
        for a in range(3):
            s.gravity[a] = float(g[a])
        s.E, s.nu = float(spec.E), float(spec.nu)
        s.p_mass, s.p_vol = float(spec.p_mass), float(spec.p_vol)
        s.bc_type, s.bc_width, s.friction_c = int(spec.bc_type), int(spec.bc_width), float(spec.friction_c)
        s.n_particles, s.n_groups = self.N, self.G
        s.group, s.act_dir = _p(self._group), _p(self._dir)
        s.ctrl_type, s.ctrl_hidden = int(spec.ctrl_type), int(spec.ctrl_hidden)
        s.ctrl_freq, s.ctrl_scale = float(spec.ctrl_freq), float(spec.ctrl_scale)
        # optional per-particle Young's modulus and mass (NULL: the scene's E and p_mass)
        E_arr, m_arr = getattr(spec, "E_arr", None), getattr(spec, "mass_arr", None)
        self._E = None if E_arr is None else _f64(E_arr).ravel()
        self._m = None if m_arr is None else _f64(m_arr).ravel()
        s.p_E, s.p_m = _p(self._E), _p(self._m)
        # optional per-wall boundary kinds and friction (NULL: bc_type and friction_c on every wall)
        wk, wc = getattr(spec, "wall_kind", None), getattr(spec, "wall_c", None)
        self._wk = None if wk is None else np.ascontiguousarray(np.asarray(wk, dtype=np.int32).ravel())
        self._wc = None if wc is None else _f64(wc).ravel()
        s.wall_kind, s.wall_c = _p(self._wk), _p(self._wc)
        self.struct = s
        self.params = _f64(spec.ctrl_params).ravel()
        self.n_nodes = int(np.prod(ng[:d]))

    @property
    def ref(self):
        return C.byref(self.struct)

    def _check(self, rc, what):
        if rc != OK:
            raise OracleError(f"{what} failed with status {rc}")

    def initial_state(self):
        sp = self.spec
        d, N = self.dim, self.N
        return (_f64(sp.x0, (N, d)), _f64(sp.v0, (N, d)), _f64(sp.C0, (N, d, d)), _f64(sp.F0, (N, d, d)))

    def controller(self, step, x, params=None, v=None):
        """Actuation a_g(t_step) from positions x (and velocities v, needed by the closed-loop form)."""
        params = self.params if params is None else _f64(params).ravel()
        act = np.zeros(max(self.G, 1))
        x = _f64(x)
        v = None if v is None else _f64(v)
        self._check(lib().oracle_controller_xv(self.ref, _p(params), int(step), _p(x), _p(v), _p(act)), "controller")
        return act[: self.G]

    def controller_adjoint(self, step, x, gact, params=None, v=None):
        """(dL/dparams, dL/dx) from dL/da; with v also dL/dv (closed-loop form)."""
        params = self.params if params is None else _f64(params).ravel()
        gp = np.zeros_like(params)
        gx = np.zeros((self.N, self.dim))
        gv = np.zeros((self.N, self.dim)) if v is not None else None
        x = _f64(x)
        v = None if v is None else _f64(v)
        gact = _f64(gact)
        self._check(lib().oracle_controller_adjoint_xv(self.ref, _p(params), int(step), _p(x), _p(v), _p(gact),
                                                       _p(gp), _p(gx), _p(gv)), "controller adjoint")
        return (gp, gx) if v is None else (gp, gx, gv)

    def step(self, act, x, v, Cm, F, want_grid=False):
        d, N = self.dim, self.N
        act = _f64(act) if self.G else np.zeros(1)
        x, v, Cm, F = _f64(x), _f64(v), _f64(Cm), _f64(F)
        x1, v1 = np.empty((N, d)), np.empty((N, d))
        C1, F1 = np.empty((N, d, d)), np.empty((N, d, d))
        gm = np.empty(self.n_nodes) if want_grid else None
        gv = np.empty((self.n_nodes, d)) if want_grid else None
        rc = lib().oracle_step(self.ref, _p(act), _p(x), _p(v), _p(Cm), _p(F), _p(x1), _p(v1), _p(C1), _p(F1),
                               _p(gm), _p(gv))
        self._check(rc, "step")
        if want_grid:
            return (x1, v1, C1, F1), (gm, gv)
        return x1, v1, C1, F1

    def step_adjoint(self, act, state, adj1, material=False):
        """((gx0, gv0, gC0, gF0), gact), plus (gE, gm) of this step with material=True."""
        d, N = self.dim, self.N
        act = _f64(act) if self.G else np.zeros(1)
        x, v, Cm, F = (_f64(a) for a in state)
        gx1, gv1, gC1, gF1 = (_f64(a) for a in adj1)
        gx0, gv0 = np.empty((N, d)), np.empty((N, d))
        gC0, gF0 = np.empty((N, d, d)), np.empty((N, d, d))
        gact = np.zeros(max(self.G, 1))
        gE = np.empty(N) if material else None
        gm = np.empty(N) if material else None
        rc = lib().oracle_step_adjoint_mat(self.ref, _p(act), _p(x), _p(v), _p(Cm), _p(F), _p(gx1), _p(gv1),
                                           _p(gC1), _p(gF1), _p(gx0), _p(gv0), _p(gC0), _p(gF0), _p(gact), _p(gE),
                                           _p(gm))
        self._check(rc, "step adjoint")
        if material:
            return (gx0, gv0, gC0, gF0), gact[: self.G], (gE, gm)
        return (gx0, gv0, gC0, gF0), gact[: self.G]

    def rollout(self, n_steps, state0=None, params=None):
        """Returns (xs, vs, Cs, Fs, acts) with xs [T+1, N, d] ... acts [T, G]."""
        d, N, G = self.dim, self.N, self.G
        params = self.params if params is None else _f64(params).ravel()
        x0, v0, C0, F0 = self.initial_state() if state0 is None else tuple(_f64(a) for a in state0)
        xs, vs = np.empty((n_steps + 1, N, d)), np.empty((n_steps + 1, N, d))
        Cs, Fs = np.empty((n_steps + 1, N, d, d)), np.empty((n_steps + 1, N, d, d))
        acts = np.empty((max(n_steps, 1), max(G, 1)))
        rc = lib().oracle_rollout(self.ref, _p(params), int(n_steps), _p(x0), _p(v0), _p(C0), _p(F0), _p(xs),
                                  _p(vs), _p(Cs), _p(Fs), _p(acts))
        self._check(rc, "rollout")
        return xs, vs, Cs, Fs, acts[:n_steps, :G]

    def backward(self, traj, seeds, params=None, material=False):
        """traj from rollout(); seeds = (gxT, gvT, gCT, gFT) with None for zero.
        Returns (gx0, gv0, gC0, gF0, gparams), plus (dL/dE_p, dL/dm_p) with material=True."""
        d, N, G = self.dim, self.N, self.G
        params = self.params if params is None else _f64(params).ravel()
        xs, vs, Cs, Fs, acts = traj
        T = xs.shape[0] - 1
        acts_full = np.zeros((max(T, 1), max(G, 1)))
        acts_full[:T, :G] = acts
        acts_p = _f64(acts_full) if G else np.zeros((max(T, 1), 1))
        sd = [None if a is None else _f64(a) for a in seeds]
        gx0, gv0 = np.empty((N, d)), np.empty((N, d))
        gC0, gF0 = np.empty((N, d, d)), np.empty((N, d, d))
        gp = np.zeros(max(params.size, 1))
        if G == 0:
            acts_p = np.zeros((max(T, 1), 1))
        gE = np.empty(N) if material else None
        gm = np.empty(N) if material else None
        rc = lib().oracle_backward_mat(self.ref, _p(params), int(params.size), int(T), _p(_f64(xs)),
                                       _p(_f64(vs)), _p(_f64(Cs)), _p(_f64(Fs)), _p(acts_p if G else np.zeros(1)),
                                       _p(sd[0]), _p(sd[1]), _p(sd[2]), _p(sd[3]), _p(gx0), _p(gv0), _p(gC0),
                                       _p(gF0), _p(gp), _p(gE), _p(gm))
        self._check(rc, "backward")
        if material:
            return gx0, gv0, gC0, gF0, gp[: params.size], gE, gm
        return gx0, gv0, gC0, gF0, gp[: params.size]


def neohookean(F, E, nu, Pbar=None):
    """(P, H_psi[Pbar]) for one d x d deformation gradient."""
    F = _f64(F)
    d = F.shape[0]
    P = np.empty((d, d))
    HP = np.empty((d, d)) if Pbar is not None else None
    pb = _f64(Pbar) if Pbar is not None else None
    rc = lib().oracle_neohookean(int(d), C.c_double(E), C.c_double(nu), _p(F), _p(pb), _p(P), _p(HP))
    if rc != OK:
        raise OracleError(f"neohookean failed with status {rc}")
    return P, HP


def bc(scene: Scene, idx, vin, gout=None):
    """Boundary projection of one node velocity (and its adjoint if ``gout`` is given)."""
    d = scene.dim
    idx_a = np.zeros(3, dtype=np.int32)
    idx_a[:d] = idx
    vin = _f64(vin)
    vout = np.empty(d)
    gin = np.empty(d) if gout is not None else None
    go = _f64(gout) if gout is not None else None
    lib().oracle_bc(scene.ref, _p(idx_a), _p(vin), _p(vout), _p(go), _p(gin))
    return (vout, gin) if gout is not None else vout
