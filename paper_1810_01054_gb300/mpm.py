"""Thin ctypes binding of libgbmpm (include/mpm.h): argument marshalling only.

Every step of the simulation and of its reverse pass runs in the library's CUDA kernels.  The
library must have been built (``python -m paper_1810_01054_gb300.build``); importing this module
without it, or calling it without a CUDA device, raises -- there is no CPU fallback.

Arrays cross the boundary as FP32, row-major: x, v [N, d]; C, F [N, d, d].  numpy arrays use
host pointers (mem_space 0); torch CUDA tensors use device pointers (mem_space 1).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbmpm.so")

MPM_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of device memory or budget", -3: "stencil left the grid",
          -4: "det F <= 0", -5: "bounded device wait expired", -6: "CUDA error", -7: "call out of order",
          -8: "too many particles in one tile", -9: "internal consistency check failed"}
IMPL_TILED, IMPL_PLAIN = 0, 1


class MPMError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({STATUS.get(status, 'unknown')})")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n_grid", C.c_int * 3),
        ("dx", C.c_float),
        ("dt", C.c_float),
        ("gravity", C.c_float * 3),
        ("E", C.c_float),
        ("nu", C.c_float),
        ("p_mass", C.c_float),
        ("p_vol", C.c_float),
        ("bc_type", C.c_int),
        ("bc_width", C.c_int),
        ("friction_c", C.c_float),
        ("n_particles", C.c_int),
        ("x0", C.c_void_p),
        ("v0", C.c_void_p),
        ("C0", C.c_void_p),
        ("F0", C.c_void_p),
        ("group", C.c_void_p),
        ("n_groups", C.c_int),
        ("act_dir", C.c_void_p),
        ("ctrl_type", C.c_int),
        ("ctrl_hidden", C.c_int),
        ("ctrl_freq", C.c_float),
        ("ctrl_scale", C.c_float),
        ("n_ctrl_params", C.c_int),
        ("ctrl_params", C.c_void_p),
        ("impl", C.c_int),
        ("mem_space", C.c_int),
        ("tile_edge", C.c_int),
    ]


class NoAllocStep(C.Structure):
    """Mirror of mpm_noalloc_step (include/mpm.h)."""
    _fields_ = [
        ("device", C.c_int),
        ("dim", C.c_int),
        ("n_grid", C.c_int * 3),
        ("dx", C.c_float),
        ("dt", C.c_float),
        ("gravity", C.c_float * 3),
        ("E", C.c_float),
        ("nu", C.c_float),
        ("p_mass", C.c_float),
        ("p_vol", C.c_float),
        ("bc_type", C.c_int),
        ("bc_width", C.c_int),
        ("friction_c", C.c_float),
        ("n_particles", C.c_int),
        ("x", C.c_void_p),
        ("v", C.c_void_p),
        ("C", C.c_void_p),
        ("F", C.c_void_p),
        ("group", C.c_void_p),
        ("n_groups", C.c_int),
        ("act_dir", C.c_void_p),
        ("act", C.c_void_p),
        ("x_out", C.c_void_p),
        ("v_out", C.c_void_p),
        ("C_out", C.c_void_p),
        ("F_out", C.c_void_p),
        ("status", C.c_void_p),
    ]


class SceneDesc64(C.Structure):
    """Mirror of mpm_scene64_desc (include/mpm.h)."""
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
        ("bc_width", C.c_int),
        ("wall_kind", C.c_int * 6),
        ("wall_c", C.c_double * 6),
        ("n_particles", C.c_int),
        ("x0", C.c_void_p),
        ("v0", C.c_void_p),
        ("C0", C.c_void_p),
        ("F0", C.c_void_p),
        ("group", C.c_void_p),
        ("n_groups", C.c_int),
        ("act_dir", C.c_void_p),
        ("n_act_steps", C.c_int),
        ("act", C.c_void_p),
    ]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "mpm_ctx_create": [C.POINTER(C.c_void_p), C.c_int, C.c_void_p],
    "mpm_ctx_destroy": [C.c_void_p],
    "mpm_sync": [C.c_void_p],
    "mpm_status_str": [C.c_int],
    "mpm_scene_create": [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(C.c_void_p)],
    "mpm_scene_destroy": [C.c_void_p],
    "mpm_scene_tile_edge": [C.c_void_p, C.POINTER(C.c_int)],
    "mpm_step": [C.c_void_p, C.c_int],
    "mpm_rollout": [C.c_void_p, C.c_int, C.c_int, C.c_size_t],
    "mpm_backward": [C.c_void_p] + [C.c_void_p] * 9 + [C.c_int],
    "mpm_get_state": [C.c_void_p, C.c_int] + [C.c_void_p] * 4 + [C.c_int],
    "mpm_get_gradients": [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int],
    "mpm_set_state": [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int, C.c_int],
    "mpm_set_ctrl_params": [C.c_void_p, C.c_void_p, C.c_int, C.c_int],
    "mpm_get_grid": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
    "mpm_scene_info": [C.c_void_p] + [C.POINTER(C.c_int)] * 4 + [C.POINTER(C.c_size_t)],
    "mpm_batch_create": [C.c_void_p, C.c_int, C.c_size_t, C.POINTER(C.c_void_p)],
    "mpm_batch_destroy": [C.c_void_p],
    "mpm_batch_admit": [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)],
    "mpm_batch_tick": [C.c_void_p, C.c_int],
    "mpm_batch_poll": [C.c_void_p, C.c_int, C.POINTER(C.c_int)],
    "mpm_batch_release": [C.c_void_p, C.c_int],
    "mpm_profile_start": [C.c_void_p, C.c_uint, C.c_int],
    "mpm_profile_read": [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "mpm_launch_count": [C.POINTER(C.c_longlong)],
    "mpm_plan_checkpoints": [C.c_int, C.c_longlong, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                             C.POINTER(C.c_int)],
    "mpm_scene_plan_rollout": [C.c_void_p, C.c_int, C.c_int, C.c_size_t, C.POINTER(C.c_int),
                               C.POINTER(C.c_longlong), C.POINTER(C.c_int)],
    "mpm_step_noalloc": [C.POINTER(NoAllocStep), C.c_void_p],
    "mpm_scene_set_tuning": [C.c_void_p, C.c_int],
    "mpm_scene_set_material": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
    "mpm_scene_set_walls": [C.c_void_p, C.c_void_p, C.c_void_p],
    "mpm_get_material_gradients": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
    "mpm_scene_launch": [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "mpm_tune_cache_lookup": [C.c_int, C.c_longlong, C.c_longlong, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "mpm_tune_cache_store": [C.c_int, C.c_longlong, C.c_longlong, C.c_int, C.POINTER(C.c_int)],
    "mpm_tune_cache_save": [C.c_char_p],
    "mpm_tune_cache_load": [C.c_char_p],
    "mpm_tune_tile_edge": [C.c_void_p, C.POINTER(SceneDesc), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)],
    "mpm64_create": [C.c_void_p, C.POINTER(SceneDesc64), C.POINTER(C.c_void_p)],
    "mpm64_destroy": [C.c_void_p],
    "mpm64_set_state": [C.c_void_p] + [C.c_void_p] * 4,
    "mpm64_set_actuation": [C.c_void_p, C.c_void_p, C.c_int],
    "mpm64_rollout": [C.c_void_p, C.c_int],
    "mpm64_get_state": [C.c_void_p, C.c_int] + [C.c_void_p] * 4,
    "mpm64_backward": [C.c_void_p] + [C.c_void_p] * 9,
    "mpm64_info": [C.c_void_p] + [C.POINTER(C.c_int)] * 4,
}

K_SORT, K_P2G, K_GRID, K_G2P, K_P2G_ADJ, K_GRID_ADJ, K_ADJ_GATHER, K_CTRL, K_PLAIN = range(9)
K_F64_P2G, K_F64_GRID, K_F64_G2P, K_F64_P2G_ADJ, K_F64_ADJ = range(9, 14)
TUNE_OFF, TUNE_AUTO, TUNE_FORCE = 0, 1, 2
TK_P2G, TK_G2P, TK_P2G_ADJ, TK_ADJ_GATHER = range(4)
TILE_KERNELS = ["p2g", "g2p", "p2g_adj", "adj_gather"]
KERNEL_NAMES = ["sort", "p2g", "grid", "g2p", "p2g_adj", "grid_adj", "adj_gather", "ctrl", "plain",
                "f64_p2g", "f64_grid", "f64_g2p", "f64_p2g_adj", "f64_adj"]


def launch_count() -> int:
    n = C.c_longlong()
    _check(lib().mpm_launch_count(C.byref(n)), "mpm_launch_count")
    return int(n.value)


def plan_checkpoints(n_steps: int, budget_states: int):
    """(forward steps over the rollout and its reverse pass, states stored at most, multi-level?)
    of the checkpoint schedule mpm_rollout takes for a budget of ``budget_states`` states."""
    f, u, m = C.c_longlong(), C.c_int(), C.c_int()
    _check(lib().mpm_plan_checkpoints(int(n_steps), int(budget_states), C.byref(f), C.byref(u), C.byref(m)),
           "mpm_plan_checkpoints")
    return f.value, u.value, bool(m.value)


def tune_cache_lookup(dim: int, particles: int, grid_tiles: int, sm_count: int):
    """Launch shapes [(ctas_per_sm, threads)] * 4 of the cache entry of this workload key, or None."""
    shape, found = (C.c_int * 8)(), C.c_int(0)
    _check(lib().mpm_tune_cache_lookup(int(dim), int(particles), int(grid_tiles), int(sm_count), shape,
                                       C.byref(found)), "mpm_tune_cache_lookup")
    return [(shape[2 * k], shape[2 * k + 1]) for k in range(4)] if found.value else None


def tune_cache_store(dim: int, particles: int, grid_tiles: int, sm_count: int, shapes):
    flat = (C.c_int * 8)(*[int(v) for sh in shapes for v in sh])
    _check(lib().mpm_tune_cache_store(int(dim), int(particles), int(grid_tiles), int(sm_count), flat),
           "mpm_tune_cache_store")


def tune_tile_edge(ctx, spec, steps: int = 64):
    """Times ``steps`` forward steps and their reverse pass of ``spec`` with 4 x 4- and with
    8 x 8-cell tiles (2D tiled scenes; 3D has one tile shape) and caches the faster edge for the
    workload, which scenes created afterwards with tile_edge 0 take.  Returns (edge, ms per step
    with 4 x 4, ms per step with 8 x 8); the times are 0 where nothing ran."""
    desc, keep, _, _ = _scene_desc(spec)
    edge = C.c_int()
    ms = (C.c_float * 2)()
    _check(lib().mpm_tune_tile_edge(ctx.handle, C.byref(desc), int(steps), C.byref(edge), ms), "mpm_tune_tile_edge")
    del keep
    return int(edge.value), float(ms[0]), float(ms[1])


def tune_cache_save(path: str):
    _check(lib().mpm_tune_cache_save(os.fsencode(path)), "mpm_tune_cache_save")


def tune_cache_load(path: str):
    _check(lib().mpm_tune_cache_load(os.fsencode(path)), "mpm_tune_cache_load")


def lib():
    """Loads libgbmpm.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1810_01054_gb300.build`")
            L = C.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_char_p if name == "mpm_status_str" else C.c_int
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != MPM_OK:
        raise MPMError(status, what)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _f32(a, shape):
    if a is None:
        return None
    if _is_torch(a):
        import torch
        t = a.detach().to(dtype=torch.float32).contiguous()
        if tuple(t.shape) != tuple(shape):
            t = t.reshape(shape)
        return t
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))


class Context:
    """A CUDA device plus the stream every call of its scenes enqueues on.  ``stream`` may be a
    torch.cuda.Stream (or raw cudaStream_t int); None creates a private stream."""

    def __init__(self, device: int = 0, stream=None):
        self.handle = None
        self._children = weakref.WeakSet()  # live scenes and batches, closed before the context
        raw = None
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream))
            # handle 0 is the legacy default stream, which the C ABI spells cudaStreamLegacy (0x1);
            # a NULL stream would make the library create a private one
            raw = C.c_void_p(handle if handle != 0 else 1)
        h = C.c_void_p()
        _check(lib().mpm_ctx_create(C.byref(h), int(device), raw), "mpm_ctx_create")
        self.handle = h
        self.device = device

    def sync(self):
        _check(lib().mpm_sync(self.handle), "mpm_sync")

    def profile_start(self, kinds, max_launches: int = 1 << 16):
        mask = 0
        for k in kinds:
            mask |= 1 << int(k)
        _check(lib().mpm_profile_start(self.handle, mask, int(max_launches)), "mpm_profile_start")

    def profile_read(self, kind):
        n, t = C.c_int(), C.c_double()
        _check(lib().mpm_profile_read(self.handle, int(kind), C.byref(n), C.byref(t)), "mpm_profile_read")
        return n.value, t.value

    def _adopt(self, child):
        self._children.add(child)

    def close(self):
        """Closes the context's batches, then its scenes, then the context itself."""
        if self.handle:
            kids = list(self._children)
            for k in kids:
                if isinstance(k, Batch):
                    k.close()
            for k in kids:
                k.close()
            _check(lib().mpm_ctx_destroy(self.handle), "mpm_ctx_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scene_desc(spec, impl=None, params=None):
    """SceneDesc of ``spec`` with the arrays it points to (kept alive by the caller), the controller
    parameter count and the number of actuation groups."""
    impl = IMPL_TILED if impl is None else impl
    d = int(spec.dim)
    N = int(np.asarray(spec.x0).shape[0]) if not _is_torch(spec.x0) else int(spec.x0.shape[0])
    G = int(np.asarray(spec.act_dir).shape[0])
    keep = []
    dev = _is_torch(spec.x0) and spec.x0.is_cuda

    def arr(a, shape):
        t = _f32(a, shape)
        keep.append(t)
        return t

    desc = SceneDesc()
    desc.dim = d
    ng = list(spec.n_grid) + [1] * (3 - len(spec.n_grid))
    for a in range(3):
        desc.n_grid[a] = int(ng[a])
    desc.dx, desc.dt = float(spec.dx), float(spec.dt)
    g = list(spec.gravity) + [0.0] * (3 - len(spec.gravity))
    for a in range(3):
        desc.gravity[a] = float(g[a])
    desc.E, desc.nu = float(spec.E), float(spec.nu)
    desc.p_mass, desc.p_vol = float(spec.p_mass), float(spec.p_vol)
    desc.bc_type, desc.bc_width, desc.friction_c = int(spec.bc_type), int(spec.bc_width), float(spec.friction_c)
    desc.n_particles = N
    desc.x0 = _ptr(arr(spec.x0, (N, d)))
    desc.v0 = _ptr(arr(spec.v0, (N, d))) if spec.v0 is not None else None
    desc.C0 = _ptr(arr(spec.C0, (N, d, d))) if spec.C0 is not None else None
    desc.F0 = _ptr(arr(spec.F0, (N, d, d))) if spec.F0 is not None else None
    if dev:
        import torch
        grp = torch.as_tensor(spec.group, dtype=torch.int32, device=spec.x0.device).contiguous()
        params_t = torch.as_tensor(spec.ctrl_params if params is None else params, dtype=torch.float32,
                                   device=spec.x0.device).contiguous()
        dirs = torch.as_tensor(spec.act_dir, dtype=torch.float32, device=spec.x0.device).contiguous()
    else:
        grp = np.ascontiguousarray(np.asarray(spec.group, dtype=np.int32))
        params_t = np.ascontiguousarray(np.asarray(spec.ctrl_params if params is None else params,
                                                   dtype=np.float32).ravel())
        dirs = np.ascontiguousarray(np.asarray(spec.act_dir, dtype=np.float32).reshape(G, d) if G else
                                    np.zeros((1, d), np.float32))
    keep += [grp, params_t, dirs]
    desc.group = _ptr(grp)
    desc.n_groups = G
    desc.act_dir = _ptr(dirs)
    desc.ctrl_type, desc.ctrl_hidden = int(spec.ctrl_type), int(spec.ctrl_hidden)
    desc.ctrl_freq, desc.ctrl_scale = float(spec.ctrl_freq), float(spec.ctrl_scale)
    n_params = int(params_t.numel() if _is_torch(params_t) else params_t.size)
    desc.n_ctrl_params = n_params
    desc.ctrl_params = _ptr(params_t)
    desc.impl = int(impl)
    desc.mem_space = 1 if dev else 0
    desc.tile_edge = int(getattr(spec, "tile_edge", 0) or 0)
    return desc, keep, n_params, G


class Scene:
    """One simulation (state, grid, controller) living on the GPU."""

    def __init__(self, ctx: Context, spec, impl: int = IMPL_TILED, params=None):
        d = int(spec.dim)
        self.ctx, self.dim = ctx, d
        self.spec = spec
        N = int(np.asarray(spec.x0).shape[0]) if not _is_torch(spec.x0) else int(spec.x0.shape[0])
        self.N = N
        desc, keep, self.n_params, G = _scene_desc(spec, impl, params)
        h = C.c_void_p()
        _check(lib().mpm_scene_create(ctx.handle, C.byref(desc), C.byref(h)), "mpm_scene_create")
        self.handle = h
        ctx._adopt(self)
        E_arr, m_arr = getattr(spec, "E_arr", None), getattr(spec, "mass_arr", None)
        if E_arr is not None or m_arr is not None:
            self.set_material(E_arr, m_arr)
        wk, wc = getattr(spec, "wall_kind", None), getattr(spec, "wall_c", None)
        if wk is not None or wc is not None:
            self.set_walls(wk, wc)
        self.G = G
        self.impl = impl

    # Every call that changes what the next reverse pass would differentiate (the state, the
    # rollout, the parameters, the material, the walls, a batch admission) bumps ``generation``;
    # the autograd Function records it and refuses a backward through a later rollout.
    generation = 0

    def _touch(self):
        self.generation += 1

    @property
    def tile_edge(self) -> int:
        """Cells per tile edge the library uses for this scene (4, or 8 for sparse 2D scenes)."""
        e = C.c_int()
        _check(lib().mpm_scene_tile_edge(self.handle, C.byref(e)), "mpm_scene_tile_edge")
        return e.value

    # ------------------------------------------------------------------ forward
    def step(self, n: int = 1):
        self._touch()
        _check(lib().mpm_step(self.handle, int(n)), "mpm_step")

    def set_tuning(self, mode: int):
        """TUNE_OFF (default shapes), TUNE_AUTO (cache, else trials: the default) or TUNE_FORCE."""
        _check(lib().mpm_scene_set_tuning(self.handle, int(mode)), "mpm_scene_set_tuning")

    def launch(self, kernel: int):
        """(ctas_per_sm, threads, tuned) of tile kernel TK_*."""
        a, t, d = C.c_int(), C.c_int(), C.c_int()
        _check(lib().mpm_scene_launch(self.handle, int(kernel), C.byref(a), C.byref(t), C.byref(d)),
               "mpm_scene_launch")
        return a.value, t.value, bool(d.value)

    def rollout(self, n_steps: int, ckpt_interval: int = 0, mem_budget: int = 0):
        self._touch()
        _check(lib().mpm_rollout(self.handle, int(n_steps), int(ckpt_interval), C.c_size_t(int(mem_budget))),
               "mpm_rollout")

    def sync(self):
        self.ctx.sync()

    # ------------------------------------------------------------------ state
    def get_state(self, step: int = -1, out=None):
        """Returns (x, v, C, F) as numpy arrays (or fills the given torch CUDA tensors)."""
        N, d = self.N, self.dim
        if out is not None:
            x, v, Cm, F = out
            _check(lib().mpm_get_state(self.handle, int(step), _ptr(x), _ptr(v), _ptr(Cm), _ptr(F), 1),
                   "mpm_get_state")
            return out
        x, v = np.empty((N, d), np.float32), np.empty((N, d), np.float32)
        Cm, F = np.empty((N, d, d), np.float32), np.empty((N, d, d), np.float32)
        _check(lib().mpm_get_state(self.handle, int(step), _ptr(x), _ptr(v), _ptr(Cm), _ptr(F), 0), "mpm_get_state")
        return x, v, Cm, F

    def set_state(self, x, v=None, Cm=None, F=None, step: int = -1):
        N, d = self.N, self.dim
        dev = _is_torch(x) and x.is_cuda
        arrs = [_f32(x, (N, d)), _f32(v, (N, d)), _f32(Cm, (N, d, d)), _f32(F, (N, d, d))]
        self._touch()
        _check(lib().mpm_set_state(self.handle, *[_ptr(a) for a in arrs], int(step), 1 if dev else 0),
               "mpm_set_state")

    def set_params(self, params):
        dev = _is_torch(params) and params.is_cuda
        p = _f32(params, (self.n_params,))
        self._touch()
        _check(lib().mpm_set_ctrl_params(self.handle, _ptr(p), self.n_params, 1 if dev else 0), "mpm_set_ctrl_params")

    def get_grid(self):
        n = int(np.prod(list(self.spec.n_grid)))
        m = np.empty(n, np.float32)
        v = np.empty((n, self.dim), np.float32)
        _check(lib().mpm_get_grid(self.handle, _ptr(m), _ptr(v), 0), "mpm_get_grid")
        return m, v

    def plan_rollout(self, n_steps: int, k: int = 0, budget: int = 0):
        """(interval, forward steps of the rollout and its reverse pass, multi-level?) of
        ``rollout(n_steps, k, budget)``; the interval is 0 with the multi-level store."""
        kk, f, m = C.c_int(), C.c_longlong(), C.c_int()
        _check(lib().mpm_scene_plan_rollout(self.handle, int(n_steps), int(k), int(budget), C.byref(kk), C.byref(f),
                                            C.byref(m)), "mpm_scene_plan_rollout")
        return int(kk.value), int(f.value), bool(m.value)

    def info(self):
        a, b, c, s = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        sb = C.c_size_t()
        _check(lib().mpm_scene_info(self.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(s), C.byref(sb)),
               "mpm_scene_info")
        return dict(n_particles=a.value, n_groups=b.value, n_ctrl_params=c.value, step=s.value,
                    state_bytes=sb.value)

    # ------------------------------------------------------------------ reverse
    def backward(self, gx=None, gv=None, gC=None, gF=None, out=None):
        """Reverse pass of the last rollout.  Seeds are dL/d(final state) (None = 0).  Returns
        (gx0, gv0, gC0, gF0, g_params) as numpy arrays, or fills ``out`` (torch CUDA tensors, the
        same five in that order) and returns it."""
        N, d = self.N, self.dim
        seeds = [_f32(gx, (N, d)), _f32(gv, (N, d)), _f32(gC, (N, d, d)), _f32(gF, (N, d, d))]
        if out is not None:
            on_dev = bool(out[0].is_cuda)
            for sd in seeds:
                if sd is not None and (not _is_torch(sd) or bool(sd.is_cuda) != on_dev):
                    raise ValueError("seeds and outputs must live in the same memory space")
            _check(lib().mpm_backward(self.handle, *[_ptr(a) for a in seeds], *[_ptr(a) for a in out],
                                      1 if on_dev else 0), "mpm_backward")
            return out
        if any(_is_torch(sd) for sd in seeds if sd is not None):
            seeds = [None if sd is None else sd.detach().cpu().numpy() for sd in seeds]
        gx0, gv0 = np.empty((N, d), np.float32), np.empty((N, d), np.float32)
        gC0, gF0 = np.empty((N, d, d), np.float32), np.empty((N, d, d), np.float32)
        gp = np.empty(max(self.n_params, 1), np.float32)
        _check(lib().mpm_backward(self.handle, *[_ptr(a) for a in seeds], _ptr(gx0), _ptr(gv0), _ptr(gC0), _ptr(gF0),
                                  _ptr(gp), 0), "mpm_backward")
        return gx0, gv0, gC0, gF0, gp[: self.n_params]

    def set_material(self, E=None, mass=None):
        """Per-particle Young's modulus and mass [N] (None keeps the scene's value); host arrays or
        CUDA tensors.  Enables dL/dE_p, dL/dm_p in the reverse pass (material_gradients)."""
        arrs = [a for a in (E, mass) if a is not None]
        on_dev = bool(arrs) and _is_torch(arrs[0]) and arrs[0].is_cuda
        conv = []
        for a in (E, mass):
            if a is None:
                conv.append(None)
            elif on_dev:
                conv.append(a.float().contiguous())
            else:
                conv.append(np.ascontiguousarray(np.asarray(a, np.float32).ravel()))
        for a in conv:
            if a is not None and (a.numel() if _is_torch(a) else a.size) != self.N:
                raise ValueError("per-particle material arrays need one entry per particle")
        self._touch()
        _check(lib().mpm_scene_set_material(self.handle, _ptr(conv[0]), _ptr(conv[1]), 1 if on_dev else 0),
               "mpm_scene_set_material")

    def set_walls(self, kind=None, c=None):
        """Per-wall boundary: kind[2 dim] (BC_STICKY / BC_SLIP / BC_OPEN), friction c[2 dim];
        wall w = 2 axis + side, low side first.  None keeps the current values."""
        nw = 2 * self.dim
        k = None if kind is None else np.ascontiguousarray(np.asarray(kind, np.int32).ravel())
        cc = None if c is None else np.ascontiguousarray(np.asarray(c, np.float32).ravel())
        for a in (k, cc):
            if a is not None and a.size != nw:
                raise ValueError(f"per-wall arrays need {nw} entries")
        self._touch()
        _check(lib().mpm_scene_set_walls(self.handle, _ptr(k), _ptr(cc)), "mpm_scene_set_walls")

    def material_gradients(self):
        """(dL/dE_p, dL/dm_p) [N] of the last finished reverse pass (per-particle material only)."""
        gE, gm = np.empty(self.N, np.float32), np.empty(self.N, np.float32)
        _check(lib().mpm_get_material_gradients(self.handle, _ptr(gE), _ptr(gm), 0), "mpm_get_material_gradients")
        return gE, gm

    def gradients(self, out=None):
        """Result of the last finished reverse pass (mpm_backward or a batched gradient request):
        (gx0, gv0, gC0, gF0, g_params) as numpy arrays, or filled into ``out`` (torch tensors)."""
        N, d = self.N, self.dim
        if out is not None:
            on_dev = bool(out[0].is_cuda)
            _check(lib().mpm_get_gradients(self.handle, *[_ptr(a) for a in out], 1 if on_dev else 0),
                   "mpm_get_gradients")
            return out
        gx0, gv0 = np.empty((N, d), np.float32), np.empty((N, d), np.float32)
        gC0, gF0 = np.empty((N, d, d), np.float32), np.empty((N, d, d), np.float32)
        gp = np.empty(max(self.n_params, 1), np.float32)
        _check(lib().mpm_get_gradients(self.handle, _ptr(gx0), _ptr(gv0), _ptr(gC0), _ptr(gF0), _ptr(gp), 0),
               "mpm_get_gradients")
        return gx0, gv0, gC0, gF0, gp[: self.n_params]

    def close(self):
        """Frees the scene (MPMError while a batch still holds it: release or close the batch)."""
        if getattr(self, "handle", None):
            _check(lib().mpm_scene_destroy(self.handle), "mpm_scene_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f64(a, shape):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


class Scene64:
    """The double-precision plain form (mpm64_*): one scene in FP64 on the GPU for accuracy
    studies (Section VI, float64 cases).  Host numpy arrays in and out.  Actuation is a per-step
    table: the spec's MPM_CTRL_TABLE parameters, or ``act`` [L, G] given here (required for other
    controller families with groups; pass np.zeros((0, G)) for a passive run)."""

    def __init__(self, ctx: Context, spec, act=None):
        if getattr(spec, "E_arr", None) is not None or getattr(spec, "mass_arr", None) is not None:
            raise ValueError("the FP64 form takes a uniform material")
        d = int(spec.dim)
        self.ctx, self.dim, self.spec = ctx, d, spec
        N = int(np.asarray(spec.x0).shape[0])
        G = int(np.asarray(spec.act_dir).shape[0])
        self.N, self.G = N, G
        if act is None:
            if int(spec.ctrl_type) == 3:  # MPM_CTRL_TABLE
                act = np.asarray(spec.ctrl_params, np.float64).reshape(int(spec.ctrl_hidden), G)
            elif G > 0:
                raise ValueError("the FP64 form takes actuation as a per-step table: pass act=[L, G]")
            else:
                act = np.zeros((0, 0))
        self._keep = []

        def arr(a, shape):
            t = _f64(a, shape)
            self._keep.append(t)
            return _ptr(t)

        desc = SceneDesc64()
        desc.dim = d
        ng = list(spec.n_grid) + [1] * (3 - len(spec.n_grid))
        for a in range(3):
            desc.n_grid[a] = int(ng[a])
        desc.dx, desc.dt = float(spec.dx), float(spec.dt)
        g = list(spec.gravity) + [0.0] * (3 - len(spec.gravity))
        for a in range(3):
            desc.gravity[a] = float(g[a])
        desc.E, desc.nu = float(spec.E), float(spec.nu)
        desc.p_mass, desc.p_vol = float(spec.p_mass), float(spec.p_vol)
        desc.bc_width = int(spec.bc_width)
        kinds = spec.wall_kind if getattr(spec, "wall_kind", None) is not None else [spec.bc_type] * (2 * d)
        cs = spec.wall_c if getattr(spec, "wall_c", None) is not None else [spec.friction_c] * (2 * d)
        for w in range(6):
            desc.wall_kind[w] = int(kinds[w]) if w < 2 * d else 2
            desc.wall_c[w] = float(cs[w]) if w < 2 * d else 0.0
        desc.n_particles = N
        desc.x0 = arr(spec.x0, (N, d))
        desc.v0 = arr(spec.v0, (N, d)) if spec.v0 is not None else None
        desc.C0 = arr(spec.C0, (N, d, d)) if spec.C0 is not None else None
        desc.F0 = arr(spec.F0, (N, d, d)) if spec.F0 is not None else None
        grp = np.ascontiguousarray(np.asarray(spec.group, dtype=np.int32).reshape(N))
        self._keep.append(grp)
        desc.group = _ptr(grp)
        desc.n_groups = G
        desc.act_dir = arr(spec.act_dir, (max(G, 1), d)) if G else None
        act = np.asarray(act, np.float64)
        self.L = int(act.shape[0]) if act.size or act.ndim == 2 else 0
        desc.n_act_steps = self.L
        desc.act = arr(act, (self.L, G)) if self.L * G else None
        h = C.c_void_p()
        _check(lib().mpm64_create(ctx.handle, C.byref(desc), C.byref(h)), "mpm64_create")
        self._keep = []
        self.handle = h
        ctx._adopt(self)

    def set_state(self, x, v=None, C_=None, F=None):
        d, N = self.dim, self.N
        a = [_f64(x, (N, d)), _f64(v, (N, d)), _f64(C_, (N, d, d)), _f64(F, (N, d, d))]
        _check(lib().mpm64_set_state(self.handle, *[_ptr(t) for t in a]), "mpm64_set_state")

    def set_actuation(self, U):
        U = np.ascontiguousarray(np.asarray(U, np.float64).reshape(-1, self.G))
        _check(lib().mpm64_set_actuation(self.handle, _ptr(U), int(U.shape[0])), "mpm64_set_actuation")
        self.L = int(U.shape[0])

    def rollout(self, n_steps: int):
        _check(lib().mpm64_rollout(self.handle, int(n_steps)), "mpm64_rollout")

    def get_state(self, step: int = -1):
        d, N = self.dim, self.N
        out = [np.empty((N, d)), np.empty((N, d)), np.empty((N, d, d)), np.empty((N, d, d))]
        _check(lib().mpm64_get_state(self.handle, int(step), *[_ptr(t) for t in out]), "mpm64_get_state")
        return tuple(out)

    def backward(self, gx=None, gv=None, gC=None, gF=None):
        """dL/d(initial x, v, C, F) and dL/dU [L, G] for seeds dL/d(final x, v, C, F)."""
        d, N = self.dim, self.N
        seeds = [_f64(gx, (N, d)), _f64(gv, (N, d)), _f64(gC, (N, d, d)), _f64(gF, (N, d, d))]
        out = [np.empty((N, d)), np.empty((N, d)), np.empty((N, d, d)), np.empty((N, d, d)),
               np.zeros((self.L, self.G))]
        _check(lib().mpm64_backward(self.handle, *[_ptr(t) for t in seeds], *[_ptr(t) for t in out]),
               "mpm64_backward")
        return tuple(out)

    def info(self):
        n, g, L, T = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().mpm64_info(self.handle, C.byref(n), C.byref(g), C.byref(L), C.byref(T)), "mpm64_info")
        return {"n_particles": n.value, "n_groups": g.value, "act_steps": L.value, "rollout_steps": T.value}

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mpm64_destroy(self.handle), "mpm64_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Scenes of one dimension advanced together by the same launches (mpm_batch_*).  A request is
    a rollout of n_steps and, with want_grad, its reverse pass seeded by loss = mean final x_0;
    results stay in the scene (Scene.get_state, Scene.gradients)."""

    def __init__(self, ctx: Context, dim: int, mem_budget: int = 0):
        h = C.c_void_p()
        _check(lib().mpm_batch_create(ctx.handle, int(dim), C.c_size_t(int(mem_budget)), C.byref(h)),
               "mpm_batch_create")
        self.handle, self.ctx, self.dim = h, ctx, dim
        ctx._adopt(self)

    def admit(self, scene: "Scene", n_steps: int, want_grad: bool) -> int:
        slot = C.c_int(-1)
        scene._touch()
        _check(lib().mpm_batch_admit(self.handle, scene.handle, int(n_steps), int(bool(want_grad)), C.byref(slot)),
               "mpm_batch_admit")
        return slot.value

    def tick(self, max_steps: int = 1):
        _check(lib().mpm_batch_tick(self.handle, int(max_steps)), "mpm_batch_tick")

    def poll(self, slot: int) -> bool:
        """True once the slot's request is finished, successfully or not (see status)."""
        return self._poll(slot)[0]

    def status(self, slot: int) -> int:
        """MPM_OK, or the error a finished request stopped with (e.g. a particle left the grid)."""
        return self._poll(slot)[1]

    def _poll(self, slot: int):
        done = C.c_int(0)
        st = lib().mpm_batch_poll(self.handle, int(slot), C.byref(done))
        if st != MPM_OK and not done.value:
            raise MPMError(st, "mpm_batch_poll")
        return bool(done.value), int(st)

    def release(self, slot: int):
        _check(lib().mpm_batch_release(self.handle, int(slot)), "mpm_batch_release")

    def close(self):
        if getattr(self, "handle", None):
            lib().mpm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def header_symbols(header_path: str):
    """Names of the functions declared in include/mpm.h."""
    import re
    text = open(header_path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm(?:64)?_[a-z0-9_]+)\s*\(", text)))
