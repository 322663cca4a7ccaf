"""Seeded synthetic scene builders for the differentiable MLS-MPM step.

This module only *builds inputs*: particle lattices, jitter, group labels,
actuation directions and controller parameters, all drawn from numpy's
seeded PCG64 generator.  It contains none of the method's arithmetic (no
weights, stresses, transfers or adjoints), so both the CUDA path and the FP64
oracle can consume the very same arrays.

The paper does not release its scenes (the falling cube of its speed table,
the 2D walker, the 3D quadruped; Section IV-A and Section V-B).  The builders
below are synthetic stand-ins with the shapes, particle counts, lattice
densities and material parameters of the five workloads this library is
measured on:

* ``walker_square_2d``  - 2D, 64x64 grid, 1024 particles, 2 sinusoid groups.
* ``walker_2d``         - 2D, 128x128 grid, ~30k particles, 4 legs, basis controller.
* ``soft_body_3d``      - 3D, 64^3 grid, ~100k particles, 16 groups, MLP controller.
* ``box_cluster_3d``    - 3D, 128^3 grid, exactly 1M particles, 64 sinusoid groups.
* ``serving_request``   - one request of the serving mix (2D or 3D box cluster).

Conventions shared by every builder:

* Node ``i`` sits at ``i*dx`` for ``i`` in ``[0, n)`` per axis; the last axis
  is the fastest-varying one in node and cell linear indices.
* Particles are seeded on a lattice of spacing ``s`` (cell-centred), each
  component jittered uniformly; ``V0 = s^d`` and ``m = rho*V0`` with rho = 1.
* ``v0 = 0``, ``C0 = 0``, ``F0 = I`` unless a builder says otherwise.
* ``dir`` of every actuation group is the vertical axis e_1 (index 1).
* Group id ``-1`` marks unactuated particles.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

CTRL_SIN = 0      # a_g(t) = A_g * sin(2*pi*freq*t)
CTRL_BASIS = 1    # a_g(t) = sum_j W_gj b_j(t), b = [sin 2pi f t, cos 2pi f t, sin 4pi f t, cos 4pi f t]
CTRL_MLP = 2      # a = scale * tanh(W3 tanh(W2 tanh(W1 z + b1) + b2) + b3), z = group centroids - body centroid
CTRL_TABLE = 3    # a_g(t_n) = U[n][g] for n < L (L = hidden), 0 after: every step's actuation a decision variable
CTRL_COM = 4      # a = scale * tanh(W z + b), z = [target, group centres of mass, group mean velocities]

BC_STICKY = 0
BC_SLIP = 1
BC_OPEN = 2       # per-wall only: the wall constrains nothing


@dataclasses.dataclass
class SceneSpec:
    """Everything needed to simulate one scene (all arrays float64 / int32)."""

    name: str
    dim: int
    n_grid: tuple
    dx: float
    dt: float
    gravity: tuple
    E: float
    nu: float
    p_mass: float
    p_vol: float
    bc_type: int
    bc_width: int
    friction_c: float
    x0: np.ndarray          # [N, d]
    v0: np.ndarray          # [N, d]
    C0: np.ndarray          # [N, d, d]
    F0: np.ndarray          # [N, d, d]
    group: np.ndarray       # [N] int32, -1 = unactuated
    act_dir: np.ndarray     # [G, d]
    ctrl_type: int
    ctrl_params: np.ndarray  # float64, layout depends on ctrl_type
    ctrl_hidden: int = 0
    ctrl_freq: float = 1.0
    ctrl_scale: float = 1.0
    n_steps: int = 1
    ckpt_interval: int = 0
    E_arr: Optional[np.ndarray] = None     # [N] per-particle Young's modulus (None: E for all)
    mass_arr: Optional[np.ndarray] = None  # [N] per-particle mass (None: p_mass for all)
    # per wall w = 2 axis + side (low side first): 0 sticky, 1 slip with friction wall_c[w], 2 open
    wall_kind: Optional[np.ndarray] = None  # [2 dim] int32 (None: bc_type on every wall)
    wall_c: Optional[np.ndarray] = None     # [2 dim] (None: friction_c on every wall)
    tile_edge: int = 0  # cells per tile edge of the tiled form (0: the library chooses; 4; 8 in 2D)

    @property
    def n_particles(self) -> int:
        return int(self.x0.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.act_dir.shape[0])

    def copy(self, **changes) -> "SceneSpec":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        for k, v in d.items():
            if isinstance(v, np.ndarray):
                d[k] = v.copy()
        d.update(changes)
        return SceneSpec(**d)


def with_material(spec: SceneSpec, seed: int, spread: float = 0.2) -> SceneSpec:
    """Copy of spec with per-particle Young's modulus and mass, each the scene's value times an
    independent factor uniform in [1 - spread, 1 + spread] (seeded).  The largest E_p must still
    satisfy the explicit-integration limit of the scene's dt."""
    rng = np.random.default_rng(seed)
    N = spec.n_particles
    E = spec.E * rng.uniform(1.0 - spread, 1.0 + spread, N)
    m = spec.p_mass * rng.uniform(1.0 - spread, 1.0 + spread, N)
    return spec.copy(E_arr=E, mass_arr=m, name=spec.name + "+material")


def n_ctrl_params(ctrl_type: int, n_groups: int, dim: int, hidden: int) -> int:
    """Parameter count of each controller family (layout documented in the header)."""
    if ctrl_type == CTRL_SIN:
        return n_groups
    if ctrl_type == CTRL_BASIS:
        return 4 * n_groups
    if ctrl_type == CTRL_MLP:
        zin = n_groups * dim
        return hidden * zin + hidden + hidden * hidden + hidden + n_groups * hidden + n_groups
    if ctrl_type == CTRL_TABLE:
        return hidden * n_groups
    if ctrl_type == CTRL_COM:
        return dim + n_groups * dim * (1 + 2 * n_groups) + n_groups
    raise ValueError(f"unknown controller type {ctrl_type}")


def com_init(rng: np.random.Generator, n_groups: int, dim: int, target) -> np.ndarray:
    """Closed-loop controller parameters: the target, W ~ N(0, 1/Z), b = 0 (Z = dim (1 + 2G))."""
    Z = dim * (1 + 2 * n_groups)
    W = rng.normal(size=(n_groups, Z)) / math.sqrt(Z)
    return np.concatenate([np.asarray(target, np.float64).ravel(), W.ravel(), np.zeros(n_groups)])


def mlp_init(rng: np.random.Generator, n_groups: int, dim: int, hidden: int) -> np.ndarray:
    """W ~ N(0, 1/fan_in), b = 0; packed W1, b1, W2, b2, W3, b3 (row-major, out x in)."""
    zin = n_groups * dim
    parts = []
    for fan_out, fan_in in ((hidden, zin), (hidden, hidden), (n_groups, hidden)):
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(fan_in), size=(fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def _lattice_box(lo, hi, s):
    """Cell-centred lattice indices (integer, spacing s) whose points lie in [lo, hi)."""
    axes = []
    for a in range(len(lo)):
        i0 = int(math.ceil(lo[a] / s - 0.5))
        i1 = int(math.ceil(hi[a] / s - 0.5))
        axes.append(np.arange(i0, max(i0, i1)))
    return axes


def _finish(name, dim, n, dx, dt, E, s, pos, group, act_dir, ctrl_type, ctrl_params, rng,
            jitter, *, hidden=0, freq=1.0, scale=1.0, n_steps=1, ckpt=0, bc_type=BC_STICKY,
            bc_width=3, friction_c=0.0, gravity=None, nu=0.3):
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    N = pos.shape[0]
    if gravity is None:
        gravity = (0.0, -9.8, 0.0)[:dim]
    vol = s ** dim
    return SceneSpec(
        name=name, dim=dim, n_grid=(n,) * dim, dx=dx, dt=dt, gravity=tuple(gravity), E=E, nu=nu,
        p_mass=1.0 * vol, p_vol=vol, bc_type=bc_type, bc_width=bc_width, friction_c=friction_c,
        x0=pos.astype(np.float64), v0=np.zeros((N, dim)), C0=np.zeros((N, dim, dim)),
        F0=np.broadcast_to(np.eye(dim), (N, dim, dim)).copy(), group=group.astype(np.int32),
        act_dir=np.asarray(act_dir, dtype=np.float64), ctrl_type=ctrl_type,
        ctrl_params=np.asarray(ctrl_params, dtype=np.float64), ctrl_hidden=hidden,
        ctrl_freq=freq, ctrl_scale=scale, n_steps=n_steps, ckpt_interval=ckpt)


def _up(dim, G):
    d = np.zeros((G, dim))
    d[:, 1] = 1.0
    return d


def walker_square_2d(seed: int = 0, *, lift_cells: float = 0.0, n_steps: int = 100) -> SceneSpec:
    """2D, 64^2 grid, dx=1/64: a 32x32 particle square at spacing dx/2 (V0 = m = s^2), jitter
    +-0.1 dx per component, lower-left corner x = 0.375, bottom at y = 3 dx (resting on the
    3-cell sticky floor band); E = 20, nu = 0.3, dt = 1e-3, 100 steps; groups = left/right
    16 columns, a_g(t) = A_g sin(2 pi t) with A = (4, -2).  ``lift_cells`` raises the square
    (a mid-air variant used by closed-form tests)."""
    rng = np.random.default_rng(seed)
    n, dx = 64, 1.0 / 64
    s = dx / 2
    ii, jj = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    x = 0.375 + (ii.ravel() + 0.5) * s
    y = 3 * dx + lift_cells * dx + (jj.ravel() + 0.5) * s
    pos = np.stack([x, y], axis=1)
    group = (ii.ravel() >= 16).astype(np.int32)
    return _finish("walker_square_2d", 2, n, dx, 1e-3, 20.0, s, pos, group, _up(2, 2), CTRL_SIN,
                   [4.0, -2.0], rng, 0.1 * dx, freq=1.0, n_steps=n_steps)


def falling_cube(dim: int, side: int, seed: int = 6, *, n_steps: int = 100) -> SceneSpec:
    """The falling elastic cube of Section IV's speed comparison (Table II): side^dim particles on
    a lattice of spacing dx/2 (side 20, 40, 80 in 3D give the table's 8,000, 64,000 and 512,000
    particles; 80 in 2D its 6,400), jitter +-0.1 dx, released from rest with its bottom 2 dx above
    the 3-cell sticky floor band, centred in x (and z), on a grid with a quarter of the cube's width
    of margin around it (at least 32 cells); E = 20, nu = 0.3, gravity, no actuation (one group,
    zero amplitude), dt at half the explicit-integration limit.  The paper gives neither grid nor
    material for this scene."""
    rng = np.random.default_rng(seed)
    cells = side // 2  # the cube's width in cells
    n = max(32, int(math.ceil(1.5 * cells)) + 8)
    dx = 1.0 / n
    s = dx / 2
    E = 20.0
    dt = 0.5 * dx * math.sqrt(1.0 / E)
    idx = np.stack(np.meshgrid(*([np.arange(side)] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    lo = np.full(dim, 0.5 * (n - cells) * dx)
    lo[1] = 5 * dx
    pos = lo + (idx + 0.5) * s
    group = np.zeros(pos.shape[0], np.int32)
    return _finish(f"falling_cube_{dim}d_{side ** dim}", dim, n, dx, dt, E, s, pos, group, _up(dim, 1),
                   CTRL_SIN, [0.0], rng, 0.1 * dx, n_steps=n_steps)


def walker_2d(seed: int = 1, *, n_steps: int = 1000) -> SceneSpec:
    """2D soft walker: 128^2 grid, dx = 1/128, body 0.5 x 0.1 on 4 legs 0.08 x 0.2 (each size
    +-10 % seeded), legs standing on the 3-cell sticky floor band, lattice spacing dx/4 (16
    particles per cell, ~30k particles), jitter +-0.1 s; E = 20, dt = 5e-4, 1000 steps,
    checkpoint every 64 steps; 4 leg groups (body unactuated) driven by the 16-parameter
    sinusoid basis at 4 Hz, W ~ N(0, 2^2)."""
    rng = np.random.default_rng(seed)
    n, dx = 128, 1.0 / 128
    s = dx / 4
    floor = 3 * dx
    jit = lambda: rng.uniform(0.9, 1.1)
    leg_w, leg_h = 0.08 * jit(), 0.2 * jit()
    body_w, body_h = 0.5 * jit(), 0.1 * jit()
    x_left = 0.5 - body_w / 2
    rects = []  # (lo, hi, group)
    for k in range(4):
        lx = x_left + k * (body_w - leg_w) / 3
        rects.append(((lx, floor), (lx + leg_w, floor + leg_h), k))
    rects.append(((x_left, floor + leg_h), (x_left + body_w, floor + leg_h + body_h), -1))
    pts, grp = [], []
    for lo, hi, g in rects:
        ax = _lattice_box(lo, hi, s)
        I, J = np.meshgrid(ax[0], ax[1], indexing="ij")
        pts.append(np.stack([(I.ravel() + 0.5) * s, (J.ravel() + 0.5) * s], axis=1))
        grp.append(np.full(I.size, g))
    pos, group = np.concatenate(pts), np.concatenate(grp)
    W = rng.normal(0.0, 2.0, size=(4, 4))
    return _finish("walker_2d", 2, n, dx, 5e-4, 20.0, s, pos, group, _up(2, 4), CTRL_BASIS,
                   W.ravel(), rng, 0.1 * s, freq=4.0, n_steps=n_steps, ckpt=64)


def _box_union(rng, dim, n, dx, s, target_lo, target_hi, *, exact=None, max_tries=200,
               side=(0.08, 0.2), floor_cells=3, region=(0.15, 0.85)):
    """Union of seeded boxes resting on the floor (bottom at y = floor_cells*dx), sampled on
    one cell-centred lattice of spacing s without duplicates.  With ``exact`` the union is
    truncated to exactly that many points (the last box is cut); otherwise boxes are added
    until the count reaches ``target_lo`` and the whole draw is repeated if it overshoots
    ``target_hi``."""
    L = int(round(1.0 / s))
    floor = floor_cells * dx
    top_limit = (n - floor_cells - 2) * dx
    for _ in range(max_tries):
        occ = np.zeros((L,) * dim, dtype=bool)
        order = []
        count = 0
        boxes = 0
        while True:
            boxes += 1
            if boxes > 4000:  # the region is saturated: keep what the union holds
                if exact is not None:
                    return np.concatenate(order)
                break
            sides = rng.uniform(side[0], side[1], size=dim)
            lo = np.empty(dim)
            for a in range(dim):
                if a == 1:
                    lo[a] = floor
                else:
                    lo[a] = rng.uniform(region[0], region[1] - sides[a])
            hi = lo + sides
            hi[1] = min(hi[1], top_limit)
            ax = _lattice_box(lo, hi, s)
            grids = np.meshgrid(*ax, indexing="ij")
            idx = tuple(g.ravel() for g in grids)
            new = ~occ[idx]
            new_idx = tuple(c[new] for c in idx)
            if exact is not None and count + new_idx[0].size >= exact:
                take = exact - count
                new_idx = tuple(c[:take] for c in new_idx)
            occ[new_idx] = True
            order.append(np.stack(new_idx, axis=1))
            count += new_idx[0].size
            if exact is not None and count >= exact:
                return np.concatenate(order)
            if exact is None and count >= target_lo:
                break
        if count <= target_hi:
            return np.concatenate(order)
    raise RuntimeError("could not draw a box union in the requested particle range")


def _bbox_groups(pos, parts):
    """Partition the particles' bounding box into a regular lattice of ``parts`` (per axis,
    0 = axis not split) and return the group id of each particle."""
    lo, hi = pos.min(axis=0), pos.max(axis=0)
    gid = np.zeros(pos.shape[0], dtype=np.int64)
    for a, k in enumerate(parts):
        if k <= 1:
            continue
        t = np.clip(((pos[:, a] - lo[a]) / max(hi[a] - lo[a], 1e-12) * k).astype(np.int64), 0, k - 1)
        gid = gid * k + t
    return gid.astype(np.int32)


def soft_body_3d(seed: int = 2, *, n_steps: int = 500) -> SceneSpec:
    """3D soft body: 64^3 grid, dx = 1/64, union of seeded boxes (sides U(0.08, 0.2)) resting on
    the floor, lattice spacing dx/2 (8 per cell), redrawn until 95k <= N <= 105k, jitter
    +-0.1 s; E = 50, dt = 5e-4, 500 steps; 16 groups = 4x4 partition of the bounding box in
    (x, z); 3-layer MLP controller 48 -> 64 -> 64 -> 16 reading group centroids relative to the
    body centroid, output scaled by E/4."""
    rng = np.random.default_rng(seed)
    n, dx = 64, 1.0 / 64
    s = dx / 2
    lat = _box_union(rng, 3, n, dx, s, 95_000, 105_000)
    pos = (lat + 0.5) * s
    group = _bbox_groups(pos, (4, 0, 4))
    params = mlp_init(rng, 16, 3, 64)
    return _finish("soft_body_3d", 3, n, dx, 5e-4, 50.0, s, pos, group, _up(3, 16), CTRL_MLP,
                   params, rng, 0.1 * s, hidden=64, scale=50.0 / 4, n_steps=n_steps)


def box_cluster_3d(seed: int = 3, *, n_particles: int = 1_000_000, n: int = 128,
                   n_steps: int = 200) -> SceneSpec:
    """3D large scene: 128^3 grid, dx = 1/128, seeded random box cluster on the floor at lattice
    spacing dx/2, exactly ``n_particles`` (the last box is truncated), jitter +-0.1 s; E = 50,
    dt = 2e-4, 200 steps; 64 groups = 4x4x4 bounding-box partition, a_g = A_g sin(2 pi t) with
    A_g ~ U(-E/4, E/4)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    s = dx / 2
    lat = _box_union(rng, 3, n, dx, s, 0, 0, exact=n_particles)
    pos = (lat + 0.5) * s
    group = _bbox_groups(pos, (4, 4, 4))
    A = rng.uniform(-50.0 / 4, 50.0 / 4, size=64)
    return _finish("box_cluster_3d", 3, n, dx, 2e-4, 50.0, s, pos, group, _up(3, 64), CTRL_SIN,
                   A, rng, 0.1 * s, n_steps=n_steps)


def serving_request(req_id: int, seed: int = 4) -> tuple:
    """One request of the serving mix: returns (SceneSpec, want_grad).  dim 2/3 at 50/50, n
    uniform in {32, 48, 64, 96, 128}, N log-uniform in [1e3, 2e5] clipped so the cluster fits,
    horizon uniform in [50, 500], 40 % forward-only / 60 % forward+gradient, a box cluster on
    the floor, E = 20 (2D) / 50 (3D), dt = 5e-4, sinusoid actuation on 4^d bbox groups."""
    rng = np.random.default_rng([seed, req_id])
    dim = int(rng.integers(2, 4))
    n = int(rng.choice([32, 48, 64, 96, 128]))
    # at most half the lattice points of the region the boxes are drawn in
    s_ = 0.5 / n
    height = 0.3 if dim == 2 else 0.2
    cap = int(0.5 * (0.7 / s_) ** (dim - 1) * (height / s_))
    N = int(min(cap, math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
    N = max(N, 64)
    T = int(rng.integers(50, 501))
    want_grad = bool(rng.uniform() < 0.6)
    dx = 1.0 / n
    s = dx / 2
    E = 20.0 if dim == 2 else 50.0
    side = (0.08, 0.3) if dim == 2 else (0.08, 0.2)
    lat = _box_union(rng, dim, n, dx, s, 0, 0, exact=N, side=side)
    pos = (lat + 0.5) * s
    parts = (4, 4) if dim == 2 else (4, 4, 4)
    group = _bbox_groups(pos, parts)
    G = 4 ** dim
    A = rng.uniform(-E / 4, E / 4, size=G)
    spec = _finish(f"serve_{req_id}", dim, n, dx, 5e-4, E, s, pos, group, _up(dim, G), CTRL_SIN, A,
                   rng, 0.1 * s, n_steps=T)
    return spec, want_grad


def billiards_2d(seed: int = 5, *, n: int = 64, radius_cells: float = 5.0, gap_cells: float = 3.0,
                 speed: float = 0.6, offset: float = 0.35, E: float = 100.0, dt: float = 1e-3,
                 n_steps: int = 1000) -> SceneSpec:
    """Two colliding elastic discs in 2D (the float64 accuracy case of Section VI, whose geometry
    the paper does not give): 64^2 grid, dx = 1/64, discs of radius 5 dx on a lattice of spacing
    dx/2 (jitter +-0.1 of it, seeded), ball A centred at (0.2, 0.5) moving at (0.6, 0), ball B at
    rest 3 dx beyond it along x and 0.35 radii higher (an oblique hit), no gravity, sticky walls
    3 cells deep; E = 100, nu = 0.3, rho = 1, dt = 1e-3 (0.64 of the explicit limit).  The
    discs first touch (share grid nodes) after about 25 steps, so a 1- or 10-step rollout has no
    collision and 100 or 1000 steps do; B leaves at ~0.43 and never reaches a wall within 1000
    steps.  Particles of A come first."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    s = dx / 2
    R = radius_cells * dx
    ca = np.array([0.2, 0.5])
    cb = ca + np.array([2 * R + gap_cells * dx, offset * R])
    pts = []
    for c in (ca, cb):
        ax = _lattice_box(c - R, c + R, s)
        I, J = np.meshgrid(ax[0], ax[1], indexing="ij")
        p = np.stack([(I.ravel() + 0.5) * s, (J.ravel() + 0.5) * s], axis=1)
        pts.append(p[np.linalg.norm(p - c, axis=1) <= R])
    na = pts[0].shape[0]
    pos = np.concatenate(pts)
    N = pos.shape[0]
    spec = _finish("billiards_2d", 2, n, dx, dt, E, s, pos, np.full(N, -1), np.zeros((0, 2)), CTRL_TABLE,
                   np.zeros(0), rng, 0.1 * s, n_steps=n_steps, bc_width=3, gravity=(0.0, 0.0))
    spec.v0[:na] = [speed, 0.0]
    return spec


def billiards_ball_a(spec: SceneSpec) -> np.ndarray:
    """Mask of ball A's particles in a billiards_2d scene (the ones moving at the start)."""
    return np.linalg.norm(spec.v0, axis=1) > 0


def blob(dim: int, n: int, n_particles: int, seed: int, *, dt: float = 1e-3, E: float = 20.0,
         nu: float = 0.3, bc_type: int = BC_STICKY, bc_width: int = 2, friction_c: float = 0.0,
         n_groups: int = 2, ctrl_type: int = CTRL_SIN, hidden: int = 8, gravity=None,
         v_scale: float = 0.0, c_scale: float = 0.0, f_scale: float = 0.0, center=None,
         radius_cells: float = 2.5, freq: float = 1.0, scale: float = 1.0,
         amp: float = 1.0) -> SceneSpec:
    """A small random particle blob for unit, FD and parity tests: positions uniform in a ball
    of ``radius_cells`` cells around ``center`` (default: grid middle), optional random
    v0/C0/F0 perturbations of the given scales, ``n_groups`` groups by particle index, random
    unit actuation directions and random controller parameters of amplitude ``amp``."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    if center is None:
        center = np.full(dim, 0.5 * (n - 1) * dx)
    center = np.asarray(center, dtype=np.float64)
    u = rng.normal(size=(n_particles, dim))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = radius_cells * dx * rng.uniform(0, 1, size=(n_particles, 1)) ** (1.0 / dim)
    pos = center + u * r
    s = dx / 2
    G = n_groups
    group = (np.arange(n_particles) % max(G, 1)).astype(np.int32) if G > 0 else np.full(n_particles, -1, np.int32)
    d = rng.normal(size=(G, dim))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    if ctrl_type == CTRL_MLP:
        params = mlp_init(rng, G, dim, hidden)
    elif ctrl_type == CTRL_COM:
        params = com_init(rng, G, dim, center + rng.uniform(-0.2, 0.2, dim))
    else:
        params = amp * rng.normal(size=n_ctrl_params(ctrl_type, G, dim, hidden))
    spec = _finish(f"blob{dim}d_{n}_{n_particles}_{seed}", dim, n, dx, dt, E, s, pos, group, d,
                   ctrl_type, params, rng, 0.0, hidden=hidden, freq=freq, scale=scale,
                   bc_type=bc_type, bc_width=bc_width, friction_c=friction_c, gravity=gravity, nu=nu)
    spec.v0 = v_scale * rng.normal(size=(n_particles, dim))
    spec.C0 = c_scale * rng.normal(size=(n_particles, dim, dim))
    spec.F0 = np.eye(dim) + f_scale * rng.normal(size=(n_particles, dim, dim))
    return spec


WORKLOADS = {
    "walker_square_2d": walker_square_2d,
    "walker_2d": walker_2d,
    "soft_body_3d": soft_body_3d,
    "box_cluster_3d": box_cluster_3d,
}
