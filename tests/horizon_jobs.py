"""Oracle side of the timed-horizon parity tests: each job runs the FP64 oracle on one of the
benchmarked workloads in a process of its own (started with spawn) and writes what the GPU side
compares against into a directory as .npy files.

Jobs (all on the seeded workloads the benchmark times):
  walker      2D walker, 31,458 particles, the whole 1000-step rollout: every 10th state and the
              full-horizon gradient of L = mean final x_0 with respect to x0, v0, C0, F0 and the
              controller parameters.
  soft        3D soft body, 95,123 particles, MLP controller, the whole 500-step rollout: every 10th
              state and the full-horizon gradient of the same loss.
  cluster_fwd 1M-particle 3D cluster, the first 50 of its 200 steps: every 10th state.
  cluster_seg 1M-particle 3D cluster, one checkpoint segment (7 steps from the initial state): the
              gradient of L = <w, x_15> + <u, v_15> with seeded weights w, u.
"""
from __future__ import annotations

import os

import numpy as np

EVERY = 10
CLUSTER_WINDOW_STEPS = 50
CLUSTER_SEGMENT = 7


def _spec(name):
    from paper_1810_01054_gb300 import scenes as S
    seeds = {"walker_2d": 1, "soft_body_3d": 2, "box_cluster_3d": 3}
    return S.WORKLOADS[name](seeds[name])


def mean_x0(N, d):
    g = np.zeros((N, d))
    g[:, 0] = 1.0 / N
    return g


def cluster_seeds(N, d):
    rng = np.random.default_rng(3)
    return rng.normal(size=(N, d)) / N, rng.normal(size=(N, d)) / N


def _save(out_dir, tag, **arrays):
    for k, a in arrays.items():
        np.save(os.path.join(out_dir, f"{tag}_{k}.npy"), a)


def _march(sc, state, n0, n1, keep_every, keep):
    """Oracle steps n0 -> n1 (controller evaluated at every step, as the rollout does), keeping
    every keep_every-th state by step number."""
    x, v, C, F = state
    for n in range(n0, n1):
        act = sc.controller(n, x, v=v)
        x, v, C, F = sc.step(act, x, v, C, F)
        if (n + 1) % keep_every == 0:
            keep[n + 1] = (x, v, C, F)
    return x, v, C, F


def full_horizon(name, out_dir):
    """Whole rollout of a benchmarked workload: every 10th state and the full-horizon gradient."""
    from oracle import oracle as O
    spec = _spec(name)
    sc = O.Scene(spec)
    T = spec.n_steps
    traj = sc.rollout(T)
    xs, vs, Cs, Fs, _ = traj
    _save(out_dir, name, xs=xs[::EVERY], vs=vs[::EVERY], Cs=Cs[::EVERY], Fs=Fs[::EVERY])
    g = sc.backward(traj, (mean_x0(sc.N, sc.dim), None, None, None))
    _save(out_dir, name, gx=g[0], gv=g[1], gC=g[2], gF=g[3], gp=g[4])
    return name


def cluster_windows(out_dir):
    from oracle import oracle as O
    spec = _spec("box_cluster_3d")
    sc = O.Scene(spec)
    keep = {0: sc.initial_state()}
    _march(sc, keep[0], 0, CLUSTER_WINDOW_STEPS, EVERY, keep)
    steps = sorted(keep)
    for i, a in enumerate(("xs", "vs", "Cs", "Fs")):
        _save(out_dir, "cluster_fwd", **{a: np.stack([keep[n][i] for n in steps])})
    return "cluster_fwd"


def cluster_segment(out_dir):
    from oracle import oracle as O
    spec = _spec("box_cluster_3d")
    sc = O.Scene(spec)
    traj = sc.rollout(CLUSTER_SEGMENT)
    wx, wv = cluster_seeds(sc.N, sc.dim)
    g = sc.backward(traj, (wx, wv, None, None))
    _save(out_dir, "cluster_seg", gx=g[0], gv=g[1], gC=g[2], gF=g[3], gp=g[4], xT=traj[0][-1], vT=traj[1][-1])
    return "cluster_seg"


def run(job, out_dir):
    if job == "walker":
        return full_horizon("walker_2d", out_dir)
    if job == "soft":
        return full_horizon("soft_body_3d", out_dir)
    if job == "cluster_fwd":
        return cluster_windows(out_dir)
    if job == "cluster_seg":
        return cluster_segment(out_dir)
    raise ValueError(job)


def load(out_dir, tag, key):
    return np.load(os.path.join(out_dir, f"{tag}_{key}.npy"))
