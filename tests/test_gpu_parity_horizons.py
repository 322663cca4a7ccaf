"""GPU parity at the benchmarked workloads over the horizons the benchmark times (FP64 oracle on
the same seeded inputs; tolerances as everywhere: forward relative 1e-4 on 10-step windows
re-synced to the oracle, gradients relative 1e-3 with cosine >= 0.999 and an element-wise bound).

  2D walker (31,458 particles, basis controller): every 10-step window of the 1000-step rollout,
      and the full-horizon gradient of L = mean final x_0 from a rollout with a checkpoint every 64
      steps, as benchmarked.
  3D soft body (95,123 particles, MLP controller): every 10-step window of the 500-step rollout, and
      the full-horizon gradient with a checkpoint every 23 steps, as benchmarked.
  1M-particle 3D cluster: the 10-step windows of the first 50 of its 200 steps, and the gradient of
      one checkpoint segment (7 steps: the interval its 4 GiB budget gives), recomputed from its
      checkpoint as in the benchmarked reverse pass.

The oracle runs in four spawned processes (tests/horizon_jobs.py) started when the module begins,
while the GPU side runs; each test waits for its own job.
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1810_01054_gb300 import scenes as S
from tests import horizon_jobs as H
from tests.parity_utils import assert_grad_close, assert_state_close, cosine, max_scaled, rel_l2

pytestmark = pytest.mark.gpu

JOB_TIMEOUT_S = 3600


@pytest.fixture(scope="module")
def jobs(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("oracle_horizons"))
    pool = mp.get_context("spawn").Pool(4)
    futs = {j: pool.apply_async(H.run, (j, out)) for j in ("soft", "cluster_seg", "cluster_fwd", "walker")}
    yield out, futs
    pool.terminate()
    pool.join()


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


def _wait(jobs, job):
    out, futs = jobs
    futs[job].get(timeout=JOB_TIMEOUT_S)
    return out


def _windows(M, ctx, spec, out, tag, n_windows):
    """Every 10-step window re-synced to the oracle's state at its start."""
    xs, vs, Cs, Fs = (H.load(out, tag, k) for k in ("xs", "vs", "Cs", "Fs"))
    gpu = M.Scene(ctx, spec)
    worst = {}
    for w in range(n_windows):
        n0 = H.EVERY * w
        gpu.set_state(xs[w], vs[w], Cs[w], Fs[w], step=n0)
        gpu.step(H.EVERY)
        got = gpu.get_state()
        ref = (xs[w + 1], vs[w + 1], Cs[w + 1], Fs[w + 1])
        for nm, a, b in zip("xvCF", got, ref):
            worst[nm] = max(worst.get(nm, 0.0), rel_l2(a, b))
        assert_state_close(got, ref)
    gpu.close()
    print(f"\n{tag}: worst 10-step window relative L2 over {n_windows} windows: "
          + ", ".join(f"{k} {v:.2e}" for k, v in worst.items()))


def _full_gradient(M, ctx, spec, out, tag, k):
    gpu = M.Scene(ctx, spec)
    gpu.rollout(spec.n_steps, k)
    xT = gpu.get_state()[0]
    g = gpu.backward(H.mean_x0(spec.n_particles, spec.dim))
    gpu.close()
    for nm, a in zip(("x0", "v0", "C0", "F0", "params"), g):
        ref = H.load(out, tag, "g" + nm[0] if nm != "params" else "gp")
        print(f"\n{tag} full-horizon dL/d{nm}: relative L2 {rel_l2(a, ref):.2e}, cosine {cosine(a, ref):.7f}, "
              f"max scaled {max_scaled(a, ref):.2e}")
        assert_grad_close(a, ref, f"{tag} dL/d{nm}")
    return xT


@pytest.mark.parametrize("part", ["windows", "gradient"])
def test_walker_over_its_1000_steps(M, ctx, jobs, part):
    spec = S.walker_2d(1)
    out = _wait(jobs, "walker")
    if part == "windows":
        _windows(M, ctx, spec, out, "walker_2d", spec.n_steps // H.EVERY)
    else:
        _full_gradient(M, ctx, spec, out, "walker_2d", 64)


@pytest.mark.parametrize("part", ["windows", "gradient"])
def test_soft_body_over_its_500_steps(M, ctx, jobs, part):
    spec = S.soft_body_3d(2)
    out = _wait(jobs, "soft")
    if part == "windows":
        _windows(M, ctx, spec, out, "soft_body_3d", spec.n_steps // H.EVERY)
    else:
        _full_gradient(M, ctx, spec, out, "soft_body_3d", 23)


def test_cluster_first_50_steps_in_windows(M, ctx, jobs):
    spec = S.box_cluster_3d(3)
    out = _wait(jobs, "cluster_fwd")
    _windows(M, ctx, spec, out, "cluster_fwd", H.CLUSTER_WINDOW_STEPS // H.EVERY)


def test_cluster_one_checkpoint_segment_gradient(M, ctx, jobs):
    spec = S.box_cluster_3d(3)
    T = H.CLUSTER_SEGMENT
    gpu = M.Scene(ctx, spec)
    gpu.rollout(T, T, 4 << 30)  # one segment: the checkpoint and T - 1 recomputed states
    wx, wv = H.cluster_seeds(spec.n_particles, 3)
    g = gpu.backward(wx, wv)
    x, v, _, _ = gpu.get_state()
    gpu.close()
    out = _wait(jobs, "cluster_seg")
    assert_state_close((x, v), (H.load(out, "cluster_seg", "xT"), H.load(out, "cluster_seg", "vT")),
                       names=("x", "v"))
    for nm, key, a in zip(("x0", "v0", "C0", "F0", "params"), ("gx", "gv", "gC", "gF", "gp"), g):
        ref = H.load(out, "cluster_seg", key)
        print(f"\ncluster segment dL/d{nm}: relative L2 {rel_l2(a, ref):.2e}, cosine {cosine(a, ref):.7f}, "
              f"max scaled {max_scaled(a, ref):.2e}")
        assert_grad_close(a, ref, f"cluster segment dL/d{nm}")


def test_cluster_plan_under_its_budgets(M, ctx):
    """The intervals mpm_rollout takes for the 1M-particle cluster's 200 steps by budget: every
    state in 32 GiB; in 4 GiB the smallest interval whose store (checkpoints, two sets of recompute
    buffers, the overlap's sorts) fits, 7 steps (29 checkpoints, 171 steps recomputed); in 1 GiB the
    multi-level store."""
    spec = S.box_cluster_3d(3)
    sc = M.Scene(ctx, spec)
    S_ = sc.info()["state_bytes"]
    T = spec.n_steps
    assert sc.plan_rollout(T, 0, 32 << 30) == (1, T, False)
    k, fwd, multi = sc.plan_rollout(T, 0, 4 << 30)
    nseg = -(-T // 7)
    assert (k, fwd, multi) == (7, 2 * T - nseg, False)
    assert (nseg + 2 * (k - 1)) * S_ <= 4 << 30
    k1, fwd1, multi1 = sc.plan_rollout(T, 0, 1 << 30)
    assert k1 == 0 and multi1 and fwd1 > 2 * T - nseg
    assert sc.plan_rollout(T, 15, 4 << 30)[:2] == (15, 2 * T - (-(-T // 15)))  # a given interval stays
    sc.close()
