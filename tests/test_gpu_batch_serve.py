"""Batched launches, the serving loop and the rollout autograd.Function (GPU).

A scene's results must be the same bits alone and inside any batch mix (tiles never span scenes
and every sum has a fixed order); requests served with continuous batching must return exactly
what they return alone; torch autograd through the rollout Function must equal the library's own
reverse pass and the FP64 oracle's gradient within the stated tolerance.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import assert_grad_close, mean_x0_seed

pytestmark = pytest.mark.gpu


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


def _k_of(T):
    return 1 if T <= 16 else int(math.ceil(math.sqrt(T)))


def _alone(M, ctx, spec, T, want_grad):
    sc = M.Scene(ctx, spec)
    sc.rollout(T, _k_of(T))
    st = sc.get_state()
    g = sc.backward(mean_x0_seed(sc.N, sc.dim)) if want_grad else None
    sc.close()
    return st, g


def _mix_2d():
    return [
        (S.blob(2, 32, 300, 1, v_scale=0.3, radius_cells=5.0, center=(0.5, 7.0 / 32), bc_width=3, amp=2.0), 23, True),
        (S.walker_square_2d(0), 40, True),
        (S.blob(2, 48, 500, 2, ctrl_type=S.CTRL_BASIS, n_groups=4, freq=4.0, radius_cells=6.0, v_scale=0.2), 17, False),
        (S.blob(2, 24, 64, 3, bc_type=S.BC_SLIP, friction_c=0.3, radius_cells=3.0, center=(0.4, 4.5 / 24)), 30, True),
    ]


def _mix_3d():
    return [
        (S.blob(3, 16, 400, 4, radius_cells=3.5, v_scale=0.3, amp=2.0), 12, True),
        (S.blob(3, 24, 900, 5, radius_cells=4.0, v_scale=0.3, ctrl_type=S.CTRL_MLP, n_groups=4, hidden=8,
                scale=3.0), 20, True),
        (S.blob(3, 20, 250, 6, radius_cells=3.0, v_scale=0.3), 9, False),
    ]


@pytest.mark.parametrize("mix", [_mix_2d, _mix_3d], ids=["2d", "3d"])
def test_batch_results_equal_alone_bitwise(M, ctx, mix):
    reqs = mix()
    alone = [_alone(M, ctx, spec, T, g) for spec, T, g in reqs]
    batch = M.Batch(ctx, reqs[0][0].dim)
    scenes, slots = [], []
    for spec, T, g in reqs:
        sc = M.Scene(ctx, spec)
        scenes.append(sc)
        slots.append(batch.admit(sc, T, g))
    assert all(s >= 0 for s in slots)
    for _ in range(10000):
        batch.tick(4)
        if all(batch.poll(s) for s in slots):
            break
    assert all(batch.poll(s) for s in slots)
    for (spec, T, g), sc, (st, grads) in zip(reqs, scenes, alone):
        got = sc.get_state()
        for a, b in zip(got, st):
            assert np.array_equal(a, b)
        if g:
            gg = sc.gradients()
            for a, b in zip(gg, grads):
                assert np.array_equal(a, b)
    for s in slots:
        batch.release(s)
    batch.close()


def test_serving_mix_equals_alone_and_reports_latency(M, ctx):
    from paper_1810_01054_gb300.serve import Server
    reqs = [(spec, T, g) for spec, T, g in _mix_2d()[:3]] + [(spec, T, g) for spec, T, g in _mix_3d()[:2]]
    alone = [_alone(M, ctx, spec, T, g) for spec, T, g in reqs]
    srv = Server(device=0, mem_fraction=0.2, tick_steps=3)
    ids = []
    for i, (spec, T, g) in enumerate(reqs):
        ids.append(srv.submit(spec, g, n_steps=T, arrival=0.002 * i))  # staggered arrivals
    srv.run()
    for rid, (spec, T, g), (st, grads) in zip(ids, reqs, alone):
        r = srv.results[rid]
        for a, b in zip((r["x"], r["v"], r["C"], r["F"]), st):
            assert np.array_equal(a, b)
        if g:
            for a, b in zip(r["grads"], grads):
                assert np.array_equal(a, b)
    p50, p99 = srv.latency_percentiles()
    assert 0 < p50 <= p99
    srv.close()


def test_serving_mix_sampled_requests_equal_alone(M, ctx):
    """60 requests of the seeded serving mix (2D and 3D box clusters, 1e3-2e5 particles, 50-500
    steps, 60 % with gradients) arrive as a Poisson stream and are served with continuous
    batching; 20 of them, sampled, run again alone and return the same bits."""
    from paper_1810_01054_gb300.serve import Server
    n = 60
    reqs = [S.serving_request(i, 4) for i in range(n)]
    rng = np.random.default_rng(0)
    arrivals = np.cumsum(rng.exponential(0.004, size=n))
    srv = Server(device=0, mem_fraction=0.3, tick_steps=8)
    ids = [srv.submit(sp, g, arrival=float(t)) for (sp, g), t in zip(reqs, arrivals)]
    srv.run()
    assert all(srv.results[i]["status"] == 0 for i in ids)
    for i in rng.choice(n, size=20, replace=False):
        sp, g = reqs[i]
        r = srv.results[ids[i]]
        st, grads = _alone(M, ctx, sp, sp.n_steps, g)
        for a, b in zip((r["x"], r["v"], r["C"], r["F"]), st):
            assert np.array_equal(a, b), i
        if g:
            for a, b in zip(r["grads"], grads):
                assert np.array_equal(a, b), i
    p50, p99 = srv.latency_percentiles()
    assert 0 < p50 <= p99
    srv.close()


def test_a_batch_keeps_one_tile_edge(M, ctx):
    """The tile kernels of a launch are instantiated for one tile edge: a batch holding scenes of
    one edge refuses another (MPM_ERR_ARG) and takes it once empty again."""
    wide = M.Scene(ctx, S.walker_square_2d(0).copy(tile_edge=8))
    narrow = M.Scene(ctx, S.walker_square_2d(0).copy(tile_edge=4))
    batch = M.Batch(ctx, 2)
    s0 = batch.admit(wide, 5, False)
    assert s0 >= 0
    with pytest.raises(M.MPMError) as e:
        batch.admit(narrow, 5, False)
    assert e.value.status == -1
    while not batch.poll(s0):
        batch.tick(8)
    batch.release(s0)
    s1 = batch.admit(narrow, 5, False)
    assert s1 >= 0
    while not batch.poll(s1):
        batch.tick(8)
    batch.release(s1)
    batch.close()


def test_admission_waits_for_memory(M, ctx):
    """A batch whose budget holds one request admits the second only after the first leaves."""
    spec = S.blob(2, 32, 200, 9, radius_cells=4.0)
    a, b = M.Scene(ctx, spec), M.Scene(ctx, spec)
    info = a.info()
    T = 25
    k = _k_of(T)
    need = ((T + k - 1) // k + k - 1) * info["state_bytes"]
    batch = M.Batch(ctx, 2, mem_budget=need + need // 2)
    s0 = batch.admit(a, T, True)
    assert s0 >= 0
    assert batch.admit(b, T, True) == -1
    while not batch.poll(s0):
        batch.tick(8)
    batch.release(s0)
    s1 = batch.admit(b, T, True)
    assert s1 >= 0
    while not batch.poll(s1):
        batch.tick(8)
    for x, y in zip(a.gradients(), b.gradients()):
        assert np.array_equal(x, y)
    batch.close()


def test_autograd_function_matches_library_and_oracle(M, ctx):
    torch = pytest.importorskip("torch")
    from paper_1810_01054_gb300.rollout import rollout
    dev = torch.device("cuda", 0)
    spec = S.walker_square_2d(0, n_steps=40)
    T = 40
    sc = M.Scene(ctx, spec)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev, requires_grad=True)
    x0, v0, C0, F0 = t(spec.x0), t(spec.v0), t(spec.C0), t(spec.F0)
    params = t(spec.ctrl_params)
    xT, vT, CT, FT = rollout(sc, T, x0, v0, C0, F0, params, ckpt_interval=8)
    loss = xT[:, 0].mean()
    loss.backward()
    torch.cuda.synchronize()
    # the library's own reverse pass on the same rollout
    sc2 = M.Scene(ctx, spec)
    sc2.rollout(T, 8)
    gx, gv, gC, gF, gp = sc2.backward(mean_x0_seed(sc2.N, 2))
    assert np.array_equal(v0.grad.cpu().numpy(), gv)
    assert np.array_equal(params.grad.cpu().numpy(), gp)
    # and the oracle
    osc = O.Scene(spec)
    traj = osc.rollout(T)
    ogx, ogv, ogC, ogF, ogp = osc.backward(traj, (mean_x0_seed(osc.N, 2), None, None, None))
    assert_grad_close(v0.grad.cpu().numpy(), ogv, "autograd dL/dv0")
    assert_grad_close(params.grad.cpu().numpy(), ogp, "autograd dL/dA")
    assert_grad_close(F0.grad.cpu().numpy(), ogF, "autograd dL/dF0")


def test_autograd_refuses_a_backward_through_a_stale_rollout(M, ctx):
    """The library differentiates a scene's latest rollout; a graph whose scene was rolled out
    again before its backward is refused instead of returning the later rollout's gradients."""
    torch = pytest.importorskip("torch")
    from paper_1810_01054_gb300.rollout import rollout
    dev = torch.device("cuda", 0)
    spec = S.walker_square_2d(0, n_steps=10)
    sc = M.Scene(ctx, spec)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev, requires_grad=True)
    leaves = lambda: (t(spec.x0), t(spec.v0), t(spec.C0), t(spec.F0), t(spec.ctrl_params))
    first = leaves()
    xT1 = rollout(sc, 10, *first)[0]
    second = leaves()
    xT2 = rollout(sc, 5, *second)[0]
    with pytest.raises(RuntimeError, match="rolled out"):
        xT1[:, 0].mean().backward()
    xT2[:, 0].mean().backward()  # the latest rollout still differentiates
    assert torch.isfinite(second[1].grad).all() and second[1].grad.abs().max() > 0
    sc.close()


def test_context_outlives_its_scenes_and_batches(M):
    """The C context refuses to go while scenes or batches use it; the binding closes them first."""
    c = M.Context(0)
    sc = M.Scene(c, S.blob(2, 16, 50, 11, radius_cells=3.0))
    b = M.Batch(c, 2)
    assert M.lib().mpm_ctx_destroy(c.handle) == -7  # MPM_ERR_STATE: nothing freed
    sc.step(2)
    c.close()
    assert sc.handle is None and b.handle is None and c.handle is None


def test_batch_crossing_the_fused_scan_threshold_equals_alone(M, ctx):
    """Tile counts above and below 2048 take different scans (separate, or inside the scatter);
    a batch whose composition moves between them as requests finish must still give every scene
    exactly its alone result.  Two 128^2 scenes (1024 tiles each) plus a 48^2 one (144 tiles)
    that finishes first: 2192 tiles, then 2048."""
    reqs = [(S.blob(2, 128, 300, 61, v_scale=0.3, radius_cells=6.0, amp=2.0), 14, True),
            (S.blob(2, 128, 250, 62, v_scale=0.3, radius_cells=5.0, amp=2.0), 30, True),
            (S.blob(2, 48, 120, 63, v_scale=0.3, radius_cells=4.0, amp=2.0), 5, True)]
    alone = [_alone(M, ctx, spec, T, g) for spec, T, g in reqs]
    batch = M.Batch(ctx, 2)
    scenes = [M.Scene(ctx, spec) for spec, _, _ in reqs]
    slots = [batch.admit(sc, T, g) for sc, (_, T, g) in zip(scenes, reqs)]
    for _ in range(1000):
        batch.tick(2)
        if all(batch.poll(s) for s in slots):
            break
    for sc, (st, grads) in zip(scenes, alone):
        for a, b in zip(sc.get_state() + sc.gradients(), st + grads):
            assert np.array_equal(a, b)
    batch.close()


def test_scene_is_driven_by_its_batch_until_released(M, ctx):
    spec = S.blob(2, 32, 200, 71, radius_cells=4.0)
    sc = M.Scene(ctx, spec)
    batch = M.Batch(ctx, 2)
    slot = batch.admit(sc, 6, True)
    for call in (lambda: sc.step(1), lambda: sc.rollout(3), lambda: sc.set_state(*[np.asarray(a) for a in
                 (spec.x0, spec.v0, spec.C0, spec.F0)]), lambda: sc.set_walls(kind=[0, 0, 0, 0]),
                 lambda: sc.set_tuning(M.TUNE_OFF), sc.close):
        with pytest.raises(M.MPMError):
            call()
    while not batch.poll(slot):
        batch.tick(4)
    g = sc.gradients()  # results can be read once the slot is done
    assert np.all(np.isfinite(g[1]))
    with pytest.raises(M.MPMError):
        sc.step(1)  # still held until released
    batch.release(slot)
    sc.step(1)
    sc.close()
    batch.close()


def test_a_failing_scene_does_not_disturb_its_batch(M, ctx):
    """One scene of a batch throws a particle out of the grid: its status reports it, and the
    other scenes still get their alone results bit for bit."""
    good = [(S.blob(2, 32, 300, 91, v_scale=0.3, radius_cells=5.0, amp=2.0), 20),
            (S.blob(2, 48, 400, 92, v_scale=0.3, radius_cells=6.0, amp=2.0), 12)]
    bad = S.blob(2, 32, 200, 93, radius_cells=4.0).copy(bc_width=0)
    bad.x0[0] = [2.6 / 32, 0.5]
    bad.v0[0] = [-800.0, 0.0]  # leaves the grid in the first step
    alone = [_alone(M, ctx, spec, T, True) for spec, T in good]
    batch = M.Batch(ctx, 2)
    scenes = [M.Scene(ctx, spec) for spec, _ in good] + [M.Scene(ctx, bad)]
    slots = [batch.admit(sc, T, True) for sc, T in zip(scenes, [20, 12, 15])]
    for _ in range(1000):
        batch.tick(4)
        if all(batch.poll(s) for s in slots):
            break
    assert [batch.status(s) for s in slots] == [0, 0, -3]
    for sc, (st, grads) in zip(scenes[:2], alone):
        for a, b in zip(sc.get_state() + sc.gradients(), st + grads):
            assert np.array_equal(a, b)
    with pytest.raises(M.MPMError) as e:
        scenes[2].get_state()
    assert e.value.status == -3
    batch.close()
    # the serving loop reports the failed request and serves the others
    from paper_1810_01054_gb300.serve import Server
    srv = Server(device=0, mem_fraction=0.2, tick_steps=4)
    ids = [srv.submit(spec, True, n_steps=T) for spec, T in good] + [srv.submit(bad, True, n_steps=15)]
    srv.run()
    assert srv.results[ids[2]]["status"] == -3
    for rid, (st, grads) in zip(ids[:2], alone):
        r = srv.results[rid]
        for a, b in zip((r["x"], r["v"], r["C"], r["F"]) + tuple(r["grads"]), st + grads):
            assert np.array_equal(a, b)
    srv.close()
