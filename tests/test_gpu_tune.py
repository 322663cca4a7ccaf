"""Launch-shape autotuning on the GPU: trial steps are ordinary steps (bitwise the same results as
the default shapes), every tile kernel ends tuned, and the next scene of the workload reuses the
cached shapes without trials."""
import numpy as np
import pytest

from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import mean_x0_seed

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


def _run(M, ctx, spec, T, k, mode):
    sc = M.Scene(ctx, spec)
    sc.set_tuning(mode)
    sc.rollout(T, k)
    st = sc.get_state()
    g = sc.backward(mean_x0_seed(sc.N, sc.dim))
    shapes = [sc.launch(kk) for kk in range(4)]
    sc.close()
    return st, g, shapes


@pytest.mark.parametrize("spec", [S.walker_square_2d(0, n_steps=40),
                                  S.blob(3, 24, 3000, 21, radius_cells=5.0, v_scale=0.3, amp=2.0)],
                         ids=["2d", "3d"])
def test_tuned_results_are_bitwise_default_and_cached(M, ctx, spec):
    T, k = 40, 8
    st0, g0, sh0 = _run(M, ctx, spec, T, k, M.TUNE_OFF)
    adj_threads = 128 if spec.dim == 3 else 256  # the adjoint gather's CTA size is fixed per dimension
    assert sh0 == [(4, 256, False), (4, 256, False), (4, 256, False), (4, adj_threads, False)]
    st1, g1, sh1 = _run(M, ctx, spec, T, k, M.TUNE_FORCE)
    for a, b in zip(st0, st1):
        assert np.array_equal(a, b)
    for a, b in zip(g0, g1):
        assert np.array_equal(a, b)
    assert all(tuned for _, _, tuned in sh1), sh1
    p2g_threads = (128, 256) if spec.dim == 2 else (256,)
    assert sh1[M.TK_P2G][1] in p2g_threads and sh1[M.TK_P2G_ADJ][1] in p2g_threads
    assert sh1[M.TK_ADJ_GATHER][1] == adj_threads
    # a new scene of the same workload takes the cached shapes at creation
    sc = M.Scene(ctx, spec)
    assert [sc.launch(kk) for kk in range(4)] == sh1
    sc.close()



def test_p2g_with_128_thread_ctas_is_bitwise_the_default(M, ctx):
    """2D P2G and adjoint scatter with 128-thread CTAs (a thread owns up to two work items) give
    the bits of the 256-thread CTAs: the work items and every sum keep their order."""
    import torch
    spec = S.blob(2, 48, 3000, 23, radius_cells=9.0, v_scale=0.3, c_scale=0.5, amp=2.0).copy(tile_edge=4)
    T, k = 24, 6
    st0, g0, _ = _run(M, ctx, spec, T, k, M.TUNE_OFF)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    shapes = [(4, 128), (4, 256), (6, 128), (4, 256)]
    M.tune_cache_store(2, spec.n_particles, (48 // 4) ** 2, sms, shapes)
    st1, g1, sh1 = _run(M, ctx, spec, T, k, M.TUNE_AUTO)  # takes the cached shapes, no trials
    assert [s[:2] for s in sh1] == shapes
    for a, b in zip(st0 + g0, st1 + g1):
        assert np.array_equal(a, b)


def test_a_batch_tunes_its_composition_and_keeps_the_bits(M, ctx):
    """A batch whose composition has no cache entry tries the candidate shapes during its own
    steps (once the composition has run 32 steps); its results stay bitwise those of the scenes run
    alone, and afterwards the key of the composition is cached for the next batch."""
    import torch
    spec = S.blob(2, 40, 700, 24, radius_cells=6.0, v_scale=0.3, amp=2.0, dt=5e-4)
    B, T = 6, 100  # long enough for both halves' trials (they start after 32 steps of a key)
    alone = []
    for _ in range(B):
        st, g, _ = _run(M, ctx, spec, T, int(np.ceil(np.sqrt(T))), M.TUNE_OFF)
        alone.append(st + g)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    probe = M.Scene(ctx, spec)
    edge = probe.tile_edge  # the library's choice for this density (the key counts its tiles)
    probe.close()
    key = (2, B * spec.n_particles, B * ((40 + edge - 1) // edge) ** 2, sms)
    assert M.tune_cache_lookup(*key) is None
    batch = M.Batch(ctx, 2)
    scenes = [M.Scene(ctx, spec) for _ in range(B)]
    slots = [batch.admit(sc, T, True) for sc in scenes]
    while not all(batch.poll(sl) for sl in slots):
        batch.tick(4)
    for sc, ref in zip(scenes, alone):
        for a, b in zip(sc.get_state() + sc.gradients(), ref):
            assert np.array_equal(a, b)
    batch.close()
    for sc in scenes:
        sc.close()
    shapes = M.tune_cache_lookup(*key)
    assert shapes is not None and shapes[M.TK_ADJ_GATHER][1] == 256


def test_dynamic_tile_scheduling_keeps_the_bits(M, ctx):
    """With more than two active tiles per CTA the forward P2G and the adjoint gather hand out
    tiles from a counter (the CTA that computes a tile varies from run to run); with fewer they
    use the fixed stride.  A 3D scene of ~1500 active tiles run under 2 CTAs per SM (counter: more
    than 4 tiles per SM) and under 8 (fixed stride) gives the same bits, over a rollout whose
    segments are recomputed (the recompute's workspace has counters of its own) and its reverse
    pass, twice in a row (the counters are back to zero after every launch)."""
    import torch
    spec = S.blob(3, 64, 150000, 31, radius_cells=26.0, v_scale=0.3, amp=2.0, bc_width=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    x = np.asarray(spec.x0)
    t = np.floor(x / spec.dx - 0.5).astype(int) // 4
    n_active = len(np.unique((t[:, 0] * 16 + t[:, 1]) * 16 + t[:, 2]))
    assert 2 * 2 * sms < n_active <= 2 * 8 * sms
    T, k = 12, 4
    res = []
    for ctas in (8, 2, 2):
        M.tune_cache_store(3, spec.n_particles, 16 ** 3, sms, [(ctas, 256), (4, 256), (4, 256), (ctas, 256)])
        st, g, sh = _run(M, ctx, spec, T, k, M.TUNE_AUTO)
        assert sh[M.TK_P2G][0] == ctas and sh[M.TK_ADJ_GATHER][0] == ctas
        res.append(st + g)
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_tile_edge_tuning_keeps_the_faster_edge_for_new_scenes(M, ctx):
    """mpm_tune_tile_edge times a 2D workload with 4 x 4- and with 8 x 8-cell tiles, returns the
    edge of the shorter pass and caches it: a scene of that workload created afterwards with
    tile_edge 0 takes it.  A 3D workload has one tile shape (nothing runs).  The workload's key
    (6,000 particles, 96^2 grid) is one no other test uses, so the cached edge changes no other
    scene of this process."""
    spec = S.blob(2, 96, 6000, 41, radius_cells=20.0, v_scale=0.3, amp=2.0)
    edge, ms4, ms8 = M.tune_tile_edge(ctx, spec, steps=32)
    print(f"\ntile edge 4: {ms4:.4f} ms/step, 8: {ms8:.4f} ms/step -> {edge}")
    assert ms4 > 0 and ms8 > 0
    assert edge == (8 if ms8 < ms4 else 4)
    sc = M.Scene(ctx, spec)
    assert sc.tile_edge == edge
    sc.close()
    assert M.tune_tile_edge(ctx, S.blob(3, 16, 200, 42, radius_cells=3.0), steps=4) == (4, 0.0, 0.0)
