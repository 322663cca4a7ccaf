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
    assert sh1[M.TK_P2G][1] == 256 and sh1[M.TK_ADJ_GATHER][1] == adj_threads
    # a new scene of the same workload takes the cached shapes at creation
    sc = M.Scene(ctx, spec)
    assert [sc.launch(kk) for kk in range(4)] == sh1
    sc.close()
