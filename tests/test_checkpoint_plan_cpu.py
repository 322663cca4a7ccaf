"""The checkpoint schedule the library plans for a memory budget (host only: mpm_plan_checkpoints
makes no CUDA call).

Below the single-level store the library plans a recursive schedule (store a state, reverse the
later part, release it, reverse the earlier part).  Its cost is checked against the same
recursion restated here, and against what any schedule must satisfy: every state kept costs no
recompute, more memory never costs more, no schedule runs fewer forward steps than the rollout,
and none stores more states than the budget allows.
"""
import functools
import math

import pytest

from paper_1810_01054_gb300 import mpm


@functools.lru_cache(maxsize=None)
def _cost(L, slots):
    """Fewest forward steps to reverse L steps from a stored start with `slots` more states."""
    best = math.inf
    for k in range(1, L + 1):  # single level: ceil(L/k) checkpoints (the start among them), k - 1 buffers
        nseg = -(-L // k)
        if nseg - 1 + k - 1 <= slots:
            best = 2 * L - nseg
            break
    if best > L and slots >= 1:
        for j in range(1, L):
            best = min(best, j + _cost(L - j, slots - 1) + _cost(j, slots))
    return best


@pytest.mark.parametrize("T", [1, 2, 7, 40, 100, 200])
@pytest.mark.parametrize("states", [3, 4, 5, 8, 11, 16])
def test_multi_level_cost_matches_the_recursion(T, states):
    fwd, used, multi = mpm.plan_checkpoints(T, states)
    assert used <= states
    k = min(T, 1 if T <= states else math.ceil(math.sqrt(T)))
    nseg = -(-T // k)
    if nseg + k - 1 <= states:  # the single-level store fits
        assert not multi and fwd == 2 * T - nseg
    else:
        assert multi and fwd == _cost(T, states - 2)


def test_every_state_kept_recomputes_nothing():
    assert mpm.plan_checkpoints(200, 0) == (200, 200, False)
    assert mpm.plan_checkpoints(200, 200) == (200, 200, False)
    # the 1M-particle cluster's budgets: 4 GiB holds 44 states of 96 MB (single level, k = 15)
    fwd, used, multi = mpm.plan_checkpoints(200, (4 << 30) // 96_000_000)
    assert not multi and used == 14 + 14 and fwd == 400 - 14


def test_more_memory_never_costs_more_and_never_less_than_the_rollout():
    """Within the multi-level regime more states never cost more forward steps.  Once the
    single-level store fits, its interval stays ceil(sqrt(T)) (it leaves room for the recompute
    to run beside the reverse steps), so its cost may exceed the best multi-level plan's just below
    that budget (at T = 200: 386 forward steps with 28 states, 383 with 27)."""
    T = 200
    prev = math.inf
    for states in range(3, 40):
        fwd, used, multi = mpm.plan_checkpoints(T, states)
        assert fwd >= T and used <= states
        if multi:
            assert fwd <= prev
            prev = fwd
        else:
            assert fwd == 2 * T - 14 and used == 28


def test_budgets_below_three_states_or_beyond_the_planner_are_refused():
    with pytest.raises(mpm.MPMError) as e:
        mpm.plan_checkpoints(200, 2)
    assert e.value.status == -2
    with pytest.raises(mpm.MPMError):
        mpm.plan_checkpoints(20000, 10)
    with pytest.raises(mpm.MPMError) as e:
        mpm.plan_checkpoints(0, 10)
    assert e.value.status == -1
