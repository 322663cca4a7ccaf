"""Host logic of the rollout autograd Function (CPU only, with a stand-in scene that records the
calls): a backward runs the reverse pass of the rollout its graph recorded, and is refused once the
scene has been rolled out, stepped or changed again since that forward."""
import pytest

torch = pytest.importorskip("torch")

from paper_1810_01054_gb300.rollout import rollout  # noqa: E402


class _FakeScene:
    """Stands in for mpm.Scene: same generation rule, outputs filled with the call counts."""

    def __init__(self, N=5, dim=2):
        self.N, self.dim, self.generation = N, dim, 0
        self.rollouts = 0
        self.backwards = 0

    def _touch(self):
        self.generation += 1

    def set_params(self, p):
        self._touch()

    def set_state(self, *a, step=-1):
        self._touch()

    def rollout(self, n, k=0, budget=0):
        self._touch()
        self.rollouts += 1

    def get_state(self, out):
        for o in out:
            o.fill_(float(self.rollouts))
        return out

    def backward(self, *seeds, out):
        self.backwards += 1
        for o in out:
            o.fill_(float(self.backwards))
        return out


def _leaves(N=5, d=2):
    mk = lambda *s: torch.zeros(*s, requires_grad=True)
    return mk(N, d), mk(N, d), mk(N, d, d), mk(N, d, d), mk(3)


def test_backward_of_the_latest_rollout_runs():
    sc = _FakeScene()
    x0, v0, C0, F0, p = _leaves()
    xT, *_ = rollout(sc, 10, x0, v0, C0, F0, p)
    xT.sum().backward()
    assert sc.backwards == 1 and torch.all(v0.grad == 1.0)


@pytest.mark.parametrize("change", ["rollout", "set_state", "set_params"])
def test_backward_through_a_stale_rollout_is_refused(change):
    sc = _FakeScene()
    x0, v0, C0, F0, p = _leaves()
    xT, *_ = rollout(sc, 10, x0, v0, C0, F0, p)
    if change == "rollout":
        rollout(sc, 10, *_leaves())
    elif change == "set_state":
        sc.set_state(None)
    else:
        sc.set_params(None)
    with pytest.raises(RuntimeError, match="rolled out"):
        xT.sum().backward()
    assert sc.backwards == 0
