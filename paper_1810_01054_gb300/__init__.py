"""GB300-native differentiable MLS-MPM (ChainQueen, arXiv 1810.01054) hot path.

The compute path is the C-ABI library ``libgbmpm.so`` (hand-written sm_103a CUDA kernels,
declared in ``include/mpm.h``); ``paper_1810_01054_gb300.mpm`` is its thin ctypes binding and
``paper_1810_01054_gb300.rollout`` the torch autograd wrapper.  Submodules are imported lazily
so that the seeded input builders in ``scenes`` load without a GPU or a built library.
"""

__all__ = ["scenes", "mpm", "rollout", "serve"]
