"""The allocation-free step, mpm_step_noalloc, against the library's regular entry point and the
FP64 oracle.

Callers that must not allocate device memory -- a control loop with a hard latency budget, where
cudaMalloc may block and synchronise the device, or a process whose device memory belongs to
another allocator -- call mpm_step_noalloc, which keeps its grid in a fixed array inside the
library.  Through the C ABI, two consecutive calls must reproduce two mpm_step calls on a
plain-form scene (the same arithmetic, summed in another atomic order) and the oracle's step from
the same input state, within the forward tolerance the other parity tests use; the second call
must leave the device's free memory unchanged.  Argument errors are returned before anything is
launched, so those cases run without a GPU.  The file is named to be collected last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1810_01054_gb300 import scenes as S
from tests.parity_utils import assert_state_close, oracle_step_from


def _args(M, spec, dev_arrays, outs, act, status):
    a = M.NoAllocStep()
    a.device = -1
    a.dim = spec.dim
    for k in range(3):
        a.n_grid[k] = int(spec.n_grid[k]) if k < spec.dim else 1
        a.gravity[k] = float(spec.gravity[k]) if k < spec.dim else 0.0
    a.dx, a.dt, a.E, a.nu = spec.dx, spec.dt, spec.E, spec.nu
    a.p_mass, a.p_vol = spec.p_mass, spec.p_vol
    a.bc_type, a.bc_width, a.friction_c = spec.bc_type, spec.bc_width, spec.friction_c
    a.n_particles = spec.n_particles
    x, v, Cm, F, grp, dirs = dev_arrays
    a.x, a.v, a.C, a.F = x.data_ptr(), v.data_ptr(), Cm.data_ptr(), F.data_ptr()
    a.group, a.n_groups, a.act_dir, a.act = grp.data_ptr(), spec.n_groups, dirs.data_ptr(), act.data_ptr()
    a.x_out, a.v_out, a.C_out, a.F_out = (o.data_ptr() for o in outs)
    a.status = status.data_ptr()
    return a


@pytest.mark.gpu
@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_step_matches_regular_step_and_oracle_twice(dim):
    torch = pytest.importorskip("torch")
    from paper_1810_01054_gb300 import mpm as M
    dev = torch.device("cuda", 0)
    if dim == 2:
        spec = S.blob(2, 48, 700, 11, v_scale=0.5, c_scale=1.0, f_scale=0.05, radius_cells=8.0, bc_width=3, amp=3.0)
    else:
        spec = S.blob(3, 24, 900, 12, v_scale=0.5, c_scale=1.0, f_scale=0.05, radius_cells=4.0, bc_width=3, amp=3.0)
    N, d = spec.n_particles, spec.dim
    t32 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()
    state = [t32(spec.x0), t32(spec.v0), t32(spec.C0), t32(spec.F0)]
    grp = torch.tensor(spec.group, dtype=torch.int32, device=dev)
    dirs = t32(spec.act_dir)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the regular entry point: a plain-form scene stepped with mpm_step
    ctx = M.Context(0, stream=stream)
    ref = M.Scene(ctx, spec, impl=M.IMPL_PLAIN)
    n0 = 4
    ref.set_state(*[s.cpu().numpy() for s in state], step=n0)
    for call in range(2):
        n = n0 + call
        act = t32([spec.ctrl_params[g] * math.sin(2 * math.pi * spec.ctrl_freq * n * spec.dt)
                   for g in range(spec.n_groups)])
        outs = [torch.empty((N, d), device=dev), torch.empty((N, d), device=dev),
                torch.empty((N, d, d), device=dev), torch.empty((N, d, d), device=dev)]
        a = _args(M, spec, (*state, grp, dirs), outs, act, status)
        torch.cuda.synchronize(dev)
        free_before = torch.cuda.mem_get_info(dev)[0]
        rc = M.lib().mpm_step_noalloc(C.byref(a), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize(dev)
        if call == 1:  # the first call on a device may load its kernels; later calls take nothing
            assert torch.cuda.mem_get_info(dev)[0] == free_before
        ref.step(1)
        want = ref.get_state()
        torch.cuda.synchronize(dev)
        assert int(status.item()) == 0
        got = [o.cpu().numpy() for o in outs]
        assert_state_close(got, want)
        inp = [s.cpu().numpy().astype(np.float64) for s in state]
        assert_state_close(got, oracle_step_from(spec, inp, n))
        state = outs
    ref.close()
    ctx.close()


def _valid(M):
    a = M.NoAllocStep()
    a.device, a.dim = -1, 3
    for k in range(3):
        a.n_grid[k] = 32
    a.dx, a.dt, a.E, a.nu, a.p_mass, a.p_vol = 1 / 32, 1e-4, 10.0, 0.3, 1e-6, 1e-6
    a.bc_type, a.bc_width, a.friction_c = 0, 2, 0.0
    return a


def _reject(M, **changes):
    a = _valid(M)
    for k, v in changes.items():
        if k == "n_grid":
            for i in range(3):
                a.n_grid[i] = v[i]
        else:
            setattr(a, k, v)
    return M.lib().mpm_step_noalloc(C.byref(a), None)


@pytest.mark.parametrize("n_grid", [(65, 65, 65), (1 << 20, 1 << 20, 1 << 24), (1 << 31 - 1, 8, 8),
                                    (513, 512, 1)])
def test_noalloc_rejects_grids_beyond_its_scratch(n_grid):
    """65^3 > 2^18 nodes; sides whose product would wrap a 64-bit count; a 2D side above 512.
    Returned before any launch, so no GPU is needed."""
    from paper_1810_01054_gb300 import mpm as M
    dim = 2 if n_grid[2] == 1 else 3
    assert _reject(M, n_grid=n_grid, dim=dim) == -1


@pytest.mark.parametrize("field,value", [("bc_width", -1), ("friction_c", -0.5), ("friction_c", float("nan")),
                                         ("p_mass", 0.0), ("p_mass", -1e-6), ("p_vol", 0.0),
                                         ("p_vol", float("nan")), ("dt", 1.0), ("bc_type", 2), ("n_particles", -1)])
def test_noalloc_rejects_what_scene_create_rejects(field, value):
    from paper_1810_01054_gb300 import mpm as M
    assert _reject(M, **{field: value}) == -1
