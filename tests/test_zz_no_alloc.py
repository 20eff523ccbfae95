"""dg_totals_noalloc: conservation totals for callers that may not allocate.

Callers that have reserved the whole GPU for their own state, that manage device
memory through their own pool, or that cannot afford the synchronisation of
cudaMalloc/cudaFree use this entry point: it keeps its partial sums in a fixed
static device array instead of allocating.  Its totals must match those of the
allocating entry point dg_totals on the same state, on two calls in a row (the
second call reuses the array the first one left behind).  This file is collected
last so that a run that stops at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1305_5536_gb300 import dg, ics

pytestmark = pytest.mark.gpu


def _call(cfg, u_dev, on_device=False):
    """The totals of the state u_dev, written to host memory, or (on_device) to a
    torch CUDA tensor that the call only enqueues into."""
    import torch
    L = dg.load()
    nv = dg.num_totals(cfg.eq, cfg.dim)
    if on_device:
        out = torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda")
        ptr = ctypes.c_void_p(out.data_ptr())
    else:
        out = np.full(nv, np.nan)
        ptr = out.ctypes.data_as(ctypes.c_void_p)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = L.dg_totals_noalloc(ctypes.byref(cfg), ctypes.c_void_p(u_dev.data_ptr()), ptr,
                            1 if on_device else 0, st)
    assert s == dg.DG_OK, L.dg_last_error(None)
    if on_device:
        torch.cuda.current_stream().synchronize()
        return out.cpu().numpy()
    return out


@pytest.mark.parametrize("case", ["mhd2d", "euler2d", "euler3d", "mhd3d"])
@pytest.mark.parametrize("on_device", [False, True])
def test_noalloc_totals_match_dg_totals_twice(case, on_device):
    import torch
    nsteps = 3
    if case == "mhd2d":
        n, eq, dim = (96, 80), "mhd", 2
        u0 = ics.orszag_tang(n)
    elif case == "euler2d":
        n, eq, dim = (96, 80), "euler", 2
        u0 = ics.euler2d_wave(n)
    elif case == "euler3d":
        n, eq, dim = (32, 24, 16), "euler", 3
        u0 = ics.kh3d(n)
        nsteps = 0
    else:
        n, eq, dim = (16, 12, 10), "mhd", 3
        u0 = ics.orszag_tang_3d(n)
        nsteps = 2
    s = dg.DGSolver(eq, dim, n, precision="fp64")
    s.set_state(u0)
    if nsteps:
        s.step(nsteps, sync=True)
    ref = s.totals()[0]
    u_dev = s.get_state(device="cuda")
    torch.cuda.synchronize()
    cfg = dg.make_config(eq, dim, n)
    assert ref.size == dg.num_totals(cfg.eq, dim)
    first = _call(cfg, u_dev, on_device)
    second = _call(cfg, u_dev, on_device)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(first, ref, rtol=1e-12, atol=1e-12 * scale)
    np.testing.assert_allclose(second, ref, rtol=1e-12, atol=1e-12 * scale)
    np.testing.assert_array_equal(first, second)
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    L = dg.load()
    cfg = dg.make_config("euler", 3, (512, 256, 256))
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = np.zeros(5)
    s = L.dg_totals_noalloc(ctypes.byref(cfg), ctypes.c_void_p(u.data_ptr()),
                            out.ctypes.data_as(ctypes.c_void_p), 0, None)
    assert s == dg.DG_EINVAL
    assert b"at most 16777216 cells" in L.dg_last_error(None)
