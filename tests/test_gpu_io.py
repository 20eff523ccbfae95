"""State transfer through the C ABI: pageable host memory (staged plane by plane
through device scratch), page-locked host memory (read and written in place by
the layout kernels) and device memory give bit-identical states, for every
equation set, both precisions and a batch of problems."""
import numpy as np
import pytest

from paper_1305_5536_gb300 import dg, ics

pytestmark = pytest.mark.gpu

CASES = [("euler", 2, (24, 20)), ("mhd", 2, (24, 20)), ("euler", 3, (8, 6, 5)),
         ("mhd", 3, (8, 6, 5))]


def _state(eq, dim, n):
    if eq == "mhd":
        return ics.orszag_tang_3d(n) if dim == 3 else ics.orszag_tang(n)
    return ics.kh3d(n, w0=0.1) if dim == 3 else ics.euler2d_wave(n, noise=1e-2)


def _three_ways(make, u):
    """Set the state from pageable, page-locked and device memory; after two
    steps read it back into all three kinds; every copy must agree bit for bit."""
    import torch
    pinned = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    dev = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    outs = []
    for src in (u, pinned, dev):
        s = make()
        s.set_state(src)
        s.step(2, sync=True)
        a = s.get_state()
        b = torch.empty(u.shape, dtype=torch.float64).pin_memory()
        s.get_state(b)
        c = s.get_state(device="cuda")
        s.close()
        np.testing.assert_array_equal(a, b.numpy())
        np.testing.assert_array_equal(a, c.cpu().numpy().reshape(a.shape))
        outs.append(a)
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    return outs[0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("eq,dim,n", CASES)
def test_state_transfer_paths_agree(eq, dim, n, prec):
    u = _state(eq, dim, n)
    out = _three_ways(lambda: dg.DGSolver(eq, dim, n, precision=prec), u)
    assert not np.array_equal(out, u)  # the steps did run


def test_state_transfer_paths_agree_batch():
    sizes = (16, 24, 40)
    cfgs = [dg.make_config("mhd", 2, (N, N), precision="fp32") for N in sizes]
    u = np.concatenate([ics.orszag_tang((N, N)).ravel() for N in sizes])
    _three_ways(lambda: dg.DGSolver(configs=cfgs), u)


def test_init_reports_enomem_when_the_state_does_not_fit():
    """Maximum sizes: a configuration the check accepts (1.95e9 cells, under its
    2e9 limit) whose state does not fit the device (3D MHD in FP64: three state
    buffers of 484 GB each).  dg_init takes the first buffer (125 GB), fails on the
    next with DG_ENOMEM and its message, frees what it took, and the device stays
    usable for the next context."""
    with pytest.raises(dg.DGError) as err:
        dg.DGSolver("mhd", 3, (1250, 1250, 1250), precision="fp64")
    assert err.value.status == dg.DG_ENOMEM
    assert "allocation" in str(err.value)
    n = (32, 32)
    s = dg.DGSolver("euler", 2, n, precision="fp64")
    s.set_state(ics.euler2d_wave(n))
    s.step(2, sync=True)
    s.close()
