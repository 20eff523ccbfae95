"""Two contexts driven from two host threads at once.

A caller that steps independent problems held in host memory can overlap one
problem's host-link transfers with another's kernels by giving each problem a
context and a stream of its own and driving each from its own host thread (the
library's calls release the GIL).  The contexts share no mutable state on the
stepping path, and the process-wide tile-shape tuning is serialised inside the
library, so each context must produce exactly the states it produces when driven
alone: set_state from page-locked host memory, steps (graph replay included),
get_state into page-locked host memory, repeated.
"""
import threading

import numpy as np
import pytest
import torch

from paper_1305_5536_gb300 import dg, ics

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eq,n,prec", [("mhd", (96, 80), "fp32"), ("mhd", (96, 80), "fp64"),
                                       ("euler", (72, 56), "fp32")])
def test_two_contexts_two_threads_match_one_context_alone(eq, n, prec):
    u0 = ics.orszag_tang(n) if eq == "mhd" else ics.euler2d_wave(n)
    ref = dg.DGSolver(eq, 2, n, precision=prec)
    ref.set_state(u0)
    ref.step(5, sync=True)
    want = ref.get_state()
    ref.close()

    host_in = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    solvers = [dg.DGSolver(eq, 2, n, precision=prec, stream=s.cuda_stream) for s in streams]
    errors = []

    def run(i):
        try:
            for _ in range(4):
                solvers[i].set_state(host_in)
                solvers[i].step(5)
                solvers[i].get_state(outs[i])
        except Exception as exc:  # reported on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    for s in solvers:
        s.close()
    assert not errors, errors
    for out in outs:
        np.testing.assert_array_equal(out.numpy(), want)
