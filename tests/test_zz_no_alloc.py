"""The allocation-free residual entry point (jz_residual_noalloc).

It serves callers that cannot let the library allocate device memory (their
memory belongs to another allocator under a fixed budget, or their loop
cannot absorb cudaMalloc/cudaFree and the device synchronisation of
cudaFree).  It uses a fixed scratch array inside the library instead.  This
file is collected last on purpose: it checks, through the C ABI, that two
calls in a row reproduce the allocating jz_residual, and that a grid larger
than the fixed scratch is refused with a clear error.
"""
import numpy as np
import pytest
import torch

from paper_2003_08746_gb300 import workloads as W
from parity import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


def test_noalloc_matches_residual_twice(jz):
    g = W.jet_grid(40, 24, 16)
    prm = W.jet_params(seed=2)
    grid = jz.Grid.from_workload(g)
    solver = jz.Solver(grid, prm)
    params = jz.make_params(prm)
    base = W.jet_state(g)
    # two different states so that the second call cannot pass on stale scratch
    states = [base + (W.random_state(g, seed=s, amp=2e-3, base_u=(0, 0, 0))
                      - W.random_state(g, seed=s, amp=0.0, base_u=(0, 0, 0))) for s in (31, 32)]
    for q in states:
        qd = torch.from_numpy(q).cuda()
        ref = torch.empty_like(qd)
        solver.residual(qd, ref)
        out = torch.full_like(qd, float("nan"))
        jz.jz_residual_noalloc(grid.h, params, qd, out)
        torch.cuda.synchronize()
        e2, em = field_errors(out.cpu().numpy(), ref.cpu().numpy())
        assert e2.max() <= 1e-12, e2
        assert em.max() <= 1e-11, em
    solver.close()
    grid.close()


def test_noalloc_rejects_grids_beyond_the_scratch(jz):
    g = W.box_grid(64, 64, 64, h=0.1)           # 68^3 padded nodes > the fixed maximum
    prm = W.box_params()
    grid = jz.Grid.from_workload(g)
    q = torch.from_numpy(W.box_state(g)).cuda()
    out = torch.empty_like(q)
    with pytest.raises(jz.JzError) as ei:
        jz.jz_residual_noalloc(grid.h, jz.make_params(prm), q, out)
    assert ei.value.code == jz.JZ_ERR_ARG
    assert "maximum" in str(ei.value)
    grid.close()
