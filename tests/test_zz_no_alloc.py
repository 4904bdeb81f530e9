"""The allocation-free residual entry point (jz_residual_noalloc).

It serves callers that cannot let the library allocate device memory (their
memory belongs to another allocator under a fixed budget, or their loop
cannot absorb cudaMalloc/cudaFree and the device synchronisation of
cudaFree).  It uses a fixed scratch array inside the library instead.  This
file is collected last on purpose: it checks, through the C ABI, that calls
in a row reproduce the allocating jz_residual without allocating (a larger
grid before a smaller one, a side stream included), and that a grid larger
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


def _noisy(g, seed):
    return W.jet_state(g) + (W.random_state(g, seed=seed, amp=2e-3, base_u=(0, 0, 0))
                             - W.random_state(g, seed=seed, amp=0.0, base_u=(0, 0, 0)))


def _check_against_residual(jz, g, q, stream=None):
    """One call of the allocation-free entry point against the allocating jz_residual; the
    call itself must allocate nothing (torch's allocator and the device's free memory are
    unchanged around it)."""
    prm = W.jet_params(seed=2)
    grid = jz.Grid.from_workload(g)
    solver = jz.Solver(grid, prm)
    qd = torch.from_numpy(q).cuda()
    ref = torch.empty_like(qd)
    solver.residual(qd, ref)
    out = torch.full_like(qd, float("nan"))
    params = jz.make_params(prm)
    if stream is not None:
        with torch.cuda.stream(stream):
            out.add_(0.0)                          # first launch on the stream before the measurement
    torch.cuda.synchronize()
    alloc0, (free0, _) = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()
    if stream is None:
        jz.jz_residual_noalloc(grid.h, params, qd, out)
    else:
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            jz.jz_residual_noalloc(grid.h, params, qd, out)      # torch's current stream is `stream`
        torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    alloc1, (free1, _) = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()
    assert alloc1 == alloc0 and free1 == free0, (alloc0, alloc1, free0, free1)
    e2, em = field_errors(out.cpu().numpy(), ref.cpu().numpy())
    assert e2.max() <= 1e-12, e2
    assert em.max() <= 1e-11, em
    solver.close()
    grid.close()


def test_noalloc_matches_residual_twice(jz):
    """Two calls in a row on different states (the second cannot pass on the first one's scratch),
    then a larger grid followed by a smaller one (what the larger one left in the array beyond
    the smaller one's range must not leak into its result), then a call on a torch side stream.
    A first call in the process looks up the array's address (and, with lazy module loading,
    loads the module that holds it), so it runs before the allocation checks."""
    g = W.jet_grid(40, 24, 16)
    prm = W.jet_params(seed=2)
    grid = jz.Grid.from_workload(g)
    qd = torch.from_numpy(W.jet_state(g)).cuda()
    out = torch.empty_like(qd)
    jz.jz_residual_noalloc(grid.h, jz.make_params(prm), qd, out)
    torch.cuda.synchronize()
    grid.close()
    for seed in (31, 32):
        _check_against_residual(jz, g, _noisy(g, seed))
    big = W.jet_grid(44, 36, 24)
    _check_against_residual(jz, big, _noisy(big, 33))
    small = W.jet_grid(20, 12, 8)
    _check_against_residual(jz, small, _noisy(small, 34))
    _check_against_residual(jz, g, _noisy(g, 35), stream=torch.cuda.Stream())


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
