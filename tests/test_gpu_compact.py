"""Compact grids (jz_grid_compact): FP32 metrics only, for meshes whose FP64 grid would not fit
next to the solver.  With a fixed time step the FP32-flux form steps bit for bit as on the full
grid (the fused kernel reads the same FP32 metrics and the boundary conditions the same FP64
surface copies); with the CFL step only the first step's rate (FP32 metrics widened) differs."""
import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W
from parity import field_errors, oracle_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


def _jet():
    g = W.jet_grid(70, 34, 16)
    noise = W.random_state(g, seed=5, amp=2e-3, base_u=(0, 0, 0)) - W.random_state(g, seed=5, amp=0.0,
                                                                                   base_u=(0, 0, 0))
    return g, W.jet_state(g) + noise


def _run(jz, g, q, prm, compact, nsteps):
    grid = jz.Grid.from_workload(g)
    if compact:
        grid.compact()
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q, 0.0)
    st = s.step(nsteps)
    out = s.get_state()
    s.close()
    grid.close()
    return out, st


def test_compact_fixed_dt_bit_identical(jz):
    g, q = _jet()
    prm = W.jet_params(seed=2, dt_fixed=2e-3)
    a, sa = _run(jz, g, q, prm, False, 6)
    b, sb = _run(jz, g, q, prm, True, 6)
    assert np.array_equal(a, b) and sa.t == sb.t
    # totals: FP64 V against FP32 V widened
    assert np.abs(np.array(sa.totals) - np.array(sb.totals)).max() <= 1e-6 * np.abs(sa.totals).max()


@pytest.mark.parametrize("dt_fixed", [0.0, 2e-3])
def test_compact_grid_against_oracle(jz, dt_fixed):
    """A compact grid (the form the paper's largest meshes run in) against the FP64 oracle
    directly: the ragged jet over 20 steps of the FP32-flux form, with the CFL step and with
    a fixed step, within the form's stated bound 1e-5 per field; the time to 1e-6."""
    g, q = _jet()
    prm = W.jet_params(seed=2, dt_fixed=dt_fixed)
    got, st = _run(jz, g, q, prm, True, 20)
    ref, t, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 20)
    e2, em = field_errors(got, ref.numpy())
    print(f"compact grid FP32-flux 20 steps vs oracle (dt_fixed={dt_fixed}): rel L2 {e2}, rel max {em}")
    assert e2.max() <= 1e-5, e2
    assert em.max() <= 1e-5, em
    assert abs(st.t - t.item()) <= 1e-6 * t.item()


def test_compact_cfl_step(jz):
    g, q = _jet()
    prm = W.jet_params(seed=2)
    a, sa = _run(jz, g, q, prm, False, 6)
    b, sb = _run(jz, g, q, prm, True, 6)
    e2, _ = field_errors(b, a)
    assert e2.max() <= 1e-6, e2
    assert abs(sa.t - sb.t) <= 1e-6 * sa.t


def test_compact_refusals_and_memory(jz):
    g = W.jet_grid(256, 128, 64)
    grid = jz.Grid.from_workload(g)
    prm = W.jet_params(seed=2)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    with pytest.raises(jz.JzError, match="still use"):
        grid.compact()
    s.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    grid.compact()
    grid.compact()                                   # idempotent
    free1, _ = torch.cuda.mem_get_info()
    padded = ((256 + 4 + 3) // 4 * 4) * (128 + 4) * (64 + 4)
    assert free1 - free0 >= 0.9 * 96 * padded          # 144 B of FP64 arrays out, 48 B of FP32 records in
    with pytest.raises(jz.JzError, match="compact"):
        jz.Solver(grid, prm, jz.JZ_PREC_FP64)
    with pytest.raises(jz.JzError, match="compact"):
        grid.metrics()
    params = jz.make_params(prm, jz.JZ_PREC_FP64)
    qd = torch.from_numpy(W.jet_state(g)).cuda()
    with pytest.raises(jz.JzError, match="compact"):
        jz.jz_residual_noalloc(grid.h, params, qd, torch.empty_like(qd))
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(qd, 0.0)
    st = s.step(2)
    assert st.min_p > 0.7
