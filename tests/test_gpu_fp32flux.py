"""FP32-flux / FP64-state form against the FP64 oracle and the FP64 GPU path.

Fluxes, dissipation and SGS terms are FP32, so the bar is the precision
variant's stated relative error, not FP64 round-off:
  * state after N steps: every field within 1e-5 relative L2 of FP64;
  * one residual evaluation: within 2e-4 relative L2 (FP32 flux values differ
    by ~1e-7 relative; the centred differences of nearly equal neighbours
    amplify that by up to ~1/h);
  * conservation on the periodic box to <= 1e-10 relative over 10 steps
    (momentum components measured against the momentum scale).
"""
import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W
from parity import field_errors, oracle_grid

pytestmark = pytest.mark.gpu

TOL_STATE = 1e-5
TOL_RES = 2e-4


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


def _jet_noise(g, seed=5, amp=2e-3):
    return W.random_state(g, seed=seed, amp=amp, base_u=(0, 0, 0)) - W.random_state(g, seed=seed, amp=0.0,
                                                                                   base_u=(0, 0, 0))


def _case(name):
    if name == "box_ragged":
        g = W.box_grid(37, 29, 19, h=0.17)
        return g, W.random_state(g, seed=21, amp=0.05), W.box_params()
    if name == "wavy":
        g = W.wavy_periodic_grid(40, 28, 20, amp=0.08)
        return g, W.smooth_state(g, seed=3, amp=0.1), W.box_params(Re=200.0)
    if name == "jet_ragged":
        g = W.jet_grid(70, 34, 16)
        return g, W.jet_state(g) + _jet_noise(g), W.jet_params(seed=2)
    if name == "jet64x32x16":
        return W.make_workload("jet64x32x16")
    if name == "box32x24x16":
        return W.make_workload("box32x24x16")
    raise KeyError(name)


@pytest.mark.parametrize("name", ["box_ragged", "wavy", "jet_ragged"])
def test_fp32flux_residual(jz, name):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    got = s.residual(q)
    ref = O.residual(oracle_grid(g), torch.from_numpy(q), O.Consts(prm)).numpy()
    e2, _ = field_errors(got, ref)
    assert e2.max() <= TOL_RES, e2


@pytest.mark.parametrize("name,nsteps", [("box32x24x16", 10), ("jet_ragged", 5), ("jet64x32x16", 20)])
def test_fp32flux_steps_vs_oracle(jz, name, nsteps):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q, 0.0)
    st = s.step(nsteps)
    got = s.get_state()
    ref, t, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), nsteps)
    e2, em = field_errors(got, ref.numpy())
    assert e2.max() <= TOL_STATE, e2
    assert abs(st.t - t.item()) <= 1e-5 * t.item()


def test_fp32flux_conservation_box(jz):
    g, q, prm = W.make_workload("box32x24x16")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q)
    st0 = s.step(0)
    st = s.step(10)
    scale = np.abs(q * grid.metrics()[9]).reshape(5, -1).sum(1)
    scale[1:4] = scale[1:4].max()           # momentum components against the momentum scale
    drift = np.abs(np.array(st.totals) - np.array(st0.totals)) / scale
    assert drift.max() < 1e-10, drift


def test_fp32flux_fixed_dt_matches_fp64_path(jz):
    """Same fixed time step: FP32-flux and FP64 GPU paths agree to the variant's bound."""
    g, q, prm = _case("jet_ragged")
    prm.dt_fixed = 2e-3
    grid = jz.Grid.from_workload(g)
    a = jz.Solver(grid, prm, jz.JZ_PREC_FP64)
    b = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    for s in (a, b):
        s.set_state(q, 0.0)
        s.step(8)
    e2, _ = field_errors(b.get_state(), a.get_state())
    assert e2.max() <= TOL_STATE, e2


def test_precision_variant_jet512_500_steps(jz):
    """Jet 512 x 256 x 128 (16.8M points), 500 steps: FP32-flux vs FP64 GPU path, every field
    within 1e-5 relative L2; and the 64 x 32 x 16 subsample of the same setup vs the oracle."""
    g, q, prm = W.make_workload("jet512x256x128")
    grid = jz.Grid.from_workload(g)
    qd = torch.from_numpy(q).cuda()
    out = {}
    for prec in (jz.JZ_PREC_FP64, jz.JZ_PREC_FP32FLUX):
        s = jz.Solver(grid, prm, prec)
        s.set_state(qd, 0.0)
        s.step(500, stats=False)
        st = s.step(0)
        res = torch.empty_like(qd)
        s.get_state(res)
        out[prec] = (res.cpu().numpy(), st)
        s.close()
    e2, em = field_errors(out[jz.JZ_PREC_FP32FLUX][0], out[jz.JZ_PREC_FP64][0])
    print(f"jet512x256x128 500 steps FP32-flux vs FP64: rel L2 {e2}, rel max {em}")
    assert e2.max() <= TOL_STATE, e2
    # subsample vs the oracle
    g, q, prm = W.make_workload("jet64x32x16")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q, 0.0)
    s.step(500, stats=False)
    got = s.get_state()
    ref, _, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 500)
    e2s, ems = field_errors(got, ref.numpy())
    print(f"jet64x32x16 500 steps FP32-flux vs oracle: rel L2 {e2s}, rel max {ems}")
    assert e2s.max() <= TOL_STATE, e2s


def test_bounded_wait_runs_out_and_context_stays_usable(jz):
    """The stage kernel's bounded mbarrier wait, run on a barrier that nothing arrives at, runs
    out and returns (no hang, no trap); afterwards the context still steps a solver."""
    timed_out, ms = jz.jz_check_wait()
    print(f"bounded wait ran out after {ms:.1f} ms")
    assert timed_out == 1
    assert 0.0 < ms < 20000.0
    g, q, prm = W.make_workload("box32x24x16")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q, 0.0)
    st = s.step(2)
    assert np.isfinite(s.get_state()).all() and st.t > 0.0
