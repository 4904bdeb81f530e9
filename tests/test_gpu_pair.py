"""Parity of the pair form (JZ_PREC_FP64PAIR: FP64 state and stage combination, fluxes,
dissipation and SGS terms in double-float arithmetic) with the CPU oracle.

The pair form stands in for the FP64 form, so it is held to the FP64 form's bars on the state:
every field <= 1e-12 relative L2 and <= 1e-11 relative max after the steps; t and dt to 1e-13.
A single residual evaluation is compared at 1e-11 relative L2: the residual is a sum of flux
differences that cancel to a few per cent of the fluxes, so its relative error is the ~2^-47
rounding of the pair arithmetic amplified by that cancellation (the state integrates it with
alpha dt).
"""
import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W
from parity import field_errors, oracle_grid

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-12
TOL_MAX = 1e-11
TOL_RES = 1e-11


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


def _case(name):
    if name == "box_ragged":
        g = W.box_grid(37, 29, 19, h=0.17)
        return g, W.random_state(g, seed=21, amp=0.05), W.box_params()
    if name == "box32x24x16":
        return W.make_workload("box32x24x16")
    if name == "wavy":
        g = W.wavy_periodic_grid(40, 28, 20, amp=0.08)
        return g, W.smooth_state(g, seed=3, amp=0.1), W.box_params(Re=200.0)
    if name == "jet_ragged":
        g = W.jet_grid(70, 34, 16)
        noise = W.random_state(g, seed=5, amp=2e-3, base_u=(0, 0, 0)) - W.random_state(g, seed=5, amp=0.0,
                                                                                      base_u=(0, 0, 0))
        return g, W.jet_state(g) + noise, W.jet_params(seed=2)
    if name == "jet64x32x16":
        return W.make_workload("jet64x32x16")
    raise KeyError(name)


@pytest.mark.parametrize("name", ["box_ragged", "wavy", "jet_ragged"])
def test_pair_residual_parity(jz, name):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    got = s.residual(q)
    ref = O.residual(oracle_grid(g), torch.from_numpy(q), O.Consts(prm)).numpy()
    e2, em = field_errors(got, ref)
    print(f"pair residual {name}: rel L2 {e2.max():.2e}, rel max {em.max():.2e}")
    assert e2.max() <= TOL_RES, e2


@pytest.mark.parametrize("name,nsteps", [("box32x24x16", 10), ("box_ragged", 3), ("wavy", 3),
                                         ("jet_ragged", 4), ("jet64x32x16", 20)])
def test_pair_rk_steps_parity(jz, name, nsteps):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    s.set_state(q, 0.25)
    st = s.step(nsteps)
    got = s.get_state()
    og, oc = oracle_grid(g), O.Consts(prm)
    ref, t, dts, R1 = O.run(og, torch.from_numpy(q), oc, nsteps, t0=0.25)
    e2, em = field_errors(got, ref.numpy())
    print(f"pair {name} {nsteps} steps: rel L2 {e2.max():.2e}, rel max {em.max():.2e}")
    assert e2.max() <= TOL_L2, e2
    assert em.max() <= TOL_MAX, em
    assert abs(st.t - t.item()) <= 1e-13 * abs(t.item())
    assert abs(st.dt - dts[-1].item()) <= 1e-13 * dts[-1].item()
    tot = O.totals(og, ref).numpy()
    scale = np.abs(ref.numpy() * og.metrics_real[9].numpy()).reshape(5, -1).sum(1)
    assert np.all(np.abs(np.array(st.totals) - tot) <= 1e-12 * scale)


def test_pair_box_conservation(jz):
    """Config 1 box: totals of Q V constant to round-off over 10 steps (the flux-form
    differences telescope; the pair rounding does not break it beyond 1e-13)."""
    g, q, prm = W.make_workload("box32x24x16")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    s.set_state(q)
    st0 = s.step(0)
    st = s.step(10)
    scale = np.abs(q * grid.metrics()[9]).reshape(5, -1).sum(1)
    drift = np.abs(np.array(st.totals) - np.array(st0.totals)) / scale
    print(f"pair box conservation drift {drift.max():.2e}")
    assert drift.max() < 1e-13


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (3, 1, 2)])
def test_pair_degenerate_periodic_boxes(jz, shape):
    g = W.box_grid(*shape, h=0.3)
    prm = W.box_params()
    q = W.random_state(g, seed=4, amp=0.05)
    grid = jz.Grid.from_workload(g)
    ref = O.residual(oracle_grid(g), torch.from_numpy(q), O.Consts(prm)).numpy()
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    got = s.residual(q)
    if np.abs(ref).max() == 0.0:
        assert np.abs(got).max() <= 1e-14
    else:
        e2, _ = field_errors(got, ref)
        assert e2.max() <= TOL_RES, e2
    qu = W.random_state(g, seed=4, amp=0.0)
    s.set_state(qu, 0.0)
    st = s.step(3)
    assert np.array_equal(s.get_state(), qu) and st.t > 0.0


def test_pair_quiescent_round_off_state(jz):
    """A jet state after one FP64 step (momenta of the quiescent region at round-off level, whose
    strain-rate squares fall below FP32's normal range): the pair residual stays finite and
    matches the FP64 form's."""
    g, q, prm = _case("jet_ragged")
    q = W.jet_state(g)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q, 0.0)
    s.step(1, stats=False)
    q1 = s.get_state()
    r64 = s.residual(q1)
    s.close()
    sp = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    rp = sp.residual(q1)
    assert np.isfinite(rp).all()
    # the mass residual of this state is ~1% of the others (the parallel jet's mass flux barely
    # varies), so every field is measured against the largest residual field norm
    scale = max(np.linalg.norm(r64[m]) for m in range(5))
    err = np.array([np.linalg.norm(rp[m] - r64[m]) for m in range(5)]) / scale
    assert err.max() <= TOL_RES, err


def test_pair_minimal_jet_grid(jz):
    g = W.jet_grid(4, 4, 4)
    prm = W.jet_params(seed=2)
    q = W.jet_state(g)
    scale = np.abs(q).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()
    grid = jz.Grid.from_workload(g)
    ref, t, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 2)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
    s.set_state(q, 0.0)
    s.step(2)
    err = np.abs(s.get_state() - ref.numpy()).reshape(5, -1).max(axis=1) / scale
    assert err.max() <= 1e-13, err


def test_pair_graph_replay_matches_plain_launches(jz):
    """Pairs of steps replayed as CUDA graphs give the same state bit for bit as plain launches
    (profiling on turns graphs off)."""
    g, q, prm = _case("jet_ragged")
    grid = jz.Grid.from_workload(g)
    out = []
    for prof in (False, True):
        s = jz.Solver(grid, prm, jz.JZ_PREC_FP64PAIR)
        s.profile(prof)
        s.set_state(q, 0.0)
        s.step(6)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_pair_adjoint_matches_fp64_adjoint(jz):
    """jz_adjoint_step on a pair-form solver (states advanced in pair arithmetic, transposed
    kernels in FP64): J and the gradient within 1e-12 of an FP64 solver's."""
    g = W.jet_grid(20, 16, 8)
    prm = W.jet_params(seed=4)
    q = W.jet_state(g)
    grid = jz.Grid.from_workload(g)
    res = []
    for prec in (jz.JZ_PREC_FP64, jz.JZ_PREC_FP64PAIR):
        s = jz.Solver(grid, prm, prec)
        s.set_state(q, 0.0)
        res.append(jz.jz_adjoint_step(s.h, np.asarray(prm.forcing_amp), 4, 2, 0.75))
        s.close()
    assert abs(res[0][0] - res[1][0]) <= 1e-12 * abs(res[0][0])
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-12 * np.abs(res[0][1]).max()


def test_pair_arithmetic_against_fp64(jz):
    """The double-float operations on 2^20 operand sets against FP64: every one within ~2^-44
    (sums and fused multiply-adds relative to the operands' magnitudes), the round trip of an
    FP64 value through a pair within 2^-46, and roots of arguments below 1e-30 (the FP32
    fallbacks) within FP32 rounding."""
    e = jz.jz_check_pair()
    print("pair arithmetic max errors:", {k: f"{v:.2e}" for k, v in e.items()})
    for k in ("add", "mul", "fma", "rcp", "sqrt", "cbrt"):
        assert e[k] <= 2.0 ** -44, (k, e[k])
    assert e["roundtrip"] <= 2.0 ** -46
    # below 1e-30 the roots are the FP32 fallbacks: FP32 rounding of the argument and result
    assert e["sqrt_tiny"] <= 2.0 ** -22 and e["cbrt_tiny"] <= 2.0 ** -21
