"""Parity of the CUDA path (through the C ABI) with the CPU oracle, FP64 form.

Element-wise comparison on the same seeded inputs.  Bar: relative L2 error of
every field <= 1e-12 (and max-abs error <= 1e-11 of the field's scale).
"""
import math

import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W
from parity import field_errors, oracle_grid

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-12
TOL_MAX = 1e-11


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
        # parallel jet plus a small seeded perturbation of every conserved variable
        noise = W.random_state(g, seed=5, amp=2e-3, base_u=(0, 0, 0)) - W.random_state(g, seed=5, amp=0.0,
                                                                                      base_u=(0, 0, 0))
        return g, W.jet_state(g) + noise, W.jet_params(seed=2)
    if name == "jet64x32x16":
        return W.make_workload("jet64x32x16")
    raise KeyError(name)


CASES = ["box_ragged", "wavy", "jet_ragged"]


@pytest.mark.parametrize("name", CASES)
def test_metrics_parity(jz, name):
    g, _, _ = _case(name)
    grid = jz.Grid.from_workload(g)
    got = grid.metrics()
    ref = oracle_grid(g).metrics_real.numpy()
    scale = np.abs(ref[:9]).max()
    assert np.abs(got[:9] - ref[:9]).max() <= 1e-13 * scale
    assert np.abs(got[9] - ref[9]).max() <= 1e-13 * np.abs(ref[9]).max()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("where", ["host", "device"])
def test_residual_parity(jz, name, where):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    if where == "host":
        got = s.residual(q)
    else:
        qd = torch.from_numpy(q).cuda()
        out = torch.empty_like(qd)
        s.residual(qd, out)
        got = out.cpu().numpy()
    ref = O.residual(oracle_grid(g), torch.from_numpy(q), O.Consts(prm)).numpy()
    e2, em = field_errors(got, ref)
    assert e2.max() <= TOL_L2, e2
    assert em.max() <= TOL_MAX, em


@pytest.mark.parametrize("name,nsteps", [("box32x24x16", 10), ("box_ragged", 3), ("wavy", 3),
                                         ("jet_ragged", 4), ("jet64x32x16", 20)])
def test_rk_steps_parity(jz, name, nsteps):
    g, q, prm = _case(name)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q, 0.25)
    st = s.step(nsteps)
    got = s.get_state()
    og, oc = oracle_grid(g), O.Consts(prm)
    ref, t, dts, R1 = O.run(og, torch.from_numpy(q), oc, nsteps, t0=0.25)
    e2, em = field_errors(got, ref.numpy())
    assert e2.max() <= TOL_L2, e2
    assert em.max() <= TOL_MAX, em
    assert abs(st.t - t.item()) <= 1e-13 * abs(t.item())
    assert abs(st.dt - dts[-1].item()) <= 1e-13 * dts[-1].item()
    assert st.steps == nsteps
    res = O.residual_l2(og, R1).item()
    assert abs(st.res_l2 - res) <= 1e-11 * res
    tot = O.totals(og, ref).numpy()
    scale = np.abs(ref.numpy() * og.metrics_real[9].numpy()).reshape(5, -1).sum(1)
    assert np.all(np.abs(np.array(st.totals) - tot) <= 1e-13 * scale)


def test_box_conservation_on_gpu(jz):
    """Config 1 box: totals of Q V constant to round-off over 10 steps on the GPU path."""
    g, q, prm = W.make_workload("box32x24x16")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q)
    st0 = s.step(0)
    st = s.step(10)
    scale = np.abs(q * grid.metrics()[9]).reshape(5, -1).sum(1)
    drift = np.abs(np.array(st.totals) - np.array(st0.totals)) / scale
    assert drift.max() < 1e-13


def test_fixed_dt_and_time(jz):
    g, q, prm = _case("jet_ragged")
    prm.dt_fixed = 1e-3
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q, 1.5)
    st = s.step(3)
    assert st.dt == 1e-3 and abs(st.t - 1.503) < 1e-14
    ref, _, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 3, t0=1.5)
    e2, _ = field_errors(s.get_state(), ref.numpy())
    assert e2.max() <= TOL_L2


def test_nonfinite_state_is_reported(jz):
    """A NaN in the state is reported as JZ_ERR_NONFINITE by the statistics (host-side check)."""
    g, q, prm = _case("box_ragged")
    q = q.copy()
    q[0, 3, 4, 5] = np.nan
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q)
    with pytest.raises(jz.JzError) as ei:
        s.step(0)
    assert ei.value.code == jz.JZ_ERR_NONFINITE


def test_jet_full_size_one_step(jz):
    """Jet 256 x 128 x 64 (2.1M points): one full RK step against the oracle."""
    g, q, prm = W.make_workload("jet256x128x64")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(torch.from_numpy(q).cuda())
    s.step(1)
    got = s.get_state()
    ref, _, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 1)
    e2, em = field_errors(got, ref.numpy())
    assert e2.max() <= TOL_L2, e2
    assert em.max() <= TOL_MAX, em


def _window_residual(g, q, prm, i, j, k, W=5):
    """Oracle residual at node (i, j, k) of a large grid from an (2W+1)^3 window around it.

    The residual at a node depends on coordinates within 3 nodes and on the state within
    2 nodes, so the window's own (wrapped, meaningless) ghost layers never reach its centre.
    """
    sl = (slice(k - W, k + W + 1), slice(j - W, j + W + 1), slice(i - W, i + W + 1))
    xyz = np.ascontiguousarray(g.xyz[(slice(None),) + sl])
    qw = np.ascontiguousarray(q[(slice(None),) + sl])
    n = 2 * W + 1
    grid = O.Grid(n, n, n, xyz, O.TOPO_PERIODIC, np.zeros((3, 3)))
    R = O.residual_padded(grid, grid.pad(torch.from_numpy(qw)), O.Consts(prm))
    return R[:, W, W, W].numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32flux"])
def test_full_size_sampled_residual(jz, precision):
    """Jet 1000 x 400 x 500 (the benchmark workload, same launch configuration): the GPU
    residual at 24 seeded interior nodes against the oracle on a window around each node."""
    g, q, prm = W.make_workload("jet1000x400x500")
    rng = np.random.Generator(np.random.PCG64(77))
    q = q + 1e-3 * rng.standard_normal(q.shape) * np.array([1, 1, 1, 1, 1])[:, None, None, None]
    grid = jz.Grid.from_workload(g)
    prec = jz.JZ_PREC_FP64 if precision == "fp64" else jz.JZ_PREC_FP32FLUX
    s = jz.Solver(grid, prm, prec)
    qd = torch.from_numpy(q).cuda()
    rd = torch.empty_like(qd)
    s.residual(qd, rd)
    nodes = [(int(rng.integers(6, g.ni - 6)), int(rng.integers(6, g.nj - 6)), int(rng.integers(6, g.nk - 6)))
             for _ in range(24)]
    tol = 1e-11 if precision == "fp64" else 2e-4
    for (i, j, k) in nodes:
        got = rd[:, k, j, i].cpu().numpy()
        ref = _window_residual(g, q, prm, i, j, k)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol * scale, (i, j, k, got, ref)
    s.close()
    grid.close()


@pytest.fixture(scope="module")
def jet64_500_ref():
    g, q, prm = W.make_workload("jet64x32x16")
    ref, _, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 500)
    return g, q, prm, ref.numpy()


@pytest.mark.parametrize("precision", ["fp64", "pair"])
def test_jet_subsample_500_steps_fp64(jz, jet64_500_ref, precision):
    """The 64 x 32 x 16 jet (the precision workload's subsample), 500 steps of the FP64 form and
    of its pair form against the oracle."""
    g, q, prm, ref = jet64_500_ref
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64 if precision == "fp64" else jz.JZ_PREC_FP64PAIR)
    s.set_state(q, 0.0)
    s.step(500, stats=False)
    got = s.get_state()
    e2, em = field_errors(got, ref)
    print(f"jet64x32x16 {precision} 500 steps vs oracle: rel L2 {e2}, rel max {em}")
    assert e2.max() <= TOL_L2, e2


def test_fp64_reciprocal_roots(jz):
    """The FP64 form's own reciprocal, cube roots and square root (third-order Householder
    steps from hardware or FP32 seeds) against IEEE division, the CUDA cbrt and IEEE sqrt on
    2^20 arguments over [1e-30, 1e30] and 0: within 2, 4 and 2 units of 2^-52 relative."""
    e_rcp, e_cbrt, e_sqrt = jz.jz_check_math()
    print(f"rcp64 {e_rcp:.3e}, cbrt_pair64 {e_cbrt:.3e}, sqrt64 {e_sqrt:.3e} max rel err")
    assert e_rcp <= 2 * 2.0 ** -52
    assert e_cbrt <= 4 * 2.0 ** -52
    assert e_sqrt <= 2 * 2.0 ** -52


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (3, 1, 2)])
def test_degenerate_periodic_boxes(jz, shape):
    """Periodic boxes one to three nodes wide (every stencil neighbour wraps onto the few
    nodes there are): residual parity with the oracle in both forms, and a uniform flow that
    stays exactly uniform."""
    g = W.box_grid(*shape, h=0.3)
    prm = W.box_params()
    q = W.random_state(g, seed=4, amp=0.05)
    grid = jz.Grid.from_workload(g)
    ref = O.residual(oracle_grid(g), torch.from_numpy(q), O.Consts(prm)).numpy()
    qu = W.random_state(g, seed=4, amp=0.0)
    for prec, tol in ((jz.JZ_PREC_FP64, TOL_L2), (jz.JZ_PREC_FP32FLUX, 2e-4)):
        s = jz.Solver(grid, prm, prec)
        got = s.residual(q)
        if np.abs(ref).max() == 0.0:
            assert np.abs(got).max() <= 1e-14
        else:
            e2, _ = field_errors(got, ref)
            assert e2.max() <= tol, (prec, e2)
        s.set_state(qu, 0.0)
        st = s.step(3)
        assert np.array_equal(s.get_state(), qu) and st.t > 0.0
        s.close()


def test_minimal_jet_grid(jz):
    """The smallest jet grid the ABI accepts (4 x 4 x 4): two steps against the oracle.  On this
    grid only the axis line lies inside the jet, and the axis average wipes its momentum in the
    first stage, so the momentum left is ~1e-7 of the initial scale: errors are measured
    against the initial state's scale per field (momentum: the largest component)."""
    g = W.jet_grid(4, 4, 4)
    prm = W.jet_params(seed=2)
    q = W.jet_state(g)
    scale = np.abs(q).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()
    grid = jz.Grid.from_workload(g)
    ref, t, _, _ = O.run(oracle_grid(g), torch.from_numpy(q), O.Consts(prm), 2)
    ref = ref.numpy()
    for prec, tol in ((jz.JZ_PREC_FP64, 1e-13), (jz.JZ_PREC_FP32FLUX, 1e-5)):
        s = jz.Solver(grid, prm, prec)
        s.set_state(q, 0.0)
        st = s.step(2)
        err = np.abs(s.get_state() - ref).reshape(5, -1).max(axis=1) / scale
        assert err.max() <= tol, (prec, err)
        assert abs(st.t - t.item()) <= 1e-6 * t.item()
        s.close()
