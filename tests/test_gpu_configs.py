"""Parity with the CPU oracle at the sizes and step counts of the named jet workloads.

* jet 256 x 128 x 64 (2.1M points), all 100 RK steps of the FP64 form, element by element;
* jet 1000 x 400 x 500 (2.0e8 points, the benchmark workload in its launch configuration):
  the GPU steps the whole grid; the oracle steps an axial slab of it (the first or the last
  40 i-planes: entrance, axis, across-axis ghosts, far field, exit), and every node farther
  from the slab's cut than the cut can reach in one step is compared;
* jet 128 x 96 x 64: the observer functional and its gradient with respect to the 32 forcing
  amplitudes against the oracle's reverse sweep (reverse-mode differentiation of its own
  forward map) over 10 steps with checkpoints every 5.

Bars as in the other parity tests: FP64 form <= 1e-12 relative L2 per field, <= 1e-11 relative
max; FP32-flux form <= 1e-5.
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


@pytest.fixture(scope="module")
def jz():
    from paper_2003_08746_gb300 import build, jz as J
    build.build()
    J.load()
    assert torch.cuda.is_available()
    return J


@pytest.fixture(scope="module")
def jet256_ref():
    """The oracle's 100 steps of the 256 x 128 x 64 jet (shared by the FP64 and pair forms)."""
    g, q, prm = W.make_workload("jet256x128x64")
    og, oc = oracle_grid(g), O.Consts(prm)
    ref, t, dts, R1 = O.run(og, torch.from_numpy(q), oc, 100)
    return g, q, prm, og, ref, t, dts, R1


@pytest.mark.parametrize("precision", ["fp64", "pair"])
def test_jet256x128x64_100_steps_fp64(jz, jet256_ref, precision):
    """The 256 x 128 x 64 jet over its 100 RK steps (CFL time step, seeded entrance forcing):
    state, time, last time step, last residual norm and totals against the oracle, for the FP64
    form and for its pair form (double-float stage arithmetic)."""
    g, q, prm, og, ref, t, dts, R1 = jet256_ref
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64 if precision == "fp64" else jz.JZ_PREC_FP64PAIR)
    s.set_state(q, 0.0)
    st = s.step(100)
    got = s.get_state()
    s.close()
    grid.close()
    e2, em = field_errors(got, ref.numpy())
    print(f"jet256x128x64 {precision} 100 steps vs oracle: rel L2 {e2}, rel max {em}")
    assert e2.max() <= TOL_L2, e2
    assert em.max() <= TOL_MAX, em
    assert abs(st.t - t.item()) <= 1e-13 * t.item()
    assert abs(st.dt - dts[-1].item()) <= 1e-13 * dts[-1].item()
    assert abs(st.res_l2 - O.residual_l2(og, R1).item()) <= 1e-11 * O.residual_l2(og, R1).item()
    tot = O.totals(og, ref).numpy()
    scale = np.abs(ref.numpy() * og.metrics_real[9].numpy()).reshape(5, -1).sum(1)
    scale[1:4] = scale[1:4].max()      # transverse momentum totals nearly cancel: momentum scale
    assert np.all(np.abs(np.array(st.totals) - tot) <= 1e-13 * scale)


# --- the 1000 x 400 x 500 jet against axial slabs of it --------------------------------------
SLAB = 40            # i-planes the oracle steps
# Nodes of the slab that the cut cannot reach in one step: the ghost coordinates and ghost
# states beyond the cut differ from the full grid's nodes, so the metrics of the plane at the
# cut and the residuals within 2 planes of it differ; every later stage carries the difference
# 2 planes further (the boundary update at the cut copies its neighbour), 9 planes in all.
# 14 keeps a margin (the CPU test of the oracle's domain of dependence checks the reach).
REACH = 14
NOISE = 2e-3


@pytest.fixture(scope="module")
def full_jet():
    """The 1000 x 400 x 500 workload with seeded Gaussian noise (standard deviation 2e-3 times
    the field's largest magnitude, at least 2e-3) on every conserved variable of the first and
    last SLAB i-planes, where the slabs are compared."""
    g, q, prm = W.make_workload("jet1000x400x500")
    rng = np.random.Generator(np.random.PCG64(31))
    for sl in (slice(0, SLAB), slice(g.ni - SLAB, g.ni)):
        q[:, :, :, sl] += NOISE * rng.standard_normal((5, g.nk, g.nj, SLAB)) * np.abs(q[:, :, :, sl]).max(
            axis=(1, 2, 3), keepdims=True).clip(min=1.0)
    return g, q, prm


def _slab(g, q, side):
    sl = slice(0, SLAB) if side == "entrance" else slice(g.ni - SLAB, g.ni)
    xyz = np.ascontiguousarray(g.xyz[:, :, :, sl])
    qs = np.ascontiguousarray(q[:, :, :, sl])
    keep = slice(0, SLAB - REACH) if side == "entrance" else slice(REACH, SLAB)
    return O.Grid(SLAB, g.nj, g.nk, xyz, O.TOPO_JET), qs, sl, keep


@pytest.fixture(scope="module")
def slab_dt(full_jet):
    """A fixed time step for the slab comparison: 0.9 x the oracle's CFL step on the entrance
    slab (the finest axial spacing of the stretched grid is at the entrance)."""
    g, q, prm = full_jet
    og, qs, _, _ = _slab(g, q, "entrance")
    return 0.9 * O.cfl_dt(og, torch.from_numpy(qs), O.Consts(prm)).item()


@pytest.fixture(scope="module")
def slab_refs(full_jet, slab_dt):
    """Oracle residual and one step (t = 0.3, fixed time step) of the entrance and exit slabs."""
    g, q, _ = full_jet
    oc = O.Consts(W.jet_params(seed=2, dt_fixed=slab_dt))
    refs = {}
    for side in ("entrance", "exit"):
        og, qs, sl, keep = _slab(g, q, side)
        Qs = torch.from_numpy(qs)
        R = O.residual(og, Qs, oc).numpy()
        Q1, t, _, _ = O.run(og, Qs, oc, 1, t0=0.3)
        refs[side] = (R, Q1.numpy(), t.item(), sl, keep)
    return refs


@pytest.mark.parametrize("precision", ["fp64", "pair", "fp32flux"])
def test_jet1000x400x500_slabs_one_step(jz, full_jet, slab_dt, slab_refs, precision):
    """One RK step of the whole 1000 x 400 x 500 grid against the oracle's step of its first and
    last 40 i-planes: every node at least 14 planes from the slab's cut (the entrance, the axis,
    the across-axis ghosts, the far field and the exit included).  Also the residual of the
    launch configuration (jz_residual on the whole grid) on the nodes at least 5 planes from
    the cut (metrics within 1 node, state within 2)."""
    g, q, _ = full_jet
    prm = W.jet_params(seed=2, dt_fixed=slab_dt)
    prec = {"fp64": jz.JZ_PREC_FP64, "pair": jz.JZ_PREC_FP64PAIR, "fp32flux": jz.JZ_PREC_FP32FLUX}[precision]
    tol2, tolm, rtol = (TOL_L2, TOL_MAX, 1e-11) if precision != "fp32flux" else (1e-5, 1e-5, 2e-4)
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, prec)
    qd = torch.from_numpy(q).cuda()
    rd = torch.empty_like(qd)
    s.residual(qd, rd)
    s.set_state(qd, 0.3)
    st = s.step(1)
    s.get_state(qd)
    s.close()
    grid.close()
    for side in ("entrance", "exit"):
        Rref, Qref, t, sl, keep = slab_refs[side]
        rk = slice(0, SLAB - 5) if side == "entrance" else slice(5, SLAB)
        r2, _ = field_errors(rd[..., sl].cpu().numpy()[..., rk], Rref[..., rk])
        e2, em = field_errors(qd[..., sl].cpu().numpy()[..., keep], Qref[..., keep])
        print(f"jet1000x400x500 {precision} {side} slab: residual rel L2 {r2.max():.2e}, "
              f"state rel L2 {e2}, rel max {em}")
        assert r2.max() <= rtol, (side, r2)
        assert e2.max() <= tol2, (side, e2)
        assert em.max() <= tolm, (side, em)
        assert abs(st.t - t) <= 1e-15 and st.dt == slab_dt
    del qd, rd
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def adj_ref():
    """The oracle's reverse sweep on the 128 x 96 x 64 adjoint workload (10 steps, r = 0.75)."""
    g, q, prm = W.make_workload("jet128x96x64", forcing_seed=4)
    og, oc = oracle_grid(g), O.Consts(prm)
    Q0 = torch.from_numpy(q)
    dt = O.cfl_dt(og, Q0, oc).item()
    obs = O.Observer(og, 0.75)
    Jo, go = O.functional_gradient(og, Q0, oc, torch.as_tensor(np.asarray(prm.forcing_amp)), 10, dt, obs)
    return g, q, prm, oc, dt, obs, Jo.item(), go.numpy()


@pytest.mark.parametrize("precision", ["fp64", "pair"])
def test_jet128x96x64_adjoint_vs_oracle_reverse_sweep(jz, adj_ref, precision):
    """The 128 x 96 x 64 adjoint workload (forcing seed 4): J and dJ/dA of the observer
    functional at r = 0.75 over 10 steps, checkpoints every 5, against the oracle's reverse
    sweep; J within the error that the 1e-12 state bar allows (J is quadratic in a pressure
    fluctuation of ~1e-5, so its relative error is not bounded by 1e-12), the gradient to 1e-9
    of its largest component."""
    g, q, prm, oc, dt, obs, Jo, go = adj_ref
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP64 if precision == "fp64" else jz.JZ_PREC_FP64PAIR)
    s.set_state(q, 0.0)
    J, gr = jz.jz_adjoint_step(s.h, np.asarray(prm.forcing_amp), 10, 5, 0.75)
    s.close()
    grid.close()
    # J = sum_n dt sum_ik w_ik (p~ - p_inf)^2 is quadratic in a small fluctuation, so its error
    # follows from the state bar: a pressure error delta_p changes J by at most
    # 2 delta_p sum dt w |p~ - p_inf| <= 2 delta_p sqrt(Wt J) (Cauchy-Schwarz, Wt = sum_n dt sum_ik w_ik),
    # with delta_p = 1e-12 p_inf.
    Wt = 10 * dt * g.nk * float(obs.w.sum())
    tol_J = 2.0 * TOL_L2 * oc.p_inf * np.sqrt(Wt * abs(Jo))
    print(f"jet128x96x64 {precision} adjoint 10 steps: J {J:.12e} vs {Jo:.12e} (bar {tol_J:.2e}), "
          f"grad max err {np.abs(gr - go).max():.2e} of {np.abs(go).max():.2e}")
    assert abs(J - Jo) <= tol_J
    assert np.abs(gr - go).max() <= 1e-9 * np.abs(go).max()
