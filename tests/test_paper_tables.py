"""The workloads and the oracle against values the paper prints (fixtures in tests/golden/,
each citing its table or section): the strong-scaling meshes A-I and the jet conditions."""
import os

from paper_2003_08746_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def _round_sig(x: float, sig: int) -> float:
    return float(f"{x:.{sig - 1}e}")


def test_paper_meshes_match_the_printed_table():
    """Axial x radial counts as printed, and axial x radial x 361 azimuthal points (first and
    last superposed, so 360 unique in the solver) round to the printed totals at the printed
    number of significant digits."""
    rows = _rows("paper_meshes.txt")
    assert [r[0] for r in rows] == sorted(W.PAPER_MESHES)
    for name, ni, nj, total in rows:
        ni, nj = int(ni), int(nj)
        assert W.PAPER_MESHES[name] == (ni, nj)
        mantissa = total.split("e")[0]
        sig = len(mantissa.replace(".", "").lstrip("0"))
        assert _round_sig(ni * nj * 361, sig) == float(total), (name, ni * nj * 361, total)


def test_jet_setup_matches_the_printed_conditions():
    """Jet Mach number, Reynolds number and domain size as printed, and the oracle's entrance
    condition in the supersonic core imposes the printed pressure and temperature ratios
    (p_j / p_inf = PR, T_j / T_inf = TR) and a velocity profile whose plateau is the printed
    Mach number."""
    import numpy as np
    import torch

    from oracle import jz_oracle as O

    v = {k: float(x) for k, x in _rows("paper_jet_setup.txt")}
    prm = W.jet_params()
    assert prm.jet_mach == v["jet_mach"] and prm.Re == v["reynolds"]
    g = W.jet_grid(12, 64, 8)
    x = g.xyz[0]
    r = np.sqrt(g.xyz[1] ** 2 + g.xyz[2] ** 2)
    assert x.min() == 0.0 and x.max() == v["domain_length"]
    assert np.isclose(r.max(), v["domain_height"], rtol=0, atol=1e-12)
    c = O.Consts(prm)
    c.amp.zero_()                                  # unforced entrance
    grid = O.Grid(g.ni, g.nj, g.nk, g.xyz, g.topology, g.period)
    one = np.ones((g.nk, g.nj, g.ni))
    p_inf = 1.0 / prm.gamma
    q = torch.from_numpy(W.conserved(one, 0.1 * one, 0 * one, 0 * one, p_inf * one))
    out = O.inflow_bc(grid, q, c, 0.0)[:, :, 1:, 0].numpy()     # entrance nodes off the axis
    core = r[:, 1:, 0] < 0.25                       # deep inside the jet: the tanh profile is flat
    assert core.sum() >= 2 * g.nk
    rho = out[0][core]
    u = out[1][core] / rho
    p = (prm.gamma - 1.0) * (out[4][core] - 0.5 * rho * u * u)
    T = prm.gamma * p / rho                         # T_inf = 1 with p_inf = 1/gamma, rho_inf = 1
    assert np.allclose(p / p_inf, v["pressure_ratio"], rtol=1e-12)
    assert np.allclose(T, v["temperature_ratio"], rtol=1e-12)
    # the entrance profile is the tanh shear layer whose plateau is the jet Mach number
    shape = 0.5 * (1.0 + np.tanh((0.5 - r[:, 1:, 0][core]) / (2.0 * prm.theta_mom)))
    assert np.allclose(u / np.sqrt(T) / shape, v["jet_mach"], rtol=1e-13)


def test_physical_constants_match_the_printed_values():
    """Pr, Pr_sgs and the Sutherland constant as printed, in the parameters and in the oracle's
    derived constants (S1 over the reference temperature)."""
    from oracle import jz_oracle as O

    v = {k: float(x) for k, x in _rows("paper_constants.txt")}
    for prm in (W.box_params(), W.jet_params()):
        assert prm.Pr == v["prandtl"] and prm.Pr_sgs == v["prandtl_sgs"] and prm.S1_K == v["sutherland_S1_K"]
        c = O.Consts(prm)
        assert c.Pr == v["prandtl"] and c.Pr_sgs == v["prandtl_sgs"]
        assert c.S_hat == v["sutherland_S1_K"] / prm.T_ref_K
