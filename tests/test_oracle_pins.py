"""Pins of the CPU oracle against what the mathematics and the paper fix.

Each test checks the oracle against a value that does not come from the
oracle itself: a closed form, an exact invariant, a textbook formula or the
linear theory of the discretisation.  The tests are chosen so that a plausible
slip (a dropped term, a wrong sign or index, a transposed operand) fails one
of them.
"""
import math

import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W

GAMMA = 1.4


def _grid(g):
    return O.Grid(g.ni, g.nj, g.nk, g.xyz, g.topology, g.period)


# ---------------------------------------------------------------------------
# c-P1  RK amplification polynomial (5-stage scheme, "2nd order")
# ---------------------------------------------------------------------------
def test_rk_amplification_polynomial():
    """q' = z q: one step must give 1 + z + z^2/2 + 3 z^3/16 + z^4/32 + z^5/128.

    The z and z^2 coefficients are those of exp(z) (second order, as the paper
    states for its 5-stage scheme); the rest is the product of the stage
    coefficients alpha = (1/4, 1/6, 3/8, 1/2, 1).
    """
    zs = torch.tensor([-0.3, -1.0, -2.5, 0.7, complex(-0.2, 1.1), complex(-1.5, -2.0)],
                      dtype=torch.complex128)
    Qn = torch.ones_like(zs)
    out, _ = O.rk_stages(Qn, lambda q: -zs * q, torch.tensor(True), 1.0, lambda q, a: q)
    expect = 1 + zs + zs ** 2 / 2 + 3 * zs ** 3 / 16 + zs ** 4 / 32 + zs ** 5 / 128
    assert torch.allclose(out, expect, rtol=0, atol=1e-15)
    # second order: local error against exp(z) scales like z^3 for small z
    z = torch.tensor([1e-2, 2e-2], dtype=torch.complex128) * complex(-1, 0.5)
    q1, _ = O.rk_stages(torch.ones_like(z), lambda q: -z * q, torch.tensor(True), 1.0, lambda q, a: q)
    err = (q1 - torch.exp(z)).abs()
    assert 6.0 < (err[1] / err[0]).item() < 10.0


# ---------------------------------------------------------------------------
# c-P2  metrics: closed forms on a uniform cylinder; free-stream preservation
# ---------------------------------------------------------------------------
def _uniform_cylinder(ni=6, nj=7, nk=8, dx=0.3, dr=0.2):
    th = 2 * math.pi * np.arange(nk) / nk
    x = dx * np.arange(ni)
    r = dr * np.arange(nj)
    xyz = np.empty((3, nk, nj, ni))
    xyz[0] = x[None, None, :]
    xyz[1] = (np.cos(th)[:, None] * r[None, :])[:, :, None]
    xyz[2] = (np.sin(th)[:, None] * r[None, :])[:, :, None]
    return O.Grid(ni, nj, nk, xyz, O.TOPO_JET), th, r, dx, dr


def test_metrics_uniform_cylinder_closed_form():
    """Discrete Thomas-Lombard metrics of x = i dx, (y, z) = j dr (cos, sin)(2 pi k/nk).

    S^xi  = (r dr s, 0, 0),   s = sin(dth)
    S^eta = dx r s (0, cos th, sin th)
    S^zeta = dx dr (0, -sin th, cos th)
    V     = dx dr r s
    (derived by hand from the centred differences; exact on every real node,
    the axis and the far-field/inflow/outflow planes included).
    """
    grid, th, r, dx, dr = _uniform_cylinder()
    nk, nj, ni = grid.nk, grid.nj, grid.ni
    dth = 2 * math.pi / nk
    s = math.sin(dth)
    TH = torch.as_tensor(th)[:, None, None].expand(nk, nj, ni)
    R = torch.as_tensor(r)[None, :, None].expand(nk, nj, ni)
    M = grid.metrics_real
    expect = torch.stack([
        R * dr * s, torch.zeros_like(R), torch.zeros_like(R),
        torch.zeros_like(R), dx * R * s * torch.cos(TH), dx * R * s * torch.sin(TH),
        torch.zeros_like(R), -dx * dr * torch.sin(TH), dx * dr * torch.cos(TH),
        dx * dr * R * s])
    assert torch.allclose(M, expect, rtol=0, atol=1e-14)
    # the axis is the singular line: zero volume and zero eta-face area there
    assert torch.all(M[9][:, 0, :] == 0)


def _uniform_state(shape, u=(0.3, 0.2, -0.1), rho=1.1, p=0.9 / GAMMA):
    one = np.ones(shape)
    return torch.from_numpy(W.conserved(rho * one, u[0] * one, u[1] * one, u[2] * one, p * one))


@pytest.mark.parametrize("kind", ["wavy", "jet"])
def test_freestream_preservation(kind):
    """A uniform flow has zero residual on a curvilinear grid (discrete metric identities)."""
    if kind == "wavy":
        g = W.wavy_periodic_grid(20, 18, 12, amp=0.1)
        prm = W.box_params()
    else:
        g = W.jet_grid(24, 20, 16)
        prm = W.jet_params()
    grid, c = _grid(g), O.Consts(prm)
    R = O.residual(grid, _uniform_state((g.nk, g.nj, g.ni)), c)
    # flux scale ~ rho u^2 + p ~ 1; a sign or index slip in any metric gives O(1e-2..1)
    assert R.abs().max().item() < 1e-12


def test_metric_identity_on_jet_grid():
    """sum_dir delta_dir(S^dir) = 0 at every updated node of a stretched jet grid."""
    g = W.jet_grid(16, 14, 12)
    grid = _grid(g)
    tot = sum(O.delta(grid.S[d], ax) for d, ax in enumerate((O.AX_I, O.AX_J, O.AX_K)))
    tot = O.real(tot)[:, grid.updated]
    assert tot.abs().max().item() < 1e-13


# ---------------------------------------------------------------------------
# c-P3  discrete conservation on the periodic box
# ---------------------------------------------------------------------------
def test_conservation_periodic_box():
    """sum Q_m V is constant over 10 steps of the box run (telescoping flux differences)."""
    g, q, prm = W.make_workload("box32x24x16")
    grid, c = _grid(g), O.Consts(prm)
    Q = torch.from_numpy(q)
    T0 = O.totals(grid, Q)
    scale = (Q.abs() * grid.metrics_real[9]).reshape(5, -1).sum(1)
    Q2, _, _, _ = O.run(grid, Q, c, 10)
    drift = ((O.totals(grid, Q2) - T0).abs() / scale)
    assert drift.max().item() < 1e-13
    assert (Q2 - Q).abs().max().item() > 1e-6       # the state did change


# ---------------------------------------------------------------------------
# c-P4 / c-P5  linear modes: entropy wave, shear wave, heat conduction
# ---------------------------------------------------------------------------
def _line_grid(n=32):
    g = W.box_grid(n, 1, 1)
    return g, _grid(g), 2 * math.pi / n


def _lam_xi(grid_h, u, a=1.0, sigma=2.0 / 3.0):
    lx = (abs(u) + a) * grid_h ** 2
    le = a * grid_h ** 2
    return lx + lx ** (1 - sigma) * 2 * le ** sigma


def _entropy_wave_prediction(n, h, u, dt, c, sigma, eps):
    th = 2 * math.pi / n
    Lam = _lam_xi(h, u, sigma=sigma)
    z = dt * complex(-Lam * c.kappa4 * 16 * math.sin(th / 2) ** 4 / h ** 3, -u / h * math.sin(th))
    P = 1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128
    return eps * (P * np.exp(1j * th * np.arange(n))).imag


@pytest.mark.parametrize("sigma,n", [(2.0 / 3.0, 32), (0.5, 8)])
def test_entropy_wave_amplification(sigma, n):
    """rho = 1 + eps sin(x), uniform u and p, inviscid: one step multiplies the mode by P(z).

    z = dt [-i (u/h) sin(th) - Lambda kappa4 16 sin^4(th/2) / h^3], th = 2 pi/n,
    Lambda the anisotropic spectral radius of the base flow (nu = 0 since p is uniform),
    for the paper-default exponent sigma = 2/3 (cube-root branch) and, on a coarse line where
    the dissipation is strong enough to tell them apart, a general exponent.
    """
    g, grid, h = _line_grid(n)
    eps, u, dt = 1e-6, 0.5, 0.05
    x = h * np.arange(n)
    one = np.ones((1, 1, n))
    q = W.conserved(1 + eps * np.sin(x)[None, None, :], u * one, 0 * one, 0 * one, one / GAMMA)
    prm = W.box_params(Re=math.inf, C_s=0.0, dt_fixed=dt, sigma=sigma)
    c = O.Consts(prm)
    Q2, _, _ = O.rk_step(grid, torch.from_numpy(q), c, 0.0)
    got = (Q2[0, 0, 0] - 1).numpy()
    pred = _entropy_wave_prediction(n, h, u, dt, c, sigma, eps)
    assert np.abs(got - pred).max() < 1e-5 * eps
    if sigma != 2.0 / 3.0:   # the coarse case distinguishes the exponent
        other = _entropy_wave_prediction(n, h, u, dt, c, 2.0 / 3.0, eps)
        assert np.abs(got - other).max() > 2e-5 * eps


def test_shear_wave_decay():
    """v = eps sin(x): advection, 4th-difference damping and viscous decay mu sin^2(th)/h^2."""
    g, grid, h = _line_grid()
    n, eps, u, dt = g.ni, 1e-6, 0.3, 0.05
    x = h * np.arange(n)
    one = np.ones((1, 1, n))
    q = W.conserved(one, u * one, eps * np.sin(x)[None, None, :], 0 * one, one / GAMMA)
    prm = W.box_params(Re=10.0, mach_ref=1.0, C_s=0.0, dt_fixed=dt)
    c = O.Consts(prm)
    mu = 0.1
    Q2, _, _ = O.rk_step(grid, torch.from_numpy(q), c, 0.0)
    th = 2 * math.pi / n
    Lam = _lam_xi(h, u)
    z = dt * complex(-Lam * c.kappa4 * 16 * math.sin(th / 2) ** 4 / h ** 3 - mu * math.sin(th) ** 2 / h ** 2,
                     -u / h * math.sin(th))
    P = 1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128
    pred = eps * (P * np.exp(1j * th * np.arange(n))).imag
    got = Q2[2, 0, 0].numpy()
    assert np.abs(got - pred).max() < 1e-5 * eps


@pytest.mark.parametrize("a", [0.1, 0.02])
def test_pressure_sensor_and_second_difference_dissipation(a):
    """Odd-even pressure p_i = p0 (1 + a (-1)^i) at rest, uniform rho, inviscid.

    The sensor |p+ - 2p + p-| / (p+ + 2p + p-) equals a at every node, so
    eps2 = kappa2 a and eps4 = max(0, kappa4 - kappa2 a) (a = 0.1: the second-difference
    branch alone; a = 0.02: both).  The centred pressure difference vanishes (p_{i+1} =
    p_{i-1}), and only the energy mode e' (-1)^i, e' = p0 a / (gamma - 1), is dissipated:
    Delta1 e = -2 e' (-1)^i, Delta3 e = 8 e' (-1)^i at every face, so
    V RHS_e = 2 L (2 eps2 + 8 eps4) e' (-1)^i with L the face spectral radius; with u = 0 the
    three radii of a node are equal (lambda = c h^2), the anisotropic scaling gives 3 lambda
    for any sigma, and L = (3 h^2 / 2)(c_even + c_odd), c = sqrt(gamma p / rho).
    """
    g, grid, h = _line_grid()
    n = g.ni
    sgn = (-1.0) ** np.arange(n)
    p0 = 1.0 / GAMMA
    one = np.ones((1, 1, n))
    q = W.conserved(one, 0 * one, 0 * one, 0 * one, (p0 * (1 + a * sgn))[None, None, :])
    c = O.Consts(W.box_params(Re=math.inf, C_s=0.0))
    R = O.residual(grid, torch.from_numpy(q), c).numpy()
    eps2 = c.kappa2 * a
    eps4 = max(0.0, c.kappa4 - eps2)
    assert (eps4 == 0.0) == (a == 0.1)
    L = 1.5 * h ** 2 * (math.sqrt(GAMMA * p0 * (1 + a)) + math.sqrt(GAMMA * p0 * (1 - a)))
    e1 = p0 * a / (GAMMA - 1.0)
    expect_e = 2.0 * L * (2.0 * eps2 + 8.0 * eps4) * e1 * sgn / h ** 3
    assert np.abs(R[:4]).max() < 1e-13
    assert np.allclose(R[4, 0, 0], expect_e, rtol=1e-12, atol=0.0)
    # the sign damps the mode: Q - dt RHS shrinks e'
    assert np.all(R[4, 0, 0] * sgn > 0)


def test_heat_flux_diffuses():
    """T = 1 + eps sin(x) at uniform p and rest: de/dt = -kappa sin^2(th)/h^2 T' (heat flows down the gradient).

    This fixes the sign of the heat flux in the energy equation (the printed
    eq. q_mod with RHS = dE/dx - dF/dx would make it anti-diffusive).
    """
    g, grid, h = _line_grid()
    n, eps = g.ni, 1e-7
    x = h * np.arange(n)
    one = np.ones((1, 1, n))
    T = 1 + eps * np.sin(x)[None, None, :]
    q = W.conserved(1.0 / T, 0 * one, 0 * one, 0 * one, one / GAMMA)
    prm = W.box_params(Re=10.0, mach_ref=1.0, C_s=0.0)
    c = O.Consts(prm)
    R = O.residual(grid, torch.from_numpy(q), c)
    kappa = 0.1 * c.Cp / c.Pr
    th = 2 * math.pi / n
    pred = -kappa * math.sin(th) ** 2 / h ** 2 * eps * np.sin(x)
    got = -R[4, 0, 0].numpy()
    assert np.abs(got - pred).max() < 1e-4 * np.abs(pred).max()


# ---------------------------------------------------------------------------
# c-P6  Sutherland and Smagorinsky, pointwise
# ---------------------------------------------------------------------------
def test_sutherland_matches_textbook_form():
    """Sutherland's law in its classical form mu0 (T/T0)^1.5 (T0 + S)/(T + S), mu0 = 1.716e-5 Pa s,
    T0 = 273.15 K, S = 110.4 K, normalised at T_ref = 288.15 K, equals mu/mu_ref of the
    non-dimensional reading (T_inf = T_ref, S1 = 110.4 K)."""
    c = O.Consts(W.box_params())
    TK = torch.tensor([200.0, 288.15, 350.0, 576.3, 1000.0], dtype=torch.float64)

    def classic(T):
        return 1.716e-5 * (T / 273.15) ** 1.5 * (273.15 + 110.4) / (T + 110.4)

    ratio = classic(TK) / classic(torch.tensor(288.15, dtype=torch.float64))
    got = O.sutherland(TK / 288.15, c) / c.mu_ref
    assert torch.allclose(got, ratio, rtol=1e-13, atol=0)
    # textbook value: mu(576.3 K)/mu(288.15 K) = 1.6416 for air
    assert abs(got[3].item() - 1.6416) < 1e-4


def test_smagorinsky_on_linear_field():
    """u_i = A_ij x_j on a uniform grid: centred gradients are exact, so
    tau = 2 (mu + rho (C_s h)^2 |S|)(S - tr(S)/3 I), |S| = sqrt(2 S:S), S = (A + A^T)/2,
    and the xi viscous flux is h^2 [tau_1x, tau_2x, tau_3x, u_i tau_ix] (uniform T)."""
    n, h = 10, 0.1
    g = W.box_grid(n, n, n, h=h)
    grid = _grid(g)
    A = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [0.2, 0.6, -0.1]])
    xyz = g.xyz
    vel = np.einsum("ij,jkmn->ikmn", A, xyz) + np.array([0.2, 0.1, 0.0])[:, None, None, None]
    one = np.ones((n, n, n))
    q = W.conserved(1.3 * one, vel[0], vel[1], vel[2], 1.3 * one / GAMMA)   # T = gamma p / rho = 1
    c = O.Consts(W.box_params(C_s=0.18))
    Qp = grid.pad(torch.from_numpy(q))
    rho, u, v, w, p, T = O.primitives(Qp, c)
    F = O.viscous_fluxes(grid, rho, u, v, w, T, c)
    S = 0.5 * (A + A.T)
    Smod = math.sqrt(2 * (S * S).sum())
    mu_eff = c.mu_ref * 1.0 + 1.3 * (0.18 * h) ** 2 * Smod     # T = 1 -> mu = mu_ref
    tau = 2 * mu_eff * (S - np.trace(S) / 3 * np.eye(3))
    sl = (slice(G2 := O.G + 3, -G2),) * 3           # nodes well away from the periodic seam
    vel_t = torch.from_numpy(vel)
    for m in range(3):
        assert torch.allclose(F[0][m][sl], torch.full_like(F[0][m][sl], h * h * tau[m, 0]), rtol=1e-11, atol=1e-16)
    energy = h * h * sum(O.real(grid.pad(vel_t[i]))[tuple(slice(3, -3) for _ in range(3))] * tau[i, 0] for i in range(3))
    assert torch.allclose(F[0][3][sl], energy, rtol=1e-11, atol=1e-16)


# ---------------------------------------------------------------------------
# c-P7  design order of accuracy (self-convergence of the residual)
# ---------------------------------------------------------------------------
def test_order_of_accuracy_curvilinear():
    """Residual of a smooth periodic state on a smooth curvilinear grid converges at order 2."""
    res = {}
    for n in (12, 24, 48):
        g = W.wavy_periodic_grid(n, n, n, amp=0.05)
        q = W.smooth_state(g, seed=3)
        grid, c = _grid(g), O.Consts(W.box_params(Re=100.0))
        R = O.residual(grid, torch.from_numpy(q), c)
        step = n // 12
        res[n] = R[:, ::step, ::step, ::step]
    e1 = (res[12] - res[24]).reshape(5, -1).norm(dim=1)
    e2 = (res[24] - res[48]).reshape(5, -1).norm(dim=1)
    order = torch.log2(e1 / e2)
    assert torch.all(order > 1.8), order
    assert torch.all(order < 2.6), order


# ---------------------------------------------------------------------------
# c-P8  acoustic pulse against the linear spherical closed form
# ---------------------------------------------------------------------------
def _pulse_error(n, L=3.0, A=1e-4, width=0.9, t_end=0.8):
    h = 2 * L / n
    g = W.box_grid(n, n, n, h=h)
    xyz = g.xyz - (L - 0.0)          # centre the box on the origin (node at 0)
    r = np.sqrt((xyz ** 2).sum(0))
    alpha = 1.0 / width ** 2
    pp = A * np.exp(-alpha * r * r)
    one = np.ones_like(r)
    p = one / GAMMA + pp
    rho = one + pp                   # isentropic: rho' = p'/a^2, a = 1
    q = W.conserved(rho, 0 * one, 0 * one, 0 * one, p)
    grid = _grid(g)
    c = O.Consts(W.box_params(Re=math.inf, C_s=0.0))
    Q = torch.from_numpy(q)
    t = 0.0
    while t < t_end - 1e-12:
        dt = min(O.cfl_dt(grid, Q, c).item(), t_end - t)
        Q, _, _ = O.rk_step(grid, Q, c, t, dt=torch.tensor(dt, dtype=torch.float64))
        t += dt
    _, _, _, _, pnum, _ = O.primitives(grid.pad(Q), c)
    pnum = O.real(pnum) - 1 / GAMMA

    def f(s):
        return A * np.exp(-alpha * s * s)
    rs = np.where(r > 1e-12, r, 1.0)
    exact = np.where(r > 1e-12, 0.5 * ((rs - t) * f(rs - t) + (rs + t) * f(rs + t)) / rs,
                     A * (1 - 2 * alpha * t * t) * np.exp(-alpha * t * t))
    inner = r < L - 0.6 - t          # before periodic images arrive
    return np.abs(pnum.numpy()[inner] - exact[inner]).max() / A


def test_acoustic_pulse_linear_closed_form():
    """Quiescent box, inviscid, Gaussian pressure pulse: r p' = [(r-t) f(r-t) + (r+t) f(r+t)]/2."""
    e_c = _pulse_error(24)
    e_f = _pulse_error(48)
    assert e_f < 0.02
    assert e_c / e_f > 4.0          # at least second-order convergence of the error


# ---------------------------------------------------------------------------
# c-P9  boundary conditions, pointwise
# ---------------------------------------------------------------------------
def _jet(ni=10, nj=8, nk=8, **kw):
    g = W.jet_grid(ni, nj, nk)
    return g, _grid(g), O.Consts(W.jet_params(**kw))


def test_outflow_bc_formula():
    """Exit: p = p_inf; u, v, w and e_int = p/((gamma-1) rho) copied from i = ni-2, so rho_b = rho_i p_inf / p_i."""
    g, grid, c = _jet()
    shp = (g.nk, g.nj, g.ni)
    one = np.ones(shp)
    q = torch.from_numpy(W.conserved(1.2 * one, 0.8 * one, 0.1 * one, -0.05 * one, 0.9 / GAMMA * one))
    out = O.outflow_bc(grid, q, c)[:, :, 1:, -1]
    rho_b = 1.2 * (1 / GAMMA) / (0.9 / GAMMA)
    exp = W.conserved(np.array(rho_b), np.array(0.8), np.array(0.1), np.array(-0.05), np.array(1 / GAMMA))
    for m in range(5):
        assert torch.allclose(out[m], torch.full_like(out[m], float(exp[m])), rtol=1e-14, atol=0)


def test_farfield_keeps_ambient_and_uses_invariants():
    g, grid, c = _jet()
    shp = (g.nk, g.nj, g.ni)
    one = np.ones(shp)
    amb = torch.from_numpy(W.conserved(one, 0 * one, 0 * one, 0 * one, one / GAMMA))
    out = O.farfield_bc(grid, amb, c)
    assert torch.allclose(out, amb, rtol=1e-15, atol=1e-15)
    # outgoing radial flow u = 0.1 n, a_int = 1.05: R+ = 0.1 + 5.25, R- = -5 ->
    # u_n = 0.175, a = 1.035, entropy from the interior.
    y, z = g.xyz[1], g.xyz[2]
    r = np.sqrt(y * y + z * z)
    nrm = np.where(r > 0, 1 / np.where(r > 0, r, 1), 0)
    rho_i, a_i = 1.0, 1.05
    p_i = rho_i * a_i ** 2 / GAMMA
    q = torch.from_numpy(W.conserved(rho_i * one, 0 * one, 0.1 * y * nrm, 0.1 * z * nrm, p_i * one))
    out = O.farfield_bc(grid, q, c)[:, :, -1, 1:-1]
    un, ab = 0.175, 1.035
    s = p_i / rho_i ** GAMMA
    rho_b = (ab * ab / (GAMMA * s)) ** (1 / 0.4)
    assert torch.allclose(out[0], torch.full_like(out[0], rho_b), rtol=1e-12)
    yb, zb = y[:, -1, 1:-1] / r[:, -1, 1:-1], z[:, -1, 1:-1] / r[:, -1, 1:-1]
    assert np.allclose(out[2].numpy(), rho_b * un * yb, rtol=1e-12, atol=1e-15)
    assert np.allclose(out[3].numpy(), rho_b * un * zb, rtol=1e-12, atol=1e-15)


def test_inflow_supersonic_core_imposed():
    g, grid, c = _jet(nj=24, forcing_amp=None)
    c.amp.zero_()
    shp = (g.nk, g.nj, g.ni)
    one = np.ones(shp)
    q = torch.from_numpy(W.conserved(one, 0.2 * one, 0 * one, 0 * one, one / GAMMA))
    out = O.inflow_bc(grid, q, c, 0.0)[:, :, 1:, 0]
    r = np.sqrt(g.xyz[1] ** 2 + g.xyz[2] ** 2)[:, 1:, 0]
    ut = 0.7 * (1 + np.tanh((0.5 - r) / 0.1))
    sup = ut >= 1
    assert sup.any() and (~sup).any()
    assert np.allclose(out[1].numpy()[sup], ut[sup], rtol=1e-14)
    assert np.allclose(out[0].numpy()[sup], 1.0, rtol=1e-15)
    # subsonic: R- from the interior (u = 0.2, a = 1), R+ from the target (a = 1)
    Rm = 0.2 - 2 / 0.4
    Rp = ut[~sup] + 2 / 0.4
    ub, ab = 0.5 * (Rp + Rm), 0.1 * (Rp - Rm)
    rho_b = ab ** 5          # (a^2/(gamma s))^(1/(gamma-1)), s = 1/gamma
    assert np.allclose(out[0].numpy()[~sup], rho_b, rtol=1e-13)
    assert np.allclose(out[1].numpy()[~sup], rho_b * ub, rtol=1e-13)


def _forcing_only(grid, c, t, m, f, A=0.01):
    """Entrance target minus the unforced profile with one nonzero amplitude A_mf: [nk][nj-1]."""
    c.amp.zero_()
    base = O.inflow_target(grid, c, t)
    c.amp[m, f] = A
    out = O.inflow_target(grid, c, t) - base
    c.amp.zero_()
    return out.numpy()


@pytest.mark.parametrize("m,f", [(3, 2), (0, 1), (7, 3)])
def test_inflow_forcing_azimuthal_mode(m, f):
    """Reading c14, azimuthal structure of the entrance forcing, pinned by a discrete Fourier
    transform over the nk unique azimuthal points (theta_k = 2 pi k / nk) of every radial line:
    a single amplitude A_mf puts all of the forcing's energy in azimuthal bins m and nk - m
    (any other mode number, or a temporal factor that depends on theta, leaks into other
    bins), and bin m carries the phase phi_mf (a sign slip in m theta conjugates it, and a
    swap with psi_mf, drawn independently, changes it)."""
    g, grid, c = _jet(ni=6, nj=40, nk=32)
    t = 0.37
    fr = _forcing_only(grid, c, t, m, f)                       # [nk][nj-1]
    X = np.fft.fft(fr, axis=0) / g.nk                          # per radial line
    line = np.abs(fr).max(axis=0) > 1e-8                       # lines where g(r) is not negligible
    assert line.sum() >= 6
    others = np.ones(g.nk, dtype=bool)
    others[m] = others[(g.nk - m) % g.nk] = False
    assert np.abs(X[others][:, line]).max() <= 1e-12 * np.abs(fr).max()
    # complex bin m = (B/2) e^{i phi} with B real (m > 0); bin 0 = B cos(phi), real
    B = (2.0 if m > 0 else 1.0) * X[m, line]
    phi = float(c.phi[m, f]) if m > 0 else 0.0
    rot = B * np.exp(-1j * phi)
    assert np.abs(rot.imag).max() <= 1e-12 * np.abs(rot).max()


@pytest.mark.parametrize("m,f", [(3, 2), (5, 0)])
def test_inflow_forcing_frequency_and_temporal_phase(m, f):
    """Reading c14, time dependence of the entrance forcing: sampled at N = 16 equal steps
    over T = 1 / (St_f U_j) at one entrance node, the forcing is a pure first harmonic of
    that period (St not multiplied by U_j, or the wrong St_f, spreads energy into other
    bins), and the phase of the first harmonic is omega t0 + psi_mf - pi/2, i.e. the
    temporal phase is psi_mf (a swap with phi_mf fails)."""
    _, grid, c = _jet(ni=6, nj=40, nk=16)
    Uj, St = c.jet_mach, c.strouhal[f]
    T = 1.0 / (St * Uj)
    N, t0 = 16, 0.123
    # the entrance node with the largest forcing over the period
    samples = np.array([_forcing_only(grid, c, t0 + n * T / N, m, f) for n in range(N)])   # [N][nk][nj-1]
    k, j = np.unravel_index(np.abs(samples).max(axis=0).argmax(), samples.shape[1:])
    x = samples[:, k, j]
    X = np.fft.fft(x) / N
    assert np.abs(X[2:N - 1]).max() <= 1e-12 * np.abs(x).max()
    assert abs(X[0]) <= 1e-12 * np.abs(x).max()
    expected = (2.0 * math.pi * St * Uj * t0 + float(c.psi[m, f]) - math.pi / 2.0)
    # the azimuthal factor cos(m theta + phi) may be negative: compare modulo pi, then its sign
    d = (np.angle(X[1]) - expected + math.pi / 2.0) % math.pi - math.pi / 2.0
    assert abs(d) <= 1e-10


def test_inflow_forcing_radial_envelope_and_amplitude():
    """Reading c14, radial envelope and scale of the forcing: on the line of largest response
    the logarithm of the forcing magnitude is a parabola in r with vertex r = 0.5, curvature
    -1/0.1^2 (a Gaussian of width 0.1 D centred on the lip), and the vertex value is
    U_j A |cos(m theta + phi) sin(omega t + psi)| (the forcing scales with U_j A)."""
    _, grid, c = _jet(ni=6, nj=60, nk=16)
    m, f, A, t = 2, 1, 0.02, 0.31
    fr = _forcing_only(grid, c, t, m, f, A=A)
    X = O.real(grid.xyz_p)[:, :, 1:, 0].numpy()               # [3][nk][nj-1] at i = 0
    r = np.sqrt(X[1] ** 2 + X[2] ** 2)
    th = np.arctan2(X[2], X[1])
    k = int(np.abs(fr).max(axis=1).argmax())
    sel = np.abs(fr[k]) > 1e-6 * np.abs(fr[k]).max()
    a2, a1, a0 = np.polyfit(r[k, sel], np.log(np.abs(fr[k, sel])), 2)
    assert abs(a2 + 100.0) <= 1e-6 * 100.0
    assert abs(-a1 / (2.0 * a2) - 0.5) <= 1e-8
    vertex = np.exp(a0 - a1 * a1 / (4.0 * a2))
    ang = abs(math.cos(m * th[k, 0] + float(c.phi[m, f])) *
              math.sin(2.0 * math.pi * c.strouhal[f] * c.jet_mach * t + float(c.psi[m, f])))
    assert abs(vertex - c.jet_mach * A * ang) <= 1e-7 * c.jet_mach * A * ang


def test_inflow_forcing_stage_times(monkeypatch):
    """Reading c14, time at which stage l imposes the entrance: t_n + alpha_l dt, with the
    low-storage coefficients alpha = (1/4, 1/6, 3/8, 1/2, 1) that the RK amplification pin
    fixes.  The boundary update of every stage is intercepted; after stage 1 the supersonic
    entrance nodes (all variables imposed) carry the target at t_n + dt/4 and not at t_n, and
    after stage 5 the target at t_n + dt."""
    g, grid, c = _jet(ni=8, nj=40, nk=16, dt_fixed=0.05)
    c.amp.zero_()
    c.amp[3, 2] = 0.05                  # strong enough to separate the stage times clearly
    q = torch.from_numpy(W.jet_state(g))
    seen = []
    orig = O.apply_bcs

    def spy(grid_, Q, c_, t):
        out = orig(grid_, Q, c_, t)
        seen.append((float(t), out.clone()))
        return out

    monkeypatch.setattr(O, "apply_bcs", spy)
    tn, dt = 0.8, 0.05
    O.rk_step(grid, q, c, tn, dt=torch.as_tensor(dt, dtype=torch.float64))
    alphas = (0.25, 1.0 / 6.0, 0.375, 0.5, 1.0)
    assert len(seen) == 5
    for (ts, _), a in zip(seen, alphas):
        assert abs(ts - (tn + a * dt)) <= 1e-15
    ut1 = O.inflow_target(grid, c, tn + 0.25 * dt).numpy()
    ut0 = O.inflow_target(grid, c, tn).numpy()
    sup = ut1 >= 1.0
    got1 = (seen[0][1][1, :, 1:, 0] / seen[0][1][0, :, 1:, 0]).numpy()
    assert np.abs(got1[sup] - ut1[sup]).max() <= 1e-14
    assert np.abs(ut1[sup] - ut0[sup]).max() >= 1e-4     # the stage time is resolved
    ut5 = O.inflow_target(grid, c, tn + dt).numpy()
    got5 = (seen[4][1][1, :, 1:, 0] / seen[4][1][0, :, 1:, 0]).numpy()
    assert np.abs(got5[sup & (ut5 >= 1.0)] - ut5[sup & (ut5 >= 1.0)]).max() <= 1e-14


def test_centerline_and_ghosts_keep_uniform_state():
    g, grid, c = _jet()
    q = _uniform_state((g.nk, g.nj, g.ni))
    assert torch.equal(O.centerline_bc(q), q)
    Qp = grid.pad(q)
    assert torch.equal(Qp, q[:, :1, :1, :1].expand_as(Qp))
    # azimuthal mode cos(theta) averages to zero on the axis
    th = torch.as_tensor(2 * math.pi * np.arange(g.nk) / g.nk)
    q2 = q.clone()
    q2[2] = torch.cos(th)[:, None, None].expand_as(q2[2])
    assert q2[2, :, 1].sum().abs() < 1e-14 and O.centerline_bc(q2)[2, :, 0].abs().max() < 1e-15


def test_ghost_map_across_axis():
    """Ghost row j = -m carries node (i, m, k + nk/2); i ghosts clamp; k wraps."""
    g, grid, c = _jet(ni=6, nj=5, nk=8)
    idx = torch.arange(g.npts, dtype=torch.float64).reshape(1, g.nk, g.nj, g.ni)
    P = grid.pad(idx)[0]
    G = O.G
    def node(i, j, k):
        return float((k * g.nj + j) * g.ni + i)
    assert P[G + 3, G - 1, G + 2] == node(2, 1, (3 + 4) % 8)
    assert P[G + 6, G - 2, G + 0] == node(0, 2, (6 + 4) % 8)
    assert P[G + 0, G + 4 + 2, G - 2] == node(0, 4, 0)
    assert P[G - 1, G + 2, G + 6] == node(5, 2, 7)


def test_cfl_dt_uniform_box():
    """dt = CFL h / (|u| + 3 a) for uniform flow along x on a cubic grid."""
    g = W.box_grid(8, 8, 8, h=0.25)
    grid = _grid(g)
    c = O.Consts(W.box_params())
    q = _uniform_state((8, 8, 8), u=(0.5, 0, 0), rho=1.0, p=1 / GAMMA)
    dt = O.cfl_dt(grid, q, c).item()
    assert abs(dt - 0.5 * 0.25 / 3.5) < 1e-15


# ---------------------------------------------------------------------------
# Symmetry pins: mirror and axis-permutation equivariance of the residual
# ---------------------------------------------------------------------------
def _random_box(n=(10, 8, 6), seed=11, h=0.3):
    g = W.box_grid(*n, h=h)
    return g, _grid(g), torch.from_numpy(W.random_state(g, seed=seed, amp=0.08))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_residual_mirror_equivariance(axis):
    """Reflect the state along one grid axis (x -> -x, flipping that velocity):
    the residual must be the reflected residual.  Any one-sided index slip in the
    dissipation faces, the sensor or the centred differences breaks this."""
    g, grid, Q = _random_box()
    c = O.Consts(W.box_params(Re=50.0))
    dim = 3 - axis                      # tensor dim of i, j, k in [5][k][j][i]
    n = Q.shape[dim]
    idx = (-torch.arange(n)) % n

    def mirror(F):
        out = F.index_select(dim, idx).clone()
        out[1 + axis] = -out[1 + axis]
        return out
    R = O.residual(grid, Q, c)
    Rm = O.residual(grid, mirror(Q), c)
    assert torch.allclose(Rm, mirror(R), rtol=0, atol=1e-13 * R.abs().max().item())


def test_residual_axis_permutation_equivariance():
    """Swap the i and j axes of a cubic periodic box together with u and v:
    the residual must swap the same way (catches transposed metric or flux components)."""
    g = W.box_grid(8, 8, 8, h=0.3)
    grid = _grid(g)
    Q = torch.from_numpy(W.random_state(g, seed=5, amp=0.08))
    c = O.Consts(W.box_params(Re=50.0))

    def swap(F):
        out = F.transpose(-1, -2).clone()
        out[[1, 2]] = out[[2, 1]]
        return out
    R = O.residual(grid, Q, c)
    Rs = O.residual(grid, swap(Q), c)
    assert torch.allclose(Rs, swap(R), rtol=0, atol=1e-13 * R.abs().max().item())


def test_jet_azimuthal_equivariance():
    """Without forcing, rotating the state by m azimuthal cells (and the Cartesian
    velocity by m dtheta) rotates the residual; this pins the across-axis ghosts."""
    g = W.jet_grid(10, 12, 8)
    grid = _grid(g)
    c = O.Consts(W.jet_params(forcing_amp=np.zeros((8, 4))))
    c.amp.zero_()
    Q = torch.from_numpy(W.random_state(g, seed=9, amp=0.05, base_u=(0.5, 0.0, 0.0)))
    m = 2
    ang = 2 * math.pi * m / g.nk
    ca, sa = math.cos(ang), math.sin(ang)

    def rot(F):
        out = torch.roll(F, shifts=m, dims=1).clone()
        y, z = out[2].clone(), out[3].clone()
        out[2] = ca * y - sa * z
        out[3] = sa * y + ca * z
        return out
    R = O.residual(grid, Q, c)
    Rr = O.residual(grid, rot(Q), c)
    assert torch.allclose(Rr, rot(R), rtol=0, atol=1e-12 * R.abs().max().item())


# ---------------------------------------------------------------------------
# c-P10  observer functional and its reverse sweep
# ---------------------------------------------------------------------------
def test_observer_weights_and_interpolation():
    """Weights sum to the lateral area 2 pi r L of the observer cylinder; a pressure field
    linear in r is interpolated exactly, so J of one state has a closed form."""
    g = W.jet_grid(20, 24, 8)
    grid = _grid(g)
    obs = O.Observer(grid, 1.3)
    L = g.xyz[0].max() - g.xyz[0].min()
    assert abs(obs.w.sum().item() * g.nk - 2 * math.pi * 1.3 * L) < 1e-10     # w_ik is the same for every k
    r = np.sqrt(g.xyz[1] ** 2 + g.xyz[2] ** 2)
    one = np.ones_like(r)
    p = 1 / GAMMA + 1e-3 * (r - 1.0)
    q = torch.from_numpy(W.conserved(one, 0 * one, 0 * one, 0 * one, p))
    c = O.Consts(W.jet_params())
    J = obs.value(q, c).item()
    expect = (1e-3 * 0.3) ** 2 * 2 * math.pi * 1.3 * L
    assert abs(J - expect) < 1e-9 * expect


def test_functional_reverse_sweep_matches_central_differences():
    """dJ/dA from the reverse sweep of the discrete forward map equals central finite
    differences (h = 1e-6) of J, component by component and along a random direction,
    within 1e-6 of the gradient's largest component."""
    g = W.jet_grid(20, 16, 8)
    prm = W.jet_params(seed=4)
    grid, c = _grid(g), O.Consts(prm)
    q = torch.from_numpy(W.jet_state(g))
    obs = O.Observer(grid, 0.75)
    dt = O.cfl_dt(grid, q, c).item()
    A = torch.as_tensor(prm.forcing_amp)
    J, gr = O.functional_gradient(grid, q, c, A, 4, dt, obs)
    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(8))
    dirs = [("comp", (0, 0)), ("comp", (2, 3)), ("dir", torch.as_tensor(rng.standard_normal((8, 4))))]
    for kind, v in dirs:
        if kind == "comp":
            d = torch.zeros_like(A)
            d[v] = 1.0
        else:
            d = v / v.norm()
        Jp = O.functional(grid, q, c, A + h * d, 4, dt, obs).item()
        Jm = O.functional(grid, q, c, A - h * d, 4, dt, obs).item()
        fd = (Jp - Jm) / (2 * h)
        ad = (gr * d).sum().item()
        assert abs(fd - ad) <= 1e-6 * gr.abs().max().item(), (kind, fd, ad)


def test_flow_statistics_closed_form():
    """u_x = a + b sin(2 pi s / S) over S samples of a full period: the time mean is a and
    the rms is |b| / sqrt(2) exactly, per node; rho varies, so u_x must be (rho u_x) / rho.
    The azimuthal average runs over k only."""
    nk, nj, ni, S = 6, 5, 7, 8
    rng = np.random.Generator(np.random.PCG64(3))
    a = torch.as_tensor(rng.uniform(0.2, 1.4, (nk, nj, ni)))
    b = torch.as_tensor(rng.uniform(-0.1, 0.1, (nk, nj, ni)))
    samples = []
    for s in range(S):
        rho = 1.0 + 0.2 * torch.as_tensor(rng.uniform(-1, 1, (nk, nj, ni)))
        u = a + b * math.sin(2 * math.pi * s / S)
        Q = torch.zeros((5, nk, nj, ni), dtype=torch.float64)
        Q[0] = rho
        Q[1] = rho * u
        Q[2] = rho * 0.3
        Q[4] = 2.0
        samples.append(Q)
    mean, rms = O.flow_statistics(samples)
    assert mean.shape == (nj, ni) and rms.shape == (nj, ni)
    assert torch.allclose(mean, a.mean(0), rtol=0, atol=1e-14)
    assert torch.allclose(rms, (b.abs() / math.sqrt(2.0)).mean(0), rtol=0, atol=1e-14)


def test_station_profile_and_potential_core():
    """Interpolation in x is exact for a field linear in x (non-uniform x, station between
    and on grid lines); the potential core ends where a piecewise-linear centreline
    profile crosses 0.95 U_j, exactly, and is None when it never does."""
    x = torch.as_tensor(np.cumsum(np.r_[0.0, np.random.Generator(np.random.PCG64(5)).uniform(0.2, 0.9, 20)]))
    nj = 4
    f = torch.stack([1.0 + (j + 1) * 0.5 * x for j in range(nj)])          # [nj][ni]
    for x0 in (float(x[3]), 0.5 * float(x[7] + x[8]), float(x[-1]), float(x[0])):
        prof = O.station_profile(f, x, x0)
        assert torch.allclose(prof, torch.tensor([1.0 + (j + 1) * 0.5 * x0 for j in range(nj)], dtype=torch.float64),
                              rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        O.station_profile(f, x, float(x[-1]) + 1.0)
    uj, xc, slope = 1.4, float(x[6]), 0.02
    axis = torch.where(x <= xc, torch.full_like(x, uj), uj * (1.0 - slope * (x - xc)))
    expect = xc + 0.05 / slope
    assert float(x[0]) < expect < float(x[-1])
    assert abs(O.potential_core_length(axis, x, uj) - expect) < 1e-12
    assert O.potential_core_length(torch.full_like(x, uj), x, uj) is None


def test_domain_of_dependence_of_one_step():
    """One RK step on an axial slab of a jet grid (its first or last planes, treated as a grid of
    its own with entrance and exit conditions at both ends) equals the step of the whole grid
    bit for bit on every node at least 10 planes from the slab's cut: the first stage changes
    the cut plane (its metrics and boundary update) and the plane next to it (ghost states
    within the stencil radius 2), and each of the four later stages carries the difference 2
    planes further, 9 planes in all.  The difference does reach 6 planes in, so the cut's
    influence is real and bounded as the stencil predicts."""
    ni, slab = 40, 24
    g = W.jet_grid(ni, 20, 8, axial_stretch=True)
    prm = W.jet_params(seed=2, dt_fixed=2e-3)
    c = O.Consts(prm)
    rng = np.random.Generator(np.random.PCG64(8))
    q = W.jet_state(g) + 2e-3 * rng.standard_normal((5, g.nk, g.nj, g.ni))
    full, _, _, _ = O.run(_grid(g), torch.from_numpy(q), c, 1, t0=0.3)
    for sl, cut in ((slice(0, slab), slab - 1), (slice(ni - slab, ni), ni - slab)):
        xyz = np.ascontiguousarray(g.xyz[..., sl])
        part, _, _, _ = O.run(O.Grid(slab, g.nj, g.nk, xyz, O.TOPO_JET), torch.from_numpy(
            np.ascontiguousarray(q[..., sl])), c, 1, t0=0.3)
        d = (part - full[..., sl]).abs().amax(dim=(0, 1, 2)).numpy()      # per plane of the slab
        dist = np.abs(np.arange(sl.start, sl.stop) - cut)
        assert d[dist >= 10].max() == 0.0
        assert d[dist == 6].max() > 1e-15
