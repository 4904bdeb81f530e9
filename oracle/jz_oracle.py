"""Plain FP64 CPU oracle of the JAZzY-style LES stage residual and RK update.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference that the
CUDA path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library never does,
and it shares no code with the CUDA sources.  It is written for obviousness,
not speed: whole-array PyTorch CPU float64 operations on ghost-padded arrays,
one step of the method per line, in the paper's order (Algorithm 2: inviscid
flux, artificial dissipation, viscous flux, RHS, stage update; then boundary
conditions after every stage).

Conventions (shared with the CUDA path as *readings*, never as code):
  * arrays are ``[..., nk+4, nj+4, ni+4]`` with two ghost layers per side
    (Sec. "Parallel Implementation Aspects": two-layer ghost points for the
    five-point dissipation stencil); index ``g`` of the padded axis is real
    index ``g - 2``.
  * ``shift(f, ax, s)[n] = f[n + s]``; entries whose source is outside the
    padded array are filled with ``FILL`` (NaN by default, so that any read
    outside the valid region shows up as NaN in the real region).
  * axes: i = -1, j = -2, k = -3 (i fastest).
  * non-dimensionalisation: rho_inf = a_inf = T_inf = 1, p_inf = 1/gamma,
    R = 1/gamma, Cp = 1/(gamma - 1), T = gamma p / rho, mu_ref = M_ref / Re.

Readings of the paper taken here (all listed in the design notes):
  heat flux diffuses (physical Fourier law, fixes the sign of eq. q_mod as
  printed); Sutherland with T_inf = 1 and S1/T_ref; Smagorinsky eddy
  viscosity with Delta = V^(1/3), sigma_kk = 0; second-order centred nodal
  differences of the transformed fluxes; Thomas-Lombard conservative metrics
  built from the same centred difference; Turkel-Vatsa scalar dissipation
  with kappa2, kappa4, sigma; low-storage 5-stage RK with
  alpha = (1/4, 1/6, 3/8, 1/2, 1); CFL time step; jet boundary conditions
  (inflow characteristic tanh profile with forcing, Riemann far field,
  pressure outflow, azimuthal average on the axis, periodic azimuth).
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64
G = 2                      # ghost layers per side
AX_I, AX_J, AX_K = -1, -2, -3
FILL = float("nan")        # value of entries shifted in from outside the array
RK_ALPHA = (0.25, 1.0 / 6.0, 0.375, 0.5, 1.0)
TOPO_PERIODIC, TOPO_JET = 1, 2


def set_fill(value: float) -> None:
    """NaN (default) flags reads outside the valid region; 0 keeps autograd finite."""
    global FILL
    FILL = value


# ---------------------------------------------------------------------------
# Array helpers
# ---------------------------------------------------------------------------
def shift(f: torch.Tensor, ax: int, s: int) -> torch.Tensor:
    """out[n] = f[n + s] along axis `ax`; out-of-range entries are FILL."""
    if s == 0:
        return f
    n = f.shape[ax]
    pad_shape = list(f.shape)
    pad_shape[ax] = abs(s)
    pad = torch.full(pad_shape, FILL, dtype=f.dtype)
    if s > 0:
        return torch.cat([f.narrow(ax, s, n - s), pad], dim=ax)
    return torch.cat([pad, f.narrow(ax, 0, n + s)], dim=ax)


def delta(f: torch.Tensor, ax: int) -> torch.Tensor:
    """Second-order centred difference in index space: (f[n+1] - f[n-1]) / 2."""
    return 0.5 * (shift(f, ax, 1) - shift(f, ax, -1))


def real(f: torch.Tensor) -> torch.Tensor:
    """Real (non-ghost) region of a padded array."""
    return f[..., G:-G, G:-G, G:-G]


class _Cbrt(torch.autograd.Function):
    """Real cube root (library cbrt), derivative 1/(3 t^2), taken as 0 at 0."""

    @staticmethod
    def forward(ctx, x):
        t = torch.from_numpy(np.cbrt(x.detach().numpy()))
        ctx.save_for_backward(t)
        return t

    @staticmethod
    def backward(ctx, g):
        (t,) = ctx.saved_tensors
        safe = torch.where(t != 0, t, torch.ones_like(t))
        return torch.where(t != 0, g / (3.0 * safe * safe), torch.zeros_like(t))


def cbrt(x: torch.Tensor) -> torch.Tensor:
    return _Cbrt.apply(x)


class _Sqrt0(torch.autograd.Function):
    """sqrt with derivative 1/(2 sqrt(x)), taken as 0 at x = 0 (subgradient convention)."""

    @staticmethod
    def forward(ctx, x):
        s = torch.sqrt(x)
        ctx.save_for_backward(s)
        return s

    @staticmethod
    def backward(ctx, g):
        (s,) = ctx.saved_tensors
        safe = torch.where(s > 0, s, torch.ones_like(s))
        return torch.where(s > 0, g / (2.0 * safe), torch.zeros_like(s))


def sqrt0(x: torch.Tensor) -> torch.Tensor:
    return _Sqrt0.apply(x)


# ---------------------------------------------------------------------------
# Parameters (derived constants computed here, independently of the library)
# ---------------------------------------------------------------------------
class Consts:
    """Derived constants of the non-dimensional formulation (Sec. LES Formulation)."""

    def __init__(self, prm):
        self.gamma = float(prm.gamma)
        self.gm1 = self.gamma - 1.0
        self.Cp = 1.0 / self.gm1                       # Cp = gamma R/(gamma-1), R = 1/gamma
        self.mu_ref = float(prm.mach_ref) / float(prm.Re)
        self.S_hat = float(prm.S1_K) / float(prm.T_ref_K)   # Sutherland constant / T_inf
        self.Pr = float(prm.Pr)
        self.Pr_sgs = float(prm.Pr_sgs)
        self.C_s = float(prm.C_s)
        self.kappa2 = float(prm.kappa2)
        self.kappa4 = float(prm.kappa4)
        self.sigma = float(prm.sigma)
        self.cfl = float(prm.cfl)
        self.dt_fixed = float(prm.dt_fixed)
        self.jet_mach = float(prm.jet_mach)
        self.theta_mom = float(prm.theta_mom)
        self.p_inf = 1.0 / self.gamma
        z = np.zeros((8, 4))
        self.amp = torch.as_tensor(z if prm.forcing_amp is None else np.asarray(prm.forcing_amp), dtype=DT)
        self.phi = torch.as_tensor(z if prm.forcing_phi is None else np.asarray(prm.forcing_phi), dtype=DT)
        self.psi = torch.as_tensor(z if prm.forcing_psi is None else np.asarray(prm.forcing_psi), dtype=DT)
        self.strouhal = [float(s) for s in prm.strouhal]


# ---------------------------------------------------------------------------
# Grid: ghost maps, padded coordinates, metrics (Algorithm 2: Calc(Jacob, Metric))
# ---------------------------------------------------------------------------
class Grid:
    """Grid topology, padded coordinates and stored metrics at every padded node.

    Stored metrics (the "area" vectors of the curvilinear transformation):
    S^xi = (xi_x, xi_y, xi_z)/J, S^eta, S^zeta and the cell volume V = 1/J,
    plus the grid constants |S^xi|, |S^eta|, |S^zeta| and Delta = V^(1/3)
    that the stage needs.
    """

    def __init__(self, ni, nj, nk, xyz, topology, period=None):
        self.ni, self.nj, self.nk = int(ni), int(nj), int(nk)
        self.topology = int(topology)
        self.period = np.zeros((3, 3)) if period is None else np.asarray(period, dtype=np.float64)
        self.shape_p = (self.nk + 2 * G, self.nj + 2 * G, self.ni + 2 * G)
        self.src = self._ghost_source_index()
        xyz = torch.as_tensor(np.asarray(xyz, dtype=np.float64)).reshape(3, self.nk, self.nj, self.ni)
        self.xyz_p = self._pad_coordinates(xyz)
        self._compute_metrics()
        self.updated = self._updated_mask()

    # --- ghost points (Sec. Parallel Implementation: two-layer ghost points) ---
    def _ghost_source_index(self) -> torch.Tensor:
        """Flat index of the real node whose state every padded node carries.

        Periodic box: wrap in all three directions.
        Jet: i clamped to [0, ni-1] (zero-order extrapolation at inflow and
        outflow); j < 0 is the across-axis neighbour (i, -j, k + nk/2); j >= nj
        copies the far-field node nj-1; k wraps (azimuthal periodicity).
        """
        ni, nj, nk = self.ni, self.nj, self.nk
        kk, jj, ii = torch.meshgrid(torch.arange(-G, nk + G), torch.arange(-G, nj + G),
                                    torch.arange(-G, ni + G), indexing="ij")
        if self.topology == TOPO_PERIODIC:
            i2, j2, k2 = ii % ni, jj % nj, kk % nk
        else:
            i2 = ii.clamp(0, ni - 1)
            below = jj < 0
            above = jj >= nj
            j2 = torch.where(below, -jj, torch.where(above, torch.full_like(jj, nj - 1), jj))
            k2 = torch.where(below, kk + nk // 2, kk) % nk
        return (k2 * nj + j2) * ni + i2

    def pad(self, f: torch.Tensor) -> torch.Tensor:
        """Fill a real array [..., nk, nj, ni] into the padded shape by the ghost map."""
        lead = f.shape[:-3]
        flat = f.reshape(*lead, -1)
        return flat[..., self.src.reshape(-1)].reshape(*lead, *self.shape_p)

    def _pad_coordinates(self, xyz: torch.Tensor) -> torch.Tensor:
        """Ghost coordinates.

        Periodic box: periodic images shifted by the period vectors.
        Jet: azimuthal wrap (no shift, the grid closes on itself), across-axis
        mirror (r -> -r, i.e. the node at (i, m, k + nk/2)), linear
        extrapolation beyond the far field and beyond the inflow/outflow planes.
        """
        ni, nj, nk = self.ni, self.nj, self.nk
        out = torch.empty((3,) + self.shape_p, dtype=DT)
        if self.topology == TOPO_PERIODIC:
            kk, jj, ii = torch.meshgrid(torch.arange(-G, nk + G), torch.arange(-G, nj + G),
                                        torch.arange(-G, ni + G), indexing="ij")
            base = self.pad(xyz)
            P = torch.as_tensor(self.period, dtype=DT)
            wi = torch.div(ii, ni, rounding_mode="floor").to(DT)
            wj = torch.div(jj, nj, rounding_mode="floor").to(DT)
            wk = torch.div(kk, nk, rounding_mode="floor").to(DT)
            for c in range(3):
                out[c] = base[c] + wi * P[0, c] + wj * P[1, c] + wk * P[2, c]
            return out
        # jet: k wrap + across-axis copy through the ghost map for real i
        base = self.pad(xyz)
        out[:] = base
        # far field: linear extrapolation in j (rows nj, nj+1) for every k
        jr = G + nj - 1
        for m in (1, 2):
            out[:, :, jr + m, :] = (1 + m) * out[:, :, jr, :] - m * out[:, :, jr - 1, :]
        # inflow / outflow: linear extrapolation in i for every (j, k)
        ir0, ir1 = G, G + ni - 1
        for m in (1, 2):
            out[..., ir0 - m] = (1 + m) * out[..., ir0] - m * out[..., ir0 + 1]
            out[..., ir1 + m] = (1 + m) * out[..., ir1] - m * out[..., ir1 - 1]
        return out

    def _compute_metrics(self):
        """Conservative metrics in the symmetric Thomas-Lombard form.

        With r = (x, y, z) and r_dir its centred index difference,
        S^xi   = [delta_zeta(r_eta x r) - delta_eta(r_zeta x r)] / 2,
        S^eta  = [delta_xi(r_zeta x r) - delta_zeta(r_xi x r)] / 2,
        S^zeta = [delta_eta(r_xi x r) - delta_xi(r_eta x r)] / 2,
        built from the same centred difference as the fluxes, so the discrete
        metric identities sum_dir delta_dir(S^dir) = 0 hold (a uniform flow is
        preserved on any grid); the vector form makes the metrics rotate with
        the grid (azimuthal equivariance on an axisymmetric mesh).
        V = 1/J is the triple product r_xi . (r_eta x r_zeta).
        """
        X = self.xyz_p
        dX = [delta(X, ax) for ax in (AX_I, AX_J, AX_K)]

        def cross(a, b):
            return torch.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])
        C = [cross(dX[d], X) for d in range(3)]
        Sx = list(0.5 * (delta(C[1], AX_K) - delta(C[2], AX_J)))
        Se = list(0.5 * (delta(C[2], AX_I) - delta(C[0], AX_K)))
        Sz = list(0.5 * (delta(C[0], AX_J) - delta(C[1], AX_I)))
        V = (dX[0] * cross(dX[1], dX[2])).sum(0)
        met = torch.stack(Sx + Se + Sz + [V])            # [10] padded, valid on real nodes
        self.metrics_real = real(met).clone()            # [10][nk][nj][ni]
        M = self.pad(self.metrics_real)                  # ghost values by the state's ghost map
        self.S = M[0:9].reshape(3, 3, *self.shape_p)     # S[dir][component]
        self.V = M[9]
        self.Smag = torch.sqrt((self.S * self.S).sum(dim=1))           # |S^dir|
        self.Delta = torch.from_numpy(np.cbrt(self.V.numpy()))         # filter width V^(1/3)
        self.invV = torch.where(self.V > 0, 1.0 / torch.where(self.V > 0, self.V, torch.ones_like(self.V)),
                                torch.zeros_like(self.V))

    def _updated_mask(self) -> torch.Tensor:
        """Real nodes advanced by the stencil (all for the box; interior for the jet)."""
        m = torch.ones((self.nk, self.nj, self.ni), dtype=torch.bool)
        if self.topology == TOPO_JET:
            m[:, 0, :] = False          # axis: azimuthal average
            m[:, -1, :] = False         # far field
            m[:, :, 0] = False          # inflow
            m[:, :, -1] = False         # outflow
        return m


# ---------------------------------------------------------------------------
# One residual evaluation (Algorithm 2: the steps from the inviscid flux to the RHS)
# ---------------------------------------------------------------------------
def primitives(Qp: torch.Tensor, c: Consts):
    """u_i = (rho u_i)/rho; p = (gamma-1)(e - rho|u|^2/2); T = gamma p / rho (p = rho R T, R = 1/gamma)."""
    rho = Qp[0]
    u, v, w = Qp[1] / rho, Qp[2] / rho, Qp[3] / rho
    p = c.gm1 * (Qp[4] - 0.5 * (Qp[1] * u + Qp[2] * v + Qp[3] * w))
    T = c.gamma * p / rho
    return rho, u, v, w, p, T


def sutherland(T: torch.Tensor, c: Consts) -> torch.Tensor:
    """Eq. (sutherland): mu = mu_ref (T/T_inf)^(3/2) (T_inf + S1)/(T + S1), T_inf = 1."""
    return c.mu_ref * (T * torch.sqrt(T)) * (1.0 + c.S_hat) / (T + c.S_hat)


def spectral_radii(grid: Grid, u, v, w, T):
    """lambda_dir = |U_dir| + a |S^dir|, U_dir = S^dir . u (volume-scaled), a = sqrt(gamma p/rho) = sqrt(T)."""
    a = torch.sqrt(T)
    lam = []
    for d in range(3):
        S = grid.S[d]
        U = S[0] * u + S[1] * v + S[2] * w
        lam.append(torch.abs(U) + a * grid.Smag[d])
    return lam


def anisotropic_scaling(lam, c: Consts):
    """Turkel-Vatsa anisotropic spectral radius, lambda_d [1 + sum_{e != d} (lambda_e/lambda_d)^sigma].

    Written as lambda_d + lambda_d^(1-sigma) sum_{e != d} lambda_e^sigma (no
    division, finite where lambda_d = 0).  sigma = 2/3 uses t = cbrt(lambda):
    lambda^(1/3) = t, lambda^(2/3) = t^2.
    """
    if abs(c.sigma - 2.0 / 3.0) < 1e-15:
        t = [cbrt(l) for l in lam]
        lo = t
        hi = [ti * ti for ti in t]
    else:
        def pw(x, e):
            safe = torch.where(x > 0, x, torch.ones_like(x))
            return torch.where(x > 0, safe ** e, torch.zeros_like(x))
        lo = [pw(l, 1.0 - c.sigma) for l in lam]
        hi = [pw(l, c.sigma) for l in lam]
    out = []
    for d in range(3):
        e1, e2 = [e for e in range(3) if e != d]
        out.append(lam[d] + lo[d] * (hi[e1] + hi[e2]))
    return out


def inviscid_flux(grid: Grid, Qp, u, v, w, p, d: int):
    """Transformed inviscid flux S^d_j E_j (eq. rhs/E): [rho U, rho u_i U + p S_i, (e + p) U]."""
    S = grid.S[d]
    U = S[0] * u + S[1] * v + S[2] * w
    return [Qp[0] * U,
            Qp[1] * U + p * S[0],
            Qp[2] * U + p * S[1],
            Qp[3] * U + p * S[2],
            (Qp[4] + p) * U]


def gradients(grid: Grid, phi):
    """Cartesian gradient at nodes by the chain rule: d phi/dx_j = J sum_dir S^dir_j delta_dir(phi).

    J = 1/V, taken as 0 on the axis where V = 0 (the gradient there only
    enters through the eta-face area, which vanishes on the axis).
    """
    dd = [delta(phi, AX_I), delta(phi, AX_J), delta(phi, AX_K)]
    return [grid.invV * (grid.S[0][j] * dd[0] + grid.S[1][j] * dd[1] + grid.S[2][j] * dd[2])
            for j in range(3)]


def viscous_fluxes(grid: Grid, rho, u, v, w, T, c: Consts):
    """Transformed viscous fluxes S^d_j F_j for d = xi, eta, zeta (eqs. tau_mod, q_mod, kappa_sgs, sgs_visc).

    tau_ij = 2 (mu + mu_sgs)(S_ij - delta_ij S_kk/3); heat flux
    (kappa + kappa_sgs) dT/dx_j enters F with the sign of physical diffusion;
    mu_sgs = rho (C_s Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij), Delta = V^(1/3);
    kappa = mu Cp/Pr, kappa_sgs = mu_sgs Cp/Pr_sgs; sigma_kk = 0.
    Returns F[d] = [F_mom_x, F_mom_y, F_mom_z, F_energy] (mass flux is zero).
    """
    gu, gv, gw, gT = gradients(grid, u), gradients(grid, v), gradients(grid, w), gradients(grid, T)
    L = [gu, gv, gw]                               # L[i][j] = d u_i / d x_j
    Sij = [[0.5 * (L[i][j] + L[j][i]) for j in range(3)] for i in range(3)]
    div = Sij[0][0] + Sij[1][1] + Sij[2][2]
    SS = sum(Sij[i][j] * Sij[i][j] for i in range(3) for j in range(3))
    Smod = sqrt0(2.0 * SS)
    mu = sutherland(T, c)
    mu_sgs = rho * (c.C_s * grid.Delta) ** 2 * Smod
    mu_eff = mu + mu_sgs
    k_eff = mu * c.Cp / c.Pr + mu_sgs * c.Cp / c.Pr_sgs
    tau = [[2.0 * mu_eff * (Sij[i][j] - (div / 3.0 if i == j else 0.0)) for j in range(3)] for i in range(3)]
    vel = [u, v, w]
    Fcart = []                                     # Cartesian viscous flux in direction j
    for j in range(3):
        energy = vel[0] * tau[0][j] + vel[1] * tau[1][j] + vel[2] * tau[2][j] + k_eff * gT[j]
        Fcart.append([tau[0][j], tau[1][j], tau[2][j], energy])
    out = []
    for d in range(3):
        S = grid.S[d]
        out.append([S[0] * Fcart[0][m] + S[1] * Fcart[1][m] + S[2] * Fcart[2][m] for m in range(4)])
    return out


def pressure_sensor(p, ax: int):
    """nu_n = |p_{n+1} - 2 p_n + p_{n-1}| / (p_{n+1} + 2 p_n + p_{n-1}) along one direction."""
    pp, pm = shift(p, ax, 1), shift(p, ax, -1)
    return torch.abs(pp - 2.0 * p + pm) / (pp + 2.0 * p + pm)


def dissipation_face_flux(Qp, Lam_d, nu, ax: int, c: Consts):
    """Turkel-Vatsa face flux at n+1/2 along one direction (stored at index n).

    d_{n+1/2} = Lambda_{n+1/2} [eps2 (Q_{n+1} - Q_n) - eps4 (Q_{n+2} - 3 Q_{n+1} + 3 Q_n - Q_{n-1})],
    eps2 = kappa2 max(nu_n, nu_{n+1}), eps4 = max(0, kappa4 - eps2),
    Lambda_{n+1/2} = (Lambda_n + Lambda_{n+1}) / 2.
    """
    nu1 = shift(nu, ax, 1)
    eps2 = c.kappa2 * torch.where(nu >= nu1, nu, nu1)
    k4 = c.kappa4 - eps2
    eps4 = torch.where(k4 > 0, k4, torch.zeros_like(k4))
    Lf = 0.5 * (Lam_d + shift(Lam_d, ax, 1))
    Q1, Q2, Qm = shift(Qp, ax, 1), shift(Qp, ax, 2), shift(Qp, ax, -1)
    d1 = Q1 - Qp
    d3 = Q2 - 3.0 * Q1 + 3.0 * Qp - Qm
    return Lf * (eps2 * d1 - eps4 * d3)


def residual_padded(grid: Grid, Qp: torch.Tensor, c: Consts) -> torch.Tensor:
    """RHS of eq. (vec-les), dQ/dt = -RHS, in curvilinear form, on the real nodes.

    V RHS = sum_dir [delta_dir(E^dir - F^dir)] - sum_dir [d_{n+1/2} - d_{n-1/2}]
    (centred flux differences plus scalar artificial dissipation).  Returned on
    every real node; only the updated nodes are used by the time step.
    """
    rho, u, v, w, p, T = primitives(Qp, c)
    lam = spectral_radii(grid, u, v, w, T)
    Lam = anisotropic_scaling(lam, c)
    Fv = viscous_fluxes(grid, rho, u, v, w, T, c)
    axes = (AX_I, AX_J, AX_K)
    acc = torch.zeros_like(Qp)
    for d in range(3):
        E = inviscid_flux(grid, Qp, u, v, w, p, d)                    # Calc(Inv. Flux)
        nu = pressure_sensor(p, axes[d])
        dface = dissipation_face_flux(Qp, Lam[d], nu, axes[d], c)     # Calc(Art. Diss.)
        H = torch.stack([E[0]] + [E[m + 1] - Fv[d][m] for m in range(4)])   # Calc(Visc. Flux)
        acc = acc + delta(H, axes[d]) - (dface - shift(dface, axes[d], -1))
    return real(acc * grid.invV)                                      # Calc(RHS Vec.)


def residual(grid: Grid, Q: torch.Tensor, c: Consts) -> torch.Tensor:
    """RHS on real nodes from an unpadded state; zero on nodes the stencil does not update."""
    R = residual_padded(grid, grid.pad(Q), c)
    return torch.where(grid.updated, R, torch.zeros_like(R))


# ---------------------------------------------------------------------------
# Boundary conditions (Sec. LES Formulation: entrance, far field, exit,
# periodicity, centerline), applied after every stage (Update(B.C., Visc.))
# ---------------------------------------------------------------------------
def _cons(rho, u, v, w, p, c: Consts):
    e = p / c.gm1 + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, e])


def _rho_from_isentrope(a2, s, c: Consts):
    """rho from a^2 = gamma p/rho and s = p/rho^gamma: rho = (a^2/(gamma s))^(1/(gamma-1))."""
    return (a2 / (c.gamma * s)) ** (1.0 / c.gm1)


def farfield_bc(grid: Grid, Q, c: Consts):
    """Riemann-invariant far field at j = nj-1, i in [1, ni-2] (reading of the garbled passage).

    n = S^eta/|S^eta|; R+ = u_int.n + 2 a_int/(gamma-1) from j = nj-2;
    R- = u_inf.n - 2 a_inf/(gamma-1) with a quiescent ambient (u_inf = 0, a_inf = 1);
    u_n = (R+ + R-)/2, a = (gamma-1)(R+ - R-)/4; tangential velocity and
    entropy p/rho^gamma from the interior where u_n > 0, else ambient.
    """
    jb = grid.nj - 1
    S = real(grid.S[1])[:, :, jb, 1:-1]          # [3][nk][ni-2]
    n = S / torch.sqrt((S * S).sum(0))
    qi = Q[:, :, jb - 1, 1:-1]
    rho_i = qi[0]
    ui = qi[1:4] / rho_i
    p_i = c.gm1 * (qi[4] - 0.5 * (qi[1:4] * ui).sum(0))
    a_i = torch.sqrt(c.gamma * p_i / rho_i)
    un_i = (ui * n).sum(0)
    Rp = un_i + 2.0 * a_i / c.gm1
    Rm = -2.0 / c.gm1
    un = 0.5 * (Rp + Rm)
    ab = 0.25 * c.gm1 * (Rp - Rm)
    out_flow = un > 0
    ut = torch.where(out_flow, ui - un_i * n, torch.zeros_like(ui))
    s = torch.where(out_flow, p_i / rho_i ** c.gamma, torch.full_like(p_i, c.p_inf))
    rho = _rho_from_isentrope(ab * ab, s, c)
    p = rho * ab * ab / c.gamma
    ub = ut + un * n
    Q = Q.clone()
    Q[:, :, jb, 1:-1] = _cons(rho, ub[0], ub[1], ub[2], p, c)
    return Q


def inflow_target(grid: Grid, c: Consts, t):
    """Jet entrance target (tanh profile + azimuthal-mode forcing) on (j in [1, nj-1], all k).

    u_x = U_j/2 [1 + tanh((0.5 - r)/(2 theta))] + U_j sum_{m,f} A_mf g(r)
    cos(m theta + phi_mf) sin(2 pi St_f U_j t + psi_mf), g = exp(-((r-0.5)/0.1)^2);
    v = w = 0, T = 1, p = 1/gamma (PR = TR = 1).
    """
    xyz = grid.xyz_p[:, G:-G, G:-G, G:-G][:, :, 1:, 0]     # [3][nk][nj-1] at i = 0
    r = torch.sqrt(xyz[1] * xyz[1] + xyz[2] * xyz[2])
    th = torch.atan2(xyz[2], xyz[1])
    Uj = c.jet_mach
    u = 0.5 * Uj * (1.0 + torch.tanh((0.5 - r) / (2.0 * c.theta_mom)))
    g = torch.exp(-((r - 0.5) / 0.1) ** 2)
    t = torch.as_tensor(t, dtype=DT)
    f = torch.zeros_like(r)
    for m in range(8):
        for q in range(4):
            tm = torch.sin(2.0 * math.pi * c.strouhal[q] * Uj * t + c.psi[m, q])
            f = f + c.amp[m, q] * torch.cos(m * th + c.phi[m, q]) * tm
    return u + Uj * g * f


def inflow_bc(grid: Grid, Q, c: Consts, t):
    """Entrance at i = 0, j in [1, nj-1] by 1-D characteristics along x.

    Supersonic target (u >= a = 1): all variables imposed.  Subsonic: R- =
    u - 2a/(gamma-1) extrapolated from i = 1; R+, entropy, v, w from the target.
    """
    ut = inflow_target(grid, c, t)
    q1 = Q[:, :, 1:, 1]
    rho1 = q1[0]
    u1 = q1[1:4] / rho1
    p1 = c.gm1 * (q1[4] - 0.5 * (q1[1:4] * u1).sum(0))
    a1 = torch.sqrt(c.gamma * p1 / rho1)
    Rm = u1[0] - 2.0 * a1 / c.gm1
    Rp = ut + 2.0 * 1.0 / c.gm1
    ub = 0.5 * (Rp + Rm)
    ab = 0.25 * c.gm1 * (Rp - Rm)
    rho_sub = _rho_from_isentrope(ab * ab, torch.full_like(ab, c.p_inf), c)
    p_sub = rho_sub * ab * ab / c.gamma
    sup = ut >= 1.0
    rho = torch.where(sup, torch.ones_like(ut), rho_sub)
    p = torch.where(sup, torch.full_like(ut, c.p_inf), p_sub)
    u = torch.where(sup, ut, ub)
    z = torch.zeros_like(ut)
    Q = Q.clone()
    Q[:, :, 1:, 0] = _cons(rho, u, z, z, p, c)
    return Q


def outflow_bc(grid: Grid, Q, c: Consts):
    """Exit at i = ni-1, j in [1, nj-1]: p imposed (p_inf); velocity and internal energy copied from i = ni-2."""
    qi = Q[:, :, 1:, -2]
    rho_i = qi[0]
    ui = qi[1:4] / rho_i
    p_i = c.gm1 * (qi[4] - 0.5 * (qi[1:4] * ui).sum(0))
    eint = p_i / (c.gm1 * rho_i)                 # internal energy per unit mass
    p = torch.full_like(p_i, c.p_inf)
    rho = p / (c.gm1 * eint)
    Q = Q.clone()
    Q[:, :, 1:, -1] = _cons(rho, ui[0], ui[1], ui[2], p, c)
    return Q


def centerline_bc(Q):
    """Axis j = 0: conserved variables of the adjacent ring j = 1 averaged over the azimuth."""
    ring = Q[:, :, 1, :].mean(dim=1, keepdim=True)          # [5][1][ni]
    Q = Q.clone()
    Q[:, :, 0, :] = ring.expand(-1, Q.shape[1], -1)
    return Q


def apply_bcs(grid: Grid, Q, c: Consts, t):
    """Update(B.C.) after a stage: far field, entrance, exit, then the axis average (jet only)."""
    if grid.topology != TOPO_JET:
        return Q
    Q = farfield_bc(grid, Q, c)
    Q = inflow_bc(grid, Q, c, t)
    Q = outflow_bc(grid, Q, c)
    Q = centerline_bc(Q)
    return Q


# ---------------------------------------------------------------------------
# Time step and the 5-stage Runge-Kutta scheme (Algorithm 2 main loop)
# ---------------------------------------------------------------------------
def cfl_dt(grid: Grid, Q, c: Consts):
    """dt = CFL / max over updated nodes of (lambda_xi + lambda_eta + lambda_zeta)/V."""
    if c.dt_fixed > 0:
        return torch.as_tensor(c.dt_fixed, dtype=DT)
    _, u, v, w, _, T = primitives(grid.pad(Q), c)
    lam = spectral_radii(grid, u, v, w, T)
    rate = real((lam[0] + lam[1] + lam[2]) * grid.invV)
    return c.cfl / rate[grid.updated].max()


def rk_stages(Qn, stage_rhs, updated, dt, bc):
    """Low-storage 5-stage Runge-Kutta (Jameson et al.; Algorithm 2, Update(Cons., alpha_l)).

    Q^(0) = Q^n; Q^(l) = Q^n - alpha_l dt RHS(Q^(l-1)) on the updated nodes,
    then bc(Q^(l), alpha_l); Q^{n+1} = Q^(5).  alpha = (1/4, 1/6, 3/8, 1/2, 1).
    """
    Qs = Qn
    rhs = []
    for a in RK_ALPHA:
        R = stage_rhs(Qs)
        rhs.append(R)
        Qs = torch.where(updated, Qn - a * dt * R, Qs)
        Qs = bc(Qs, a)
    return Qs, rhs


def rk_step(grid: Grid, Q, c: Consts, t, dt=None):
    """One time step of the solver with boundary conditions after each stage.

    Returns (Q^{n+1}, dt, RHS of stage 1).
    """
    if dt is None:
        dt = cfl_dt(grid, Q, c)
    Qs, rhs = rk_stages(Q, lambda q: residual_padded(grid, grid.pad(q), c), grid.updated, dt,
                        lambda q, a: apply_bcs(grid, q, c, t + a * dt))
    return Qs, dt, rhs[0]


def run(grid: Grid, Q, c: Consts, nsteps: int, t0: float = 0.0):
    """nsteps time steps; returns (Q, t, list of dt, RHS of stage 1 of the last step)."""
    t = torch.as_tensor(t0, dtype=DT)
    dts = []
    R1 = None
    for _ in range(nsteps):
        Q, dt, R1 = rk_step(grid, Q, c, t)
        t = t + dt
        dts.append(dt)
    return Q, t, dts, R1


def totals(grid: Grid, Q):
    """Conservation totals sum over real nodes of Q_m V."""
    V = grid.metrics_real[9]
    return (Q * V).reshape(5, -1).sum(dim=1)


def residual_l2(grid: Grid, R):
    """RMS over updated nodes of the density residual."""
    r = R[0][grid.updated]
    return torch.sqrt((r * r).mean())


# ---------------------------------------------------------------------------
# Observer functional and its discrete adjoint (reverse sweep by autograd)
# ---------------------------------------------------------------------------
class Observer:
    """Cylindrical observer surface r = r_obs of a jet grid.

    Pressure on the surface is interpolated linearly in r between the
    bracketing grid lines j_o, j_o + 1 (the radial coordinate of a jet grid
    depends on j only); the surface weights are w_ik = r_obs dtheta dx_i with
    the trapezoid dx_i of the axial coordinate.
    """

    def __init__(self, grid: Grid, r_obs: float):
        X = real(grid.xyz_p)
        r = torch.sqrt(X[1, 0, :, 0] ** 2 + X[2, 0, :, 0] ** 2)       # r_j at i = 0, k = 0
        below = (r <= r_obs).nonzero().flatten()
        self.j0 = int(below.max())
        if self.j0 >= grid.nj - 1:
            raise ValueError("observer radius beyond the far field")
        self.beta = float((r_obs - r[self.j0]) / (r[self.j0 + 1] - r[self.j0]))
        x = X[0, 0, 0, :]
        dx = torch.empty_like(x)
        dx[1:-1] = 0.5 * (x[2:] - x[:-2])
        dx[0] = 0.5 * (x[1] - x[0])
        dx[-1] = 0.5 * (x[-1] - x[-2])
        self.w = (r_obs * (2.0 * math.pi / grid.nk)) * dx              # [ni], same for every k

    def value(self, Q, c: Consts):
        """sum_{i,k} w_ik (p~_ik - p_inf)^2 for one state Q."""
        def pres(q):
            return c.gm1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0])
        p0 = pres(Q[:, :, self.j0, :])
        p1 = pres(Q[:, :, self.j0 + 1, :])
        pt = (1.0 - self.beta) * p0 + self.beta * p1
        return (self.w * (pt - c.p_inf) ** 2).sum()


def functional(grid: Grid, Q0, c: Consts, amps, nsteps: int, dt, obs: Observer, t0: float = 0.0):
    """J = sum_{n=1..N} dt sum_ik w_ik (p~_ik(Q^n) - p_inf)^2 with the forcing amplitudes `amps`
    ([8][4]) and a frozen time step dt; each step is recomputed in the backward pass."""
    from torch.utils.checkpoint import checkpoint
    c.amp = amps
    dt = torch.as_tensor(dt, dtype=DT)
    Q = Q0
    J = torch.zeros((), dtype=DT)
    for n in range(nsteps):
        t = torch.as_tensor(t0 + n * float(dt), dtype=DT)
        Q = checkpoint(lambda q, a, t=t: rk_step(grid, q, c, t, dt=dt)[0], Q, amps, use_reentrant=False)
        J = J + dt * obs.value(Q, c)
    return J


def functional_gradient(grid: Grid, Q0, c: Consts, amps, nsteps: int, dt, obs: Observer, t0: float = 0.0):
    """(J, dJ/dA) by reverse-mode differentiation of the discrete forward map (the oracle's reverse sweep)."""
    old = FILL
    set_fill(0.0)                     # keep shifted-in entries finite for the backward pass
    try:
        A = torch.as_tensor(amps, dtype=DT).clone().requires_grad_(True)
        J = functional(grid, Q0, c, A, nsteps, dt, obs, t0)
        (g,) = torch.autograd.grad(J, A)
    finally:
        set_fill(old)
    return J.detach(), g


# ---------------------------------------------------------------------------
# Flow statistics (Sec. "Validation": time-averaged axial velocity on the
# centreline and in radial profiles at fixed x/D, rms of the axial velocity,
# potential-core length where the centreline mean drops to 95% of U_j)
# ---------------------------------------------------------------------------
def flow_statistics(samples):
    """Time statistics of the axial velocity u_x = (rho u_x) / rho over a list of states
    Q [5][nk][nj][ni]: per node the mean and the rms about it (population definitions,
    two passes), each then averaged over the azimuth k.  Returns (mean, rms), [nj][ni]."""
    U = torch.stack([Q[1] / Q[0] for Q in samples])            # [S][nk][nj][ni]
    mean = U.mean(dim=0)
    rms = torch.sqrt(((U - mean) ** 2).mean(dim=0))
    return mean.mean(dim=0), rms.mean(dim=0)


def station_profile(field, x, x0: float):
    """Radial profile of field [nj][ni] at axial position x0: linear interpolation in x
    between the two i lines that bracket x0 (x [ni] increasing)."""
    x = torch.as_tensor(x, dtype=DT)
    if not (float(x[0]) <= x0 <= float(x[-1])):
        raise ValueError("station outside the axial range")
    i1 = int((x >= x0).nonzero().flatten()[0])
    if i1 == 0:
        return field[:, 0].clone()
    i0 = i1 - 1
    w = (x0 - x[i0]) / (x[i1] - x[i0])
    return (1.0 - w) * field[:, i0] + w * field[:, i1]


def potential_core_length(axis_mean, x, u_jet: float, frac: float = 0.95):
    """First axial position where the centreline mean velocity axis_mean [ni] falls below
    frac * u_jet, interpolated linearly between the bracketing i lines; None if it never does."""
    x = torch.as_tensor(x, dtype=DT)
    thr = frac * u_jet
    below = (axis_mean < thr).nonzero().flatten()
    if below.numel() == 0:
        return None
    i1 = int(below[0])
    if i1 == 0:
        return float(x[0])
    i0 = i1 - 1
    w = (axis_mean[i0] - thr) / (axis_mean[i0] - axis_mean[i1])
    return float(x[i0] + w * (x[i1] - x[i0]))


def make(xyz, ni, nj, nk, topology, period, prm):
    """Convenience: (Grid, Consts) from plain arrays and a parameter object."""
    return Grid(ni, nj, nk, xyz, topology, period), Consts(prm)
