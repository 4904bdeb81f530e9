"""Seeded synthetic workloads: grids, initial states and inflow-forcing draws.

This module is the only code shared by the CUDA path, the CPU oracle and the
benchmark.  It produces plain FP64 arrays (NumPy, seeded PCG64) and holds none
of the solver's arithmetic: no metrics, fluxes, dissipation, boundary
conditions or time stepping.  The initial states are written as conserved
variables using the definition of the total energy per unit volume
(e = p/(gamma-1) + rho|u|^2/2, paper Sec. "Large Eddy Simulation Formulation"),
which is how the state vector Q is defined, not a step of the method.

Non-dimensionalisation (ambient reference state): rho_inf = 1, a_inf = 1,
T_inf = 1, p_inf = 1/gamma; lengths in jet diameters D.

Shapes follow the paper's jet workloads (axial x radial x azimuthal meshes,
Table "mesh" of Sec. "Scalability setup"; 30 D x 10 D domain) and the periodic
box used for conservation and linear-mode checks.

Array layout everywhere: C-order ``[..., nk, nj, ni]`` (i fastest), i.e. the
coordinate array is ``xyz[3][nk][nj][ni]`` and the state ``q[5][nk][nj][ni]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4

# Topology codes shared with the C ABI (include/jz.h).
TOPO_PERIODIC = 1
TOPO_JET = 2


# ---------------------------------------------------------------------------
# Parameter sets (plain numbers; derived constants are computed by each side)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class FlowParams:
    """Physical and numerical parameters of one run (plain inputs)."""

    gamma: float = GAMMA
    Pr: float = 0.72          # paper: Prandtl number of air
    Pr_sgs: float = 0.9       # paper: SGS Prandtl number for static closures
    Re: float = 1.0e4         # Reynolds number built on U_ref = mach_ref * a_inf
    mach_ref: float = 0.5
    T_ref_K: float = 288.15   # dimensional ambient temperature for Sutherland
    S1_K: float = 110.4       # Sutherland constant, paper eq. (sutherland)
    C_s: float = 0.18         # Smagorinsky constant (0 reproduces the paper's runs)
    kappa2: float = 0.25      # Turkel-Vatsa 2nd-difference coefficient
    kappa4: float = 1.0 / 64  # Turkel-Vatsa 4th-difference coefficient
    sigma: float = 2.0 / 3.0  # anisotropy exponent of the spectral-radius scaling
    cfl: float = 0.5
    dt_fixed: float = 0.0     # > 0: fixed time step instead of the CFL step
    # jet inflow (used only on the jet topology)
    jet_mach: float = 1.4     # U_j / a_inf
    theta_mom: float = 0.05   # momentum thickness of the tanh profile (units of D)
    forcing_amp: np.ndarray | None = None    # [8][4]
    forcing_phi: np.ndarray | None = None    # [8][4] azimuthal phase
    forcing_psi: np.ndarray | None = None    # [8][4] temporal phase
    strouhal: tuple = (0.2, 0.4, 0.6, 0.8)


N_MODES = 8
N_FREQ = 4


def forcing_draw(seed: int, amp_max: float = 1.0e-3):
    """Seeded inflow-forcing draw: amplitudes U[0, amp_max], phases U[0, 2pi).

    Returns (amp, phi, psi), each of shape [8 azimuthal modes][4 frequencies].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=(N_MODES, N_FREQ))
    psi = rng.uniform(0.0, 2.0 * math.pi, size=(N_MODES, N_FREQ))
    amp = rng.uniform(0.0, amp_max, size=(N_MODES, N_FREQ))
    return amp, phi, psi


def box_params(**kw) -> FlowParams:
    """Periodic-box run: Mach 0.5 reference flow, Re = 1e4, Smagorinsky SGS."""
    p = FlowParams(Re=1.0e4, mach_ref=0.5, C_s=0.18)
    return dataclasses.replace(p, **kw)


def jet_params(seed: int = 2, **kw) -> FlowParams:
    """Jet run: M = 1.4 perfectly expanded unheated jet, Re = 1.57e6 (Sec. Scalability setup)."""
    amp, phi, psi = forcing_draw(seed)
    p = FlowParams(Re=1.57e6, mach_ref=1.4, C_s=0.18, jet_mach=1.4, theta_mom=0.05,
                   forcing_amp=amp, forcing_phi=phi, forcing_psi=psi)
    return dataclasses.replace(p, **kw)


# ---------------------------------------------------------------------------
# Grids
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    ni: int
    nj: int
    nk: int
    xyz: np.ndarray              # [3][nk][nj][ni] float64
    topology: int
    period: np.ndarray           # [3 directions i,j,k][3 components] shift vectors

    @property
    def npts(self) -> int:
        return self.ni * self.nj * self.nk


def box_grid(ni: int, nj: int, nk: int, h: float | None = None) -> Grid:
    """Uniform Cartesian triply periodic box with spacing h (default 2*pi/ni)."""
    h = 2.0 * math.pi / ni if h is None else h
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    xyz = np.stack([i * h, j * h, k * h]).astype(np.float64)
    period = np.diag([ni * h, nj * h, nk * h]).astype(np.float64)
    return Grid(ni, nj, nk, np.ascontiguousarray(xyz), TOPO_PERIODIC, period)


def wavy_periodic_grid(ni: int, nj: int, nk: int, amp: float = 0.08, seed: int = 7) -> Grid:
    """Smooth, randomly phased curvilinear distortion of a periodic box.

    x = L * (s + amp * sum of periodic sines of (s, t, u)), with s, t, u the
    normalised index coordinates; every displacement is periodic in all three
    indices, so the grid tiles space with the box periods.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = np.array([2.0 * math.pi, 1.5 * math.pi, 1.0 * math.pi])
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    s, t, u = i / ni, j / nj, k / nk
    ph = rng.uniform(0, 2 * math.pi, size=(3, 3))
    xyz = np.empty((3, nk, nj, ni))
    base = (s, t, u)
    for c in range(3):
        d = (np.sin(2 * math.pi * s + ph[c, 0]) * np.sin(2 * math.pi * t + ph[c, 1])
             * np.sin(2 * math.pi * u + ph[c, 2]))
        xyz[c] = L[c] * (base[c] + amp * d)
    period = np.diag(L).astype(np.float64)
    return Grid(ni, nj, nk, np.ascontiguousarray(xyz), TOPO_PERIODIC, period)


def stretched_coordinate(n: int, length: float, ratio: float, centre: float, width: float,
                         samples: int = 200001) -> np.ndarray:
    """n points on [0, length], spacing growing from the point `centre` outwards.

    The spacing is proportional to 1 + (ratio - 1) * tanh(|s - centre| / width):
    finest at `centre`, `ratio` times coarser far from it.  The map is built by
    integrating the inverse spacing on a fine sample and inverting it, so the
    first point is exactly 0 and the last exactly `length`.
    """
    s = np.linspace(0.0, length, samples)
    dens = 1.0 / (1.0 + (ratio - 1.0) * np.tanh(np.abs(s - centre) / width))
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(s))])
    cum *= (n - 1) / cum[-1]
    out = np.interp(np.arange(n, dtype=np.float64), cum, s)
    out[0], out[-1] = 0.0, length
    return out


def jet_grid(ni: int, nj: int, nk: int, length: float = 30.0, radius: float = 10.0,
             radial_ratio: float = 10.0, axial_stretch: bool = False) -> Grid:
    """Cylindrical jet grid: axial x, radial r (tanh-stretched at r = 0.5 D), azimuthal theta.

    j = 0 lies on the jet axis (r = 0); the nk azimuthal points are unique,
    theta_k = 2 pi k / nk (the paper's superposed first/last point is dropped),
    so nk must be even for the across-axis neighbours.  y = r cos(theta),
    z = r sin(theta).
    """
    if nk % 2:
        raise ValueError("jet grid needs an even azimuthal point count")
    if axial_stretch:
        x = stretched_coordinate(ni, length, 4.0, 0.0, 5.0)
    else:
        x = np.linspace(0.0, length, ni)
    r = stretched_coordinate(nj, radius, radial_ratio, 0.5, 0.5)
    th = 2.0 * math.pi * np.arange(nk) / nk
    xyz = np.empty((3, nk, nj, ni))
    xyz[0] = x[None, None, :]
    xyz[1] = (np.cos(th)[:, None] * r[None, :])[:, :, None]
    xyz[2] = (np.sin(th)[:, None] * r[None, :])[:, :, None]
    return Grid(ni, nj, nk, np.ascontiguousarray(xyz), TOPO_JET, np.zeros((3, 3)))


def jet_grid_device(ni: int, nj: int, nk: int, device="cuda", length: float = 30.0, radius: float = 10.0,
                    radial_ratio: float = 10.0, axial_stretch: bool = False):
    """The jet_grid recipe built on a torch device (for meshes too large to build quickly
    on the host): the 1-D axes come from the same NumPy code, the 3-D coordinate array
    [3][nk][nj][ni] is formed on the device."""
    import torch
    if nk % 2:
        raise ValueError("jet grid needs an even azimuthal point count")
    x = stretched_coordinate(ni, length, 4.0, 0.0, 5.0) if axial_stretch else np.linspace(0.0, length, ni)
    r = stretched_coordinate(nj, radius, radial_ratio, 0.5, 0.5)
    th = 2.0 * math.pi * np.arange(nk) / nk
    xt = torch.as_tensor(x, dtype=torch.float64, device=device)
    rt = torch.as_tensor(r, dtype=torch.float64, device=device)
    ct = torch.as_tensor(np.cos(th), dtype=torch.float64, device=device)
    st = torch.as_tensor(np.sin(th), dtype=torch.float64, device=device)
    xyz = torch.empty((3, nk, nj, ni), dtype=torch.float64, device=device)
    xyz[0] = xt[None, None, :]
    xyz[1] = (ct[:, None] * rt[None, :])[:, :, None]
    xyz[2] = (st[:, None] * rt[None, :])[:, :, None]
    return xyz


def jet_state_device(xyz, jet_mach: float = 1.4, theta_mom: float = 0.05, gamma: float = GAMMA):
    """jet_state on a torch device: parallel tanh jet, uniform rho and p."""
    import torch
    r = torch.sqrt(xyz[1] * xyz[1] + xyz[2] * xyz[2])
    u = 0.5 * jet_mach * (1.0 + torch.tanh((0.5 - r) / (2.0 * theta_mom)))
    q = torch.zeros((5,) + tuple(r.shape), dtype=torch.float64, device=xyz.device)
    q[0] = 1.0
    q[1] = u
    q[4] = (1.0 / gamma) / (gamma - 1.0) + 0.5 * u * u
    return q


# Paper's Table "mesh" (axial x radial points; 361 azimuthal points with the first and
# last superposed -> 360 unique).
PAPER_MESHES = {"A": (128, 128), "B": (256, 128), "C": (256, 256), "D": (512, 256), "E": (512, 512),
                "F": (1024, 512), "G": (1024, 1024), "H": (2048, 1024), "I": (1700, 1700)}


# ---------------------------------------------------------------------------
# Initial states (conserved variables [rho, rho u, rho v, rho w, e])
# ---------------------------------------------------------------------------
def conserved(rho, u, v, w, p, gamma: float = GAMMA) -> np.ndarray:
    """Stack the conserved vector Q from primitive fields (definition of e)."""
    e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, rho * w, e]).astype(np.float64))


def box_state(grid: Grid, seed: int = 1, mach: float = 0.5, noise: float = 1.0e-3,
              gamma: float = GAMMA) -> np.ndarray:
    """Uniform Mach `mach` flow along x plus i.i.d. N(0, noise^2) velocity noise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = (grid.nk, grid.nj, grid.ni)
    du = rng.standard_normal(size=(3,) + shp) * noise
    rho = np.ones(shp)
    p = np.full(shp, 1.0 / gamma)
    return conserved(rho, mach + du[0], du[1], du[2], p, gamma)


def jet_state(grid: Grid, jet_mach: float = 1.4, theta_mom: float = 0.05,
              gamma: float = GAMMA) -> np.ndarray:
    """Parallel jet: the unforced tanh profile extruded along x, uniform rho and p."""
    y, z = grid.xyz[1], grid.xyz[2]
    r = np.sqrt(y * y + z * z)
    u = 0.5 * jet_mach * (1.0 + np.tanh((0.5 - r) / (2.0 * theta_mom)))
    shp = r.shape
    return conserved(np.ones(shp), u, np.zeros(shp), np.zeros(shp), np.full(shp, 1.0 / gamma), gamma)


def smooth_state(grid: Grid, seed: int = 3, amp: float = 0.05, gamma: float = GAMMA) -> np.ndarray:
    """Smooth periodic state (one Fourier mode per field, random phases).

    Used for order-of-accuracy and parity checks on periodic grids; every field
    is periodic in the index coordinates.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k, j, i = np.meshgrid(np.arange(grid.nk), np.arange(grid.nj), np.arange(grid.ni), indexing="ij")
    s, t, u = 2 * math.pi * i / grid.ni, 2 * math.pi * j / grid.nj, 2 * math.pi * k / grid.nk
    ph = rng.uniform(0, 2 * math.pi, size=(5, 3))
    f = [np.sin(s + ph[c, 0]) * np.cos(t + ph[c, 1]) * np.sin(u + ph[c, 2]) for c in range(5)]
    rho = 1.0 + amp * f[0]
    return conserved(rho, 0.4 + amp * f[1], amp * f[2], amp * f[3], (1.0 + amp * f[4]) / gamma, gamma)


def random_state(grid: Grid, seed: int, amp: float = 0.05, base_u=(0.3, 0.1, -0.1),
                 gamma: float = GAMMA) -> np.ndarray:
    """I.i.d. noisy state around a uniform flow (exercises every stencil branch)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = (grid.nk, grid.nj, grid.ni)
    n = rng.standard_normal(size=(5,) + shp) * amp
    rho = 1.0 + n[0]
    p = (1.0 + n[4]) / gamma
    return conserved(rho, base_u[0] + n[1], base_u[1] + n[2], base_u[2] + n[3], p, gamma)


# ---------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped runs)
# ---------------------------------------------------------------------------
WORKLOADS = {
    "box32x24x16": dict(kind="box", shape=(32, 24, 16), steps=10),
    "jet256x128x64": dict(kind="jet", shape=(256, 128, 64), steps=100),
    "jet512x256x128": dict(kind="jet", shape=(512, 256, 128), steps=500),
    "jet64x32x16": dict(kind="jet", shape=(64, 32, 16), steps=500),
    "jet128x96x64": dict(kind="jet", shape=(128, 96, 64), steps=200),
    "jet1000x400x500": dict(kind="jet", shape=(1000, 400, 500), steps=20, axial_stretch=True),
}


def make_workload(name: str, forcing_seed: int = 2):
    """Grid, initial state and parameters of a named workload."""
    w = WORKLOADS[name]
    ni, nj, nk = w["shape"]
    if w["kind"] == "box":
        g = box_grid(ni, nj, nk)
        return g, box_state(g, seed=1), box_params()
    g = jet_grid(ni, nj, nk, axial_stretch=w.get("axial_stretch", False))
    prm = jet_params(seed=forcing_seed)
    return g, jet_state(g, prm.jet_mach, prm.theta_mom), prm
