"""Flow statistics of the axial velocity (jz_stats_*) against the oracle.

Bar: the GPU states agree with the oracle's to <= 1e-12 relative, so u_x = (rho u_x)/rho
agrees to ~1e-12 absolute (|u_x| <= U_j = 1.4); the mean and the rms are 1-Lipschitz in the
samples' sup-norm, hence both must agree to 1e-11 absolute.  Welford accumulation (GPU)
against the two-pass definition (oracle) differs only in rounding, far below that."""
import math

import numpy as np
import pytest
import torch

from oracle import jz_oracle as O
from paper_2003_08746_gb300 import workloads as W
from parity import oracle_grid

pytestmark = pytest.mark.gpu

TOL = 1e-11


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
    return g, W.jet_state(g) + noise, W.jet_params(seed=2)


def test_flow_stats_vs_oracle(jz):
    """A sample after every second step over 12 steps (6 samples), FP64 form."""
    g, q, prm = _jet()
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm)
    s.set_state(q, 0.0)
    s.stats_begin(2)
    s.step(12, stats=False)
    mean, rms, n = s.stats_read()
    assert n == 6
    og, oc = oracle_grid(g), O.Consts(prm)
    Q, t = torch.from_numpy(q), torch.zeros((), dtype=torch.float64)
    samples = []
    for step in range(1, 13):
        Q, dt, _ = O.rk_step(og, Q, oc, t)
        t = t + dt
        if step % 2 == 0:
            samples.append(Q)
    om, orms = O.flow_statistics(samples)
    assert np.abs(mean - om.numpy()).max() <= TOL
    assert np.abs(rms - orms.numpy()).max() <= TOL
    assert orms.max().item() > 1e-6                 # the check is not vacuous
    # stations and potential core through the library's host helpers vs the oracle's
    x = g.xyz[0, 0, 0, :]
    for x0 in (2.5, 5.0):
        prof = jz.jz_station_profile(mean, x, x0)
        assert np.abs(prof - O.station_profile(om, x, x0).numpy()).max() <= TOL
    xc = jz.jz_potential_core(mean[0], x, prm.jet_mach)
    xo = O.potential_core_length(om[0], x, prm.jet_mach)
    assert (xc is None) == (xo is None)
    if xc is not None:
        assert abs(xc - xo) <= 1e-9


def test_single_sample_exact(jz):
    """One sample: the mean is the azimuthal average of u_x of the state and the rms is 0."""
    g, q, prm = _jet()
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    s.set_state(q, 0.0)
    s.step(3, stats=False)
    s.stats_begin(0)
    s.stats_sample()
    mean, rms, n = s.stats_read()
    Q = s.get_state()
    assert n == 1 and np.all(rms == 0.0)
    # u_x by the library's reciprocal (about 1 ulp) and summed in another order: a few ulp of U_j
    assert np.abs(mean - (Q[1] / Q[0]).mean(axis=0)).max() <= 1e-14
    # restart: begin again clears the accumulators
    s.stats_begin(1)
    s.step(2, stats=False)
    assert s.stats_read()[2] == 2
    s.stats_end()
    with pytest.raises(jz.JzError):
        s.stats_read()


def test_flow_stats_full_size_sampled(jz):
    """Jet 1000 x 400 x 500, FP32-flux form, 3 samples (one per step): mean and rms on 64
    sampled (i, j) lines equal the same statistics formed by torch from the three states."""
    g, q, prm = W.make_workload("jet1000x400x500")
    grid = jz.Grid.from_workload(g)
    s = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    qd = torch.from_numpy(q).cuda()
    del q
    s.set_state(qd, 0.0)
    s.stats_begin(1)
    rng = np.random.Generator(np.random.PCG64(11))
    ii = rng.integers(0, g.ni, 64)
    jj = rng.integers(0, g.nj, 64)
    us = []
    for _ in range(3):
        s.step(1, stats=False)
        s.get_state(qd)
        us.append((qd[1][:, jj, ii] / qd[0][:, jj, ii]).cpu().numpy())   # [nk][64]
    U = np.stack(us)
    m = U.mean(axis=0)
    r = np.sqrt(((U - m) ** 2).mean(axis=0))
    mean = torch.empty((g.nj, g.ni), dtype=torch.float64, device="cuda")
    rms = torch.empty_like(mean)
    assert jz.jz_stats_read(s.h, mean, rms) == 3
    torch.cuda.synchronize()
    assert np.abs(mean.cpu().numpy()[jj, ii] - m.mean(axis=0)).max() <= 1e-13
    assert np.abs(rms.cpu().numpy()[jj, ii] - r.mean(axis=0)).max() <= 1e-12
    s.close()
    grid.close()
