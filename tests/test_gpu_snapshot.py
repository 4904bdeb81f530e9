"""Snapshots (checkpoint / restart): continuing from jz_load_snapshot reproduces an
uninterrupted run bit for bit, in both precision forms; mismatched or damaged files are
rejected with an error, not loaded."""
import numpy as np
import pytest
import torch

from paper_2003_08746_gb300 import workloads as W

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
    return g, W.jet_state(g) + noise, W.jet_params(seed=2)


@pytest.mark.parametrize("prec_name", ["JZ_PREC_FP64", "JZ_PREC_FP32FLUX"])
def test_restart_is_bit_exact(jz, tmp_path, prec_name):
    prec = getattr(jz, prec_name)
    g, q, prm = _jet()
    grid = jz.Grid.from_workload(g)
    a = jz.Solver(grid, prm, prec)
    a.set_state(q, 0.0)
    a.step(3, stats=False)
    path = tmp_path / "snap.bin"
    a.save(path)
    q_saved = a.get_state()
    st_a = a.step(4)
    qa = a.get_state()
    b = jz.Solver(grid, prm, prec)
    b.load(path)
    st_b = b.step(4)
    qb = b.get_state()
    assert np.array_equal(qa, qb)
    assert st_a.t == st_b.t and st_a.dt == st_b.dt and st_a.steps == st_b.steps == 7
    assert st_a.totals[:] == st_b.totals[:]
    head, qf = jz.read_snapshot(path)
    assert np.array_equal(qf, q_saved)
    assert (head["ni"], head["nj"], head["nk"], head["topology"]) == (g.ni, g.nj, g.nk, g.topology)
    assert head["steps"] == 3 and head["precision"] == prec
    # the FP32-flux form's stage 5 leaves the next step's CFL rate (stored); the FP64 form
    # reduces it in the next step's first stage, so nothing is stored
    assert head["flags"] == (1 if prec == jz.JZ_PREC_FP32FLUX else 0)


def test_cross_precision_load(jz, tmp_path):
    """An FP64 snapshot continues in the FP32-flux form (the CFL rate is reduced afresh)."""
    g, q, prm = _jet()
    grid = jz.Grid.from_workload(g)
    a = jz.Solver(grid, prm, jz.JZ_PREC_FP64)
    a.set_state(q, 0.0)
    a.step(2, stats=False)
    a.save(tmp_path / "s.bin")
    b = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    b.load(tmp_path / "s.bin")
    c = jz.Solver(grid, prm, jz.JZ_PREC_FP32FLUX)
    c.set_state(a.get_state(), a.step(0).t)
    sb, sc = b.step(3), c.step(3)
    assert np.array_equal(b.get_state(), c.get_state()) and sb.t == sc.t


def test_rejects_mismatch_and_damage(jz, tmp_path):
    g, q, prm = _jet()
    grid = jz.Grid.from_workload(g)
    a = jz.Solver(grid, prm)
    a.set_state(q, 0.0)
    a.step(1, stats=False)
    path = tmp_path / "s.bin"
    a.save(path)
    raw = path.read_bytes()
    # other grid shape
    g2 = W.jet_grid(72, 34, 16)
    other = jz.Solver(jz.Grid.from_workload(g2), prm)
    with pytest.raises(jz.JzError, match="does not match"):
        other.load(path)
    # other parameters
    other = jz.Solver(grid, W.jet_params(seed=2, C_s=0.1))
    with pytest.raises(jz.JzError, match="different parameters"):
        other.load(path)
    b = jz.Solver(grid, prm)
    # one flipped data byte
    bad = bytearray(raw)
    bad[jz.SNAPSHOT_HEADER_BYTES + 12345] ^= 0x10
    (tmp_path / "bad.bin").write_bytes(bytes(bad))
    with pytest.raises(jz.JzError, match="hash mismatch"):
        b.load(tmp_path / "bad.bin")
    # truncated, not a snapshot, missing
    (tmp_path / "short.bin").write_bytes(raw[:-8])
    with pytest.raises(jz.JzError, match="short file"):
        b.load(tmp_path / "short.bin")
    (tmp_path / "junk.bin").write_bytes(b"x" * 400)
    with pytest.raises(jz.JzError, match="not a version-1 snapshot"):
        b.load(tmp_path / "junk.bin")
    with pytest.raises(jz.JzError, match="cannot open"):
        b.load(tmp_path / "missing.bin")
    # the solver that refused the damaged files still loads the good one
    b.load(path)
    assert np.array_equal(b.get_state(), a.get_state())
