"""Shared helpers of the parity tests (comparison metrics, oracle/GPU set-up)."""
import numpy as np
import torch

from oracle import jz_oracle as O


def field_errors(got, ref):
    """Per-field relative L2 and max-abs errors, as arrays of 5.

    Mass and energy are normalised by their own norm; the three momentum
    components by the largest momentum-component norm (zero-mean or tiny
    components are measured against the momentum scale).
    """
    got, ref = np.asarray(got), np.asarray(ref)
    l2 = np.array([np.linalg.norm(ref[m]) for m in range(5)])
    mx = np.array([np.abs(ref[m]).max() for m in range(5)])
    den_l2 = l2.copy()
    den_mx = mx.copy()
    den_l2[1:4] = l2[1:4].max()
    den_mx[1:4] = mx[1:4].max()
    den_l2 = np.where(den_l2 > 0, den_l2, 1.0)
    den_mx = np.where(den_mx > 0, den_mx, 1.0)
    e2 = np.array([np.linalg.norm(got[m] - ref[m]) for m in range(5)]) / den_l2
    em = np.array([np.abs(got[m] - ref[m]).max() for m in range(5)]) / den_mx
    return e2, em


def oracle_grid(g):
    return O.Grid(g.ni, g.nj, g.nk, g.xyz, g.topology, g.period)
