"""Shared helpers of the GPU parity tests."""
import numpy as np

import oracle


def parity_tol(m, k, i, j, tol_cfg):
    """The acceptance bound: max(fixed tolerance, 10 x the method's own
    sensitivity to rounding order, measured by the oracle)."""
    floor = oracle.sensitivity_floor(m, k, i, j)
    return max(tol_cfg, 10.0 * floor), floor


def oracle_block(m, k, i, j):
    ref, st, _ = oracle.bri_block(m, k, i, j, memo=True)
    assert st == oracle.OK
    return ref


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)
