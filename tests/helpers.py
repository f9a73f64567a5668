"""Shared helpers of the GPU parity tests."""
import numpy as np

import oracle


def parity_tol(m, k, i, j, tol_cfg, pad_last=False):
    """The acceptance bound: max(fixed tolerance, 10 x the method's own
    sensitivity to rounding order, measured by the oracle)."""
    floor = oracle.sensitivity_floor(m, k, i, j, pad_last=pad_last)
    return max(tol_cfg, 10.0 * floor), floor


def oracle_block(m, k, i, j, pad_last=False):
    ref, st, _ = oracle.bri_block(m, k, i, j, memo=True, pad_last=pad_last)
    assert st == oracle.OK
    return ref


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)
