"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (one sweep from an identical state, same alpha):
  FP32 storage: 1e-5 rad; FP16 storage: 2e-3 rad against the oracle's
  binary16-storage mode. Near-ties -- an angular difference within 2^-20 turn
  of 0 or 1/2, or a phase within 2^-20 turn of a DWT window edge, where an
  FP32 and an FP64 evaluation may legitimately branch differently -- may take
  either branch: the oracle is re-run with each combination of branches for
  those items and the closest is kept. They must stay below 0.1% of edges.
"""
import itertools
import math

import numpy as np

TIE_EPS = 2.0 ** -20
TOL_F32 = 1e-5
TOL_F16 = 2e-3
# bfloat16 storage cannot meet 2e-3 rad (its quantum is 2^-9 turn = 1.2e-2 rad
# near 1/2); against the oracle's bfloat16-storage mode the bound is one
# quantum (a binary32-vs-FP64 difference can move a rounding by one step)
TOL_BF16 = 2 * math.pi * 2 ** -9 * 1.05


def circ_rad(a, b):
    d = np.mod(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64), 1.0)
    return 2 * math.pi * np.minimum(d, 1.0 - d)


def one_sweep_error(orc, g, x0, x_gpu, alpha, sweep, *, storage=0, max_enum=10, **kw):
    """Max circular error (rad) of one GPU sweep against the oracle, allowing
    either branch at near-ties. Returns (error, n_ties)."""
    x_or, ties = orc.sweep(g, x0, alpha, sweep, storage=storage, tie_eps=TIE_EPS, **kw)
    err = float(circ_rad(x_or, x_gpu).max())
    if len(ties) == 0:
        return err, 0
    ties = ties[:max_enum]
    best = err
    nforce = g.m + g.n * (2 if kw.get("h") is not None else 1)
    for signs in itertools.product((1, -1), repeat=len(ties)):
        force = np.zeros(nforce, dtype=np.int8)
        force[ties] = signs
        xf, _ = orc.sweep(g, x0, alpha, sweep, storage=storage, force=force, **kw)
        best = min(best, float(circ_rad(xf, x_gpu).max()))
    return best, len(ties)


def bf16_exact_turns(x):
    """Round turns to bfloat16 in the representation [-1/2, 1/2), back to [0,1)."""
    import torch
    x = np.asarray(x, dtype=np.float64)
    g = np.where(x >= 0.5, x - 1.0, x)
    g = torch.tensor(g).to(torch.bfloat16).to(torch.float64).numpy()
    return np.mod(np.where(g < 0, g + 1.0, g), 1.0)


def f16_exact_turns(x):
    """Round turns to binary16 in the representation [-1/2, 1/2), back to [0,1)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.where(x >= 0.5, x - 1.0, x).astype(np.float16).astype(np.float64)
    return np.mod(np.where(g < 0, g + 1.0, g), 1.0)
