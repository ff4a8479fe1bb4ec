"""Helpers of the GPU parity tests.

Near-tie tolerances.  The oracle computes similarities in FP64; the kernels
compute squared distances in FP32.  A decision of the method (the expansion
test, a climb, the order of two list entries) can legitimately go the other
way on the GPU only when the oracle's relative margin for it is below what
FP32 rounding can move.  The bounds follow the kernels' summation order:

* row gathers (search, update, cross, re-score): a lane holds e = DP/G
  elements of a row.  FP32 and BF16 rows: four running sums of e/4 squared
  differences each (fused multiply-adds), added in two levels, then log2(G)
  butterfly steps; with the rounding of each difference the relative error
  of d2 is at most (e/4 + log2(G) + 4) u, u = 2^-24.  FP8 rows: one running
  sum of e products and the rounding of the scaled value,
  (e + log2(G) + 5) u.  A similarity 1/(1 + sqrt(d2)) adds about 3 u more,
  e (the expansion) is rounded to FP32 (u).  A comparison cannot flip when
  the margin exceeds eps_d2 + 8 u; the tests flag margins below twice that.
* the exact-graph kernel adds all DP products of a pair in order:
  eps_d2 <= (DP + 2) u, flagged below 2 (DP + 10) u.

Decisions with smaller margins are "ambiguous": they are counted and
reported, excluded from the bit-exact comparison, and bounded in number.
"""
from __future__ import annotations

import math

import numpy as np

U = 2.0 ** -24
DPS = (16, 32, 64, 96, 128, 256)


def padded(d: int) -> int:
    return next(dp for dp in DPS if d <= dp)


def _group(nc: int) -> int:
    return 8 if nc % 8 == 0 else 4 if nc % 4 == 0 else 2 if nc % 2 == 0 else 1


def gather_tol(d: int, storage: int = 0) -> float:
    dp = padded(d)
    e = {0: 4, 1: 8, 2: 16}[storage]
    nc = dp // e
    g = _group(nc)
    per_lane = dp // g
    if storage == 2:
        eps = (per_lane + math.log2(g) + 5) * U
    else:
        eps = (per_lane / 4 + math.log2(g) + 4) * U
    return 2.0 * (eps + 8 * U)


def exact_tol(d: int) -> float:
    return 2.0 * (padded(d) + 10) * U


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def cuda_tensor(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()
