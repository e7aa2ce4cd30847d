"""Refinement indicator and one adaptation step (oracle; test infrastructure).

The paper refines and coarsens blocks by cell-average thresholds (Sec. 5,
its convection test) and for the cylinder by divergence/curl (Sec. 6) without
giving a formula; reading R16 fixes one:

  * per cell, g = 2 |(K_{e_1}, ..., K_{e_d})| / K_0 for the density, where
    K_0 is the mean mode and K_{e_a} the mode of degree one along axis a
    (P_1(xi) = xi), i.e. h |grad rho| / rho_mean on a cube cell of edge h;
    the block's indicator is the largest g over its cells;
  * a leaf is refined if its indicator exceeds refine_above and its level is
    below max_level; the 2:1 closure may refine more;
  * then, visiting the leaves in canonical order, a parent whose 2^d
    children are all leaves (after the refinement) with indicators below
    coarsen_below is coarsened when its first child (all position bits
    even) is met, unless that would break 2:1 face balance;
  * the state follows by copy, split (Eqs. (11)-(12)) or combine
    (Eqs. (13)-(14)), Sec. 3.4.
"""
from __future__ import annotations

import copy

import numpy as np

from . import basis as B
from .dg import Solver
from .forest import BalanceError


def indicator(S, U):
    """Largest g over each leaf's cells (rho = variable 0)."""
    d, N = S.d, S.ops.N
    modes = B.mode_indices(d, N)
    lin = [m for m, k in enumerate(modes) if sum(k) == 1]   # e_a, axis order
    lin.sort(key=lambda m: [a for a in range(d) if modes[m][a] == 1][0])
    out = np.zeros(len(S.leaves))
    for li in range(len(S.leaves)):
        K0 = U[li, 0, 0, :]
        if N == 1:
            continue  # no degree-one modes: the indicator is 0
        grad = np.sqrt(np.sum(U[li, 0, lin, :] ** 2, axis=0))
        out[li] = np.max(2.0 * grad / K0)
    return out


def adapt(S, U, refine_above, coarsen_below, max_level, g=None):
    """One adaptation; returns (new solver, new state, blocks refined by the
    flags, parents coarsened).  g: per-leaf indicator (default indicator(S, U));
    U may be None for a topology-only step (the state returned is then None)."""
    if g is None:
        g = indicator(S, U)
    F = copy.deepcopy(S.F)
    flagged = [k for i, k in enumerate(S.leaves) if g[i] > refine_above and k[1] < max_level]
    if flagged:
        F.refine(flagged)
    low = {k for i, k in enumerate(S.leaves) if g[i] < coarsen_below}
    d = S.d
    n_coarse = 0
    for key in list(F.leaves()):
        r, lev, pos = key
        if lev <= 1 or any(x & 1 for x in pos):
            continue
        if not F.is_leaf(key):
            continue  # coarsened already with an earlier sibling
        parent = (r, lev - 1, tuple(x >> 1 for x in pos))
        kids = [(r, lev, tuple(2 * parent[2][a] + b[a] for a in range(d)))
                for b in B.all_corner_bits(d)]
        if not all(F.tree.get(k) is True and k in low for k in kids):
            continue
        try:
            F.coarsen([parent])
            n_coarse += 1
        except BalanceError:
            pass
    S2 = Solver(F, S.p, gamma=S.gamma, cfl=S.cfl, nonconforming=S.nonconforming, limiter=S.limiter,
                boundary=S.boundary)
    return S2, None if U is None else S2.regrid_state(S, U), len(flagged), n_coarse


__all__ = ["indicator", "adapt"]
