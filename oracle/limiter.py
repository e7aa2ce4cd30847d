"""Positivity-preserving scaling limiter (oracle; test infrastructure).

The paper names limiters for its cylinder case (Sec. 6) without details;
reading R17 takes the scaling limiter of Zhang & Shu (J. Comput. Phys. 229,
2010) applied to every cell after every Runge-Kutta stage:

  * the cell mean u_bar is the J-weighted average sum_q w_q J_q u_q /
    sum_q w_q J_q over the volume Gauss points (the limiter keeps it);
  * the check points are the volume Gauss points and the Gauss points of the
    2d faces (the values the face fluxes see);
  * eps_rho = eps * rho_bar, eps_p = eps * p(u_bar);
  * density: theta_1 = min(1, (rho_bar - eps_rho) / (rho_bar - min rho)),
    u~ = u_bar + theta_1 (u - u_bar);
  * pressure: at every check point with p(u~) < eps_p, t solves
    p(u_bar + t (u~ - u_bar)) = eps_p in [0, 1] (a quadratic in t, since
    rho p / (gamma - 1) = E rho - |m|^2 / 2); theta_2 = min of those t (1 if
    none); the limited polynomial is u_bar + theta_2 (u~ - u_bar).

A cell whose mean itself has rho_bar <= 0 or p(u_bar) <= 0 is left alone
and reported.
"""
from __future__ import annotations

import numpy as np

from . import basis as B
from .euler import primitives


def _pressure_root(ubar, du, eps_p, gamma):
    """Smallest t in [0, 1] with p(ubar + t du) = eps_p (du = u~ - ubar at one
    point, where p(ubar + du) < eps_p <= p(ubar))."""
    d = len(ubar) - 2
    g1 = gamma - 1.0
    rb, mb, Eb = ubar[0], ubar[1:1 + d], ubar[d + 1] - eps_p / g1
    dr, dm, dE = du[0], du[1:1 + d], du[d + 1]
    # f(t) = (E(t) - eps_p/(gamma-1)) rho(t) - |m(t)|^2 / 2 = a t^2 + b t + c
    a = dE * dr - 0.5 * float(dm @ dm)
    b = Eb * dr + dE * rb - float(mb @ dm)
    c = Eb * rb - 0.5 * float(mb @ mb)
    if abs(a) < 1e-300:
        return min(1.0, max(0.0, -c / b))
    disc = max(b * b - 4.0 * a * c, 0.0)
    roots = [(-b - np.sqrt(disc)) / (2.0 * a), (-b + np.sqrt(disc)) / (2.0 * a)]
    inside = [t for t in roots if 0.0 <= t <= 1.0]
    return min(inside) if inside else 0.0


def positivity_limit(S, U, eps, gamma=None):
    """Returns (limited state, number of cells changed, number of cells with
    an inadmissible mean)."""
    gamma = S.gamma if gamma is None else gamma
    ops, d, nv = S.ops, S.d, S.nv
    # check points: volume Gauss points, then each face's Gauss points
    pts = [ops.Phi] + [ops.faces[f][2] for f in range(2 * d)]
    Pchk = np.concatenate(pts, axis=0)                       # (P, M)
    out = U.copy()
    changed = bad = 0
    for li in range(len(S.leaves)):
        J, _ = S.geo_vol[li]
        for c in range(U.shape[3]):
            K = U[li, :, :, c]                               # (nv, M)
            wj = ops.wq * J[c]
            uq = ops.Phi @ K.T                               # (Q, nv)
            ubar = (wj @ uq) / wj.sum()
            rb, _, pb = primitives(ubar[None], gamma)
            if not (rb[0] > 0 and pb[0] > 0):
                bad += 1
                continue
            eps_r, eps_p = eps * rb[0], eps * pb[0]
            vals = Pchk @ K.T                                # (P, nv)
            rmin = vals[:, 0].min()
            th1 = 1.0 if rmin >= eps_r else min(1.0, (rb[0] - eps_r) / (rb[0] - rmin))
            vt = ubar + th1 * (vals - ubar)
            _, _, p = primitives(vt, gamma)
            th2 = 1.0
            for k in np.nonzero(p < eps_p)[0]:
                th2 = min(th2, _pressure_root(ubar, vt[k] - ubar, eps_p, gamma))
            theta = th1 * th2
            if theta < 1.0:
                changed += 1
                # nodal-free form: the mean is mode 0's J-weighted value; scale
                # the polynomial about the constant ubar
                Kbar = np.zeros_like(K)
                Kbar[:, 0] = ubar                            # P_0 = 1
                out[li, :, :, c] = Kbar + theta * (K - Kbar)
    return out, changed, bad


__all__ = ["positivity_limit"]
