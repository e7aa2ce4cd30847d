"""Tensor Legendre basis and Gauss-Legendre quadrature (oracle; test infrastructure).

Sec. 2 (after Eq. 3) takes phi_i from a complete polynomial space; the reading
used here is the tensor space Q^p with unnormalised Legendre polynomials P_k
per axis (mode index m = sum_a k_a N^a, N = p + 1, x fastest).
"""
from __future__ import annotations

import itertools

import numpy as np


def legendre(k, x):
    """P_k(x) by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, float)
    p0 = np.ones_like(x)
    if k == 0:
        return p0
    p1 = x.copy()
    for j in range(1, k):
        p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
    return p1


def legendre_deriv(k, x):
    """P_k'(x) from P'_{j+1} = P'_{j-1} + (2j+1) P_j."""
    x = np.asarray(x, float)
    d = [np.zeros_like(x), np.ones_like(x)]
    if k < 2:
        return d[k]
    for j in range(1, k):
        d.append(d[j - 1] + (2 * j + 1) * legendre(j, x))
    return d[k]


def gauss(N):
    """N-point Gauss-Legendre nodes and weights on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(N)
    return x, w


def mode_indices(d, N):
    """List of multi-indices k (tuple over axes), ordered by m = sum k_a N^a."""
    return [tuple((m // N ** a) % N for a in range(d)) for m in range(N ** d)]


def tensor_points(d, N):
    """Volume Gauss points (Q x d) and weights (Q), q = sum q_a N^a."""
    x, w = gauss(N)
    pts = np.zeros((N ** d, d))
    wts = np.ones(N ** d)
    for q in range(N ** d):
        for a in range(d):
            qa = (q // N ** a) % N
            pts[q, a] = x[qa]
            wts[q] *= w[qa]
    return pts, wts


def face_points(d, N, axis, side):
    """Gauss points on face (axis, side) of [-1,1]^d.

    Returns reference points (N^(d-1) x d) with xi_axis = -1 (side 0) or +1
    (side 1), and the (d-1)-dimensional weights.  Face point index is
    sum_j q_{t_j} N^j over the tangential axes t_j in increasing order.
    """
    x, w = gauss(N)
    tang = [a for a in range(d) if a != axis]
    nf = N ** (d - 1)
    pts = np.zeros((nf, d))
    wts = np.ones(nf)
    for f in range(nf):
        for j, t in enumerate(tang):
            qj = (f // N ** j) % N
            pts[f, t] = x[qj]
            wts[f] *= w[qj]
        pts[f, axis] = 1.0 if side else -1.0
    return pts, wts


def eval_basis(points, N):
    """Phi[i, m] = prod_a P_{k_a}(xi_a) at arbitrary reference points."""
    points = np.atleast_2d(points)
    d = points.shape[1]
    P = [[legendre(k, points[:, a]) for k in range(N)] for a in range(d)]
    out = np.ones((points.shape[0], N ** d))
    for m, k in enumerate(mode_indices(d, N)):
        for a in range(d):
            out[:, m] *= P[a][k[a]]
    return out


def eval_basis_grad(points, N):
    """dPhi[i, m, a] = d phi_m / d xi_a at arbitrary reference points."""
    points = np.atleast_2d(points)
    d = points.shape[1]
    P = [[legendre(k, points[:, a]) for k in range(N)] for a in range(d)]
    dP = [[legendre_deriv(k, points[:, a]) for k in range(N)] for a in range(d)]
    out = np.ones((points.shape[0], N ** d, d))
    for m, k in enumerate(mode_indices(d, N)):
        for g in range(d):
            for a in range(d):
                out[:, m, g] *= dP[a][k[a]] if a == g else P[a][k[a]]
    return out


def all_corner_bits(d):
    return [tuple((c >> a) & 1 for a in range(d)) for c in range(2 ** d)]


def lattice(d, n):
    """Cell multi-indices of an n^d block, x fastest."""
    return [tuple((c // n ** a) % n for a in range(d)) for c in range(n ** d)]


__all__ = ["legendre", "legendre_deriv", "gauss", "mode_indices", "tensor_points",
           "face_points", "eval_basis", "eval_basis_grad", "all_corner_bits",
           "lattice", "itertools"]
