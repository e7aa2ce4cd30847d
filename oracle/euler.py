"""Compressible Euler flux and Lax-Friedrichs numerical flux (oracle; test infrastructure).

Eq. (2) gives U = (rho, rho u, rho v, E) and the fluxes F_1, F_2 in 2D; the
3D system adds rho w and F_3 in the same pattern.  Eq. (23) closes it with
p = rho e (gamma - 1), so p = (gamma - 1)(E - rho |u|^2 / 2).
Eq. (5) is the Lax-Friedrichs flux; see reading R3 in ``oracle/__init__``.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def primitives(U, gamma=GAMMA):
    """U[..., nv] -> (rho, vel[..., d], p)."""
    d = U.shape[-1] - 2
    rho = U[..., 0]
    vel = U[..., 1:1 + d] / rho[..., None]
    E = U[..., d + 1]
    p = (gamma - 1.0) * (E - 0.5 * rho * np.sum(vel * vel, axis=-1))
    return rho, vel, p


def physical_flux(U, gamma=GAMMA):
    """F[..., nv, d]: column j is the flux F_j of Eq. (2) (extended to 3D)."""
    d = U.shape[-1] - 2
    rho, vel, p = primitives(U, gamma)
    E = U[..., d + 1]
    F = np.zeros(U.shape + (d,))
    for j in range(d):
        F[..., 0, j] = rho * vel[..., j]
        for a in range(d):
            F[..., 1 + a, j] = rho * vel[..., a] * vel[..., j] + (p if a == j else 0.0)
        F[..., d + 1, j] = vel[..., j] * (E + p)
    return F


def sound_speed(U, gamma=GAMMA):
    rho, _, p = primitives(U, gamma)
    return np.sqrt(gamma * p / rho)


def lax_friedrichs(UL, UR, n, gamma=GAMMA):
    """Eq. (5) with reading R3.

    UL, UR: [..., nv]; n: [..., d] unit normal pointing from L to R.
    F = 1/2 [ (F(UL) + F(UR)) . n + alpha (UL - UR) ],
    alpha = max(|u_L.n| + c_L, |u_R.n| + c_R) (the largest absolute
    eigenvalue of the normal flux Jacobian on either side).
    """
    FL = np.einsum("...vj,...j->...v", physical_flux(UL, gamma), n)
    FR = np.einsum("...vj,...j->...v", physical_flux(UR, gamma), n)
    _, vL, _ = primitives(UL, gamma)
    _, vR, _ = primitives(UR, gamma)
    aL = np.abs(np.sum(vL * n, axis=-1)) + sound_speed(UL, gamma)
    aR = np.abs(np.sum(vR * n, axis=-1)) + sound_speed(UR, gamma)
    alpha = np.maximum(aL, aR)
    return 0.5 * (FL + FR + alpha[..., None] * (UL - UR))
