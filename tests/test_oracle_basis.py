"""Pins for the oracle's basis, quadrature and Euler flux (closed forms)."""
import os

import numpy as np
import pytest

from oracle import basis as B
from oracle import euler as E

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_gauss_exact_to_degree_2N_minus_1(N):
    x, w = B.gauss(N)
    for k in range(2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    k = 2 * N  # first degree the rule cannot integrate
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


def test_legendre_closed_forms():
    x = np.linspace(-1, 1, 17)
    assert np.allclose(B.legendre(0, x), 1)
    assert np.allclose(B.legendre(1, x), x)
    assert np.allclose(B.legendre(2, x), (3 * x ** 2 - 1) / 2, atol=1e-15)
    assert np.allclose(B.legendre(3, x), (5 * x ** 3 - 3 * x) / 2, atol=1e-15)
    assert np.allclose(B.legendre_deriv(2, x), 3 * x, atol=1e-15)
    assert np.allclose(B.legendre_deriv(3, x), (15 * x ** 2 - 3) / 2, atol=1e-14)
    for k in range(6):
        assert B.legendre(k, np.array([1.0]))[0] == pytest.approx(1.0)
        assert B.legendre(k, np.array([-1.0]))[0] == pytest.approx((-1.0) ** k)


def test_legendre_orthogonality():
    x, w = B.gauss(10)
    for k in range(5):
        for l in range(5):
            v = np.sum(w * B.legendre(k, x) * B.legendre(l, x))
            assert abs(v - (2.0 / (2 * k + 1) if k == l else 0.0)) < 1e-14


def test_tensor_mode_order():
    pts = np.array([[0.3, -0.7], [0.9, 0.2]])
    Phi = B.eval_basis(pts, 3)
    # m = k_x + 3 k_y: m=1 -> P1(x), m=3 -> P1(y), m=5 -> P2(x) P1(y)
    assert np.allclose(Phi[:, 1], pts[:, 0])
    assert np.allclose(Phi[:, 3], pts[:, 1])
    assert np.allclose(Phi[:, 5], (3 * pts[:, 0] ** 2 - 1) / 2 * pts[:, 1])
    G = B.eval_basis_grad(pts, 3)
    assert np.allclose(G[:, 5, 0], 3 * pts[:, 0] * pts[:, 1])
    assert np.allclose(G[:, 5, 1], (3 * pts[:, 0] ** 2 - 1) / 2)


def _golden_flux():
    rows = {}
    for line in open(os.path.join(GOLD, "euler_flux.txt")):
        if line.startswith("#") or not line.strip():
            continue
        dim, name, *vals = line.split()
        rows[(dim, name)] = np.array([float(v) for v in vals])
    return rows


@pytest.mark.parametrize("d", [2, 3])
def test_euler_flux_golden(d):
    g = _golden_flux()
    U = g[(f"{d}d", "U")]
    F = E.physical_flux(U[None])[0]
    for j in range(d):
        assert np.allclose(F[:, j], g[(f"{d}d", f"F{j + 1}")], rtol=0, atol=1e-14)


def test_lax_friedrichs_consistency_and_antisymmetry():
    rng = np.random.default_rng(1)
    for d in (2, 3):
        nv = d + 2
        U = np.zeros((20, nv))
        U[:, 0] = 1 + 0.2 * rng.random(20)
        U[:, 1:1 + d] = 0.3 * rng.standard_normal((20, d))
        U[:, -1] = 3 + rng.random(20)
        V = U.copy()
        V[:, 0] += 0.1
        V[:, -1] += 0.3
        n = rng.standard_normal((20, d))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        F = np.einsum("pvj,pj->pv", E.physical_flux(U), n)
        assert np.allclose(E.lax_friedrichs(U, U, n), F, atol=1e-14)
        assert np.allclose(E.lax_friedrichs(U, V, n), -E.lax_friedrichs(V, U, -n), atol=1e-14)
        # dissipative sign (reading R3): for a jump in density only, at rest,
        # the LF mass flux carries mass from the denser side
        W = U.copy()
        W[:, 1:1 + d] = 0
        Z = W.copy()
        Z[:, 0] += 0.5
        Z[:, -1] = W[:, -1]
        assert np.all(E.lax_friedrichs(Z, W, n)[:, 0] > 0)
