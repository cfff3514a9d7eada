"""Pins of oracle.basis: Gauss exactness, Legendre closed forms, mode sets."""
import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss(n)
    for d in range(2 * n):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    # and not beyond: degree 2n is not integrated exactly
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


def test_legendre_closed_forms():
    x = np.linspace(-1, 1, 7)
    assert np.allclose(basis.leg(0, x), 1)
    assert np.allclose(basis.leg(1, x), x)
    assert np.allclose(basis.leg(2, x), 0.5 * (3 * x ** 2 - 1))
    assert np.allclose(basis.leg(3, x), 0.5 * (5 * x ** 3 - 3 * x))
    assert np.allclose(basis.dleg(3, x), 0.5 * (15 * x ** 2 - 3))
    for i in range(5):
        assert basis.leg(i, 1.0) == pytest.approx(1.0)
        assert basis.leg(i, -1.0) == pytest.approx((-1.0) ** i)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_mode_sets(k):
    P = basis.modes_2d(k, "P")
    Q = basis.modes_2d(k, "Q")
    assert len(P) == (k + 1) * (k + 2) // 2
    assert len(Q) == (k + 1) ** 2
    assert Q[: len(P)] == P
    assert all(i + j <= k for (i, j) in P)
    if k >= 1:
        assert P[:3] == [(0, 0), (1, 0), (0, 1)]


@pytest.mark.parametrize("k,b", [(1, "P"), (2, "P"), (2, "Q"), (3, "Q")])
def test_mass_matrix_is_diagonal(k, b):
    B = basis.Basis2D(k, b, nq=k + 2)
    M = 0.25 * np.einsum("q,qm,qn->mn", B.wvol, B.phi_vol, B.phi_vol)
    assert np.allclose(M, np.diag(B.mass), atol=1e-14)
