"""Legendre modal bases and Gauss--Legendre rules on the reference cell.

The DG space V_h of Sec. 2.1 holds, on each cell K, polynomials of degree <= k
(P^k) or of degree <= k in each variable (Q^k).  The modal basis on the
reference cell [-1, 1]^d is the tensor product of Legendre polynomials
P_i(xi) P_j(eta).  Gauss rules come from numpy's ``leggauss``; Legendre values
and derivatives from ``numpy.polynomial.legendre``.  Test infrastructure only.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(n):
    """n-point Gauss--Legendre rule on [-1, 1]: (nodes, weights)."""
    return npleg.leggauss(n)


def leg(i, x):
    """Legendre polynomial P_i evaluated at x (P_i(1) = 1)."""
    c = np.zeros(i + 1)
    c[i] = 1.0
    return npleg.legval(np.asarray(x, dtype=np.float64), c)


def dleg(i, x):
    """Derivative P_i'(x)."""
    c = np.zeros(i + 1)
    c[i] = 1.0
    return npleg.legval(np.asarray(x, dtype=np.float64), npleg.legder(c))


def modes_1d(k):
    """Mode list of the 1D space P^k: [0, 1, ..., k]."""
    return list(range(k + 1))


def modes_2d(k, basis):
    """Mode list [(i, j), ...] of P^k (i + j <= k) or Q^k (i, j <= k).

    Ordering (an interface shared with the CUDA library's state layout):
    by total degree d = i + j ascending, and inside one degree by i
    descending.  P^k is therefore a prefix of Q^k, and modes 0, 1, 2 are
    always (0,0), (1,0), (0,1).
    """
    out = []
    dmax = k if basis == "P" else 2 * k
    for d in range(dmax + 1):
        for i in range(d, -1, -1):
            j = d - i
            if i <= k and j <= k:
                out.append((i, j))
    return out


def mass_1d(k):
    """Diagonal of the 1D mass matrix on the reference cell divided by |K|:
    (1/|K|) int_K P_i^2 = 1/(2i+1)."""
    return np.array([1.0 / (2 * i + 1) for i in range(k + 1)])


def mass_2d(modes):
    """(1/|K|) int_K (P_i P_j)^2 = 1/((2i+1)(2j+1)) for each mode."""
    return np.array([1.0 / ((2 * i + 1) * (2 * j + 1)) for (i, j) in modes])


class Basis1D:
    """Tables of the 1D P^k basis at the n-point Gauss rule and at xi = +-1."""

    def __init__(self, k, nq=None):
        self.k = k
        self.nm = k + 1
        self.nq = k + 1 if nq is None else nq
        self.xq, self.wq = gauss(self.nq)
        # phi[q, m] = P_m(xi_q),  dphi[q, m] = P_m'(xi_q)
        self.phi = np.stack([leg(m, self.xq) for m in range(self.nm)], axis=1)
        self.dphi = np.stack([dleg(m, self.xq) for m in range(self.nm)], axis=1)
        self.phi_r = np.array([leg(m, 1.0) for m in range(self.nm)])
        self.phi_l = np.array([leg(m, -1.0) for m in range(self.nm)])
        self.mass = mass_1d(k)


class Basis2D:
    """Tables of the 2D P^k / Q^k basis on [-1,1]^2.

    Volume points are the tensor Gauss rule (q = a * nq + b for xi_a, eta_b);
    each face carries the nq-point Gauss rule of its edge.
    """

    def __init__(self, k, basis, nq=None):
        self.k = k
        self.basis = basis
        self.modes = modes_2d(k, basis)
        self.nm = len(self.modes)
        self.nq = k + 1 if nq is None else nq
        x, w = gauss(self.nq)
        self.x1, self.w1 = x, w
        xi = np.repeat(x, self.nq)      # q = a*nq + b  ->  xi_a
        eta = np.tile(x, self.nq)       #               ->  eta_b
        self.xi, self.eta = xi, eta
        self.wvol = np.repeat(w, self.nq) * np.tile(w, self.nq)
        self.phi_vol = np.stack([leg(i, xi) * leg(j, eta) for (i, j) in self.modes], axis=1)
        self.dxi_vol = np.stack([dleg(i, xi) * leg(j, eta) for (i, j) in self.modes], axis=1)
        self.deta_vol = np.stack([leg(i, xi) * dleg(j, eta) for (i, j) in self.modes], axis=1)
        one = np.ones_like(x)
        # face tables [p, m]: E at xi=+1, W at xi=-1, N at eta=+1, S at eta=-1
        self.phi_face = {
            "E": np.stack([leg(i, one) * leg(j, x) for (i, j) in self.modes], axis=1),
            "W": np.stack([leg(i, -one) * leg(j, x) for (i, j) in self.modes], axis=1),
            "N": np.stack([leg(i, x) * leg(j, one) for (i, j) in self.modes], axis=1),
            "S": np.stack([leg(i, x) * leg(j, -one) for (i, j) in self.modes], axis=1),
        }
        self.mass = mass_2d(self.modes)
