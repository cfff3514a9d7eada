"""Linear stability: maximum CFL numbers of Table 1.1.

The paper's von Neumann analysis is omitted from its text; here the same
quantity is computed by brute force: for 1D linear advection u_t + u_x = 0
with the upwind flux on a periodic mesh of N cells, the one-step map of a
scheme is linear, so its matrix G(lambda) (lambda = dt/h) is assembled by
applying one step to every unit vector, and the maximum CFL number is the
largest lambda with spectral radius rho(G) <= 1 (bisection).  Test
infrastructure only.
"""
import numpy as np

from .dg1d import DG1D
from .physics import Advection


def step_matrix(k, N, lam, step):
    dg = DG1D(np.linspace(0.0, 1.0, N + 1), k, Advection([1.0]))
    h = 1.0 / N
    n = N * (k + 1)
    G = np.empty((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        G[:, col] = step(dg, e.reshape(N, 1, k + 1), 0.0, lam * h).reshape(-1)
    return G


def spectral_radius(k, N, lam, step):
    return np.max(np.abs(np.linalg.eigvals(step_matrix(k, N, lam, step))))


def max_cfl(k, step, N=32, lo=0.02, hi=0.6, tol=1e-4, growth=1e-10):
    """Largest lambda in [lo, hi] with rho(G(lambda)) <= 1 + growth."""
    assert spectral_radius(k, N, lo, step) <= 1 + growth
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if spectral_radius(k, N, mid, step) <= 1 + growth:
            lo = mid
        else:
            hi = mid
    return lo
