"""Exact solutions used to pin the oracle (Sec. 4.1).  Test infrastructure.

Every function returns conserved variables with the variable index last.
"""
import numpy as np

from .physics import Euler


def sine_advection(x, t, beta=1.0):
    """u = sin(x - beta t): Sec. 4.1.1 boundary-error example (Table 4.4)."""
    return np.sin(x - beta * t)[..., None]


def euler1d_sine(x, t, gamma=1.4):
    """rho = 1 + 0.2 sin(pi (x - t)), w = 1, p = 1 (Table 4.2)."""
    ph = Euler(gamma, 1)
    rho = 1.0 + 0.2 * np.sin(np.pi * (x - t))
    return ph.conserved(rho, [np.ones_like(x)], np.ones_like(x))


def euler2d_sine(X, Y, t, gamma=1.4, w=0.7, v=0.3):
    """rho = 1 + 0.2 sin(pi (x + y - (w + v) t)), (w, v) = (0.7, 0.3), p = 1
    (Table 4.5)."""
    ph = Euler(gamma, 2)
    rho = 1.0 + 0.2 * np.sin(np.pi * (X + Y - (w + v) * t))
    return ph.conserved(rho, [w + 0 * X, v + 0 * X], 1.0 + 0 * X)


def isentropic_vortex(X, Y, t, gamma=1.4, eps=5.0, xc=5.0, yc=5.0, mean=(1.0, 1.0),
                      period=None):
    """Isentropic vortex translated by the mean flow (not in the paper; the
    standard smooth 2D Euler test):
        du, dv = eps/(2 pi) exp((1 - r^2)/2) (-ybar, xbar)
        T = 1 - (gamma - 1) eps^2 / (8 gamma pi^2) exp(1 - r^2)
        rho = T^(1/(gamma-1)),  p = rho^gamma.
    ``period`` = (Lx, Ly) wraps the centre into a periodic box."""
    ph = Euler(gamma, 2)
    cx = xc + mean[0] * t
    cy = yc + mean[1] * t
    xb = X - cx
    yb = Y - cy
    if period is not None:
        Lx, Ly = period
        xb = xb - Lx * np.round(xb / Lx)
        yb = yb - Ly * np.round(yb / Ly)
    r2 = xb * xb + yb * yb
    amp = eps / (2 * np.pi) * np.exp(0.5 * (1 - r2))
    w = mean[0] - amp * yb
    v = mean[1] + amp * xb
    T = 1 - (gamma - 1) * eps * eps / (8 * gamma * np.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1.0 / (gamma - 1))
    p = rho ** gamma
    return ph.conserved(rho, [w, v], p)
