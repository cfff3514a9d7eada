"""Seeded synthetic inputs and problem data shared by the tests, the bench and
the CPU oracle's callers.

This module holds problem definitions (initial data, boundary states, random
ensembles) and nothing of the cRKDG method's arithmetic: no basis, no
quadrature, no projection, no flux and no time stepping.  Both sides of every
parity test take their inputs from here and discretise them with their own
code.

Contents
  splitmix64           counter-based 64-bit generator (Steele, Lea, Flood 2014)
  random_modal_state   smooth random modal states for operator parity tests
  vortex_ic            isentropic vortex (strength eps, mean flow (1, 1))
  sine_wave_2d         rho = 1 + 0.2 sin(pi (x + y)), (0.7, 0.3), p = 1
  dmr_states           Mach-10 double Mach reflection states (Rankine--Hugoniot)
  riemann_ensemble     four-quadrant Riemann problems of uneven sizes
  shock_vortex         stationary Mach 1.1 normal shock + weak vortex
"""
import math

import numpy as np

GAMMA = 1.4
MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15; z = mix(state).  Published
    constants of the generator; uniform doubles use the top 53 bits."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0):
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def conserved(rho, w, v, p, gamma=GAMMA):
    """Conserved 2D Euler state (rho, rho w, rho v, E), variable index last."""
    rho, w, v, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, w, v, p)))
    E = p / (gamma - 1.0) + 0.5 * rho * (w * w + v * v)
    return np.stack([rho, rho * w, rho * v, E], axis=-1)


def n_modes(k, basis):
    return (k + 1) * (k + 2) // 2 if basis == "P" else (k + 1) ** 2


def mode_degrees(k, basis):
    """Total degree of every mode in the library's mode order (by total
    degree, then first index descending)."""
    out = []
    dmax = k if basis == "P" else 2 * k
    for d in range(dmax + 1):
        for i in range(d, -1, -1):
            if i <= k and d - i <= k:
                out.append(d)
    return np.array(out)


def random_modal_state(ny, nx, k, basis, physics, seed, amp=0.05):
    """Random modal coefficients u[y, x, v, m] (FP64) that stay physical:
    averages from smooth random primitives, higher modes small and decaying
    with degree.  physics: 'euler' (4 variables) or 'advection' (1)."""
    rng = np.random.default_rng(seed)
    nm = n_modes(k, basis)
    deg = mode_degrees(k, basis)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, size=8)
    sx = 2 * np.pi / max(nx, 1)
    sy = 2 * np.pi / max(ny, 1)
    f = lambda a, b: np.sin(a * sx * xx + ph[b]) * np.cos(a * sy * yy + ph[b + 1])
    if physics == "euler":
        rho = 1.0 + 0.3 * f(1, 0) + 0.05 * rng.uniform(-1, 1, size=(ny, nx))
        w = 0.5 * f(1, 2) + 0.05 * rng.uniform(-1, 1, size=(ny, nx))
        v = 0.5 * f(2, 4) + 0.05 * rng.uniform(-1, 1, size=(ny, nx))
        p = 1.0 + 0.3 * f(1, 6) + 0.05 * rng.uniform(-1, 1, size=(ny, nx))
        avg = conserved(rho, w, v, p)
    else:
        avg = (np.sin(sx * xx + ph[0]) * np.cos(sy * yy + ph[1]))[..., None] + 0.1 * rng.normal(size=(ny, nx, 1))
    nv = avg.shape[-1]
    u = np.zeros((ny, nx, nv, nm))
    u[..., 0] = avg
    for m in range(1, nm):
        u[..., m] = amp * np.abs(avg) * rng.normal(size=(ny, nx, nv)) / (2.0 ** deg[m])
    return u


def random_modal_state_1d(nx, k, nv, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    u = np.zeros((nx, nv, k + 1))
    x = np.arange(nx) * 2 * np.pi / nx
    u[:, :, 0] = (1.0 + 0.3 * np.sin(x))[:, None] if nv == 3 else np.sin(x)[:, None]
    if nv == 3:
        w = 0.5 * np.cos(x)
        p = 1.0 + 0.2 * np.sin(2 * x)
        rho = u[:, 0, 0]
        u[:, 1, 0] = rho * w
        u[:, 2, 0] = p / (GAMMA - 1) + 0.5 * rho * w * w
    for m in range(1, k + 1):
        u[:, :, m] = amp * np.abs(u[:, :, 0]) * rng.normal(size=(nx, nv)) / 2.0 ** m
    return u


# -- smooth problems ---------------------------------------------------------------
def vortex_ic(X, Y, t=0.0, eps=5.0, center=(5.0, 5.0), mean=(1.0, 1.0), period=(10.0, 10.0),
              gamma=GAMMA):
    """Isentropic vortex: perturbation eps/(2 pi) exp((1-r^2)/2) (-ybar, xbar)
    of the mean flow, temperature 1 - (gamma-1) eps^2/(8 gamma pi^2) exp(1-r^2),
    rho = T^(1/(gamma-1)), p = rho^gamma.  The centre moves with the mean flow
    and is wrapped into the periodic box."""
    xb = X - (center[0] + mean[0] * t)
    yb = Y - (center[1] + mean[1] * t)
    if period is not None:
        xb = xb - period[0] * np.round(xb / period[0])
        yb = yb - period[1] * np.round(yb / period[1])
    r2 = xb * xb + yb * yb
    a = eps / (2 * math.pi) * np.exp(0.5 * (1 - r2))
    T = 1 - (gamma - 1) * eps * eps / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
    rho = T ** (1 / (gamma - 1))
    return conserved(rho, mean[0] - a * yb, mean[1] + a * xb, rho ** gamma, gamma)


def sine_wave_2d(X, Y, t=0.0):
    rho = 1 + 0.2 * np.sin(np.pi * (X + Y - t))
    return conserved(rho, 0.7 + 0 * X, 0.3 + 0 * X, 1 + 0 * X)


# -- double Mach reflection -----------------------------------------------------------
def normal_shock(mach, rho1=1.4, p1=1.0, gamma=GAMMA):
    """State behind a normal shock of Mach number ``mach`` moving into gas at
    rest (rho1, p1): returns (rho2, p2, u2 lab-frame speed behind the shock,
    shock speed s)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    s = mach * c1
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (m2 - 1))
    u2 = s * (1 - rho1 / rho2)
    return rho2, p2, u2, s


def dmr_states(gamma=GAMMA):
    """Pre- and post-shock conserved states of the double Mach reflection:
    a Mach 10 shock at 60 degrees to the wall (the shock normal points along
    (cos 30, -sin 30)) moving into rho = 1.4, p = 1 at rest.  Also returns the
    wall start x0 = 1/6 and the speed of the shock's x-intercept, 20/sqrt(3)
    for Mach 10 (shock line x = x0 + (y + s t / sin 60 ... ) / tan 60)."""
    rho2, p2, u2, s = normal_shock(10.0, 1.4, 1.0, gamma)
    ang = math.pi / 6
    post = conserved(rho2, u2 * math.cos(ang), -u2 * math.sin(ang), p2, gamma)
    pre = conserved(1.4, 0.0, 0.0, 1.0, gamma)
    return {"pre": pre, "post": post, "x0": 1.0 / 6.0, "shock_speed": s,
            "slope": 1.0 / math.sqrt(3.0), "xspeed": s / math.cos(ang)}


def dmr_shock_x(y, t, st):
    """x-position of the incident shock at height y and time t:
    x = 1/6 + y/sqrt(3) + t * (shock speed / cos 30)."""
    return st["x0"] + st["slope"] * y + st["xspeed"] * t


def dmr_ic(X, Y, st=None):
    st = dmr_states() if st is None else st
    post = X < dmr_shock_x(Y, 0.0, st)
    return np.where(post[..., None], st["post"], st["pre"])


# -- four-quadrant Riemann ensemble ------------------------------------------------------
def _vacuum_ok(a, b, normal, gamma, margin):
    """Pressure-positivity (no vacuum) test for the 1D Riemann problem across
    a quadrant boundary: 2 (c_a + c_b)/(gamma - 1) > (u_b - u_a) . n + margin."""
    ca = math.sqrt(gamma * a[3] / a[0])
    cb = math.sqrt(gamma * b[3] / b[0])
    du = (b[1 + normal] - a[1 + normal])
    return 2 * (ca + cb) / (gamma - 1) > du + margin


def riemann_ensemble(n_problems=256, seed=20230713, sizes=(64, 128, 256, 512), gamma=GAMMA,
                     margin=0.5):
    """Four-quadrant Riemann problems on [0,1]^2 split at (0.5, 0.5), seeded
    with SplitMix64.  Each problem draws its mesh size N from ``sizes``
    (N x N cells) and four primitive states (rho, w, v, p) with rho, p in
    U[0.1, 1.5] and w, v in U[-1, 1]; quadrant order NE, NW, SW, SE.  A
    problem whose adjacent quadrants fail the vacuum test (margin 0.5) is
    redrawn.  Returns a list of dicts {N, prim[4][4]}."""
    g = SplitMix64(seed)
    out = []
    while len(out) < n_problems:
        N = sizes[g.next_u64() % len(sizes)]
        prim = []
        for q in range(4):
            prim.append((g.uniform(0.1, 1.5), g.uniform(-1.0, 1.0), g.uniform(-1.0, 1.0),
                         g.uniform(0.1, 1.5)))
        ne, nw, sw, se = prim
        pairs = [(nw, ne, 0), (sw, se, 0), (se, ne, 1), (sw, nw, 1)]
        if all(_vacuum_ok(a, b, n, gamma, margin) for (a, b, n) in pairs):
            out.append({"N": N, "prim": prim})
    return out


def riemann_ic(X, Y, prim, gamma=GAMMA):
    ne, nw, sw, se = [conserved(*p, gamma=gamma) for p in prim]
    east = X >= 0.5
    north = Y >= 0.5
    return np.where((north & east)[..., None], ne,
                    np.where(north[..., None], nw, np.where(east[..., None], se, sw)))


# -- shock-vortex interaction ----------------------------------------------------------------
def shock_vortex(X, Y, mach=1.1, eps=0.3, center=(0.25, 0.5), radius=0.05, shock_x=0.5,
                 gamma=GAMMA):
    """Stationary Mach-1.1 normal shock at x = 0.5 on [0, 2] x [0, 1] with a
    weak isentropic vortex upstream.  Upstream: rho = 1, p = 1, w = mach * c;
    downstream from Rankine--Hugoniot in the shock frame.  The vortex has the
    isentropic-vortex form above with lengths scaled by ``radius``."""
    c1 = math.sqrt(gamma)
    w1 = mach * c1
    rho2, p2, du, _ = normal_shock(mach, 1.0, 1.0, gamma)
    w2 = w1 - du
    xb = (X - center[0]) / radius
    yb = (Y - center[1]) / radius
    r2 = xb * xb + yb * yb
    a = eps / (2 * math.pi) * np.exp(0.5 * (1 - r2))
    T = 1 - (gamma - 1) * eps * eps / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
    rho_up = T ** (1 / (gamma - 1))
    up = conserved(rho_up, w1 - a * yb, a * xb, rho_up ** gamma, gamma)
    down = conserved(rho2 + 0 * X, w2 + 0 * X, 0 * X, p2 + 0 * X, gamma)
    return np.where((X < shock_x)[..., None], up, down)
