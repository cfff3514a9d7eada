"""TVB-minmod limiter on 2D Cartesian meshes, applied in characteristic fields.

The paper applies "the standard TVB minmod limiters" of Cockburn and Shu's
RKDG paper on multidimensional systems (Sec. 4.2), once per cRKDG step at the
final stage (Remark 2.2), with parameter M (M = 50 for the double Mach
reflection, Sec. 4.2.2).  The paper does not print the limiter; the reading
implemented here (parity unpinned against the paper; pinned by invariants):

  per direction (x shown; y alike with mode (0,1), dy, N/S neighbours):
    a1 = u_(1,0)                (the xi-slope coefficient of the cell)
    a2 = ubar_E - ubar_K,  a3 = ubar_K - ubar_W
  for systems, project onto characteristic fields with L_x(ubar_K) = R_x^{-1},
  R_x the right eigenvectors of d f_x / d u at the cell average;
  modified minmod, per field:
    mt = a1                     if |a1| <= M dx^2
    mt = minmod(a1, a2, a3)     otherwise   (minmod = s min|.| if all signs
                                              equal s, else 0)
  the cell is troubled if mt != a1 in any field of x or y.  A troubled cell
  keeps its average, gets u_(1,0) = R_x mt_x, u_(0,1) = R_y mt_y, and all
  other modes are set to zero.

Ghost averages across a boundary: periodic -> neighbour across the domain;
outflow -> own average; reflect -> own average with the normal momentum
negated; ('dirichlet', g) -> g at the ghost-cell centre and time t;
('custom', h) -> h(own average, ghost-cell centre, t).
Test infrastructure only.
"""
import numpy as np

from .physics import Euler


def minmod3(a, b, c):
    s = np.sign(a)
    same = (np.sign(b) == s) & (np.sign(c) == s)
    m = np.minimum(np.minimum(np.abs(a), np.abs(b)), np.abs(c))
    return np.where(same, s * m, 0.0)


def tvb_minmod(a1, a2, a3, Mh2):
    return np.where(np.abs(a1) <= Mh2, a1, minmod3(a1, a2, a3))


def ghost_average(dg, side, avg, t):
    """Average of the ghost cell beyond a non-periodic side, from the own
    averages of the boundary cells avg (n, nv)."""
    bc = dg.bc[side]
    axis = 0 if side in ("E", "W") else 1
    if bc == "outflow":
        return avg.copy()
    if bc == "reflect":
        out = avg.copy()
        out[:, 1 + axis] = -out[:, 1 + axis]
        return out
    if side in ("E", "W"):
        X = np.full(dg.ny, dg.x1 + 0.5 * dg.dx if side == "E" else dg.x0 - 0.5 * dg.dx)
        Y = dg.yc
    else:
        X = dg.xc
        Y = np.full(dg.nx, dg.y1 + 0.5 * dg.dy if side == "N" else dg.y0 - 0.5 * dg.dy)
    kind, fn = bc
    if kind == "dirichlet":
        return np.asarray(fn(X, Y, t), dtype=np.float64) + 0 * avg
    return np.asarray(fn(avg, X, Y, t), dtype=np.float64)


def neighbour_averages(dg, avg, t):
    nb = {"E": np.roll(avg, -1, axis=1), "W": np.roll(avg, 1, axis=1),
          "N": np.roll(avg, -1, axis=0), "S": np.roll(avg, 1, axis=0)}
    if dg.bc["E"] != "periodic":
        nb["E"][:, -1] = ghost_average(dg, "E", avg[:, -1], t)
        nb["W"][:, 0] = ghost_average(dg, "W", avg[:, 0], t)
    if dg.bc["N"] != "periodic":
        nb["N"][-1, :] = ghost_average(dg, "N", avg[-1, :], t)
        nb["S"][0, :] = ghost_average(dg, "S", avg[0, :], t)
    return nb


def tvb_limit(dg, u, M, t, force=None):
    """Return (limited copy of u, boolean troubled-cell map).  ``force``
    (optional boolean map) replaces the TVB troubled-cell test: the cells it
    marks get the TVB-minmod reconstruction, the others are kept (the way a
    learned indicator's decisions are applied)."""
    u = np.array(u, dtype=np.float64, copy=True)
    if dg.B.nm < 3:
        return u, np.zeros((dg.ny, dg.nx), dtype=bool)
    avg = u[..., 0]                                   # [y, x, v]
    nb = neighbour_averages(dg, avg, t)
    systems = isinstance(dg.phys, Euler)
    # every cell at once; per cell and direction: (a1, a2, a3) as above
    ax = (u[..., :, 1], nb["E"] - avg, avg - nb["W"])
    ay = (u[..., :, 2], nb["N"] - avg, avg - nb["S"])
    mv = lambda A, a: np.einsum("yxij,yxj->yxi", A, a)    # per-cell matrix times vector
    if systems:
        Rx = dg.phys.right_eigenvectors(avg, 0)           # [y, x, 4, 4]
        Ry = dg.phys.right_eigenvectors(avg, 1)
        Lx, Ly = np.linalg.inv(Rx), np.linalg.inv(Ry)
        cx = [mv(Lx, a) for a in ax]
        cy = [mv(Ly, a) for a in ay]
    else:
        cx, cy = list(ax), list(ay)
    mx = tvb_minmod(cx[0], cx[1], cx[2], M * dg.dx * dg.dx)
    my = tvb_minmod(cy[0], cy[1], cy[2], M * dg.dy * dg.dy)
    if force is None:
        flags = np.any(mx != cx[0], axis=-1) | np.any(my != cy[0], axis=-1)
    else:
        flags = np.asarray(force, dtype=bool).copy()
    newx = mv(Rx, mx) if systems else mx
    newy = mv(Ry, my) if systems else my
    out = u.copy()
    f = flags
    out[f, :, 1] = newx[f]
    out[f, :, 2] = newy[f]
    out[f, :, 3:] = 0.0
    return out, flags


def make_limiter(dg, M):
    """limiter(u, t) -> limited u, for use with the step functions."""
    return lambda u, t: tvb_limit(dg, u, M, t)[0]


# ---------------------------------------------------------------------------
# Positivity-preserving scaling (Zhang and Shu, J. Comput. Phys. 229 (2010),
# "On positivity-preserving high order discontinuous Galerkin schemes for
# compressible Euler equations on rectangular meshes").  Not part of the
# paper's method: an option applied after the TVB limiter, at the same final
# stage, for strong shocks (the Mach 10 double Mach reflection).  Per cell,
# with ubar the average and u_q the values at the scheme's own points (the
# volume Gauss points and the Gauss points of the four faces):
#   1. theta_1 = min(1, (rhobar - eps) / (rhobar - min_q rho_q)) if
#      min_q rho_q < eps; the density's non-constant modes are scaled by it;
#   2. for every point with p(u_q) < eps, t_q in [0, 1] solves
#      p(ubar + t (u_q - ubar)) = eps (a quadratic in t after multiplying by
#      rho); theta_2 = min_q t_q scales every non-constant mode.
# The average is unchanged.  eps = 1e-10 (a reading).
def positivity_points(dg):
    """Basis values at the volume points and the face points: (npts, nm)."""
    return np.concatenate([dg.B.phi_vol] + [dg.B.phi_face[s] for s in ("E", "W", "N", "S")], axis=0)


def positivity_limit(dg, u, eps=1e-10):
    u = np.array(u, dtype=np.float64, copy=True)
    if not isinstance(dg.phys, Euler) or dg.B.nm < 2:
        return u
    g = dg.phys.gamma
    P = positivity_points(dg)
    # step 1: density
    rho_q = np.einsum("yxm,qm->yxq", u[..., 0, :], P)
    rbar = u[..., 0, 0]
    rmin = rho_q.min(axis=-1)
    th1 = np.where(rmin < eps, np.minimum(1.0, (rbar - eps) / np.maximum(rbar - rmin, 1e-300)), 1.0)
    u[..., 0, 1:] *= th1[..., None]
    # step 2: pressure
    uq = np.einsum("yxvm,qm->yxqv", u, P)
    ub = u[..., :, 0]
    d = uq - ub[:, :, None, :]
    dr, de = d[..., 0], d[..., -1]
    dm = d[..., 1:-1]
    rb, eb = ub[..., 0][..., None], ub[..., -1][..., None]
    mb = ub[..., 1:-1][:, :, None, :]
    k = eps / (g - 1.0)
    a = dr * de - 0.5 * np.sum(dm * dm, axis=-1)
    b = rb * de + eb * dr - np.sum(mb * dm, axis=-1) - k * dr
    c = rb * eb - 0.5 * np.sum(mb * mb, axis=-1) - k * rb
    gval = a + b + c                       # value at t = 1
    bad = gval < 0.0
    # smallest root in (0, 1) of a t^2 + b t + c with c > 0 > a + b + c
    disc = np.sqrt(np.maximum(b * b - 4 * a * c, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        q = -0.5 * (b + np.where(b >= 0, disc, -disc))
        r1 = np.where(q != 0, c / q, np.inf)
        r2 = np.where(a != 0, q / a, np.inf)
    r = np.where((r1 > 0) & (r1 <= 1), r1, np.inf)
    r = np.minimum(r, np.where((r2 > 0) & (r2 <= 1), r2, np.inf))
    r = np.where(np.isfinite(r), r, 0.0)
    t = np.where(bad, r, 1.0)
    th2 = t.min(axis=-1)
    u[..., :, 1:] *= th2[..., None, None]
    return u
