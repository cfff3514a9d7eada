"""2D discontinuous Galerkin operators on uniform Cartesian meshes and the
RKDG / cRKDG steps (Sec. 2, extended to systems and two dimensions as the
paper's Sec. 4.1.2 and 4.2.2 do).

State u[y, x, v, m] with the modes of ``basis.modes_2d``.  On the cell
K = [x_l, x_l + dx] x [y_l, y_l + dy] with reference coordinates (xi, eta):

  M_m (div f)_m = - int_K f . grad phi_m + sum_{e in dK} int_e G_e phi_m
  M_m = dx dy / ((2i+1)(2j+1))

  G_e = f(u^int) . nu_e                 local operator, eq. (2.7)
  G_e = fhat(u^int, u^ext; nu_e)        DG operator, eq. (2.3)

Integrals use the (k+1)-point Gauss rule per direction (a reading: the paper
does not state its quadrature).  In reference coordinates
  (div f)_m = (2i+1)(2j+1)/2 * [ (X_m^face - X_m^vol)/dx + (Y_m^face - Y_m^vol)/dy ]
  X_m^vol  = sum_q w_q f_x(u_q) dphi_m/dxi (q),  X_m^face = sum_p w_p (G_E phi_m(1,eta_p) + G_W phi_m(-1,eta_p))
and likewise in y.

Boundary conditions (one per side W, E, S, N) give the exterior trace at a
boundary face point from the interior trace, the point and the time:
  'periodic'                neighbour across the domain
  'outflow'                 u^ext = u^int
  'reflect'                 u^ext = u^int with the normal momentum negated
  ('dirichlet', g)          u^ext = g(x, y, t)
  ('custom', h)             u^ext = h(u^int, x, y, t)
For stage i the boundary time is t^n + c_i dt; in cRKDG boundary data enter
only the final stage (Sec. 3.4).  Test infrastructure only.
"""
import numpy as np


def _einsum(*a):
    """np.einsum with contraction-order optimisation (same sums)."""
    return np.einsum(*a, optimize=True)


from .basis import Basis2D
from .physics import lf_flux

SIDES = ("W", "E", "S", "N")
# (axis, outward sign) of every side
NORMAL = {"E": (0, 1.0), "W": (0, -1.0), "N": (1, 1.0), "S": (1, -1.0)}


class DG2D:
    def __init__(self, nx, ny, box, k, basis, phys, bc, nq=None):
        self.nx, self.ny = nx, ny
        self.x0, self.x1, self.y0, self.y1 = box
        self.dx = (self.x1 - self.x0) / nx
        self.dy = (self.y1 - self.y0) / ny
        self.xc = self.x0 + (np.arange(nx) + 0.5) * self.dx
        self.yc = self.y0 + (np.arange(ny) + 0.5) * self.dy
        self.k = k
        self.B = Basis2D(k, basis, nq)
        self.phys = phys
        self.nv = phys.nv
        self.bc = dict(bc)
        # 1 / (2 * mass_m) = (2i+1)(2j+1)/2
        self.cm = 0.5 / self.B.mass

    # -- coordinates ---------------------------------------------------------------
    def volume_points(self, B=None):
        """(X, Y) of the volume quadrature points, shape (ny, nx, nq*nq)."""
        B = self.B if B is None else B
        X = self.xc[None, :, None] + 0.5 * self.dx * B.xi[None, None, :]
        Y = self.yc[:, None, None] + 0.5 * self.dy * B.eta[None, None, :]
        return np.broadcast_arrays(X, Y)

    def face_points(self, side):
        """(X, Y) of the face quadrature points of every cell on one side,
        shape (ny, nx, nq)."""
        p = self.B.x1
        if side in ("E", "W"):
            xf = self.xc + (0.5 if side == "E" else -0.5) * self.dx
            X = xf[None, :, None] + 0 * p[None, None, :]
            Y = self.yc[:, None, None] + 0.5 * self.dy * p[None, None, :]
        else:
            yf = self.yc + (0.5 if side == "N" else -0.5) * self.dy
            X = self.xc[None, :, None] + 0.5 * self.dx * p[None, None, :]
            Y = yf[:, None, None] + 0 * p[None, None, :]
        return np.broadcast_arrays(X, Y)

    def project(self, fn, nq=None):
        """L2 projection of fn(X, Y) -> (..., nv) with an nq-point Gauss rule
        per direction (default k + 3): u_m = (1/mass_m) (1/4) sum_q w_q g(x_q) phi_m(q)."""
        B = Basis2D(self.k, self.B.basis, nq if nq is not None else self.k + 3)
        X, Y = self.volume_points(B)
        vals = np.asarray(fn(X, Y), dtype=np.float64)
        c = _einsum("q,yxqv,qm->yxvm", B.wvol, vals, B.phi_vol)
        return 0.25 * c / B.mass

    def project_point_values(self, vals):
        """Projection from values at this discretisation's own volume points,
        vals[y, x, q, v] (the rule of ``volume_points()``)."""
        c = _einsum("q,yxqv,qm->yxvm", self.B.wvol, vals, self.B.phi_vol)
        return 0.25 * c / self.B.mass

    # -- pieces of the operators -----------------------------------------------------
    def volume(self, u):
        """(X^vol, Y^vol) = sum_q w_q f_{x,y}(u(x_q)) d(phi_m)/d(xi, eta)(q)."""
        uq = _einsum("yxvm,qm->yxqv", u, self.B.phi_vol)
        fx = self.phys.flux(uq, 0)
        fy = self.phys.flux(uq, 1)
        vx = _einsum("q,yxqv,qm->yxvm", self.B.wvol, fx, self.B.dxi_vol)
        vy = _einsum("q,yxqv,qm->yxvm", self.B.wvol, fy, self.B.deta_vol)
        return vx, vy

    def traces(self, u):
        """Interior traces at the face points of each side: (ny, nx, nq, nv)."""
        return {s: _einsum("yxvm,pm->yxpv", u, self.B.phi_face[s]) for s in SIDES}

    def face_integral(self, G):
        """X^face and Y^face from the normal fluxes G[side] (ny, nx, nq, nv)."""
        w = self.B.x1 * 0 + self.B.w1
        fx = sum(_einsum("p,yxpv,pm->yxvm", w, G[s], self.B.phi_face[s]) for s in ("E", "W"))
        fy = sum(_einsum("p,yxpv,pm->yxvm", w, G[s], self.B.phi_face[s]) for s in ("N", "S"))
        return fx, fy

    def combine(self, facex, facey, vx, vy):
        return self.cm[None, None, None, :] * ((facex - vx) / self.dx + (facey - vy) / self.dy)

    def exterior(self, tr, t):
        """Exterior traces for every face of every cell, with boundary data
        at time t."""
        ext = {
            "E": np.roll(tr["W"], -1, axis=1),
            "W": np.roll(tr["E"], 1, axis=1),
            "N": np.roll(tr["S"], -1, axis=0),
            "S": np.roll(tr["N"], 1, axis=0),
        }
        for side in SIDES:
            bc = self.bc[side]
            if bc == "periodic":
                continue
            sl = {"E": (slice(None), -1), "W": (slice(None), 0),
                  "N": (-1, slice(None)), "S": (0, slice(None))}[side]
            uint = tr[side][sl]
            X, Y = self.face_points(side)
            ext[side][sl] = self.boundary_state(bc, side, uint, X[sl], Y[sl], t)
        return ext

    def boundary_state(self, bc, side, uint, X, Y, t):
        axis, _ = NORMAL[side]
        if bc == "outflow":
            return uint.copy()
        if bc == "reflect":
            out = uint.copy()
            out[..., 1 + axis] = -out[..., 1 + axis]
            return out
        kind, fn = bc
        if kind == "dirichlet":
            return np.asarray(fn(X, Y, t), dtype=np.float64) + 0 * uint
        if kind == "custom":
            return np.asarray(fn(uint, X, Y, t), dtype=np.float64)
        raise ValueError(bc)

    # -- operators ---------------------------------------------------------------------
    def L_loc(self, u):
        """Local operator of eq. (2.7): face terms f(u^int) . nu_e."""
        vx, vy = self.volume(u)
        tr = self.traces(u)
        G = {}
        for s in SIDES:
            axis, sign = NORMAL[s]
            G[s] = sign * self.phys.flux(tr[s], axis)
        fx, fy = self.face_integral(G)
        return self.combine(fx, fy, vx, vy)

    def L_dg(self, u, t):
        """DG operator of eq. (2.3) with the LF flux of Sec. 2.1 and boundary
        data at time t."""
        vx, vy = self.volume(u)
        tr = self.traces(u)
        ext = self.exterior(tr, t)
        G = {}
        for s in SIDES:
            axis, sign = NORMAL[s]
            G[s] = lf_flux(self.phys, tr[s], ext[s], axis, sign)
        fx, fy = self.face_integral(G)
        return self.combine(fx, fy, vx, vy)

    # -- diagnostics ---------------------------------------------------------------------
    def averages(self, u):
        return u[..., 0]

    def total(self, u):
        """sum_K |K| ubar_K for every variable (the conserved totals of eq. (3.4))."""
        return np.sum(u[..., 0], axis=(0, 1)) * self.dx * self.dy

    def max_speed(self, u):
        """max_K ( s_x(ubar_K)/dx + s_y(ubar_K)/dy ) over cell averages."""
        avg = u[..., 0]
        return np.max(self.phys.speed(avg, 0) / self.dx + self.phys.speed(avg, 1) / self.dy)


def cfl_dt_2d(dg, u, cfl):
    """dt = CFL / max_K ( s_x/dx + s_y/dy ) at cell averages (reading of the
    paper's 2D "CFL number", Sec. 4.1.2 / 4.2.2)."""
    return cfl / dg.max_speed(u)


def crkdg_step(dg, u, t, dt, tab, limiter=None):
    """One cRKDG step, eq. (2.8), with the limiter (if any) applied once, to
    u^{n+1} (Remark 2.2)."""
    A, b, c, s = tab["A"], tab["b"], tab["c"], tab["s"]
    stages, Lloc = [u], []
    for i in range(1, s):
        Lloc.append(dg.L_loc(stages[i - 1]))
        stages.append(u - dt * sum(A[i, j] * Lloc[j] for j in range(i)))
    upd = sum(b[i] * dg.L_dg(stages[i], t + c[i] * dt) for i in range(s) if b[i] != 0.0)
    out = u - dt * upd
    return limiter(out, t + dt) if limiter is not None else out


def rkdg_step(dg, u, t, dt, tab, limiter=None):
    """One RKDG step in Butcher form, eq. (2.6); the limiter follows every
    stage (Sec. 4.2)."""
    A, b, c, s = tab["A"], tab["b"], tab["c"], tab["s"]
    lim = limiter if limiter is not None else (lambda v, tt: v)
    stages, L = [u], []
    for i in range(1, s):
        L.append(dg.L_dg(stages[i - 1], t + c[i - 1] * dt))
        stages.append(lim(u - dt * sum(A[i, j] * L[j] for j in range(i)), t + c[i] * dt))
    L.append(dg.L_dg(stages[s - 1], t + c[s - 1] * dt))
    return lim(u - dt * sum(b[i] * L[i] for i in range(s)), t + dt)


def run(dg, u, t0, T, step, dt=None, cfl=None, max_steps=None):
    """March to T with fixed dt (last step clipped) or the CFL dt."""
    t, n = t0, 0
    while t < T - 1e-14 * max(1.0, abs(T)):
        if max_steps is not None and n >= max_steps:
            break
        d = dt if dt is not None else cfl_dt_2d(dg, u, cfl)
        d = min(d, T - t)
        u = step(u, t, d)
        t += d
        n += 1
    return u, n, t


def rkdg_ssp_step(dg, u, t, dt, order, limiter=None):
    """RKDG in the Shu--Osher SSP-RK2 / SSP-RK3 forms (convex combinations of
    forward Euler steps, Sec. 3.2.1) with the limiter after every stage
    (Sec. 4.2); boundary data of the stages at t, t + dt (, t + dt/2)."""
    lim = limiter if limiter is not None else (lambda v, tt: v)
    if order == 2:
        u1 = lim(u - dt * dg.L_dg(u, t), t + dt)
        return lim(0.5 * u + 0.5 * (u1 - dt * dg.L_dg(u1, t + dt)), t + dt)
    if order == 3:
        u1 = lim(u - dt * dg.L_dg(u, t), t + dt)
        u2 = lim(0.75 * u + 0.25 * (u1 - dt * dg.L_dg(u1, t + dt)), t + 0.5 * dt)
        return lim(u / 3.0 + 2.0 / 3.0 * (u2 - dt * dg.L_dg(u2, t + 0.5 * dt)), t + dt)
    raise ValueError(order)
