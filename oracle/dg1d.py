"""1D discontinuous Galerkin operators and the RKDG / cRKDG time steps.

Follows Sec. 2 of the paper on a 1D mesh of cells K_j = [x_{j-1/2}, x_{j+1/2}]
with the Legendre basis of ``basis.Basis1D`` (u[x, v, m]).

  DG operator (eq. (2.3)):  int_K (div^DG f) v = - int_K f(u) v' + fhat v |_faces
  local operator (eq. (2.7)): the same with fhat replaced by the interior
                              trace f(u^int) . nu (no neighbour data)
  RKDG (eq. (2.6)):  every stage uses div^DG
  cRKDG (eq. (2.8)): inner stages use div^loc, the update uses div^DG
  Shu--Osher SSP forms and the non-conservative variant of eq. (3.1)

Boundary data for a stage i are taken at t^n + c_i dt (Sec. 2.1, remark
after eq. (2.6); Sec. 3.4).  Test infrastructure only.
"""
import numpy as np

from .basis import Basis1D
from .physics import godunov_burgers


class DG1D:
    """P^k DG discretisation of u_t + f(u)_x = 0 on a 1D mesh.

    nodes : cell interfaces x_{1/2} < ... < x_{N+1/2}
    bc    : (left, right); each 'periodic', 'outflow' or ('dirichlet', g)
            with g(t) -> exterior state (nv,) at that boundary
    flux  : 'lf' (Lax--Friedrichs, local alpha) or 'godunov' (Burgers only)
    """

    def __init__(self, nodes, k, phys, bc=("periodic", "periodic"), flux="lf", nq=None):
        self.nodes = np.asarray(nodes, dtype=np.float64)
        self.h = np.diff(self.nodes)
        self.xc = 0.5 * (self.nodes[1:] + self.nodes[:-1])
        self.n = len(self.h)
        self.k = k
        self.B = Basis1D(k, nq)
        self.phys = phys
        self.bc = bc
        self.flux_kind = flux
        # (2m+1) / h_j : inverse of the diagonal mass matrix
        self.minv = (2.0 * np.arange(k + 1) + 1.0)[None, :] / self.h[:, None]

    # -- element quantities ------------------------------------------------
    def points(self):
        """Physical coordinates of the volume quadrature points, shape (N, nq)."""
        return self.xc[:, None] + 0.5 * self.h[:, None] * self.B.xq[None, :]

    def project(self, fn, nq=None):
        """L2 projection Pi of a function fn(x) -> (..., nv) onto V_h, by an
        nq-point Gauss rule (default k + 3)."""
        B = Basis1D(self.k, nq if nq is not None else self.k + 3)
        x = self.xc[:, None] + 0.5 * self.h[:, None] * B.xq[None, :]
        vals = np.asarray(fn(x), dtype=np.float64).reshape(self.n, B.nq, -1)
        # coefficient m = (2m+1)/2 * sum_q w_q u(x_q) P_m(xi_q)
        c = np.einsum("q,xqv,qm->xvm", B.wq, vals, B.phi)
        return c * (2.0 * np.arange(self.k + 1) + 1.0) / 2.0

    def evaluate(self, u, xi):
        """Values of u_h at reference points xi in every cell: (N, len(xi), nv)."""
        phi = np.stack([np.polynomial.legendre.legval(xi, np.eye(self.k + 1)[m])
                        for m in range(self.k + 1)], axis=1)
        return np.einsum("xvm,qm->xqv", u, phi)

    def averages(self, u):
        return u[:, :, 0]

    # -- operators -----------------------------------------------------------
    def volume(self, u):
        """sum_q w_q f(u(x_q)) P_m'(xi_q): the reference-cell form of
        int_K f(u_h) v' dx (the factors h/2 and 2/h cancel)."""
        uq = np.einsum("xvm,qm->xqv", u, self.B.phi)
        f = self.phys.flux(uq, 0)
        return np.einsum("q,xqv,qm->xvm", self.B.wq, f, self.B.dphi)

    def traces(self, u):
        """(u(x_{j-1/2}^+), u(x_{j+1/2}^-)) for every cell: left and right traces."""
        left = np.einsum("xvm,m->xv", u, self.B.phi_l)
        right = np.einsum("xvm,m->xv", u, self.B.phi_r)
        return left, right

    def L_loc(self, u):
        """Local operator div^loc f of eq. (2.7): face terms use the cell's own
        traces, f(u^int) . nu, with nu = +1 on the right and -1 on the left."""
        left, right = self.traces(u)
        fr = self.phys.flux(right, 0)
        fl = -self.phys.flux(left, 0)
        face = fr[:, :, None] * self.B.phi_r[None, None, :] + fl[:, :, None] * self.B.phi_l[None, None, :]
        return self.minv[:, None, :] * (face - self.volume(u))

    def interface_states(self, u, t):
        """States (uL, uR) on the N+1 interfaces x_{i-1/2}, i = 0..N."""
        left, right = self.traces(u)
        nv = u.shape[1]
        uL = np.empty((self.n + 1, nv))
        uR = np.empty((self.n + 1, nv))
        uL[1:] = right
        uR[:-1] = left
        if self.bc[0] == "periodic":
            uL[0] = right[-1]
            uR[-1] = left[0]
        else:
            for side, bc in (("L", self.bc[0]), ("R", self.bc[1])):
                if side == "L":
                    uL[0] = uR[0] if bc == "outflow" else bc[1](t)
                else:
                    uR[-1] = uL[-1] if bc == "outflow" else bc[1](t)
        return uL, uR

    def numerical_flux(self, uL, uR):
        """Flux through an interface in the +x direction."""
        if self.flux_kind == "godunov":
            return godunov_burgers(uL, uR)
        fl = self.phys.flux(uL, 0)
        fr = self.phys.flux(uR, 0)
        alpha = np.maximum(self.phys.speed(uL, 0), self.phys.speed(uR, 0))
        return 0.5 * (fl + fr - alpha[:, None] * (uR - uL))

    def L_dg(self, u, t):
        """DG operator div^DG f of eq. (2.3) with boundary data at time t."""
        uL, uR = self.interface_states(u, t)
        F = self.numerical_flux(uL, uR)          # (N+1, nv)
        fr = F[1:]                                # right face, nu = +1
        fl = -F[:-1]                              # left face,  nu = -1
        face = fr[:, :, None] * self.B.phi_r[None, None, :] + fl[:, :, None] * self.B.phi_l[None, None, :]
        return self.minv[:, None, :] * (face - self.volume(u))


# -- time steps ------------------------------------------------------------------
def crkdg_step(dg, u, t, dt, tab):
    """One cRKDG step, eq. (2.8):
       u^(i)   = u^n - dt sum_{j<i} a_ij div^loc f(u^(j))
       u^{n+1} = u^n - dt sum_i b_i div^DG f(u^(i)),  stage i at t + c_i dt."""
    A, b, c, s = tab["A"], tab["b"], tab["c"], tab["s"]
    stages, Lloc = [u], []
    for i in range(1, s):
        Lloc.append(dg.L_loc(stages[i - 1]))
        stages.append(u - dt * sum(A[i, j] * Lloc[j] for j in range(i)))
    upd = sum(b[i] * dg.L_dg(stages[i], t + c[i] * dt) for i in range(s) if b[i] != 0.0)
    return u - dt * upd


def rkdg_step(dg, u, t, dt, tab, limiter=None):
    """One RKDG step in Butcher form, eq. (2.6): every stage uses div^DG.
    An optional limiter is applied to every stage value and to u^{n+1}."""
    A, b, c, s = tab["A"], tab["b"], tab["c"], tab["s"]
    lim = limiter if limiter is not None else (lambda v, tt: v)
    stages, L = [u], []
    for i in range(1, s):
        L.append(dg.L_dg(stages[i - 1], t + c[i - 1] * dt))
        stages.append(lim(u - dt * sum(A[i, j] * L[j] for j in range(i)), t + c[i] * dt))
    L.append(dg.L_dg(stages[s - 1], t + c[s - 1] * dt))
    return lim(u - dt * sum(b[i] * L[i] for i in range(s)), t + dt)


def rkdg_ssp_step(dg, u, t, dt, order, limiter=None):
    """RKDG with the Shu--Osher SSP-RK2 / SSP-RK3 forms (convex combinations
    of forward Euler steps, Sec. 3.2.1), limiter after every stage."""
    lim = limiter if limiter is not None else (lambda v, tt: v)
    if order == 2:
        u1 = lim(u - dt * dg.L_dg(u, t), t + dt)
        return lim(0.5 * u + 0.5 * (u1 - dt * dg.L_dg(u1, t + dt)), t + dt)
    if order == 3:
        u1 = lim(u - dt * dg.L_dg(u, t), t + dt)
        u2 = lim(0.75 * u + 0.25 * (u1 - dt * dg.L_dg(u1, t + dt)), t + 0.5 * dt)
        return lim(u / 3.0 + 2.0 / 3.0 * (u2 - dt * dg.L_dg(u2, t + 0.5 * dt)), t + dt)
    raise ValueError(order)


def shu_osher_crkdg_wrong_step(dg, u, t, dt, order):
    """The suboptimal, non-conservative variant of Sec. 3.2.1: div^DG replaced
    by div^loc in the inner stages of the *Shu--Osher* form (eq. (3.1) for
    SSP-RK2; the same substitution for SSP-RK3)."""
    if order == 2:
        u1 = u - dt * dg.L_loc(u)
        return 0.5 * u + 0.5 * (u1 - dt * dg.L_dg(u1, t + dt))
    if order == 3:
        u1 = u - dt * dg.L_loc(u)
        u2 = 0.75 * u + 0.25 * (u1 - dt * dg.L_loc(u1))
        return u / 3.0 + 2.0 / 3.0 * (u2 - dt * dg.L_dg(u2, t + 0.5 * dt))
    raise ValueError(order)


def cfl_dt_1d(dg, u, cfl):
    """dt = CFL * min_j h_j / max_j |f'(ubar_j)| from cell averages."""
    avg = dg.averages(u)
    s = dg.phys.speed(avg, 0)
    return cfl * np.min(dg.h) / np.max(s)


def run(dg, u, t0, T, step, dt=None, cfl=None):
    """March from t0 to T with a fixed dt (last step clipped) or a CFL dt.
    ``step(u, t, dt)`` advances one step.  Returns (u, nsteps)."""
    t, n = t0, 0
    while t < T - 1e-14 * max(1.0, abs(T)):
        d = dt if dt is not None else cfl_dt_1d(dg, u, cfl)
        d = min(d, T - t)
        u = step(u, t, d)
        t += d
        n += 1
    return u, n
