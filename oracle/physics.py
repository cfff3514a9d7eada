"""Physical fluxes and the Lax--Friedrichs numerical flux (Sec. 2.1).

Conservation law  u_t + div f(u) = 0  (eq. (2.1)).  Systems used by the
paper's tests (Sec. 4): linear advection f = beta u, Burgers f = u^2/2,
1D Euler (rho, rho w, E) and 2D Euler (rho, rho w, rho v, E) with
E = p/(gamma-1) + rho |vel|^2 / 2.

The Lax--Friedrichs flux of Sec. 2.1 is
    fhat = 1/2 ( f(u_int).nu + f(u_ext).nu - alpha (u_ext - u_int) ),
    alpha = max |d f/d u . nu|.
For linear advection alpha = |beta . nu| and fhat is the upwind flux
(Remark 3.5 / Sec. 4.1.1).  For Euler the paper uses the *local* LF flux;
the reading taken here: alpha is evaluated per face quadrature point and per
RK stage as max(|vel.nu| + c) over the two traces, with c = 0 where
gamma p / rho < 0 (alpha is undefined for such non-hyperbolic point values).

Arrays carry the variable index last: u[..., v].  Test infrastructure only.
"""
import numpy as np


class Advection:
    """f(u) = beta u, beta constant (scalar, nv = 1)."""

    def __init__(self, beta):
        self.beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
        self.nv = 1

    def flux(self, u, axis):
        return self.beta[axis] * u

    def speed(self, u, axis):
        return np.abs(self.beta[axis]) * np.ones(u.shape[:-1])


class Burgers:
    """f(u) = u^2 / 2 (scalar, 1D)."""

    nv = 1

    def flux(self, u, axis):
        return 0.5 * u * u

    def speed(self, u, axis):
        return np.abs(u[..., 0])


class Euler:
    """Compressible Euler equations in d = 1 or 2 dimensions.

    Conserved variables: (rho, rho w, E) in 1D, (rho, rho w, rho v, E) in 2D.
    """

    def __init__(self, gamma=1.4, dim=2):
        self.gamma = float(gamma)
        self.dim = dim
        self.nv = dim + 2

    def primitive(self, u):
        rho = u[..., 0]
        vel = [u[..., 1 + d] / rho for d in range(self.dim)]
        E = u[..., -1]
        kin = 0.5 * rho * sum(v * v for v in vel)
        p = (self.gamma - 1.0) * (E - kin)
        return rho, vel, p

    def flux(self, u, axis):
        rho, vel, p = self.primitive(u)
        vn = vel[axis]
        E = u[..., -1]
        out = np.empty_like(u)
        out[..., 0] = rho * vn
        for d in range(self.dim):
            out[..., 1 + d] = u[..., 1 + d] * vn + (p if d == axis else 0.0)
        out[..., -1] = vn * (E + p)
        return out

    def sound(self, u):
        """c = sqrt(gamma p / rho); a state with gamma p / rho < 0 (a point
        value past a strong shock) is not hyperbolic and d f / d u has no
        real eigenvalues there: the reading taken is c = 0."""
        rho, vel, p = self.primitive(u)
        return np.sqrt(np.maximum(self.gamma * p / rho, 0.0))

    def speed(self, u, axis):
        """|vel . nu| + c, the spectral radius of d f / d u . nu (LF alpha)."""
        rho, vel, p = self.primitive(u)
        return np.abs(vel[axis]) + self.sound(u)

    def conserved(self, rho, vel, p):
        """Conserved state from primitive (rho, [w, v], p); trailing axis = variable."""
        rho = np.asarray(rho, dtype=np.float64)
        vel = [np.asarray(v, dtype=np.float64) + 0 * rho for v in vel]
        p = np.asarray(p, dtype=np.float64) + 0 * rho
        kin = 0.5 * rho * sum(v * v for v in vel)
        comps = [rho] + [rho * v for v in vel] + [p / (self.gamma - 1.0) + kin]
        return np.stack(comps, axis=-1)

    def right_eigenvectors(self, u, axis):
        """Columns = right eigenvectors of d f_axis / d u at the state u (2D
        only), for the eigenvalues (vn - c, vn, vn, vn + c).  Standard
        scaling: first component 1 for the acoustic and entropy waves.
        u[..., 4] -> R[..., 4, 4] (one matrix per state)."""
        assert self.dim == 2
        rho, vel, p = self.primitive(u)
        w, v = vel
        c = np.sqrt(self.gamma * p / rho)
        H = (u[..., -1] + p) / rho
        q2 = w * w + v * v
        one, zero = np.ones_like(w), np.zeros_like(w)
        if axis == 0:
            rows = [[one, one, zero, one],
                    [w - c, w, zero, w + c],
                    [v, v, one, v],
                    [H - w * c, 0.5 * q2, v, H + w * c]]
        else:
            rows = [[one, one, zero, one],
                    [w, w, one, w],
                    [v - c, v, zero, v + c],
                    [H - v * c, 0.5 * q2, w, H + v * c]]
        return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)


def lf_flux(phys, uint, uext, axis, sign):
    """Lax--Friedrichs flux fhat . nu on a face with outward normal
    nu = sign * e_axis, at every point: 1/2 (f(u_int).nu + f(u_ext).nu
    - alpha (u_ext - u_int)), alpha = max over both traces of |f'(u).nu|
    (local, per point)."""
    fi = sign * phys.flux(uint, axis)
    fe = sign * phys.flux(uext, axis)
    alpha = np.maximum(phys.speed(uint, axis), phys.speed(uext, axis))
    return 0.5 * (fi + fe - alpha[..., None] * (uext - uint))


def godunov_burgers(ul, ur):
    """Exact Riemann (Godunov) flux for Burgers, f = u^2/2, left state ul,
    right state ur (flux in +x direction)."""
    f = lambda s: 0.5 * s * s
    out = np.where(ul <= ur,
                   np.where((ul <= 0) & (0 <= ur), 0.0, np.minimum(f(ul), f(ur))),
                   np.maximum(f(ul), f(ur)))
    return out
