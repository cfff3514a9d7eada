"""Helpers that set up one problem on both sides of a parity test: the CUDA
library through the C ABI (paper_2307_06471_gb300.binding) and the FP64 CPU
oracle.  Boundary conditions are described once and translated to each
side; layouts are converted between the oracle's u[y, x, v, m] and the
library's planes [v, m, y, x].  Inputs come from crkdg_inputs only."""
import numpy as np

from oracle import tableaux as OTB
from oracle.dg1d import DG1D
from oracle.dg2d import DG2D
from oracle.physics import Advection, Euler

TAB_NAMES = {"midpoint": OTB.MIDPOINT, "heun2": OTB.HEUN, "heun3": OTB.HEUN3, "ssprk3": OTB.SSPRK3,
             "rk4": OTB.RK4, "euler": OTB.EULER}


def to_planes(u):
    """oracle [y, x, v, m] (2D) or [x, v, m] (1D) -> library [v, m, y, x]."""
    if u.ndim == 3:
        return np.ascontiguousarray(np.transpose(u, (1, 2, 0))[:, :, None, :])
    return np.ascontiguousarray(np.transpose(u, (2, 3, 0, 1)))


def from_planes(p, dim=2):
    if dim == 1:
        return np.ascontiguousarray(np.transpose(p[:, :, 0, :], (2, 0, 1)))
    return np.ascontiguousarray(np.transpose(p, (2, 3, 0, 1)))


def _reflect(u, axis):
    out = np.array(u, dtype=np.float64, copy=True)
    out[..., 1 + axis] = -out[..., 1 + axis]
    return out


def gpu_bc(desc):
    """(type, fn, params) of the C ABI for one side."""
    from paper_2307_06471_gb300 import binding as B
    kind = desc[0]
    if kind == "periodic":
        return B.BC_PERIODIC, 0, None
    if kind == "outflow":
        return B.BC_OUTFLOW, 0, None
    if kind == "reflect":
        return B.BC_REFLECT, 0, None
    if kind == "const":
        return B.BC_DIRICHLET, B.FN_CONST, list(desc[1])
    if kind == "sine":
        return B.BC_DIRICHLET, B.FN_SINE, list(desc[1:])
    if kind == "sine_prod":
        return B.BC_DIRICHLET, B.FN_SINE_PROD, list(desc[1:])
    if kind == "dmr_bottom":
        return B.BC_DIRICHLET, B.FN_DMR_BOTTOM, list(desc[1]) + [desc[2]]
    if kind == "dmr_top":
        return B.BC_DIRICHLET, B.FN_DMR_TOP, list(desc[1]) + list(desc[2]) + [desc[3], desc[4], desc[5]]
    raise ValueError(desc)


def oracle_bc(desc, axis):
    kind = desc[0]
    if kind in ("periodic", "outflow", "reflect"):
        return kind
    if kind == "const":
        st = np.asarray(desc[1], dtype=np.float64)
        return ("dirichlet", lambda X, Y, t: np.broadcast_to(st, np.shape(X) + st.shape).copy())
    if kind == "sine":
        A, kx, ky, w, ph = desc[1:]
        return ("dirichlet", lambda X, Y, t: (A * np.sin(kx * X + ky * Y - w * t + ph))[..., None])
    if kind == "sine_prod":
        A, kx, cx, ky, cy = desc[1:]
        return ("dirichlet", lambda X, Y, t: (A * np.sin(kx * (X - cx * t)) * np.sin(ky * (Y - cy * t)))[..., None])
    if kind == "dmr_bottom":
        post, x0 = np.asarray(desc[1]), desc[2]
        return ("custom", lambda u, X, Y, t: np.where((np.asarray(X) < x0)[..., None], post, _reflect(u, axis)))
    if kind == "dmr_top":
        post, pre, x0, sy, st = np.asarray(desc[1]), np.asarray(desc[2]), desc[3], desc[4], desc[5]
        return ("dirichlet", lambda X, Y, t: np.where((np.asarray(X) < x0 + sy * np.asarray(Y) + st * t)[..., None],
                                                      post, pre))
    raise ValueError(desc)


def make_pair_2d(nx, ny, box, k, basis, physics, tab, bcs, precision, gamma=1.4, beta=(1.0, 0.5)):
    """bcs: dict side -> description.  Returns (Solver, DG2D)."""
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    sides = ("W", "E", "S", "N")
    codes = [gpu_bc(bcs[s]) for s in sides]
    mesh = B.make_mesh(2, nx, ny, box, [c[0] for c in codes], [c[1] for c in codes], [c[2] for c in codes])
    phys_id = B.EULER if physics == "euler" else B.ADVECTION
    prec = {"f64": B.F64, "f32": B.F32, "f32c": B.F32C, "f32d": B.F32D}[precision]
    solver = B.Solver(mesh, k, B.BASIS_P if basis == "P" else B.BASIS_Q, GTB.BY_NAME[tab], phys_id, prec,
                      gamma=gamma, beta=beta)
    ph = Euler(gamma, 2) if physics == "euler" else Advection(list(beta))
    obc = {s: oracle_bc(bcs[s], 0 if s in ("W", "E") else 1) for s in sides}
    dg = DG2D(nx, ny, box, k, basis, ph, obc)
    return solver, dg


def make_pair_1d(nx, box, k, physics, tab, bcs, precision, gamma=1.4, beta=1.0):
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    codes = [gpu_bc(bcs[0]), gpu_bc(bcs[1])]
    mesh = B.make_mesh(1, nx, 1, box, [codes[0][0], codes[1][0], 0, 0], [codes[0][1], codes[1][1], 0, 0],
                       [codes[0][2], codes[1][2], None, None])
    phys_id = B.EULER if physics == "euler" else B.ADVECTION
    solver = B.Solver(mesh, k, B.BASIS_P, GTB.BY_NAME[tab], phys_id, B.F64 if precision == "f64" else B.F32,
                      gamma=gamma, beta=(beta, 0.0))
    ph = Euler(gamma, 1) if physics == "euler" else Advection([beta])

    def obc1(d):
        if d[0] in ("periodic", "outflow"):
            return d[0]
        if d[0] == "const":
            st = np.asarray(d[1], dtype=np.float64)
            return ("dirichlet", lambda t: st)
        if d[0] == "sine":
            A, kx, ky, w, phs = d[1:]
            x = box[0]
            return ("dirichlet", lambda t: np.array([A * np.sin(kx * x - w * t + phs)]))
        raise ValueError(d)
    dg = DG1D(np.linspace(box[0], box[1], nx + 1), k, ph, bc=(obc1(bcs[0]), obc1(bcs[1])))
    return solver, dg


def rel_err(a, b, vaxis=-2):
    """Largest error relative to the scale of its own variable: max over the
    conserved variables v of max|a_v - b_v| / s_v, with s_v = max|b_v| over
    all cells and modes (the oracle layout [..., v, m] has v at axis -2; pass
    vaxis=0 for library planes [v, m, y, x]).  A variable whose own scale is
    below 1 % of max(1, max|b|) -- a component that is zero in the reference,
    such as the momentum of a state at rest -- is measured against that
    floor instead.  Each variable is held to its own size, so the largest
    variable (the energy of a strong shock, hundreds of times the density)
    cannot hide an error in a small one."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), vaxis, 0)
    b = np.moveaxis(np.asarray(b, dtype=np.float64), vaxis, 0)
    floor = 1e-2 * max(1.0, float(np.max(np.abs(b))))
    return max(float(np.max(np.abs(a[v] - b[v]))) / max(float(np.max(np.abs(b[v]))), floor)
               for v in range(b.shape[0]))


def tvb_margin(dg, u, t, M, cells):
    """Smallest distance of a TVB-minmod decision of the listed patch cells
    from a tie, relative to the size of the compared numbers.  Per cell,
    direction and characteristic field (the oracle's reading: a1 the slope
    mode, a2/a3 the forward/backward average differences, projected with the
    left eigenvectors at the cell average) the decision flips where
    |a1| = M h^2 (the TVB threshold) or, above it, where |a1| equals the
    smaller of |a2|, |a3| with all signs equal (minmod returns a1 itself:
    not troubled, else troubled).  Each distance is divided by the largest
    magnitude entering it, the sum of |L_fj| |u_j| over the projected
    vector."""
    from oracle.limiter import neighbour_averages
    avg = u[..., 0]
    nb = neighbour_averages(dg, avg, t)
    best = np.inf
    for (cy, cx) in cells:
        ab = avg[cy, cx]
        for axis, (m, hi, lo, h) in enumerate(((1, "E", "W", dg.dx), (2, "N", "S", dg.dy))):
            L = np.linalg.inv(dg.phys.right_eigenvectors(ab, axis))
            vecs = (u[cy, cx, :, m], nb[hi][cy, cx] - ab, ab - nb[lo][cy, cx])
            a = [L @ v for v in vecs]
            scale = [np.abs(L) @ np.abs(v) for v in vecs]
            thr = M * h * h
            for f in range(4):
                best = min(best, abs(abs(a[0][f]) - thr) / max(thr, scale[0][f], 1e-300))
                same = np.sign(a[1][f]) == np.sign(a[0][f]) == np.sign(a[2][f])
                if abs(a[0][f]) > thr and same:
                    other = min(abs(a[1][f]), abs(a[2][f]))
                    sc = max(scale[0][f], scale[1][f], scale[2][f], 1e-300)
                    best = min(best, abs(abs(a[0][f]) - other) / sc)
    return best


def positivity_root_tie(dg, lim_cell, got_cell, eps, e32=2.0 ** -24):
    """Whether an FP32 result `got_cell` [v, m] of the positivity scaling that
    misses the value band against the oracle is the oracle's scaling with its
    pressure factor taken within FP32 rounding of a near-double root.

    The scaling (Zhang and Shu, applied after the TVB limiter; `lim_cell` is
    its input) multiplies the density's non-constant modes by theta1 and then
    every non-constant mode by theta2, the smallest root in (0, 1] of
    a t^2 + b t + c over the points where the pressure at t = 1 is below eps.
    A root r = (-b -+ sqrt(D)) / 2a moves by dD / (4 |a| sqrt(D)) when the
    discriminant D = b^2 - 4ac moves by dD; FP32 rounding of b^2 and 4ac
    gives dD of a few e32 (b^2 + 4|ac|), so the root moves by about
    e32 (b^2 + 4|ac|) / D * |r2 - r1| / 4, large where the roots nearly
    coincide (D small against b^2).  theta1 is a well-conditioned quotient.

    Accepted when: the cell average is unchanged; the non-constant modes are
    those of `lim_cell` times theta2' (and the oracle's theta1 for the
    density) to FP32 rounding; and |theta2' - theta2| is within 4 e32
    (b^2 + 4|ac|) / D |r2 - r1| + 1e-6 at the point that binds theta2."""
    from oracle.limiter import positivity_points
    P = positivity_points(dg)
    lim = np.asarray(lim_cell, dtype=np.float64)
    got = np.asarray(got_cell, dtype=np.float64)
    g = dg.phys.gamma
    if not np.array_equal(got[:, 0], lim[:, 0]):
        return False
    # theta1 and the points' quadratics, in FP64
    rho = P @ lim[0]
    rb = lim[0, 0]
    th1 = min(1.0, (rb - eps) / (rb - rho.min())) if rho.min() < eps else 1.0
    u = lim.copy()
    u[0, 1:] *= th1
    d = (u @ P.T) - u[:, :1]
    ub = u[:, 0]
    k = eps / (g - 1.0)
    a = d[0] * d[-1] - 0.5 * np.sum(d[1:-1] ** 2, axis=0)
    b = ub[0] * d[-1] + ub[-1] * d[0] - ub[1:-1] @ d[1:-1] - k * d[0]
    c = ub[0] * ub[-1] - 0.5 * np.sum(ub[1:-1] ** 2) - k * ub[0]
    th2, bound = 1.0, 1e-6
    for q in np.where(a + b + c < 0.0)[0]:
        D = b[q] * b[q] - 4.0 * a[q] * c
        sq = np.sqrt(max(D, 0.0))
        qq = -0.5 * (b[q] + (sq if b[q] >= 0 else -sq))
        roots = [r for r in ((c / qq) if qq != 0 else np.inf, (qq / a[q]) if a[q] != 0 else np.inf) if 0 < r <= 1]
        r = min(roots) if roots else 0.0
        if r < th2:
            th2 = r
            spread = sq / abs(a[q]) if a[q] != 0 else 0.0
            bound = 4.0 * e32 * (b[q] * b[q] + 4.0 * abs(a[q] * c)) / max(D, 1e-300) * spread + 1e-6
    # theta2' of the result: the momentum and energy modes' common factor
    sel = [(v, m) for v in range(1, lim.shape[0]) for m in range(1, lim.shape[1])
           if abs(lim[v, m]) > 1e-3 * np.max(np.abs(lim[v, 1:]))]
    th2g = float(np.median([got[v, m] / lim[v, m] for v, m in sel]))
    for v in range(lim.shape[0]):
        f = th2g * (th1 if v == 0 else 1.0)
        if np.max(np.abs(got[v, 1:] - f * lim[v, 1:])) > 4e-6 * max(np.max(np.abs(lim[v])), 1e-30):
            return False
    return abs(th2g - th2) <= bound
