"""Algorithmic work of one fused cRKDG step per cell (for roofline figures).

Counts the floating-point operations of the quadrature form of one cRKDG
step for one interior cell (halo recomputation excluded): every point
value, face trace and projection as a direct sum over the modes, as eq.
(2.3) and (2.7) define them; an FMA counts 2, add/sub/mul/div/sqrt/max
count 1.  Products with a zero derivative-table entry are not counted;
products with zero point values are.  The count is the method's and does
not follow implementation shortcuts: the 2D step kernel forms the east/west
(north/south) traces and face projections from even- and odd-mode partial
sums (phi_m(-1, eta) = (-1)^i phi_m(1, eta)), about 13 % fewer operations
for P^2 than counted here.

Bytes: u^n is read once and u^{n+1} written once per cell: 2 * NDOF * size,
plus, with the limiter, the neighbours' averages (served by L1/L2 in the
kernel, so not counted as algorithmic traffic).
"""
import numpy as np
from numpy.polynomial import legendre as L

FLUX2 = {"euler": 18, "advection": 2}     # both axes at one point
FLUXN = {"euler": 17, "advection": 1}     # one axis + wave speed
LIMITER = {"euler": 2 * (40 + 3 * 32 + 4 * 8 + 32), "advection": 2 * 12}


def _modes(k, basis):
    out = []
    dmax = k if basis == "P" else 2 * k
    for d in range(dmax + 1):
        for i in range(d, -1, -1):
            if i <= k and d - i <= k:
                out.append((i, d - i))
    return out


def _nonzero_derivative_entries(k, basis):
    x, w = L.leggauss(k + 1)
    leg = lambda i, t: L.legval(t, np.eye(k + 1)[i])
    dleg = lambda i, t: L.legval(t, L.legder(np.eye(k + 1)[i])) if i > 0 else 0.0 * t
    n = 0
    for (i, j) in _modes(k, basis):
        for a in range(k + 1):
            for b in range(k + 1):
                gx = w[a] * w[b] * dleg(i, x[a]) * leg(j, x[b])
                gy = w[a] * w[b] * leg(i, x[a]) * dleg(j, x[b])
                n += (abs(gx) > 1e-15) + (abs(gy) > 1e-15)
    return n


def step_flops_per_cell(k, basis, physics, A, b, limiter=False):
    """FLOPs of one cRKDG step for one cell (2D)."""
    nv = 4 if physics == "euler" else 1
    nq = k + 1
    nqv = nq * nq
    nm = len(_modes(k, basis))
    ndof = nv * nm
    s = len(b)
    nzd = _nonzero_derivative_entries(k, basis)
    f = 0
    for i in range(s):
        need_L = i < s - 1
        need_flux = b[i] != 0.0
        if not (need_L or need_flux):
            continue
        f += sum(2 * ndof + 1 for j in range(i) if A[i][j] != 0.0)     # stage state
        f += 2 * nqv * nv * nm + nqv * FLUX2[physics]                   # evaluate + flux
        f += nqv * 2 * nv + 2 * nzd * nv                                 # volume projection
        f += 4 * 2 * nq * nv * nm                                        # face traces
        if need_L:
            f += 4 * nq * FLUXN[physics] + 8 * nq * nv * nm + 2 * ndof   # local face terms, L_i
        if need_flux:
            f += 2 * ndof                                                # b_i * volume
            f += 2 * nq * (2 * FLUXN[physics] + 1 + 5 * nv)              # LLF on E and S faces
    f += ndof * (6 * nq + 5) + ndof * (2 * nq + 3)                       # final update, north face
    if limiter:
        f += LIMITER[physics]
    return f


def step_bytes_per_cell(k, basis, physics, elem_bytes):
    nv = 4 if physics == "euler" else 1
    return 2 * nv * len(_modes(k, basis)) * elem_bytes
