"""Error norms of a DG solution against an exact function.

The paper prints L^2 and L^infinity errors (Sec. 4) without stating the
normalisation.  Reading taken (pinned against Table 4.4): the L^2 norm is the
plain integral norm, (int |e|^2)^{1/2}, and L^infinity is the maximum of |e|
over the sample points; both are computed with an nq-point Gauss rule per
direction in every cell (default nq = 5).  L^1 is reported both as the
integral and divided by |Omega| (mean absolute error).  Test infrastructure.
"""
import numpy as np

from .basis import Basis1D, gauss, leg


def errors_1d(dg, u, exact, var=0, nq=5):
    """exact(x) -> (..., nv).  Returns dict(L1, L1_mean, L2, Linf)."""
    xq, wq = gauss(nq)
    x = dg.xc[:, None] + 0.5 * dg.h[:, None] * xq[None, :]
    phi = np.stack([leg(m, xq) for m in range(dg.k + 1)], axis=1)
    uh = np.einsum("xvm,qm->xqv", u, phi)[..., var]
    ue = np.asarray(exact(x), dtype=np.float64).reshape(dg.n, nq, -1)[..., var]
    e = np.abs(uh - ue)
    jac = 0.5 * dg.h[:, None] * wq[None, :]
    vol = np.sum(dg.h)
    l1 = np.sum(jac * e)
    return {"L1": l1, "L1_mean": l1 / vol, "L2": np.sqrt(np.sum(jac * e * e)),
            "Linf": np.max(e)}


def errors_2d(dg, u, exact, var=0, nq=5, mask=None):
    """exact(x, y) -> (..., nv) on the 2D mesh of ``dg``.  Same keys.
    ``mask`` (ny, nx) restricts the norms to the selected cells."""
    xq, wq = gauss(nq)
    X = dg.xc[None, :, None, None] + 0.5 * dg.dx * xq[None, None, :, None]
    Y = dg.yc[:, None, None, None] + 0.5 * dg.dy * xq[None, None, None, :]
    X, Y = np.broadcast_arrays(X, Y)
    phi = np.stack([leg(i, xq)[:, None] * leg(j, xq)[None, :] for (i, j) in dg.B.modes], axis=-1)
    uh = np.einsum("yxvm,abm->yxabv", u, phi)[..., var]
    ue = np.asarray(exact(X, Y), dtype=np.float64)[..., var]
    e = np.abs(uh - ue)
    w2 = (wq[:, None] * wq[None, :]) * (0.25 * dg.dx * dg.dy)
    vol = dg.nx * dg.ny * dg.dx * dg.dy
    if mask is not None:
        e = e[mask]
        vol = np.count_nonzero(mask) * dg.dx * dg.dy
    l1 = np.sum(w2 * e)
    return {"L1": l1, "L1_mean": l1 / vol, "L2": np.sqrt(np.sum(w2 * e * e)),
            "Linf": np.max(e)}
