"""The tie bands the FP32 parity tests use, pinned on the CPU: a cell whose
FP32 result may differ from the FP64 oracle is accepted only where FP32
rounding explains the difference.  The positivity root band (Zhang and Shu's
pressure factor theta2, the smallest root of a quadratic) accepts a factor
moved by the measured FP32 error at a near-double root and rejects the same
error at a well-conditioned root, and rejects a wrong density factor theta1,
a changed average or a result that is not a scaling of its input."""
import numpy as np

import crkdg_inputs as inp
from oracle.limiter import positivity_limit
from tests.pairing import DG2D, Euler, from_planes, oracle_bc, positivity_root_tie, to_planes

EPS = 1e-10


def _cells():
    """Rows 200..205 of the seeded random P^2 Euler state the limiter pass
    test uses (130 columns), rounded to FP32 as the FP32 path holds it; the
    positivity scaling is per cell, so a slice of rows stands alone."""
    u = inp.random_modal_state(2000, 130, 2, "P", "euler", seed=31, amp=0.5)[200:206]
    u = from_planes(to_planes(u).astype(np.float32).astype(np.float64))
    bc = {s: oracle_bc(("periodic",), 0 if s in ("W", "E") else 1) for s in "WESN"}
    dg = DG2D(130, 6, (0, 1, 0, 6 / 37.0), 2, "P", Euler(1.4, 2), bc)
    return dg, u, positivity_limit(dg, u, EPS)


def _scaled(cell, f_rho, f):
    out = cell.copy()
    out[0, 1:] *= f_rho
    out[1:, 1:] *= f
    return out


def test_positivity_root_band():
    dg, u, w = _cells()
    near = (3, 44)   # row 203: theta2's point has roots 0.9775 and 1.0020 (D / b^2 ~ 8e-5)
    assert not np.array_equal(w[near], u[near])
    assert positivity_root_tie(dg, u[near], w[near], EPS)
    # the FP32 pass's measured error at this cell (theta2 + 8.4e-6) is inside the band
    th2_err = 1.0 + 8.6e-6
    assert positivity_root_tie(dg, u[near], _scaled(w[near], th2_err, th2_err), EPS)
    # errors that FP32 rounding cannot make
    assert not positivity_root_tie(dg, u[near], _scaled(w[near], 1.001, 1.001), EPS)   # theta2
    assert not positivity_root_tie(dg, u[near], _scaled(w[near], 1.0001, 1.0), EPS)   # theta1
    avg = w[near].copy()
    avg[0, 0] *= 1.0 + 1e-7
    assert not positivity_root_tie(dg, u[near], avg, EPS)
    mixed = w[near].copy()
    mixed[1, 2] *= 1.001   # not one factor for every mode
    assert not positivity_root_tie(dg, u[near], mixed, EPS)
    # well-conditioned roots: the oracle's result is accepted, theta2 2e-5 off is not
    acted = np.argwhere(np.any(w != u, axis=(2, 3)))
    assert len(acted) >= 10
    n_well = 0
    for (cy, cx) in acted:
        if (cy, cx) == near:
            continue
        assert positivity_root_tie(dg, u[cy, cx], w[cy, cx], EPS)
        if not positivity_root_tie(dg, u[cy, cx], _scaled(w[cy, cx], 1 + 2e-5, 1 + 2e-5), EPS):
            n_well += 1
    assert n_well >= 10
