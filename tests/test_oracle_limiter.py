"""Pins of the oracle's TVB-minmod limiter (reading of Sec. 4.2; the paper
does not print the limiter, so these are invariants, not printed values)."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import tableaux as TB
from oracle.dg2d import DG2D, crkdg_step
from oracle.limiter import make_limiter, minmod3, tvb_limit
from oracle.physics import Advection, Euler

PER = {s: "periodic" for s in "WESN"}
OUT = {s: "outflow" for s in "WESN"}


def test_minmod_closed_forms():
    assert minmod3(np.array(1.0), np.array(2.0), np.array(3.0)) == 1.0
    assert minmod3(np.array(-3.0), np.array(-2.0), np.array(-5.0)) == -2.0
    assert minmod3(np.array(1.0), np.array(-2.0), np.array(3.0)) == 0.0
    assert minmod3(np.array(0.0), np.array(1.0), np.array(1.0)) == 0.0


def test_eigenvectors_diagonalise_the_jacobian():
    """R diag(lambda) R^{-1} equals the flux Jacobian, obtained here by
    central differences of the flux."""
    ph = Euler(1.4, 2)
    u = inp.conserved(1.3, 0.4, -0.7, 2.1)
    for axis in (0, 1):
        R = ph.right_eigenvectors(u, axis)
        rho, vel, p = ph.primitive(u)
        c = np.sqrt(1.4 * p / rho)
        vn = vel[axis]
        lam = np.diag([vn - c, vn, vn, vn + c])
        J = np.empty((4, 4))
        for j in range(4):
            e = np.zeros(4)
            e[j] = 1e-6
            J[:, j] = (ph.flux(u + e, axis) - ph.flux(u - e, axis)) / 2e-6
        assert np.allclose(R @ lam @ np.linalg.inv(R), J, atol=1e-7)


def _euler_dg(n=10, bc=PER, k=2):
    return DG2D(n, n, (0, 1, 0, 1), k, "P", Euler(1.4, 2), bc)


def test_averages_are_preserved_and_high_modes_cleared():
    dg = _euler_dg()
    u = inp.random_modal_state(10, 10, 2, "P", "euler", seed=11, amp=0.8)
    v, flags = tvb_limit(dg, u, 0.0, 0.0)
    assert flags.any()
    assert np.array_equal(v[..., 0], u[..., 0])
    assert np.all(v[flags][..., 3:] == 0)
    assert np.array_equal(v[~flags], u[~flags])


def test_smooth_data_with_large_M_is_untouched():
    dg = _euler_dg()
    u = inp.random_modal_state(10, 10, 2, "P", "euler", seed=12)
    v, flags = tvb_limit(dg, u, 1e8, 0.0)
    assert not flags.any()
    assert np.array_equal(u, v)


def test_linear_data_is_not_flagged():
    """A linear function: a1 equals both neighbour differences (in scalar and
    in characteristic fields alike), so minmod returns a1."""
    dg = DG2D(8, 8, (0, 1, 0, 1), 2, "P", Advection([1.0, 1.0]), OUT)
    u = dg.project(lambda X, Y: (2 * X - 3 * Y)[..., None])
    # the outflow ghost copies the cell itself: drop the boundary ring
    v, flags = tvb_limit(dg, u, 0.0, 0.0)
    assert not flags[1:-1, 1:-1].any()


def test_step_profile_flags_only_cells_at_the_jump():
    dg = _euler_dg(n=12, bc=OUT)
    u = dg.project(lambda X, Y: np.where((X < 0.52)[..., None], inp.conserved(1.0, 0, 0, 1.0),
                                         inp.conserved(0.125, 0, 0, 0.1)))
    # M h^2 > 0 keeps roundoff-level slopes of the constant cells unflagged
    v, flags = tvb_limit(dg, u, 1.0, 0.0)
    # the jump sits inside column 6; its neighbours are constant (a1 = 0)
    assert flags[:, 6].all()
    assert not flags[:, :6].any() and not flags[:, 7:].any()


def test_limiter_is_idempotent_on_its_output():
    dg = _euler_dg()
    u = inp.random_modal_state(10, 10, 2, "P", "euler", seed=13, amp=0.8)
    v, _ = tvb_limit(dg, u, 10.0, 0.0)
    w, _ = tvb_limit(dg, v, 10.0, 0.0)
    assert np.max(np.abs(w - v)) < 1e-12


def test_conservation_with_limiter():
    dg = _euler_dg(n=8)
    u = inp.random_modal_state(8, 8, 2, "P", "euler", seed=14, amp=0.2)
    lim = make_limiter(dg, 1.0)
    m0 = dg.total(u)
    for _ in range(5):
        u = crkdg_step(dg, u, 0.0, 0.002, TB.SSPRK3, limiter=lim)
    assert np.all(np.abs(dg.total(u) - m0) <= 1e-13 * np.abs(m0))


def test_reflective_ghost_negates_normal_momentum():
    from oracle.limiter import neighbour_averages
    bc = {"W": "reflect", "E": "reflect", "S": "reflect", "N": "reflect"}
    dg = _euler_dg(n=4, bc=bc)
    u = inp.random_modal_state(4, 4, 2, "P", "euler", seed=15)
    nb = neighbour_averages(dg, u[..., 0], 0.0)
    a = u[..., 0]
    assert np.allclose(nb["W"][:, 0, 1], -a[:, 0, 1]) and np.allclose(nb["W"][:, 0, 2], a[:, 0, 2])
    assert np.allclose(nb["N"][-1, :, 2], -a[-1, :, 2]) and np.allclose(nb["N"][-1, :, 1], a[-1, :, 1])


# -- positivity-preserving scaling (Zhang and Shu 2010; an option outside the paper) --------
def test_positivity_scaling_closed_form_density():
    """P^1 density rho = rb + s xi with s > rb: the smallest point value is at
    the east/west faces, rb - s, so theta_1 = (rb - eps) / s exactly."""
    from oracle.limiter import positivity_limit
    dg = DG2D(1, 1, (0, 1, 0, 1), 1, "P", Euler(1.4, 2), PER)
    rb, s, eps = 1.0, 3.0, 1e-10
    u = np.zeros((1, 1, 4, 3))
    u[0, 0, :, 0] = inp.conserved(rb, 0.0, 0.0, 10.0)
    u[0, 0, 0, 1] = s
    v = positivity_limit(dg, u, eps)
    assert v[0, 0, 0, 1] == pytest.approx(s * (rb - eps) / s, rel=1e-14)
    assert np.array_equal(v[..., 0], u[..., 0])


def test_positivity_scaling_closed_form_pressure():
    """theta_2 from a quadratic worked by hand.  P^1 state with averages
    rho = 1, rho w = 1, rho v = 0, E = 0.6 (p = 0.04) and xi-slopes
    d rho = 0.3, d(rho w) = 0.8 (all other slopes 0).  Along the segment
    ubar + t (u_q - ubar) to a point with xi = 1 (every east-face point)
        rho(t) = 1 + 0.3 t,   rho w(t) = 1 + 0.8 t,   E(t) = 0.6,
    and p(t) = eps, i.e. rho (E - k) - (rho w)^2 / 2 = 0 with k = eps/(gamma-1):
        (1 + 0.3 t)(0.6 - k) - (1 + 0.8 t)^2 / 2 = 0
        <=>  0.32 t^2 + (0.8 - 0.3 (0.6 - k)) t - (0.1 - k) = 0.
    A point with xi = x in (0, 1) reaches the same state at t / x, later; the
    west points (xi < 0) have positive pressure (rho w < 1 there), and the
    density stays >= 0.7, so theta_1 = 1 and theta_2 is the positive root.
    Every non-constant mode of every variable is scaled by theta_2."""
    from oracle.limiter import positivity_limit, positivity_points
    dg = DG2D(1, 1, (0, 1, 0, 1), 1, "P", Euler(1.4, 2), PER)
    eps = 1e-3
    k = eps / 0.4
    u = np.zeros((1, 1, 4, 3))
    u[0, 0, :, 0] = (1.0, 1.0, 0.0, 0.6)
    u[0, 0, 0, 1] = 0.3
    u[0, 0, 1, 1] = 0.8
    a, b, c = 0.32, 0.8 - 0.3 * (0.6 - k), -(0.1 - k)
    theta = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)
    assert 0.1 < theta < 0.2
    v = positivity_limit(dg, u, eps)
    assert np.array_equal(v[..., 0], u[..., 0])
    assert v[0, 0, 0, 1] == pytest.approx(0.3 * theta, rel=1e-12)
    assert v[0, 0, 1, 1] == pytest.approx(0.8 * theta, rel=1e-12)
    assert np.all(v[0, 0, 2:, 1:] == 0.0) and np.all(v[0, 0, :2, 2] == 0.0)
    # the east-face points land on p = eps exactly, no point below it
    rho, _, p = dg.phys.primitive(np.einsum("yxvm,qm->yxqv", v, positivity_points(dg)))
    assert p.min() == pytest.approx(eps, rel=1e-9)
    assert rho.min() > 0.9


def test_positivity_scaling_invariants():
    from oracle.limiter import positivity_limit, positivity_points
    dg = _euler_dg(n=12)
    u = inp.random_modal_state(12, 12, 2, "P", "euler", seed=31)
    assert np.array_equal(positivity_limit(dg, u), u)        # physical data untouched
    bad = u.copy()
    bad[..., 1:] *= 40.0                                     # large oscillations: negative p, rho
    P = positivity_points(dg)
    uq = np.einsum("yxvm,qm->yxqv", bad, P)
    assert (dg.phys.primitive(uq)[2] < 0).any()
    v = positivity_limit(dg, bad, 1e-10)
    assert np.array_equal(v[..., 0], bad[..., 0])
    rho, _, p = dg.phys.primitive(np.einsum("yxvm,qm->yxqv", v, P))
    assert rho.min() >= 1e-10 * (1 - 1e-6) and p.min() >= 1e-10 * (1 - 1e-3) - 1e-12


def _x_profile_state(avg, a1, nm=6, ny=3, hi=0.1):
    """Scalar P^2 state on a periodic 4 x 3 mesh of [0,1]^2, constant in y:
    cell averages avg[x], x-slope coefficients a1[x], y-slopes 0, every
    second-degree mode hi."""
    u = np.zeros((ny, len(avg), 1, nm))
    for x in range(len(avg)):
        u[:, x, 0, 0] = avg[x]
        u[:, x, 0, 1] = a1[x]
    u[..., 3:] = hi
    return u


@pytest.mark.parametrize("M,flagged,slopes", [
    # worked by hand (periodic, dx = 1/4): cell 0 sees differences (+1, -6),
    # cell 1 (+2, +1), cell 2 (+3, +2), cell 3 (-6, +3)
    (0.0, [True, True, False, True], [0.0, 1.0, 1.0, 0.0]),
    # M dx^2 = 0.25: |a1| = 0.2 of cell 3 is below it and stays
    (4.0, [True, True, False, False], [0.0, 1.0, 1.0, -0.2]),
])
def test_scalar_tvb_minmod_worked_example(M, flagged, slopes):
    dg = DG2D(4, 3, (0, 1, 0, 1), 2, "P", Advection([1.0, 0.0]), PER)
    u = _x_profile_state([0.0, 1.0, 3.0, 6.0], [0.5, 2.0, 1.0, -0.2])
    v, flags = tvb_limit(dg, u, M, 0.0)
    assert np.array_equal(flags, np.tile(np.array(flagged), (3, 1)))
    for x in range(4):
        assert np.all(v[:, x, 0, 1] == slopes[x])
        assert np.all(v[:, x, 0, 2] == 0.0)                       # y-slopes stay 0
        assert np.all(v[:, x, 0, 3:] == (0.0 if flagged[x] else 0.1))
        assert np.all(v[:, x, 0, 0] == u[:, x, 0, 0])


def test_euler_entropy_wave_limits_like_scalar_density():
    """At rest with uniform pressure, a density-only profile lies entirely in
    the entropy field (its left eigenvector row is (1, 0, 0, -b1) with the
    energy slope 0, the acoustic rows vanish on it), so the characteristic
    limiter acts on the density slope exactly as the scalar minmod and leaves
    momentum and energy slopes at 0."""
    dg = DG2D(4, 3, (0, 1, 0, 1), 2, "P", Euler(1.4, 2), PER)
    avg_rho = [1.0, 2.0, 4.0, 7.0]
    a1 = [0.5, 2.0, 1.0, -0.2]
    u = np.zeros((3, 4, 4, 6))
    for x in range(4):
        u[:, x, :, 0] = inp.conserved(avg_rho[x], 0.0, 0.0, 1.0)
        u[:, x, 0, 1] = a1[x]
    v, flags = tvb_limit(dg, u, 0.0, 0.0)
    assert np.array_equal(flags, np.tile(np.array([True, True, False, True]), (3, 1)))
    want = [0.0, 1.0, 1.0, 0.0]
    for x in range(4):
        assert np.allclose(v[:, x, 0, 1], want[x], rtol=0, atol=1e-12)
        assert np.allclose(v[:, x, 1:, 1], 0.0, rtol=0, atol=1e-12)
        assert np.allclose(v[:, x, :, 2], 0.0, rtol=0, atol=1e-12)
