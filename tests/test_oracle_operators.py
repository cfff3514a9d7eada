"""Pins of the oracle's spatial operators and time steps against closed forms
and exact invariants of the paper (Sec. 2, Sec. 3.1--3.5)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import crkdg_inputs as inp
from oracle import tableaux as TB
from oracle.dg1d import DG1D, crkdg_step as crkdg1, rkdg_step as rkdg1
from oracle.dg2d import DG2D, crkdg_step as crkdg2, rkdg_step as rkdg2
from oracle.physics import Advection, Euler

PER = {s: "periodic" for s in "WESN"}


def test_local_operator_1d_is_exact_derivative():
    """div^loc(beta u) = Pi d/dx(beta u) = beta u' for u in P^k (Sec. 2.2)."""
    rng = np.random.default_rng(1)
    k, N, beta = 3, 6, -1.7
    nodes = np.sort(rng.uniform(0, 1, N + 1))
    dg = DG1D(nodes, k, Advection([beta]))
    u = rng.normal(size=(N, 1, k + 1))
    L = dg.L_loc(u)
    for j in range(N):
        d = npleg.legder(u[j, 0]) * 2.0 / dg.h[j] * beta
        d = np.concatenate([d, np.zeros(k + 1 - len(d))])
        assert np.max(np.abs(L[j, 0] - d)) < 1e-11 * max(1, np.max(np.abs(d)))


@pytest.mark.parametrize("basis", ["P", "Q"])
def test_local_operator_2d_is_exact_derivative(basis):
    """Same identity in 2D: beta_x u_x + beta_y u_y, computed here from the
    Legendre series by numpy's legder in each direction."""
    rng = np.random.default_rng(2)
    k, bx, by = 3, 0.6, -1.3
    dg = DG2D(3, 2, (0, 1.5, 0, 1.0), k, basis, Advection([bx, by]), PER)
    u = rng.normal(size=(2, 3, 1, dg.B.nm))
    L = dg.L_loc(u)
    idx = {mn: m for m, mn in enumerate(dg.B.modes)}
    for y in range(2):
        for x in range(3):
            C = np.zeros((k + 1, k + 1))
            for m, (i, j) in enumerate(dg.B.modes):
                C[i, j] = u[y, x, 0, m]
            dX = npleg.legder(C, axis=0) * 2 / dg.dx
            dY = npleg.legder(C, axis=1) * 2 / dg.dy
            D = np.zeros((k + 1, k + 1))
            D[: dX.shape[0], :] += bx * dX
            D[:, : dY.shape[1]] += by * dY
            for (i, j), m in idx.items():
                assert abs(L[y, x, 0, m] - D[i, j]) < 1e-11
            # the derivative of a P^k polynomial has no component outside P^k
            for i in range(k + 1):
                for j in range(k + 1):
                    if (i, j) not in idx:
                        assert abs(D[i, j]) < 1e-11


def test_free_stream_is_preserved():
    """A constant state: div^loc f = div^DG f = 0 (consistency of the flux)."""
    ph = Euler(1.4, 2)
    dg = DG2D(5, 4, (0, 1, 0, 1), 2, "Q", ph, PER)
    u = np.zeros((4, 5, 4, dg.B.nm))
    u[..., 0] = inp.conserved(1.3, 0.4, -0.2, 0.9)
    assert np.max(np.abs(dg.L_loc(u))) < 1e-12
    assert np.max(np.abs(dg.L_dg(u, 0.0))) < 1e-12


def fv_forward_euler_lf(avg, dt, dx, dy, phys):
    """First-order finite-volume forward Euler with the local LF flux, written
    independently of the DG code: the k = 0 limit of cRKDG."""
    def F(a, b, axis):
        fa = phys.flux(a, axis)
        fb = phys.flux(b, axis)
        al = np.maximum(phys.speed(a, axis), phys.speed(b, axis))
        return 0.5 * (fa + fb) - 0.5 * al[..., None] * (b - a)
    Fx = F(avg, np.roll(avg, -1, axis=1), 0)  # flux through east faces
    Fy = F(avg, np.roll(avg, -1, axis=0), 1)
    return avg - dt / dx * (Fx - np.roll(Fx, 1, axis=1)) - dt / dy * (Fy - np.roll(Fy, 1, axis=0))


@pytest.mark.parametrize("tab", [TB.HEUN3, TB.SSPRK3, TB.RK4, TB.MIDPOINT])
def test_k0_collapses_to_forward_euler_fv(tab):
    """P^0: div^loc f = 0 (Sec. 3.3), every inner stage equals u^n and, since
    sum b_i = 1, cRKDG is forward-Euler LF finite volumes."""
    ph = Euler(1.4, 2)
    dg = DG2D(6, 5, (0, 1.2, 0, 1.0), 0, "P", ph, PER)
    u = inp.random_modal_state(5, 6, 0, "P", "euler", seed=3)
    assert np.max(np.abs(dg.L_loc(u))) == 0.0
    dt = 0.01
    a = crkdg2(dg, u, 0.0, dt, tab)[..., 0]
    b = fv_forward_euler_lf(u[..., 0], dt, dg.dx, dg.dy, ph)
    assert np.max(np.abs(a - b)) < 1e-13


def test_conservation_periodic_2d():
    """Cell-average form eq. (3.4): totals are conserved to roundoff."""
    ph = Euler(1.4, 2)
    dg = DG2D(8, 6, (0, 1, 0, 1), 2, "P", ph, PER)
    u = inp.random_modal_state(6, 8, 2, "P", "euler", seed=4)
    m0 = dg.total(u)
    for n in range(30):
        u = crkdg2(dg, u, 0.0, 0.002, TB.SSPRK3)
    m1 = dg.total(u)
    assert np.all(np.abs(m1 - m0) <= 1e-13 * np.abs(m0) + 1e-15)


def test_shu_osher_variant_breaks_conservation():
    """eq. (3.2): the Shu--Osher substitution updates with div^loc and is not
    conservative (Sec. 3.2.1) -- a negative control of the test above."""
    from oracle.dg1d import shu_osher_crkdg_wrong_step
    ph = Euler(1.4, 1)
    dg = DG1D(np.linspace(0, 1, 11), 1, ph)
    u = inp.random_modal_state_1d(10, 1, 3, seed=5, amp=0.2)
    tot = lambda v: np.sum(v[:, :, 0] * dg.h[:, None], axis=0)
    u1 = shu_osher_crkdg_wrong_step(dg, u, 0.0, 0.01, 2)
    assert np.max(np.abs(tot(u1) - tot(u))) > 1e-8
    u2 = crkdg1(dg, u, 0.0, 0.01, TB.HEUN)
    assert np.max(np.abs(tot(u2) - tot(u))) < 1e-14


def _changed_cells(a, b):
    return np.argwhere(np.any(a != b, axis=tuple(range(2, a.ndim))))


def test_stencil_1d_brute_force():
    """Proposition 3.1: cRKDG changes only the cell and its two neighbours;
    RKDG with s stages reaches 2s+1 cells (Fig. 3.1)."""
    ph = Euler(1.4, 1)
    N, j0 = 16, 8
    dg = DG1D(np.linspace(0, 1, N + 1), 2, ph)
    u = inp.random_modal_state_1d(N, 2, 3, seed=6)
    v = u.copy()
    v[j0] += 1e-3 * np.abs(u[j0])
    for tab in (TB.HEUN3, TB.RK4):
        a = crkdg1(dg, u, 0.0, 1e-3, tab)
        b = crkdg1(dg, v, 0.0, 1e-3, tab)
        ch = np.flatnonzero(np.any(a != b, axis=(1, 2)))
        assert list(ch) == [j0 - 1, j0, j0 + 1]
        a = rkdg1(dg, u, 0.0, 1e-3, tab)
        b = rkdg1(dg, v, 0.0, 1e-3, tab)
        ch = np.flatnonzero(np.any(a != b, axis=(1, 2)))
        s = tab["s"]
        assert list(ch) == list(range(j0 - s, j0 + s + 1))


def test_stencil_2d_brute_force():
    """2D: cRKDG reaches the 5-point stencil; RKDG the diamond |i|+|j| <= s."""
    ph = Euler(1.4, 2)
    n, c = 9, 4
    dg = DG2D(n, n, (0, 1, 0, 1), 1, "P", ph, PER)
    u = inp.random_modal_state(n, n, 1, "P", "euler", seed=7)
    v = u.copy()
    v[c, c] += 1e-3 * np.abs(u[c, c])
    tab = TB.SSPRK3
    a, b = crkdg2(dg, u, 0.0, 1e-3, tab), crkdg2(dg, v, 0.0, 1e-3, tab)
    got = {tuple(p) for p in _changed_cells(a, b)}
    assert got == {(c, c), (c - 1, c), (c + 1, c), (c, c - 1), (c, c + 1)}
    a, b = rkdg2(dg, u, 0.0, 1e-3, tab), rkdg2(dg, v, 0.0, 1e-3, tab)
    got = {tuple(p) for p in _changed_cells(a, b)}
    want = {(c + i, c + j) for i in range(-3, 4) for j in range(-3, 4) if abs(i) + abs(j) <= 3}
    assert got == want


def lwdg_form(dg, u, dt, p):
    """Eq. (3.9): u - dt div^DG(beta sum_{i<p} dt^i/(i+1)! L_h^i u),
    L_h = -div^loc(beta .): the LWDG form of Theorem 3.3."""
    acc = np.zeros_like(u)
    term = u.copy()
    fact = 1.0
    for i in range(p):
        fact *= (i + 1)
        acc = acc + dt ** i / fact * term
        term = -dg.L_loc(term)
    return u - dt * dg.L_dg(acc, 0.0)


@pytest.mark.parametrize("k,tabs", [(2, (TB.HEUN3, TB.SSPRK3)), (3, (TB.RK4, TB.RK38)), (1, (TB.MIDPOINT, TB.HEUN))])
def test_linear_update_is_tableau_independent_and_lwdg(k, tabs):
    """Theorem 3.3: for linear advection with the upwind flux every p-stage,
    p-th order tableau gives the same cRKDG update, equal to eq. (3.9)."""
    dg = DG2D(7, 5, (0, 1.4, 0, 1.0), k, "P", Advection([1.0, -0.5]), PER)
    u = inp.random_modal_state(5, 7, k, "P", "advection", seed=8)
    dt = 0.02
    ref = lwdg_form(dg, u, dt, tabs[0]["s"])
    for tab in tabs:
        got = crkdg2(dg, u, 0.0, dt, tab)
        assert np.max(np.abs(got - ref)) < 1e-13


def test_upwind_p0_advection_is_first_order_upwind():
    """For beta > 0 the LF flux is upwind (Remark 3.5): P^0 one step is
    u_j - lambda (u_j - u_{j-1})."""
    N = 12
    dg = DG1D(np.linspace(0, 1, N + 1), 0, Advection([2.0]))
    u = np.random.default_rng(9).normal(size=(N, 1, 1))
    dt = 0.01
    got = crkdg1(dg, u, 0.0, dt, TB.SSPRK3)[:, 0, 0]
    lam = 2.0 * dt * N
    want = u[:, 0, 0] - lam * (u[:, 0, 0] - np.roll(u[:, 0, 0], 1))
    assert np.max(np.abs(got - want)) < 1e-14


def test_rkdg_ssp_2d_matches_butcher_form_for_linear_problems():
    """For linear advection SSP-RK3 in Shu--Osher form and in Butcher form
    are the same method: one step agrees to roundoff."""
    from oracle.dg2d import rkdg_ssp_step
    dg = DG2D(7, 6, (0, 1.4, 0, 1.2), 2, "P", Advection([1.0, 0.5]), PER)
    u = inp.random_modal_state(6, 7, 2, "P", "advection", seed=31)
    a = rkdg_ssp_step(dg, u, 0.0, 0.01, 3)
    b = rkdg2(dg, u, 0.0, 0.01, TB.SSPRK3)
    assert np.max(np.abs(a - b)) < 1e-14
