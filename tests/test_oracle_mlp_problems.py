"""Pins of the oracle MLP (finite differences, closed forms) and of the
problem data (exact solutions satisfy the PDE; Rankine--Hugoniot balance)."""
import math

import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import mlp
from oracle.physics import Euler
from oracle.problems import isentropic_vortex


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    P = mlp.init_params(rng, sizes=(40, 16, 16, 16, 1))
    X = rng.normal(size=(12, 40))
    y = (rng.uniform(size=12) < 0.4).astype(float)

    def loss(P):
        z, _ = mlp.forward(P, X)
        return mlp.bce_with_logits(z, y, pos_weight=3.0)[0]

    z, cache = mlp.forward(P, X)
    _, dz = mlp.bce_with_logits(z, y, pos_weight=3.0)
    g = mlp.backward(P, cache, dz)
    for key in ("W", "b"):
        for l in range(4):
            A = P[key][l]
            idx = [tuple(rng.integers(0, s) for s in A.shape) for _ in range(4)]
            for ix in idx:
                old = A[ix]
                A[ix] = old + 1e-6
                lp = loss(P)
                A[ix] = old - 1e-6
                lm = loss(P)
                A[ix] = old
                fd = (lp - lm) / 2e-6
                assert abs(fd - g[key][l][ix]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9


def test_bce_closed_forms():
    z = np.zeros(4)
    y = np.array([0.0, 1.0, 0.0, 1.0])
    L, dz = mlp.bce_with_logits(z, y, pos_weight=1.0)
    assert L == pytest.approx(math.log(2.0))
    assert np.allclose(dz, (0.5 - y) / 4)


def test_adam_first_step_is_signed_lr():
    P = {"W": [np.array([[1.0, -2.0]])], "b": [np.array([0.5])]}
    G = {"W": [np.array([[0.3, -4.0]])], "b": [np.array([-1e-3])]}
    st = {}
    mlp.adam_update(P, G, st, lr=0.01, eps=0.0)
    assert np.allclose(P["W"][0], [[0.99, -1.99]])
    assert np.allclose(P["b"][0], [0.51])


def test_features_scale_invariance():
    """Scaling every deviation from the cell average by c > 0 leaves the 36
    normalised features unchanged and shifts the 4 scale features by log10 c."""
    rng = np.random.default_rng(1)
    u = rng.normal(size=(3, 3, 4, 6))
    nb = {s: rng.normal(size=(3, 3, 4)) for s in "EWNS"}
    f1 = mlp.features(u, nb, 50.0, 0.01)
    c = 7.0
    u2 = u.copy()
    u2[..., 1:] *= c
    nb2 = {s: u[..., 0] + c * (nb[s] - u[..., 0]) for s in nb}
    f2 = mlp.features(u2, nb2, 50.0, 0.01)
    assert np.allclose(f1[:, :36], f2[:, :36])
    assert np.allclose(f2[:, 36:], np.clip(f1[:, 36:] + math.log10(c), -8, 8))


def test_vortex_is_an_exact_solution():
    """Residual of u_t + f_x + g_y by central differences is O(h^2)."""
    ph = Euler(1.4, 2)
    X, Y = np.meshgrid(np.linspace(3, 7, 9), np.linspace(3, 7, 9), indexing="xy")
    res = []
    for h in (1e-2, 5e-3):
        ut = (isentropic_vortex(X, Y, 0.3 + h) - isentropic_vortex(X, Y, 0.3 - h)) / (2 * h)
        fx = (ph.flux(isentropic_vortex(X + h, Y, 0.3), 0) - ph.flux(isentropic_vortex(X - h, Y, 0.3), 0)) / (2 * h)
        gy = (ph.flux(isentropic_vortex(X, Y + h, 0.3), 1) - ph.flux(isentropic_vortex(X, Y - h, 0.3), 1)) / (2 * h)
        res.append(np.max(np.abs(ut + fx + gy)))
    assert res[1] < 0.3 * res[0] and res[1] < 1e-3
    # the shared input module states the same field
    a = inp.vortex_ic(X, Y, 0.3)
    assert np.allclose(a, isentropic_vortex(X, Y, 0.3, period=(10, 10)), atol=1e-13)


def test_dmr_states_satisfy_rankine_hugoniot():
    """In the frame moving with the shock, mass, momentum and energy fluxes
    across the shock balance."""
    st = inp.dmr_states()
    ph = Euler(1.4, 2)
    n = np.array([math.cos(math.pi / 6), -math.sin(math.pi / 6)])
    s = st["shock_speed"]

    def frame_flux(U):
        rho, (w, v), p = ph.primitive(U)
        un = w * n[0] + v * n[1] - s
        E = p / 0.4 + 0.5 * rho * un * un
        return np.array([rho * un, rho * un * un + p, un * (E + p)])

    a, b = frame_flux(st["pre"]), frame_flux(st["post"])
    assert np.allclose(a, b, rtol=1e-13, atol=1e-12)
    rho2, (w2, v2), p2 = ph.primitive(st["post"])
    assert rho2 == pytest.approx(8.0) and p2 == pytest.approx(116.5)
    assert math.hypot(w2, v2) == pytest.approx(8.25)
    assert st["xspeed"] == pytest.approx(20 / math.sqrt(3))


def test_riemann_ensemble_is_reproducible_and_in_range():
    a = inp.riemann_ensemble(16)
    b = inp.riemann_ensemble(16)
    assert a == b
    for pr in a:
        assert pr["N"] in (64, 128, 256, 512)
        for (rho, w, v, p) in pr["prim"]:
            assert 0.1 <= rho <= 1.5 and 0.1 <= p <= 1.5 and -1 <= w <= 1 and -1 <= v <= 1


def test_splitmix64_reference_values():
    """First outputs for seed 1234567, as published with the generator's
    reference implementation."""
    g = inp.SplitMix64(1234567)
    got = [g.next_u64() for _ in range(3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]
