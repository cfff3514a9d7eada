"""The isentropic-vortex configuration at its full size (320 x 320 Q^2 cells,
classical RK4, periodic [0,10]^2, CFL 0.1; the largest mesh of the FP32 /
FP64 convergence and matched-L1 comparison), every output element of the
CUDA path (the default launch shape of a solver of that mesh) against the
FP64 oracle run on the whole mesh: three steps from the oracle's projection
of the vortex, with the oracle's CFL time step.

Bands: FP64 1e-12 (rel_err per variable); the deviation form (CRKDG_F32D)
2e-6 of the three steps' increment and 1e-7 of the state (the bands of
tests/test_gpu_deviation.py, derived there); plain FP32 2e-5 of the state
(it misses the increment band: its flux roundings are O(eps |f|), the
reason the deviation form exists)."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import tableaux as OTB
from oracle.dg2d import cfl_dt_2d, crkdg_step
from tests.pairing import from_planes, make_pair_2d, rel_err, to_planes

pytestmark = pytest.mark.gpu

N, STEPS, CFL = 320, 3, 0.1
PER = {s: ("periodic",) for s in "WESN"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def oracle_run():
    gs, dg = make_pair_2d(N, N, (0, 10, 0, 10), 2, "Q", "euler", "rk4", PER, "f64")
    gs.close()
    u0 = dg.project(lambda X, Y: inp.vortex_ic(X, Y))
    dt = cfl_dt_2d(dg, u0, CFL)
    w, t = u0.copy(), 0.0
    for _ in range(STEPS):
        w = crkdg_step(dg, w, t, dt, OTB.RK4)
        t += dt
    return u0, dt, w


def _inc_err(got, want, u):
    d = np.moveaxis(got - want, -2, 0)
    w = np.moveaxis(want - u, -2, 0)
    return max(float(np.max(np.abs(d[v]))) / float(np.max(np.abs(w[v]))) for v in range(d.shape[0]))


@pytest.mark.parametrize("prec", ["f64", "f32d", "f32"])
def test_vortex_320_every_cell_against_the_oracle(prec, oracle_run):
    u0, dt, want = oracle_run
    gs, _ = make_pair_2d(N, N, (0, 10, 0, 10), 2, "Q", "euler", "rk4", PER, prec)
    gs.set_state(to_planes(u0), 0.0)
    m0 = gs.conservation()
    for _ in range(STEPS):
        gs.step(dt)
    got = from_planes(gs.get_state())
    m1 = gs.conservation()
    assert gs.sync() == (0, 0)
    gs.close()
    if prec == "f64":
        assert rel_err(got, want) < 1e-12
        assert np.max(np.abs(m1 - m0) / np.abs(m0)) < 1e-13
    elif prec == "f32d":
        assert _inc_err(got, want, u0) < 2e-6
        assert rel_err(got, want) < 1e-7
        assert np.max(np.abs(m1 - m0) / np.abs(m0)) < 1e-10
    else:
        assert rel_err(got, want) < 2e-5
