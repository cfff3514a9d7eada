"""Edge cases of the step on the GPU against the FP64 oracle: degenerate
meshes (one cell, one row, one column, two rows or columns: a cell that is
its own periodic neighbour, halo lanes and rows that wrap onto the cells
they border), a large mesh checked through a property that holds at any
size (data depending on x only gives identical rows, on y only identical
columns, and those equal the oracle's one-row / one-column run), and steps
of zero length (rejected on the host; copies on the device at t_end)."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import tableaux as OTB
from oracle.dg2d import cfl_dt_2d, crkdg_step
from tests.pairing import from_planes, make_pair_2d, rel_err, to_planes

pytestmark = pytest.mark.gpu

PER = {s: ("periodic",) for s in "WESN"}
OUT = {s: ("outflow",) for s in "WESN"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (7, 1), (31, 2), (2, 31), (30, 3)])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_degenerate_meshes_match_the_oracle(nx, ny, bc):
    gs, dg = make_pair_2d(nx, ny, (0, 1, 0, 1), 2, "P", "euler", "ssprk3", PER if bc == "periodic" else OUT, "f64")
    u = inp.random_modal_state(ny, nx, 2, "P", "euler", seed=60 + nx + ny)
    gs.set_state(to_planes(u), 0.0)
    dt = 0.2 * cfl_dt_2d(dg, u, 1.0)
    w, t = u, 0.0
    for _ in range(2):
        gs.step(dt)
        w = crkdg_step(dg, w, t, dt, OTB.SSPRK3)
        t += dt
    got = from_planes(gs.get_state())
    assert rel_err(got, w) < 1e-13
    assert gs.sync() == (0, 0)
    gs.close()


def _wave(X, Y, along):
    """A smooth periodic density/pressure wave moving with the flow along one
    axis, constant along the other."""
    s = X if along == "x" else Y
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * s)
    p = 1.0 + 0.1 * np.cos(2 * np.pi * s)
    w = np.full_like(s, 0.4) if along == "x" else np.full_like(s, 0.1)
    v = np.full_like(s, 0.1) if along == "x" else np.full_like(s, 0.4)
    return inp.conserved(rho, w, v, p)


@pytest.mark.parametrize("along", ["x", "y"])
def test_large_mesh_rows_and_columns_agree_with_a_thin_oracle_run(along):
    """FP32, 4096 x 2048 cells (x wave) or 2048 x 4096 (y wave) in the
    default launch shape, three steps: every row (column) equals the first
    bitwise — each computes the same arithmetic on the same data — and the
    first equals the oracle's 4096 x 1 (1 x 4096) periodic run within the
    FP32 band."""
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    n_long, n_short = 4096, 2048
    nx, ny = (n_long, n_short) if along == "x" else (n_short, n_long)
    mesh = B.make_mesh(2, nx, ny, (0.0, 1.0, 0.0, 1.0), [B.BC_PERIODIC] * 4)
    s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, B.F32)
    # the thin oracle mesh: the cells of the full mesh along the wave, one
    # cell of the full mesh's size across it (periodic: its own neighbour)
    if along == "x":
        g1, dg1 = make_pair_2d(n_long, 1, (0, 1.0, 0, 1.0 / n_short), 2, "P", "euler", "ssprk3", PER, "f32")
    else:
        g1, dg1 = make_pair_2d(1, n_long, (0, 1.0 / n_short, 0, 1.0), 2, "P", "euler", "ssprk3", PER, "f32")
    g1.close()
    u1 = dg1.project(lambda X, Y: _wave(X, Y, along))
    u1 = from_planes(to_planes(u1).astype(np.float32).astype(np.float64))
    # the full state: the thin run's cells repeated across the other axis
    u = np.repeat(u1, n_short, axis=0) if along == "x" else np.repeat(u1, n_short, axis=1)
    s.set_state(to_planes(u), 0.0)
    dt = 0.3 * cfl_dt_2d(dg1, u1, 1.0)
    w, t = u1, 0.0
    for _ in range(3):
        s.step(dt)
        w = crkdg_step(dg1, w, t, dt, OTB.SSPRK3)
        t += dt
    got = s.get_state()   # planes [v, m, y, x]
    assert s.sync() == (0, 0)
    s.close()
    if along == "x":
        first = got[:, :, :1, :]
        assert np.array_equal(got, np.broadcast_to(first, got.shape))
        assert rel_err(from_planes(first), w) < 2e-5
    else:
        first = got[:, :, :, :1]
        assert np.array_equal(got, np.broadcast_to(first, got.shape))
        assert rel_err(from_planes(first), w) < 2e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_zero_time_step_leaves_the_state(prec):
    """A host step with dt = 0 is rejected before anything runs; device-driven
    steps at t = t_end (dt = min(cfl / max speed, t_end - t) = 0) copy the
    state unchanged and leave t where it is."""
    from paper_2307_06471_gb300 import binding as B
    gs, _ = make_pair_2d(45, 37, (0, 1, 0, 1), 2, "P", "euler", "ssprk3", PER, prec)
    u = inp.random_modal_state(37, 45, 2, "P", "euler", seed=61)
    gs.set_state(to_planes(u), 0.25)
    before = gs.get_state()
    with pytest.raises(B.CrkdgError):
        gs.step(0.0)
    gs.advance(3, 0.5, 0.25)
    assert np.array_equal(gs.get_state(), before)
    assert gs.time() == 0.25
    assert gs.sync() == (0, 0)
    gs.close()
