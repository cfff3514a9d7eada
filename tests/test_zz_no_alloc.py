"""The no-allocation reduction entry point (crkdg_reduce_state_noalloc).

Some callers cannot allocate device memory themselves -- code inside a host
framework that owns the memory pool, or code running while a graph is being
captured.  This entry point takes the state and an output buffer the caller
already owns and keeps its scratch in a fixed device array inside the
library.  The tests compare its results with the allocating entry points
(crkdg_cfl_dt and crkdg_conservation) on two calls in a row, in 2D and 1D
(Euler and advection), and check that a non-physical cell is reported in the
status element of the output.  They sit in a file pytest collects last, so a
run that stops at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import crkdg_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


def _call(dev_u, dim, nx, ny, nm, phys, prec, dx, dy, beta, n_out):
    """Two calls in a row into a caller-owned device buffer; returns both."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    L = B.lib()
    out = torch.zeros(n_out, dtype=torch.float64, device="cuda")
    cbeta = (C.c_double * 2)(*beta)
    stream = torch.cuda.current_stream().cuda_stream
    res = []
    for _ in range(2):
        out.fill_(-1.0)
        rc = L.crkdg_reduce_state_noalloc(C.c_void_p(dev_u.data_ptr()), dim, nx, ny, nm, phys, prec, dx, dy, 1.4,
                                          cbeta, C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == 0, L.crkdg_noalloc_last_error().decode()
        torch.cuda.synchronize()
        res.append(out.cpu().numpy())
    return res


def _device(planes, prec):
    import torch
    return torch.tensor(planes, dtype=torch.float32 if prec == "f32" else torch.float64, device="cuda").contiguous()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_reduction_matches_allocating_entry_points(prec):
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    nx, ny, k = 301, 77, 2
    mesh = B.make_mesh(2, nx, ny, (0.0, 3.0, 0.0, 1.0), [B.BC_PERIODIC] * 4)
    P = B.F32 if prec == "f32" else B.F64
    s = B.Solver(mesh, k, B.BASIS_P, GTB.SSPRK3, B.EULER, P)
    u = inp.random_modal_state(ny, nx, k, "P", "euler", seed=77)
    planes = np.ascontiguousarray(np.transpose(u, (2, 3, 0, 1)))
    s.set_state(planes, 0.0)
    dt = s.cfl_dt(0.5)
    sums = s.conservation()
    # the caller's own device buffers: state (same values as the context's) and output
    for res in _call(_device(planes, prec), 2, nx, ny, s.n_modes, B.EULER, P, 3.0 / nx, 1.0 / ny, (0.0, 0.0), 2 + 4):
        assert res[0] == pytest.approx(0.5 / dt, rel=1e-13)
        assert np.allclose(res[1:5], sums, rtol=1e-12, atol=1e-14)
        assert res[5] == 0.0                                   # no status bit on a physical state
    s.close()


@pytest.mark.parametrize("physics", ["euler", "advection"])
def test_noalloc_reduction_1d(physics):
    """1D meshes: ny and dy are ignored (a caller passing any dy gets the
    totals of cells of width dx, as crkdg_conservation computes them)."""
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    nx, k = 203, 2
    nv = 3 if physics == "euler" else 1
    phys = B.EULER if physics == "euler" else B.ADVECTION
    mesh = B.make_mesh(1, nx, 1, (0.0, 2.0), [B.BC_PERIODIC, B.BC_PERIODIC, 0, 0])
    s = B.Solver(mesh, k, B.BASIS_P, GTB.SSPRK3, phys, B.F64, beta=(-1.5, 0.0))
    u = inp.random_modal_state_1d(nx, k, nv, seed=5)
    planes = np.ascontiguousarray(np.transpose(u, (1, 2, 0))[:, :, None, :])
    s.set_state(planes, 0.0)
    dt = s.cfl_dt(0.3)
    sums = s.conservation()
    for res in _call(_device(planes, "f64"), 1, nx, 7, s.n_modes, phys, B.F64, 2.0 / nx, 0.25, (-1.5, 0.0),
                     2 + nv):
        assert res[0] == pytest.approx(0.3 / dt, rel=1e-13)
        assert np.allclose(res[1:1 + nv], sums, rtol=1e-12, atol=1e-14)
        assert res[1 + nv] == 0.0
    s.close()


def test_noalloc_reports_nonphysical_cells():
    """A cell average with negative density (set on the host) and a NaN cell
    come back as status bits in out[1 + nv]; the maximum wave speed alone
    would not show the NaN."""
    from paper_2307_06471_gb300 import binding as B
    nx, ny, k = 64, 32, 1
    u = inp.random_modal_state(ny, nx, k, "P", "euler", seed=9)
    planes = np.ascontiguousarray(np.transpose(u, (2, 3, 0, 1)))
    neg = planes.copy()
    neg[0, 0, 5, 7] = -0.5
    res = _call(_device(neg, "f64"), 2, nx, ny, 3, B.EULER, B.F64, 1.0 / nx, 1.0 / ny, (0.0, 0.0), 6)
    for r in res:
        assert int(r[5]) & B.ST_NONPHYSICAL
    nan = planes.copy()
    nan[3, 0, 20, 30] = np.nan
    res = _call(_device(nan, "f32"), 2, nx, ny, 3, B.EULER, B.F32, 1.0 / nx, 1.0 / ny, (0.0, 0.0), 6)
    for r in res:
        assert np.isfinite(r[0])
        assert int(r[5]) & (B.ST_NONPHYSICAL | B.ST_NAN)
    # a physical state afterwards: the bits of the earlier calls are gone
    res = _call(_device(planes, "f64"), 2, nx, ny, 3, B.EULER, B.F64, 1.0 / nx, 1.0 / ny, (0.0, 0.0), 6)
    assert res[-1][5] == 0.0


def test_noalloc_rejects_bad_sizes():
    from paper_2307_06471_gb300 import binding as B
    L = B.lib()
    rc = L.crkdg_reduce_state_noalloc(C.c_void_p(16), 2, 1 << 16, 1 << 15, 6, B.EULER, B.F32, 1.0, 1.0, 1.4, None,
                                      C.c_void_p(16), None)
    assert rc == B.EINVAL
    assert b"2^30" in L.crkdg_noalloc_last_error()
