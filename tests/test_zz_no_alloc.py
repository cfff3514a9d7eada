"""The no-allocation reduction entry point (crkdg_reduce_state_noalloc).

Some callers cannot allocate device memory themselves -- code inside a host
framework that owns the memory pool, or code running while a graph is being
captured.  This entry point takes the state and an output buffer the caller
already owns and keeps its scratch in a fixed device array inside the
library.  The test compares its results with the allocating entry points
(crkdg_cfl_dt and crkdg_conservation) on two calls in a row.  It sits in a
file pytest collects last, so a run that stops at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import crkdg_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_reduction_matches_allocating_entry_points(prec):
    import torch
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
    tdt = torch.float32 if prec == "f32" else torch.float64
    dev_u = torch.tensor(planes, dtype=tdt, device="cuda").contiguous()
    out = torch.zeros(1 + 4, dtype=torch.float64, device="cuda")
    L = B.lib()
    beta = (C.c_double * 2)(0.0, 0.0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(-1.0)
        rc = L.crkdg_reduce_state_noalloc(C.c_void_p(dev_u.data_ptr()), 2, nx, ny, s.n_modes, B.EULER, P,
                                          3.0 / nx, 1.0 / ny, 1.4, beta, C.c_void_p(out.data_ptr()),
                                          C.c_void_p(stream))
        assert rc == 0, L.crkdg_noalloc_last_error().decode()
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        assert res[0] == pytest.approx(0.5 / dt, rel=1e-13)
        assert np.allclose(res[1:], sums, rtol=1e-12, atol=1e-14)
    s.close()


def test_noalloc_rejects_bad_sizes():
    from paper_2307_06471_gb300 import binding as B
    L = B.lib()
    rc = L.crkdg_reduce_state_noalloc(C.c_void_p(16), 2, 1 << 16, 1 << 15, 6, B.EULER, B.F32, 1.0, 1.0, 1.4, None,
                                      C.c_void_p(16), None)
    assert rc == B.EINVAL
    assert b"2^30" in L.crkdg_noalloc_last_error()
