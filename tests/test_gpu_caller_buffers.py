"""A context whose state lives in caller-owned device memory
(crkdg_create_on_buffers): two PyTorch tensors hold the ping-pong copies.
The context starts from the first tensor's contents, its steps equal those of
a context with its own state bit for bit (and the FP64 oracle), the copy that
crkdg_current_state names holds the result, crkdg_destroy leaves the tensors
alone, and host memory or misaligned device addresses are rejected."""
import ctypes as C

import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import tableaux as OTB
from oracle.dg2d import cfl_dt_2d, crkdg_step
from tests.pairing import from_planes, make_pair_2d, rel_err, to_planes

pytestmark = pytest.mark.gpu

PER = {s: ("periodic",) for s in "WESN"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_state_in_caller_owned_tensors(prec):
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    nx, ny, steps = 45, 37, 3
    P = B.F32 if prec == "f32" else B.F64
    tdt = torch.float32 if prec == "f32" else torch.float64
    npdt = np.float32 if prec == "f32" else np.float64
    own, dg = make_pair_2d(nx, ny, (0, 1, 0, 1), 2, "P", "euler", "ssprk3", PER, prec)
    u = inp.random_modal_state(ny, nx, 2, "P", "euler", seed=71)
    planes = to_planes(u).astype(npdt)
    own.set_state(planes.astype(np.float64), 0.0)
    dt = 0.2 * cfl_dt_2d(dg, u, 1.0)
    for _ in range(steps):
        own.step(dt)
    ref = own.get_state()
    own.close()

    nbytes = B.state_bytes(own.mesh, 2, B.BASIS_P, B.EULER, P)
    assert nbytes == planes.nbytes
    ta = torch.from_numpy(planes.ravel().copy()).to("cuda")
    tb = torch.full_like(ta, float("nan"))
    assert ta.element_size() * ta.numel() == nbytes
    torch.cuda.synchronize()
    s = B.Solver(own.mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, P, state_buffers=(ta.data_ptr(), tb.data_ptr()))
    assert s.current_state() == (0, ta.data_ptr())
    assert np.array_equal(s.get_state(), planes.astype(np.float64))   # starts as the first tensor
    for _ in range(steps):
        s.step(dt)
    which, ptr = s.current_state()
    assert (which, ptr) == (steps % 2, (ta if steps % 2 == 0 else tb).data_ptr())
    got = s.get_state()
    assert s.sync() == (0, 0)
    s.close()
    torch.cuda.synchronize()
    cur = (ta if which == 0 else tb).cpu().numpy().reshape(planes.shape)
    assert np.array_equal(cur.astype(np.float64), got)
    assert np.array_equal(got, ref)   # the same kernels on the same data
    w = u.copy()
    t = 0.0
    for _ in range(steps):
        w = crkdg_step(dg, w, t, dt, OTB.SSPRK3)
        t += dt
    assert rel_err(from_planes(got), w) < (1e-12 if prec == "f64" else 2e-5)
    # the tensors outlive the context
    tb.mul_(2.0)
    torch.cuda.synchronize()
    assert torch.isfinite(tb).all()


def test_host_and_misaligned_buffers_are_rejected():
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    mesh = B.make_mesh(2, 16, 8, (0.0, 1.0, 0.0, 1.0), [B.BC_PERIODIC] * 4)
    n = B.state_bytes(mesh, 2, B.BASIS_P, B.EULER, B.F32) // 4
    ta = torch.zeros(n + 16, dtype=torch.float32, device="cuda")
    tb = torch.zeros(n + 16, dtype=torch.float32, device="cuda")
    host = torch.zeros(n, dtype=torch.float32, pin_memory=True)
    for a, b in ((host.data_ptr(), tb.data_ptr()), (ta.data_ptr() + 4, tb.data_ptr())):
        with pytest.raises(B.CrkdgError):
            B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, B.F32, state_buffers=(a, b))
    # a context on the valid pair still works after the rejections
    s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, B.F32, state_buffers=(ta.data_ptr(), tb.data_ptr()))
    assert s.current_state()[0] == 0
    assert s.sync() == (0, 0)
    s.close()
