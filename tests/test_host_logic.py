"""Host-side logic without a GPU: argument validation of the C ABI (every
check runs before the first CUDA call) and the multi-rank aggregation of
bench.py over torch.distributed with the gloo backend (world size 2)."""
import ctypes as C
import os
import socket

import numpy as np
import pytest


@pytest.fixture(scope="module")
def B():
    from paper_2307_06471_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _create(B, mesh, k=2, basis=0, flux=0, tab=None, gamma=1.4, physics=1, precision=0, beta=(1.0, 0.0)):
    from paper_2307_06471_gb300 import tableaux as T
    t = tab if tab is not None else B.make_tableau(*T.SSPRK3)
    out = C.c_void_p()
    pp = (C.c_double * 2)(*beta)
    return B.lib().crkdg_create(C.byref(mesh), k, basis, flux, C.byref(t), gamma, physics, precision, pp, None,
                                C.byref(out))


def test_create_rejects_bad_arguments_before_touching_the_gpu(B):
    per = [B.BC_PERIODIC] * 4
    good = B.make_mesh(2, 8, 8, (0, 1, 0, 1), per)
    assert _create(B, good, k=4) == B.EUNSUPPORTED
    assert _create(B, good, basis=7) == B.EINVAL
    assert _create(B, good, flux=3) == B.EINVAL
    assert _create(B, good, physics=9) == B.EINVAL
    assert _create(B, good, precision=9) == B.EINVAL
    assert _create(B, good, gamma=1.0) == B.EINVAL
    assert _create(B, good, physics=B.ADVECTION, precision=B.F32C) == B.EUNSUPPORTED
    assert _create(B, B.make_mesh(3, 8, 8, (0, 1, 0, 1), per)) == B.EINVAL
    assert _create(B, B.make_mesh(2, 0, 8, (0, 1, 0, 1), per)) == B.EINVAL
    assert _create(B, B.make_mesh(2, 8, 8, (1, 1, 0, 1), per)) == B.EINVAL
    mixed = B.make_mesh(2, 8, 8, (0, 1, 0, 1), [B.BC_PERIODIC, B.BC_OUTFLOW, B.BC_PERIODIC, B.BC_PERIODIC])
    assert _create(B, mixed) == B.EINVAL
    refl = B.make_mesh(2, 8, 8, (0, 1, 0, 1), [B.BC_REFLECT] * 4)
    assert _create(B, refl, physics=B.ADVECTION) == B.EINVAL
    bad_fn = B.make_mesh(2, 8, 8, (0, 1, 0, 1), [B.BC_DIRICHLET, B.BC_OUTFLOW, B.BC_OUTFLOW, B.BC_OUTFLOW],
                         [9, 0, 0, 0])
    assert _create(B, bad_fn) == B.EINVAL
    implicit = B.make_tableau([[0.5, 0.0], [0.5, 0.0]], [0.5, 0.5])
    assert _create(B, good, tab=implicit) == B.EINVAL
    too_many = B.Tableau()
    too_many.s = 7
    assert _create(B, good, tab=too_many) == B.EINVAL
    assert b"tableau" in B.lib().crkdg_last_error()


def test_state_bytes_and_caller_buffer_checks(B):
    """crkdg_state_bytes from the layout (cells x variables x modes, 4 or 8
    bytes, two plane sets for the compensated states), and the checks of
    crkdg_create_on_buffers that come before any CUDA call."""
    from paper_2307_06471_gb300 import tableaux as T
    per = [B.BC_PERIODIC] * 4
    m2 = B.make_mesh(2, 30, 7, (0, 1, 0, 1), per)
    m1 = B.make_mesh(1, 50, 1, (0, 1, 0, 1), per)
    assert B.state_bytes(m2, 2, B.BASIS_P, B.EULER, B.F32) == 30 * 7 * 4 * 6 * 4
    assert B.state_bytes(m2, 2, B.BASIS_Q, B.EULER, B.F64) == 30 * 7 * 4 * 9 * 8
    assert B.state_bytes(m2, 3, B.BASIS_P, B.ADVECTION, B.F32) == 30 * 7 * 1 * 10 * 4
    assert B.state_bytes(m2, 2, B.BASIS_Q, B.EULER, B.F32D) == 30 * 7 * 4 * 9 * 4 * 2
    assert B.state_bytes(m1, 2, B.BASIS_Q, B.EULER, B.F64) == 50 * 3 * 3 * 8   # 1D: P^k, 3 variables
    n = C.c_size_t()
    assert B.lib().crkdg_state_bytes(C.byref(m2), 4, B.BASIS_P, B.EULER, B.F32, C.byref(n)) == B.EINVAL
    assert B.lib().crkdg_state_bytes(C.byref(m2), 2, B.BASIS_P, B.EULER, 9, C.byref(n)) == B.EINVAL
    t = B.make_tableau(*T.SSPRK3)
    pp = (C.c_double * 2)(1.0, 0.0)
    out = C.c_void_p()
    nb = B.state_bytes(m2, 2, B.BASIS_P, B.EULER, B.F32)

    def make(a, b):
        return B.lib().crkdg_create_on_buffers(C.byref(m2), 2, B.BASIS_P, B.FLUX_LLF, C.byref(t), 1.4, B.EULER,
                                               B.F32, pp, None, C.c_void_p(a), C.c_void_p(b), C.byref(out))
    base = 1 << 40   # never dereferenced: every case fails a check first
    assert make(0, base) == B.EINVAL                      # null
    assert make(base + 4, base + 2 * nb) == B.EINVAL      # misaligned
    assert make(base, base + nb - 16) == B.EINVAL         # overlapping
    assert out.value is None


def test_batch_create_rejects_bad_arguments(B):
    from paper_2307_06471_gb300 import tableaux as T
    arr = (B.BatchProblem * 1)(B.BatchProblem(8, 8, 0.0, 1.0, 0.0, 1.0))
    tab = B.make_tableau(*T.SSPRK3)
    out = C.c_void_p()
    L = B.lib()
    bc_ok = (C.c_int * 4)(*([B.BC_OUTFLOW] * 4))
    bc_bad = (C.c_int * 4)(B.BC_DIRICHLET, 1, 1, 1)
    assert L.crkdg_batch_create(C.cast(arr, C.c_void_p), 1, bc_bad, 2, 0, C.byref(tab), 1.4, 0, None,
                                C.byref(out)) == B.EINVAL
    assert L.crkdg_batch_create(C.cast(arr, C.c_void_p), 1, bc_ok, 5, 0, C.byref(tab), 1.4, 0, None,
                                C.byref(out)) == B.EUNSUPPORTED
    assert L.crkdg_batch_create(C.cast(arr, C.c_void_p), 0, bc_ok, 2, 0, C.byref(tab), 1.4, 0, None,
                                C.byref(out)) == B.EINVAL
    empty = (B.BatchProblem * 1)(B.BatchProblem(8, 8, 1.0, 1.0, 0.0, 1.0))
    assert L.crkdg_batch_create(C.cast(empty, C.c_void_p), 1, bc_ok, 2, 0, C.byref(tab), 1.4, 0, None,
                                C.byref(out)) == B.EINVAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dev_ms = [10.0, 12.5][rank]            # rank 1 is the slowest
    ms, value, n = bench.aggregate(dev_ms, 1000, 4)
    q.put((rank, ms, value, n))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, n in res:
        assert n == 2
        assert ms == 12.5                               # max over ranks
        assert value == pytest.approx(2 * 1000 * 4 / 12.5e-3)
