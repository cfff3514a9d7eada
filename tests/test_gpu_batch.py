"""Batched ensembles: every problem of a batch evolves exactly as it does
alone (same per-cell arithmetic, same device-computed dt sequence), problems
stop at their own t_end, and a batched problem agrees with the FP64 oracle."""
import numpy as np
import pytest

import crkdg_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


def _problems():
    ens = inp.riemann_ensemble(6, sizes=(16, 24, 40, 64))
    boxes = [(0.0, 1.0, 0.0, 1.0), (0.0, 1.0, 0.0, 1.0), (-0.5, 0.5, 0.0, 1.0), (0.0, 1.0, 0.0, 1.0),
             (0.0, 1.0, 0.25, 1.25), (0.0, 1.0, 0.0, 1.0)]
    probs = []
    for i, e in enumerate(ens):
        N = e["N"]
        ny = N if i % 2 == 0 else N // 2 + 3          # some non-square meshes
        probs.append((N, ny, boxes[i], e["prim"]))
    return probs


def _ic(prim, box):
    cx = 0.5 * (box[0] + box[1])
    cy = 0.5 * (box[2] + box[3])
    return lambda X, Y: inp.riemann_ic(X - cx + 0.5, Y - cy + 0.5, prim)


@pytest.mark.parametrize("mode", ["pass", "fused"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_equals_single_problem_runs(prec, mode):
    """The batch's limiter runs as a pass over every problem before the
    batched step (default) or inside its load.  Each problem evolves like the
    same problem alone in the same limit mode: bitwise, except for the FP32
    limiter pass, whose arithmetic is compiled into a kernel of its own for
    the batch (the compiler may fuse its multiply-adds differently from the
    single-problem pass): there to FP32 rounding (measured 1.2e-7 absolute
    on states of order 1 after ten steps; the band is 1e-5 of each
    variable's scale)."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    P = B.F32 if prec == "f32" else B.F64
    LM = B.LIMIT_PASS if mode == "pass" else B.LIMIT_FUSED
    probs = _problems()
    stream = torch.cuda.Stream()
    bt = B.Batch([(nx, ny, box) for (nx, ny, box, _) in probs], 2, B.BASIS_P, GTB.SSPRK3, P,
                 stream=stream.cuda_stream)
    bt.set_launch(seg_rows=8, warps_per_block=4)
    bt.set_limit_mode(LM)
    for i, (nx, ny, box, prim) in enumerate(probs):
        bt.project_function(i, _ic(prim, box))
    bt.limit(50.0)
    bt.positivity(1e-10)
    done = bt.run(0.16, 10.0, steps_per_graph=5, max_graphs=2)   # 10 steps, nobody done
    assert done == 0
    for i, (nx, ny, box, prim) in enumerate(probs):
        mesh = B.make_mesh(2, nx, ny, box, [B.BC_OUTFLOW] * 4)
        s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, P, stream=stream.cuda_stream)
        s.set_launch(seg_rows=8, warps_per_block=4)
        s.set_limit_mode(LM)
        s.project_function(_ic(prim, box))
        s.limit(50.0)
        s.positivity(1e-10)
        s.advance(10, 0.16, 10.0)
        want = s.get_state()
        got = bt.get_state(i)
        if prec == "f32" and mode == "pass":
            for v in range(4):
                assert np.max(np.abs(got[v] - want[v])) <= 1e-5 * max(np.max(np.abs(want[v])), 1e-2), (i, v)
        else:
            assert np.array_equal(got, want), i
        t, steps, status = bt.info(i)
        assert steps == 10 and status == 0
        exact = not (prec == "f32" and mode == "pass")
        assert t == pytest.approx(s.time(), rel=0 if exact else 1e-6, abs=0)
        s.close()
    bt.close()


def test_batch_problems_stop_at_t_end():
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    probs = _problems()
    stream = torch.cuda.Stream()
    bt = B.Batch([(nx, ny, box) for (nx, ny, box, _) in probs], 1, B.BASIS_P, GTB.MIDPOINT, B.F32,
                 stream=stream.cuda_stream)
    for i, (nx, ny, box, prim) in enumerate(probs):
        bt.project_function(i, _ic(prim, box))
    bt.limit(50.0)
    bt.positivity(1e-10)
    T = 0.02
    done = bt.run(0.2, T, steps_per_graph=16, max_graphs=100)
    assert done == len(probs)
    steps = []
    for i in range(len(probs)):
        t, n, st = bt.info(i)
        assert t == pytest.approx(T, rel=1e-12) and st == 0
        steps.append(n)
    assert len(set(steps)) > 1          # uneven problems took different step counts
    bt.close()


def test_batched_problem_matches_oracle_f64():
    import torch
    from oracle import tableaux as OTB
    from oracle.dg2d import DG2D, cfl_dt_2d, crkdg_step
    from oracle.limiter import positivity_limit, tvb_limit
    from oracle.physics import Euler
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    probs = _problems()[:3]
    stream = torch.cuda.Stream()
    bt = B.Batch([(nx, ny, box) for (nx, ny, box, _) in probs], 2, B.BASIS_P, GTB.SSPRK3, B.F64,
                 stream=stream.cuda_stream)
    for i, (nx, ny, box, prim) in enumerate(probs):
        bt.project_function(i, _ic(prim, box))
    bt.limit(50.0)
    bt.positivity(1e-10)
    bt.run(0.16, 10.0, steps_per_graph=3, max_graphs=1)
    nx, ny, box, prim = probs[2]
    dg = DG2D(nx, ny, box, 2, "P", Euler(1.4, 2), {s: "outflow" for s in "WESN"})
    X, Y = dg.volume_points()
    u = dg.project_point_values(_ic(prim, box)(X, Y))
    lim = lambda v, t: positivity_limit(dg, tvb_limit(dg, v, 50.0, t)[0], 1e-10)
    w = lim(u, 0.0)
    t = 0.0
    for _ in range(3):
        dt = cfl_dt_2d(dg, w, 0.16)
        w = crkdg_step(dg, w, t, dt, OTB.SSPRK3, limiter=lim)
        t += dt
    got = np.transpose(bt.get_state(2), (2, 3, 0, 1))
    assert np.max(np.abs(got - w)) / np.max(np.abs(w)) < 1e-12
    bt.close()
