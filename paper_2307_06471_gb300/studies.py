"""Measurement studies beside the headline bench (python -m
paper_2307_06471_gb300.studies <name>): each prints one JSON line.

  ensemble  batched four-quadrant Riemann ensemble (256 problems, N from
            {64,128,256,512}, P^2, SSP-RK3, TVB M=50 + positivity, FP32 or
            FP64): DOF-updates/s of the batched, graph-replayed steps
  vortex    isentropic vortex, Q^2, RK4, CFL 0.1, periodic [0,10]^2, to T:
            density L1 error, order over the sizes, FP64 total drift, time
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np
from numpy.polynomial import legendre as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _modes(k, basis):
    out = []
    dmax = k if basis == "P" else 2 * k
    for d in range(dmax + 1):
        for i in range(d, -1, -1):
            if i <= k and d - i <= k:
                out.append((i, d - i))
    return out


def density_l1(state, k, basis, box, exact, nq=5):
    """Mean absolute density error of planes [v][m][y][x] against exact(X, Y)
    with an nq-point Gauss rule per direction."""
    nv, nm, ny, nx = state.shape
    x0, x1, y0, y1 = box
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    g, w = L.leggauss(nq)
    modes = _modes(k, basis)
    P = lambda i, t: L.legval(t, np.eye(k + 1)[i])
    phi = np.stack([np.outer(P(i, g), P(j, g)) for (i, j) in modes])         # (m, a, b)
    rho = np.einsum("myx,mab->yxab", state[0], phi)
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    X = xc[None, :, None, None] + 0.5 * dx * g[None, None, :, None]
    Y = yc[:, None, None, None] + 0.5 * dy * g[None, None, None, :]
    X, Y = np.broadcast_arrays(X, Y)
    e = np.abs(rho - exact(X, Y)[..., 0])
    return float(np.sum(e * np.outer(w, w)) * 0.25 / (nx * ny))


def vortex(sizes=(80, 160, 320), T=10.0, precision="f32", cfl=0.1):
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    P = {"f32": B.F32, "f64": B.F64, "f32c": B.F32C}[precision]
    stream = torch.cuda.Stream()
    rows = []
    for N in sizes:
        mesh = B.make_mesh(2, N, N, (0.0, 10.0, 0.0, 10.0), [B.BC_PERIODIC] * 4)
        s = B.Solver(mesh, 2, B.BASIS_Q, GTB.RK4, B.EULER, P, stream=stream.cuda_stream)
        s.project_function(lambda X, Y: inp.vortex_ic(X, Y))
        m0 = s.conservation()
        e0 = density_l1(s.get_state(), 2, "Q", (0, 10, 0, 10), lambda X, Y: inp.vortex_ic(X, Y))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = 0
        while True:
            s.advance(200, cfl, T, capture=True)
            steps += 200
            if s.time() >= T * (1 - 1e-14):
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        u = s.get_state()
        err = density_l1(u, 2, "Q", (0, 10, 0, 10), lambda X, Y: inp.vortex_ic(X, Y, T))
        m1 = s.conservation()
        code, st = s.sync()
        rows.append({"N": N, "L1_density": err, "L1_projection": e0, "wall_s": wall,
                     "dof_updates_per_s": N * N * 36 * steps / wall, "mass_drift_rel": float(abs(m1[0] - m0[0]) / m0[0]),
                     "energy_drift_rel": float(abs(m1[3] - m0[3]) / m0[3]), "status": st})
        s.close()
    for a, b in zip(rows[:-1], rows[1:]):
        b["order"] = math.log(a["L1_density"] / b["L1_density"]) / math.log(b["N"] / a["N"])
    return {"study": "vortex", "precision": precision, "T": T, "basis": "Q2", "tableau": "rk4", "cfl": cfl,
            "rows": rows}


def ensemble(n=256, steps=40, precision="f32", seed=20230713, autotune=True):
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    P = B.F32 if precision == "f32" else B.F64
    ens = inp.riemann_ensemble(n, seed=seed)
    stream = torch.cuda.Stream()
    bt = B.Batch([(e["N"], e["N"], (0.0, 1.0, 0.0, 1.0)) for e in ens], 2, B.BASIS_P, GTB.SSPRK3, P,
                 stream=stream.cuda_stream)
    for i, e in enumerate(ens):
        bt.project_function(i, lambda X, Y: inp.riemann_ic(X, Y, e["prim"]))
    bt.limit(50.0)
    bt.positivity(1e-10)
    tuned = bt.autotune(0.16) if autotune else None
    bt.run(0.16, 0.2, steps_per_graph=4, max_graphs=1)      # warm-up, graph capture
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    bt.run(0.16, 0.2, steps_per_graph=steps, max_graphs=1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    stat = [bt.info(i) for i in range(n)]
    out = {"study": "ensemble", "precision": precision, "problems": n, "total_cells": bt.total_cells,
           "dof": bt.total_cells * 24, "steps": steps, "ms_per_step": ms / steps,
           "dof_updates_per_s": bt.total_cells * 24 * steps / (ms * 1e-3), "tasks": bt.n_tasks,
           "autotune_us": tuned, "nonzero_status": sum(1 for s in stat if s[2]),
           "sizes": {str(N): sum(1 for e in ens if e["N"] == N) for N in (64, 128, 256, 512)}}
    bt.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["vortex", "ensemble"])
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--sizes", default="80,160,320")
    ap.add_argument("--T", type=float, default=10.0)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--n", type=int, default=256)
    a = ap.parse_args()
    if a.study == "vortex":
        r = vortex(tuple(int(x) for x in a.sizes.split(",")), a.T, a.precision)
    else:
        r = ensemble(a.n, a.steps, a.precision)
    print(json.dumps(r, default=float))
