"""Measurement studies beside the headline bench (python -m
paper_2307_06471_gb300.studies <name>): each prints one JSON line.

  ensemble  batched four-quadrant Riemann ensemble (256 problems, N from
            {64,128,256,512}, P^2, SSP-RK3, TVB M=50 + positivity, FP32 or
            FP64): DOF-updates/s of the batched, graph-replayed steps
  vortex    isentropic vortex, Q^2, RK4, CFL 0.1, periodic [0,10]^2, to T:
            density L1 error, order over the sizes, FP64 total drift, time
  compact   cRKDG against the original RKDG (Shu--Osher SSP-RK3, limiter
            every stage) on the 1920 x 480 double Mach reflection: device
            time per step and per unit simulated time at the paper's CFL
  learned   learned troubled-cell indicator: labels from ensemble runs,
            training with the library's kernels, evaluation on the
            shock-vortex problem (miss / false-flag rates against TVB, L1 vs an
            FP64 TVB run, DOF-updates/s with and without the network)
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


def vortex_run(N, T, precision, stream_handle, cfl=0.1, chunk=100):
    """One isentropic-vortex run (Q^2, RK4, periodic [0,10]^2) to T with
    device-driven steps (CUDA-graph replays of `chunk` steps): density L1 at
    T against the exact translated vortex, wall time of the stepping (host
    clock around the synchronised run), steps, DOF-updates/s, FP64 totals
    drift, device status."""
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    P = {"f32": B.F32, "f64": B.F64, "f32c": B.F32C, "f32d": B.F32D}[precision]
    mesh = B.make_mesh(2, N, N, (0.0, 10.0, 0.0, 10.0), [B.BC_PERIODIC] * 4)
    s = B.Solver(mesh, 2, B.BASIS_Q, GTB.RK4, B.EULER, P, stream=stream_handle)
    s.project_function(lambda X, Y: inp.vortex_ic(X, Y))
    m0 = s.conservation()
    e0 = density_l1(s.get_state(), 2, "Q", (0, 10, 0, 10), lambda X, Y: inp.vortex_ic(X, Y))
    n0 = s.step_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while True:
        s.advance(chunk, cfl, T, capture=True)
        if s.time() >= T * (1 - 1e-14):
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    steps = s.step_count() - n0
    u = s.get_state()
    err = density_l1(u, 2, "Q", (0, 10, 0, 10), lambda X, Y: inp.vortex_ic(X, Y, T))
    m1 = s.conservation()
    code, st = s.sync()
    s.close()
    return {"precision": precision, "N": N, "T": T, "L1_density": err, "L1_projection": e0, "wall_s": wall,
            "steps": steps, "dof_updates_per_s": N * N * 36 * steps / wall,
            "mass_drift_rel": float(abs(m1[0] - m0[0]) / m0[0]),
            "energy_drift_rel": float(abs(m1[3] - m0[3]) / m0[3]), "status": st}


def precision_rates(N=1280, steps=40, warmup=5, variants=("f32", "f32c", "f32d", "f64")):
    """Device-timed step rate of the vortex configuration (Q^2, RK4,
    periodic) on an N x N mesh that fills the GPU (1280^2: 59M DOF; the
    state copies, 236 MB per FP32 plane set, exceed L2), per precision:
    `steps` device-driven steps (dt from each step's own reduction) between
    CUDA events on the solver's stream, after `warmup` steps."""
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    stream = torch.cuda.Stream()
    out = {}
    for v in variants:
        P = {"f32": B.F32, "f64": B.F64, "f32c": B.F32C, "f32d": B.F32D}[v]
        mesh = B.make_mesh(2, N, N, (0.0, 10.0, 0.0, 10.0), [B.BC_PERIODIC] * 4)
        s = B.Solver(mesh, 2, B.BASIS_Q, GTB.RK4, B.EULER, P, stream=stream.cuda_stream)
        s.project_function(lambda X, Y: inp.vortex_ic(X, Y))
        s.advance(warmup, 0.1, 10.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            s.step_device()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        code, st = s.sync()
        out[v] = {"ms_per_step": ms, "dof_updates_per_s": N * N * 36 / (ms * 1e-3), "status": st}
        s.close()
    return {"workload": "isentropic vortex, Q2, RK4, %dx%d, %d device-driven steps" % (N, N, steps), "rates": out}


def matched_l1(T=1.0, fp64_sizes=(80, 120, 160, 240, 320), fp32_sizes=(80, 160, 320),
               variants=("f32", "f32c", "f32d")):
    """Time to a given accuracy: the vortex to T in FP64 on fp64_sizes and in
    each FP32 variant on fp32_sizes.  Each FP32 run is matched to an FP64 run
    (the same mesh if its L1 is within 10 % of FP64's there, else the coarsest
    FP64 mesh whose L1 is at most the FP32 run's); the speedup is that FP64
    run's wall time over the FP32 run's.  Per variant the best matched run is
    reported."""
    import torch
    stream = torch.cuda.Stream()
    runs = [vortex_run(N, T, "f64", stream.cuda_stream) for N in fp64_sizes]
    f64 = {r["N"]: r for r in runs}
    best = {}
    for v in variants:
        for N in fp32_sizes:
            r = vortex_run(N, T, v, stream.cuda_stream)
            runs.append(r)
            same = f64.get(N)
            if same is not None and r["L1_density"] <= 1.1 * same["L1_density"]:
                m = same
            else:
                ok = [f for f in sorted(f64.values(), key=lambda f: f["N"]) if f["L1_density"] <= r["L1_density"]]
                m = ok[0] if ok else None
            if m is None:
                continue
            rec = {"variant": v, "N": N, "L1": r["L1_density"], "wall_s": r["wall_s"],
                   "fp64_N": m["N"], "fp64_L1": m["L1_density"], "fp64_wall_s": m["wall_s"],
                   "speedup_vs_fp64": m["wall_s"] / r["wall_s"]}
            if v not in best or rec["speedup_vs_fp64"] > best[v]["speedup_vs_fp64"]:
                best[v] = rec
    return {"workload": "isentropic vortex (strength 5, mean flow (1,1)), [0,10]^2 periodic, Q2, RK4, CFL 0.1, "
                        "T=%g" % T, "runs": runs, "matched": best}


def vortex(sizes=(80, 160, 320), T=10.0, precision="f32", cfl=0.1):
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    P = {"f32": B.F32, "f64": B.F64, "f32c": B.F32C, "f32d": B.F32D}[precision]
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


def ensemble(n=256, steps=40, precision="f32", seed=20230713, autotune=True, limit_mode="pass"):
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
    bt.set_limit_mode(B.LIMIT_PASS if limit_mode == "pass" else B.LIMIT_FUSED)
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
    out = {"study": "ensemble", "precision": precision, "limit_mode": limit_mode, "problems": n,
           "total_cells": bt.total_cells,
           "dof": bt.total_cells * 24, "steps": steps, "ms_per_step": ms / steps,
           "dof_updates_per_s": bt.total_cells * 24 * steps / (ms * 1e-3), "tasks": bt.n_tasks,
           "autotune_us": tuned, "nonzero_status": sum(1 for s in stat if s[2]),
           "sizes": {str(N): sum(1 for e in ens if e["N"] == N) for N in (64, 128, 256, 512)}}
    bt.close()
    return out


# -- learned troubled-cell indicator ----------------------------------------------------------
def _shock_vortex_solver(B, GTB, inp, nx, ny, precision, stream):
    st_up = inp.conserved(1.0, 1.1 * math.sqrt(1.4), 0.0, 1.0)
    mesh = B.make_mesh(2, nx, ny, (0.0, 2.0, 0.0, 1.0), [B.BC_DIRICHLET, B.BC_OUTFLOW, B.BC_OUTFLOW, B.BC_OUTFLOW],
                       [B.FN_CONST, 0, 0, 0], [list(st_up), None, None, None])
    s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, precision, stream=stream)
    s.project_function(lambda X, Y: inp.shock_vortex(X, Y))
    s.limit(50.0)
    s.positivity(1e-10)
    return s


def learned(n_train_members=200, snapshots=3, steps_between=40, epochs=6, eval_n=(512, 256), T=0.35,
            perf_n=(2048, 2048), perf_steps=100, seed=20230713, pos_weights=None):
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    M = 50.0
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    out = {"study": "learned", "M": M}
    # 1. labels from batched runs of the method itself (config-4 ensemble)
    ens = inp.riemann_ensemble(256, seed=seed)
    bt = B.Batch([(e["N"], e["N"], (0.0, 1.0, 0.0, 1.0)) for e in ens], 2, B.BASIS_P, GTB.SSPRK3, B.F32, stream=sh)
    for i, e in enumerate(ens):
        bt.project_function(i, lambda X, Y: inp.riemann_ic(X, Y, e["prim"]))
    bt.limit(M)
    bt.positivity(1e-10)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    feats = {"train": [], "val": []}
    labels = {"train": [], "val": []}
    for snap in range(snapshots):
        bt.run(0.16, 0.2, steps_per_graph=steps_between, max_graphs=1)
        for i, e in enumerate(ens):
            n = e["N"] * e["N"]
            X = torch.empty(n, 40, device="cuda")
            y = torch.empty(n, device="cuda")
            bt.features(i, X.data_ptr(), y.data_ptr(), M)
            keep = (y > 0.5) | (torch.rand(n, device="cuda", generator=g) < 0.05)   # all positives, 5 % negatives
            part = "train" if i < n_train_members else "val"
            feats[part].append(X[keep])
            labels[part].append(y[keep])
    bt.close()
    Xtr, ytr = torch.cat(feats["train"]).contiguous(), torch.cat(labels["train"]).contiguous()
    Xva, yva = torch.cat(feats["val"]).contiguous(), torch.cat(labels["val"]).contiguous()
    npos = float(ytr.sum().item())
    out["train_samples"] = len(ytr)
    out["train_positive_frac"] = npos / len(ytr)
    out["negative_keep_frac"] = 0.05
    # 3. shock-vortex evaluation (config 5): FP64 TVB reference and FP32 TVB once
    nx, ny = eval_n

    def run(prec, net=None):
        s = _shock_vortex_solver(B, GTB, inp, nx, ny, prec, sh)
        if net is not None:
            s.set_indicator(net)
        while s.time() < T * (1 - 1e-12):
            s.advance(100, 0.16, T)
        res = {"state": s.get_state(), "status": s.sync()[1]}
        if net is not None:
            n = nx * ny
            X = torch.empty(n, 40, device="cuda")
            y = torch.empty(n, device="cuda")
            s.features(X.data_ptr(), y.data_ptr(), M)
            z = torch.empty(n, device="cuda")
            net.predict(X.data_ptr(), n, z.data_ptr())
            lab, prd = y > 0.5, z > 0
            band = (z > -1.3862943611198906) & (z < 1.3862943611198906)
            res.update(tvb_flagged=int(lab.sum()), miss=float((lab & ~prd).sum() / max(lab.sum(), 1)),
                       false=float((~lab & prd).sum() / max((~lab).sum(), 1)), band=float(band.float().mean()))
        s.close()
        return res

    ref = run(B.F64)["state"][0, 0]
    cells = nx * ny
    tvb32 = run(B.F32)
    out["L1_density_f32_tvb"] = float(np.abs(tvb32["state"][0, 0] - ref).sum() / cells)
    out["eval_mesh"] = "%dx%d" % eval_n
    out["T"] = T
    # 2. training with the library's kernels, one network per class weight
    # (pos_weight = keep fraction restores the natural class prior; 1.0 and
    # the balanced weight over-weight positives)
    nets = []
    out["networks"] = []
    for pw in pos_weights if pos_weights else (0.05, 0.25, (len(ytr) - npos) / max(npos, 1.0)):
        net = B.MLP(seed=1, stream=sh)
        t0 = time.perf_counter()
        loss = net.train(Xtr.data_ptr(), ytr.data_ptr(), len(ytr), epochs=epochs, batch=1024, lr=1e-3, pos_weight=pw,
                         seed=7)
        row = {"pos_weight": pw, "train_seconds": time.perf_counter() - t0, "final_train_loss": loss}
        zva = torch.empty(len(yva), device="cuda")
        net.predict(Xva.data_ptr(), len(yva), zva.data_ptr())
        pred, pos = zva > 0, yva > 0.5
        row["val_miss_rate_subsampled"] = float((pos & ~pred).sum() / max(pos.sum(), 1))
        row["val_false_rate_subsampled"] = float((~pos & pred).sum() / max((~pos).sum(), 1))
        r = run(B.F32, net)
        row.update(eval_miss_rate=r["miss"], eval_false_rate=r["false"], eval_band_fallback_frac=r["band"],
                   eval_tvb_flagged=r["tvb_flagged"], status=r["status"],
                   L1_density=float(np.abs(r["state"][0, 0] - ref).sum() / cells))
        out["networks"].append(row)
        nets.append(net)
    net = nets[0]
    # 4. throughput at 2048 x 2048 (device steps, L2 not a factor at 403 MB)
    nx, ny = perf_n
    # (the network in the limiter pass, the default limit mode, and fused
    # into the step's load)
    # (the network in the limiter pass on the tcgen05 tensor cores -- the
    # default -- or with mma.sync, and fused into the step's load)
    for name, prec, use_net, fused, mma in (("f32_tvb", B.F32, False, False, False),
                                            ("f32_mlp", B.F32, True, False, False),
                                            ("f32_mlp_pass_mma_sync", B.F32, True, False, True),
                                            ("f32_mlp_fused", B.F32, True, True, True),
                                            ("f64_tvb", B.F64, False, False, False)):
        s = _shock_vortex_solver(B, GTB, inp, nx, ny, prec, sh)
        if use_net:
            s.set_indicator(net)
            s.set_indicator_engine(B.MLP_MMA_SYNC if mma else B.MLP_TCGEN05)
        if fused:
            s.set_limit_mode(B.LIMIT_FUSED)
        n_steps = perf_steps if prec == B.F32 else max(5, perf_steps // 10)
        s.advance(3, 0.16, 10.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            s.step_device()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n_steps
        out["dof_per_s_" + name] = nx * ny * 24 / (ms * 1e-3)
        out["ms_per_step_" + name] = ms
        s.close()
    out["perf_mesh"] = "%dx%d" % perf_n
    for n_ in nets:
        n_.close()
    return out


def indicator_rates(N=2048, steps=30, seed=5):
    """Device time per step of the shock-vortex problem (P^2, SSP-RK3, FP32,
    N x N) with the TVB test and with a network (seeded, untrained, logit
    band [-2, 2] so that both the network and the TVB fallback decide) in the
    limiter pass on the tcgen05 tensor cores, in the pass with mma.sync, and
    fused into the step's load; `steps` device-driven steps between CUDA
    events after 3 warm-up steps."""
    import torch
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    net = B.MLP(seed=seed, stream=sh)
    out = {"study": "indicator_rates", "mesh": "%dx%d" % (N, N), "steps": steps}
    for name, use, engine, fused in (("tvb", False, None, False), ("pass_tcgen05", True, B.MLP_TCGEN05, False),
                                     ("pass_mma_sync", True, B.MLP_MMA_SYNC, False), ("fused_mma_sync", True, None, True)):
        s = _shock_vortex_solver(B, GTB, inp, N, N, B.F32, sh)
        if use:
            s.set_indicator(net, -2.0, 2.0)
        if engine is not None:
            s.set_indicator_engine(engine)
        if fused:
            s.set_limit_mode(B.LIMIT_FUSED)
        s.advance(3, 0.16, 10.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s.step_device()
        e1.record(stream)
        torch.cuda.synchronize()
        out["ms_per_step_" + name] = e0.elapsed_time(e1) / steps
        out["status_" + name] = s.sync()[1]
        s.close()
    net.close()
    return out


def compact(nx=1920, ny=480, steps=100, precision="f32"):
    """cRKDG (limiter pass + one fused step launch) against the original RKDG (SSP-RK3
    in Shu--Osher form, limiter after every stage) on the double Mach
    reflection, each at the paper's CFL for P^2 (0.16 and 0.18, Sec. 4.2)."""
    import torch
    import crkdg_inputs as inp
    import bench
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    P = B.F32 if precision == "f32" else B.F64
    stream = torch.cuda.Stream()
    st = inp.dmr_states()
    out = {"study": "compact", "mesh": "%dx%d" % (nx, ny), "precision": precision, "steps": steps}
    for name, cfl in (("crkdg", 0.16), ("rkdg", 0.18)):
        mesh, _ = bench.dmr_mesh(B, inp, nx, ny)
        s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.EULER, P, stream=stream.cuda_stream)
        s.project_function(lambda X, Y: inp.dmr_ic(X, Y, st))
        s.limit(50.0)
        s.positivity(1e-10)
        for _ in range(5):
            dt = s.cfl_dt(cfl)
            s.step(dt) if name == "crkdg" else s.rkdg_step(dt, 3)
        torch.cuda.synchronize()
        t0 = s.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(steps):
            dt = s.cfl_dt(cfl)                       # host dt for both (same overhead)
            e0.record(stream)
            s.step(dt) if name == "crkdg" else s.rkdg_step(dt, 3)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        sim = s.time() - t0
        out[name] = {"cfl": cfl, "ms_per_step": ms / steps, "sim_time": sim,
                     "device_ms_per_unit_time": ms / sim, "status": s.sync()[1],
                     # cRKDG: limiter pass + fused step + its one-block finalize; RKDG:
                     # 3 x (limiter pass, DG forward-Euler pass + finalize) + 2 linear
                     # combinations + the time update
                     "launches_per_step": 3 if name == "crkdg" else 12,
                     "operator_passes_per_step": 1 if name == "crkdg" else 3,
                     "limiter_passes_per_step": 1 if name == "crkdg" else 3}
        s.close()
    out["rkdg_over_crkdg_time_to_solution"] = out["rkdg"]["device_ms_per_unit_time"] / out["crkdg"]["device_ms_per_unit_time"]
    return out


def advection1d(N=160, steps=1600):
    """u_t + u_x = 0 on periodic [0, 2 pi], u0 = sin x, P^2, SSP-RK3,
    dt = 0.1 h (CFL 0.1), T = 2 pi: the whole run in one single-block launch.
    L1 / Linf error of u against sin(x - T) = sin x, and the mass drift."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    mesh = B.make_mesh(1, N, 1, (0.0, 2 * math.pi, 0.0, 1.0), [B.BC_PERIODIC] * 4)
    s = B.Solver(mesh, 2, B.BASIS_P, GTB.SSPRK3, B.ADVECTION, B.F64, beta=(1.0, 0.0))
    s.project_function(lambda X: np.sin(X)[..., None])
    m0 = s.conservation()
    dt = 2 * math.pi / steps
    s.run_fixed(1, dt)                      # warm-up (module load)
    s.project_function(lambda X: np.sin(X)[..., None])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.run_fixed(steps, dt)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    u = s.get_state()[0, :, 0, :]            # [m][x]
    g, w = L.leggauss(5)
    h = 2 * math.pi / N
    xc = (np.arange(N) + 0.5) * h
    X = xc[None, :] + 0.5 * h * g[:, None]
    uh = sum(u[m][None, :] * L.legval(g, np.eye(3)[m])[:, None] for m in range(3))
    e = np.abs(uh - np.sin(X - 2 * math.pi))
    m1 = s.conservation()
    out = {"study": "advection1d", "N": N, "steps": steps, "wall_s": wall, "us_per_step": 1e6 * wall / steps,
           "L1_mean": float(np.sum(e * w[:, None]) * 0.5 * h / (2 * math.pi)), "Linf": float(e.max()),
           "mass_drift_abs": float(abs(m1[0] - m0[0])), "launches": 1}
    s.close()
    return out


def advection2d_inflow(sizes=(10, 20, 40, 80), T=0.4, k=3, basis="Q"):
    """Cartesian analogue of the paper's 2D boundary-error example: u_t + u_x
    + u_y = 0 on [-1,1]^2, u0 = sin(pi x) sin(pi y), exact data
    sin(pi (x - t)) sin(pi (y - t)) imposed on the inflow sides (W, S) at the
    stage times of the final stage, outflow E, N; P^3/Q^3 with RK4 and
    dt = h/30 (FP64).  L2 error and order."""
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    rows = []
    pp = [1.0, math.pi, 1.0, math.pi, 1.0]
    for N in sizes:
        mesh = B.make_mesh(2, N, N, (-1.0, 1.0, -1.0, 1.0), [B.BC_DIRICHLET, B.BC_OUTFLOW, B.BC_DIRICHLET, B.BC_OUTFLOW],
                           [B.FN_SINE_PROD, 0, B.FN_SINE_PROD, 0], [pp, None, pp, None])
        s = B.Solver(mesh, k, B.BASIS_Q if basis == "Q" else B.BASIS_P, GTB.RK4, B.ADVECTION, B.F64,
                     beta=(1.0, 1.0))
        s.project_function(lambda X, Y: (np.sin(math.pi * X) * np.sin(math.pi * Y))[..., None])
        h = 2.0 / N
        n = int(math.ceil(T / (h / 30)))
        for _ in range(n):
            s.step(T / n)
        u = s.get_state()
        nm = len(_modes(k, basis))
        g, w = L.leggauss(k + 3)
        P = lambda i, t: L.legval(t, np.eye(k + 1)[i])
        phi = np.stack([np.outer(P(i, g), P(j, g)) for (i, j) in _modes(k, basis)])
        uh = np.einsum("myx,mab->yxab", u[0], phi)
        xc = -1 + (np.arange(N) + 0.5) * h
        X = xc[None, :, None, None] + 0.5 * h * g[None, None, :, None]
        Y = xc[:, None, None, None] + 0.5 * h * g[None, None, None, :]
        e = uh - np.sin(math.pi * (X - T)) * np.sin(math.pi * (Y - T))
        l2 = math.sqrt(float(np.sum(e * e * np.outer(w, w)) * 0.25 * h * h))
        rows.append({"N": N, "L2": l2, "steps": n})
        s.close()
    for a, b in zip(rows[:-1], rows[1:]):
        b["order"] = math.log(a["L2"] / b["L2"]) / math.log(b["N"] / a["N"])
    return {"study": "advection2d_inflow", "k": k, "basis": basis, "T": T, "rows": rows}


def advection_hbm(N=4096, steps=200, k=2, basis="Q"):
    """2D linear advection u_t + u_x + 0.5 u_y = 0, periodic [0,1]^2, Q^2,
    SSP-RK3, FP32, N x N cells (4096^2: 151M DOF, 604 MB per state copy, far
    above L2), in both operator forms of the step: the quadrature form (the
    fused Euler machinery with a trivial flux) and the modal form for linear
    fluxes; each against the HBM roofline (u^n read + u^{n+1} written per
    step) and the FP32 one."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    from paper_2307_06471_gb300.workcount import step_bytes_per_cell, step_flops_per_cell
    build.build()
    stream = torch.cuda.Stream()
    mesh = B.make_mesh(2, N, N, (0.0, 1.0, 0.0, 1.0), [B.BC_PERIODIC] * 4)
    s = B.Solver(mesh, k, B.BASIS_Q if basis == "Q" else B.BASIS_P, GTB.SSPRK3, B.ADVECTION, B.F32,
                 beta=(1.0, 0.5), stream=stream.cuda_stream)
    s.project_function(lambda X, Y: (np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y))[..., None])
    h = 1.0 / N
    dt = 0.1 / (1.0 / h + 0.5 / h)
    cells = N * N
    nm = len(_modes(k, basis))
    A, b = GTB.SSPRK3
    fpc = step_flops_per_cell(k, basis, "advection", A, b)
    bpc = step_bytes_per_cell(k, basis, "advection", 4)
    peaks = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                        "MEASURED_PEAKS.json")))
    hbm_peak = float(peaks.get("hbm_gbs", 6787.9))
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    out = {"study": "advection_hbm", "N": N, "k": k, "basis": basis, "steps": steps, "bytes_per_cell": bpc,
           "flop_per_cell_quadrature": fpc}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, form in (("quadrature", B.FORM_QUADRATURE), ("modal", B.FORM_AUTO)):
        s.set_operator_form(form)
        for _ in range(5):
            s.step(dt)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                s.step(dt)
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = bpc * cells / (ms * 1e-3) / 1e9
        row = {"ms_per_step": ms, "dof_updates_per_s": cells * nm / (ms * 1e-3), "hbm_gbs": gbs,
               "hbm_frac_of_measured": gbs / hbm_peak}
        if name == "quadrature":
            tf = fpc * cells / (ms * 1e-3) / 1e12
            row.update({"tflops": tf, "fp32_frac": tf / fp32_peak})
        out[name] = row
    out["status"] = s.sync()[1]
    s.close()
    return out


def dmr_full(nx=1920, ny=480, k=2, T=0.2, cfl=None, precision="f32"):
    """The double Mach reflection run to T = 0.2 (Sec. 4.2): P^k, SSP-RK3,
    TVB M = 50 + positivity scaling, CFL 0.16 for P^2 and 0.3 for P^1 (the
    paper's numbers), device-driven steps with the run state (t, dt, max wave
    speed) read back after every step.  Reports the step count, the whole
    run's wall time and rate, and the final state's density and pressure
    ranges (cell averages) and troubled-cell count."""
    import torch
    import crkdg_inputs as inp
    import bench
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()
    cfl = cfl or (0.16 if k == 2 else 0.3)
    stream = torch.cuda.Stream()
    st = inp.dmr_states()
    mesh, _ = bench.dmr_mesh(B, inp, nx, ny)
    s = B.Solver(mesh, k, B.BASIS_P, GTB.SSPRK3, B.EULER, B.F32 if precision == "f32" else B.F64,
                 stream=stream.cuda_stream)
    s.project_function(lambda X, Y: inp.dmr_ic(X, Y, st))
    s.limit(50.0)
    s.positivity(1e-10)
    cap = 40000
    mon = torch.zeros(cap, 5, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.advance(1, cfl, T)
    s.run_state_async(mon[0].data_ptr())
    n = 1
    while True:
        if n % 256 == 0:
            stream.synchronize()
            if mon[n - 1, 0] >= T * (1 - 1e-12) or mon[n - 1, 1] <= 0.0:
                break
        if n >= cap:
            break
        s.step_device()
        s.run_state_async(mon[n].data_ptr())
        n += 1
    code, status = s.sync()
    wall = time.perf_counter() - t0
    r = mon[:n].numpy()
    steps = int(np.count_nonzero(np.concatenate([[1.0], r[:-1, 1]]) > 0.0))
    troubled = s.troubled_count()
    u = s.get_state()
    rho = u[0, 0]
    mx, my, E = u[1, 0], u[2, 0], u[3, 0]
    p = 0.4 * (E - 0.5 * (mx * mx + my * my) / rho)
    nm = u.shape[1]
    s.close()
    return {"study": "dmr_full", "mesh": "%dx%d" % (nx, ny), "k": k, "cfl": cfl, "T": float(r[n - 1, 0]),
            "steps": steps, "wall_s": wall, "dof_updates_per_s": nx * ny * 4 * nm * steps / wall,
            "status": status, "code": code, "rho_min": float(rho.min()), "rho_max": float(rho.max()),
            "p_min": float(p.min()), "p_max": float(p.max()), "troubled_last_step": int(troubled)}


def build_lib():
    from paper_2307_06471_gb300 import build
    build.build()


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["vortex", "ensemble", "learned", "compact", "advection1d", "advection2d",
                                     "advection_hbm", "dmr_full", "precision_rates", "matched_l1",
                                     "indicator_rates"])
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--sizes", default="80,160,320")
    ap.add_argument("--T", type=float, default=10.0)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--limit-mode", default="pass", choices=["pass", "fused"])
    a = ap.parse_args()
    if a.study == "vortex":
        r = vortex(tuple(int(x) for x in a.sizes.split(",")), a.T, a.precision)
    elif a.study == "learned":
        r = learned()
    elif a.study == "compact":
        r = compact(precision=a.precision)
    elif a.study == "advection1d":
        r = advection1d()
    elif a.study == "advection2d":
        r = advection2d_inflow()
    elif a.study == "advection_hbm":   # --sizes N,steps (a smaller case, e.g. for a profiler)
        r = advection_hbm(*(int(v) for v in a.sizes.split(",")[:2])) if a.sizes != "80,160,320" else advection_hbm()
    elif a.study == "precision_rates":   # --sizes N --steps K --precision f32,f32d,...
        build_lib()
        r = precision_rates(int(a.sizes.split(",")[0]) if a.sizes != "80,160,320" else 1280, a.steps,
                            variants=tuple(a.precision.split(",")) if a.precision != "f32" else
                            ("f32", "f32c", "f32d", "f64"))
    elif a.study == "indicator_rates":   # --sizes N --steps K
        build_lib()
        r = indicator_rates(int(a.sizes.split(",")[0]) if a.sizes != "80,160,320" else 2048, a.steps)
    elif a.study == "matched_l1":
        build_lib()
        r = matched_l1(T=a.T if a.T != 10.0 else 1.0)
    elif a.study == "dmr_full":
        r = dmr_full(*(int(v) for v in a.sizes.split(",")[:3])) if a.sizes != "80,160,320" else dmr_full()
    else:
        r = ensemble(a.n, a.steps, a.precision, limit_mode=a.limit_mode)
    print(json.dumps(r, default=float))
