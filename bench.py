#!/usr/bin/env python3
"""Throughput of the compact RKDG (cRKDG) time step on GB300.

Workload (one GPU): the double Mach reflection of the paper's Sec. 4.2.2 --
2D Euler (gamma = 1.4), Mach 10 shock at 60 degrees, [0,4] x [0,1],
1920 x 480 cells, P^2 (24 DOF per cell), SSP-RK3 in Butcher form, TVB-minmod
limiter M = 50 once per step followed by the positivity-preserving scaling
(Zhang--Shu; needed at Mach 10), FP32 bulk with FP64 CFL / conservation
reductions, CFL 0.16.  Synthetic: the analytic initial data, advanced W
warm-up steps before timing.

A "step" is one full cRKDG time step (the previous step's limiter, all inner
stages, the final DG stage with boundary data, the FP64 reductions that give
the next dt) -- three launches: the limiter pass, the fused step kernel with
dt read on the device, and its one-block finalize (slot reduction, next dt).

value  : DOF-updates/s = cells * 24 * K / (sum of per-step device times),
         CUDA events on the solver's stream around each step, L2 flushed
         between timed steps, outside the events (256 MiB written, then
         256 MiB of another buffer read, so the flush's own dirty lines are
         written back before the events; --flush write: the write alone).
e2e    : the same metric through the C ABI with host buffers, wall clock:
         upload of the FP64 initial state from pinned host memory, K
         device-driven steps (dt from each step's own reduction) with each
         step's run state (t, dt, max wave speed) read back asynchronously
         into pinned memory, download of the FP64 state into pinned memory.
roofline : the fused step kernel (with its finalize) against the FP32 FMA
         peak measured on this GPU by the library's probe (alu_peaks: FP32,
         packed FP32x2 and FP64 FMA rates), HBM GB/s as context.
fp64_arm : the same DMR workload with the FP64 state (CRKDG_F64), device
         timed the same way over --fp64-steps steps.
matched_l1 : the isentropic vortex (Q^2, RK4, CFL 0.1, T = --matched-T) in
         FP64 on 80/120/160/240/320^2 and, on 80/160/320^2, in FP32, the
         compensated FP32 state and
         the deviation-form FP32 step (CRKDG_F32D) on the same meshes; each
         FP32 run matched to the FP64 run of at most its density L1 error;
         speedup = FP64 wall time / FP32 wall time (host clock, synchronised
         device-driven runs).
--impl reference : the FP64 CPU oracle (numpy) on a bounded sample of the
         same workload (a 240 x 60 mesh of the same problem), timed on the
         host cores; rank 0 only.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(name="dmr_1920x480_P2_ssprk3_tvb50_f32", nx=1920, ny=480, k=2, basis="P", tab="ssprk3", M=50.0,
          pp_eps=1e-10, cfl=0.16, T=0.2, box=(0.0, 4.0, 0.0, 1.0))
METRIC = "2D Euler P2 cRKDG DOF-updates/s"
UNIT = "DOF-updates/s"
SAMPLE = dict(nx=240, ny=60)      # bounded oracle sample of the same problem

# ncu dram traffic of the step kernel for this workload, per launch, and the
# hash of the kernel sources it was taken with (None until captured)
TRAFFIC = {"bytes": 138982144, "src_hash": "a4da2c6e8e44eed5"}


def kernel_src_hash():
    """Hash of the step kernel's sources without their comments: a change of
    code (not of a comment) voids the recorded traffic."""
    import re
    h = hashlib.sha256()
    for f in ("step2d.cuh", "common.cuh", "limiter.cuh", "tables.cuh"):
        with open(os.path.join(ROOT, "paper_2307_06471_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()[:16]


def dmr_mesh(B, inp, nx, ny):
    st = inp.dmr_states()
    post, pre = list(st["post"]), list(st["pre"])
    bc = [B.BC_DIRICHLET, B.BC_OUTFLOW, B.BC_DIRICHLET, B.BC_DIRICHLET]
    fn = [B.FN_CONST, 0, B.FN_DMR_BOTTOM, B.FN_DMR_TOP]
    params = [post, None, post + [st["x0"]], post + pre + [st["x0"], st["slope"], st["xspeed"]]]
    return B.make_mesh(2, nx, ny, WL["box"], bc, fn, params), st


def make_solver(stream_handle, nx, ny, precision="f32"):
    import crkdg_inputs as inp
    from paper_2307_06471_gb300 import binding as B
    from paper_2307_06471_gb300 import tableaux as GTB
    mesh, st = dmr_mesh(B, inp, nx, ny)
    s = B.Solver(mesh, WL["k"], B.BASIS_P, GTB.BY_NAME[WL["tab"]], B.EULER, B.F32 if precision == "f32" else B.F64,
                 stream=stream_handle)
    s.project_function(lambda X, Y: inp.dmr_ic(X, Y, st))
    s.limit(WL["M"])
    s.positivity(WL["pp_eps"])
    return s


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def alu_peaks(stream_handle):
    """FP32 (scalar and packed FP32x2) and FP64 FMA peaks of this GPU,
    measured by the library's FMA probe (crkdg_alu_peak) just before the
    timed region."""
    from paper_2307_06471_gb300 import binding as B
    out = {}
    for name, kind in (("f32", B.PEAK_F32), ("f32x2", B.PEAK_F32X2), ("f64", B.PEAK_F64)):
        tf, ms, sms = B.alu_peak(kind, reps=9, stream=stream_handle)
        out[name] = {"tflops": tf, "ms_per_launch": ms}
    out["sms"] = sms
    return out


class L2Flush:
    """Between timed steps: write a 256 MiB buffer (larger than the 126 MB
    L2), then (mode "write+read", the default) read another 256 MiB buffer,
    so that the write's dirty lines are written back during the flush and
    not by the timed kernels that evict them."""

    def __init__(self, mode):
        import torch
        n = 256 * 1024 * 1024 // 4
        self.mode = mode
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(n, dtype=torch.float32, device="cuda") if mode == "write+read" else None
        self.sink = torch.zeros(1, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.zero_()
        if self.r is not None:
            self.sink.copy_(self.r.sum())

    def describe(self):
        return ("flushed between timed steps: 256 MiB written" +
                (", then 256 MiB of another buffer read (the write-backs land in the flush)"
                 if self.r is not None else ""))


def timed_steps(s, stream, flush, steps, use_pass):
    """Device times (ms) of `steps` whole steps, each bracketed by CUDA events
    on the solver's stream, L2 flushed before each (outside the events):
    (total, mean limiter pass, mean step kernel + finalize)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush()
        starts[i].record(stream)
        if use_pass:
            s.apply_limit()        # limiter pass of the previous step's final stage (in place)
        mids[i].record(stream)
        s.step_device()            # fused cRKDG step kernel + its one-block finalize
        ends[i].record(stream)
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    lim = sum(a.elapsed_time(b) for a, b in zip(starts, mids)) / steps
    ker = sum(a.elapsed_time(b) for a, b in zip(mids, ends)) / steps
    return total, lim, ker


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_sample(nx, ny, steps, warm=1, procs=1):
    """Run the FP64 oracle on the bounded sample in `procs` single-threaded
    child processes at once; returns (aggregate DOF-updates/s, seconds of
    the slowest copy, steps per copy)."""
    code = r"""
import json, sys, time, os
sys.path.insert(0, %r)
import numpy as np
import crkdg_inputs as inp
from oracle import tableaux as TB
from oracle.dg2d import DG2D, crkdg_step, cfl_dt_2d
from oracle.limiter import tvb_limit, positivity_limit
from oracle.physics import Euler
nx, ny, steps, warm = %d, %d, %d, %d
st = inp.dmr_states()
post, pre = st['post'], st['pre']
def refl(u, axis):
    o = np.array(u, copy=True); o[..., 1 + axis] = -o[..., 1 + axis]; return o
bc = {'W': ('dirichlet', lambda X, Y, t: np.broadcast_to(post, np.shape(X) + (4,)).copy()), 'E': 'outflow',
      'S': ('custom', lambda u, X, Y, t: np.where((np.asarray(X) < st['x0'])[..., None], post, refl(u, 1))),
      'N': ('dirichlet', lambda X, Y, t: np.where((np.asarray(X) < st['x0'] + st['slope'] * np.asarray(Y) + st['xspeed'] * t)[..., None], post, pre))}
dg = DG2D(nx, ny, (0, 4, 0, 1), 2, 'P', Euler(1.4, 2), bc)
u = dg.project(lambda X, Y: inp.dmr_ic(X, Y, st), nq=3)
lim = lambda v, t: positivity_limit(dg, tvb_limit(dg, v, 50.0, t)[0], 1e-10)
u = lim(u, 0.0)
t = 0.0
for i in range(warm + steps):
    if i == warm:
        t0 = time.perf_counter()
    dt = cfl_dt_2d(dg, u, 0.16)
    u = crkdg_step(dg, u, t, dt, TB.SSPRK3, limiter=lim)
    t += dt
el = time.perf_counter() - t0
print(json.dumps({'sec': el, 'steps': steps, 'dofs': nx * ny * 24}))
""" % (ROOT, nx, ny, steps, warm)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    # procs single-threaded copies at once, one per host core: the sample's
    # steps are independent of each other's, so the aggregate is
    # procs * DOF * steps over the slowest copy's time
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    res = []
    for pr in ps:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    sec = max(d["sec"] for d in res)
    return procs * res[0]["dofs"] * res[0]["steps"] / sec, sec, res[0]["steps"]


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return rank, ws


def aggregate(dev_ms, dof_per_rank, steps):
    """Whole-job figures of N independent replicas: the slowest rank's device
    time (max over ranks) and value = N * DOF * steps / that time."""
    ws = 1
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            import torch
            ws = dist.get_world_size()
            dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
            t = torch.tensor([float(dev_ms)], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dev_ms = float(t.item())
    except ImportError:
        pass
    return dev_ms, ws * dof_per_rank * steps / (dev_ms * 1e-3), ws


def run_reference(args):
    rank, ws = dist_init()
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    # bound the run to a few minutes: ~0.3 s per oracle step at 240 x 60
    nx, ny = SAMPLE["nx"], SAMPLE["ny"]
    if steps > 300:
        nx, ny = 120, 30
    ncores = os.cpu_count() or 1
    rate, sec, n = oracle_sample(nx, ny, steps, warm=max(1, min(args.warmup, 3)), procs=ncores)
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / n, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL["name"], "sample_mesh": "%dx%d" % (nx, ny), "k": 2, "basis": "P",
                       "tableau": "ssprk3", "limiter": "tvb M=50"},
            "impl": "reference",
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": "FP64 numpy oracle, DMR %dx%d P2 SSP-RK3 + TVB + positivity, %d steps in "
                                       "each of %d single-threaded copies run at once (one per host core), "
                                       "aggregate rate; %s" % (nx, ny, n, ncores, cpu_model())},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=float))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 arm of the same workload")
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--no-matched-l1", action="store_true", help="skip the vortex comparison at matched L1")
    ap.add_argument("--flush", default="write+read", choices=["write", "write+read"],
                    help="L2 flush between timed steps (see L2Flush)")
    ap.add_argument("--matched-T", type=float, default=1.0)
    ap.add_argument("--limit-mode", default="pass", choices=["pass", "fused"],
                    help="pending limiter as a separate pass before the step kernel, or fused into its load")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    import numpy as np
    import torch

    rank, ws = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2307_06471_gb300 import build
    from paper_2307_06471_gb300.workcount import step_bytes_per_cell, step_flops_per_cell
    from paper_2307_06471_gb300 import tableaux as GTB
    build.build()

    nx, ny = WL["nx"], WL["ny"]
    cells = nx * ny
    dof = cells * 24
    stream = torch.cuda.Stream()
    s = make_solver(stream.cuda_stream, nx, ny)
    from paper_2307_06471_gb300 import binding as B
    use_pass = args.limit_mode == "pass"
    s.set_limit_mode(B.LIMIT_PASS if use_pass else B.LIMIT_FUSED)
    if args.autotune:
        s.autotune()
    seg_rows, wpb = s.get_launch()
    flush = L2Flush(args.flush)

    # measured FP32 / FP64 FMA peaks (the roofline's denominator), before the
    # timed region
    alu = alu_peaks(stream.cuda_stream)
    # warm-up: device-driven steps (first dt from a reduction of the state)
    s.advance(args.warmup, WL["cfl"], WL["T"])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        dev_ms, lim_ms, step_kernel_ms = timed_steps(s, stream, flush, args.steps, use_pass)
    code, status = s.sync()
    t_sim = s.time()
    dev_ms, value, _ = aggregate(dev_ms, dof, args.steps)
    ms_per_step = dev_ms / args.steps

    A, b = GTB.BY_NAME[WL["tab"]]
    # the step kernel's own work: the limiter's counts there only when it runs fused
    fpc = step_flops_per_cell(WL["k"], WL["basis"], "euler", A, b, limiter=not use_pass)
    bpc = step_bytes_per_cell(WL["k"], WL["basis"], "euler", 4)
    clocks = clk.summary()
    peaks, peak_kind = measured_peaks()
    fp32_peak = alu["f32"]["tflops"]              # measured: FP32 FMA probe on this GPU
    # roofline of the dominant kernel (the fused step) from its own event-timed
    # duration; the limiter pass is HBM bound: it reads the 24 modes of every
    # cell (neighbour averages hit L1/L2) and rewrites only the limited cells
    achieved = fpc * cells / (step_kernel_ms * 1e-3) / 1e12
    hbm = bpc * cells / (step_kernel_ms * 1e-3) / 1e9
    lim_bytes = 24 * 4 * cells
    limit_pass = ({"ms": lim_ms, "read_bytes": lim_bytes, "gbs": lim_bytes / (lim_ms * 1e-3) / 1e9,
                   "frac_of_measured_hbm": lim_bytes / (lim_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
                  if use_pass else None)
    traffic = TRAFFIC["bytes"] if TRAFFIC["src_hash"] == kernel_src_hash() else None

    e2e = None
    if not args.no_e2e:
        estream = torch.cuda.Stream()
        import crkdg_inputs as inp  # noqa: F401
        s2 = make_solver(estream.cuda_stream, nx, ny)
        s2.advance(args.warmup, WL["cfl"], WL["T"])
        # FP64 host state (input of the timed run) and the output buffer, both
        # in pinned host memory
        host = torch.empty(tuple(s2.shape), dtype=torch.float64, pin_memory=True).numpy()
        s2.get_state(out=host)
        out = torch.empty(tuple(s2.shape), dtype=torch.float64, pin_memory=True).numpy()
        mon = torch.zeros(args.steps, 5, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.set_state(host, 0.0)
        s2.limit(WL["M"])
        s2.positivity(WL["pp_eps"])
        # device-driven run: dt from the step's own FP64 reduction; each step's
        # run state (t, dt, max wave speed) is read back asynchronously
        s2.advance(1, WL["cfl"], WL["T"])
        s2.run_state_async(mon[0].data_ptr())
        for i in range(1, args.steps):
            s2.step_device()
            s2.run_state_async(mon[i].data_ptr())
        code2, _ = s2.sync()
        s2.get_state(out=out)
        wall = time.perf_counter() - t0
        assert code2 == 0 and bool((mon[:, 1] > 0).all())
        e2e = {"value": ws * dof * args.steps / wall, "unit": UNIT,
               "h2d_bytes_per_step": host.nbytes // args.steps,
               "d2h_bytes_per_step": 40 + out.nbytes // args.steps,
               "note": "FP64 host state in pinned memory uploaded once (rounded to FP32 on the GPU), device-driven steps "
                       "(crkdg_step_device), the run state (t, dt, max wave speed) read back every step "
                       "into pinned memory, state downloaded once into pinned memory (widened to FP64 on the GPU); bytes "
                       "per step = transfers / steps"}
        s2.close()

    # the same workload in FP64 on the GPU (the reference precision): the
    # same state after the warm-up, device-timed the same way
    fp64_arm = None
    if not args.no_fp64:
        s64 = make_solver(stream.cuda_stream, nx, ny, precision="f64")
        s64.set_limit_mode(B.LIMIT_PASS if use_pass else B.LIMIT_FUSED)
        s64.advance(args.warmup, WL["cfl"], WL["T"])
        n64 = min(args.steps, args.fp64_steps)
        t64, l64, k64 = timed_steps(s64, stream, flush, n64, use_pass)
        c64, st64 = s64.sync()
        fp64_arm = {"value": dof * n64 / (t64 * 1e-3), "unit": UNIT, "ms_per_step": t64 / n64, "steps": n64,
                    "limit_pass_ms": l64 if use_pass else None, "step_kernel_ms": k64, "status": st64,
                    "fp32_speedup": (t64 / n64) / ms_per_step,
                    "note": "CRKDG_F64: the same DMR workload and launch sequence with an FP64 state and FP64 "
                            "arithmetic (GB300's FP64 FMA rate is the f64 entry of alu_peaks)"}
        s64.close()

    # the headline comparison at matched L1 error: the isentropic vortex (the
    # paper-style exact-solution test, Q^2 RK4) to a short T in FP64 and in the
    # FP32 variants, each FP32 run matched to the FP64 run of equal or lower
    # error (same mesh within 10 %, else the coarsest FP64 mesh that reaches it)
    matched = None
    if rank == 0 and ws == 1 and not args.no_matched_l1:
        from paper_2307_06471_gb300 import studies
        matched = studies.matched_l1(T=args.matched_T)
        # the same precisions' step rates on a mesh that fills the GPU (the
        # 320^2 vortex holds ~3 warps per SM, so its rates are latency bound)
        matched["rates_full_gpu"] = studies.precision_rates()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        rate1, sec1, n1 = oracle_sample(SAMPLE["nx"], SAMPLE["ny"], 30)
        rate, sec, n = oracle_sample(SAMPLE["nx"], SAMPLE["ny"], 10, procs=ncores)
        cpu = {"value": rate, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": "FP64 numpy oracle, DMR %dx%d P2 SSP-RK3 + TVB + positivity, %d steps in each of %d "
                         "single-threaded copies run at once (one per host core; %.1f s), aggregate rate; %s"
                         % (SAMPLE["nx"], SAMPLE["ny"], n, ncores, sec, cpu_model()),
               "single_thread": {"value": rate1, "cores": 1, "steps": n1, "sec": sec1}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WL["name"], "cells": cells, "dof_per_cell": 24, "k": 2, "basis": "P",
                           "tableau": "ssprk3", "limiter": "tvb M=50 + positivity scaling (once per step)", "cfl": WL["cfl"],
                           "reductions": "fp64", "l2": flush.describe(),
                           "launch": {"seg_rows": seg_rows, "warps_per_block": wpb},
                           "limit_mode": "separate pass + fused step" if use_pass else "fused into the step's load",
                           "parallelism": "replicas" if ws > 1 else "single"},
                "roofline": {"kernel": "step2d_kernel<float,2,P,Euler>", "kernel_ms": step_kernel_ms,
                             "kernel_ms_covers": "the step launch and its one-block finalize launch "
                                                 "(reduction of the per-warp slots, next dt)",
                             "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": achieved / fp32_peak, "traffic": traffic,
                             "peak_note": "measured: FP32 FMA probe (crkdg_alu_peak, scalar FFMA chains, %d SMs, "
                                          "median of 9 launches) on this GPU just before the timed region"
                                          % alu["sms"],
                             "flop_per_cell": fpc, "hbm_gbs": hbm, "hbm_frac_of_measured": hbm / peaks["hbm_gbs"],
                             "hbm_peak_source": peak_kind},
                "limit_pass": limit_pass, "alu_peaks": alu, "fp64_arm": fp64_arm, "matched_l1": matched,
                "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps * (3 if use_pass else 2),
                "status": {"code": code, "bits": status, "t_sim": t_sim},
                "cpu_baseline": cpu}
        print(json.dumps(line, default=float))
    s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
