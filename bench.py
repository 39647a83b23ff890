"""Benchmark of the MFWH hot path on GB300.

One step = one GMRES(20) cycle of the MFWH solve of the 1025^2, N_f = 8
workload, from a zero initial guess: b = Pi(0) (one forced wave solve), 20
Arnoldi steps on (I - S) V = b (one homogeneous wave solve, two Gram-Schmidt
passes and a Givens update each), the solution update, and the Helmholtz
residual check of the result.  Every wave solve is N_t leapfrog steps fused
with the N_f filter accumulations and, on the last step, the B^{-1} solve.

Metric: Gpts/s = interior grid points x time steps x wave solves / time.
With --solve, one unrestarted GMRES solve to a relative residual of 1e-8 is
timed as well (time to solution).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--solve]

Multi-GPU (torchrun): every rank solves its own independent problem (seed
offset by the rank); no data-path collective; weak scaling.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RESTART = 20
TOL = 1e-8
MAX_ITERS = RESTART          # one restart cycle per step
SOLVE_MAX_ITERS = 800        # unrestarted solve for the time to solution
WORD = 8  # float64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve", action="store_true", help="also time one unrestarted solve to 1e-8")
    ap.add_argument("--no-tts", action="store_true",
                    help="skip the time to a 1e-6 Helmholtz residual (FP64 and mixed arms)")
    ap.add_argument("--tts-inner", type=float, default=1e-6,
                    help="inner GMRES tolerance of the time-to-solution arms")
    ap.add_argument("--tts-relax", type=float, default=1e-2,
                    help="mixed arm: FP32 products once the inner residual is below this")
    ap.add_argument("--time-block", type=int, default=0,
                    help="leapfrog steps per kernel launch (0 = library default)")
    ap.add_argument("--tile-shape", type=int, default=0,
                    help="tile shape of the blocked kernels (library's tile_shape)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 wave-solve leg")
    ap.add_argument("--fp32-only", action="store_true",
                    help="run only the FP32 leg and print it (for profiling its kernel)")
    ap.add_argument("--batched", action="store_true",
                    help="run the batched workload (independent 2D problems solved concurrently)")
    ap.add_argument("--batch", type=int, default=48, help="problems in the batched workload")
    ap.add_argument("--default-batch", type=int, default=16,
                    help="problems of the batched workload in the default line's batched leg")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the default line's batched leg (lockstep and concurrent solves)")
    ap.add_argument("--batch-iters", type=int, default=10,
                    help="GMRES(10) Arnoldi steps per problem in the batched workload")
    ap.add_argument("--batch-mem-gb", type=float, default=180.0,
                    help="device-memory budget of the batched workload")
    ap.add_argument("--warm-start", action="store_true",
                    help="train the warm-start network on MFWH solutions and compare GMRES from "
                         "its prediction with GMRES from zero")
    ap.add_argument("--cnn", action="store_true",
                    help="time the warm-start network's forward pass and training step (tensor-"
                         "core convolutions) on a synthetic batch")
    ap.add_argument("--cnn-batch", type=int, default=48, help="images per batch with --cnn")
    ap.add_argument("--ws-n", type=int, default=128, help="cells per axis of the warm-start workload")
    ap.add_argument("--ws-train", type=int, default=683, help="training problems (6 samples each)")
    ap.add_argument("--ws-test", type=int, default=24, help="held-out problems")
    ap.add_argument("--ws-epochs", type=int, default=15)
    ap.add_argument("--ws-gen-seconds", type=float, default=300.0,
                    help="time limit of the training-data generation")
    ap.add_argument("--oracle-timings", action="store_true",
                    help="with --impl reference: also the oracle's times on the 65^2, 1025^2 "
                         "and 257^3 workloads")
    ap.add_argument("--small", action="store_true",
                    help="the 65^2, N_f = 2 workload on the GPU (fixed-point and GMRES times)")
    ap.add_argument("--implicit-scaling", action="store_true",
                    help="implicit fourth-order MFWH from 129^2 to 2049^2 (the paper's MG table);"
                         " with --cube its 3D analogue from 33^3 to 129^3")
    ap.add_argument("--implicit", action="store_true",
                    help="implicit trapezoidal time stepping (multigrid) beside explicit FP64")
    ap.add_argument("--cube-n", type=int, default=256,
                    help="cells per axis of the 3D workload (256: the 257^3 configuration)")
    ap.add_argument("--cube", action="store_true",
                    help="run the 3D two-layer workload (257^3, N_f = 4, GMRES(15) cycle)")
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi (for runs under a profiler)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 rate of GB300 from its unit counts: 152 SMs x 2 FP64 FMA lanes per SM and cycle (the
# peak ncu reports for DFMA on sm_103) x 2 flops x the 2070 MHz maximum SM clock = 1.259
# TFLOP/s (the nominal figure is 1.25).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def bytes_per_point_step(nf, forced):
    """Algorithmic HBM bytes of one unblocked leapfrog+filter point-step:
    read W^n, W^{n-1}, q_m (and f_m when forced), write W^{n+1}, q_m."""
    return (3 + (3 if forced else 2) * nf) * WORD


def blocked_bytes_per_point_launch(nf, forced):
    """Algorithmic HBM bytes per interior point of one temporally blocked FP64 launch (any
    number of steps): read and write both wave levels and the N_f float-pair filter sums,
    and read the N_f forcing grids once when forced."""
    return (4 + 2 * nf + (nf if forced else 0)) * WORD


def flops_per_point_step(nf, forced, dim=2):
    """FP64 flops of one point-step as the step kernel executes them: dim adds for the
    neighbour pairs, dim + 1 FMAs for the leapfrog (the centre term with W^{n-1} and one per
    axis), N_f FMAs for the forcing when forced; an FMA counts 2.  The float-pair split of
    W^{n+1} and the N_f filter updates run on the integer and FP32 pipes and are not counted."""
    fma = dim + 1 + (nf if forced else 0)
    return 2 * fma + dim


def kernel_traffic(profile, kernel_key):
    """dram bytes per launch from a committed ncu summary, if it is for this kernel source."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != kernel_key:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _code_only(text):
    """Source text without comments and without whitespace, so that the hash of a kernel's
    source changes with its code and not with its comments."""
    import re
    text = re.sub(rb"/\*.*?\*/", b"", text, flags=re.S)
    text = re.sub(rb"//[^\n]*", b"", text)
    return re.sub(rb"\s+", b"", text)


def _region(path, end_marker):
    with open(os.path.join(ROOT, "paper_2507_23613_gb300", "csrc", path), "rb") as fh:
        text = fh.read()
    cut = text.find(end_marker.encode())
    return _code_only(text if cut < 0 else text[:cut])


def kernel_source_key():
    """Hash of the FP64 step kernels' source: wave.cu up to the residual kernels, the
    kernel argument structs of kernels.h and the float-pair filter sums (fpair.cuh)."""
    h = hashlib.sha256()
    h.update(_region("wave.cu", "// ---- Helmholtz residual"))
    h.update(_region("kernels.h", "// Arguments of one temporally blocked launch"))
    h.update(_region("fpair.cuh", "\0"))
    return h.hexdigest()[:16]


def blocked_kernel_source_key():
    """Hash of the FP64 temporally blocked kernels' source (wave_tb_kernels.cuh), their
    argument structs (kernels.h) and the float-pair arithmetic (fpair.cuh)."""
    h = hashlib.sha256()
    h.update(_region("wave_tb_kernels.cuh", "\0"))
    h.update(_region("kernels.h", "// ---- FP32 path"))
    h.update(_region("fpair.cuh", "\0"))
    return h.hexdigest()[:16]


def fp32_kernel_source_key():
    """Hash of the FP32 blocked kernel's source (wave32_kernels.cuh)."""
    h = hashlib.sha256()
    h.update(_region("wave32_kernels.cuh", "// ---- init and conversion"))
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_sample_problem(make, steps):
    """The oracle's problem for the workload inputs.<make[0]>(**make[1]), cut to its first
    `steps` time steps (test infrastructure)."""
    from oracle import wave as W
    from paper_2507_23613_gb300 import inputs
    import copy
    wl = getattr(inputs, make[0])(**make[1])
    g = W.Grid(wl.n, wl.length)
    prob = W.make_problem(g, wl.omega, wl.forcing, c2=wl.c2, cfl=wl.cfl, n_p=wl.n_p)
    n_full = prob.setup.n_t
    sub = copy.copy(prob)
    sub.setup = copy.copy(prob.setup)
    sub.setup.n_t = min(steps, n_full)
    sub.setup.w = prob.setup.w[:sub.setup.n_t + 1]
    return sub, wl, n_full


def _oracle_worker(make, steps, commands, results):
    """One host process of the CPU baseline: build the sample once, then time the oracle's
    homogeneous map over it each time a command arrives (None ends the process)."""
    from oracle import wave as W
    sub, wl, _ = _oracle_sample_problem(make, steps)
    v = np.zeros_like(wl.forcing)
    results.put(None)                       # ready
    while commands.get() is not None:
        t0 = time.perf_counter()
        W.apply_Pi(sub, v, forced=False)
        results.put(time.perf_counter() - t0)


class OracleRig:
    """The oracle's map (test infrastructure, timed as it stands) on the host cores: `workers`
    processes (default: all cores), each running the homogeneous map of the workload
    inputs.<make[0]>(**make[1]) on the full grid for the same bounded number of time steps,
    numpy single-threaded in each.  The number of steps is calibrated on one process to take
    about budget_s / 4 .. budget_s; one sample is all processes' point-steps over the slowest
    process's time, started together."""

    def __init__(self, make, budget_s=15.0, workers=None):
        import multiprocessing as mp
        from oracle import wave as W
        self.workers = workers or os.cpu_count() or 1
        steps = 4
        while True:
            sub, wl, n_full = _oracle_sample_problem(make, steps)
            t0 = time.perf_counter()
            W.apply_Pi(sub, np.zeros_like(wl.forcing), forced=False)
            dt = time.perf_counter() - t0
            if dt > budget_s / 4 or steps >= n_full:
                break
            steps = min(n_full, int(steps * max(2.0, budget_s / max(dt, 1e-3))))
        self.steps, self.n_full, self.wl, self.last_dt = steps, n_full, wl, dt
        self.procs = []
        if self.workers > 1:
            ctx = mp.get_context("spawn")
            keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")
            saved = {k: os.environ.get(k) for k in keys}
            os.environ.update({k: "1" for k in keys})
            self.results = ctx.Queue()
            self.cmds = [ctx.Queue() for _ in range(self.workers)]
            for c in self.cmds:
                pr = ctx.Process(target=_oracle_worker, args=(make, steps, c, self.results),
                                 daemon=True)
                pr.start()
                self.procs.append(pr)
            for k, val in saved.items():
                if val is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = val
            for _ in self.procs:
                self.results.get(timeout=900)       # every worker has built its sample

    def run(self):
        """One sample: Gpts/s and a description."""
        if self.procs:
            for c in self.cmds:
                c.put(1)
            self.last_dt = max(self.results.get(timeout=900) for _ in self.procs)
        wl = self.wl
        pts = wl.interior_points * self.steps * self.workers
        return {"value": pts / self.last_dt / 1e9, "unit": "Gpts/s", "cores": self.workers,
                "kind": "oracle",
                "sample": (f"numpy oracle, homogeneous map, {self.workers} process(es) x "
                           f"{self.steps} of {self.n_full} leapfrog+filter steps each on the full "
                           f"{'x'.join(str(k + 1) for k in wl.n)} grid, N_f={wl.nf}, slowest "
                           f"{self.last_dt:.1f} s, numpy single-threaded per process")}

    def close(self):
        for c in getattr(self, "cmds", []):
            c.put(None)
        for pr in self.procs:
            pr.join(timeout=60)
        self.procs = []


def cpu_baseline(make, budget_s=15.0, workers=None):
    """One sample of the oracle on the host cores (OracleRig)."""
    rig = OracleRig(make, budget_s, workers)
    try:
        return rig.run()
    finally:
        rig.close()


def oracle_timings(args):
    """The FP64 oracle timed on the host (part of the reference arm): the 65^2 workload in
    full (40 fixed-point iterations, and GMRES to 1e-8), the 1025^2 and 257^3 maps on a
    bounded number of steps with the per-step rate extrapolated to a whole map (labelled as
    such)."""
    from oracle import wave as W
    from paper_2507_23613_gb300 import inputs
    out = {"cores": 1, "kind": "oracle",
           "note": "the 65^2 runs use one core; the 1025^2 and 257^3 samples use all cores"}
    wl = inputs.square_small()
    g = W.Grid(wl.n, wl.length)
    prob = W.make_problem(g, wl.omega, wl.forcing, cfl=wl.cfl, n_p=wl.n_p)
    t0 = time.perf_counter()
    W.fixed_point_iteration(prob, np.zeros_like(wl.forcing), 40)
    t_fpi = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, ginfo = W.gmres(prob, restart=20, tol=1e-8, max_iters=400)
    t_gm = time.perf_counter() - t0
    out["square65_nf2"] = {"fpi40_s": round(t_fpi, 3), "gmres_1e-8_s": round(t_gm, 3),
                           "gmres_iterations": ginfo.iterations, "n_t": prob.setup.n_t}
    for name, make in (("square1025_nf8", ("square_large", {"seed": args.seed})),
                       ("cube257_nf4", ("cube_layered", {"seed": args.seed + 1000}))):
        wl = getattr(inputs, make[0])(**make[1])
        info = cpu_baseline(make, budget_s=10.0)
        n_t = W.make_problem(W.Grid(wl.n, wl.length), wl.omega, wl.forcing, c2=wl.c2,
                             cfl=wl.cfl, n_p=wl.n_p).setup.n_t
        per_map = wl.interior_points * n_t / (info["value"] * 1e9)
        out[name] = {"gpts_s": round(info["value"], 4), "sample": info["sample"], "n_t": n_t,
                     "map_s_extrapolated": round(per_map, 1)}
    return out


def run_small(args):
    """The 65^2, N_f = 2 workload on the GPU through the C ABI: 40 fixed-point iterations and
    GMRES(20) to 1e-8 from zero (wall time around each synchronous call)."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import build, inputs
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    wl = inputs.square_small()
    s = M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(), n_p=wl.n_p,
                 cfl=wl.cfl)
    v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
    s.solve_fpi(v, 40)                                   # warm-up
    torch.cuda.synchronize()
    v.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.solve_fpi(v, 40)
    torch.cuda.synchronize()
    t_fpi = time.perf_counter() - t0
    v.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = s.solve_gmres(v, restart=20, tol=1e-8, max_iters=400, raise_on_error=False)
    torch.cuda.synchronize()
    t_gm = time.perf_counter() - t0
    s.close()
    print(json.dumps({"metric": "65^2 N_f = 2 solve times", "unit": "s", "value": round(t_gm, 4),
                      "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": "square65_nf2"},
                      "fpi40_s": round(t_fpi, 4), "gmres_1e-8_s": round(t_gm, 4),
                      "gmres_iterations": info["iterations"]}), flush=True)


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle (test infrastructure, timed as it stands) on all host
    cores (OracleRig), one bounded sample of the bench workload per step."""
    if rank != 0:
        return
    from paper_2507_23613_gb300 import inputs
    make = ("square_large", {"seed": args.seed})
    wl = inputs.square_large(args.seed)
    rig = OracleRig(make, budget_s=4.0)
    try:
        for _ in range(args.warmup):
            rig.run()
        per = []
        info = None
        for _ in range(args.steps):
            info = rig.run()
            per.append(info["value"])
    finally:
        rig.close()
    value = statistics.mean(per)
    line = {"impl": "reference", "metric": "stencil Gpts/s (+N_f filters)", "value": value,
            "unit": "Gpts/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, rig.n_full),
            "cpu_baseline": {**info, "value": value},
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.oracle_timings:
        line["oracle_timings"] = oracle_timings(args)
    print(json.dumps(line), flush=True)


def fp32_bytes_per_point_launch(nf, forced):
    """Algorithmic HBM bytes per interior point of one blocked FP32 launch (any depth T):
    read and write W and D (4 B each) and the Kahan pairs (2 x 4 B per frequency), read the
    FP32 forcing when forced."""
    return 4 * (4 + 4 * nf + (nf if forced else 0))


def fp32_leg(args, wl, f_dev, stream, n_t):
    """The same GMRES(20) cycle with FP32 wave solves (increment form, filter partial sums
    folded into Kahan pairs once per blocked launch), and the FP32 map's error per
    frequency against the FP64 map."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import _lib
    s32 = M.Solver(wl.n, wl.length, wl.omega, f_dev, stream=stream.cuda_stream, n_p=wl.n_p,
                   cfl=wl.cfl, precision=_lib.PREC_FP32_BLOCKSUM)
    v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")

    def cycle():
        with torch.cuda.stream(stream):
            v.zero_()
        info = s32.solve_gmres(v, restart=RESTART, tol=TOL, max_iters=MAX_ITERS,
                               raise_on_error=False)
        ms, step_launches, launches = s32.last_timing()
        return info, ms, step_launches, launches + 1

    for _ in range(max(1, args.warmup)):
        cycle()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [cycle() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    pi_apps = sum(i[0]["pi_applications"] for i in infos)
    forced_apps = len(infos)
    step_ms = sum(i[1] for i in infos)
    step_launches = sum(i[2] for i in infos)
    alg = wl.interior_points * (forced_apps * fp32_bytes_per_point_launch(wl.nf, True)
                                + (pi_apps - forced_apps) * fp32_bytes_per_point_launch(wl.nf, False))
    launches_per_pi = step_launches / max(pi_apps, 1)
    alg_bytes = alg * launches_per_pi
    gbs = alg_bytes / (step_ms * 1e-3) / 1e9
    hbm_peak, peak_kind = peaks()
    # error of one FP32 map against the FP64 map, per frequency
    rng = np.random.default_rng(11)
    x = rng.normal(size=wl.forcing.shape) * 0.01
    g = x.reshape(wl.nf, wl.n[1] + 1, wl.n[0] + 1)
    g[:, [0, -1], :] = 0.0
    g[:, :, [0, -1]] = 0.0
    xd = torch.from_numpy(x).cuda()
    o32 = torch.empty_like(xd)
    o64 = torch.empty_like(xd)
    s64 = M.Solver(wl.n, wl.length, wl.omega, f_dev, stream=stream.cuda_stream, n_p=wl.n_p,
                   cfl=wl.cfl)
    with torch.cuda.stream(stream):
        s32.apply_Pi(xd, o32, forced=True)
        s64.apply_Pi(xd, o64, forced=True)
    torch.cuda.synchronize()
    a = o32.cpu().numpy().reshape(wl.nf, -1)
    b = o64.cpu().numpy().reshape(wl.nf, -1)
    err = (np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)).tolist()
    s64.close()
    s32.close()
    return {"precision": "fp32 wave steps, Kahan filter pairs folded per launch, FP64 Arnoldi",
            "value": round(wl.interior_points * n_t * pi_apps / (elapsed * 1e-3) / 1e9, 3),
            "unit": "Gpts/s", "ms_per_step": round(elapsed / args.steps, 3),
            "roofline": {"bound": "hbm", "kernel": "k_tb2d32 (blocked FP32 leapfrog + filters)",
                         "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(gbs / hbm_peak, 4), "peak_source": peak_kind,
                         "alg_bytes_per_launch": round(alg_bytes / max(step_launches, 1)),
                         "avg_launch_us": round(step_ms * 1e3 / max(step_launches, 1), 2),
                         "steps_per_launch": round(n_t / launches_per_pi, 2),
                         "traffic": kernel_traffic("k_tb2d32_square1025_nf8.txt",
                                                   fp32_kernel_source_key())},
            "pi_rel_err_vs_fp64_per_freq": [float(f"{e:.3e}") for e in err],
            "rel_residual_after_cycle": infos[-1][0]["rel_residual"]}


def run_batched(args):
    """The full batched workload (--batch problems, autotuned blocking), one JSON line."""
    import torch
    from paper_2507_23613_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    print(json.dumps(batched_solves(args, args.batch, tune=True)), flush=True)


def batched_solves(args, count, tune):
    """Independent 2D problems (sizes 257^2..2049^2, N_f 1..16) solved concurrently: one
    host thread and one stream per problem, each wave solve one CUDA-graph launch, FP32 wave
    solves with compensated filter sums; blocking depth and tile from the autotuner (tune) or
    the library defaults.  Reports the per-problem solve times (p50, p99) and the aggregate
    stencil rate; then the same solves in lockstep, one graph launch per application of the map
    across the batch.  Returns the result as a dict."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import _lib, inputs
    M._lib.load()
    prec = _lib.PREC_FP32_BLOCKSUM
    restart = 10
    chosen, seed, mem = [], args.seed + 5000, 0.0
    t_gen = time.perf_counter()
    while len(chosen) < count and seed < args.seed + 5000 + 50 * count:
        wl = inputs.batch_workload(seed)
        seed += 1
        try:
            s = M.plan(M.make_problem(wl.n, wl.length, wl.omega, n_p=wl.n_p, cfl=wl.cfl,
                                      precision=prec)[0])
        except M.MfwhError:
            continue                      # ill-conditioned filter system: draw again
        need = wl.forcing.size * (148 + 8 * (restart - 10)) / 1e9
        if mem + need > args.batch_mem_gb:
            continue
        mem += need
        chosen.append((wl, s.n_t))
    t_gen = time.perf_counter() - t_gen
    t_tune = time.perf_counter()
    tuned = [M.autotune(wl.n, wl.length, wl.omega, n_p=wl.n_p, cfl=wl.cfl, precision=prec)
             if tune else (0, 0, 0.0) for wl, _ in chosen]
    t_tune = time.perf_counter() - t_tune
    # smaller problems on higher-priority streams, so that they are not queued behind the
    # long wave solves of the large ones
    lo_pri, hi_pri = torch.cuda.Stream.priority_range()
    streams = [torch.cuda.Stream(priority=hi_pri if wl.n[0] <= 512 else lo_pri)
               for wl, _ in chosen]
    solvers, xs = [], []
    for (wl, _), (tb, shape, _), st in zip(chosen, tuned, streams):
        s = M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(),
                     stream=st.cuda_stream, n_p=wl.n_p, cfl=wl.cfl, precision=prec,
                     time_block=tb, tile_shape=shape)
        s.set_graphs(True)
        solvers.append(s)
        xs.append(torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda"))
    # warm-up: one solve of one Arnoldi step each captures the graphs
    M.solve_batch(solvers, xs, restart=1, tol=0.0, max_iters=1, raise_on_error=False)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, infos, secs = M.solve_batch(solvers, xs, restart=restart, tol=0.0,
                                    max_iters=args.batch_iters, raise_on_error=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    pts = sum((wl.n[0] - 1) * (wl.n[1] - 1) * n_t * info["pi_applications"]
              for (wl, n_t), info in zip(chosen, infos))
    # the same solves in lockstep: one graph launch per application of the map across the batch
    bstream = torch.cuda.Stream()
    for x in xs:
        x.zero_()
    M.solve_batch_graph(solvers, xs, restart=1, tol=0.0, max_iters=1, stream=bstream.cuda_stream,
                        raise_on_error=False)           # warm-up
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lst, linfos, lsecs = M.solve_batch_graph(solvers, xs, restart=restart, tol=0.0,
                                             max_iters=args.batch_iters,
                                             stream=bstream.cuda_stream, raise_on_error=False)
    torch.cuda.synchronize()
    lwall = time.perf_counter() - t0
    lpts = sum((wl.n[0] - 1) * (wl.n[1] - 1) * n_t * info["pi_applications"]
               for (wl, n_t), info in zip(chosen, linfos))
    lockstep = {"value": round(lpts / lwall / 1e9, 3), "unit": "Gpts/s (aggregate)",
                "p50_s": round(float(np.percentile(lsecs, 50)), 3),
                "p99_s": round(float(np.percentile(lsecs, 99)), 3), "wall_s": round(lwall, 3),
                "graph_launches": 1 + args.batch_iters, "status": lst,
                "per_problem_s": [round(float(x), 3) for x in lsecs],
                "note": "mfwh_solve_batch_graph: every application of the map is one CUDA-graph "
                        "launch whose branches are the problems' wave solves"}
    sizes = [wl.n[0] + 1 for wl, _ in chosen]
    line = {"metric": "batched MFWH: per-problem GMRES solve time", "impl": "native",
            "value": round(pts / wall / 1e9, 3), "unit": "Gpts/s (aggregate)",
            "p50_s": round(float(np.percentile(secs, 50)), 3),
            "p99_s": round(float(np.percentile(secs, 99)), 3),
            "max_s": round(float(np.max(secs)), 3), "wall_s": round(wall, 3),
            "n_gpus": 1, "dtype": "f32 wave steps / f64 Krylov", "data": "synthetic",
            "config": {"workload": f"batch{len(chosen)}_2d_sizes257-2049_nf1-16_omega5-80",
                       "problems": len(chosen),
                       "size_counts": {str(k + 1): sizes.count(k + 1) for k in inputs.BATCH_SIZES},
                       "nf": [wl.nf for wl, _ in chosen], "n_t": [n for _, n in chosen],
                       "solver": f"GMRES({restart}), {args.batch_iters} Arnoldi steps per problem",
                       "blocking": ("autotuned " + str([list(t[:2]) for t in tuned])) if tune
                                   else "library defaults (16 FP32 steps per launch)",
                       "device_gb": round(mem, 1)},
            "status": st, "generate_s": round(t_gen, 1), "autotune_s": round(t_tune, 1),
            "lockstep": lockstep}
    for s in solvers:
        s.close()
    return line


def run_cube(args):
    """The 3D workload: 257^3 unit cube, 7-point Laplacian, c = 1.0 / 1.5 split at z = 0.5,
    N_f = 4 frequencies in [8, 30], one GMRES(15) cycle from zero with FP64 and with FP32
    wave solves (FP64 Arnoldi); Gpts/s, HBM fraction of the step kernel, and the FP32 map's
    error against the FP64 map per frequency."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import _lib, build, inputs
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    wl = inputs.cube_layered(args.seed + 1000, n=args.cube_n)
    lay = wl.layer
    f = torch.from_numpy(wl.forcing).cuda()
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()
    out = {"metric": "stencil Gpts/s (+N_f filters), 3D", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": f"cube{wl.n[0] + 1}_nf{wl.nf}_two_layer_gmres15_cycle",
                      "grid": [k + 1 for k in wl.n], "nf": wl.nf,
                      "omega": [round(float(o), 3) for o in wl.omega],
                      "c": [lay["c_lo"], lay["c_hi"]], "interface_z": lay["interface"]}}
    x = torch.from_numpy(np.random.default_rng(3).normal(size=wl.forcing.shape) * 0.01).cuda()
    maps = {}
    legs = (("fp64", _lib.PREC_FP64, 1), ("fp32_tb1", _lib.PREC_FP32_BLOCKSUM, 1),
            ("fp32_tb2", _lib.PREC_FP32_BLOCKSUM, 2), ("fp32_tb4", _lib.PREC_FP32_BLOCKSUM, 4))
    for name, prec, tb in legs:
        s = M.Solver(wl.n, wl.length, wl.omega, f, stream=stream.cuda_stream, n_p=wl.n_p,
                     cfl=wl.cfl, c_lo=lay["c_lo"], c_hi=lay["c_hi"], interface=lay["interface"],
                     layer_axis=lay["axis"], precision=prec, time_block=tb)
        n_t = s.setup["n_t"]
        v = torch.zeros_like(f)
        s.solve_gmres(v, restart=15, tol=0.0, max_iters=1, raise_on_error=False)   # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            v.zero_()
        torch.cuda.synchronize()
        ev0.record(stream)
        info = s.solve_gmres(v, restart=15, tol=0.0, max_iters=15, raise_on_error=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        step_ms, step_launches, _ = s.last_timing()
        apps = info["pi_applications"]
        interior = (wl.n[0] - 1) * (wl.n[1] - 1) * (wl.n[2] - 1)
        w = 8 if name == "fp64" else 4
        # per launch and interior point: read W^n, the previous level or D, the filter state;
        # write them (FP32: W, D and the Kahan pairs, once per launch of `tb` steps)
        per_pt = (3 + 2 * wl.nf) * w if name == "fp64" else (4 + 4 * wl.nf) * 4
        gbs = interior * per_pt * step_launches / (step_ms * 1e-3) / 1e9
        kern = ("k_step<NF,3>" if name == "fp64" else
                ("k_step32<NF,3>" if tb == 1 else f"k_tb3d32<NF,{2 if tb <= 2 else 4}>"))
        out[name] = {"value": round(interior * n_t * apps / (ms * 1e-3) / 1e9, 3),
                     "unit": "Gpts/s", "ms_per_cycle": round(ms, 1), "n_t": n_t,
                     "time_block": tb,
                     "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                                  "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                                  "peak_source": peak_kind, "kernel": kern,
                                  "avg_launch_us": round(step_ms * 1e3 / max(step_launches, 1),
                                                         2)}}
        o = torch.empty_like(x)
        with torch.cuda.stream(stream):
            s.apply_Pi(x, o, forced=True)
        torch.cuda.synchronize()
        maps[name] = o.cpu().numpy().reshape(wl.nf, -1)
        s.close()
    for name in ("fp32_tb1", "fp32_tb2", "fp32_tb4"):
        a, b = maps[name], maps["fp64"]
        out[name]["pi_rel_err_vs_fp64_per_freq"] = [
            float(f"{e:.3e}") for e in np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)]
    best = max(("fp32_tb1", "fp32_tb2", "fp32_tb4"), key=lambda k: out[k]["value"])
    out["fp32"] = dict(out[best], leg=best)
    print(json.dumps(out), flush=True)


def implicit_bytes_per_point(nf, forced, cycles_per_solve, dim=2):
    """Algorithmic bytes per interior point of one implicit step (FP64): the V-cycles at the
    finest level (2 red-black sweeps before and 1 after the coarse correction, each reading u
    and f and writing u; the residual pass reading u, f and writing r; full weighting reading
    r and writing the coarse f and u; prolongation reading the coarse u and updating u),
    scaled by the coarser levels' share (1/(1 - 2^-dim)), the converged pre-smoothing and
    residual test, and the update of W, q and the next right-hand side."""
    w = 8
    fine = 3 * 3 * w + 3 * w + (w + 2 * w / 2 ** dim) + (2 * w + w / 2 ** dim)
    cyc = fine / (1.0 - 2.0 ** -dim)
    check = 2 * 3 * w + 3 * w
    update = 4 * w + (3 if forced else 2) * nf * w
    return cycles_per_solve * cyc + check + update


def run_implicit(args):
    """Implicit trapezoidal time stepping (10 steps per shortest period, multigrid step solves
    to 1e-10) on the 1025^2, N_f = 8, N_p = 2 workload: one GMRES(20) cycle from zero, timed
    beside the explicit FP64 cycle of the same problem; ms per wave solve, multigrid cycles
    per step, and the step kernel's achieved bandwidth on the algorithmic byte model."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import build, inputs
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    layer = {}
    restart = RESTART
    if args.cube:
        # the 3D workload instead: 257^3, two layers, N_f = 4, GMRES(15)
        wl = inputs.cube_layered(args.seed + 1000)
        lay = wl.layer
        layer = dict(c_lo=lay["c_lo"], c_hi=lay["c_hi"], interface=lay["interface"],
                     layer_axis=lay["axis"])
        restart = 15
    else:
        wl = inputs.square_large(args.seed)
    dim = len(wl.n)
    f = torch.from_numpy(wl.forcing).cuda()
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()
    res = {}
    for name, kw in (("implicit", dict(time_stepping="implicit")), ("explicit", {})):
        s = M.Solver(wl.n, wl.length, wl.omega, f, stream=stream.cuda_stream, n_p=wl.n_p,
                     cfl=wl.cfl, **kw, **layer)
        n_t = s.setup["n_t"]
        v = torch.zeros_like(f)
        for _ in range(max(1, args.warmup)):
            s.solve_gmres(v, restart=restart, tol=0.0, max_iters=restart, raise_on_error=False)
        if name == "implicit":
            s.mg_stats(reset=True)
        ms_tot, step_ms, step_l, launches, apps = 0.0, 0.0, 0, 0, 0
        for _ in range(max(1, args.steps)):
            with torch.cuda.stream(stream):
                v.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            info = s.solve_gmres(v, restart=restart, tol=0.0, max_iters=restart,
                                 raise_on_error=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_tot += ev0.elapsed_time(ev1)
            a, b, c = s.last_timing()
            step_ms += a
            step_l += b
            launches += c
            apps += info["pi_applications"]
        k = max(1, args.steps)
        r = {"n_t": n_t, "dt": s.setup["dt"], "ms_per_cycle": round(ms_tot / k, 2),
             "ms_per_wave_solve": round(step_ms / apps, 3),
             "pi_applications_per_cycle": apps / k,
             "rel_residual_after_cycle": info["rel_residual"],
             "gpu_launches_per_cycle": launches / k}
        if name == "implicit":
            st = s.mg_stats()
            cps = st["cycles"] / max(st["solves"], 1)
            r.update({"mg_levels": st["levels"], "mg_cycles_per_step": round(cps, 3),
                      "mg_unconverged_steps": st["unconverged"]})
            interior = wl.interior_points
            # one forced map per cycle, the rest homogeneous
            per_app = [implicit_bytes_per_point(wl.nf, i == 0, cps, dim) for i in range(apps // k)]
            alg = interior * n_t * sum(per_app) * k
            gbs = alg / (step_ms * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                             "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                             "peak_source": peak_kind, "kernel": f"k_imp_step<{dim}>",
                             "alg_bytes_per_launch": round(alg / step_l),
                             "avg_launch_us": round(step_ms * 1e3 / step_l, 2),
                             "note": "2D: finest-level multigrid arrays are L2-resident"}
        if args.solve:
            # time to solution: unrestarted GMRES to 1e-8 (the paper's solver), and FP64
            # defect correction to max_m r_h <= 1e-6 (inner GMRES to 1e-6 relative)
            for key, fn in (("gmres_1e-8", lambda vv: s.solve_gmres(
                                vv, restart=SOLVE_MAX_ITERS, tol=TOL, max_iters=SOLVE_MAX_ITERS,
                                raise_on_error=False)),
                            ("refined_rh_1e-6", lambda vv: s.solve_refined(
                                vv, target=1e-6, inner_tol=1e-6, restart=1000, max_iters=3000,
                                raise_on_error=False))):
                with torch.cuda.stream(stream):
                    v.zero_()
                if name == "implicit":
                    s.mg_stats(reset=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = fn(v)
                torch.cuda.synchronize()
                r[key] = {"seconds": round(time.perf_counter() - t0, 2),
                          "status": int(info["status"]), "arnoldi_steps": info["iterations"],
                          "pi_applications": info["pi_applications"],
                          "rel_residual": info["rel_residual"],
                          "max_helmholtz_residual": float(np.max(info["helmholtz_residual"]))}
                if name == "implicit":
                    st = s.mg_stats()
                    r[key]["mg_cycles_per_step"] = round(st["cycles"] / max(st["solves"], 1), 3)
        res[name] = r
        s.close()
    out = {"metric": "implicit vs explicit FP64 MFWH wave solve", "unit": "ms",
           "value": res["implicit"]["ms_per_wave_solve"], "higher_is_better": False,
           "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{wl.name}_implicit_gmres{restart}_cycle",
                      "grid": [k_ + 1 for k_ in wl.n], "nf": wl.nf, "n_p": wl.n_p,
                      "steps_per_period": 10, "mg_tol": 1e-10},
           "implicit": res["implicit"], "explicit": res["explicit"],
           "speedup_per_wave_solve": round(res["explicit"]["ms_per_wave_solve"]
                                           / res["implicit"]["ms_per_wave_solve"], 3)}
    print(json.dumps(out), flush=True)


# The paper's multigrid scaling table (Figure squareGridCpuScaling: square, order 4, implicit
# time stepping, the three-frequency problem of eq. Nf3parameters, Ogmg to 1e-10 on a CPU):
# grid spacing -> (wave solves, multigrid cycles per solve, CPU seconds).
PAPER_MG_TABLE = {64: (22, 7.1, 5.6), 128: (22, 7.0, 14.3), 256: (22, 7.0, 49.9),
                  512: (20, 6.7, 169.8), 1024: (20, 6.7, 690.9), 2048: (20, 6.7, 2862.0)}


def run_implicit_scaling(args):
    """O(N) check of implicit MFWH with multigrid on GB300: the three-frequency problem of
    eq. Nf3parameters on the unit square, fourth-order operator, implicit trapezoidal steps
    (10 per shortest period, multigrid to 1e-10), unrestarted GMRES to 1e-10, from 129^2 to
    2049^2 (65^2 is below the library's minimum grid for fourth-order implicit stepping).
    With --cube, the same on its 3D analogue from 33^3 to 129^3."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import build, inputs
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    rows = []
    cube = args.cube
    for n in ((32, 64, 128) if cube else (128, 256, 512, 1024, 2048)):
        wl = inputs.paper_three_frequency_cube(n) if cube else inputs.paper_three_frequency(n)
        f = torch.from_numpy(wl.forcing).cuda()
        s = M.Solver(wl.n, wl.length, wl.omega, f, n_p=wl.n_p, order=4, time_stepping="implicit")
        v = torch.zeros_like(f)
        s.solve_gmres(v, restart=5, tol=0.0, max_iters=5, raise_on_error=False)   # warm-up
        v.zero_()
        s.mg_stats(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = s.solve_gmres(v, restart=300, tol=1e-10, max_iters=300, raise_on_error=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        st = s.mg_stats()
        pts = (n + 1) ** len(wl.n)
        paper = None if cube else PAPER_MG_TABLE[n]
        rows.append({"grid": [n + 1] * len(wl.n), "points": pts, "n_t": s.setup["n_t"],
                     "wave_solves": info["pi_applications"], "gmres_status": int(info["status"]),
                     "rel_residual": info["rel_residual"],
                     "max_helmholtz_residual": float(np.max(info["helmholtz_residual"])),
                     "mg_cycles_per_step": round(st["cycles"] / max(st["solves"], 1), 2),
                     "mg_unconverged_steps": st["unconverged"], "seconds": round(sec, 3),
                     "us_per_point": round(sec / pts * 1e6, 3)})
        if paper:
            rows[-1]["paper_cpu"] = {"wave_solves": paper[0], "mg_cycles": paper[1],
                                     "seconds": paper[2]}
        s.close()
    out = {"metric": "implicit MFWH time to 1e-10 vs grid (O(N) scaling)", "unit": "s",
           "value": rows[-1]["seconds"], "higher_is_better": False, "n_gpus": 1, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": ("paper3freq_cube_order4_implicit" if cube
                                   else "paper3freq_square_order4_implicit"),
                                          "omega": [5.1, 10.1, 15.1], "n_p": 2, "order": 4,
                                          "steps_per_period": 10, "mg_tol": 1e-10,
                                          "gmres_tol": 1e-10},
           "rows": rows,
           "paper_context": ("none: the paper's scaling study is 2D" if cube else
                             "Figure squareGridCpuScaling: CPU (Ogmg) seconds on the paper's "
                             "machine; a different machine and solver, quoted as context")}
    print(json.dumps(out), flush=True)


def conv_flops(layers, channels, in_channels, pixels):
    """Tensor-core FLOPs of one forward pass of the warm-start network: 2 x pixels x 9 taps x
    Cin x Cout per 3 x 3 layer (in_channels -> channels, channels -> channels, ..., -> 1)."""
    chans = [in_channels] + [channels] * (layers - 1) + [1]
    return 2 * 9 * pixels * sum(a * b for a, b in zip(chans[:-1], chans[1:]))


def run_cnn(args):
    """The warm-start network's kernels on a synthetic batch (129^2 images, the warm-start
    workload's grid, 2 input channels, 5 layers of 32 channels): forward passes (implicit-GEMM
    convolutions on tcgen05) and training steps (forward, input and weight gradients, Adam)."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    B, H = args.cnn_batch, args.ws_n + 1
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    x = torch.randn((B, 2, H, H), generator=g, device="cuda", dtype=torch.float32)
    t = torch.randn((B, 1, H, H), generator=g, device="cuda", dtype=torch.float32)
    mask = torch.ones((B, 1, H, H), device="cuda", dtype=torch.float32)
    y = torch.empty((B, 1, H, H), device="cuda", dtype=torch.float32)
    net = M.CNN(layers=5, channels=32, in_channels=2, seed=args.seed)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        net.forward(x, y)
        net.train_step(x, t, mask, 1e-4)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for _ in range(args.steps):
        net.forward(x, y)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(args.steps):
        net.train_step(x, t, mask, 1e-4)
    ev[3].record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1]) / args.steps
    train_ms = ev[2].elapsed_time(ev[3]) / args.steps
    flops = conv_flops(5, 32, 2, B * H * H)
    peak = 1973.9
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peak = float(json.load(fh).get("bf16_tflops", peak))
    tf = flops / (fwd_ms * 1e-3) / 1e12
    net.close()
    print(json.dumps({
        "metric": "warm-start network forward TFLOP/s (BF16 tensor cores)", "value": round(tf, 2),
        "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "cnn5x32_batch%d_%dx%d" % (B, H, H), "layers": 5, "channels": 32},
        "forward_ms": round(fwd_ms, 3), "train_step_ms": round(train_ms, 3),
        "roofline": {"bound": "tensor", "achieved": round(tf, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(tf / peak, 4),
                     "flops_per_forward": flops,
                     "note": "K = 9 Cin <= 288 and N = Cout <= 32 per implicit GEMM: far too "
                             "little reuse per operand byte for the tensor peak"}}), flush=True)


def run_warm_start(args):
    """Learned warm start: MFWH-converged FP64 solutions of seeded problems train the network
    (inputs f_m / max|f_m| and omega_m / 45, target the shape V_m / max|V_m|, amplitude fitted to
    the Helmholtz residual at prediction time); held-out problems are then solved by GMRES to
    1e-6 from zero and from the network's prediction."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import _lib, build, inputs
    torch.cuda.set_device(0)
    build.build()
    M._lib.load()
    restart, omega_scale, group = 800, 45.0, 48
    n = args.ws_n
    H = W = n + 1
    # training data from batched FP64 solves
    xs, ts, gen_t0, seed, solved, iters = [], [], time.perf_counter(), args.seed + 9000, 0, []
    while solved < args.ws_train and time.perf_counter() - gen_t0 < args.ws_gen_seconds:
        wls = []
        while len(wls) < min(group, args.ws_train - solved):
            wl = inputs.warm_start_workload(seed, n=n)
            seed += 1
            try:
                M.plan(M.make_problem(wl.n, wl.length, wl.omega, n_p=wl.n_p, cfl=wl.cfl)[0])
            except M.MfwhError:
                continue
            wls.append(wl)
        streams = [torch.cuda.Stream() for _ in wls]
        sol = [M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(),
                        stream=st.cuda_stream, n_p=wl.n_p, cfl=wl.cfl) for wl, st in zip(wls, streams)]
        for s in sol:
            s.set_graphs(True)
        vs = [torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda") for wl in wls]
        torch.cuda.synchronize()
        _, infos, _ = M.solve_batch(sol, vs, restart=restart, tol=1e-8, max_iters=restart,
                                    raise_on_error=False)
        for s, v, info in zip(sol, vs, infos):
            if info["rel_residual"] < 1e-7:
                x = torch.empty((s.nf, 2, H, W), dtype=torch.float32, device="cuda")
                t = torch.empty((s.nf, 1, H, W), dtype=torch.float32, device="cuda")
                s.warm_start_data(v, x, t, omega_scale)
                xs.append(x)
                ts.append(t)
                iters.append(info["iterations"])
            s.close()
        solved += len(wls)
    gen_s = time.perf_counter() - gen_t0
    X = torch.cat(xs)
    T = torch.cat(ts)
    mask = torch.ones((H, W), dtype=torch.float32, device="cuda")
    mask[0, :] = mask[-1, :] = 0
    mask[:, 0] = mask[:, -1] = 0
    # training
    net = M.CNN(layers=5, channels=32, in_channels=2, seed=args.seed)
    S, bs = X.shape[0], 32
    gen = torch.Generator().manual_seed(args.seed)
    tr_t0 = time.perf_counter()
    losses = []
    for ep in range(args.ws_epochs):
        lr = 1e-3 if ep < 0.7 * args.ws_epochs else 2e-4
        perm = torch.randperm(S, generator=gen).cuda()
        ep_loss = []
        for i in range(0, S - bs + 1, bs):
            idx = perm[i:i + bs]
            ep_loss.append(net.train_step(X[idx].contiguous(), T[idx].contiguous(), mask, lr))
        losses.append(float(np.mean(ep_loss)))
    train_s = time.perf_counter() - tr_t0
    # held-out comparison
    rows = []
    for k in range(args.ws_test):
        wl = inputs.warm_start_workload(args.seed + 50000 + k, n=n)
        try:
            s = M.Solver(wl.n, wl.length, wl.omega, torch.from_numpy(wl.forcing).cuda(),
                         n_p=wl.n_p, cfl=wl.cfl)
        except M.MfwhError:
            continue
        res = {}
        for mode in ("zero", "cnn"):
            v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kept, ratio0 = (False, 1.0)
            if mode == "cnn":
                kept, ratio0 = s.warm_start(net, v, omega_scale)
            info = s.solve_gmres(v, restart=restart, tol=1e-6, max_iters=restart,
                                 raise_on_error=False)
            res[mode] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                         "kept": kept, "start_residual_ratio": float(ratio0),
                         "rel_residual": info["rel_residual"]}
        rows.append(res)
        s.close()
    med = lambda key, mode: float(np.median([r[mode][key] for r in rows]))
    line = {"metric": "learned warm start: GMRES iterations and time to 1e-6, CNN start vs zero",
            "impl": "native", "unit": "iterations",
            "value": med("iterations", "cnn"), "zero_start_iterations": med("iterations", "zero"),
            "cnn_seconds_median": round(med("seconds", "cnn"), 4),
            "zero_seconds_median": round(med("seconds", "zero"), 4),
            "kept_fraction": float(np.mean([r["cnn"]["kept"] for r in rows])),
            "cnn_start_residual_ratio_median": med("start_residual_ratio", "cnn"),
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": "bf16 network (fp32 accumulate), f64 MFWH",
            "config": {"workload": f"warm_start_square{H}_nf6_omega15-45_np2",
                       "network": "5 layers, 3x3, 32 channels, inputs (f/max|f|, omega/45)",
                       "training_samples": int(S), "training_problems": solved,
                       "training_solve_iterations_median": float(np.median(iters)),
                       "epochs": args.ws_epochs, "batch": bs,
                       "loss_first_last_epoch": [losses[0], losses[-1]],
                       "generate_s": round(gen_s, 1), "train_s": round(train_s, 1),
                       "test_problems": len(rows)},
            "per_problem": [{m: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                 for kk, vv in r[m].items()} for m in r} for r in rows]}
    print(json.dumps(line), flush=True)
    net.close()


TTS_TARGET = 1e-6          # max_m r_h of the time-to-solution arms
TTS_RESTART = 800          # no restart within the step budget
TTS_MAX_ITERS = 1000       # Arnoldi steps per arm at most


def time_to_solution(args, wl, f_dev, stream, solver):
    """Wall time to max_m r_h <= 1e-6 (eq. errorAndResid) on the bench workload from zero, for
    two arms on the same GPU: FP64 (refinement with FP64 products: an FP64 GMRES solve,
    repeated on the FP64 residual until r_h meets the target) and mixed precision (the same
    refinement whose inner solves switch to FP32 wave solves once their residual is below
    --tts-relax: relaxed inexact Krylov products).  Each arm: seconds, Arnoldi steps,
    refinements, final max r_h, and whether the target was reached."""
    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import _lib
    out = {"target_max_rh": TTS_TARGET, "start": "zero", "inner_tol": args.tts_inner,
           "restart": TTS_RESTART, "max_iters": TTS_MAX_ITERS}
    s32 = M.Solver(wl.n, wl.length, wl.omega, f_dev, stream=stream.cuda_stream, n_p=wl.n_p,
                   cfl=wl.cfl, precision=_lib.PREC_FP32_BLOCKSUM)
    for name, call in (
            ("fp64", lambda v: solver.solve_refined(
                v, target=TTS_TARGET, inner_tol=args.tts_inner, restart=TTS_RESTART,
                max_iters=TTS_MAX_ITERS, max_refinements=8, raise_on_error=False)),
            ("mixed_relaxed_fp32", lambda v: s32.solve_relaxed(
                v, target=TTS_TARGET, inner_tol=args.tts_inner, relax_below=args.tts_relax,
                restart=TTS_RESTART, max_iters=TTS_MAX_ITERS, max_refinements=8,
                raise_on_error=False))):
        v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = call(v)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        rh = float(np.max(info["helmholtz_residual"]))
        out[name] = {"seconds": round(secs, 2), "arnoldi_steps": info["iterations"],
                     "refinements": info["refinements"], "max_helmholtz_residual": rh,
                     "reached": bool(info["status"] == _lib.OK and rh <= TTS_TARGET)}
        del v
        torch.cuda.empty_cache()
    out["mixed_relaxed_fp32"]["relax_below"] = args.tts_relax
    s32.close()
    return out


def workload_config(wl, n_t):
    return {"workload": f"square{wl.n[0] + 1}x{wl.n[1] + 1}_nf{wl.nf}_np{wl.n_p}_gmres{RESTART}_cycle",
            "step": "one GMRES(20) cycle from zero: b = Pi(0), 20 Arnoldi steps, update, residual check",
            "grid": [wl.n[0] + 1, wl.n[1] + 1], "nf": wl.nf, "n_p": wl.n_p, "n_t": n_t,
            "omega_band": [10.0, 60.0], "gaussian_b": 400.0, "cfl": wl.cfl,
            "restart": RESTART, "tol": TOL,
            "precision": "fp64 wave levels, steps and filter solve; filter sums as float pairs",
            "l2": "working set (forcing, accumulators, Krylov basis: > 1 GB) is larger than L2"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.batched:
        return run_batched(args) if rank == 0 else None
    if args.implicit:
        return run_implicit(args) if rank == 0 else None
    if args.small:
        return run_small(args) if rank == 0 else None
    if args.implicit_scaling:
        return run_implicit_scaling(args) if rank == 0 else None
    if args.cube:
        return run_cube(args) if rank == 0 else None
    if args.warm_start:
        return run_warm_start(args) if rank == 0 else None
    if args.cnn:
        return run_cnn(args) if rank == 0 else None

    import torch
    import paper_2507_23613_gb300 as M
    from paper_2507_23613_gb300 import build, inputs

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    M._lib.load()

    from paper_2507_23613_gb300 import multi
    wl = inputs.square_large(multi.problem_seed(args.seed, rank))
    stream = torch.cuda.Stream()
    f_dev = torch.from_numpy(wl.forcing).cuda()
    if args.fp32_only:
        from paper_2507_23613_gb300 import _lib
        n_t32 = M.plan(M.make_problem(wl.n, wl.length, wl.omega, n_p=wl.n_p, cfl=wl.cfl)[0]).n_t
        print(json.dumps({"fp32": fp32_leg(args, wl, f_dev, stream, n_t32)}), flush=True)
        return
    solver = M.Solver(wl.n, wl.length, wl.omega, f_dev, stream=stream.cuda_stream,
                      n_p=wl.n_p, cfl=wl.cfl, time_block=args.time_block,
                      tile_shape=args.tile_shape)
    n_t = solver.setup["n_t"]
    N = wl.forcing.size
    v = torch.zeros(wl.forcing.shape, dtype=torch.float64, device="cuda")

    def one_step():
        with torch.cuda.stream(stream):
            v.zero_()
        info = solver.solve_gmres(v, restart=RESTART, tol=TOL, max_iters=MAX_ITERS,
                                  raise_on_error=False)
        if info["status"] not in (M._lib.OK, M._lib.ERR_NOT_CONVERGED):
            raise M.MfwhError(info["status"], "GMRES cycle failed")
        ms, step_launches, launches = solver.last_timing()
        return info, ms, step_launches, launches + 1

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(one_step())
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()

    pi_apps = sum(i[0]["pi_applications"] for i in infos)
    forced_apps = sum(1 for _ in infos)          # one forced map (b) per solve
    homog_apps = pi_apps - forced_apps
    pts_steps = wl.interior_points * n_t * pi_apps
    step_ms_total = sum(i[1] for i in infos)
    step_launches = sum(i[2] for i in infos)
    launches = sum(i[3] for i in infos)
    alg_bytes = wl.interior_points * n_t * (forced_apps * bytes_per_point_step(wl.nf, True)
                                           + homog_apps * bytes_per_point_step(wl.nf, False))
    alg_flops = wl.interior_points * n_t * (forced_apps * flops_per_point_step(wl.nf, True)
                                           + homog_apps * flops_per_point_step(wl.nf, False))
    achieved_gbs = alg_bytes / (step_ms_total * 1e-3) / 1e9
    achieved_tf = alg_flops / (step_ms_total * 1e-3) / 1e12
    hbm_peak, peak_kind = peaks()

    # whole-job numbers: max time over ranks, points summed over ranks
    value, t_max, total_pts = multi.weak_scaling_rate(elapsed_ms, pts_steps, dist, "cuda")

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        f_host = torch.from_numpy(wl.forcing).pin_memory()
        v_host = torch.zeros(wl.forcing.shape, dtype=torch.float64).pin_memory()
        e2e_steps = max(1, args.steps)
        e_pts = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            v_host.zero_()
            solver.set_forcing(f_host)
            info = solver.solve_gmres(v_host.numpy(), restart=RESTART, tol=TOL, max_iters=MAX_ITERS,
                                      raise_on_error=False)
            e_pts += wl.interior_points * n_t * info["pi_applications"]
        e_s = time.perf_counter() - t0
        e2e = {"value": e_pts / e_s / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": 2 * N * WORD, "d2h_bytes_per_step": N * WORD,
               "note": "forcing and initial guess copied from pinned host memory, solution read back, every step"}

    tts = None if args.no_tts else time_to_solution(args, wl, f_dev, stream, solver)
    solve = None
    if args.solve:
        with torch.cuda.stream(stream):
            v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = solver.solve_gmres(v, restart=SOLVE_MAX_ITERS, tol=TOL, max_iters=SOLVE_MAX_ITERS,
                                  raise_on_error=False)
        solve = {"seconds": round(time.perf_counter() - t0, 3), "tol": TOL, "restart": "none",
                 "converged": info["status"] == M._lib.OK, "iterations": info["iterations"],
                 "rel_residual": info["rel_residual"],
                 "max_helmholtz_residual": float(np.max(info["helmholtz_residual"]))}

    fp32 = None if args.no_fp32 else fp32_leg(args, wl, f_dev, stream, n_t)
    batched = None
    if not args.no_batched and rank == 0:
        batched = batched_solves(args, args.default_batch, tune=False)

    if rank != 0:
        return
    # Steps per launch, from the library's own launch count (ceil(N_t / depth) per map).
    launches_per_map = step_launches / max(pi_apps, 1)
    depth = max(1, int(round(n_t / launches_per_map)))
    t_hbm = alg_bytes / (hbm_peak * 1e9)
    t_alu = alg_flops / (FP64_PEAK_TFLOPS * 1e12)
    unblocked = {"unit": "GB/s", "achieved": round(achieved_gbs, 1),
                 "frac": round(achieved_gbs / hbm_peak, 4),
                 "bytes_per_point_step": [bytes_per_point_step(wl.nf, False),
                                          bytes_per_point_step(wl.nf, True)]}
    if depth == 1:
        traffic = kernel_traffic("k_step_square1025_nf8.txt", kernel_source_key())
        kernel = "k_step/k_last (leapfrog + N_f filters, one step per launch)"
        if t_hbm >= t_alu:
            roof = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(achieved_gbs / hbm_peak, 4)}
        else:
            roof = {"bound": "alu", "achieved": round(achieved_tf, 4), "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4)}
        roof["alg_bytes_per_launch"] = round(alg_bytes / max(step_launches, 1))
    else:
        # Blocked launches move (4 + 2 N_f (+ N_f forced)) words per point whatever their depth;
        # the bound is the FP64 pipe (5 FP64 instructions per homogeneous point-step).
        blk_bytes = wl.interior_points * (
            forced_apps * -(-n_t // depth) * blocked_bytes_per_point_launch(wl.nf, True)
            + homog_apps * -(-n_t // depth) * blocked_bytes_per_point_launch(wl.nf, False))
        blk_gbs = blk_bytes / (step_ms_total * 1e-3) / 1e9
        shape = args.tile_shape if args.time_block else 5
        pipe = depth <= 4 and shape == 5 and wl.nf <= 8
        traffic = (kernel_traffic("k_tb2d_pipe_square1025_nf8.txt", blocked_kernel_source_key())
                   if pipe else None)
        kernel = ("k_tb2d_pipe (%d leapfrog steps + N_f filters per pass, persistent CTAs "
                  "copying the next tile while stepping one)" % depth if pipe else
                  "k_tb2d (%d leapfrog steps + N_f filters per launch)" % depth)
        roof = {"bound": "alu", "achieved": round(achieved_tf, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4),
                "alg_bytes_per_launch": round(blk_bytes / max(step_launches, 1)),
                "blocked_hbm": {"unit": "GB/s", "achieved": round(blk_gbs, 1),
                                "frac": round(blk_gbs / hbm_peak, 4)},
                "unblocked_byte_model": unblocked,
                "steps_per_launch": depth}
    roof.update({"traffic": traffic, "kernel": kernel, "peak_source": peak_kind,
                 "peak_note": ("alu peak derived from unit counts: 152 SMs x 2 FP64 FMA lanes x "
                               "2 flops x 2.07 GHz; hbm peak " + peak_kind),
                 "avg_launch_us": round(step_ms_total * 1e3 / max(step_launches, 1), 2),
                 "hbm_frac": round(achieved_gbs / hbm_peak, 4),
                 "fp64_alu_frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4)})
    line = {
        "metric": "stencil Gpts/s (+N_f filters)", "value": round(value, 3), "unit": "Gpts/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, n_t),
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "e2e": e2e,
        "cycle": {"pi_applications_per_step": pi_apps / args.steps,
                  "gmres_iterations_per_step": sum(i[0]["iterations"] for i in infos) / args.steps,
                  "rel_residual_after_cycle": infos[-1][0]["rel_residual"],
                  "max_helmholtz_residual": float(np.max(infos[-1][0]["helmholtz_residual"]))},
        "time_to_solution": tts,
        "unrestarted_solve_1e-8": solve,
        "fp32": fp32,
        "batched": batched,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(("square_large", {"seed": multi.problem_seed(
            args.seed, rank)}), budget_s=8.0)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
