"""Benchmark of one full hybrid LB/FD step (FD update + flame sensor + thermodynamic pressure +
LB stream/collide) on the reactive swirl-burner workload (384 x 192 x 192 cells, D3Q27,
6 species, 2-step chemistry, thickened flame with sensor, closed-domain thermodynamic pressure).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Metric: million lattice-cell updates per second of the full
step (MLUPS), FP32 populations and arithmetic; the same step with FP16 shifted population
storage is reported beside it. N > 1 runs independent replicas (one per GPU, weak scaling).
The state (~4.3 GB FP32) is larger than L2, so no flush is needed between steps.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c4_swirl_reactive_3d"
METRIC = "MLUPS per full hybrid step (LB + FD + chemistry + P_th), % of HBM roofline"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_time_ms(ms, world):
    """Max over ranks of a rank's timed-region duration (ms): the whole-job time of the
    replicas. Uses the initialised process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def model_bytes(wl, kernel, storage):
    """Algorithmic bytes per fluid cell of one launch: every array the kernel must touch, once.
    LB stream-collide: populations read and written (2 Q S), velocity written (d F), rho and
    Lambda read (2 F), the mask (1). FD update: T and Y_k read and written (2 (1 + K) F), velocity
    read (d F), the mask (1), rho and Lambda written (2 F). F = 8 bytes for FP64 fields, else 4;
    S = 8, 4 or 2 for FP64, FP32 or FP16 populations."""
    d = wl.cfg["dim"]
    Q = 27 if d == 3 else 9
    F = 8 if storage == "f64" else 4
    S = {"f64": 8, "f32": 4, "f16": 2}[storage]
    thermal = bool(wl.cfg.get("thermal"))
    K = len(wl.cfg.get("species", [])) if thermal else 0
    if kernel == "lb_stream_collide":
        return 2 * Q * S + d * F + (2 * F if thermal else 0) + 1
    if kernel == "fd_update":
        return 2 * (1 + K) * F + d * F + 1 + 2 * F
    return None


def job_value(cells, steps, world, ms):
    """Whole-job throughput in MLUPS: every rank advances its own copy of the workload."""
    return cells * steps * world / (ms * 1e-3) / 1e6


def _timed_steps(solver, steps, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver.synchronize()
    e0.record(solver.stream)
    solver.step(steps)
    e1.record(solver.stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_variant(wl, storage, steps, warmup, torch, profile_steps, stats=0, probes=0):
    from paper_2207_11567_gb300 import from_workload
    wl.cfg["storage"] = storage
    s = from_workload(wl)
    if stats:
        s.stats_control(1, stats)
    if probes:
        import numpy as np
        fluid = np.nonzero(np.asarray(wl.mask).reshape(-1) == 0)[0]
        s.set_probes(fluid[np.linspace(0, fluid.size - 1, probes).astype(np.int64)], capacity=steps + warmup + 16)
    s.step(warmup)
    s.synchronize()
    ms = _timed_steps(s, steps, torch)
    # per-kernel CUDA-event timing on the library's stream (direct launches)
    s.profile(True)
    s.step(profile_steps)
    kt = s.kernel_times()
    s.profile(False)
    kb = s.kernel_bytes()
    out = {"ms": ms, "kernels": {k: {"ms_avg": (t / n if n else 0.0), "launches": n, "bytes": kb[k]}
                                 for k, (t, n) in kt.items()}}
    s.close()
    return out


def e2e_run(wl, steps, torch):
    """User call sequence through the C ABI with host buffers in pinned memory: initial fields
    uploaded from the host, K steps, fields read back into host memory; all inside the timed
    region. Returns (seconds, host-to-device bytes, device-to-host bytes)."""
    import numpy as np
    from paper_2207_11567_gb300 import Solver
    from paper_2207_11567_gb300 import _lib as L
    wl.cfg["storage"] = "f32"

    def pinned(a):
        if a is None:
            return None
        t = torch.empty(np.asarray(a).size, dtype=torch.float64, pin_memory=True)
        v = t.numpy()
        v[:] = np.asarray(a, dtype=np.float64).reshape(-1)
        return v

    T, Y, u, P = pinned(wl.T), pinned(wl.Y), pinned(wl.u), pinned(wl.P_h)
    s = Solver(wl.cfg, wl.mask, wl.inlet_u)
    bits = L.F_T | L.F_Y | L.F_U | L.F_PH
    if not wl.cfg.get("thermal"):
        bits &= ~(L.F_T | L.F_Y)
    out = torch.empty(L.lib.lbm_fields_size(s.ctx, bits), dtype=torch.float64, pin_memory=True).numpy()
    s.synchronize()
    t0 = time.perf_counter()
    s.set_fields(T=T, Y=Y, u=u, P_h=P)
    s.step(steps)
    s.fields(bits, out=out)
    t1 = time.perf_counter()
    h2d = 8 * sum(a.size for a in (T, Y, u, P) if a is not None)
    d2h = 8 * out.size
    s.close()
    return t1 - t0, h2d, d2h


def oracle_sample(max_seconds=20.0):
    """The FP64 CPU oracle as it stands on a bounded sample of the same workload: a reduced
    reactive swirl domain (48 x 24 x 24 cells, same physics and parameters), timed per step."""
    import torch
    import workloads as W
    from oracle.step import Oracle
    wl = W.generate.swirl_3d(48, 24, 24, reactive=True, seed=0)
    o = Oracle(wl.cfg, wl.mask, wl.inlet_u)
    st = o.init_state(T=wl.T, Y=wl.Y, u=wl.u, P_h=wl.P_h)
    st = o.step(st)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < max_seconds:
        st = o.step(st)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": wl.N * n / dt / 1e6, "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, reactive swirl {wl.cfg['nx']}x{wl.cfg['ny']}x{wl.cfg['nz']} "
                      f"({wl.N} cells) cut from the same workload family, {n} steps in {dt:.1f} s"}


def adjoint_bench(args):
    """Gradient of the fuel consumption after K = 2000 steps of the 512 x 128 chamber (inlet
    profile of 128 values and initial temperature field), checkpoints every 100 steps: forward
    and backward wall time with device synchronisation (FP32), their ratio, and an FP64 check of
    the gradient against central differences along 16 seeded directions (numpy Philox) at
    h = 1e-4 and h = 1e-6, with the FP32 gradient's distance to the FP64 one.

    The problem starts from the chamber's fields (T, Y, u, P_h) --adj-spinup steps after its
    ignition state (FP64 run, nominal inlet; 0 starts at the ignition state itself), restarted
    with equilibrium populations: in the first ~200 steps after ignition the fuel diffuses into
    the hot kernel at tiny mass fractions, where the order-0.5 rate law has slopes ~Y^-1/2 and
    the exact derivative of the discrete map reaches 1e33."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2207_11567_gb300 import AdjointProblem, Solver
    from paper_2207_11567_gb300 import _lib as L
    torch.cuda.set_device(0)
    wl = W.make("c5_adjoint_2d")
    K, C = (args.adj_steps or wl.steps), 100
    inlet0 = np.asarray(wl.inlet_u, dtype=np.float64).reshape(2, -1)
    T0, Y0, u0, P0 = np.asarray(wl.T, dtype=np.float64).reshape(-1), wl.Y, wl.u, wl.P_h
    if args.adj_spinup:
        s = Solver(dict(wl.cfg, storage="f64"), wl.mask, inlet0)
        s.set_fields(T=T0, Y=Y0, u=u0, P_h=P0, g_pert=wl.g_pert)
        s.step(args.adj_spinup)
        f = s.fields(L.F_T | L.F_Y | L.F_U | L.F_PH)
        s.close()
        T0, Y0, u0, P0 = f["T"], f["Y"], f["u"], f["P_h"]

    def problem(storage, n_steps=K):
        cfg = dict(wl.cfg)
        cfg["storage"] = storage
        return AdjointProblem(cfg, wl.mask, Y0, u0=u0, P_h0=P0, g_pert=None if args.adj_spinup else wl.g_pert,
                              n_steps=n_steps, checkpoint_every=C, fuel=0)

    pb = problem("f32")
    for _ in range(max(1, args.warmup)):
        pb.forward(inlet0, T0)
        pb.backward()
    fwd, bwd = [], []
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J32 = pb.forward(inlet0, T0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            gin32, gT32 = pb.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fwd.append(t1 - t0)
            bwd.append(t2 - t1)
    pb.close()
    tf, tb = statistics.median(fwd), statistics.median(bwd)
    fd = {}
    if not args.no_fd_check:
        fluid = (np.asarray(wl.mask).reshape(-1) == 0).astype(np.float64)
        p = problem("f64")
        J64 = p.forward(inlet0, T0)
        gin, gT = (v.cpu().numpy() for v in p.backward())

        def check(h):
            """|AD - FD| / sum |grad_i d_i| along args.fd_dirs Philox directions (seed 2207)."""
            rng = np.random.Generator(np.random.Philox(2207))
            errs = []
            for _ in range(args.fd_dirs):
                di = rng.standard_normal(inlet0.shape) * (inlet0 != 0) * 0.1 * np.abs(inlet0).max()
                dT = rng.standard_normal(T0.shape) * fluid * 10.0
                fdv = (p.forward(inlet0 + h * di, T0 + h * dT) - p.forward(inlet0 - h * di, T0 - h * dT)) / (2 * h)
                ad = float((gin * di).sum() + (gT * dT).sum())
                errs.append(abs(ad - fdv) / float(np.abs(gin * di).sum() + np.abs(gT * dT).sum()))
            return {"K": K, "h": h, "max_err": max(errs), "median_err": statistics.median(errs)}

        checks = [check(1e-4), check(1e-6)]
        p.close()
        g32 = np.concatenate([gin32.double().cpu().numpy().ravel(), gT32.double().cpu().numpy().ravel()])
        g64 = np.concatenate([gin.ravel(), gT.ravel()])
        fin = bool(np.isfinite(g32).all())
        fd = {"directions": args.fd_dirs, "err_measure": "|AD - FD| / sum |grad_i d_i|, FP64",
              "h_1e-4": checks[0], "h_1e-6": checks[1], "max_abs_grad": float(np.abs(g64).max()),
              "J_f64": J64, "J_f32": J32, "f32_grad_finite": fin,
              "f32_vs_f64_grad_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)) if fin else None}
    N = wl.N
    line = {"metric": "adjoint / forward time ratio, gradient of fuel consumption w.r.t. inlet profile and T0",
            "value": tb / tf, "unit": "x", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f32", "data": "synthetic", "scaling": "weak", "vs_baseline": None,
            "config": {"workload": "c5_adjoint_2d", "grid": [wl.cfg["nx"], wl.cfg["ny"]], "cells": N, "K": K,
                       "start": (f"restart {args.adj_spinup} FP64 steps after ignition" if args.adj_spinup
                                 else "ignition state"),
                       "checkpoint_every": C, "lattice": "D2Q9", "species": len(wl.cfg["species"])},
            "forward_s": tf, "backward_s": tb, "forward_mlups": N * K / tf / 1e6, "backward_mlups": N * K / tb / 1e6,
            "gradient_check": fd, "clocks": clk.summary()}
    print(json.dumps(line))


def horizon_run(args):
    """The benchmark workload over its stated horizon: the 384 x 192 x 192 reactive burner (FP32,
    closed-domain pressure, flame sensor) stepped args.horizon steps from its initial state, with
    P_th, max |u| and the range of T over the fluid cells every args.horizon_every steps (a run that
    goes non-finite shows it in these values; nothing waits on it)."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2207_11567_gb300 import from_workload
    from paper_2207_11567_gb300 import _lib as L
    torch.cuda.set_device(0)
    wl = W.make(args.workload)
    if args.open_domain:
        wl.cfg["closed_domain"] = False
    s = from_workload(wl)
    fluid = torch.as_tensor(np.asarray(wl.mask).reshape(-1) == 0, device="cuda")
    rows, done = [], 0
    t0 = time.perf_counter()
    while done < args.horizon:
        n = min(args.horizon_every, args.horizon - done)
        s.step(n)
        done += n
        sc = s.scalars()
        try:
            f = s.fields(L.F_T | L.F_U, device=True)
        except L.HLBMError as e:  # the library reports a non-finite velocity of any step
            rows.append({"step": done, "P_th": sc["P_th"], "finite": False, "status": str(e)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            break
        u = f["u"][:, fluid]
        T = f["T"][fluid]
        rows.append({"step": done, "P_th": sc["P_th"], "u_max": float(u.abs().max()), "T_min": float(T.min()),
                     "T_max": float(T.max()), "finite": bool(torch.isfinite(u).all() and torch.isfinite(T).all())})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    s.close()
    print(json.dumps({"metric": "horizon run of the benchmark workload", "workload": args.workload,
                      "closed_domain": not args.open_domain, "steps": args.horizon,
                      "seconds": time.perf_counter() - t0, "trajectory": rows}))


def small_bench(args):
    """Workloads whose state fits in L2 (C1 planar flame, FP64; C2 chamber, FP32): each timed step
    runs after an L2 flush (a 256 MB write), timed alone with CUDA events on the library's
    stream; the back-to-back rate (L2-resident state, CUDA graphs) is reported beside it."""
    import torch
    import workloads as W
    from paper_2207_11567_gb300 import from_workload
    torch.cuda.set_device(0)
    wl = W.make(args.workload)
    storage = wl.cfg["storage"]
    s = from_workload(wl)
    s.step(max(3, args.warmup))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step = []
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.zero_()
            s._after_torch()
            e0.record(s.stream)
            s.step(1)
            e1.record(s.stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
        s.synchronize()
        back_ms = _timed_steps(s, args.steps, torch)
    s.profile(True)
    s.step(10)
    kt = s.kernel_times()
    s.profile(False)
    kb = s.kernel_bytes()
    flame = None
    if wl.cfg.get("thermal") and wl.cfg["dim"] == 2:
        s.synchronize()
        t0 = time.perf_counter()
        L = s.flame_length(0.5, wl.cfg.get("T_in", 300.0), 1950.0)
        flame = {"length_cells": L, "ms_wall": 1e3 * (time.perf_counter() - t0),
                 "note": "lbm_flame_length at c = 0.5, wall time including the host read of the partial sums"}
    s.close()
    ms = statistics.mean(per_step)
    kern = {k: {"ms": t / n, "GB/s": kb[k] / (t / n * 1e-3) / 1e9} for k, (t, n) in kt.items() if n}
    dominant = max(kern, key=lambda k: kern[k]["ms"])
    peak, peak_kind = _peaks()
    ach = kern[dominant]["GB/s"]
    N = wl.N
    line = {"metric": "MLUPS per full hybrid step (LB + FD + chemistry)", "value": N / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
            "config": {"workload": args.workload, "grid": [wl.cfg["nx"], wl.cfg["ny"]], "cells": N,
                       "lattice": "D2Q9", "species": len(wl.cfg.get("species", [])), "storage": storage,
                       "l2": "state fits in L2: 256 MB L2 flush before every timed step, each step timed alone"},
            "steps_per_s": 1e3 / ms,
            "back_to_back": {"value": N * args.steps / (back_ms * 1e-3) / 1e6, "unit": "MLUPS",
                             "steps_per_s": 1e3 * args.steps / back_ms,
                             "note": "no flush, L2-resident state, CUDA graphs over step pairs"},
            "gpu_launches": sum(1 for k in kt.values() if k[1]) * args.steps,
            "roofline": {"bound": "hbm", "kernel": dominant, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "peak_kind": peak_kind, "traffic": None,
                         "note": "algorithmic bytes / CUDA-event time of the kernel in a back-to-back step"},
            "kernels": kern, "clocks": clk.summary(), "flame_length": flame}
    print(json.dumps(line))


def flame_tool_bench(args):
    """The 1-D free-flame tool on the planar flame's mixture (one-step chemistry, 4 species,
    phi = 0.83, 300 K): a 256 x 1 channel run until the consumption speed is steady, with the
    thickening factors 1 and 4, FP32. Reports the time to the converged flame (device steps and
    the tool's host control every 200 steps, wall clock) and the flame it finds."""
    import torch
    import workloads as W
    from paper_2207_11567_gb300 import from_workload
    from paper_2207_11567_gb300.flame1d import free_flame
    torch.cuda.set_device(0)
    runs = {}
    for F in (1.0, 4.0):
        wl = W.generate.flame_2d(nx=256, ny=1, storage="f32", seed=0, width_cells=20.0 * F)
        wl.cfg["thicken_F"] = F
        s = from_workload(wl)
        s.step(max(3, args.warmup))
        s.synchronize()
        t0 = time.perf_counter()
        sol = free_flame(s, chunk=200, max_steps=400000)
        s.synchronize()
        wall = time.perf_counter() - t0
        s.close()
        runs[f"F={F:g}"] = {"converged": sol.converged, "steps": sol.steps, "seconds": wall,
                            "steps_per_s": sol.steps / wall, "S_L_m_s": sol.S_L, "delta_L_m": sol.delta_L,
                            "T_b_K": sol.T_b, "Y_b": [float(v) for v in sol.Y_b]}
    total = sum(r["seconds"] for r in runs.values())
    line = {"metric": "1-D free flame: wall time to a converged flame (F = 1 and F = 4)", "value": total,
            "unit": "s", "n_gpus": 1, "steps": sum(r["steps"] for r in runs.values()), "warmup": max(3, args.warmup),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "flame1d_tool", "grid": [256, 1], "chunk": 200,
                       "mixture": "CH4/air phi 0.83, one-step chemistry, unity Lewis numbers"},
            "runs": runs}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default="full", choices=["full", "mid"],
                    help="mid: 192x96x96 cut of the same workload family, for small profiler captures")
    ap.add_argument("--only", default=None, choices=["f32", "f16"],
                    help="time one storage variant only (profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=["c4_swirl_reactive_3d", "c3_swirl_cold_3d",
                                                             "c2_chamber_2d", "c1_flame_2d", "c5_adjoint_2d",
                                                             "flame1d_tool"],
                    help="benchmark configuration (default: the reactive swirl burner)")
    ap.add_argument("--no-fd-check", action="store_true", help="c5: skip the FP64 finite-difference check")
    ap.add_argument("--fd-dirs", type=int, default=16, help="c5: directions of the finite-difference check")
    ap.add_argument("--adj-steps", type=int, default=0, help="c5: steps K (default: the workload's 2000)")
    ap.add_argument("--adj-spinup", type=int, default=400,
                    help="c5: start from the chamber's fields this many steps after ignition (0: the ignition state)")
    ap.add_argument("--stats", type=int, default=0,
                    help="with --only: sample running statistics every N steps during the timed steps")
    ap.add_argument("--probes", type=int, default=0,
                    help="with --only: record N probe cells after every step during the timed steps")
    ap.add_argument("--varcp", action="store_true",
                    help="variable species heat capacities (c_p,k(T) polynomials) in the energy equation")
    ap.add_argument("--mixavg", action="store_true",
                    help="mixture-averaged species diffusion (synthetic pair Lewis numbers)")
    ap.add_argument("--curved", action="store_true",
                    help="c3/c4: interpolated bounce-back on the injector cylinders and the exhaust cone")
    ap.add_argument("--horizon", type=int, default=0,
                    help="c3/c4: step the workload this many steps and print P_th, u and T every --horizon-every")
    ap.add_argument("--horizon-every", type=int, default=500)
    ap.add_argument("--open-domain", action="store_true", help="--horizon: hold P_th constant (open domain)")
    args = ap.parse_args()
    if args.horizon and args.impl == "ours":
        horizon_run(args)
        return
    if args.workload == "c5_adjoint_2d" and args.impl == "ours":
        adjoint_bench(args)
        return
    if args.workload == "flame1d_tool" and args.impl == "ours":
        flame_tool_bench(args)
        return
    if args.workload in ("c1_flame_2d", "c2_chamber_2d") and args.impl == "ours" and not args.only:
        small_bench(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        cb = oracle_sample(max_seconds=max(5.0, min(60.0, 2.0 * args.steps)))
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload, "sample": cb["sample"]},
                "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                            "d2h_bytes_per_step": 0}, "vs_baseline": None}
        print(json.dumps(line))
        return

    import torch
    import workloads as W
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()

    def make():
        if args.case == "mid":
            return W.generate.swirl_3d(192, 96, 96, reactive=args.workload != "c3_swirl_cold_3d", seed=0,
                                       curved=args.curved)
        if args.curved:
            size = (384, 192, 192) if args.workload == "c4_swirl_reactive_3d" else (256, 128, 128)
            return W.generate.swirl_3d(*size, reactive=args.workload == "c4_swirl_reactive_3d", seed=0,
                                       curved=True)
        return W.make(args.workload)

    if args.varcp:
        from workloads.configs import variable_cp
        make_plain = make

        def make():
            wl = make_plain()
            if wl.cfg.get("thermal"):
                variable_cp(wl.cfg)
            return wl
    if args.mixavg:
        from workloads.configs import mixture_averaged
        make_plain2 = make

        def make():
            wl = make_plain2()
            if wl.cfg.get("thermal"):
                mixture_averaged(wl.cfg)
            return wl
    if args.only:
        r = run_variant(make(), args.only, args.steps, args.warmup, torch, profile_steps=2, stats=args.stats,
                        probes=args.probes)
        print(json.dumps({"case": args.case, "storage": args.only, "ms_per_step": r["ms"] / args.steps,
                          "kernels": r["kernels"]}))
        return
    wl = make()
    # FP16-storage variant first (its own solver), then the FP32 headline
    f16 = run_variant(make(), "f16", args.steps, args.warmup, torch, profile_steps=10)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(dev_index) as clk:
        f32 = run_variant(wl, "f32", args.steps, args.warmup, torch, profile_steps=10)
    ms = job_time_ms(f32["ms"], world)
    if world > 1:
        torch.distributed.barrier()
    e2e_s, h2d, d2h = (1.0, 0, 0) if args.no_e2e else e2e_run(make(), args.steps, torch)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    N = wl.N
    import numpy as np
    n_fluid = int((np.asarray(wl.mask).reshape(-1) == 0).sum())
    value = job_value(N, args.steps, world, ms)
    peak, peak_kind = _peaks()
    kern = f32["kernels"]
    dominant = max(kern, key=lambda k: kern[k]["ms_avg"] * kern[k]["launches"])
    dk = kern[dominant]
    model = model_bytes(wl, dominant, "f32")
    alg_bytes = model * n_fluid if model else dk["bytes"]
    achieved = alg_bytes / (dk["ms_avg"] * 1e-3) / 1e9
    traffic, warp_inst = None, None
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            prof = json.load(f)
            traffic = prof.get(f"{dominant}:{args.workload}:f32") or None
            warp_inst = prof.get(f"{dominant}:{args.workload}:f32:warp_inst") or None
    except Exception:
        traffic = None
    # instruction-issue roof: 152 SMs x 4 schedulers x 1 warp instruction per cycle x 32 lanes at
    # the sampled SM clock (thread instructions per second)
    clk_summary = clk.summary()
    sm_hz = (clk_summary.get("sm_mhz") or 2070.0) * 1e6
    issue_peak = 152 * 4 * 32 * sm_hz
    issue = None
    if warp_inst and not args.curved:
        ach = warp_inst * 32 / (dk["ms_avg"] * 1e-3)
        issue = {"achieved": ach / 1e12, "peak": issue_peak / 1e12, "unit": "T thread-instructions/s",
                 "frac": ach / issue_peak, "warp_inst_per_launch": warp_inst,
                 "note": "ncu instruction count of the same kernel (192x96x96 capture x8), live CUDA-event time"}
    per_step_launches = sum(1 for k in kern.values() if k["launches"])
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "value_fluid_cells": job_value(n_fluid, args.steps, world, ms),
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "grid": [wl.cfg["nx"], wl.cfg["ny"], wl.cfg["nz"]], "cells": N,
                   "fluid_cells": n_fluid,
                   "lattice": "D3Q27" if wl.cfg["dim"] == 3 else "D2Q9", "collision": "cumulant+smagorinsky",
                   "species": len(wl.cfg.get("species", [])) if wl.cfg.get("thermal") else 0,
                   "reactions": len(wl.cfg.get("reactions", [])) if wl.cfg.get("thermal") else 0,
                   "thicken_F": wl.cfg.get("thicken_F"), "flame_sensor": wl.cfg.get("flame_sensor"),
                   "closed_domain": wl.cfg.get("closed_domain"), "storage": "f32",
                   "parallelism": f"replicas{world}", "walls": "interpolated" if args.curved else "half-way",
                   "l2": f"state {wl.N * (27 if wl.cfg['dim'] == 3 else 9) * 8 / 1e9:.2f} GB of populations > L2, no flush needed"},
        "e2e": {"value": N * args.steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "note": "set_fields from pinned host memory + K steps + get_fields into pinned host memory, "
                        "through the C ABI"},
        "gpu_launches": per_step_launches * args.steps,
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "bytes_per_launch": alg_bytes, "bytes_per_fluid_cell": model, "fluid_cells": n_fluid,
                     "kernel_extra_bytes_per_launch": dk["bytes"] - alg_bytes, "ms_per_launch": dk["ms_avg"],
                     "issue": issue,
                     "note": "achieved = algorithmic bytes (model_bytes per fluid cell x fluid cells) / CUDA-event "
                             "time of the kernel; kernel_extra_bytes_per_launch: words the kernel moves beyond "
                             "the model (32-bit link / stencil words instead of the 1-byte mask, the flame "
                             "sensor's F_loc in and out)"},
        "kernels": {k: {"ms": v["ms_avg"],
                        "GB/s": ((model_bytes(wl, k, "f32") or 0) * n_fluid or v["bytes"]) / (v["ms_avg"] * 1e-3) / 1e9
                        if v["ms_avg"] else 0.0}
                    for k, v in kern.items() if v["launches"]},
        "fp16_storage": {"value": N * args.steps * world / (f16["ms"] * 1e-3) / 1e6, "unit": "MLUPS",
                         "ms_per_step": f16["ms"] / args.steps,
                         "lb_ms": f16["kernels"]["lb_stream_collide"]["ms_avg"],
                         "lb_GB/s": model_bytes(wl, "lb_stream_collide", "f16") * n_fluid
                         / (f16["kernels"]["lb_stream_collide"]["ms_avg"] * 1e-3) / 1e9},
        "clocks": clk_summary,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample()
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
