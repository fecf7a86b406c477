#!/usr/bin/env python
"""Throughput of the WP-CCC hot path on GB300: RK4 steps per second.

Workload: the two-centre p + H calculation (Z_T = Z_P = 1): hydrogenic n <= 4
plus 10 Coulomb wave-packet pseudostates per l <= 3 on each centre (N_T = N_P =
190, N = 380 coupled amplitudes), a 48 x 48 Gauss-Laguerre x Gauss-Legendre
(eta, tau) rule, v = 1.5 a.u., 32 impact parameters uniform in [0.2, 12] a.u.,
z from -50 to 50 a.u. with h = 0.1 (1000 RK4 steps per path).  Inputs are
synthetic (generated basis, straight-line paths).

One bench step advances all 32 paths by STEP_RK4 consecutive RK4 steps (the
steps of the run are consecutive and centred on z = 0) through the public call
wpccc_propagate: matrix elements at every z it needs, the solve S X = H, the
RK4 sweep.  `value` counts RK4 steps of all paths on all ranks per second of
device time.

By default (--precision auto) the run times the plain FP64 form and then the
reduced-precision forms on the same steps from the same initial amplitudes;
the headline `value` is the fastest form whose probabilities stay within 1e-6
(absolute) of the FP64 form's, and every timed form is listed under `forms`
with its rate and measured error.  `e2e` times the headline form again with
the amplitudes copied in from pinned host memory and the probabilities copied
back every step.

--impl reference times the FP64 CPU oracle (the test oracle of this repository)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched/mixed vs plain FP64 RK4 steps/s at ≤1e-6 prob error; % FP64 peak"
UNIT = "RK4 steps/s"
WORKLOAD = "p_H_2c_n4l3"
STEP_RK4 = 16           # RK4 steps of every path per bench step
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_DFMA_MEASURED_TFLOPS = 1.20   # FMA microbenchmark on this machine's GB300 (all SMs, register operands)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_FFMA_MEASURED_TFLOPS = 69.9


# forms of the batched bench: (precision mode, refinement sweeps, name)
BATCH_FORMS = ((0, 2, "fp64"), (4, 2, "fp64-tensor-core"), (5, 4, "fp64-tc-refined"), (5, 2, "mixed-fp64-tc-elements"),
               (3, 2, "mixed-tensor-core"))

SOLVE_MODES = {"stage": lambda w: w.SOLVE_STAGE, "matrix": lambda w: w.SOLVE_MATRIX, "schur": lambda w: w.SOLVE_SCHUR}


def _measured_peak(key: str, fallback: float) -> float:
    """A peak from MEASURED_PEAKS.json (measured on the GB300s), else the stated fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError, TypeError):
        return fallback


BF16_MEASURED_TFLOPS = _measured_peak("bf16_tflops", 1900.0)               # burst: a kernel timed alone
BF16_SUSTAINED_TFLOPS = _measured_peak("bf16_tflops_sustained", 1700.0)    # a kernel timed inside a long step
HBM_MEASURED_GBS = _measured_peak("hbm_gbs", 6800.0)
CONFIG_DESC_C6 = ("two-centre bare C6+ on H (Z_T=1, Z_P=6): hydrogenic n<=6 + 20 Coulomb wave-packet bins per "
                  "l<=5 (k<=4) on each centre, all m, N_T=N_P=811, N=1622; 128x48 (eta,tau) nodes; Nr=2000 to "
                  "100 a.u.; v=2; 16 b uniform in [0.5,15]; the paper's geometric z-grid, z_min=1e-3, "
                  "|z|<=50, 500 nodes per side (1000 RK4 steps)")
CONFIG_DESC = ("two-centre p+H (Z_T=Z_P=1): hydrogenic n<=4 + 10 Coulomb wave-packet bins per l<=3 (k<=3) "
               "on each centre, all m, N_T=N_P=190, N=380; 48x48 (eta,tau) nodes; Nr=2000 to 100 a.u.; "
               "v=1.5; 32 b uniform in [0.2,12]; z in [-50,50], h=0.1")


CONFIG_DESC_LI = ("differentiation form: two-centre p + Li-like one-electron target, model potential "
                  "V(r) = -[1 + 2 e^{-a r}(1 + b r)]/r with a, b drawn within 5% of (3.0, 1.5) (seed 0); target: "
                  "box eigenstates n<=4 without the core 1s + 10 wave packets per l<=3 (k<=3); projectile "
                  "hydrogen-like n<=4 + 10 wave packets per l<=3; all m, N = 379; 48x48 (eta,tau) nodes; v = 1.5; "
                  "32 b uniform in [0.2,12]; z in [-50,50], h = 0.1; observables: capture and 2p excitation; "
                  "theta = (Z_p, a, b)")


def _reasons(mask: int) -> list:
    names = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
             0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
             0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}
    return [n for b, n in names.items() if mask & b]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running. start() returns once
    the first sample has arrived (or after 3 s), so that sampling is live when the timed region begins."""

    def __init__(self, index: int, cmd=None):
        self.index = index
        self.cmd = cmd
        self.samples = []
        self.proc = None
        self.thread = None
        self.first = threading.Event()

    def start(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active"
        cmd = self.cmd or ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                           "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        self.first.wait(timeout=3.0)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 4:
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), float(parts[2]), int(parts[3], 16)))
                    self.first.set()
                except ValueError:
                    pass

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        mask = 0
        for s in self.samples:
            mask |= s[3]
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "power_w_max": max(s[2] for s in self.samples),
                "reasons": _reasons(mask & ~0x1), "samples": len(self.samples)}


def cpu_oracle_rate(basis, paths, n_steps: int, path_index: int = 16) -> dict:
    """The FP64 oracle, as it stands, on one path for n_steps RK4 steps (host cores)."""
    from oracle import wpccc_oracle as O
    b = float(paths.b[path_index])
    v = float(paths.v[path_index])
    zg = paths.z[path_index]
    k0 = 500 - n_steps // 2                      # steps around closest approach
    seg = zg[k0:k0 + n_steps + 1]
    c0 = O.initial_state(basis)
    t0 = time.perf_counter()
    O.rk4_path(lambda z: O.coupling_M(basis, b, v, z), seg, c0)
    dt = time.perf_counter() - t0
    threads = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        threads = max(int(i.get("num_threads", 1)) for i in threadpool_info()) or threads
    except Exception:
        pass
    return {"value": n_steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"1 path (b={b:.3f}), {n_steps} RK4 steps around z=0 of the same workload, "
                      f"{dt:.1f} s; numpy/LAPACK with {threads} threads"}


def run_reference(args) -> None:
    import wpccc_inputs as wi
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    basis, paths = wi.config_inputs(WORKLOAD)
    per_step = 2                                  # RK4 steps of one path per bench step
    for _ in range(args.warmup):
        cpu_oracle_rate(basis, paths, per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_rate(basis, paths, per_step)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    cb = cpu_oracle_rate(basis, paths, per_step)
    cb["value"] = value
    cb["sample"] = f"each step: 1 path, {per_step} RK4 steps of the same workload"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": CONFIG_DESC, "form": "FP64 CPU oracle"},
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_batch(args) -> dict:
    """Batched form: six speeds (bases of different size), 64 paths each, uneven step counts (the
    same z extent at h = 0.1 v/1.5), captured into one CUDA graph with autotuned chunk schedules.
    Timed against the same sets propagated by separate wpccc_propagate calls (plain FP64 form)."""
    import torch
    import wpccc_inputs as wi
    import paper_2403_04252_gb300 as w
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    step_ref = args.rk4_per_step if args.rk4_per_step != STEP_RK4 else 4
    sets_in = wi.batch_inputs()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v_, basis_, paths_ = sets_in[2]
        cpu = cpu_oracle_rate(basis_, paths_, 3, path_index=32)
    sets, c = [], []
    for v, basis, paths in sets_in:
        g = w.Basis(basis, device=local)
        g.set_workspace_limit(8 << 30)
        g.set_solve_mode(SOLVE_MODES[args.solve_mode](w))
        zg = paths.z[0]
        n = zg.size - 1
        k = max(1, int(round(step_ref * 1.5 / v)))          # same z extent at every speed
        k0 = n // 2 - k // 2
        seg = zg[k0:k0 + k + 1]
        sets.append((g, paths.b, v, seg))
        t = torch.zeros((paths.n_paths, g.N), dtype=torch.complex128, device=dev)
        t[:, 0] = 1.0
        c.append(t)
    units = sum(b.size * (seg.size - 1) for (_, b, _, seg) in sets)
    stream = torch.cuda.current_stream(dev)

    def reset_amplitudes():
        for t in c:
            t.zero_()
            t[:, 0] = 1.0

    def build(mode: int, iters: int):
        for g, _, _, _ in sets:
            g.set_refine_iters(iters)
        reset_amplitudes()
        t0 = time.perf_counter()
        bt = w.Batch(sets, c, precision_mode=mode, autotune=True)
        return bt, time.perf_counter() - t0

    def time_form(mode: int, iters: int) -> dict:
        """builds the batch graph of one form, warms it up, times args.steps launches"""
        bt, t_create = build(mode, iters)
        for _ in range(args.warmup):
            bt.launch()
        bt.status()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bt.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks_f = sampler.stop()
        bt.status()
        ms_f = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms_f], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_f = float(t.item())
        chunk_f, tuned_f = bt.info()
        P_f = np.concatenate([w.probabilities(t).cpu().numpy().ravel() for t in c])
        bt.close()
        return {"mode": mode, "iters": iters, "ms": ms_f, "value": world * units * args.steps / (ms_f / 1e3),
                "clocks": clocks_f, "P": P_f, "create_s": t_create, "chunk_steps": chunk_f, "tuned": tuned_f}

    # the batched graph in the FP64-accurate forms and the fastest refined form; the headline is the
    # fastest within 1e-6 of the plain FP64 graph on the same launches
    forms = {}
    for mode, iters, name in BATCH_FORMS:
        try:
            forms[name] = time_form(mode, iters)
        except w.WpcccError as exc:
            forms[name] = {"unsupported": str(exc)}
            continue
        forms[name]["err"] = float(np.abs(forms[name]["P"] - forms["fp64"]["P"]).max())
    ok = [n for n, f in forms.items() if "unsupported" not in f and f["err"] <= 1e-6]
    head = max(ok, key=lambda n: forms[n]["value"])
    H = forms[head]
    mode, iters = H["mode"], H["iters"]
    ms, value, clocks, t_create = H["ms"], H["value"], H["clocks"], H["create_s"]
    chunk_steps, tuned = H["chunk_steps"], H["tuned"]
    batch, _ = build(mode, iters)
    for _ in range(args.warmup):
        batch.launch()
    batch.status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the same sets, one wpccc_propagate call per set after another, profiled per kernel
    for g, _, _, _ in sets:
        g.profile_enable(True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for (g, b, v, seg), cc in zip(sets, c):
            g.propagate(b, v, seg, c=cc, precision_mode=mode)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    prof = {}
    for g, _, _, _ in sets:
        for kname, (kms, kn) in g.profile_read().items():
            a = prof.setdefault(kname, [0.0, 0])
            a[0] += kms
            a[1] += kn
        g.profile_enable(False)
    # end to end: amplitudes from pinned host memory, probabilities back, per launch
    c_host = [torch.zeros(t.shape, dtype=torch.complex128).pin_memory() for t in c]
    for t in c_host:
        t[:, 0] = 1.0
    P_host = [torch.empty(t.shape, dtype=torch.float64).pin_memory() for t in c]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for t, th in zip(c, c_host):
            t.copy_(th, non_blocking=True)
        batch.launch()
        for t, ph in zip(c, P_host):
            ph.copy_(w.probabilities(t), non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = sum(t.numel() * 16 for t in c_host)
    d2h = sum(t.numel() * 8 for t in P_host)
    # roofline of every kernel category (from the profiled separate calls: the same kernels), the work
    # summed over the six bases; the dominant category (largest device time) is the line's `roofline`
    work = {}
    cat_meta = {}
    for (g, b, v, seg), (vv, basis, _) in zip(sets, sets_in):
        evals = args.steps * b.size * (2 * (seg.size - 1) + 1)
        n_half = int(sum(1 for m in basis.P.st_m if m >= 0))
        cats = _category_rooflines(basis, mode, args.solve_mode, basis.N, n_half)
        cats["rk4"] = (_rk4_flops_per_step(mode, args.solve_mode, basis.N, basis.T.N, basis.P.N),
                       ("alu", FP64_PEAK_TFLOPS, "TFLOP/s"), "k_rk4")
        for k, (per_unit, meta, name) in cats.items():
            n_units = args.steps * b.size * (seg.size - 1) if k == "rk4" else evals
            work[k] = work.get(k, 0.0) + per_unit * n_units
            cat_meta[k] = (meta, name)

    def roof_b(key: str) -> dict:
        k_ms, k_n = prof[key]
        (bound, peak, unit), name = cat_meta[key]
        ach = work[key] / (k_ms / 1e3) / (1e9 if unit == "GB/s" else 1e12)
        return {"bound": bound, "kernel": name, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "traffic": None, "peak_source": _peak_source(bound, peak), "launch_ms_avg": k_ms / max(k_n, 1)}

    timed = {k: prof[k][0] for k in work if k in prof and prof[k][1] > 0}
    dom = max(timed, key=lambda k: timed[k])
    roofline_b = roof_b(dom)
    roofline_b["by_kernel"] = {k: {kk: vv for kk, vv in roof_b(k).items()
                                   if kk in ("kernel", "bound", "achieved", "peak", "unit", "frac")}
                               | {"ms": timed[k], "share": timed[k] / sum(timed.values())} for k in timed}
    roofline_b["timing"] = "kernel times from the same sets' separate, profiled wpccc_propagate calls"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 4: "bf16-slices(fp64-accurate)+f64", 3: "bf16x4-slices+f32+f64"}.get(
                mode, "bf16-slices(fp64-accurate)+f32+f64"),
            "data": "synthetic",
            "config": {"workload": "batched form: two-centre p+H at v in {0.5,0.8,1.2,2,3,4}, pseudostates per "
                                   "l = round(8+8(v-0.5)/3.5) = 8..16 (k<=3), hydrogenic n<=4, l<=3, all m, "
                                   "72 x 48 (eta, tau) nodes "
                                   f"(N = {[g.N for g, _, _, _ in sets]}); 64 b uniform in [0.2,12] per speed "
                                   "(384 paths); h = 0.1 v/1.5 (step count proportional to 1/v)",
                       "bench_step": "one CUDA graph launch advancing every path through the same z extent "
                                     f"(RK4 steps per speed {[int(seg.size - 1) for _, _, _, seg in sets]}), "
                                     "centred on z = 0; each launch recomputes all elements and solves",
                       "form": f"batched, {head} (precision mode {mode}, {iters} refinement sweeps): all six "
                               "bases' chunk pipelines captured into one CUDA graph, concurrent streams, autotuned "
                               f"chunk schedules; solve mode {args.solve_mode}",
                       "l2": "inputs larger than L2 (S and H of one launch: several GB)"},
            "batched_vs_separate_calls": {"separate_calls_value": world * units * args.steps / (ms_seq / 1e3),
                                          "speedup": ms_seq / ms},
            "autotune": {"chunk_steps": [int(x) for x in chunk_steps],
                         "ms_per_rk4_step": [float(x) for x in tuned], "create_s": t_create},
            "roofline": roofline_b,
            "kernel_ms_separate_calls": {k: v_[0] for k, v_ in prof.items()},
            "forms": {n: ({"value": f["value"], "ms_per_step": f["ms"] / args.steps, "create_s": f["create_s"],
                           "max_abs_prob_error_vs_fp64": f["err"],
                           "meets_fp64_bar": bool(np.all(np.abs(f["P"] - forms["fp64"]["P"])
                                                         <= 1e-10 * np.maximum(forms["fp64"]["P"], 1e-4)))}
                          if "unsupported" not in f else f) for n, f in forms.items()},
            "speedup_vs_plain_fp64": value / forms["fp64"]["value"],
            "prob_error": {"max_abs": H["err"], "bound": 1e-6,
                           "against": "the plain FP64 batch graph on the same launches (whose amplitudes equal "
                                      "separate plain FP64 calls bit for bit, tests/test_gpu_parity.py)"},
            "e2e": {"value": world * units * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(n for _, n in prof.values())), "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    batch.close()
    for g, _, _, _ in sets:
        g.close()
    return line


def oracle_gradient_rate(basis, paths, gw, n_steps: int, path_index: int = 8) -> dict:
    """The oracle's forward-mode gradient (every line of Algorithm 1 differentiated) on one path, a few
    steps around z = 0, on the host cores."""
    from oracle import wpccc_oracle as O
    zg = paths.z[path_index]
    k0 = zg.size // 2
    seg = zg[k0:k0 + n_steps + 1]
    b, v = float(paths.b[path_index]), float(paths.v[path_index])
    t0 = time.perf_counter()
    O.gradient(basis, b, v, seg, gw)
    dt = time.perf_counter() - t0
    return {"value": n_steps / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 path (b={b:.3f}), {n_steps} RK4 steps around z=0 with the forward-mode gradient of "
                      f"two observables w.r.t. 3 parameters, {dt:.1f} s; numpy/LAPACK on the host cores"}


def run_one_centre_large(args) -> None:
    """One-centre p + H at l <= 10 (N = 4257): the plain FP64 form with the RK4 vectors in global memory
    (the shared-memory sweep holds N <= ~2840).  One bench step advances every path by a few RK4 steps
    around closest approach; every position's D_T is assembled (N^2 complex, 290 MB)."""
    import torch
    import wpccc_inputs as wi
    import paper_2403_04252_gb300 as w
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    basis, paths = wi.config_inputs("p_H_1c_n10l10")
    g = w.Basis(basis, device=local)
    g.set_workspace_limit(int((args.workspace_gb or 64.0) * (1 << 30)))
    N = g.N
    n_paths = paths.n_paths if args.paths <= 0 else min(args.paths, paths.n_paths)
    b = paths.b[:n_paths]
    v = float(paths.v[0])
    zg = paths.z[0]
    STEP = args.rk4_per_step if args.rk4_per_step != STEP_RK4 else 4
    first = max(0, (zg.size - 1) // 2 - (args.warmup + args.steps) * STEP // 2)

    def segment(k):
        a = first + k * STEP
        return zg[a:a + STEP + 1]
    c = torch.zeros((n_paths, N), dtype=torch.complex128, device=dev)
    c[:, 0] = 1.0
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        g.propagate(b, v, segment(k), c=c)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    g.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        g.propagate(b, v, segment(args.warmup + k), c=c)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = g.profile_read()
    g.profile_enable(False)
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    P = w.probabilities(c).cpu().numpy()
    norm_dev = float(np.abs(P.sum(axis=1) - 1.0).max())
    value = world * n_paths * STEP * args.steps / (ms / 1e3)
    # end to end: amplitudes from pinned host memory, probabilities back, every step
    c_host = torch.zeros((n_paths, N), dtype=torch.complex128).pin_memory()
    c_host[:, 0] = 1.0
    P_host = torch.empty((n_paths, N), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        c.copy_(c_host, non_blocking=True)
        g.propagate(b, v, segment(args.warmup + k), c=c)
        P_host.copy_(w.probabilities(c), non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # roofline: the RK4 sweep, four FP64 matrix-vector products of 8 N^2 flops per path-step, against
    # the element assembly (the direct blocks of Eq. 6)
    rk_ms, rk_n = prof["rk4"]
    rk_flops = 4.0 * 8.0 * N * N * n_paths * STEP * args.steps
    ach = rk_flops / (rk_ms / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "one-centre p+H (Z=1): hydrogenic n<=10 + 32 Coulomb wave-packet bins per l<=10 "
                                   f"(k<=2), all m, N={N}; v=2 (100 keV); {n_paths} b in [0.5, 8]; z in [-40, 40], "
                                   "h=0.1",
                       "form": "plain FP64, M = -(i/v) D_T; RK4 vectors in global memory (one launch per RK4 "
                               "stage, GPU-wide matrix-vector products)",
                       "bench_step": f"{STEP} RK4 steps of each path, consecutive segments centred on z = 0",
                       "l2": f"inputs larger than L2: D_T of one position is {16 * N * N / 1e6:.0f} MB"},
            "norm_deviation": norm_dev,
            "roofline": {"bound": "alu", "kernel": "k_rk4_wide", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "FP64 pipe from unit counts and clocks (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                         "launch_ms_avg": rk_ms / max(rk_n, 1)},
            "kernel_ms": {k: v_[0] for k, v_ in prof.items()},
            "e2e": {"value": world * n_paths * STEP * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": c_host.numel() * 16, "d2h_bytes_per_step": P_host.numel() * 8},
            "gpu_launches": int(sum(n for _, n in prof.values())), "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if dist:
        dist.destroy_process_group()


def run_grad(args) -> None:
    """Differentiation form: wpccc_propagate_adjoint (forward sweep with checkpoints, reverse sweep
    with recomputation, element adjoint) on consecutive segments of the 32 paths, timed against the
    plain FP64 propagation of the same segments; a sampled full-size check against central
    differences of the GPU's own propagation."""
    import torch
    import wpccc_inputs as wi
    import paper_2403_04252_gb300 as w
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    basis, paths = wi.li_inputs(seed=0)
    gw = wi.observable_weights(basis)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_gradient_rate(basis, paths, gw, 3)
    g = w.Basis(basis, device=local)
    g.set_workspace_limit(int((args.workspace_gb or 16.0) * (1 << 30)))
    n_paths = paths.n_paths if args.paths <= 0 else min(args.paths, paths.n_paths)
    bs = paths.b[:n_paths]
    zg = paths.z[0]
    S = args.rk4_per_step if args.rk4_per_step != STEP_RK4 else 50
    K = max(1, min(args.checkpoint_every, S))
    n_seg = args.warmup + 2 * args.steps + 1
    k0 = max(0, (zg.size - 1) // 2 - (n_seg * S) // 2)

    def segment(k: int):
        a = k0 + k * S
        return zg[a:a + S + 1]
    c = torch.zeros((n_paths, g.N), dtype=torch.complex128, device=dev)
    c[:, 0] = 1.0
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        g.propagate_adjoint(bs, 1.5, segment(k), gw, checkpoint_every=K, c=c)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    g.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        _, P, J = g.propagate_adjoint(bs, 1.5, segment(args.warmup + k), gw, checkpoint_every=K, c=c)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = g.profile_read()
    g.profile_enable(False)
    finite = bool(torch.isfinite(J).all().item())
    # the plain FP64 form on the next segments
    e0.record(stream)
    for k in range(args.steps):
        g.propagate(bs, 1.5, segment(args.warmup + args.steps + k), c=c)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms, ms_fwd], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_fwd = float(t[0].item()), float(t[1].item())
    units = n_paths * S
    value = world * units * args.steps / (ms / 1e3)
    # end to end: amplitudes from pinned host memory, observables and gradients back
    c_host = torch.zeros((n_paths, g.N), dtype=torch.complex128).pin_memory()
    c_host[:, 0] = 1.0
    P_host = torch.empty((n_paths, gw.shape[0]), dtype=torch.float64).pin_memory()
    J_host = torch.empty((n_paths, gw.shape[0], g.n_par), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        c.copy_(c_host, non_blocking=True)
        _, P, J = g.propagate_adjoint(bs, 1.5, segment(args.warmup + k), gw, checkpoint_every=K, c=c)
        P_host.copy_(P, non_blocking=True)
        J_host.copy_(J, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # sampled full-size check: one path, 20 steps around z = 0, against central differences
    fd_check = None
    if rank == 0 and not args.no_fd_check:
        zs = zg[(zg.size - 1) // 2 - 10:(zg.size - 1) // 2 + 11]
        bsel = [float(paths.b[8])]
        _, _, Jc = g.propagate_adjoint(bsel, 1.5, zs, gw, checkpoint_every=7)
        Jc = Jc.cpu().numpy()[0]
        a0, b0 = basis.mp_a, basis.mp_b
        th0 = (1.0, a0, b0)
        fd_check = {"path": "b=%.3f, 20 RK4 steps around z=0" % bsel[0], "checkpoint_every": 7}
        for h in (1e-5, 1e-4):
            rel = []
            for p in range(3):
                vals = []
                for sg in (1.0, -1.0):
                    th = list(th0)
                    th[p] += sg * h
                    gb = w.Basis(wi.li_basis(Z_p=th[0], a=th[1], b=th[2]), device=local)
                    cc = gb.propagate(bsel, 1.5, zs)
                    vals.append((w.probabilities(cc).cpu().numpy() @ gw.T)[0])
                    gb.close()
                fd = (vals[0] - vals[1]) / (2 * h)
                rel.append(float(np.max(np.abs(fd - Jc[:, p]) / np.maximum(np.abs(Jc[:, p]), 1e-300))))
            fd_check[f"max_rel_diff_h{h:g}"] = dict(zip(("Z_p", "a", "b"), rel))
        fd_check["dP_dtheta"] = {o: dict(zip(("Z_p", "a", "b"), map(float, Jc[i])))
                                 for i, o in enumerate(("capture", "2p_excitation"))}
    flops = {"mol_gemm": 0.0, "solve": 0.0}
    n_half = int(sum(1 for m in basis.P.st_m if m >= 0))
    # positions evaluated per call: the forward sweep (2 per step + 1 per segment) and the reverse sweep
    evals = args.steps * n_paths * 2 * (2 * S + -(-S // K))
    flops["mol_gemm"] = 8.0 * basis.T.N * n_half * basis.quad.G * evals
    flops["solve"] = (8.0 / 3.0) * basis.N ** 3 * evals
    dom = max(prof, key=lambda k: prof[k][0])
    dom_f = dom if dom in flops else "mol_gemm"
    achieved = flops[dom_f] / (prof[dom_f][0] / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CONFIG_DESC_LI, "paths": n_paths,
                       "bench_step": f"wpccc_propagate_adjoint over {S} RK4 steps of each path (checkpoint every "
                                     f"{K}): observables and their gradient w.r.t. (Z_p, a, b); consecutive "
                                     "segments centred on z = 0",
                       "form": "differentiation: forward sweep with checkpoints, reverse sweep recomputing S, H "
                               "and LU per segment, adjoint RK4 and node-level adjoint of the element assembly",
                       "l2": "inputs larger than L2 (S and H of one segment: ~15 GB)"},
            "forms": {"adjoint": {"value": value, "ms_per_step": ms / args.steps},
                      "plain_fp64_forward": {"value": world * units * args.steps / (ms_fwd / 1e3),
                                             "ms_per_step": ms_fwd / args.steps}},
            "adjoint_cost_vs_forward": ms / ms_fwd,
            "gradient_finite": finite,
            "fd_check": fd_check,
            "kernel_ms": {k: v_[0] for k, v_ in prof.items()},
            "roofline": {"bound": "alu", "kernel": {"mol_gemm": "k_mol_gemm<double>",
                                                           "solve": "k_lu_solve"}[dom_f],
                         "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "FP64 pipe from unit counts and clocks (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                         "dominant_category": dom},
            "e2e": {"value": world * units * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": c_host.numel() * 16,
                    "d2h_bytes_per_step": P_host.numel() * 8 + J_host.numel() * 8},
            "gpu_launches": int(sum(n for _, n in prof.values())), "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if dist:
        dist.destroy_process_group()


# algorithmic bytes or flops per position of each kernel category, and the peak each is measured against
def _category_rooflines(basis, mode: int, solve_mode: str, N: int, n_half: int) -> dict:
    """Per position (evaluation of S and H at one z): the work each category of kernels must do, as the
    method defines it, with the bound and peak that apply.  Contraction: K and Q over the full N_T x N_P
    block, 4 real flops per node each (8 N_T N_P G; the q -> -q reflection lets the kernels form only the
    n_half projectile columns with q >= 0, and the tensor-core forms issue 10 or 28 bf16 slice products per
    algorithmic product: neither changes the algorithmic count).  Factorisation: the Schur complement's
    lower triangle and its Cholesky factor (4 N_P^2 N_T + 4/3 N_P^3), or LU (8/3 N^3).  Node tables and
    rotation/direct blocks are bound by memory: the bytes they must write (node tables of the layout the
    form uses; S and H)."""
    NT, NP_, G = basis.T.N, basis.P.N, basis.quad.G
    mixed = mode in (1, 2, 3, 5)
    tc = mode in (3, 4, 5)
    slices = 3 if mode == 3 else 7
    nradT, nradP = basis.T.n_rad, basis.P.n_rad
    lT = int(max(basis.T.rad_l)) if nradT else 0
    lP = int(max(basis.P.rad_l)) if nradP else 0
    nlqT, nlqP = (lT + 1) * (lT + 2) // 2, (lP + 1) * (lP + 2) // 2
    dmax = lT + lP
    if tc:
        node_bytes = slices * 2 * NT * G * 2 + (n_half + 2 * (dmax + 1)) * G * 8
    elif mode == 1:
        node_bytes = (NT + n_half) * G * 4 + 2 * (dmax + 1) * G * 8
    else:
        node_bytes = (nradT + nradP + nlqT + nlqP) * G * 8 + 2 * (dmax + 1) * G * 16
    if solve_mode == "schur":
        f_solve = 4.0 * NP_ * NP_ * NT + (4.0 / 3.0) * NP_ ** 3
    else:
        f_solve = (8.0 / 3.0 + (8.0 if (solve_mode == "matrix" and not mixed) else 0.0)) * N ** 3
    mol_name = {1: "k_mol_gemm_f32q", 3: "k_mol_tc64<4>", 4: "k_mol_tc64<7>", 5: "k_mol_tc64<7>"}.get(
        mode, "k_mol_gemm<double>")
    solve_name = (("k_schur_factor<float>" if solve_mode == "schur" else "k_lu_factor_f32") if mixed
                  else ("k_schur_factor<double>" if solve_mode == "schur" else "k_lu_solve"))
    mol_peak = (("tensor", BF16_SUSTAINED_TFLOPS, "TFLOP/s") if tc else
                ("alu", FP32_PEAK_TFLOPS, "TFLOP/s") if mode == 1 else ("alu", FP64_PEAK_TFLOPS, "TFLOP/s"))
    return {
        "node_tables": (float(node_bytes), ("hbm", HBM_MEASURED_GBS, "GB/s"),
                        "k_node_tables<float>" if (tc or mode == 1) else "k_node_tables<double>"),
        "mol_gemm": (8.0 * NT * NP_ * G, mol_peak, mol_name),
        "rotate_direct": (float(2 * 16 * N * N + 2 * 16 * NT * n_half), ("hbm", HBM_MEASURED_GBS, "GB/s"),
                          "k_rotate+k_direct"),
        "solve": (f_solve, ("alu", FP32_PEAK_TFLOPS if mixed else FP64_PEAK_TFLOPS, "TFLOP/s"), solve_name),
    }


def _peak_source(bound: str, peak: float) -> str:
    if bound == "hbm":
        return "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    if bound == "tensor":
        return ("measured sustained bf16 dense tensor peak (MEASURED_PEAKS.json bf16_tflops_sustained; the kernel "
                "is timed inside the step) against the method's algorithmic flops, not the bf16 slice products "
                "the kernel issues")
    if peak == FP32_PEAK_TFLOPS:
        return ("FP32 pipe from unit counts and clocks (152 SMs x 128 FFMA/clk x 2.07 GHz); "
                f"measured FFMA microbenchmark {FP32_FFMA_MEASURED_TFLOPS} TFLOP/s")
    return ("FP64 pipe from unit counts and clocks (152 SMs x 2 DFMA/clk x 2.07 GHz); "
            f"measured DFMA microbenchmark {FP64_DFMA_MEASURED_TFLOPS} TFLOP/s")


def _rk4_flops_per_step(mode: int, solve_mode: str, N: int, NT: int, NP_: int) -> float:
    """RK4 per path-step (FP64): 4 applications of M; matrix form X y, stage form H y + two triangles,
    Schur form H y, K^+ t_T, K x_P and two triangles of N_P; refined forms H y, two preconditioner solves
    and one residual S x (off-diagonal blocks)."""
    mixed = mode in (1, 2, 3, 5)
    schur = solve_mode == "schur"
    if mixed:
        solve_once = (16.0 * NT * NP_ + 8.0 * NP_ * NP_) if schur else 8.0 * N * N
        return 4.0 * (8.0 * N * N + 2.0 * solve_once + 16.0 * NT * NP_)
    if schur:
        return 4.0 * (8.0 * N * N + 16.0 * NT * NP_ + 8.0 * NP_ * NP_)
    return {"matrix": 32.0, "stage": 64.0}[solve_mode] * N * N


# DRAM bytes per position of a kernel on a workload, measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over a capture of whole launches, divided by the positions): only kernels whose code
# is unchanged since the capture are listed (the others report traffic null)
MEASURED_TRAFFIC_PER_POSITION = {
    # ncu over 33 positions of the p + H workload, precision mode 3: (314.0 + 17.5) MB and (3.7 + 263.2) MB
    ("p_H_2c_n4l3", "k_mol_tc64<4>"): 10.05e6,
    ("p_H_2c_n4l3", "k_node_tables<float>"): 8.09e6,
}


def run_fixed_speed(args, sub: bool = False) -> dict:
    """One fixed-speed workload (p + H, or C6+ on H): every precision form timed on the same consecutive
    segments of all paths; the headline is the fastest form within 1e-6 of the plain FP64 form both on the
    timed segments and, for p + H, over whole paths of a subset of impact parameters."""
    import torch
    import wpccc_inputs as wi

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c6 = args.workload == "C6_H_2c_n6l5"

    basis, paths = wi.config_inputs(args.workload)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(basis, paths, 40 if not c6 else 1, path_index=min(16, paths.n_paths // 2))

    import paper_2403_04252_gb300 as w
    g = w.Basis(basis, device=local)
    ws_gb = args.workspace_gb or (16.0 if not c6 else 96.0)
    g.set_workspace_limit(int(ws_gb * (1 << 30)))
    g.set_solve_mode(SOLVE_MODES[args.solve_mode](w))
    n_paths = paths.n_paths if args.paths <= 0 else min(args.paths, paths.n_paths)
    N = g.N
    zg = paths.z[0]
    n_total = zg.size - 1
    b = paths.b[:n_paths]
    v = paths.v[:n_paths]
    if world > 1:
        # weak scaling: every rank takes n_paths impact parameters of a world-times finer scan of the
        # same range (no data-path collective: the paths are independent)
        from paper_2403_04252_gb300.dist import shard_impact_parameters
        b0, b1, _ = wi.CONFIGS[args.workload]["b"]
        b = shard_impact_parameters(b0, b1, n_paths, rank, world)
    STEP = args.rk4_per_step
    stream = torch.cuda.current_stream(dev)

    # the bench steps cover consecutive segments centred on closest approach (z = 0), where the
    # couplings are strongest; they wrap around if more steps are asked for than the path holds
    first = max(0, n_total // 2 - (args.warmup + args.steps) * STEP // 2)

    def segment(k: int):
        k0 = (first + k * STEP) % (n_total - STEP + 1)
        return zg[k0:k0 + STEP + 1]

    def reduce_max(x: float) -> float:
        from paper_2403_04252_gb300.dist import max_over_ranks
        return max_over_ranks(x, device=dev)

    def measure(form: int) -> dict:
        """warm-up, then the device-timed steps of one form; returns its rate and final amplitudes.
        Forms 0-5 are the precision modes; form 6 is mode 5 with four refinement sweeps per stage."""
        prec = 5 if form == 6 else form
        g.set_refine_iters(4 if form == 6 else 2)
        c = torch.zeros((n_paths, N), dtype=torch.complex128, device=dev)
        c[:, 0] = 1.0
        for k in range(args.warmup):
            g.propagate(b, v, segment(k), c=c, precision_mode=prec)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        g.profile_enable(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            g.propagate(b, v, segment(args.warmup + k), c=c, precision_mode=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = reduce_max(e0.elapsed_time(e1))
        prof = g.profile_read()
        g.profile_enable(False)
        if dist:
            dist.barrier()
        P = w.probabilities(c).cpu().numpy()
        g.set_refine_iters(2)
        return {"prec": form, "ms": ms, "value": world * n_paths * STEP * args.steps / (ms / 1e3),
                "prof": prof, "clocks": clocks, "P": P}

    names = {0: "fp64", 1: "mixed", 2: "mixed-fp64-elements", 3: "mixed-tensor-core", 4: "fp64-tensor-core",
             5: "mixed-fp64-tc-elements", 6: "fp64-tc-refined"}
    forms = {}
    if args.precision == "auto":
        forms[0] = measure(0)
        for prec in (4, 6, 1, 3, 5, 2):
            if prec == 2 and any(forms[p].get("err", 1.0) <= 1e-6 for p in forms if p != 0):
                break
            try:
                forms[prec] = measure(prec)
            except w.WpcccError as exc:      # e.g. a basis the tensor-core form does not take
                forms[prec] = {"prec": prec, "unsupported": str(exc)}
                continue
            forms[prec]["err"] = float(np.abs(forms[prec]["P"] - forms[0]["P"]).max())
    else:
        head = {v_: k for k, v_ in names.items()}[args.precision]
        forms[head] = measure(head)
        if head >= 1:
            ref = measure(0)
            forms[head]["err"] = float(np.abs(forms[head]["P"] - ref["P"]).max())
            forms[0] = ref

    # whole paths (untimed) of a stated subset of impact parameters: every form against the plain FP64 form
    whole = None
    if args.whole_path_paths > 0 and not c6 and world == 1:
        k = min(args.whole_path_paths, n_paths)
        idx = np.unique(np.linspace(0, n_paths - 1, k).round().astype(int))
        P_ref = None
        whole = {"paths": idx.tolist(), "b": [float(x) for x in b[idx]], "rk4_steps_per_path": int(n_total),
                 "forms": {}}
        for p in sorted(forms):
            if "unsupported" in forms[p]:
                continue
            prec = 5 if p == 6 else p
            g.set_refine_iters(4 if p == 6 else 2)
            P = w.probabilities(g.propagate(b[idx], v[idx], zg, precision_mode=prec)).cpu().numpy()
            g.set_refine_iters(2)
            if p == 0:
                P_ref = P
            e = float(np.abs(P - P_ref).max())
            forms[p]["whole_err"] = e
            whole["forms"][names[p]] = {
                "max_abs_prob_error_vs_fp64": e,
                "meets_fp64_bar": bool(np.all(np.abs(P - P_ref) <= 1e-10 * np.maximum(P_ref, 1e-4)))}
    if args.precision == "auto":
        ok = [p for p in forms if p == 0 or (forms[p].get("err", 1.0) <= 1e-6 and forms[p].get("whole_err", 0.0) <= 1e-6)]
        head = max(ok, key=lambda p: forms[p]["value"])
    H = forms[head]
    prec, ms, prof, clocks, value = H["prec"], H["ms"], H["prof"], H["clocks"], H["value"]
    mode = 5 if prec == 6 else prec          # the library's precision mode of the headline form
    g.set_refine_iters(4 if prec == 6 else 2)

    # ---- end to end through the public API with host buffers, headline form
    c_host = torch.zeros((n_paths, N), dtype=torch.complex128).pin_memory()
    c_host[:, 0] = 1.0
    P_host = torch.empty((n_paths, N), dtype=torch.float64).pin_memory()
    c_dev = torch.empty((n_paths, N), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        c_dev.copy_(c_host, non_blocking=True)
        g.propagate(b, v, segment(args.warmup + k), c=c_dev, precision_mode=mode)
        P = w.probabilities(c_dev)
        P_host.copy_(P, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0)
    seg_bytes = 8 * (STEP + 1) * n_paths + 8 * 2 * n_paths + 4 * n_paths  # z nodes, b, v, n_z
    h2d = c_host.numel() * 16 + seg_bytes
    d2h = P_host.numel() * 8

    # ---- roofline: every kernel category of the headline form against its bound; the dominant one
    # (largest device time) is the line's `roofline`
    NT, NP_, G = basis.T.N, basis.P.N, basis.quad.G
    n_half = int(sum(1 for m in basis.P.st_m if m >= 0))
    evals = args.steps * n_paths * (2 * STEP + 1)
    cats = _category_rooflines(basis, mode, args.solve_mode, N, n_half)
    cats["rk4"] = (_rk4_flops_per_step(mode, args.solve_mode, N, NT, NP_), ("alu", FP64_PEAK_TFLOPS, "TFLOP/s"),
                   "k_rk4")
    issued = {3: 10.0, 4: 28.0, 5: 28.0}.get(mode)

    def roof(key: str) -> dict:
        k_ms, k_launches = prof[key]
        per_unit, (bound, peak, unit), k_name = cats[key]
        units = n_paths * STEP * args.steps if key == "rk4" else evals
        work = per_unit * units
        ach = work / (k_ms / 1e3) / (1e9 if unit == "GB/s" else 1e12)
        per_pos = MEASURED_TRAFFIC_PER_POSITION.get((args.workload, k_name))
        r = {"bound": bound, "kernel": k_name, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
             "traffic": per_pos * evals / max(k_launches, 1) if (per_pos and key != "rk4") else None,
             "peak_source": _peak_source(bound, peak), "launch_ms_avg": k_ms / max(k_launches, 1),
             ("bytes_per_launch" if unit == "GB/s" else "flop_per_launch"): work / max(k_launches, 1),
             "work_per_unit": per_unit, "unit_of_work": "path-step" if key == "rk4" else "position"}
        if key == "mol_gemm" and issued:
            r["issued_bf16_tflops"] = issued * 8.0 * NT * n_half * G * evals / (k_ms / 1e3) / 1e12
            r["issued_note"] = (f"bf16 slice products issued ({int(issued)} per algorithmic product, q >= 0 "
                                "columns only)")
        return r

    timed = {k: prof[k][0] for k in cats if k in prof and prof[k][1] > 0}
    dom = max(timed, key=lambda k: timed[k])
    roofline = roof(dom)
    roofline["by_kernel"] = {k: {kk: vv for kk, vv in roof(k).items() if kk in ("kernel", "bound", "achieved",
                                                                                   "peak", "unit", "frac",
                                                                                   "launch_ms_avg")}
                             | {"ms": timed[k], "share": timed[k] / sum(timed.values())} for k in timed}
    roofline["streams"] = ("RK4 sweeps run on a second stream, overlapping the next chunk's element kernels and "
                           "factorisation on the caller's stream; shares are of the summed kernel time")
    total_flops = (cats["mol_gemm"][0] + cats["solve"][0]) * evals + cats["rk4"][0] * n_paths * STEP * args.steps
    launches = int(sum(n for _, n in prof.values()))
    form_desc = {0: "plain FP64, all paths batched; S^-1 applied "
                    + {"stage": "per RK4 stage from LU factors",
                       "schur": "per RK4 stage through the Cholesky factor of the Schur complement I - K^+ K",
                       "matrix": "as X = S^-1 H with N right-hand sides (the paper's ZGESV form)"}[args.solve_mode],
                 1: "mixed precision: Eq. 9 contraction and the factors of S on the FP32 pipe, FP64 "
                    "node tables, refinement and RK4; all paths batched",
                 2: "mixed precision with FP64 elements: factors of S on the FP32 pipe, FP64 refinement and RK4",
                 3: "mixed precision, tensor-core contraction: Eq. 9 on tcgen05 (four fixed-point bf16 slices, ten "
                    "slice products into exact FP32 accumulators), FP32 factors of S, FP64 refinement and RK4; all "
                    "paths batched",
                 4: "FP64-accurate: Eq. 9 contraction emulated on tcgen05 (seven bf16 slices per operand, 28 "
                    "slice products, exact level accumulators, double-float sums), FP64 solve and RK4",
                 5: "mixed precision with FP64-accurate tensor-core elements: FP32 factors of S, FP64 refinement "
                    "and RK4",
                 6: "FP64-accurate, refined: tensor-core elements to FP64 accuracy, FP32 factors of S as the "
                    "preconditioner of four FP64 refinement sweeps per RK4 stage, FP64 RK4"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 3: "bf16x4-slices+f32+f64", 4: "bf16-slices(fp64-accurate)+f64",
                      5: "bf16-slices(fp64-accurate)+f32+f64",
                      6: "bf16-slices(fp64-accurate)+f32+f64"}.get(prec, "f32+f64"), "data": "synthetic",
            "config": {"workload": CONFIG_DESC if not c6 else CONFIG_DESC_C6, "paths": n_paths,
                       "form": form_desc[prec],
                       "bench_step": f"{STEP} RK4 steps of each of the {n_paths} paths per rank, consecutive "
                                     "segments centred on z = 0",
                       "l2": "inputs larger than L2: S and H of one step are "
                             f"{2 * 16 * N * N * n_paths * (2 * STEP + 1) / 1e9:.1f} GB"},
            "forms": {names[p]: ({"value": f["value"], "ms_per_step": f["ms"] / args.steps,
                                  "max_abs_prob_error_vs_fp64": f.get("err", 0.0),
                                  **({"whole_path_max_abs_prob_error_vs_fp64": f["whole_err"]}
                                     if "whole_err" in f else {}),
                                  "kernel_ms": {k: v_[0] for k, v_ in f["prof"].items()}}
                                 if "unsupported" not in f else {"unsupported": f["unsupported"]})
                      for p, f in forms.items()},
            "speedup_vs_plain_fp64": value / forms[0]["value"],
            "fp64_accurate_forms": {
                "bar": "max |dP| <= 1e-10 max(P, 1e-4) against the plain FP64 form on the same steps",
                **{names[p]: {"value": forms[p]["value"], "speedup_vs_plain_fp64": forms[p]["value"] / forms[0]["value"],
                              "max_abs_prob_error_vs_fp64": forms[p].get("err", 0.0),
                              "meets_fp64_bar": bool(np.all(np.abs(forms[p]["P"] - forms[0]["P"])
                                                            <= 1e-10 * np.maximum(forms[0]["P"], 1e-4)))}
                   for p in (0, 4, 6) if p in forms and "unsupported" not in forms[p]}},
            "prob_error": {"max_abs": H.get("err", 0.0), "bound": 1e-6,
                           "against": "the plain FP64 form on the same steps (itself within 1e-10 of the oracle)",
                           "rk4_steps_per_path": (args.warmup + args.steps) * STEP,
                           **({"whole_path_max_abs": H.get("whole_err", 0.0)} if whole else {})},
            "whole_path_check": whole,
            "roofline": roofline,
            "algorithmic_tflops_whole_step": total_flops / (ms / 1e3) / 1e12,
            "matrix_elements_per_s": world * evals * (NT * NT + NP_ * NP_ + 3 * NT * NP_) / (ms / 1e3),
            "kernel_ms": {k: v_[0] for k, v_ in prof.items()},
            "e2e": {"value": world * n_paths * STEP * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    g.close()
    return line


_SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "forms", "speedup_vs_plain_fp64",
             "fp64_accurate_forms", "prob_error", "whole_path_check", "roofline", "e2e", "cpu_baseline", "clocks",
             "kernel_ms", "kernel_ms_separate_calls", "batched_vs_separate_calls", "autotune", "gpu_launches")


def _sub_entry(line: dict) -> dict:
    return {k: line[k] for k in _SUB_KEYS if k in line}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", type=int, default=0, help="use only the first P paths (0: all of the workload)")
    ap.add_argument("--rk4-per-step", type=int, default=STEP_RK4)
    ap.add_argument("--solve-mode", default="auto", choices=["auto", "stage", "matrix", "schur"],
                    help="S^-1 per RK4 stage through the Schur complement's Cholesky factor (schur), from pivoted LU "
                         "factors (stage), or as X = S^-1 H (matrix); auto = schur (the Cholesky factor needs a "
                         "positive-definite S, i.e. the workloads' converged (eta, tau) rules)")
    ap.add_argument("--workload", default=None, choices=["p_H_2c_n4l3", "C6_H_2c_n6l5", "p_H_2c_batch6v",
                                                         "pLi_2c_grad", "p_H_1c_n10l10"],
                    help="run one workload only.  Default: the p + H headline (p_H_2c_n4l3: two-centre p + H, "
                         "N = 380, 32 paths) with the batched velocity scan (p_H_2c_batch6v: six speeds, "
                         "N = 316..572, 64 paths each, one graph launch) and the precision workload "
                         "(C6_H_2c_n6l5: bare C6+ on H, N = 1622, 16 paths) carried in `workloads`; "
                         "pLi_2c_grad: p + Li-like model-potential target (N = 379, 32 paths), observables and "
                         "their gradient by the adjoint; p_H_1c_n10l10: one-centre p + H at l <= 10 (N = 4257)")
    ap.add_argument("--no-sub-workloads", action="store_true",
                    help="default run: skip the velocity-scan and C6+ entries")
    ap.add_argument("--whole-path-paths", type=int, default=4,
                    help="p + H: impact parameters (evenly spread, the smallest included) whose whole 1000-step "
                         "paths every form runs untimed, against the plain FP64 form; 0 skips the check")
    ap.add_argument("--checkpoint-every", type=int, default=25, help="pLi_2c_grad: RK4 steps per checkpoint")
    ap.add_argument("--no-fd-check", action="store_true", help="pLi_2c_grad: skip the central-difference sample")
    ap.add_argument("--workspace-gb", type=float, default=0.0, help="0: 16 GB (p + H) or 96 GB (C6+ on H)")
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "fp64", "mixed", "mixed-fp64-elements", "mixed-tensor-core", "fp64-tensor-core",
                             "mixed-fp64-tc-elements", "fp64-tc-refined"],
                    help="auto: time plain FP64 and the reduced-precision forms, report the fastest form whose "
                         "probabilities stay within 1e-6 of the FP64 form on the same steps")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.solve_mode == "auto":
        args.solve_mode = "schur"
    if args.impl == "reference":
        args.workload = args.workload or WORKLOAD
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "p_H_2c_batch6v":
        line = run_batch(args)
    elif args.workload == "pLi_2c_grad":
        run_grad(args)
        return
    elif args.workload == "p_H_1c_n10l10":
        run_one_centre_large(args)
        return
    elif args.workload is not None:
        line = run_fixed_speed(args)
    else:
        args.workload = WORKLOAD
        line = run_fixed_speed(args)
        if world == 1 and not args.no_sub_workloads:
            # the batched and precision workloads of the metric, each with its own forms, errors, roofline,
            # end-to-end rate and CPU baseline; a few bench steps each, so the whole run stays within minutes
            import copy
            sub = {}
            a = copy.copy(args)
            a.workload, a.steps, a.warmup, a.rk4_per_step = "p_H_2c_batch6v", min(args.steps, 3), 3, STEP_RK4
            sub["p_H_2c_batch6v"] = _sub_entry(run_batch(a))
            a = copy.copy(args)
            a.workload, a.steps, a.warmup, a.rk4_per_step = "C6_H_2c_n6l5", min(args.steps, 2), 3, STEP_RK4
            a.whole_path_paths = 0
            sub["C6_H_2c_n6l5"] = _sub_entry(run_fixed_speed(a, sub=True))
            line["workloads"] = sub
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
