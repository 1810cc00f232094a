"""Benchmark of the Riccati sweep: trajectory-steps/s, FP32 batched against
the plain FP64 sweep on the same grains.

One step = one pass of the whole hot path over the workload: rotate Delta and
A onto the lattices, the Riccati sweep (all angle pairs, lines and Matsubara
energies, propagator and energy sums fused), rotate-back with the
Fermi-surface average, then gap update, current and free energy.  Boundary
values carry over from step to step (Delta and A frozen: burn-in sweeps).

Default workload (c3): 64 seeded grains, discs and random convex polygons of
radius 10-40 xi0 at grid spacing 0.2 xi0, s or d_{x2-y2} pairing, t uniform in
[0.05, 0.8] with the Matsubara cutoff 16 pi kB Tc (10-160 energies), 0-5 flux
quanta, 64-256 Fermi angles; Delta = bulk guess x (1 + 0.05 Z).  The line also
carries the plain FP64 batch on the same grains (`fp64_plain`), the C-ABI
end-to-end step with host buffers (`e2e`) and the errors of four grains
against the FP64 oracle.

Other workloads: c2 (d_{x2-y2} square rotated by 45 deg, side 50 xi0, 256^2,
128 angles, t = 0.1, 80 energies, 0.5 flux quanta, kappa = 80), c4, c5,
annulus (--workload).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c4|c5|annulus]
    python bench.py --impl reference      # the FP64 CPU oracle on this host
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2205_15000_b300 import ranks  # noqa: E402
from paper_2205_15000_b300 import workloads as W  # noqa: E402

METRIC = "Riccati trajectory-steps/s"
WORKLOAD = "c2_diamond_dx2y2_256sq_128ang_80eps"
# algorithmic FP32 lane-operations of the sweep per (angle pair, sample, energy):
# two closed-form steps (coefficients gamma_h, E, K: 34; application of the
# Moebius map: 18) and one propagator/energy-sum evaluation (21), with the terms
# that depend only on the segment (Delta, the Doppler shift, its length) shared by
# the energies and not counted; MUFU operations counted separately (15)
ALG_FP32_OPS_PER_PSE = 2 * (34 + 18) + 21
ALG_MUFU_OPS_PER_PSE = 2 * 7 + 1
# the implicit midpoint stepper: a quadratic per step (41 FP32 ops, 3 MUFU; ell zr
# shared by the energies) with the same propagator evaluation
ALG_OPS_PER_PSE = {"closed": ALG_FP32_OPS_PER_PSE, "midpoint": 2 * 41 + 21}
# the adjoint sweep (closed-form step) per (angle pair, sample, energy), counted the
# same way from its arithmetic: pass 1 one step (34 + 18); pass 2 the forward
# segment's Moebius coefficients (40), their mirror for beta (17), beta's step (20),
# the step derivatives (112), the coefficient cotangents (19) and the propagator
# cotangents at the sample (80); pass 3 beta's coefficients (40), derivatives (112)
# and cotangents (21); 23 MUFU operations
ALG_ADJ_OPS_PER_PSE = (34 + 18) + (40 + 17 + 20 + 112 + 19 + 80) + (40 + 112 + 21)
SM_COUNT_B300 = 148
FP32_LANES_PER_SM = 128
# FP64 pipe: ncu reports sm__inst_executed_pipe_fp64 peak 0.0625 warp instructions
# per cycle per SM on B300, i.e. 2 lanes per cycle per SM
FP64_LANES_PER_SM = 2


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries) every 2 ms by a thread that runs exactly while
    the timed steps run.  Falls back to the nvidia-smi sampler when NVML cannot be
    opened."""

    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
               "sw_power_cap": 0x4, "hw_power_brake_slowdown": 0x80}
    NVML_CLOCK_SM = 1

    def __init__(self, device_index, smi_path):
        import ctypes
        import threading
        self.samples, self.reasons, self.smax = [], set(), None
        self.stop_flag = threading.Event()
        self.thread = None
        self.smi = None
        self.smi_path, self.index = smi_path, device_index
        try:
            import torch
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit")
            want = str(torch.cuda.get_device_properties(device_index).uuid)
            want = want if want.startswith("GPU-") else "GPU-" + want
            n = ctypes.c_uint(0)
            nv.nvmlDeviceGetCount_v2(ctypes.byref(n))
            handle = None
            for i in range(n.value):
                h = ctypes.c_void_p()
                if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(i), ctypes.byref(h)) != 0:
                    continue
                buf = ctypes.create_string_buffer(96)
                if nv.nvmlDeviceGetUUID(h, buf, ctypes.c_uint(96)) == 0 and buf.value.decode() == want:
                    handle = h
                    break
            if handle is None:
                raise RuntimeError("no NVML device with the CUDA device's UUID")
            clk = ctypes.c_uint(0)
            if nv.nvmlDeviceGetMaxClockInfo(handle, ctypes.c_int(self.NVML_CLOCK_SM), ctypes.byref(clk)) != 0:
                raise RuntimeError("nvmlDeviceGetMaxClockInfo")
            self.smax = float(clk.value)
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.nvml, self.h = nv, handle
        except Exception:
            self.nvml = None
            self.smi = _sample_clocks_start(smi_path)

    def _run(self):
        import ctypes
        nv, h = self.nvml, self.h
        clk, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self.stop_flag.is_set():
            if nv.nvmlDeviceGetClockInfo(h, ctypes.c_int(self.NVML_CLOCK_SM), ctypes.byref(clk)) == 0:
                self.samples.append(float(clk.value))
            if self.reason_fn(h, ctypes.byref(r)) == 0:
                for name, bit in self.REASONS.items():
                    if r.value & bit:
                        self.reasons.add(name)
            self.stop_flag.wait(0.002)

    def start(self):
        if self.nvml is not None:
            import threading
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()
        return self

    def stop(self):
        if self.nvml is None:
            return _sample_clocks_stop(*(self.smi or (None, None)), self.smi_path, self.index)
        self.stop_flag.set()
        if self.thread is not None:
            self.thread.join(timeout=5)
        if not self.samples:
            return None
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.smax,
                "reasons": sorted(self.reasons), "samples": len(self.samples),
                "source": "NVML every 2 ms during the timed steps"}


def _sample_clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def _sample_clocks_stop(proc, f, path, device_index=0):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    except Exception:
        return None
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def _measured_fma_peak():
    """The library's measured FP32 lane-FMA rate (packed and scalar chains, the larger;
    Gop/s), taken after the timed steps; None when it cannot be measured."""
    from paper_2205_15000_b300 import sc
    try:
        return max(sc.sc_debug_fma_rate(True), sc.sc_debug_fma_rate(False)) / 1e9
    except Exception:
        return None


def _profiled_traffic(workload, precision, fused=False):
    """DRAM bytes (read + write) of the dominant kernel per sweep from the ncu
    capture recorded in profiles/sweep_traffic.json for this workload,
    precision and batch layout (sweep launches with or without the lattice
    transfers as work items), or None when no capture of the current build is
    recorded."""
    try:
        with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as f:
            entries = json.load(f)
    except Exception:
        return None
    for tr in entries if isinstance(entries, list) else [entries]:
        if tr.get("precision") == precision and tr.get("workload") == workload and \
                bool(tr.get("fused_transfers", False)) == bool(fused):
            return tr.get("dram_bytes_per_sweep", tr.get("dram_bytes_per_launch"))
    return None


def cpu_oracle_sample(p, delta, aind, n_sweeps=1, angle_subset=16, keep=None):
    """The FP64 oracle on this host: the same grain and energies with a subset
    of the Fermi angles (a bounded sample); returns steps/s and details.  With
    `keep` (a dict), the last sweep's outputs and the mask are stored in it."""
    import oracle
    q = dict(p)
    q["n_angles"] = angle_subset
    g = oracle.OracleGeom(q)
    # steps of the sample: n_e * sum over pairs and lines of 2 (n_samples + 1)
    L = g.lines()
    ns = np.maximum(L["m1"] - L["m0"] + 1, 0)
    steps = q["n_energies"] * int(np.sum(2 * (ns + 1)))
    ex = None
    t0 = time.perf_counter()
    for _ in range(n_sweeps):
        o = g.full_sweep(delta, aind, ex)
        ex = o["exit"]
    dt = time.perf_counter() - t0
    if keep is not None:
        keep["out"] = o
        keep["mask"] = g.mask().astype(bool)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": steps * n_sweeps / dt, "unit": "trajectory-steps/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{n_sweeps} FP64 sweep(s) of the same grain and {q['n_energies']} energies with "
                      f"{angle_subset} of {p['n_angles']} Fermi angles ({steps} steps per sweep), {dt:.2f} s"}


def _errors_vs_oracle(p, delta, precision, keep, n_sweeps=2):
    """Max-norm errors of Delta_new, j and F(R) (relative to the oracle's max over
    the grain) after n_sweeps sweeps from fresh boundary values, the library in
    `precision` against the FP64 oracle on the same inputs."""
    from paper_2205_15000_b300 import sc
    ctx = sc.Context(p, precision=precision)
    ctx.set_fields(delta)
    for _ in range(n_sweeps):
        ctx.sweep()
    r = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ctx.outputs().items()}
    o, m = keep["out"], keep["mask"]

    def rel(a, b):
        return float(np.max(np.abs(a[m] - b[m])) / max(np.max(np.abs(b[m])), 1e-300))
    return {"delta_new": rel(r["delta_new"], o["delta_new"]), "j": rel(r["j"], o["j"]),
            "F": rel(r["F"], o["F"]),
            "F_total": abs(r["F_total"] - o["F_total"]) / abs(o["F_total"]),
            "tolerance": {"delta_new": 1e-5, "j": 1e-4, "F": 1e-4},
            "norm": f"max over the grain, relative to the oracle's max; {n_sweeps} sweep(s) from fresh boundary values"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, delta, aind = W.c2_diamond_d()
    vals, secs = [], []
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_oracle_sample(p, delta, aind, 1, 16)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(dt)
            cb = r
    v = float(statistics.mean(vals))
    # a step of this arm is one bounded sample of the workload (16 of the 128 angles)
    line = {"metric": METRIC, "value": v, "unit": "trajectory-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(statistics.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": cb["sample"],
                       "step": "one bounded sample (one FP64 oracle sweep over 16 of the 128 angles)"},
            "cpu_baseline": {"value": v, "unit": "trajectory-steps/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2205_15000_b300 import sc

    world, rank, local = ranks.env_ranks()
    torch.cuda.set_device(local)
    dist = ranks.init("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    if args.workload == "c4":
        p, delta, aind = W.c4_disc_d()
        workload = "c4_disc_d_128sq_64ang_40eps_vortex"
    elif args.workload == "c5":
        p, delta, aind = W.c5_square_d()
        workload = "c5_square_d_1024sq_256ang_160eps_20vortices"
    elif args.workload == "annulus":
        p, delta, aind = W.annulus_d()
        workload = "annulus_dx2y2_R25_r10_256sq_128ang_80eps_solenoid"
    else:
        p, delta, aind = W.c2_diamond_d(n=args.grid, n_angles=args.angles)
        workload = WORKLOAD if (args.grid, args.angles) == (256, 128) else \
            f"c2_reduced_{args.grid}sq_{args.angles}ang_80eps"
    p["stepper"] = args.stepper
    if args.adjoint_checkpoint:  # adjoint: forward gamma kept every k samples and recomputed
        p["adjoint_checkpoint"] = args.adjoint_checkpoint
        workload += f"_ckpt{args.adjoint_checkpoint}"
    if args.energies:  # another energy count on the same grain (profiling the wide layouts)
        p["n_energies"] = args.energies
        workload += f"_{args.energies}eps"
    if args.lanes:  # a fixed lane layout (profiling a small case in the layout of a large one)
        workload += f"_lanes{args.lanes}"
    if args.energy_sum == "ozaki":
        # Ozaki's poles up to the same energy cutoff (eps_c = 16 pi kB Tc)
        p["energy_sum"] = "ozaki"
        p["n_energies"] = W.ozaki_poles_for_cutoff(p["t"])
        workload += f"_ozaki{p['n_energies']}"
    ctx = sc.Context(p, precision=args.precision, lanes_per_line=args.lanes, record_timings=True)
    info = ctx.info
    stream = torch.cuda.current_stream()
    d_delta = torch.view_as_real(torch.as_tensor(delta, dtype=torch.complex128)).contiguous().to(dev)
    sc.sc_set_fields(ctx.h, d_delta, None, True, stream)
    dn = torch.empty((p["ny"], p["nx"], 2), dtype=torch.float64, device=dev)
    jj = torch.empty_like(dn)
    FF = torch.empty((p["ny"], p["nx"]), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    gd = torch.empty((p["ny"], p["nx"], 2), dtype=torch.float64, device=dev)
    ga = torch.empty_like(gd)

    def step():
        sc.sc_riccati_sweep(ctx.h, stream)
        sc.sc_gap_update(ctx.h, dn, True, False, stream)
        sc.sc_current(ctx.h, jj, True, stream)
        sc.sc_free_energy(ctx.h, FF, True, False, stream)
        if args.adjoint:  # gradient of F_total with respect to Delta(R) and A_ind(R)
            sc.sc_sweep_adjoint(ctx.h, None, None, None, 1.0, gd, ga, True, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ranks.barrier(dist)
    torch.cuda.synchronize()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_r{rank}_{os.getpid()}.csv")
    sampler = ClockSampler(local, clk_path) if rank == 0 else None
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern = []  # per timed step: (rotate, sweep, rotate_back) from the library's events
    if sampler:
        sampler.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
        ki = sc.sc_get_info(ctx.h)  # waits for this step's sweep kernels
        kern.append((ki.ms_rotate, ki.ms_sweep, ki.ms_rotate_back, ki.ms_adjoint))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    sweep_ms = statistics.mean(k[1] for k in kern)
    kernels_ms = {"rotate": statistics.mean(k[0] for k in kern), "sweep": sweep_ms,
                  "rotate_back": statistics.mean(k[2] for k in kern)}
    if args.adjoint:
        kernels_ms["adjoint_sweep"] = statistics.mean(k[3] for k in kern)
    clocks = sampler.stop() if sampler else None

    # end to end through the public API with host buffers: every step copies its
    # input Delta from pinned host memory and reads Delta_new, j and F back into
    # pinned host memory.  Uploads and read-backs run on two more streams through
    # double-buffered device staging, so that step i+1's upload and step i-1's
    # read-back overlap step i's sweep; L2 is flushed at the start of every step,
    # inside the timed region.
    pin_delta = torch.view_as_real(torch.as_tensor(delta, dtype=torch.complex128)).contiguous().pin_memory()
    h_out = [[torch.empty((p["ny"], p["nx"], 2), dtype=torch.float64).pin_memory(),
              torch.empty((p["ny"], p["nx"], 2), dtype=torch.float64).pin_memory(),
              torch.empty((p["ny"], p["nx"]), dtype=torch.float64).pin_memory()] for _ in range(2)]
    d_in = [torch.empty_like(pin_delta, device=dev) for _ in range(2)]
    d_out = [[torch.empty_like(h, device=dev) for h in h_out[0]] for _ in range(2)]
    cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()
    e2e_ms = []
    e2e_enqueue_ms = None
    n_e2e = max(5, min(args.steps, 20)) if not args.no_e2e else 0
    if n_e2e:
        def e2e_steps(n_steps):
            ev_in = [torch.cuda.Event() for _ in range(n_steps)]
            ev_used = [torch.cuda.Event() for _ in range(n_steps)]
            ev_out = [torch.cuda.Event() for _ in range(n_steps)]
            ev_read = [torch.cuda.Event() for _ in range(n_steps)]
            for i in range(n_steps):
                b = i % 2
                with torch.cuda.stream(cs_in):
                    if i >= 2:
                        cs_in.wait_event(ev_used[i - 2])  # the buffer's previous upload was consumed
                    d_in[b].copy_(pin_delta, non_blocking=True)
                    ev_in[i].record(cs_in)
                stream.wait_event(ev_in[i])
                if i >= 2:
                    stream.wait_event(ev_read[i - 2])    # the output buffers were read back
                flush.fill_(float(i))
                sc.sc_set_fields(ctx.h, d_in[b], None, True, stream)
                ev_used[i].record(stream)
                sc.sc_riccati_sweep(ctx.h, stream)
                sc.sc_gap_update(ctx.h, d_out[b][0], True, False, stream)
                sc.sc_current(ctx.h, d_out[b][1], True, stream)
                sc.sc_free_energy(ctx.h, d_out[b][2], True, False, stream)
                ev_out[i].record(stream)
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(ev_out[i])
                    for h_, d_ in zip(h_out[b], d_out[b]):
                        h_.copy_(d_, non_blocking=True)
                    ev_read[i].record(cs_out)
            t_enq = time.perf_counter()
            torch.cuda.synchronize()
            return t_enq

        e2e_steps(3)  # untimed: the copy stream's and the pinned buffers' first use
        t0 = time.perf_counter()
        t_enq = e2e_steps(n_e2e)
        e2e_ms = [(time.perf_counter() - t0) * 1e3 / n_e2e]
        e2e_enqueue_ms = (t_enq - t0) * 1e3 / n_e2e
    h2d = pin_delta.numel() * 8
    d2h = sum(h.numel() for h in h_out[0]) * 8

    # loop glue outside the timed step: the induced vector potential (App. D) from
    # the last current, zero-padded FFT convolution on the device
    vp_ms = None
    if p["kappa"] > 0 and math.isfinite(p["kappa"]):
        vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(6)]
        for a_, b_ in vev:
            a_.record(stream)
            sc.sc_update_vector_potential(ctx.h, stream)
            b_.record(stream)
        torch.cuda.synchronize()
        vp_ms = statistics.median(a_.elapsed_time(b_) for a_, b_ in vev[1:])

    steps_per_step = info.steps_per_sweep
    total_ms_max = ranks.max_over_ranks(dist, total_ms, dev)
    ranks.barrier(dist)
    value = ranks.throughput(steps_per_step * args.steps, world, total_ms_max * 1e-3)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peaks = _measured_peaks()
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0)
    # issue roofline of the arithmetic pipe the sweep runs on: 148 SMs x lanes per
    # cycle (FP32: 128; FP64: 2) x max SM clock
    lanes = FP32_LANES_PER_SM if args.precision == "fp32" else FP64_LANES_PER_SM
    peak_gops = SM_COUNT_B300 * lanes * sm_max * 1e6 / 1e9
    peak_note = ("FP32 lane issue 148 SM x 128 x max SM clock (derived)" if args.precision == "fp32" else
                 "FP64 pipe 148 SM x 2 lanes/cycle (ncu pipe peak) x max SM clock (derived); the IEEE "
                 "division, square root, exp and sin/cos sequences run on the same pipe")
    pse = info.points_per_sweep // 2  # (pair, sample, energy) combinations per sweep
    # the same arithmetic in either precision (transcendentals not counted)
    ops = pse * ALG_OPS_PER_PSE[args.stepper]
    achieved = ops / (sweep_ms * 1e-3) / 1e9
    traffic = _profiled_traffic(workload, args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": "trajectory-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": workload, "grid": [p["nx"], p["ny"]], "n_angles": p["n_angles"],
                   "n_energies": p["n_energies"], "t": p["t"], "pairing": "dx2y2",
                   "flux_quanta": p["flux_quanta"], "precision": args.precision, "stepper": args.stepper,
                   "energy_sum": args.energy_sum,
                   "steps_per_sweep": steps_per_step, "l2": "flushed between timed steps",
                   "parallelism": f"replicas{world}",
                   "step": "forward sweep + outputs" + (" + adjoint of F_total" if args.adjoint else ""),
                   "grain": dict({k: p[k] for k in ("nx", "ny", "h", "t", "n_angles", "n_energies",
                                                    "flux_quanta", "pairing")},
                                 gauge=p.get("gauge", "symmetric"), parts=len(p.get("parts") or []))},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": traffic,
                     "kernel": "sweep_kernel", "ms_per_launch": sweep_ms,
                     "kernels_ms_per_step": kernels_ms, "peak_note": peak_note,
                     "ops_per_unit": f"{ALG_OPS_PER_PSE[args.stepper]} lane-operations per (angle pair, sample, "
                                     "energy), the optimised formulation, terms that depend only on the segment "
                                     "excluded"},
        "e2e": ({"value": steps_per_step / (statistics.median(e2e_ms) * 1e-3),
                 "unit": "trajectory-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "ms_per_step": statistics.median(e2e_ms), "host_enqueue_ms_per_step": e2e_enqueue_ms}
                if e2e_ms else None),
        # per step: (FP32: field conversion,) rotate, sweep, rotate-back, outputs;
        # adjoint: output cotangents, transposed rotate-back, adjoint sweep, transposed rotate
        # a step: (FP32: field conversion,) rotate, sweep, (energy-block sums,)
        # rotate-back, outputs and their final sums; the adjoint's launches on top
        "gpu_launches": ((6 if args.precision == "fp32" else 5) + (1 if p["n_energies"] > 32 * 8 else 0)
                         + (4 if args.adjoint else 0)) * args.steps,
        "loop_glue": ({"vector_potential_ms": vp_ms, "method": "zero-padded FFT convolution, FP64",
                       "outside_timed_region": True} if vp_ms is not None else None),
        "clocks": clocks,
        "wall_s": t_wall,
    }
    if args.precision == "fp32":
        pm = _measured_fma_peak()
        if pm:
            line["roofline"]["peak_measured"] = pm
            line["roofline"]["frac_of_measured"] = achieved / pm
            line["roofline"]["peak_measured_note"] = ("sc_debug_fma_rate after the timed steps: 8 blocks of 256 "
                                                      "threads per SM, 8 independent FMA chains per thread")
    if args.adjoint and args.stepper == "closed":
        adj_ms = kernels_ms["adjoint_sweep"]
        adj_ach = pse * ALG_ADJ_OPS_PER_PSE / (adj_ms * 1e-3) / 1e9
        line["roofline_adjoint"] = {
            "bound": "alu", "achieved": adj_ach, "peak": peak_gops, "unit": "Gop/s", "frac": adj_ach / peak_gops,
            "kernel": "adjoint_sweep_kernel", "ms_per_launch": adj_ms, "over_forward_sweep": adj_ms / sweep_ms,
            "ops_per_unit": f"{ALG_ADJ_OPS_PER_PSE} lane-operations per (angle pair, sample, energy): three "
                            "passes, counted like the sweep's"}
    if not args.no_cpu_baseline and (args.workload in ("c2", "annulus") or args.errors):
        # the large grain: one full oracle sweep (minutes on the host cores), opt-in
        n_sw = 1 if args.workload == "c5" else 2
        keep = {}
        line["cpu_baseline"] = cpu_oracle_sample(p, delta, aind, n_sw, p["n_angles"], keep)
        line["errors_vs_fp64_oracle"] = _errors_vs_oracle(p, delta, args.precision, keep, n_sw)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _c3_members_for_errors(grains, steps):
    """Members whose outputs are compared with the oracle: the smallest and the
    largest by trajectory-steps per sweep, then the s-wave and the d-wave member
    nearest the median size among the rest (discs and polygons both occur)."""
    order = sorted(range(len(grains)), key=lambda i: steps[i])
    pick = [order[0], order[-1]]
    med = steps[order[len(order) // 2]]
    for pairing in (0, 1):
        rest = [i for i in order if i not in pick and grains[i][0]["pairing"] == pairing]
        if rest:
            pick.append(min(rest, key=lambda i: abs(steps[i] - med)))
    return pick


def _c3_reference_members(grains, steps):
    """The bounded sample one step of the reference arm sweeps: the members at
    the 1/8, 3/8 and 5/8 points of the size order (about 2e8 trajectory-steps)."""
    order = sorted(range(len(grains)), key=lambda i: steps[i])
    n = len(order)
    return [order[n // 8], order[(3 * n) // 8], order[(5 * n) // 8]]


def _oracle_steps(p):
    import oracle
    L = oracle.OracleGeom(p).lines()
    ns = np.maximum(L["m1"] - L["m0"] + 1, 0)
    return p["n_energies"] * int(np.sum(2 * (ns + 1)))


def _member_outputs(m):
    o = m.outputs()
    return {"delta_new": o["delta_new"].cpu().numpy(), "j": o["j"].cpu().numpy(),
            "F": o["F"].cpu().numpy(), "F_total": o["F_total"]}


def _rel_errors(r, o, m):
    def rel(a, b):
        return float(np.max(np.abs(a[m] - b[m])) / max(np.max(np.abs(b[m])), 1e-300))
    return {"delta_new": rel(r["delta_new"], o["delta_new"]), "j": rel(r["j"], o["j"]),
            "F": rel(r["F"], o["F"]), "F_total": abs(r["F_total"] - o["F_total"]) / abs(o["F_total"])}


def run_reference_batch(args):
    """Reference arm on the batched workload: each step is one FP64 oracle sweep
    (with outputs) of a fixed bounded sample of the 64 grains."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    grains = W.c3_batch(n_grains=args.grains, seed=3)
    steps = [_oracle_steps(p) for p, _, _ in grains]
    sub = _c3_reference_members(grains, steps)
    geoms = [oracle.OracleGeom(grains[i][0]) for i in sub]
    n_steps = sum(steps[i] for i in sub)
    secs = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for g, i in zip(geoms, sub):
            g.full_sweep(grains[i][1], None, None)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            secs.append(dt)
    v = n_steps * len(secs) / sum(secs)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"one FP64 oracle sweep with outputs of grains {sub} of the {args.grains} "
              f"({n_steps} trajectory-steps, {statistics.mean(secs):.2f} s)")
    line = {"metric": METRIC, "value": v, "unit": "trajectory-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(statistics.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"c3_batch_{args.grains}_grains", "sample": sample,
                       "step": "one bounded sample of the batched workload (3 of its grains)"},
            "cpu_baseline": {"value": v, "unit": "trajectory-steps/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """The batched form: 64 seeded grains (discs and convex polygons, radius
    10-40 xi0, h = 0.2, s/d pairing, t in [0.05, 0.8], 0-5 flux quanta, 64-256
    angles) swept by persistent launches fed by one work list, iterations
    replayed as captured CUDA graphs; every member's gap update, current and
    free energy included in a step.  Beside the FP32 batch: the plain FP64
    batch on the same grains, the C-ABI end-to-end step with host buffers, and
    the errors of four members against the FP64 oracle."""
    import torch
    from paper_2205_15000_b300 import sc

    world, rank, local = ranks.env_ranks()
    torch.cuda.set_device(local)
    dist = ranks.init("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    grains = W.c3_batch(n_grains=args.grains, seed=3 + rank)
    for p, _, _ in grains:
        p["stepper"] = args.stepper
        if args.energy_sum == "ozaki":
            p["energy_sum"] = "ozaki"
            p["n_energies"] = W.ozaki_poles_for_cutoff(p["t"])
    workload = f"c3_batch_{args.grains}_grains" + ("" if args.stepper == "closed" else f"_{args.stepper}") + \
        ("" if args.energy_sum == "matsubara" else "_ozaki")
    stream = torch.cuda.current_stream()
    want_oracle = not args.no_cpu_baseline and rank == 0

    b = sc.Batch([p for p, _, _ in grains], precision=args.precision, energies_per_lane=args.ept)
    for (p, d, _), m in zip(grains, b.members):
        m.set_fields(d)
    msteps = [m.info.steps_per_sweep for m in b.members]
    check = _c3_members_for_errors(grains, msteps)
    ept = b.autotune(stream) if not args.ept else args.ept
    if args.transfers != "auto":
        b.set_fused_transfers(args.transfers == "fused")
    # outputs of the checked members after two sweeps from fresh boundary values,
    # in the layout that is timed
    got = {}
    if want_oracle:
        b.reset_boundary()
        b.run(2, True, stream)
        torch.cuda.synchronize()
        got[args.precision] = {i: _member_outputs(b.members[i]) for i in check}
    b.run(args.warmup, True, stream)
    torch.cuda.synchronize()
    info = b.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ranks.barrier(dist)
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_r{rank}_{os.getpid()}.csv")
    sampler = ClockSampler(local, clk_path) if rank == 0 else None
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ksweep = []
    if sampler:
        sampler.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        b.run(1, True, stream)
        ev[i][1].record(stream)
        flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
        ksweep.append(b.info().ms_sweep)  # waits for this step's sweep launches
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop() if sampler else None
    total_ms = ranks.max_over_ranks(dist, float(sum(a.elapsed_time(c) for a, c in ev)), dev)
    value = ranks.throughput(info.steps_per_sweep * args.steps, world, total_ms * 1e-3)
    sweep_ms = statistics.mean(ksweep)

    # end to end through the public API with host buffers: every step uploads all
    # members' Delta from pinned host memory into device staging, sets them
    # (sc_batch_set_fields), runs one batch iteration (sc_batch_run with outputs)
    # and reads every member's Delta_new, j and F back (sc_batch_get_outputs into
    # device staging, then one copy into pinned host memory).  Uploads and
    # read-backs run on two more streams through double-buffered staging.
    e2e = None
    if not args.no_e2e:
        npt = [p["nx"] * p["ny"] for p, _, _ in grains]
        off = np.concatenate([[0], np.cumsum(npt)]).astype(np.int64)
        tot = int(off[-1])
        h_in = torch.empty((tot, 2), dtype=torch.float64).pin_memory()
        for (p, d, _), o0 in zip(grains, off[:-1]):
            h_in[o0:o0 + p["nx"] * p["ny"]] = torch.view_as_real(
                torch.as_tensor(np.ascontiguousarray(d, np.complex128).reshape(-1)))
        # outputs of all members: Delta_new (complex), then j (2 reals), then F
        d_in = [torch.empty((tot, 2), dtype=torch.float64, device=dev) for _ in range(2)]
        d_out = [torch.empty(5 * tot, dtype=torch.float64, device=dev) for _ in range(2)]
        h_out = [torch.empty(5 * tot, dtype=torch.float64).pin_memory() for _ in range(2)]
        cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()

        def e2e_steps(n_steps):
            ev_in = [torch.cuda.Event() for _ in range(n_steps)]
            ev_used = [torch.cuda.Event() for _ in range(n_steps)]
            ev_out = [torch.cuda.Event() for _ in range(n_steps)]
            ev_read = [torch.cuda.Event() for _ in range(n_steps)]
            for i in range(n_steps):
                k = i % 2
                with torch.cuda.stream(cs_in):
                    if i >= 2:
                        cs_in.wait_event(ev_used[i - 2])  # the buffer's previous upload was consumed
                    d_in[k].copy_(h_in, non_blocking=True)
                    ev_in[i].record(cs_in)
                stream.wait_event(ev_in[i])
                if i >= 2:
                    stream.wait_event(ev_read[i - 2])  # the output staging was read back
                flush.fill_(float(i))
                sc.sc_batch_set_fields(b.h, d_in[k], True, stream)
                ev_used[i].record(stream)
                sc.sc_batch_run(b.h, 1, True, stream)
                sc.sc_batch_get_outputs(b.h, d_out[k][:2 * tot], d_out[k][2 * tot:4 * tot], d_out[k][4 * tot:],
                                        True, stream)
                ev_out[i].record(stream)
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(ev_out[i])
                    h_out[k].copy_(d_out[k], non_blocking=True)
                    ev_read[i].record(cs_out)
            t_enq = time.perf_counter()
            torch.cuda.synchronize()
            return t_enq

        e2e_steps(3)  # untimed: the copy streams' and the pinned buffers' first use
        n_e2e = max(5, min(args.steps, 20))
        t0 = time.perf_counter()
        t_enq = e2e_steps(n_e2e)
        e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
        e2e = {"value": info.steps_per_sweep / (e2e_ms * 1e-3), "unit": "trajectory-steps/s",
               "h2d_bytes_per_step": int(h_in.numel() * 8), "d2h_bytes_per_step": int(h_out[0].numel() * 8),
               "ms_per_step": e2e_ms, "host_enqueue_ms_per_step": (t_enq - t0) * 1e3 / n_e2e,
               "steps": n_e2e}
    fp32_launches = info.sweep_launches
    launches_per_iteration = info.launches_per_iteration
    fp32_lane_fill = info.steps_per_sweep / max(info.lane_steps_per_sweep, 1)
    last = b.info()
    classes = [{"energies_per_lane": last.class_ept[k], "blocks_per_sm": last.class_blocks_per_sm[k],
                "ms": last.class_ms[k]} for k in range(last.sweep_launches)]
    # with the transfers inside the sweep launches, the sweep kernel alone is also
    # timed in the separate layout (same classes and blocks per SM), after the
    # timed steps, so that its own roofline fraction is reported beside the
    # fused launches'
    separate = None
    if last.fused_transfers:
        b.set_fused_transfers(False)
        b.run(2, True, stream)
        ms_sep = []
        for i in range(5):
            b.run(1, True, stream)
            flush.fill_(float(i))
            ms_sep.append(b.info().ms_sweep)
        torch.cuda.synchronize()
        separate = {"ms_per_sweep": statistics.mean(ms_sep), "steps": 5}
    b.close()
    del b

    # the plain FP64 batch on the same grains (same work list and launch scheme;
    # its energies-per-lane bound left at the library's default)
    fp64 = None
    if args.precision == "fp32" and not args.no_fp64:
        b64 = sc.Batch([p for p, _, _ in grains], precision="fp64")
        for (p, d, _), m in zip(grains, b64.members):
            m.set_fields(d)
        b64.run(2, True, stream)  # the first sweep from fresh boundary values, then one replay
        torch.cuda.synchronize()
        if want_oracle:
            got["fp64"] = {i: _member_outputs(b64.members[i]) for i in check}
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.fp64_steps)]
        k64 = []
        for a_, c_ in ev64:
            a_.record(stream)
            b64.run(1, True, stream)
            c_.record(stream)
            flush.fill_(1.0)
            k64.append(b64.info().ms_sweep)
        torch.cuda.synchronize()
        ms64 = sum(a_.elapsed_time(c_) for a_, c_ in ev64) / len(ev64)
        i64 = b64.info()
        v64 = i64.steps_per_sweep / (ms64 * 1e-3)
        sm_max = (clocks or {}).get("sm_max_mhz") or 2032.0
        pk64 = SM_COUNT_B300 * FP64_LANES_PER_SM * sm_max * 1e6 / 1e9
        ach64 = (i64.steps_per_sweep // 2) * ALG_OPS_PER_PSE[args.stepper] / (statistics.mean(k64) * 1e-3) / 1e9
        fp64 = {"value": v64, "unit": "trajectory-steps/s", "ms_per_step": ms64, "steps": len(ev64),
                "warmup": 2, "energies_per_lane": i64.energies_per_lane, "sweep_launches": i64.sweep_launches,
                "speedup_fp32_over_fp64": value / v64,
                "roofline": {"bound": "alu", "achieved": ach64, "peak": pk64, "unit": "Gop/s",
                             "frac": ach64 / pk64, "ms_per_sweep": statistics.mean(k64),
                             "peak_note": "FP64 pipe 148 SM x 2 lanes/cycle (ncu pipe peak) x max SM clock (derived)"}}
        b64.close()
        del b64

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    pse = info.steps_per_sweep // 2  # ~ (pair, sample, energy) combinations
    achieved = pse * ALG_OPS_PER_PSE[args.stepper] / (sweep_ms * 1e-3) / 1e9
    lanes = FP32_LANES_PER_SM if args.precision == "fp32" else FP64_LANES_PER_SM
    peak_gops = SM_COUNT_B300 * lanes * ((clocks or {}).get("sm_max_mhz") or 2032.0) * 1e6 / 1e9
    traffic = _profiled_traffic(workload, args.precision, last.fused_transfers)
    pm = _measured_fma_peak() if args.precision == "fp32" else None
    line = {
        "metric": METRIC, "value": value, "unit": "trajectory-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": workload, "grains": args.grains,
                   "steps_per_sweep": info.steps_per_sweep, "work_items": info.n_items,
                   "energies_per_lane": ept, "precision": args.precision, "stepper": args.stepper,
                   "energy_sum": args.energy_sum, "lane_fill": fp32_lane_fill,
                   "sweep_launches": fp32_launches, "sweep_classes": classes,
                   "two_part_members": last.split_members,
                   "autotune_split_ms": {"with_parts": last.split_ms_on, "without": last.split_ms_off},
                   "fused_transfers": bool(last.fused_transfers), "transfer_items": last.transfer_items,
                   "autotune_fuse_ms": {"with_transfer_items": last.fuse_ms_on, "without": last.fuse_ms_off},
                   "min_lanes_per_line": last.min_lanes_per_line,
                   "step": "one batch iteration: every member's rotate, the sweep, rotate-back and outputs",
                   "ms_iteration": last.ms_iteration,
                   "l2": "flushed between timed steps", "parallelism": f"replicas{world}",
                   "cuda_graph": "one graph per iteration parity"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": traffic,
                     "kernel": f"sweep_kernel ({fp32_launches} launches back to back per sweep)"
                     + (", which also run most members' rotations and rotate-backs as work items"
                        if last.fused_transfers else ""),
                     "ms_per_sweep": sweep_ms,
                     "ops_per_unit": f"{ALG_OPS_PER_PSE[args.stepper]} FP32 lane-operations per (angle pair, "
                                     "sample, energy): the optimised closed-form formulation, terms that depend "
                                     "only on the segment excluded",
                     "peak_note": ("FP32" if args.precision == "fp32" else "FP64")
                     + " lane issue 148 SM x lanes/cycle x max SM clock (derived)",
                     "peak_measured": pm, "frac_of_measured": (achieved / pm) if pm else None,
                     "sweep_kernel_alone": None if separate is None else dict(
                         separate, frac=pse * ALG_OPS_PER_PSE[args.stepper] / (separate["ms_per_sweep"] * 1e-3)
                         / 1e9 / peak_gops,
                         note="the same class launches without the transfer work items (transfers in launches "
                              "of their own), 5 steps after the timed ones"),
                     "peak_measured_note": "sc_debug_fma_rate after the timed steps: 8 blocks of 256 threads per SM, "
                                           "8 independent FMA chains per thread"},
        "fp64_plain": fp64,
        "e2e": e2e,
        # one iteration: (FP32) the field conversion and rotation over all members,
        # one sweep launch per energies-per-lane class, energy-block sums, the
        # rotate-back (one launch per component count present), outputs and final sums
        "gpu_launches": launches_per_iteration * args.steps,
        "clocks": clocks,
        "wall_s": t_wall,
    }
    if want_oracle:
        import oracle
        errs, secs, n_steps = {}, 0.0, 0
        for i in check:
            p, d, _ = grains[i]
            g = oracle.OracleGeom(p)
            mk = g.mask().astype(bool)
            # the first sweep is the timed CPU sample; the second (from its exit
            # values) completes the two sweeps the errors are taken after
            t0 = time.perf_counter()
            o = g.full_sweep(d, None, None)
            secs += time.perf_counter() - t0
            n_steps += msteps[i]
            o = g.full_sweep(d, None, o["exit"])
            errs[str(i)] = {"grain": {"shape": "disc" if p["shape_kind"] == 0 else "polygon",
                                      "pairing": "s" if p["pairing"] == 0 else "dx2y2", "grid": p["nx"],
                                      "n_angles": p["n_angles"], "n_energies": p["n_energies"],
                                      "t": p["t"], "flux_quanta": p["flux_quanta"],
                                      "steps_per_sweep": msteps[i]}}
            for prec, res in got.items():
                errs[str(i)][prec] = _rel_errors(res[i], o, mk)
        worst = {k: max(errs[str(i)][args.precision][k] for i in check) for k in ("delta_new", "j", "F")}
        line["errors_vs_fp64_oracle"] = {
            "members": errs, "worst_" + args.precision: worst,
            "tolerance": {"delta_new": 1e-5, "j": 1e-4, "F": 1e-4},
            "within_tolerance": all(worst[k] <= tol for k, tol in (("delta_new", 1e-5), ("j", 1e-4), ("F", 1e-4))),
            "norm": "max over the grain, relative to the oracle's max; 2 sweeps from fresh boundary values"}
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = {
            "value": n_steps / secs, "unit": "trajectory-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"the first FP64 oracle sweep with outputs of grains {check} of the {args.grains} "
                      f"(a subset: the smallest, the largest, an s-wave and a d-wave grain; "
                      f"{n_steps} trajectory-steps, {secs:.1f} s; their second sweeps, for the errors, untimed)"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the accelerator comparison of App. E (its table of examples (a)-(g)) at the
# example configuration's numerics: 20 points per xi0, 32 Fermi momenta,
# energy cutoff 16 (units 2 pi kB Tc) with Ozaki's sums, convergence 1e-5
# ---------------------------------------------------------------------------
PAPER_ACCEL_TABLE = {  # iterations printed in the paper (F: not converged in 10^4)
    "a_dwave_chiral": (80, 34, 25, 37), "b_dwave_octagon": (71, 33, 25, 32),
    "c_dwave_plus_swave": (69, 36, 30, 33), "d_dwave_phase_crystal": (3027, 809, 1054, 439),
    "e_swave_abrikosov_lattice": (1001, 313, 211, 133), "f_swave_disc_meissner": ("F", "F", 20, 43),
    "g_swave_disc_vortex": ("F", "F", 45, 42),
}


def _bulk_amplitude(pairing, t, tc_ratio, eps, w, n_angles=32):
    """Bulk |Delta| of one component alone at its T_c (initial guess only):
    t sum_p w_p <eta^2 / sqrt(eps_p^2 + Delta^2 eta^2)> = ln(t / tc) + t sum_p w_p / eps_p."""
    phi = 2 * math.pi * np.arange(n_angles) / n_angles
    eta2 = {0: np.ones_like(phi), 1: 2 * np.cos(2 * phi) ** 2, 2: 2 * np.sin(2 * phi) ** 2}[pairing]
    D = math.log(t / tc_ratio) + t * float(np.sum(w / eps))
    f = lambda d: t * float(np.mean(np.sum(w[None, :] * eta2[:, None] / np.sqrt(eps[None, :] ** 2 + d * d * eta2[:, None]), axis=1))) - D  # noqa: E731
    if f(1e-9) <= 0:
        return 0.0
    lo, hi = 1e-9, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
    return 0.5 * (lo + hi)


def accel_examples(ppx=20.0):
    """Parameters and initial fields of the table's examples.  Readings where
    the paper is silent: the octagon of (b) has side 10; (c) takes T_c^s =
    0.6 T_c; (d) removes a right-angled corner with legs of 7 xi0 from the
    square of side 25 and places its vortex at (-20, -20) from the centre;
    vortices of (e) and (g) sit at the centre; components start at their own
    bulk amplitudes, the second chiral component with phase pi/2."""
    h = 1.0 / ppx
    common = dict(n_angles=32, energy_sum="ozaki")
    ex = []
    p = W.disc(12.5, int(round(25 * ppx)), t=0.5, pairing=2, kappa=0.0, **common)
    p["components"] = [(2, 1.0), (1, 1.0)]
    ex.append(("a_dwave_chiral", p, [(0.0, 1.0), (0.25, 1.0)], []))
    vx, vy = W.regular_polygon((0.0, 0.0), 8, 10.0)
    p = W.polygon(vx, vy, h, margin=1.0, t=0.5, pairing=1, kappa=0.0, **common)
    ex.append(("b_dwave_octagon", p, [(0.0, 1.0)], []))
    p = W.disc(12.5, int(round(25 * ppx)), t=0.5, pairing=2, kappa=0.0, **common)
    p["components"] = [(2, 1.0), (0, 0.6)]
    ex.append(("c_dwave_plus_swave", p, [(0.0, 1.0), (0.0, 0.6)], []))
    sq = W.polygon_part([-12.5, 12.5, 12.5, -12.5], [-12.5, -12.5, 12.5, 12.5])
    cut = W.polygon_part([5.5, 19.5, 19.5], [12.5, -1.5, 12.5], add=False)
    p = W.composite([sq, cut], h, margin=1.0, t=0.1, pairing=1, kappa=100.0, **common)
    ex.append(("d_dwave_phase_crystal", p, [(0.0, 1.0)], [((-20.0, -20.0), -1)]))
    p = W.square(25.0, int(round(25 * ppx)), t=0.2, pairing=0, kappa=10.0, flux_quanta=20.0, **common)
    ex.append(("e_swave_abrikosov_lattice", p, [(0.0, 1.0)], [((0.0, 0.0), -13)]))
    p = W.disc(15.0, int(round(30 * ppx)), t=0.5, pairing=0, kappa=5.0, flux_quanta=0.5, **common)
    ex.append(("f_swave_disc_meissner", p, [(0.0, 1.0)], []))
    p = W.disc(15.0, int(round(30 * ppx)), t=0.5, pairing=0, kappa=5.0, flux_quanta=1.5, **common)
    ex.append(("g_swave_disc_vortex", p, [(0.0, 1.0)], [((0.0, 0.0), -1)]))
    return ex


def run_accel_table(args):
    import torch
    from paper_2205_15000_b300 import sc
    kinds = ["picard", "polyak", "barzilai-borwein", "congacc"]
    tol, max_iter = 1e-5, args.accel_max_iter
    out = {}
    only = set(args.accel_only.split(",")) if args.accel_only else None
    kinds = [k for k in kinds if not args.accel_kinds or k in args.accel_kinds.split(",")]
    for name, p, comps, vortices in accel_examples(args.accel_ppx):
        if only and name.split("_")[0] not in only:
            continue
        p["n_energies"] = W.ozaki_poles_for_cutoff(p["t"], 16.0)
        probe = sc.Context(p, host_only=True)
        eps, w = sc.sc_energy_grid(probe.h, p["n_energies"])
        X, Y = W.grid_xy(p)
        chi = np.zeros_like(X)
        for (cx, cy), wnd in vortices:
            chi += wnd * np.arctan2(Y - cy, X - cx)
        pair_list = [c[0] for c in p["components"]] if p.get("components") else [p["pairing"]]
        d0 = np.stack([_bulk_amplitude(pc, p["t"], tcr, eps, w) * np.exp(1j * (chi + 2 * math.pi * shift))
                       for pc, (shift, tcr) in zip(pair_list, comps)])
        d0 = d0[0] if len(comps) == 1 else d0
        magn = p["kappa"] > 0 and math.isfinite(p["kappa"])
        def iteration(ctx, m, prm, prev):
            """One sweep + residuals + accelerator step of the Python loop; prev holds
            (j, F) of the previous iteration."""
            ctx.sweep()
            o = ctx.outputs()
            d_in, a_in = ctx.fields()
            dn = o["delta_new"].reshape(d_in.shape)
            # Eq. global_error per order-parameter component (l2 over the grain), and
            # the change of j, A_ind and F between iterations
            dd = (dn - d_in).reshape(-1, *m.shape)[:, m]
            din = d_in.reshape(-1, *m.shape)[:, m]
            errs = [float(torch.linalg.vector_norm(dd[c]) / max(float(torch.linalg.vector_norm(din[c])), 1e-300))
                    for c in range(dd.shape[0])]
            j = o["j"]
            if prev[0] is not None:
                errs.append(float(torch.linalg.vector_norm(j - prev[0]) / max(float(torch.linalg.vector_norm(prev[0])), 1e-30)))
                errs.append(abs(o["F_total"] - prev[1]) / max(abs(prev[1]), 1e-300))
            prev[0], prev[1] = j.clone(), o["F_total"]
            ctx.accelerate(prm)
            if magn:
                _, a_out = ctx.fields()
                na = float(torch.linalg.vector_norm(a_in))
                errs.append(float(torch.linalg.vector_norm(a_out - a_in)) / na if na > 0 else 1.0)
            return errs

        # untimed warm-up of both loops: plan creation, module loads, torch's first kernels
        warm = sc.Context(p, precision=args.precision)
        warm.set_fields(d0)
        mw = torch.as_tensor(warm.mask().astype(bool), device="cuda")
        for kind in kinds:
            prev = [None, None]
            for _ in range(2):
                iteration(warm, mw, sc.accel_params(kind), prev)
            warm.self_consistency(sc.accel_params(kind), max_iter=2, tol=0.0, check_every=1)
        torch.cuda.synchronize()
        del warm
        res = {}
        for kind in kinds:
            ctx = sc.Context(p, precision=args.precision)
            ctx.set_fields(d0)
            m = torch.as_tensor(ctx.mask().astype(bool), device="cuda")
            prm = sc.accel_params(kind)
            prev = [None, None]
            conv = None
            hist = []
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for it in range(1, max_iter + 1):
                errs = iteration(ctx, m, prm, prev)
                if it % 10 == 1:
                    hist.append(max(errs))
                if it > 1 and max(errs) < tol:
                    conv = it
                    break
            torch.cuda.synchronize()
            py_ms = (time.perf_counter() - t0) * 1e3 / it
            # the same iterations through the native loop (sc_self_consistency), residual
            # read only at the end
            n_nat = min(it, 200)
            ctx2 = sc.Context(p, precision=args.precision)
            ctx2.set_fields(d0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ctx2.self_consistency(prm, max_iter=n_nat, tol=0.0, check_every=1 << 30)
            torch.cuda.synchronize()
            native_ms = (time.perf_counter() - t1) * 1e3 / n_nat
            res[kind] = {"iterations": conv if conv is not None else f"not converged in {max_iter}",
                         "ms_per_iteration": py_ms, "native_ms_per_iteration": native_ms,
                         "final_residual": max(errs), "residual_every_10": hist if args.accel_history else None}
        out[name] = {"ours": res, "paper": dict(zip(kinds, PAPER_ACCEL_TABLE[name])),
                     "grid": [p["nx"], p["ny"]], "ozaki_poles": p["n_energies"]}
        print(json.dumps({name: out[name]}), flush=True)
    print(json.dumps({"metric": "self-consistency iterations to 1e-5", "unit": "iterations",
                      "higher_is_better": False, "config": {"workload": "accelerator_table_app_e",
                                                            "points_per_xi0": args.accel_ppx, "n_angles": 32,
                                                            "energy_cutoff": 16, "energy_sum": "ozaki",
                                                            "precision": args.precision},
                      "examples": out}), flush=True)
    return 0


def run_ldos(args):
    """LDOS sweeps (Sec. 2): the C4 grain (d-wave disc R 25, 128^2, 64 angles,
    t 0.2, one vortex) at 64 real energies spanning [-Delta0, Delta0] with the
    broadening 0.05 Delta0 (Delta0 = the bulk gap maximum), 20 retarded sweeps
    per call (boundary burn-in) and the rotate-back; steps counted as in the
    Matsubara sweep (both directions, every segment, every energy)."""
    import torch
    from paper_2205_15000_b300 import sc
    world, rank, local = ranks.env_ranks()
    torch.cuda.set_device(local)
    dist = ranks.init("nccl")
    p, delta, _ = W.c4_disc_d()
    d0 = math.sqrt(2.0) * W.BULK_GUESS[("dx2y2", 0.2)]
    energies = np.linspace(-d0, d0, 64)
    n_burnin = 20
    ctx = sc.Context(p, precision=args.precision)
    ctx.set_fields(delta)
    info = ctx.info
    stream = torch.cuda.current_stream()
    out = torch.empty((len(energies), p["ny"], p["nx"]), dtype=torch.float64, device="cuda")
    per_call = n_burnin * len(energies) * (info.steps_per_sweep // p["n_energies"])
    for _ in range(args.warmup):
        sc.sc_ldos(ctx.h, energies, 0.05 * d0, n_burnin, out, True, stream)
    torch.cuda.synchronize()
    ranks.barrier(dist)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in ev:
        a_.record(stream)
        sc.sc_ldos(ctx.h, energies, 0.05 * d0, n_burnin, out, True, stream)
        b_.record(stream)
    torch.cuda.synchronize()
    ms = [a_.elapsed_time(b_) for a_, b_ in ev]
    total = ranks.max_over_ranks(dist, float(sum(ms)), torch.device("cuda", local))
    value = ranks.throughput(per_call * args.steps, world, total * 1e-3)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.median(ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": "c4_ldos_128sq_64ang_64energies_vortex", "n_energies": len(energies),
                       "broadening": 0.05 * d0, "burnin_sweeps_per_step": n_burnin,
                       "steps_per_call": per_call, "precision": args.precision,
                       "step": "sc_ldos: retarded sweeps with burn-in + rotate-back"},
            "gpu_launches": (2 + n_burnin + 1) * args.steps,
        }), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--energy-sum", default="matsubara", choices=["matsubara", "ozaki"],
                    help="Matsubara energies below the cutoff, or Ozaki's poles reaching it")
    ap.add_argument("--stepper", default="closed", choices=["closed", "midpoint"],
                    help="integrator along a line: closed-form step or implicit midpoint rule (App. C)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=256, help="grid side (reduced cases for profiling)")
    ap.add_argument("--angles", type=int, default=128, help="Fermi angles (reduced cases for profiling)")
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c4", "c5", "annulus"],
                    help="c3 (default): 64 grains swept as one batch; c2: one 256^2 d-wave [110] grain; "
                         "c4: d-wave disc with a vortex (128^2); c5: 1024^2 d-wave square, 20 vortices; "
                         "annulus: d-wave annulus R> 25, R< 10 (256^2), solenoid gauge")
    ap.add_argument("--adjoint", action="store_true", help="add the adjoint sweep (gradient of F) to a step")
    ap.add_argument("--adjoint-checkpoint", type=int, default=0,
                    help="adjoint: keep the forward gamma every k samples and recompute (0: park every sample)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--errors", action="store_true",
                    help="c4/c5: also run the FP64 oracle on the whole grain (c5: one sweep, minutes on "
                         "the host cores) and report the errors of Delta_new, j and F")
    ap.add_argument("--energies", type=int, default=0, help="energy count (0: the workload's own)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 2, 4, 8, 16, 32],
                    help="energy lanes per line (0: the library's choice)")
    ap.add_argument("--grains", type=int, default=64)
    ap.add_argument("--ept", type=int, default=0,
                    help="batch bound on energies per lane (0: chosen by sc_batch_autotune)")
    ap.add_argument("--no-fp64", action="store_true", help="batch: skip the plain FP64 comparison arm")
    ap.add_argument("--transfers", default="auto", choices=["auto", "fused", "separate"],
                    help="batch: members' rotations and rotate-backs as work items of the sweep launches "
                         "(fused), in launches of their own (separate), or as sc_batch_autotune chooses (auto)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="batch: timed steps of the plain FP64 arm")
    ap.add_argument("--ldos", action="store_true", help="time the LDOS sweeps on the c4 grain (64 energies)")
    ap.add_argument("--accel-table", action="store_true",
                    help="iterations of the four accelerators on the examples of App. E's table")
    ap.add_argument("--accel-ppx", type=float, default=20.0, help="points per xi0 for --accel-table")
    ap.add_argument("--accel-max-iter", type=int, default=10000)
    ap.add_argument("--accel-only", default="", help="comma-separated example letters, e.g. a,d")
    ap.add_argument("--accel-kinds", default="", help="comma-separated accelerators")
    ap.add_argument("--accel-history", action="store_true", help="record the residual every 10 iterations")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference_batch(args) if args.workload == "c3" else run_reference(args)
    if args.accel_table:
        return run_accel_table(args)
    if args.ldos:
        return run_ldos(args)
    if args.workload == "c3":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
