#!/usr/bin/env python
"""Throughput of the phase-field twin step on GB300.

Default workload: the 256^3 polycrystal (64 Voronoi grains with random
orientations, all six {10-12} variants, 8 random nuclei, -2% along z), FP32
fields and FFTs with FP64 reductions, Moulinec-Suquet tolerance 1e-6.  A step
is one full pf_step: the Moulinec-Suquet solve to tolerance, the driving
forces and the Allen-Cahn update.  Metric: voxel-steps/s.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

METRIC = "voxel-steps/s per PF step (FFT+Green+update), mixed vs FP64; % HBM roofline"
UNIT = "voxel-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
KERNEL_SRC = os.path.join(ROOT, "paper_2302_13612_gb300", "csrc", "pf_kernels.cu")


def hbm_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(ms, dist=None):
    """Elapsed milliseconds of the slowest rank (measurement only; the data
    path of the instances has no collective)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(n_voxels, steps, world, ms_max):
    """Whole-job voxel-steps/s: every rank advances its own instance."""
    return world * n_voxels * steps / (ms_max / 1e3)


def workload(name, steps, rank=0):
    from paper_2302_13612_gb300 import inputs as I
    if name == "poly256":
        return I.config3(steps=steps, seed=1003 + rank), \
            "256^3 polycrystal, 64 grains, 6 variants, -2% zz (cfg 3)"
    if name == "poly128":
        return I.config3(steps=steps, n=128, seed=1003 + rank), \
            "128^3 polycrystal, 64 grains, 6 variants, -2% zz (cfg 3 recipe at 128^3, for profiler captures)"
    if name == "pillar128":
        return I.config2(steps=steps, seed=1002 + rank), \
            "128^3 single-crystal pillar, 2 variants, plastic strain, ramp to -4% (cfg 2)"
    if name == "pillar512":
        return I.config5(steps=steps, seed=1005 + rank), \
            "512^3 single-crystal pillar, 2 variants, plastic strain, ramp (cfg 5)"
    if name == "plain32":
        return I.config1(steps=steps), "32^3 single crystal, 1 variant, homogeneous (cfg 1)"
    raise SystemExit(f"unknown workload {name}")


# --------------------------------------------------------------------------
# algorithmic bytes per launch (each field read or written once)
# --------------------------------------------------------------------------
def bytes_per_launch(name, w, esz, warm_degree=3, warm_points=0):
    nz, ny, nx = w.shape
    N = nx * ny * nz
    nh = ny * nz * (nx // 2 + 1)   # complex values per half-spectrum component
    c = 2 * esz
    V = w.V
    ep = 6 * N * esz if w.eps_p is not None else 0
    gr = 2 * N if w.grain is not None else 0
    table = {
        "x_fwd_tau": 6 * N * esz + V * N * esz + ep + gr + 6 * nh * c,
        "x_fwd_drive": 6 * N * esz + V * N * esz + ep + gr + V * nh * c,
        "y_pass_ms": 2 * 6 * nh * c,
        "y_pass_pf": 2 * V * nh * c,
        "z_green": 2 * 6 * nh * c,
        "z_helmholtz": 2 * V * nh * c,
        "x_inv_eps": 6 * nh * c + 2 * 6 * N * esz,
        "x_inv_f": V * nh * c + V * N * esz,
        "c0_sum": V * N * esz + gr,
        # degree d (steady state): the strain and d histories in, the start and
        # one history slot out
        "warm_start": ((warm_points or warm_degree + 1) + 2) * 6 * N * esz,
    }
    return table.get(name)


CSRC = os.path.dirname(KERNEL_SRC)
# the sources each profiled kernel is compiled from (its translation unit and
# the headers it includes)
DEVICE_HEADERS = ("pf_device.cuh", "pf_fft.cuh", "pf_f2.cuh", "pf_internal.h", "pf_tma.cuh")
KERNEL_SRCS = {"x_fwd_tau": ("pf_xfix.cu", "pf_xfix.cuh", "pf_pfa.cuh", "pf_dft32.cuh") + DEVICE_HEADERS}


def src_hash(files):
    hsh = hashlib.sha256()
    for f in files:
        hsh.update(open(os.path.join(CSRC, f), "rb").read())
    return hsh.hexdigest()[:16]


def traffic_for(kernel, workload_name):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since those counters were taken."""
    try:
        src = src_hash(KERNEL_SRCS[kernel])
        for line in open(TRAFFIC_FILE):
            kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
            if kv.get("kernel") == kernel and kv.get("workload") == workload_name and kv.get("src") == src:
                return float(kv["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


FP64_FILE = os.path.join(ROOT, "profiles", "fp64_flops.txt")
# the sources of the kernels the FP64 step runs (the generic passes)
FP64_SRCS = ("pf_k_xfwd.cu", "pf_k_xinv.cu", "pf_k_yz.cu", "pf_kernels.cu") + DEVICE_HEADERS


def fp64_src_hash():
    return src_hash(FP64_SRCS)


def fp64_flops(workload_name):
    """Executed FP64 flops per voxel of one Moulinec-Suquet pass and of the
    phase-field update of the FP64 step (ncu instruction counts, FMA = 2),
    from the committed summary, or None when the kernel sources changed
    since those counts were taken."""
    try:
        src = fp64_src_hash()
        for line in open(FP64_FILE):
            kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
            if kv.get("workload") == workload_name and kv.get("src") == src:
                return float(kv["flops_per_voxel_pass"]), float(kv["flops_per_voxel_update"])
    except (OSError, ValueError, KeyError):
        pass
    return None


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
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
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on a bounded sample
# --------------------------------------------------------------------------
def oracle_sample(n_sample, steps, warmup):
    """Time the oracle stepping the polycrystal recipe on an n_sample^3 grid
    (same structure as the 256^3 workload: 64 grains, 6 variants)."""
    from oracle import pf_oracle as O
    from paper_2302_13612_gb300 import inputs as I
    w = I.config3(steps=steps + warmup, n=n_sample)
    st = O.state_from_workload(w)
    for k in range(warmup):
        st.step(w.E[k])
    t0 = time.perf_counter()
    for k in range(steps):
        st.step(w.E[warmup + k])
    dt = time.perf_counter() - t0
    return w.nvox * steps / dt, dt, w


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.ref_n
    value, dt, w = oracle_sample(n, args.steps, args.warmup)
    cores = os.cpu_count()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"polycrystal recipe of the 256^3 workload at {n}^3 (64 grains, 6 variants)",
                   "grid": [n, n, n]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle steps of the polycrystal recipe at {n}^3 "
                                   f"after {args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2302_13612_gb300 import pf

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    pf.load_library()
    total = max(args.warmup + args.steps + 2, args.warmup + 2 + 12)
    w, desc = workload(args.workload, total, rank)
    N = w.nvox
    stream = torch.cuda.current_stream()
    prec = args.precision
    dt = torch.float64 if prec == "fp64" else torch.float32
    cfg = pf.config_for(w, precision=prec, ms_tol=args.ms_tol, stream=stream.cuda_stream,
                        warm_degree=args.warm_degree, warm_points=args.warm_points, autotune=args.autotune)
    h = pf.Handle(cfg, 1, grain_R=w.grain_R)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    f_d = dev(w.f.reshape(w.V, N))
    ep_d = None if w.eps_p is None else dev(w.eps_p.reshape(6, N))
    g_d = None if w.grain is None else torch.from_numpy(w.grain.reshape(N).astype(np.int16)).cuda()
    h.set_fields(0, f_d, ep_d, g_d, None, mem=pf.PF_MEM_DEVICE)
    torch.cuda.synchronize()

    # warm-up
    h.step(w.E[: args.warmup][None])
    torch.cuda.synchronize()

    # timed region: inputs resident in HBM; per-kernel events on the launch stream
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    h.timing(True)
    barrier()
    torch.cuda.synchronize()
    l0 = h.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    code, info = h.step(w.E[args.warmup: args.warmup + args.steps][None])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = h.launch_count() - l0
    table = h.timing_table()
    h.timing(False)
    clk = clocks.stop()
    n_ms_mean = info[0].n_ms_total / args.steps
    ms = max_over_ranks(ms, dist)
    value = aggregate_rate(N, args.steps, world, ms)

    # the same steps as one CUDA graph launch (device-side pass control)
    graph = None
    if args.graph or not args.no_extras:
        cfgg = pf.config_for(w, precision=prec, ms_tol=args.ms_tol, stream=stream.cuda_stream, use_graph=1,
                             warm_degree=args.warm_degree, warm_points=args.warm_points, autotune=args.autotune)
        hg = pf.Handle(cfgg, 1, grain_R=w.grain_R)
        hg.set_fields(0, f_d, ep_d, g_d, None, mem=pf.PF_MEM_DEVICE)
        hg.step(w.E[: args.warmup][None])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, ig = hg.step(w.E[args.warmup: args.warmup + args.steps][None])
        e1.record(stream)
        torch.cuda.synchronize()
        msg = max_over_ranks(e0.elapsed_time(e1), dist)
        graph = {"value": aggregate_rate(N, args.steps, world, msg), "ms_per_step": msg / args.steps,
                 "n_ms_mean": ig[0].n_ms_total / args.steps}
        hg.close()

    # the same steps with each solve started from the last strain alone
    plain_warm = None
    if not args.no_extras and args.warm_degree != 0:
        cfgp = pf.config_for(w, precision=prec, ms_tol=args.ms_tol, stream=stream.cuda_stream, warm_degree=0,
                             autotune=args.autotune)
        hp = pf.Handle(cfgp, 1, grain_R=w.grain_R)
        hp.set_fields(0, f_d, ep_d, g_d, None, mem=pf.PF_MEM_DEVICE)
        hp.step(w.E[: args.warmup][None])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, ip = hp.step(w.E[args.warmup: args.warmup + args.steps][None])
        e1.record(stream)
        torch.cuda.synchronize()
        msp = max_over_ranks(e0.elapsed_time(e1), dist)
        plain_warm = {"value": aggregate_rate(N, args.steps, world, msp), "ms_per_step": msp / args.steps,
                      "n_ms_mean": ip[0].n_ms_total / args.steps}
        hp.close()

    # end to end through the C ABI with host buffers: each step the host hands
    # over the plastic strain and reads back the twin fractions and <sigma>
    e2e = None
    if not args.no_extras:
        pin = lambda shape, d: torch.empty(shape, dtype=d).pin_memory().numpy()
        npdt = np.float64 if prec == "fp64" else np.float32
        ep_h = pin((6, N), dt)
        ep_h[...] = 0.0 if w.eps_p is None else w.eps_p.reshape(6, N)
        f_h = pin((w.V, N), dt)
        esz = np.dtype(npdt).itemsize
        k_e2e = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(k_e2e):
            h.set_plastic_strain(0, ep_h)
            _, inf2 = h.step(w.E[args.warmup + k][None, None])
            h.lib.pf_get_fields(h.h, 0, f_h.ctypes.data, None, pf.PF_MEM_HOST)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": world * N * k_e2e / te, "unit": UNIT,
               "h2d_bytes_per_step": 6 * N * esz + 48, "d2h_bytes_per_step": w.V * N * esz + 48,
               "steps": k_e2e, "what": "per step: plastic strain H2D from pinned memory, pf_step, "
                                        "twin fractions and <sigma> D2H"}
        if w.eps_p is None:
            h.set_plastic_strain(0, None)

    # the plain FP64 GPU step on the same workload (the mixed-vs-FP64 ratio)
    fp64 = None
    if not args.no_extras and prec != "fp64":
        torch.cuda.synchronize()
        cfg64 = pf.config_for(w, precision="fp64", ms_tol=args.ms_tol, stream=stream.cuda_stream,
                              warm_degree=args.warm_degree, warm_points=args.warm_points, autotune=args.autotune)
        h64 = pf.Handle(cfg64, 1, grain_R=w.grain_R)
        f64 = torch.from_numpy(w.f.reshape(w.V, N)).cuda()
        ep64 = None if w.eps_p is None else torch.from_numpy(w.eps_p.reshape(6, N)).cuda()
        h64.set_fields(0, f64, ep64, g_d, None, mem=pf.PF_MEM_DEVICE)
        # as many warm-up steps as the FP32 run has history when its timed steps
        # start (the extrapolated warm start holds up to warm_degree + 1 solutions)
        w64 = max(1, min(args.warmup + 2, total - 12))
        h64.step(w.E[:w64][None])
        k64 = 10
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, i64 = h64.step(w.E[w64:w64 + k64][None])
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        v64 = N * k64 / (ms64 / 1e3)
        fp64 = {"value": v64 * world, "ms_per_step": ms64 / k64, "n_ms_mean": i64[0].n_ms_total / k64,
                "speedup_fp32_over_fp64": value / (v64 * world)}
        h64.close()
        del f64, ep64

    # roofline of the dominant kernel
    esz = 8 if prec == "fp64" else 4
    peak, peak_kind = hbm_peak()
    kernels = {}
    tot_ms = sum(v[0] for v in table.values()) or 1.0
    for name, (kms, cnt) in table.items():
        b = bytes_per_launch(name, w, esz, args.warm_degree, args.warm_points)
        avg = kms / cnt
        kernels[name] = {"ms_total": round(kms, 4), "launches": cnt, "ms_avg": round(avg, 5),
                         "share": round(kms / tot_ms, 4),
                         "GB_s": round(b / (avg / 1e3) / 1e9, 1) if b else None}
    bpl = lambda k: bytes_per_launch(k, w, esz, args.warm_degree, args.warm_points)
    dom = max((k for k in kernels if bpl(k)), key=lambda k: kernels[k]["ms_total"])
    b = bytes_per_launch(dom, w, esz, args.warm_degree, args.warm_points)
    ach = b / (kernels[dom]["ms_avg"] / 1e3) / 1e9
    step_bytes = sum((bpl(k) or 0) * v["launches"] for k, v in kernels.items())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_kind": f"{peak_kind} (copy bandwidth)",
                "traffic": traffic_for(dom, args.workload), "algorithmic_bytes_per_launch": b,
                "step_effective_GB_s": round(step_bytes / (ms / 1e3) / 1e9, 1),
                "step_effective_frac": round(step_bytes / (ms / 1e3) / 1e9 / peak, 4)}

    # the survey's pass model of the step (fused xy passes; FP32 bytes per
    # voxel-step n_MS (194 + 4V) + 74 + 20V, doubled in FP64), with n_MS of this run
    model = (n_ms_mean * (194 + 4 * w.V) + 74 + 20 * w.V) * (esz / 4.0)
    roofline["step_model_B_per_voxel"] = round(model, 1)
    roofline["step_model_GB_s"] = round(model * N * args.steps / (ms / 1e3) / 1e9, 1)
    roofline["step_model_frac"] = round(roofline["step_model_GB_s"] / peak, 4)

    # measured arithmetic peaks (FMA chains, CUDA events) and the FP64 step
    # against the FP64 one: executed FP64 flops per voxel-step from the ncu
    # counts in profiles/ (n_MS passes plus the update)
    alu = None
    if not args.no_extras:
        alu = {k: round(pf.fma_peak(i, stream.cuda_stream) / 1e12, 3)
               for i, k in enumerate(("fp32_tflops", "fp32x2_tflops", "fp64_tflops"))}
        if fp64 is not None:
            fl = fp64_flops(args.workload)
            if fl is not None:
                per_step = fp64["n_ms_mean"] * fl[0] + fl[1]
                ach = per_step * N / (fp64["ms_per_step"] / 1e3) / 1e12
                fp64["roofline"] = {"bound": "fp64", "achieved": round(ach, 3), "peak": alu["fp64_tflops"],
                                    "unit": "TFLOP/s", "frac": round(ach / alu["fp64_tflops"], 4),
                                    "peak_kind": "measured (FMA chains)", "flops_per_voxel_step": round(per_step, 1)}
            fp64["fp32_step_hbm_frac"] = roofline["frac"]

    # precision: the FP32 and mixed steps against the FP64 GPU step from the
    # same fields (three steps, the FP64 step at a tight tolerance), relative
    # L2 and max errors of f, sigma and the <sigma> curve; and the mixed step's rate
    precision = None
    if not args.no_extras and prec != "fp64":
        precision = precision_errors(w, args, stream, f_d, ep_d, g_d)
        torch.cuda.synchronize()
        cfgm = pf.config_for(w, precision="mixed", ms_tol=args.ms_tol, stream=stream.cuda_stream,
                             warm_degree=args.warm_degree, warm_points=args.warm_points, autotune=args.autotune)
        hm = pf.Handle(cfgm, 1, grain_R=w.grain_R)
        hm.set_fields(0, f_d, ep_d, g_d, None, mem=pf.PF_MEM_DEVICE)
        hm.step(w.E[: args.warmup][None])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, im = hm.step(w.E[args.warmup: args.warmup + args.steps][None])
        e1.record(stream)
        torch.cuda.synchronize()
        msm = max_over_ranks(e0.elapsed_time(e1), dist)
        precision["mixed_step"] = {"value": aggregate_rate(N, args.steps, world, msm), "ms_per_step": msm / args.steps,
                                   "n_ms_mean": im[0].n_ms_total / args.steps,
                                   "speedup_over_fp64": (aggregate_rate(N, args.steps, world, msm) / fp64["value"])
                                   if fp64 else None}
        hm.close()

    # the batched form (48 uneven instances, one CUDA graph launch per call)
    batch = None
    if not args.no_extras:
        batch = batch_measure(args, rank, world, dist, steps=max(3, min(args.steps, 10)), warmup=3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        v_cpu, t_cpu, wc = oracle_sample(args.ref_n, 1, 1)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"1 FP64 oracle step (after 1 warm-up step) of the polycrystal recipe at "
                         f"{args.ref_n}^3, {t_cpu:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "mixed": "bf16x3+f32", "fp64": "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": desc, "grid": list(w.shape[::-1]), "variants": w.V,
                       "grains": len(w.grain_R), "precision": f"{prec} fields and FFTs, fp64 reductions",
                       "ms_tol": args.ms_tol, "n_ms_mean": n_ms_mean,
                       "autotune": bool(args.autotune),
                       "warm_start": "last strain" if args.warm_degree == 0 else
                       (f"degree-{args.warm_degree} least-squares fit to the last {args.warm_points} solutions"
                        if args.warm_points > args.warm_degree + 1 else
                        f"degree-{args.warm_degree} extrapolation through the last {args.warm_degree + 1} solutions"),
                       "l2": "working set > 1 GB per instance, larger than the 129 MB L2; no flush",
                       "parallelism": f"{world} independent instance(s), one per GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "fp64_step": fp64, "graph_step": graph, "plain_warm_start_step": plain_warm,
            "kernels": kernels, "alu_peaks": alu, "batch_step": batch, "precision_errors": precision,
        }
        print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def precision_errors(w, args, stream, f_d, ep_d, g_d, steps=3):
    """Relative errors of the FP32 and mixed steps against the FP64 GPU step,
    all three started from the same fields and advanced by the same mean
    strains with the same pass counts: f after the steps, the stress field
    of the last solved pair and the <sigma> curve of every step."""
    import torch

    from paper_2302_13612_gb300 import pf

    N = w.nvox
    res = {}
    ref = None
    for prec in ("fp64", "fp32", "mixed"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        h = pf.handle_for_device(w, prec, dict(ms_tol=0.0, ms_max_it=3, stream=stream.cuda_stream,
                                               warm_degree=args.warm_degree, warm_points=args.warm_points,
                                               autotune=args.autotune), f_d.to(dt),
                                 None if ep_d is None else ep_d.to(dt), g_d)
        curve = []
        for k in range(steps):
            _, info = h.step(w.E[k][None, None])
            curve.append(list(info[0].mean_sigma))
        f, _ = h.get_fields(0, want_eps=False)
        _, sig = h.stress(0)
        h.close()
        out = (np.asarray(f, np.float64), np.asarray(sig, np.float64), np.asarray(curve))
        if ref is None:
            ref = out
            continue
        rl2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        rmx = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
        res[prec] = {"f_rel_l2": rl2(out[0], ref[0]), "f_rel_max": rmx(out[0], ref[0]),
                     "sigma_rel_l2": rl2(out[1], ref[1]), "sigma_rel_max": rmx(out[1], ref[1]),
                     "mean_sigma_curve_rel_max": rmx(out[2], ref[2])}
    res["what"] = (f"{steps} steps from the same fields, 3 Moulinec-Suquet passes each, against the FP64 GPU step "
                   f"(which matches the FP64 oracle to 1e-12 on the parity grids)")
    return res


def batch_measure(args, rank, world, dist, steps, warmup):
    """The batched form: args.batch independent instances with grids drawn
    from {64, 80, 96, 120, 128, 160}^3 in one handle, each pf_step call one
    CUDA graph launch advancing every instance (parallel graph branches).
    Returns its rate, time per step and the step's effective bandwidth."""
    import torch

    from paper_2302_13612_gb300 import inputs as I
    from paper_2302_13612_gb300 import pf

    n_inst = args.batch
    total = warmup + steps
    ws = [I.config4_instance(rank * n_inst + i, steps=total) for i in range(n_inst)]
    stream = torch.cuda.current_stream()
    h = pf.batch_handle_for(ws, precision="fp32" if args.precision == "fp64" else args.precision,
                            ms_tol=args.ms_tol, use_graph=1, stream=stream.cuda_stream,
                            warm_degree=args.warm_degree, warm_points=args.warm_points, autotune=args.autotune)
    nvox = sum(w.nvox for w in ws)
    E = np.stack([w.E for w in ws])
    h.step(E[:, :warmup])
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = h.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    code, infos = h.step(E[:, warmup:])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    clk = clocks.stop()
    value = aggregate_rate(nvox, steps, world, ms)
    esz = 4
    step_bytes = 0.0
    model_bytes = 0.0
    for w, inf in zip(ws, infos):
        n_ms = inf.n_ms_total / steps
        per_pass = sum(bytes_per_launch(k, w, esz) for k in ("x_fwd_tau", "y_pass_ms", "z_green", "x_inv_eps")) \
            + bytes_per_launch("y_pass_ms", w, esz)
        update = sum(bytes_per_launch(k, w, esz) for k in ("x_fwd_drive", "z_helmholtz", "x_inv_f", "c0_sum")) \
            + 2 * bytes_per_launch("y_pass_pf", w, esz)
        if args.warm_degree:
            update += bytes_per_launch("warm_start", w, esz, args.warm_degree, args.warm_points)
        step_bytes += n_ms * per_pass + update
        model_bytes += (n_ms * (194 + 4 * w.V) + 74 + 20 * w.V) * w.nvox
    peak, peak_kind = hbm_peak()
    eff = step_bytes * steps / (ms / 1e3) / 1e9
    meff = model_bytes * steps / (ms / 1e3) / 1e9
    out = {
        "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
        "instances": n_inst, "voxels": nvox,
        "n_ms_mean": sum(i.n_ms_total for i in infos) / (steps * n_inst),
        "workload": f"{n_inst} independent instances, grids from {{64,80,96,120,128,160}}^3, 1-3 variants, "
                    f"one CUDA graph launch per call (cfg 4)",
        "grids": [list(w.shape[::-1]) for w in ws[:8]] + (["..."] if n_inst > 8 else []),
        "roofline": {"bound": "hbm", "kernel": "whole step (graph)", "achieved": round(eff, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(eff / peak, 4), "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "traffic": None, "step_model_GB_s": round(meff, 1), "step_model_frac": round(meff / peak, 4)},
        # kernels run inside the graph: per instance and step C0 (2), step begin (1),
        # each pass 6 + 1 decision, the update (6) and the step end (1); the
        # extrapolated warm start adds 2 per step
        "gpu_launches": sum((10 + (2 if args.warm_degree else 0)) * steps + 7 * i.n_ms_total for i in infos),
        "graph_launches": h.launch_count() - l0, "clocks": clk, "status": code,
    }
    h.close()
    return out


def run_batch(args):
    """--workload batch: the batched form as the bench line."""
    import torch

    from paper_2302_13612_gb300 import pf

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pf.load_library()
    b = batch_measure(args, rank, world, dist, args.steps, args.warmup)
    if rank == 0:
        line = {
            "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "instances": b["instances"], "voxels": b["voxels"],
                       "n_ms_mean": b["n_ms_mean"], "warm_degree": args.warm_degree,
                       "autotune": bool(args.autotune), "grids": b["grids"],
                       "l2": "working set of the batch > 1 GB; no flush"},
            "roofline": b["roofline"], "gpu_launches": b["gpu_launches"], "graph_launches": b["graph_launches"],
            "clocks": b["clocks"], "status": b["status"],
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    # four untimed steps: the degree-3 extrapolated warm start holds its four
    # solutions from the first timed step on
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poly256",
                    choices=["poly256", "poly128", "pillar128", "pillar512", "plain32", "batch"])
    ap.add_argument("--batch", type=int, default=48, help="instances of the batch workload")
    ap.add_argument("--graph", action="store_true", help="run the timed steps as CUDA graph launches")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed", "fp64"],
                    help="mixed: FP32 with the y transforms on the BF16 tensor cores (three-term splits)")
    ap.add_argument("--ms-tol", type=float, default=1e-6)
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="time candidate pass shapes and FFT radix orders at the first step (warm-up)")
    ap.add_argument("--warm-degree", type=int, default=3, choices=[0, 1, 2, 3, 4, 5],
                    help="degree of the extrapolated start of each step's Moulinec-Suquet passes")
    ap.add_argument("--warm-points", type=int, default=0, choices=[0, 2, 3, 4, 5, 6],
                    help="solutions the warm start holds (more than degree + 1: least-squares fit)")
    ap.add_argument("--ref-n", type=int, default=64, help="grid of the oracle's bounded sample")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e, FP64 and CPU legs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
