#!/usr/bin/env python
"""Benchmark: resolvent actions/s of the batched randomized-SVD time march.

One step = one full randomized SVD of the workload (every direct and adjoint
march plus the per-frequency QR / SVD glue) through rsv_gains_modes.  One
resolvent action = one test vector x one frequency through one march.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank marches its own
independent copy of the workload (frequency / test-vector blocks are
independent problems), so the job is weak-scaled with no data-path
collective; the time is the max over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "resolvent actions/s (test vectors x freqs) at <=1e-4 gain error"
L2_FLUSH_BYTES = 512 << 20


def marches_per_step(w) -> int:
    return 2 * w.n_power_iter + 2


def n_instances(w) -> int:
    return len(w.system.n) if type(w.system).__name__ == "GL1D" else 1


def actions_per_step(w) -> int:
    return marches_per_step(w) * w.k * w.n_omega * n_instances(w)


def workload(name: str):
    return W.ALL[name]()


def default_precision(name: str) -> str:
    return "fp64" if name == "c1" else "fp32"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (also exercised by the CPU gloo tests)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed_offset(rank: int) -> int:
    """Each rank marches an independent test block (weak scaling)."""
    return 1000 * rank


def max_over_ranks(value: float, group=None, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# per-kernel roofline model
# ---------------------------------------------------------------------------
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


# DRAM bytes (read + write) per launch group of a category's kernels over one time tile,
# from ncu captures of the same kernels at the same rows per launch, keyed by (workload,
# category, tile steps, rows per launch).  An entry is dropped whenever the kernel it
# describes changes.  Sources (summaries in profiles/):
#   dense march  dense_tc_march_c2.txt: one 256-step launch, 84.35 MB read + 24.63 MB written
#   1-D march    gl1d_tile_c5.txt: one 127-step launch, 754.9 MB read + 344.4 MB written
#   2-D march    adr2d_stage_c3.txt: the four stage kernels of one step at 16 vectors,
#                558.5 MB per step, scaled by 255 steps (traffic per step is constant)
TRAFFIC = {
    ("dense_hermite_gl_n1024_k32_w256_trm", "march", 256, 32768):
        {"bytes": 108.98e6, "src": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"},
    ("gl_batch64_k8_w64_ssrm", "march", 127, 365184):
        {"bytes": 1.0993e9, "src": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"},
    ("adr2d_1024x512_k16_w128_ssrm", "march", 255, 8388608):
        {"bytes": 255 * 558.5e6, "src": "ncu dram bytes of the four stage kernels of one step x 255 steps"},
}

FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
FP64_ALU_TFLOPS = 1.25                                # nominal FP64 rate of the part


def kernel_model(cat, w, prec, tile, groups, ms_total, rows, path):
    """Roofline record of one kernel category: algorithmic work per launch / average launch time.

    Units of work per launch (one time tile of S steps):
      synthesis  rows x n_omega x n_tau complex (8 flop) or real-output (4 flop) multiply-adds
      analysis   rows x n_omega x S multiply-adds (8 flop complex state, 4 flop real state)
      march      dense: 8 n^2 k flop per step (one dense complex product, tensor cores);
                 1-D kind (state held on chip for the whole tile): the forcing tile read
                 (2S+1 stage times), the snapshot tile written (S steps) and the state read
                 and written once, (3S + 3) state passes per tile;
                 2-D whole-step kernel: 6 state passes per step (state read and written,
                 forcing read at the three stage times, snapshot written);
                 per-stage kernels: 15 state passes per step (12 for four stage read/write
                 pairs, 2 forcing reads, 1 snapshot write)
    """
    peaks = load_peaks()
    avg_s = ms_total / max(groups, 1) / 1e3
    S = tile
    dense = "kind=dense" in path
    se = (8 if prec == "fp64" else 4) * (1 if w.real_state else 2)
    alu_peak = FP64_ALU_TFLOPS if prec == "fp64" else FP32_ALU_TFLOPS
    cflop = 4 if w.real_state else 8
    tc_contract = "contractions=tcgen05" in path
    if cat in ("synthesis", "analysis") and tc_contract:
        peak_tc = peaks["bf16_tflops"] * 1.1 / 2.25
    if cat == "synthesis":
        n_tau = S if dense else 2 * S + 1
        work = rows * w.n_omega * n_tau * cflop
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if prec != "fp64" else "nominal FP64"
        if tc_contract:
            bound, peak, src = "tensor", peak_tc, "measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)"
    elif cat == "analysis":
        work = rows * w.n_omega * S * cflop
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if prec != "fp64" else "nominal FP64"
        if tc_contract:
            bound, peak, src = "tensor", peak_tc, "measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)"
    elif cat == "march" and dense and "tcgen05" in path:
        work = 8.0 * w.n * w.n * w.k * S
        peak = peaks["bf16_tflops"] * 1.1 / 2.25
        bound, unit, per = "tensor", "TFLOP/s", 1e12
        src = "measured bf16 x nominal tf32/bf16 ratio (1.1/2.25); 3xTF32 split products counted once"
    elif cat == "march" and dense:
        work = 8.0 * w.n * w.n * w.k * S
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived FP32 CUDA-core rate"
    elif cat == "march" and "whole-step" in path:
        work = 6.0 * rows * se * S
        bound, unit, peak, per = "hbm", "GB/s", peaks["hbm_gbs"], 1e9
        src = peaks["src"] + " copy bandwidth"
    elif cat == "march" and "kind=gl1d" in path:
        work = (3.0 * S + 3.0) * rows * se
        bound, unit, peak, per = "hbm", "GB/s", peaks["hbm_gbs"], 1e9
        src = peaks["src"] + " copy bandwidth"
    else:
        work = 15.0 * rows * se * S
        bound, unit, peak, per = "hbm", "GB/s", peaks["hbm_gbs"], 1e9
        src = peaks["src"] + " copy bandwidth"
    achieved = work / avg_s / per
    traffic = TRAFFIC.get((w.name, cat, S, rows))
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic["bytes"] if traffic else None, "traffic_src": traffic["src"] if traffic else None,
            "kernel": cat, "work_per_launch": work, "avg_launch_ms": avg_s * 1e3, "peak_src": src}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample, in a subprocess with one thread
# ---------------------------------------------------------------------------
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import frequencies, march, operators
w = W.ALL[{name!r}]()
g = frequencies.make_grid(w.omegas, w.dt)
kind = type(w.system).__name__
a = (W.hermite_gl_matrix(w.system) if kind == "Dense" else
     operators.gl1d(w.system) if kind == "GL1D" else
     operators.adr2d(w.system) if kind == "ADR2D" else operators.adv3d(w.system))
fh = W.test_block(w)
total, first, forced = march.schedule(g, w.variant, w.n_transient_windows, w.tail_steps)
steps = min({steps}, total)
t0 = time.perf_counter()
march.march(a, g, fh, variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps,
            real_state=w.real_state, stop_after=steps)
dt = time.perf_counter() - t0
print(json.dumps({{"seconds": dt, "steps": steps, "total_steps": int(total), "first": int(first)}}))
"""


def cpu_baseline(name: str, target_seconds: float = 15.0):
    w = workload(name)
    if w.n * w.k * w.n_omega > (1 << 31):
        return {"value": None, "unit": "actions/s", "cores": 1, "kind": "oracle",
                "sample": f"not run: the FP64 oracle would hold {w.n * w.k * w.n_omega * 16 / 2**30:.0f} GiB "
                          "of complex128 test block and accumulators on the host"}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    big = w.n * w.k * w.n_omega > (1 << 28)
    probe = 3 if big else (10 if type(w.system).__name__ in ("Dense", "ADV3D") else 100)
    r = subprocess.run([sys.executable, "-c", CPU_SNIPPET.format(root=ROOT, name=name, steps=probe)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per_step = d["seconds"] / d["steps"]
    steps = max(probe, min(d["total_steps"], int(target_seconds / per_step)))
    if steps > probe:
        r = subprocess.run([sys.executable, "-c", CPU_SNIPPET.format(root=ROOT, name=name, steps=steps)],
                           capture_output=True, text=True, env=env, timeout=900)
        if r.returncode != 0:
            return {"value": None, "error": r.stderr[-400:]}
        d = json.loads(r.stdout.strip().splitlines()[-1])
        per_step = d["seconds"] / d["steps"]
    # one march = total_steps steps and yields k * n_omega (* instances) actions
    march_s = per_step * d["total_steps"]
    actions = w.k * w.n_omega * n_instances(w)
    return {"value": actions / march_s, "unit": "actions/s", "cores": 1, "kind": "oracle",
            "sample": f"{d['steps']} of the {d['total_steps']} steps of one direct march of {w.name} "
                      f"(FP64 numpy oracle, one thread), extrapolated to the full march",
            "seconds": d["seconds"]}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def subspace_angle_max(ma, mb, segs):
    """Largest principal angle (radians) between span(ma[j, :, seg]) and span(mb[j, :, seg])."""
    worst = 0.0
    for j in range(ma.shape[0]):
        for off, ln in segs:
            qa, _ = np.linalg.qr(ma[j, :, off:off + ln].astype(np.complex128).T)
            qb, _ = np.linalg.qr(mb[j, :, off:off + ln].T)
            sv = np.linalg.svd(qa.conj().T @ qb, compute_uv=False)
            worst = max(worst, float(np.arccos(np.clip(sv.min(), -1.0, 1.0))))
    return worst


def fp64_single_vector(w, dense, omega_dev, opts, stream, n_t):
    """The plain comparator: the FP64 path marching one test vector (one direct march)."""
    import torch
    from paper_2008_10904_gb300 import rsv
    steps = (w.n_transient_windows + 1) * n_t if w.variant == "ssrm" else n_t + w.tail_steps
    cost = float(w.n) * w.n_omega * steps
    if cost > 5e11:
        return {"value": None, "unit": "actions/s",
                "impl": "FP64 GPU march, one test vector", "note": "not run: its FP64 CUDA-core forcing synthesis "
                f"alone would take tens of seconds ({cost:.1e} point-frequency-steps)"}
    op64 = rsv.create_for_workload(w, rsv.RSV_PREC_FP64, stream=stream.cuda_stream, dense_matrix=dense)
    x1 = omega_dev[:, :1, :].to(torch.complex128).contiguous()
    y1 = torch.empty_like(x1)
    ms = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rsv.rsv_march_direct(op64, x1, 1, y1, **opts)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    rsv.rsv_destroy_operator(op64)
    return {"value": w.n_omega * n_instances(w) / (ms[-1] / 1e3), "unit": "actions/s",
            "impl": "FP64 GPU march of one test vector (the library's FP64 path, k = 1), second of two runs",
            "ms_per_march": ms[-1]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2008_10904_gb300 import build as B
    from paper_2008_10904_gb300 import rsv

    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        dist.barrier()
    rsv.load()
    name = args.workload
    w = workload(name)
    prec_name = args.precision or default_precision(name)
    prec = rsv.RSV_PREC_FP64 if prec_name == "fp64" else rsv.RSV_PREC_FP32
    cdt = torch.complex128 if prec_name == "fp64" else torch.complex64
    dense = W.hermite_gl_matrix(w.system) if type(w.system).__name__ == "Dense" else None
    stream = torch.cuda.current_stream()
    op = rsv.create_for_workload(w, prec, stream=stream.cuda_stream, dense_matrix=dense)
    n_t, h = rsv.rsv_set_frequencies(op, w.omegas)
    path = rsv.rsv_describe(op)
    opts = rsv.march_opts_for(w, tile_steps=args.tile)
    big = w.n * w.k * w.n_omega > (1 << 29)
    if big:   # draw per frequency row straight into a pinned host block (no full complex128 copy)
        pinned = torch.empty((w.n_omega, w.k, w.n), dtype=torch.complex64, pin_memory=True)
        for j in range(w.n_omega):
            pinned[j].copy_(torch.from_numpy(W.test_block_row(w, j, seed_offset=rank_seed_offset(rank))))
        omega_dev = pinned.to(device="cuda", dtype=cdt)
    else:
        omega_host = W.test_block(w, seed_offset=rank_seed_offset(rank))
        omega_dev = torch.from_numpy(omega_host).to(device="cuda", dtype=cdt)
        pinned = torch.from_numpy(omega_host.astype(np.complex128 if prec_name == "fp64" else np.complex64)).pin_memory()
    ninst = n_instances(w)
    gains = np.zeros((ninst, w.n_omega, w.n_modes))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        rsv.rsv_gains_modes(op, omega_dev, w.k, w.n_power_iter, w.n_modes, gains, **opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timed region: device-resident inputs, L2 flushed between steps (outside the events)
    sampler = ClockSampler(local)
    sampler.start()
    rsv.rsv_profile_reset(op)
    rsv.rsv_profile_enable(op, True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    rsv.rsv_profile_enable(op, False)
    clocks = sampler.stop()
    prof = {c: rsv.rsv_profile_read(op, i) for i, c in enumerate(rsv.PROFILE_CATEGORIES)}  # (groups, kernels, ms)
    sec_max = max_over_ranks(total_ms / 1e3, device="cuda")
    value = job_throughput(actions_per_step(w) * args.steps, ws, sec_max)
    gains_timed = gains.copy()

    # end to end through the public API: pinned host test block in, gains on the host out
    h2d = pinned.numel() * pinned.element_size()
    d2h = gains.nbytes
    e2e_ms = 0.0
    for _ in range(max(1, args.steps)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        omega_dev.copy_(pinned, non_blocking=True)
        step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_sec = max_over_ranks(e2e_ms / 1e3, device="cuda")
    e2e_value = job_throughput(actions_per_step(w) * max(1, args.steps), ws, e2e_sec)

    # accuracy: the timed path's gains against the FP64 path (itself parity-tested against the oracle)
    acc = None
    if prec_name != "fp64" and not args.skip_accuracy and dense is None and w.n * w.k * w.n_omega < 2 ** 27:
        # response modes of both paths (untimed calls) for the subspace angle
        m32 = torch.empty((w.n_omega, w.n_modes, w.n), dtype=torch.complex64, device="cuda")
        g32 = np.zeros_like(gains)
        rsv.rsv_gains_modes(op, omega_dev, w.k, w.n_power_iter, w.n_modes, g32, response_modes=m32, **opts)
        op64 = rsv.create_for_workload(w, rsv.RSV_PREC_FP64, stream=stream.cuda_stream, dense_matrix=dense)
        g64 = np.zeros_like(gains)
        m64 = torch.empty((w.n_omega, w.n_modes, w.n), dtype=torch.complex128, device="cuda")
        rsv.rsv_gains_modes(op64, omega_dev.to(torch.complex128), w.k, w.n_power_iter, w.n_modes, g64,
                            response_modes=m64, **opts)
        segs = [rsv.rsv_instance_range(op64, i) for i in range(ninst)]
        rsv.rsv_destroy_operator(op64)
        acc = {"gain_rel_err_max": float(np.max(np.abs(gains_timed - g64) / np.abs(g64))),
               "subspace_angle_max_rad": subspace_angle_max(m32.cpu().numpy(), m64.cpu().numpy(), segs),
               "vs": "FP64 GPU path (parity-tested against the FP64 oracle to 1e-10)",
               "angle": f"largest principal angle between the leading-{w.n_modes} response-mode spans, "
                        "over frequencies and instances"}
    elif prec_name == "fp64":
        acc = {"gain_rel_err_max": 0.0, "vs": "FP64 path itself (parity-tested against the oracle to 1e-10)"}

    path = rsv.rsv_describe(op)   # now includes the tile / group sizes the marches used
    dom = max(prof, key=lambda c: prof[c][2])
    desc = dict(kv.split("=", 1) for kv in path.split() if "=" in kv)
    tile = int(desc.get("tile", args.tile or 256))
    rows = int(desc.get("group", w.k)) * w.n
    roof = kernel_model(dom, w, prec_name, tile, prof[dom][0], prof[dom][2], rows, path)
    launches = sum(v[1] for v in prof.values())
    steps_per_march = {"ssrm": (w.n_transient_windows + 1) * n_t, "trm": n_t + w.tail_steps}[w.variant]
    out = {
        "metric": METRIC, "value": value, "unit": "actions/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec_name == "fp64" else "f32",
        "data": "synthetic (seeded Gaussian test vectors, workload of the config)",
        "config": {"workload": w.name, "n": w.n, "k": w.k, "n_omega": w.n_omega, "variant": w.variant,
                   "steps_per_window": n_t, "h": h, "steps_per_march": steps_per_march,
                   "marches_per_step": marches_per_step(w), "actions_per_step": actions_per_step(w),
                   "power_iterations": w.n_power_iter, "precision": prec_name,
                   "l2": "flushed between steps (512 MiB write outside the timed events)",
                   "parallelism": f"independent replicas x{ws}", "path": path},
        "e2e": {"value": e2e_value, "unit": "actions/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernel_ms": {c: {"groups": v[0], "kernels": v[1], "ms": v[2]} for c, v in prof.items()},
        "roofline": roof,
        "clocks": clocks,
        "accuracy": acc,
    }
    rsv.rsv_destroy_operator(op)
    out["fp64_single_vector"] = (fp64_single_vector(w, dense, omega_dev, opts, stream, n_t)
                                 if args.comparator else None)
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(name)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    w = workload(name)
    vals = []
    for _ in range(args.warmup):          # untimed: the short probe march only
        cpu_baseline(name, target_seconds=0.0)
    t0 = time.perf_counter()
    last = None
    for _ in range(max(1, args.steps)):
        last = cpu_baseline(name, target_seconds=args.ref_seconds)
        if last.get("value"):
            vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals) if vals else None
    out = {"metric": METRIC, "value": v, "unit": "actions/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": w.name, "n": w.n, "k": w.k, "n_omega": w.n_omega, "variant": w.variant},
           "cpu_baseline": dict(last or {}, value=v),
           "e2e": {"value": v, "unit": "actions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(W.ALL), default="c2")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default=None)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--comparator", action="store_true",
                    help="also time the FP64 path marching one test vector (two direct marches, untimed in value)")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
