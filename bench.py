#!/usr/bin/env python
"""Benchmark: resolvent actions/s of the batched time march.

Default step (--step march): one march of the whole workload, alternately
direct and adjoint, followed by the CholeskyQR2 orthonormalisation of its
Fourier block per frequency: one half-iteration of the block power
iteration, so the step covers every stage of the method (twiddles,
synthesis, RK4 operator stages, streaming DFT, schedule, per-frequency block
algebra).  --step rsvd makes one step a whole randomized SVD through
rsv_gains_modes.  One resolvent action = one test vector x one frequency
through one march; a march step yields k x n_omega (x instances) actions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c4] [--step march|rsvd]
                  [--impl ours|reference]

The default workload is the 3-D boundary-layer system (256 x 128 x 128 x 3
state, 8 test vectors, 64 frequencies, steady-state method with three
transient windows): the largest configuration that fits one GPU.

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
import platform
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
ACC_FREQS = 4        # frequencies of the accuracy sample (the first ones of the grid)
ACC_K = 3            # test vectors of the accuracy sample (= the leading gains compared)


def marches_per_rsvd(w) -> int:
    return 2 * w.n_power_iter + 2


def n_instances(w) -> int:
    return len(w.system.n) if type(w.system).__name__ == "GL1D" else 1


def actions_per_march(w) -> int:
    return w.k * w.n_omega * n_instances(w)


def actions_per_step(w, step_kind="march") -> int:
    return actions_per_march(w) * (marches_per_rsvd(w) if step_kind == "rsvd" else 1)


def steps_per_march(w, n_t) -> int:
    return (w.n_transient_windows + 1) * n_t if w.variant == "ssrm" else n_t + w.tail_steps


def workload(name: str):
    return W.ALL[name]()


def default_precision(name: str) -> str:
    return "fp64" if name == "c1" else "fp32"


def big_block(w, k=None) -> bool:
    return w.n * (k or w.k) * w.n_omega > (1 << 29)


def sub_workload(w, omegas=None, k=None, n_power_iter=None):
    """The workload with fewer frequencies (the first ones of its grid: same window and step) or vectors."""
    return W.Workload(w.name, w.system, w.omegas if omegas is None else omegas, w.dt, k or w.k, w.variant,
                      n_transient_windows=w.n_transient_windows, tail_steps=w.tail_steps,
                      n_power_iter=w.n_power_iter if n_power_iter is None else n_power_iter, n_modes=w.n_modes,
                      real_state=w.real_state, seed=w.seed)


def seeded_block(w, k=None, seed_offset=0, dtype=None):
    """A seeded test block [n_omega][k][n] on the device.

    Small blocks are the workload's own (workloads.test_block, the inputs the oracle tests share).
    Blocks above 2^24 entries are drawn on the device by torch's seeded generator with the same
    distribution, (N(0,1) + i N(0,1)) / sqrt(2) per entry and a real N(0,1) row at w = 0 for
    real-state systems: drawing tens of GB of Gaussians on the host takes minutes.
    """
    import torch
    dtype = dtype or torch.complex64
    kk = k or w.k
    if w.n * kk * w.n_omega <= (1 << 24):
        return torch.from_numpy(W.test_block(w, k=kk, seed_offset=seed_offset)).to(device="cuda", dtype=dtype)
    g = torch.Generator(device="cuda")
    g.manual_seed(w.seed + seed_offset)
    x = torch.randn((w.n_omega, kk, w.n), dtype=dtype, device="cuda", generator=g)   # re, im ~ N(0, 1/2)
    for j, om in enumerate(w.omegas):
        if w.real_state and om == 0.0:
            x[j] = (x[j].real * math.sqrt(2.0)).to(dtype)
    return x


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
#   1-D march    gl1d_pack_c5.txt: one 127-step launch of the packed kernel (one wave of 152
#                CTAs x 3072 slots), 750.9 MB read + 340.2 MB written
#   2-D march    adr2d_pair_c3.txt: the two stage-pair kernels of one step at 16 vectors,
#                342.9 MB per step, scaled by 255 steps (traffic per step is constant)
#   3-D march    adv3d_pair_c4.txt: the two stage-pair kernels of one step at 2 vectors,
#                1347.6 MB per step, scaled by 255 steps
TRAFFIC = {
    ("dense_hermite_gl_n1024_k32_w256_trm", "march", 256, 32768):
        {"bytes": 108.98e6, "src": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"},
    ("gl_batch64_k8_w64_ssrm", "march", 127, 365184):
        {"bytes": 1.0911e9, "src": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"},
    ("adr2d_1024x512_k16_w128_ssrm", "march", 255, 8388608):
        {"bytes": 255 * 342.9e6, "src": "ncu dram bytes of the two stage-pair kernels of one step x 255 steps"},
    ("adv3d_256x128x128x3_k8_w64_ssrm", "march", 255, 25165824):
        {"bytes": 255 * 1347.6e6, "src": "ncu dram bytes of the two stage-pair kernels of one step x 255 steps"},
}

FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
REF_TOTAL_S = 150.0                                   # CPU seconds of the reference arm's timed steps
FP64_ALU_TFLOPS = 1.25                                # nominal FP64 rate of the part


def kernel_model(cat, w, prec, tile, groups, ms_total, rows, path):
    """Roofline record of one kernel category: algorithmic work per launch / average launch time.

    Units of work per launch (one time tile of S steps):
      synthesis  rows x n_omega x n_tau complex (8 flop) or real-output (4 flop) multiply-adds
      analysis   rows x n_omega x S multiply-adds (8 flop complex state, 4 flop real state)
      march      dense: 8 n^2 k flop per step (one dense complex product, tensor cores);
                 1-D kind (state held on chip for the whole tile): the forcing tile read
                 (2S+1 stage times), the snapshot tile written (S steps) and the state read
                 and written once, (3S + 3) state passes per tile; in FP64 (bound by the FP64
                 rate, not by bytes) 122 flop per point and step: four evaluations of
                 k = A x + f (three complex multiply-adds, 24 flop), the three stage inputs
                 u + c k (4 flop each) and the update u + h/6 (k1 + 2 k2 + 2 k3 + k4) (14 flop);
                 2-D whole-step kernel: 6 state passes per step (state read and written,
                 forcing read at the three stage times, snapshot written);
                 per-stage and stage-pair kernels (2-D, 3-D): 15 state passes per step, the
                 algorithmic model of one RK4 step (12 for four stage read/write pairs,
                 2 forcing reads, 1 snapshot write), whatever the kernels actually move
    """
    peaks = load_peaks()
    avg_s = ms_total / max(groups, 1) / 1e3
    S = tile
    dense = "kind=dense" in path
    se = (8 if prec == "fp64" else 4) * (1 if w.real_state else 2)
    alu_peak = FP64_ALU_TFLOPS if prec == "fp64" else FP32_ALU_TFLOPS
    cflop = 4 if w.real_state else 8
    tc_contract = "contractions=tcgen05" in path
    # kernels timed inside a step of seconds: the sustained bf16 rate x the nominal TF32/bf16 ratio
    peak_tc = peaks["bf16_tflops_sustained"] * 1.1 / 2.25
    tc_src = "measured sustained bf16 x nominal tf32/bf16 ratio (1.1/2.25)"
    if cat == "synthesis":
        n_tau = S if dense else 2 * S + 1
        work = rows * w.n_omega * n_tau * cflop
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if prec != "fp64" else "nominal FP64"
        if tc_contract:
            bound, peak, src = "tensor", peak_tc, tc_src
    elif cat == "analysis":
        work = rows * w.n_omega * S * cflop
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if prec != "fp64" else "nominal FP64"
        if tc_contract:
            bound, peak, src = "tensor", peak_tc, tc_src
    elif cat == "march" and dense and "tcgen05" in path:
        work = 8.0 * w.n * w.n * w.k * S
        peak = peak_tc
        bound, unit, per = "tensor", "TFLOP/s", 1e12
        src = tc_src + "; 3xTF32 split products counted once"
    elif cat == "march" and dense:
        work = 8.0 * w.n * w.n * w.k * S
        bound, unit, peak, per = "alu", "TFLOP/s", alu_peak, 1e12
        src = "derived FP32 CUDA-core rate"
    elif cat == "march" and "whole-step" in path:
        work = 6.0 * rows * se * S
        bound, unit, peak, per = "hbm", "GB/s", peaks["hbm_gbs"], 1e9
        src = peaks["src"] + " copy bandwidth"
    elif cat == "march" and "kind=gl1d" in path and prec == "fp64":
        work = 122.0 * rows * S
        bound, unit, peak, per = "alu", "TFLOP/s", FP64_ALU_TFLOPS, 1e12
        src = "nominal FP64"
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
# CPU baseline: the oracle on a bounded sample, in a subprocess
# ---------------------------------------------------------------------------
# The oracle marches k_s vectors for `steps` steps of the workload's schedule from the start;
# its cost per step is proportional to the vectors it carries, so the full march of k vectors
# is extrapolated as (seconds / steps) x steps_per_march x k / k_s.  Blocks too large for the
# host (the 3-D workload) march one vector whose single seeded row serves every frequency
# (the same work as distinct rows; drawing 64 rows of 12.6 M Gaussians would take a minute).
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import frequencies, march, operators
w = W.ALL[{name!r}]()
g = frequencies.make_grid(w.omegas, w.dt)
kind = type(w.system).__name__
a = (W.hermite_gl_matrix(w.system) if kind == "Dense" else
     operators.gl1d(w.system) if kind == "GL1D" else
     operators.adr2d(w.system) if kind == "ADR2D" else operators.adv3d(w.system))
ks = {k_sample}
if {one_row}:
    row = W.test_block_row(w, 0, k=ks).astype(np.complex128)
    if w.real_state:
        row = row.real.astype(np.complex128)
    fh = np.broadcast_to(row, (w.n_omega, ks, w.n))
else:
    fh = W.test_block(w, k=ks)
total, first, forced = march.schedule(g, w.variant, w.n_transient_windows, w.tail_steps)
steps = min({steps}, total)
secs = []
for r in range({warmup} + {repeats}):
    t0 = time.perf_counter()
    march.march(a, g, fh, variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps,
                real_state=w.real_state, stop_after=steps if r >= {warmup} else 0)
    secs.append(time.perf_counter() - t0)
print(json.dumps({{"seconds": secs[-1], "samples": secs[{warmup}:], "steps": steps, "total_steps": int(total),
                  "first": int(first)}}))
"""


def _oracle_sample(name, steps, k_sample, one_row, threads, warmup=0, repeats=1):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", CPU_SNIPPET.format(root=ROOT, name=name, steps=steps,
                                                                 k_sample=k_sample, one_row=one_row,
                                                                 warmup=warmup, repeats=repeats)],
                       capture_output=True, text=True, env=env, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-600:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model() -> str:
    """The host CPU's model name (x86: /proc/cpuinfo; Arm: lscpu), else the machine type."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_baseline(name: str, target_seconds: float = 15.0, warmup: int = 0, repeats: int = 1):
    """The oracle, as it stands, on the host's cores (BLAS threads), on a bounded sample of one march.

    A short probe sizes the sample to about target_seconds; with repeats > 1 the sample is timed
    that many times in one process (after `warmup` untimed runs of the oracle's set-up path, no
    steps) and `samples` lists each value.
    """
    w = workload(name)
    cores = os.cpu_count() or 1
    huge = w.n * w.k * w.n_omega > (1 << 28)
    k_sample = 1 if huge else w.k
    one_row = w.n * w.n_omega > (1 << 28)
    probe = 1 if huge else (10 if type(w.system).__name__ in ("Dense", "ADV3D") else 100)
    try:
        d = _oracle_sample(name, probe, k_sample, one_row, cores)
        steps = max(probe, min(d["total_steps"], int(target_seconds / (d["seconds"] / d["steps"]))))
        d = _oracle_sample(name, steps, k_sample, one_row, cores, warmup, repeats)
    except (RuntimeError, subprocess.TimeoutExpired) as e:
        return {"value": None, "unit": "actions/s", "cores": cores, "kind": "oracle", "error": str(e)[-400:]}
    per_step = d["seconds"] / d["steps"]
    scale = d["total_steps"] * (w.k / k_sample) / d["steps"]
    samples = [actions_per_march(w) / (t * scale) for t in d["samples"]]
    march_s = per_step * d["total_steps"] * (w.k / k_sample)
    sample = (f"{d['steps']} of the {d['total_steps']} steps of one direct march of {w.name} with "
              f"{k_sample} of its {w.k} test vectors (FP64 numpy/scipy oracle, {cores} BLAS threads; sparse "
              f"products single-threaded), extrapolated to the full march of all vectors")
    if one_row:
        sample += "; one seeded test-vector row serves every frequency (same work, fewer random draws)"
    return {"value": actions_per_march(w) / march_s, "unit": "actions/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "sample": sample, "seconds": d["seconds"], "samples": samples}


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


def accuracy_record(w, prec_name, dense, stream, rank):
    """Gain accuracy of the timed precision on a bounded sample of the workload.

    Sample: the full grid and schedule, the first ACC_FREQS frequencies (same window and step),
    ACC_K test vectors, no power iteration (Y = R Omega, Q = qr(Y), W = R^H Q, svd).  The FP32
    randomized SVD against the FP64 path's (itself parity-tested against the FP64 oracle to 1e-10)
    on the same test vectors: the leading gains' largest relative difference and the largest
    principal angle between the response-mode spans.
    """
    import torch
    from paper_2008_10904_gb300 import rsv
    if prec_name == "fp64":
        return {"gain_rel_err_max": 0.0, "vs": "FP64 path itself (parity-tested against the oracle to 1e-10)"}
    ws = sub_workload(w, omegas=w.omegas[:ACC_FREQS], k=ACC_K, n_power_iter=0)
    nm, ninst = ACC_K, n_instances(ws)
    x = seeded_block(ws, seed_offset=rank_seed_offset(rank), dtype=torch.complex128)
    opts = rsv.march_opts_for(ws)
    t0 = time.perf_counter()
    res = {}
    low = rsv.RSV_PREC_BF16_STATE if prec_name == "bf16" else rsv.RSV_PREC_FP32
    for prec, cdt in ((low, torch.complex64), (rsv.RSV_PREC_FP64, torch.complex128)):
        op = rsv.create_for_workload(ws, prec, stream=stream.cuda_stream, dense_matrix=dense)
        gains = np.zeros((ninst, ws.n_omega, nm))
        modes = torch.empty((ws.n_omega, nm, ws.n), dtype=cdt, device="cuda")
        rsv.rsv_gains_modes(op, x.to(cdt), ws.k, ws.n_power_iter, nm, gains, response_modes=modes, **opts)
        segs = [rsv.rsv_instance_range(op, i) for i in range(ninst)]
        rsv.rsv_destroy_operator(op)
        res[prec] = (gains, modes.cpu().numpy())
        del modes
    del x
    torch.cuda.empty_cache()
    g32, m32 = res[low]
    g64, m64 = res[rsv.RSV_PREC_FP64]
    return {"gain_rel_err_max": float(np.max(np.abs(g32 - g64) / np.abs(g64))),
            "subspace_angle_max_rad": subspace_angle_max(m32, m64, segs),
            "vs": "FP64 GPU path (parity-tested against the FP64 oracle to 1e-10), same test vectors",
            "sample": f"full grid and schedule, first {ws.n_omega} frequencies, {ws.k} test vectors, no power "
                      f"iteration, leading {nm} gains",
            "angle": f"largest principal angle between the leading-{nm} response-mode spans, over frequencies "
                     "and instances",
            "seconds": time.perf_counter() - t0}


def fp64_single_vector(w, dense, stream, n_t, rank):
    """The plain comparator: the library's FP64 path marching one test vector for all frequencies.

    Timed over one window of N_T steps (forced and analysed: SSRM with no transient window), the
    second of two runs, and scaled to the workload's steps per march.
    """
    import torch
    from paper_2008_10904_gb300 import rsv
    w1 = sub_workload(w, k=1)
    try:
        op64 = rsv.create_for_workload(w1, rsv.RSV_PREC_FP64, stream=stream.cuda_stream, dense_matrix=dense)
    except rsv.RsvError as e:
        return {"value": None, "note": f"not run: {e}"}
    x1 = seeded_block(w1, seed_offset=rank_seed_offset(rank), dtype=torch.complex128)
    y1 = torch.empty_like(x1)
    ms = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rsv.rsv_march_direct(op64, x1, 1, y1, variant="ssrm", n_transient_windows=0)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    rsv.rsv_destroy_operator(op64)
    del x1, y1
    torch.cuda.empty_cache()
    per_march_ms = ms[-1] * steps_per_march(w, n_t) / n_t
    return {"value": w.n_omega * n_instances(w) / (per_march_ms / 1e3), "unit": "actions/s",
            "impl": "FP64 GPU march of one test vector (the library's FP64 path, k = 1)",
            "sample": f"one window of {n_t} steps (second of two runs), scaled to {steps_per_march(w, n_t)} steps",
            "ms_per_march": per_march_ms}


def one_frequency_march(rsv, op, w, bufs, opts, stream, step_ms):
    """The frequencies one at a time (the cost the paper compares against, Sec. 2.4): one march of the
    same schedule with only the first frequency (same window and steps: the grid spacing is kept),
    timed after one untimed run, times n_omega, against the measured step (one march of all
    frequencies and its orthonormalisation)."""
    import torch
    dw = float(w.omegas[1] - w.omegas[0]) if w.n_omega > 1 else 0.0
    rsv.rsv_set_frequencies(op, w.omegas[:1], dw)
    x1 = bufs[0][:1].contiguous()
    y1 = torch.empty_like(x1)
    ms = 0.0
    for r in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rsv.rsv_march_direct(op, x1, w.k, y1, **opts)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    rsv.rsv_set_frequencies(op, w.omegas)
    all_ms = ms * w.n_omega
    return {"ms_per_single_frequency_march": ms, "ms_all_frequencies_one_at_a_time": all_ms,
            "value": w.k * w.n_omega / (all_ms / 1e3), "unit": "actions/s",
            "speedup_of_all_at_once": all_ms / step_ms,
            "sample": f"one march of frequency {w.omegas[0]:g} alone (same window and steps, {w.k} vectors), "
                      f"second of two runs, times {w.n_omega} frequencies"}


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
    prec = {"fp64": rsv.RSV_PREC_FP64, "fp32": rsv.RSV_PREC_FP32, "bf16": rsv.RSV_PREC_BF16_STATE}[prec_name]
    cdt = torch.complex128 if prec_name == "fp64" else torch.complex64
    dense = W.hermite_gl_matrix(w.system) if type(w.system).__name__ == "Dense" else None
    stream = torch.cuda.current_stream()
    op = rsv.create_for_workload(w, prec, stream=stream.cuda_stream, dense_matrix=dense)
    n_t, h = rsv.rsv_set_frequencies(op, w.omegas)
    opts = rsv.march_opts_for(w, tile_steps=args.tile)
    # the seeded test block, resident on the device and pinned on the host for the end-to-end runs
    x0 = seeded_block(w, seed_offset=rank_seed_offset(rank), dtype=cdt)
    pinned = torch.empty((w.n_omega, w.k, w.n), dtype=cdt, pin_memory=True)
    pinned.copy_(x0)
    bufs = [x0, None]
    ninst = n_instances(w)
    step_kind = args.step
    if step_kind == "march":
        bufs[1] = torch.empty_like(bufs[0])
        rfac = np.zeros((w.n_omega, ninst, w.k, w.k), dtype=np.complex128)
    gains = np.zeros((ninst, w.n_omega, w.n_modes))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    counter = [0]

    def step(read_r=False):
        """One step; read_r: also bring the step's result (R factors / gains) to the host."""
        if step_kind == "rsvd":
            rsv.rsv_gains_modes(op, bufs[0], w.k, w.n_power_iter, w.n_modes, gains, **opts)
            return
        i = counter[0]
        src, dst = bufs[i % 2], bufs[(i + 1) % 2]
        (rsv.rsv_march_adjoint if i % 2 else rsv.rsv_march_direct)(op, src, w.k, dst, **opts)
        rsv.rsv_orthonormalize(op, dst, w.k, rfac if read_r else None)
        counter[0] += 1

    # measured tile length and vector group (untimed): one timed tile per candidate configuration
    tuned = None
    if args.tile == 0 and not args.no_autotune:
        t_s, t_g = rsv.rsv_autotune(op, bufs[0], w.k, **opts)
        tuned = {"tile": t_s, "group": t_g, "chosen_by": "rsv_autotune: one timed tile per candidate "
                 "(default tile and half of it x groups of k, k/2, k/4, 1 that fit), least time per vector-step"}
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
    value = job_throughput(actions_per_step(w, step_kind) * args.steps, ws, sec_max)
    path = rsv.rsv_describe(op)   # includes the tile / group sizes the marches used

    # end to end through the public API: each step copies its input block from pinned host memory
    # and reads its result back (march step: the R factors of the orthonormalisation; rSVD: gains)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    h2d = pinned.numel() * pinned.element_size()
    d2h = rfac.nbytes if step_kind == "march" else gains.nbytes
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if step_kind == "rsvd":
            bufs[0].copy_(pinned, non_blocking=True)
            step(read_r=True)
        else:
            # the host-input march: per-vector-group copies on a second stream overlap the march
            i = counter[0]
            dst = bufs[(i + 1) % 2]
            (rsv.rsv_march_adjoint_host if i % 2 else rsv.rsv_march_direct_host)(op, pinned, w.k, dst, **opts)
            rsv.rsv_orthonormalize(op, dst, w.k, rfac)
            counter[0] += 1
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_sec = max_over_ranks(e2e_ms / 1e3, device="cuda")
    e2e_value = job_throughput(actions_per_step(w, step_kind) * e2e_steps, ws, e2e_sec)
    single = None
    if step_kind == "march" and not args.no_single_frequency:
        single = one_frequency_march(rsv, op, w, bufs, opts, stream, step_ms=total_ms / max(args.steps, 1))
    rsv.rsv_destroy_operator(op)
    del bufs, flush, pinned
    torch.cuda.empty_cache()

    dom = max(prof, key=lambda c: prof[c][2])
    desc = dict(kv.split("=", 1) for kv in path.split() if "=" in kv)
    tile = int(desc.get("tile", args.tile or 256))
    rows = int(desc.get("group", w.k)) * w.n
    roof = kernel_model(dom, w, prec_name, tile, prof[dom][0], prof[dom][2], rows, path)
    launches = sum(v[1] for v in prof.values())
    acc = None if args.skip_accuracy else accuracy_record(w, prec_name, dense, stream, rank)
    comp = None if args.no_comparator else fp64_single_vector(w, dense, stream, n_t, rank)
    out = {
        "metric": METRIC, "value": value, "unit": "actions/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "f32 (bf16 state storage)"}[prec_name],
        "data": "synthetic (seeded Gaussian test vectors, workload of the config)",
        "config": {"workload": w.name, "n": w.n, "k": w.k, "n_omega": w.n_omega, "variant": w.variant,
                   "steps_per_window": n_t, "h": h, "steps_per_march": steps_per_march(w, n_t),
                   "step": ("one march (alternately direct and adjoint) + CholeskyQR2 of its block per "
                            "frequency: half an iteration of the block power iteration"
                            if step_kind == "march" else "one randomized SVD (all marches + glue)"),
                   "actions_per_step": actions_per_step(w, step_kind),
                   "power_iterations": w.n_power_iter, "precision": prec_name,
                   "l2": "flushed between steps (512 MiB write outside the timed events); state blocks exceed L2",
                   "parallelism": f"independent replicas x{ws}", "path": path,
                   "tiles": tuned or {"chosen_by": "memory rule" if args.tile == 0 else f"--tile {args.tile}"}},
        "e2e": {"value": e2e_value, "unit": "actions/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "ms_per_step": e2e_ms / e2e_steps,
                "h2d": ("rsv_march_*_host: each vector group's slice copied from pinned memory on a second stream "
                        "while the previous group marches" if step_kind == "march" else
                        "one copy of the block from pinned memory before the step")},
        "gpu_launches": launches,
        "kernel_ms": {c: {"groups": v[0], "kernels": v[1], "ms": v[2]} for c, v in prof.items()},
        "roofline": roof,
        "clocks": clocks,
        "accuracy": acc,
        "fp64_single_vector": comp,
        "one_frequency_at_a_time": single,
    }
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(name, target_seconds=args.ref_seconds)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of one march of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    w = workload(name)
    t0 = time.perf_counter()
    # each step's sample: about --ref-seconds of CPU work, less when the K steps would exceed about
    # REF_TOTAL_S in all (never less than one step of the workload)
    per_step_s = min(args.ref_seconds, REF_TOTAL_S / max(1, args.steps))
    last = cpu_baseline(name, target_seconds=per_step_s, warmup=args.warmup, repeats=max(1, args.steps))
    wall = time.perf_counter() - t0
    vals = last.get("samples") or []
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
    ap.add_argument("--workload", choices=sorted(W.ALL), default="c4")
    ap.add_argument("--step", choices=["march", "rsvd"], default="march")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default=None,
                    help="bf16: the 3-D workload's march state stored in BF16 (arithmetic in FP32)")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true", help="keep the memory rule's tile and group")
    ap.add_argument("--no-single-frequency", action="store_true",
                    help="skip the one-frequency-at-a-time comparison march")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end measurement (<= --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--no-comparator", action="store_true",
                    help="skip the FP64 one-test-vector comparator (one window, scaled to a march)")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
