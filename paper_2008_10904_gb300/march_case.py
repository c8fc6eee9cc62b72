"""One direct (or adjoint) march of a named workload, for profilers.

  python -m paper_2008_10904_gb300.march_case --workload c3 [--k 16] [--n-omega 8] [--tile 16]
         [--precision fp32|fp64|bf16] [--adjoint] [--repeat 2] [--full-schedule]

Runs the workload's operator through rsv_march_direct / rsv_march_adjoint
with a seeded Gaussian test block drawn on the device, optionally cut to
fewer test vectors (--k) and fewer frequencies (--n-omega: the first M of the
workload's grid, so the window length and step count per window stay those
of the full workload).  By default the schedule is one forced window (TRM
with no tail); --full-schedule uses the workload's own SSRM / TRM schedule.
The last repetition runs with the per-category kernel profiler on and one
JSON line is printed: the path description, steps per window, and per
category (synthesis / march / analysis / glue) the tile groups, kernels
launched and milliseconds.  Nothing here is checked against anything: the
parity tests do that.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--n-omega", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--precision", choices=["fp32", "fp64", "bf16"], default="fp32")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--full-schedule", action="store_true")
    args = ap.parse_args(argv)

    import torch
    import workloads as W
    from paper_2008_10904_gb300 import build, rsv

    build.build()
    rsv.load()
    full = W.ALL[args.workload]()
    k = args.k or full.k
    om = full.omegas[:args.n_omega] if args.n_omega else full.omegas
    if args.full_schedule:
        w = W.Workload(full.name, full.system, om, full.dt, k, full.variant,
                       n_transient_windows=full.n_transient_windows, tail_steps=full.tail_steps,
                       real_state=full.real_state, seed=full.seed)
    else:
        w = W.Workload(full.name, full.system, om, full.dt, k, "trm", tail_steps=0,
                       real_state=full.real_state, seed=full.seed)
    prec = {"fp32": rsv.RSV_PREC_FP32, "fp64": rsv.RSV_PREC_FP64, "bf16": rsv.RSV_PREC_BF16_STATE}[args.precision]
    cdt = torch.complex128 if args.precision == "fp64" else torch.complex64
    dense = W.hermite_gl_matrix(w.system) if type(w.system).__name__ == "Dense" else None
    op = rsv.create_for_workload(w, prec, dense_matrix=dense)
    n_t, h = rsv.rsv_set_frequencies(op, w.omegas)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.seed)
    x = torch.randn((w.n_omega, k, w.n), dtype=cdt, device="cuda", generator=gen)
    if w.real_state and w.omegas[0] == 0.0:
        x[0] = x[0].real.to(cdt)      # the zero frequency of a real march carries a real coefficient
    y = torch.empty_like(x)
    opts = rsv.march_opts_for(w, tile_steps=args.tile)
    march = rsv.rsv_march_adjoint if args.adjoint else rsv.rsv_march_direct
    for r in range(max(1, args.repeat)):
        last = r == max(1, args.repeat) - 1
        if last:
            torch.cuda.synchronize()
            rsv.rsv_profile_reset(op)
            rsv.rsv_profile_enable(op, True)
        march(op, x, k, y, **opts)
        torch.cuda.synchronize()
    rsv.rsv_profile_enable(op, False)
    prof = {c: rsv.rsv_profile_read(op, i) for i, c in enumerate(rsv.PROFILE_CATEGORIES)}
    print(json.dumps({"workload": w.name, "n": w.n, "k": k, "n_omega": w.n_omega, "steps_per_window": n_t,
                      "h": h, "adjoint": args.adjoint, "path": rsv.rsv_describe(op),
                      "kernel_ms": {c: {"groups": v[0], "kernels": v[1], "ms": v[2]} for c, v in prof.items()}}),
          flush=True)
    rsv.rsv_destroy_operator(op)


if __name__ == "__main__":
    main()
