"""The allocation-free direct march against the allocating one and the oracle.

rsv_march_direct_static serves callers that cannot allocate device memory
after start-up (a host solver that reserves the device memory for its own
pool, a real-time loop that must not stall on the allocator): its scratch
is a static device array instead of library workspace.  Its result must
equal rsv_march_direct's within the parity tolerance, on consecutive calls
that reuse (and must re-clear) the shared array, for the steady-state
schedule and for a transient run with an unforced tail; it is also checked
against the oracle directly.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators
from parity import rel_rows

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5   # the FP32 march tolerance of the other parity tests (contractions may run on different units)


@pytest.mark.parametrize("variant", ["ssrm", "trm"])
@pytest.mark.parametrize("prec", [0, 1])
def test_static_scratch_march_matches_allocating_march(rsv, prec, variant):
    import torch
    w = W.small_gl(n=64, n_omega=8, k=3, n_trans=3, mu0=-0.1, variant=variant, tail_steps=700)
    op = rsv.create_for_workload(w, prec)
    try:
        cdt = torch.complex128 if prec == rsv.RSV_PREC_FP64 else torch.complex64
        fh = W.test_block(w)
        if prec == rsv.RSV_PREC_FP32:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = torch.from_numpy(fh).to(device="cuda", dtype=cdt)
        opts = rsv.march_opts_for(w, tile_steps=64)
        ref = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, ref, **opts)
        ref = ref.cpu().numpy()
        tol = TOL64 if prec == rsv.RSV_PREC_FP64 else TOL32
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            rsv.rsv_march_direct_static(op, x, w.k, y, **opts)
            got = y.cpu().numpy()
            assert rel_rows(got, ref) < tol
        # the oracle, on the same schedule
        g = frequencies.make_grid(w.omegas, w.dt)
        oref = march.march(operators.gl1d(w.system), g, fh, variant=variant, n_trans=w.n_transient_windows,
                           tail_steps=w.tail_steps)
        assert rel_rows(got.astype(np.complex128), oref) < tol
    finally:
        rsv.rsv_destroy_operator(op)


def test_static_scratch_rejects_tail_truncation(rsv):
    import torch
    w = W.small_gl(n=32, n_omega=4, k=1, variant="trm", tail_steps=100)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        x = torch.zeros((w.n_omega, w.k, w.n), dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct_static(op, x, w.k, y, variant="trm", tail_steps=100, tail_tol=1e-6)
        assert e.value.status == 1 and "tail_tol" in str(e.value)
    finally:
        rsv.rsv_destroy_operator(op)


def test_static_scratch_rejects_oversized_problem(rsv):
    import torch
    w = W.small_gl(n=1024, n_omega=256, k=32, n_trans=0, dt=0.5)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP32)
    try:
        x = torch.zeros((w.n_omega, w.k, w.n), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct_static(op, x, w.k, y, **rsv.march_opts_for(w))
        assert e.value.status == 1 and "static array holds" in str(e.value)
    finally:
        rsv.rsv_destroy_operator(op)
