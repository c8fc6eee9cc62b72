"""The allocation-free direct march against the allocating one.

rsv_march_direct_static serves callers that cannot allocate device memory
after start-up (a fixed memory budget, a thread recording a CUDA stream
capture, a real-time loop): its scratch is a static device array instead of
library workspace.  Its result must equal rsv_march_direct's within the
parity tolerance, on consecutive calls that reuse (and must re-clear) the
shared array.  This file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5   # the FP32 march tolerance of the other parity tests (contractions may run on different units)


@pytest.mark.parametrize("prec", [0, 1])
def test_static_scratch_march_matches_allocating_march(rsv, prec):
    import torch
    w = W.small_gl(n=64, n_omega=8, k=3, n_trans=3, mu0=-0.1)
    op = rsv.create_for_workload(w, prec)
    try:
        cdt = torch.complex128 if prec == rsv.RSV_PREC_FP64 else torch.complex64
        x = torch.from_numpy(W.test_block(w)).to(device="cuda", dtype=cdt)
        opts = rsv.march_opts_for(w, tile_steps=64)
        ref = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, ref, **opts)
        ref = ref.cpu().numpy()
        tol = TOL64 if prec == rsv.RSV_PREC_FP64 else TOL32
        for _ in range(2):
            y = torch.full_like(x, float("nan"))
            rsv.rsv_march_direct_static(op, x, w.k, y, **opts)
            got = y.cpu().numpy()
            assert np.abs(got - ref).max() / np.abs(ref).max() < tol
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
