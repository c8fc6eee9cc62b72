"""GPU parity of the TRM record truncated by the state norm (Sec. 2.2) against the oracle.

With tail_tol > 0 the library ends the unforced tail at the first tile end, at
or after the end of the forcing window, where every vector's norm is at most
tail_tol times its largest tile-end norm so far.  The oracle applies the same
rule at the same check points (multiples of the tile length), so both stop
after the same number of steps and the Fourier coefficients agree element by
element (FP64 1e-10, FP32 2e-5).  The truncation error itself against the
closed-form resolvent is pinned on the oracle in tests/test_oracle_pins.py.
"""
import numpy as np
import pytest

import workloads as W
from parity import gain_rel, rel_rows
from oracle import frequencies, march, operators

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 2e-5}


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)




def _case(kind):
    if kind == "gl1d":
        w = W.small_gl(n=40, n_omega=8, k=3, variant="trm", tail_steps=0, mu0=-0.1)
        return w, operators.gl1d(w.system), None, 50
    if kind == "dense":
        sysm = W.Dense(n=48, x_half_width=20.0)
        w = W.Workload("dense_tail", sysm, np.linspace(-1.0, 1.0, 8), 0.02, 3, "trm")
        a = W.hermite_gl_matrix(sysm)
        return w, a, a, 64
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4, visc=0.05)   # abscissa -0.026
    dx = sysm.lx / (sysm.nx + 1)
    w = W.Workload("adr_tail", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, 2, "trm", real_state=True,
                   seed=W.SEED_BASE + 36)
    return w, operators.adr2d(sysm), None, 40


@pytest.mark.parametrize("kind", ["gl1d", "dense", "adr2d"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_trm_norm_truncated_tail(rsv, kind, prec, adjoint):
    w, a, dense, tile = _case(kind)
    g = frequencies.make_grid(w.omegas, w.dt)
    cap, tol = 400 * g.n_t, 1e-6
    op = rsv.create_for_workload(w, prec, dense_matrix=dense)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, variant="trm", tail_steps=cap, tile_steps=tile, tail_tol=tol)
        desc = dict(kv.split("=", 1) for kv in rsv.rsv_describe(op).split() if "=" in kv)
        ref, steps = march.march(a, g, fh, variant="trm", tail_steps=cap, adjoint=adjoint, real_state=w.real_state,
                                 tail_tol=tol, check_every=tile, return_steps=True)
        assert g.n_t <= steps < g.n_t + cap           # the rule ended the tail before the cap
        assert int(desc["steps"]) == steps
        assert rel_rows(y.cpu().numpy().astype(np.complex128), ref) < TOL[prec]
    finally:
        rsv.rsv_destroy_operator(op)


def test_tail_tol_rejected_when_negative(rsv):
    w, _, _, _ = _case("gl1d")
    op = rsv.create_for_workload(w, 0)
    try:
        x = _dev(W.test_block(w), 0)
        with pytest.raises(RuntimeError):
            rsv.rsv_march_direct(op, x, w.k, x * 0, variant="trm", tail_steps=100, tail_tol=-1.0)
    finally:
        rsv.rsv_destroy_operator(op)
