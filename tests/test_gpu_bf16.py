"""GPU checks of the BF16-state march (RSV_PREC_BF16_STATE, 3-D kind) against the FP64 oracle.

BF16 keeps 8 significant bits: every stored state or stage value is rounded
to within 2^-8 (3.9e-3) of itself, four times per step, and the system
carries those errors for as long as it remembers (a random walk over its
decay time).  The test's tolerance comes from that arithmetic, evaluated
for this case: a numpy march of the same scheme whose stored state and stage
inputs are rounded to BF16 (round to nearest even) gives the expected error
level against the oracle, and the GPU march must stay within three times it
(rounding order differs; measured, the two agree to three digits).  Gains:
the randomized SVD on BF16 state inherits errors of that order in its basis;
one FP64 refinement pass cuts the gain error severalfold but not to 1e-4.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators
from parity import gain_rel, rel_rows

pytestmark = pytest.mark.gpu


def _case(k=2):
    sysm = W.ADV3D(nx=24, ny=12, nz=12, lx=20.0, ly=10.0, lz=10.0, visc=0.02)
    dx = sysm.lx / (sysm.nx + 1)
    om = np.array([0.04 * np.pi * 5 * j for j in range(6)])
    return W.Workload("adv_bf16", sysm, om, 0.5 * dx, k, "ssrm", n_transient_windows=2, real_state=True,
                      seed=W.SEED_BASE + 46)


def _bf16(x):
    """Round to BF16 (nearest even) and back to float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    r = ((b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _emulated_bf16_march(a, g, fh, n_trans):
    """The RK4 scheme with the state and the stage inputs stored in BF16 (accumulator in FP32)."""
    om = g.omegas
    wts = np.where(om == 0.0, 1.0, 2.0)
    nom, kk, n = fh.shape
    h = g.h
    u = np.zeros((n, kk))
    out = np.zeros((nom, kk, n), dtype=np.complex128)
    total, first = (n_trans + 1) * g.n_t, n_trans * g.n_t
    syn = lambda t: march.synthesize(fh, om, t, True, wts)
    f32 = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)
    for s in range(total):
        t = s * h
        if s >= first:
            out += np.exp(-1j * om * t)[:, None, None] * u.T[None]
        f0, fm, f1 = syn(t), syn(t + 0.5 * h), syn(t + h)
        k1 = a @ u + f0
        x = _bf16(u + 0.5 * h * k1)
        acc = f32(u + h / 6 * k1)
        k2 = a @ x + fm
        x = _bf16(u + 0.5 * h * k2)
        acc = f32(acc + h / 3 * k2)
        k3 = a @ x + fm
        x = _bf16(u + h * k3)
        acc = f32(acc + h / 3 * k3)
        k4 = a @ x + f1
        u = _bf16(acc + h / 6 * k4)
    return out / g.n_t


@pytest.mark.parametrize("adjoint", [False, True])
def test_bf16_state_march_within_derived_tolerance(rsv, adjoint):
    import torch
    w = _case()
    a = operators.adv3d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_BF16_STATE)
    try:
        assert "bf16" in rsv.rsv_describe(op)
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = torch.from_numpy(fh).to(device="cuda", dtype=torch.complex64)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w, 32))
        aa = a.T.tocsr() if adjoint else a
        kw = dict(variant="ssrm", n_trans=w.n_transient_windows, real_state=True)
        ref = march.march(a, g, fh, adjoint=adjoint, **kw)
        if adjoint:
            gneg = frequencies.make_grid(-w.omegas, w.dt, dw=g.dw)
            emu = _emulated_bf16_march(aa, gneg, fh, w.n_transient_windows)
        else:
            emu = _emulated_bf16_march(aa, g, fh, w.n_transient_windows)
        e_emu = rel_rows(emu, ref)
        e_gpu = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        print(f"BF16 state: emulated {e_emu:.2e}, GPU {e_gpu:.2e}")
        assert 1e-5 < e_emu < 0.1
        assert e_gpu < 3.0 * e_emu, (e_gpu, e_emu)
    finally:
        rsv.rsv_destroy_operator(op)


def test_bf16_rsvd_refined_in_fp64(rsv):
    """Randomized SVD on BF16 state (12 vectors, 8 power iterations), then one FP64 refinement pass
    on its forcing basis, against the FP64 path's refinement of its own rSVD basis.  The BF16 march
    errors of a few percent leave the BF16 basis far from the leading singular subspace (measured:
    gains 0.35 off); the Rayleigh-Ritz pass squares the basis error and cuts the gain error more than
    fivefold (measured: 0.03), but BF16 state does not reach the 1e-4 accuracy target here."""
    import torch
    w = _case(k=12)
    opts = rsv.march_opts_for(w, 32)
    x = torch.from_numpy(W.test_block(w)).cuda()
    res = {}
    for name, prec, cdt in (("bf16", rsv.RSV_PREC_BF16_STATE, torch.complex64),
                            ("fp64", rsv.RSV_PREC_FP64, torch.complex128)):
        op = rsv.create_for_workload(w, prec)
        try:
            g = np.zeros((1, w.n_omega, w.k))
            v = torch.empty((w.n_omega, w.k, w.n), dtype=cdt, device="cuda")
            rsv.rsv_gains_modes(op, x.to(cdt), w.k, 8, w.k, g, forcing_modes=v, **opts)
            res[name] = (g[:, :, :3], v.to(torch.complex128).contiguous())
        finally:
            rsv.rsv_destroy_operator(op)
    op64 = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        refined = {}
        for name in ("bf16", "fp64"):
            gr = np.zeros((1, w.n_omega, 3))
            rsv.rsv_refine_gains(op64, res[name][1], w.k, 3, gr, **opts)
            refined[name] = gr
    finally:
        rsv.rsv_destroy_operator(op64)
    e_raw = gain_rel(res["bf16"][0], refined["fp64"])
    e_ref = gain_rel(refined["bf16"], refined["fp64"])
    print(f"BF16 rSVD gain error {e_raw:.2e}, after FP64 refinement {e_ref:.2e}")
    assert e_ref < 0.2 * e_raw
