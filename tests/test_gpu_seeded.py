"""GPU check of the seeded randomized SVD (rsv_gains_modes_seeded): the library draws the test block
from the SplitMix64 stream through the Box-Muller transform, and its gains equal the oracle's block
randomized SVD on the oracle's draw of the same seed (1e-10 in FP64, 1e-4 per gain in FP32)."""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, rsvd
from parity import gain_rel

pytestmark = pytest.mark.gpu


def _gl():
    return W.small_gl(n=48, n_omega=6, k=3, n_trans=4, mu0=-0.1), False


def _adr():
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4)
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_seeded", sysm, np.linspace(0.0, 4.0, 6), 0.5 * dx, 3, "ssrm", n_transient_windows=2,
                      real_state=True, seed=W.SEED_BASE + 81), True


@pytest.mark.parametrize("make,prec", [(_gl, 0), (_adr, 0), (_adr, 1)])
def test_seeded_rsvd_matches_oracle(rsv, make, prec):
    w, real = make()
    seed = 20081090
    op = rsv.create_for_workload(w, prec)
    try:
        opts = rsv.march_opts_for(w)
        gains = np.zeros((1, w.n_omega, 2))
        rsv.rsv_gains_modes_seeded(op, w.k, 1, 2, seed, gains, **opts)
        again = np.zeros_like(gains)
        rsv.rsv_gains_modes_seeded(op, w.k, 1, 2, seed, again, **opts)
        assert np.array_equal(gains, again)
        real_rows = [j for j, o in enumerate(w.omegas) if real and o == 0.0]
        om = rsvd.gaussian_test_block(seed, w.n_omega, w.k, w.n, real_rows=real_rows)
        a = operators.gl1d(w.system) if not real else operators.adr2d(w.system)
        g = frequencies.make_grid(w.omegas, w.dt)
        kw = dict(variant="ssrm", n_trans=w.n_transient_windows, real_state=real)
        md = lambda b: march.march(a, g, b, **kw)
        ma = lambda b: march.march(a, g, b, adjoint=True, **kw)
        ref, _, _ = rsvd.block_rsvd(md, ma, om, 1, 2, real_rows=real_rows)
        e = gain_rel(gains, ref)
        assert e < (1e-10 if prec == 0 else 1e-4), e
    finally:
        rsv.rsv_destroy_operator(op)
