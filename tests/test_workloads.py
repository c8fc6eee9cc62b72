"""The seeded input generators (shared by the oracle tests and the GPU path; no method arithmetic)."""
import numpy as np

import workloads as W


def test_test_block_is_seeded_and_shaped():
    w = W.small_gl(n=40, n_omega=8, k=3)
    a, b = W.test_block(w), W.test_block(w)
    assert a.shape == (8, 3, 40) and a.dtype == np.complex128
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.test_block(w, seed_offset=1000))   # bench ranks differ
    # unit-variance complex Gaussian entries
    assert abs(np.mean(np.abs(a) ** 2) - 1.0) < 0.2


def test_real_state_zero_frequency_row_is_real():
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4)
    w = W.Workload("adr", sysm, np.linspace(0.0, 4.0, 8), 0.5, 2, "ssrm", real_state=True)
    blk = W.test_block(w)
    assert np.all(blk[0].imag == 0.0) and np.any(blk[1].imag != 0.0)
    row0 = W.test_block_row(w, 0)
    assert row0.dtype == np.complex64 and np.all(row0.imag == 0.0)


def test_row_generator_is_seeded_per_row():
    w = W.small_gl(n=40, n_omega=8, k=3)
    r3 = W.test_block_row(w, 3)
    assert r3.shape == (3, 40)
    assert np.array_equal(r3, W.test_block_row(w, 3))
    assert not np.array_equal(r3, W.test_block_row(w, 4))
    allrows = np.stack([W.test_block_row(w, j) for j in range(8)])
    assert abs(np.mean(np.abs(allrows) ** 2) - 1.0) < 0.2
