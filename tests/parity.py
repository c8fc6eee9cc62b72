"""Error measures shared by the GPU parity tests.

Gains differ across frequencies by an order of magnitude or more (about 17x
between the strongest and weakest frequency of the 1-D workload), so every
comparison is normalised per frequency: an error in a weak frequency's row is
measured against that row, not against the block's largest entry.
"""
import numpy as np


def rel_rows(got, ref):
    """Largest per-frequency relative error of a coefficient block.

    Blocks are [n_omega][k][n]: for each frequency row j, max|got_j - ref_j| / max|ref_j|,
    and the largest over j.  A 2-D array is one row.
    """
    got = np.asarray(got)
    ref = np.asarray(ref)
    if ref.ndim < 3:
        return float(np.abs(got - ref).max() / np.abs(ref).max())
    m = ref.shape[0]
    num = np.abs(got - ref).reshape(m, -1).max(axis=1)
    den = np.abs(ref).reshape(m, -1).max(axis=1)
    return float((num / den).max())


def gain_rel(got, ref):
    """Largest relative error of individual gains (each gain against itself)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float((np.abs(got - ref) / np.abs(ref)).max())


def subspace_cos(a, b):
    """Smallest cosine of the principal angles between the row spaces of a and b (rows = vectors)."""
    qa, _ = np.linalg.qr(np.asarray(a, dtype=np.complex128).T)
    qb, _ = np.linalg.qr(np.asarray(b, dtype=np.complex128).T)
    return float(np.linalg.svd(qa.conj().T @ qb, compute_uv=False).min())
