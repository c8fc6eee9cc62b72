"""Host-side helpers of bench.py that need no GPU."""
import numpy as np

import bench


def test_subspace_angle_of_bench():
    """bench.subspace_angle_max: zero for the same span (any basis, any phase), the known angle
    for a rotated span, per instance segment."""
    rng = np.random.default_rng(5)
    n, m = 40, 3
    a = rng.standard_normal((2, m, n)) + 1j * rng.standard_normal((2, m, n))
    mix = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    b = np.einsum("jmn,mk->jkn", a, mix) * np.exp(0.7j)            # same spans, other basis
    segs = [(0, 25), (25, 15)]
    assert bench.subspace_angle_max(a, b, segs) < 1e-6
    # rotate one basis vector of one segment by theta out of the span
    theta = 0.3
    q, _ = np.linalg.qr(a[0, :, 0:25].T)
    perp = rng.standard_normal(25) + 0j
    perp -= q @ (q.conj().T @ perp)
    perp /= np.linalg.norm(perp)
    c = b.copy()
    c[0, :, 0:25] = np.stack([q[:, 0] * np.cos(theta) + perp * np.sin(theta), q[:, 1], q[:, 2]])
    assert abs(bench.subspace_angle_max(a, c, segs) - theta) < 1e-9
