"""The oracle's closed-form RK4 resolvent against stored values derived symbolically.

tests/golden/scalar_rk4_resolvent.txt holds R_h(w) for scalar systems
du/dt = lam u + e^{i w t} stepped by classical RK4 (Sec. 2.1 Eq.
systemFreqDomain, time-discretised), solved from the four stage equations
with sympy by tests/golden/make_scalar_rk4.py.  The oracle writes the same
map as (zI - M)^{-1}(h/6)G; a dropped term, a wrong stage weight or a
misplaced half-step phase in either shows up here.  The oracle's march is
pinned to that closed form in test_oracle_pins.py.
"""
import os

import numpy as np

from oracle import resolvent

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    out = []
    for ln in open(os.path.join(HERE, "golden", "scalar_rk4_resolvent.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        lr, li, h, w, rr, ri = (float(x) for x in ln.split())
        out.append((complex(lr, li), h, w, complex(rr, ri)))
    return out


def test_scalar_rk4_resolvent_matches_symbolic_derivation():
    rows = _rows()
    assert len(rows) == 6
    for lam, h, w, ref in rows:
        got = resolvent.rk4_discrete(np.array([[lam]]), w, h)[0, 0]
        assert abs(got - ref) <= 1e-12 * abs(ref), (lam, h, w, got, ref)


def test_diagonal_system_is_the_scalar_map_per_entry():
    """A diagonal A decouples into the scalar maps of the fixture."""
    rows = _rows()
    for h in sorted({r[1] for r in rows}):
        sel = [r for r in rows if r[1] == h]
        for lam, _, w, ref in sel:
            a = np.diag([lam, -1.0, lam])
            r = resolvent.rk4_discrete(a, w, h)
            assert abs(r[0, 0] - ref) <= 1e-12 * abs(ref) and abs(r[2, 2] - ref) <= 1e-12 * abs(ref)
            assert abs(r[0, 1]) == 0.0 and abs(r[2, 0]) == 0.0
