"""Decay run that sets the SSRM transient length (oracle).

Sec. 2.3: the time after which transients have vanished, so that the state
follows the periodic steady state, is estimated from a prior run in which
the norm of a random initial condition falls to a prescribed small value.
Here that run is the unforced RK4 march u_{s+1} = M u_s (the step of the
march module with zero forcing) from a seeded random state u_0:

  * it stops at the first check point s (every `check_every` steps) where
    ||u_s|| <= tol ||u_0||: the decay length is s steps;
  * a state that grows past `growth_limit` ||u_0||, or turns non-finite, at
    a check point marks the system as unstable: a stable system is what the
    method assumes (Sec. 2.1), and the norm of an unstable one never falls;
  * reaching `max_steps` without either is reported as well.

The SSRM then forces ceil(s / N_T) transient windows before the analysed
window of N_T steps.

The random initial state comes from a counter-based generator, SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value i of stream `seed` is mix64(seed + (i + 1) * G) with
G = 0x9E3779B97F4A7C15 and the finaliser

    z ^= z >> 30;  z *= 0xBF58476D1CE4E5B9
    z ^= z >> 27;  z *= 0x94D049BB133111EB
    z ^= z >> 31

(all arithmetic modulo 2**64).  Its top 53 bits give a double in [0, 1),
mapped to [-1, 1): u = 2 (z >> 11) 2**-53 - 1, exact in binary64.  A complex
state takes entry p = values 2p (real part) and 2p + 1 (imaginary part); a
real state takes entry p = value p.
"""
from __future__ import annotations

import math

import numpy as np

from . import march as _march

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Values 0 .. count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + i * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """count doubles in [-1, 1) from the top 53 bits of each SplitMix64 value."""
    z = splitmix64(seed, count) >> np.uint64(11)
    return 2.0 * z.astype(np.float64) * 2.0 ** -53 - 1.0


def initial_state(n: int, seed: int, complex_state: bool) -> np.ndarray:
    """The probe's random initial state (length n)."""
    if complex_state:
        v = uniform_pm1(seed, 2 * n)
        return v[0::2] + 1j * v[1::2]
    return uniform_pm1(seed, n)


def decay_probe(a, h: float, u0, tol: float, max_steps: int, check_every: int = 1,
                growth_limit: float = 1e6, instances=None):
    """Unforced RK4 march from u0 with step h until ||u|| <= tol ||u0|| at a check point.

    `instances` lists (offset, size) of the independent diagonal blocks of a
    batched system; the ratio is then the largest of the blocks' own ratios
    ||u_i|| / ||u0_i|| (every block must have decayed).
    Returns (steps, ratio, status): steps marched, the ratio there, and
    status "decayed", "grew" (ratio above growth_limit or non-finite at a check
    point) or "cap" (max_steps marched without either).
    """
    u = np.array(u0).reshape(-1, 1)
    segs = instances or [(0, u.shape[0])]
    n0 = [float(np.linalg.norm(u[o:o + s])) for o, s in segs]
    zero = np.zeros_like(u)
    ratio = 1.0
    for step in range(1, max_steps + 1):
        u = _march.rk4_step(a, u, h, zero, zero, zero)
        if step % check_every == 0 or step == max_steps:
            ratio = max(float(np.linalg.norm(u[o:o + s])) / n for (o, s), n in zip(segs, n0))
            if not math.isfinite(ratio) or ratio > growth_limit:
                return step, ratio, "grew"
            if ratio <= tol:
                return step, ratio, "decayed"
    return max_steps, ratio, "cap"


def transient_windows(decay_len: int, n_t: int) -> int:
    """SSRM transient windows covering a decay length of decay_len steps (windows of n_t steps)."""
    return -(-int(decay_len) // int(n_t))
