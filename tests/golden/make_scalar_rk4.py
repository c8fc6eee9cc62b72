"""Writes scalar_rk4_resolvent.txt: the steady-state response of one classical
RK4 step to periodic forcing, for scalar systems du/dt = lam u + e^{i w t}.

The value is derived here symbolically, from the four RK4 stage equations
themselves (forcing sampled at t_n, t_n + h/2, t_n + h) and the periodic
ansatz u_n = R e^{i w t_n}; nothing here uses the oracle's closed form or any
library code of this repository.  Re-run with `python tests/golden/make_scalar_rk4.py`.
"""
import os

import sympy as sp

lam, h, w, R, t = sp.symbols("lam h w R t", complex=True)
E = sp.exp(sp.I * w * t)
f = lambda tt: sp.exp(sp.I * w * tt)
u = R * E
k1 = lam * u + f(t)
k2 = lam * (u + h / 2 * k1) + f(t + h / 2)
k3 = lam * (u + h / 2 * k2) + f(t + h / 2)
k4 = lam * (u + h * k3) + f(t + h)
u_next = u + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
# periodic steady state: u_{n+1} = R e^{i w (t + h)}
eq = sp.expand(sp.simplify((u_next - R * f(t + h)) / E))
R_sol = sp.solve(sp.Eq(eq, 0), R)[0]

cases = [(-0.3 + 0.5j, 0.01, 0.7), (-0.1 - 0.2j, 0.05, -1.3), (-0.6, 0.2, 0.0),
         (-0.05 + 1.0j, 0.02, 1.0), (-2.0 + 0.0j, 0.1, 3.0), (-0.8 + 4.0j, 0.05, -4.0)]
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scalar_rk4_resolvent.txt")
with open(out, "w") as fh:
    fh.write("# Steady-state RK4 response R_h(w) of du/dt = lam u + e^{i w t} (Sec. 2.1 Eq. systemFreqDomain,\n")
    fh.write("# time-discretised by classical RK4 with the forcing sampled at t_n, t_n + h/2, t_n + h).\n")
    fh.write("# Derived symbolically from the stage equations by tests/golden/make_scalar_rk4.py (sympy, 30 digits).\n")
    fh.write("# columns: Re lam, Im lam, h, w, Re R_h, Im R_h\n")
    for l, hh, ww in cases:
        v = complex(sp.N(R_sol.subs({lam: l, h: hh, w: ww}), 30))
        fh.write(f"{l.real!r} {complex(l).imag!r} {hh!r} {ww!r} {v.real:.17e} {v.imag:.17e}\n")
print("wrote", out)
