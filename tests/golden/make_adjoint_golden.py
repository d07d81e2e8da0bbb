"""Writes adjoint_512_400.txt: FP64 oracle values for the dispersivity-inversion problem at its
configured size (2D 512^2 lattice, h = 1.3 dx, Wendland C2, 400 steps of Eq. 8-9 at a fixed dt).

Only the oracle and the seeded inputs are used.  The target field C* is the oracle's state after
400 steps with theta* = (alpha_L, alpha_T, D_m) = (2e-2, 2e-3, 1e-6), rounded to FP32 (the
precision the GPU library receives it in); the misfit is J = 1/2 sum_a (C_a^N - C*_a)^2 at
theta = (1e-2, 1e-3, 1e-6).  Recorded: dt, J, dJ/dtheta by the oracle's tangent-linear model, and
dJ/dtheta by FP64 central differences with eps = 1e-4 theta_k.  The dispersion tensor is Eq. 3, the
rate Eq. 4-5 and the step Eq. 8-9 (Sec. 2); the inversion problem is derived from them (the paper
has no adjoint).

Usage: python tests/golden/make_adjoint_golden.py   (a few minutes on a multi-core host)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2108_09488_gb300 import inputs  # noqa: E402

THETA = np.array([1e-2, 1e-3, 1e-6])
THETA_STAR = np.array([2e-2, 2e-3, 1e-6])
SIDE, H_DX, NSTEPS = 512, 1.3, 400
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_512_400.txt")


def problem():
    """The plume, its FP64 positions and C^0, the oracle keyword arguments and the FP32 target."""
    p = inputs.Plume(dim=2, side=SIDE, h_over_dx=H_DX, alpha_L=THETA[0], alpha_T=THETA[1], D_m=THETA[2])
    xq, C = p.initial_state()
    x = inputs.from_fixed(xq, p.boxv)
    D = oracle.dispersion_tensor(p.velocity, *THETA)
    dt = oracle.dt_rule(D, p.h)
    kw = dict(m=p.mass, rho=1.0, box=p.boxv, kind=0, H=p.support, gamma=4.0, dt=dt, nsteps=NSTEPS)
    _, Cstar = oracle.misfit(x, p.velocity, C.astype(np.float64), theta=THETA_STAR, target=np.zeros(p.n), **kw)
    target = Cstar.astype(np.float32).astype(np.float64)
    return p, x, C, kw, target


def main():
    oracle.build()
    t0 = time.time()
    p, x, C, kw, target = problem()
    C0 = C.astype(np.float64)
    J, g = oracle.misfit_gradient_tlm(x, p.velocity, C0, theta=THETA, target=target, **kw)
    fd = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-4 * THETA[k]
        Jp, _ = oracle.misfit(x, p.velocity, C0, theta=THETA + e, target=target, **kw)
        Jm, _ = oracle.misfit(x, p.velocity, C0, theta=THETA - e, target=target, **kw)
        fd.append((Jp - Jm) / (2 * e[k]))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle values, written by tests/golden/make_adjoint_golden.py (see its docstring)\n")
        f.write(f"# 2D {SIDE}^2 lattice, h = {H_DX} dx, Wendland C2, {NSTEPS} steps of Eq. 8-9; theta = "
                f"{[float(t) for t in THETA]}, theta* = {[float(t) for t in THETA_STAR]}; target rounded to FP32\n")
        f.write(f"dt {kw['dt']!r}\n")
        f.write(f"J {J!r}\n")
        f.write("grad_tlm " + " ".join(repr(float(v)) for v in g) + "\n")
        f.write("grad_fd " + " ".join(repr(float(v)) for v in fd) + "\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s: J={J!r} tlm={g} fd={fd}")


if __name__ == "__main__":
    main()
