"""Writes precision_<case>.txt: the FP64 oracle's concentrations after the full run of each
configured plume, at a fixed seeded sample of particles, for the FP32-versus-FP64 drift check of
tests/test_gpu_precision.py.

Only the oracle and the seeded inputs are used.  Each run starts from the FP32-rounded initial
state the GPU library receives (Eq. 11 at the lattice positions) and takes the configured number
of predictor-corrector steps (Eq. 8-9; the rate Eq. 4-5 with the tensor of Eq. 3) at the time step
of the lambda_max rule (0.1 h^2 / lambda_max(D)), positions advanced in FP64.  Cases: the 64^2
plume (200 steps, every particle), the 256^2 ladder rung at alpha_L/alpha_T = 1, 10, 100 (1000
steps each) and the 3D plume on a 32^3 lattice with h = 2 dx (500 steps); 2048 sampled particles
for the last four.

Usage: python tests/golden/make_precision_golden.py [case ...]   (about ten minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2108_09488_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLE = 2048
SAMPLE_SEED = 4242


def cases():
    """name -> (plume, steps, sampled)"""
    return {
        "lattice64": (inputs.lattice_2d_64(), 200, False),
        "ladder256_r1": (inputs.ladder_2d(256, 1), 1000, True),
        "ladder256_r10": (inputs.ladder_2d(256, 10), 1000, True),
        "ladder256_r100": (inputs.ladder_2d(256, 100), 1000, True),
        "cube32": (inputs.cube_3d_128(side=32), 500, True),
    }


def sample_indices(n, sampled):
    if not sampled:
        return np.arange(n)
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, min(SAMPLE, n), replace=False))


def run(name, plume, steps, sampled):
    xq, C = plume.initial_state()
    x = inputs.from_fixed(xq, plume.boxv)
    D = oracle.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
    dt = oracle.dt_rule(D, plume.h)
    _, Cn, pairs = oracle.step(x, plume.velocity, C.astype(np.float64), plume.mass, plume.rho, plume.boxv,
                               plume.kernel, plume.support, plume.dim + 2.0, plume.alpha_L, plume.alpha_T,
                               plume.D_m, dt, nsteps=steps)
    idx = sample_indices(plume.n, sampled)
    path = os.path.join(HERE, f"precision_{name}.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle concentrations after the full run, written by tests/golden/make_precision_golden.py\n")
        f.write(f"# {plume.name}: {plume.n} particles, {steps} steps of Eq. 8-9 at dt = {dt!r}\n")
        f.write(f"steps {steps}\n")
        f.write(f"dt {dt!r}\n")
        f.write(f"linf_all {float(np.max(np.abs(Cn)))!r}\n")
        f.write(f"mass_all {float(np.sum(plume.mass * Cn))!r}\n")
        f.write("# index C\n")
        for i in idx:
            f.write(f"{int(i)} {float(Cn[i])!r}\n")
    return path


def main():
    oracle.build()
    want = sys.argv[1:] or list(cases())
    for name, (plume, steps, sampled) in cases().items():
        if name not in want:
            continue
        t0 = time.time()
        path = run(name, plume, steps, sampled)
        print(f"{name}: {path} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
