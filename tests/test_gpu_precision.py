"""FP32 against FP64 over whole runs: the configured plumes (64^2 for 200 steps, the 256^2 ladder
rung at alpha_L/alpha_T = 1, 10, 100 for 1000 steps, the 3D plume on a 32^3 lattice for 500 steps)
run through the C ABI and are compared with the FP64 oracle's run of the same steps, stored by
tests/golden/make_precision_golden.py at a fixed sample of particles (all of them at 64^2).

Reported (pytest -s): the relative drift max|C_gpu - C_oracle| / max|C_oracle| after the full run,
and the relative change of the total solute sum m C on the GPU.  The drift is gated by the FP32
rounding budget of the update: each step rounds C^{l+1/2} and C^{l+1} to FP32, at most
2 * 2^-24 of max|C| per step, and the FP32 rate adds at most 1e-5 of the step's increment, which
is far smaller; added up linearly over the steps that gives steps * 2^-23.  The solute sum is
conserved exactly by Eq. 4's antisymmetric pair terms in exact arithmetic (Sec. 2.2), so its
relative change is gated by the same per-step FP32 budget.
"""
import os

import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = {
    "lattice64": inputs.lattice_2d_64,
    "ladder256_r1": lambda: inputs.ladder_2d(256, 1),
    "ladder256_r10": lambda: inputs.ladder_2d(256, 10),
    "ladder256_r100": lambda: inputs.ladder_2d(256, 100),
    "cube32": lambda: inputs.cube_3d_128(side=32),
}
# walks: the library's default choice and the paired branch-free walk over trimmed rows
WALKS = {"default": {}, "paired-trimmed": {"flags": 25}}


def _golden(name):
    g = {"idx": [], "C": []}
    with open(os.path.join(HERE, "golden", f"precision_{name}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            a, b = line.split()
            if a in ("steps", "dt", "linf_all", "mass_all"):
                g[a] = float(b)
            else:
                g["idx"].append(int(a))
                g["C"].append(float(b))
    g["idx"] = np.array(g["idx"])
    g["C"] = np.array(g["C"])
    return g


@pytest.fixture(scope="module")
def lib(adelib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return adelib


@pytest.mark.parametrize("walk", sorted(WALKS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_full_run_drift_against_fp64_oracle(lib, name, walk):
    import torch
    plume = CASES[name]()
    g = _golden(name)
    steps = int(g["steps"])
    xq, C = plume.initial_state()
    sim = lib.Simulation(lib.params_for(plume, dt=g["dt"], **WALKS[walk]), xq, C)
    assert sim.info.dt == g["dt"]
    m0 = sim.stats().mass
    sim.run(steps, stats=False)
    torch.cuda.synchronize()
    st = sim.stats()
    Cg = sim.C.cpu().numpy().astype(np.float64)
    drift = float(np.max(np.abs(Cg[g["idx"]] - g["C"])) / g["linf_all"])
    mass_change = (st.mass - m0) / m0
    budget = steps * 2.0 ** -23
    print(f"\n{name} [{walk}]: {steps} steps, drift vs FP64 oracle {drift:.3e} (budget {budget:.1e}), "
          f"mass change {mass_change:.3e}, C_min {st.c_min:.3e}")
    assert st.status == 0
    assert drift <= budget
    assert abs(mass_change) <= budget
    sim.close()
