"""Paper-scale resolution (Sec. 2.3 scaling relations, Table 1; Sec. 3 test model): Wendland C4
with support h, thousands of neighbours per particle, irregular (jittered) particles and
dispersivity ratios alpha_T/alpha_L down to 0.001, through the C ABI against the FP64 oracle.

Bars as for the ladder: max |gpu - oracle| / max |oracle| <= 1e-5 for dC/dt and for one step's
increment; in-support pair counts exact.
"""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu

RATE_TOL = 1e-5


@pytest.fixture(scope="module")
def lib(adelib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return adelib


def _args(plume, C):
    return (plume.velocity, np.asarray(C, dtype=np.float64), plume.mass, plume.rho, plume.boxv,
            plume.kernel, plume.support, plume.dim + 2.0, plume.alpha_L, plume.alpha_T, plume.D_m)


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("side,ratio", [(96, 0.1), (96, 0.001), (160, 0.01)])
def test_paper_scale_rate_parity(lib, orc, side, ratio):
    plume = inputs.paper_plume(side, ratio)
    xq, C = plume.initial_state()
    sim = lib.Simulation(lib.params_for(plume), xq, C)
    r, pairs = orc.rate(inputs.from_fixed(xq, plume.boxv), *_args(plume, C))
    assert pairs > 1000 * plume.n                       # thousands of neighbours per particle
    assert _rel(sim.rate().cpu().numpy(), r) <= RATE_TOL
    assert sim.count_pairs() == pairs


def test_paper_scale_one_step_parity(lib, orc):
    plume = inputs.paper_plume(96, 0.001)
    xq, C = plume.initial_state()
    sim = lib.Simulation(lib.params_for(plume), xq, C)
    assert sim.info.dt == plume.dt
    sim.step(1)
    xq1, C1 = sim.state()
    xo, Co, _ = orc.step(inputs.from_fixed(xq, plume.boxv), *_args(plume, C), plume.dt)
    dC_orc = Co - C
    tol = RATE_TOL * np.max(np.abs(dC_orc)) + np.max(np.abs(Co)) * 2.0 ** -24
    assert np.max(np.abs(C1.astype(np.float64) - C - dC_orc)) <= tol
    d = np.abs(inputs.from_fixed(xq1, plume.boxv) - xo)
    assert np.minimum(d, 1.0 - d).max() <= 2.0 ** -32


def test_paper_scale_1m_sampled(lib, orc):
    """Table 1's first row: 10^6 irregular particles, ~31,500 neighbours (h = 0.0999 L), in the
    launch configuration bench.py times (autotuned); sampled particles against the oracle."""
    plume = inputs.paper_plume(1000, 0.1)
    xq, C = plume.initial_state()
    sim = lib.Simulation(lib.params_for(plume), xq, C)
    sim.autotune()
    r = sim.rate().cpu().numpy()
    sel = np.random.default_rng(7).choice(plume.n, 1500, replace=False).astype(np.int32)
    r_orc, pairs = orc.rate_at(sel, inputs.from_fixed(xq, plume.boxv), *_args(plume, C))
    assert pairs > 30000 * sel.size
    assert np.max(np.abs(r[sel] - r_orc)) <= RATE_TOL * np.max(np.abs(r))


@pytest.mark.parametrize("k", [1, 3, 6])
def test_big_cells_bit_exact(lib, orc, k):
    """Wide kernels put hundreds of particles in a cell (about 440 per cell at one cell per support
    radius here), which the cell build orders warp-cooperatively: permutation and start table are
    still bit-exact against the oracle's stable counting sort."""
    plume = inputs.paper_plume(96, 0.1)
    xq, C = plume.initial_state()
    sim = lib.Simulation(lib.params_for(plume, cell_subdiv=k), xq, C)
    sim.build_cells()
    perm, cs = sim.cells()
    assert np.max(np.diff(cs)) > 32 or k > 1
    perm_o, cs_o = orc.sort_cells(orc.cell_keys(xq, np.array(sim.info.nc)), sim.info.ncells)
    assert np.array_equal(perm, perm_o) and np.array_equal(cs, cs_o)
    r, _ = orc.rate(inputs.from_fixed(xq, plume.boxv), *_args(plume, C))
    assert _rel(sim.rate().cpu().numpy(), r) <= RATE_TOL
