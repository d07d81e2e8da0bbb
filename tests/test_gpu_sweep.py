"""Parameter sweep (many dispersivity sets on one plume sharing the particles, the uniform
velocity and the time step) through the C ABI against the FP64 oracle, one oracle run per set.

Bars as for the single plume: dC/dt and the step increment max |gpu - oracle| / max |oracle| <= 1e-5
per set; pair counts exact; graph replay bitwise equal to plain steps.
"""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu

RATE_TOL = 1e-5

# 11 sets: groups of 8, 2 and 1 launches; isotropic, alpha_L < alpha_T, large D_m, all zero
THETA = np.array([[1e-2, 1e-3, 1e-6], [1e-3, 1e-3, 1e-6], [1e-1, 1e-3, 0.0], [2e-2, 2e-3, 1e-6],
                  [1e-3, 1e-2, 1e-6], [5e-3, 5e-4, 1e-4], [0.0, 0.0, 0.0], [3e-2, 1e-4, 1e-6],
                  [1e-2, 1e-2, 0.0], [4e-2, 4e-3, 1e-5], [7e-3, 7e-5, 1e-6]])


@pytest.fixture(scope="module")
def lib(adelib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return adelib


def _fields(plume, xq, P):
    """P different seeded Gaussian plumes (Eq. 11) on the same particles."""
    x = inputs.from_fixed(xq, plume.boxv)
    rng = np.random.default_rng(11)
    out = []
    for _ in range(P):
        x0 = rng.uniform(0.2, 0.8, size=plume.dim)
        out.append(inputs.gaussian_plume(x, plume.boxv, x0, rng.uniform(0.04, 0.08)))
    return np.array(out, dtype=np.float32)


def _oracle_rate(orc, plume, xq, C, th):
    return orc.rate(inputs.from_fixed(xq, plume.boxv), plume.velocity, C.astype(np.float64), plume.mass,
                    plume.rho, plume.boxv, plume.kernel, plume.support, plume.dim + 2.0, *th)


def _rel(a, b):
    b = np.asarray(b, np.float64)
    m = np.max(np.abs(b))
    return 0.0 if m == 0 else float(np.max(np.abs(np.asarray(a, np.float64) - b)) / m)


CASES = {
    "2d-256-ladder": (lambda: inputs.ladder_2d(256, 10), THETA),
    "2d-96-c4-jitter": (lambda: inputs.Plume(dim=2, side=96, h_over_dx=4.245, kernel=inputs.WENDLAND_C4,
                                             jitter=0.3, seed=4), THETA[:6]),
    "3d-24-jitter": (lambda: inputs.Plume(dim=3, side=24, h_over_dx=1.7, jitter=0.4, seed=5), THETA[:3]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sweep_rate_parity(lib, orc, name):
    mk, theta = CASES[name]
    plume = mk()
    xq, _ = plume.initial_state()
    C = _fields(plume, xq, len(theta))
    sw = lib.Sweep(lib.params_for(plume), xq, C, theta)
    r = sw.rate().cpu().numpy()
    pairs_set = None
    for k, th in enumerate(theta):
        r_o, pairs = _oracle_rate(orc, plume, xq, C[k], th)
        if not np.any(th):
            assert np.all(r[k] == 0.0)
        else:
            assert _rel(r[k], r_o) <= RATE_TOL, k
        pairs_set = pairs
    assert sw.count_pairs() == pairs_set


def test_sweep_one_step_parity_and_common_dt(lib, orc):
    plume = inputs.ladder_2d(256, 10)
    xq, _ = plume.initial_state()
    theta = THETA[:5]
    C = _fields(plume, xq, len(theta))
    sw = lib.Sweep(lib.params_for(plume), xq, C, theta)
    dts = [orc.dt_rule(orc.dispersion_tensor(plume.velocity, *th), plume.h) for th in theta if np.any(th)]
    assert sw.info.dt == pytest.approx(min(dts), rel=1e-14)
    sw.step(1)
    xq1, C1 = sw.state()
    x = inputs.from_fixed(xq, plume.boxv)
    for k, th in enumerate(theta):
        xo, Co, _ = orc.step(x, plume.velocity, C[k].astype(np.float64), plume.mass, plume.rho, plume.boxv,
                             plume.kernel, plume.support, 4.0, *th, sw.info.dt)
        dC = Co - C[k]
        tol = RATE_TOL * np.max(np.abs(dC)) + np.max(np.abs(Co)) * 2.0 ** -24
        assert np.max(np.abs(C1[k].astype(np.float64) - C[k] - dC)) <= tol, k
    d = np.abs(inputs.from_fixed(xq1, plume.boxv) - xo)
    assert np.minimum(d, 1.0 - d).max() <= 2.0 ** -32


def test_sweep_run_graph_equals_step_bitwise_and_stats(lib):
    plume = inputs.ladder_2d(256, 10)
    xq, _ = plume.initial_state()
    C = _fields(plume, xq, len(THETA))
    a = lib.Sweep(lib.params_for(plume), xq, C, THETA)
    b = lib.Sweep(lib.params_for(plume), xq, C, THETA)
    a.step(6)
    b.run(6)
    xa, Ca = a.state()
    xb, Cb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ca.view(np.uint32), Cb.view(np.uint32))
    st = b.stats()
    for k in range(len(THETA)):
        c = Cb[k].astype(np.float64)
        assert st[k].mass == pytest.approx(plume.mass * c.sum(), rel=1e-12)
        assert st[k].c_min == c.min() and st[k].c_max == c.max() and st[k].status == 0
    # count, the one-pass scan, place, order; the sets' gather; 2 per group (3 groups)
    assert a.launches_per_step() == 4 + 1 + 2 * 3


def test_sweep_matches_single_plume_contexts(lib):
    """Each set of the sweep against a single-plume context with the same parameters and dt (a
    different arithmetic for Dcal: Kc form vs a u + b), two steps."""
    plume = inputs.ladder_2d(256, 10)
    xq, _ = plume.initial_state()
    theta = THETA[[0, 2, 4]]
    C = _fields(plume, xq, len(theta))
    sw = lib.Sweep(lib.params_for(plume, cell_subdiv=3), xq, C, theta)
    sw.step(2)
    _, Cs = sw.state()
    for k, th in enumerate(theta):
        sim = lib.Simulation(lib.params_for(plume, alpha_L=th[0], alpha_T=th[1], D_m=th[2], dt=sw.info.dt,
                                            cell_subdiv=3, flags=lib.FLAG_DIRECT), xq, C[k])
        sim.step(2)
        _, Ck = sim.state()
        dC = Ck.astype(np.float64) - C[k]
        # both sides round C to FP32 after each of the two steps
        tol = 2 * RATE_TOL * np.max(np.abs(dC)) + 4 * np.max(np.abs(C[k])) * 2.0 ** -24
        assert np.max(np.abs(Cs[k].astype(np.float64) - C[k] - dC)) <= tol, k
        sim.close()
