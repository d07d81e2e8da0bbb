"""Cattaneo's hyperbolic form (Eq. 14) through the C ABI against the oracle's FP64 Cattaneo step.

The GPU state is (x, C, Q) with Q = dC/dt the relaxing flux; the oracle's step is pinned in
tests/test_oracle_cattaneo.py.  Bars: C increments and Q within 1e-5 of the largest oracle value
(plus one FP32 rounding of C); positions within 2^-32 of the box per step.
"""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu

RATE_TOL = 1e-5
VARIANTS = {"direct": 1, "tiled": 2, "branched": 4, "paired": 17}


@pytest.fixture(scope="module")
def lib(adelib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return adelib


def _args(plume):
    return (plume.mass, plume.rho, plume.boxv, plume.kernel, plume.support, plume.dim + 2.0,
            plume.alpha_L, plume.alpha_T, plume.D_m)


def _oracle(orc, plume, xq, C, Q, dt, tau, nsteps):
    x = inputs.from_fixed(xq, plume.boxv)
    return orc.step_cattaneo(x, plume.velocity, C.astype(np.float64), Q, *_args(plume), dt, tau,
                             nsteps=nsteps)


def _check(plume, C, xq_g, C_g, Q_g, xo, Co, Qo, nsteps):
    dC = Co - C
    tol = RATE_TOL * np.max(np.abs(dC)) + nsteps * np.max(np.abs(Co)) * 2.0 ** -24
    assert np.max(np.abs(C_g.astype(np.float64) - C - dC)) <= tol
    assert np.max(np.abs(Q_g.astype(np.float64) - Qo)) <= RATE_TOL * np.max(np.abs(Qo))
    d = np.abs(inputs.from_fixed(xq_g, plume.boxv) - xo)
    assert np.minimum(d, 1.0 - d).max() <= nsteps * 2.0 ** -32


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_cattaneo_fickian_flux_steps(lib, orc, variant):
    """Q(0) = R(C(0)) computed on the GPU (ade_set_flux with NULL), three steps, tau = 2 dt, for
    every interaction variant (the update lives in their shared epilogue)."""
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    D = orc.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
    tau = 2.0 * orc.dt_rule(D, plume.h)
    sim = lib.Simulation(lib.params_for(plume, tau=tau, flags=VARIANTS[variant]), xq, C)
    assert sim.info.dt == pytest.approx(orc.dt_rule(D, plume.h), rel=1e-14)
    sim.set_flux()
    Q0 = sim.flux().cpu().numpy().astype(np.float64)
    r0, _ = orc.rate(inputs.from_fixed(xq, plume.boxv), plume.velocity, C.astype(np.float64),
                     *_args(plume))
    assert np.max(np.abs(Q0 - r0)) <= RATE_TOL * np.max(np.abs(r0))
    sim.step(3)
    xq3, C3 = sim.state()
    Q3 = sim.flux().cpu().numpy()
    xo, Co, Qo, _ = _oracle(orc, plume, xq, C, Q0, sim.info.dt, tau, 3)
    _check(plume, C, xq3, C3, Q3, xo, Co, Qo, 3)


def test_cattaneo_given_flux_3d_c4_and_dt_cap(lib, orc):
    """A given flux (Q(0) = 0: the plume starts at rest) in 3D with the C4 kernel; tau below the
    parabolic step caps dt at tau."""
    plume = inputs.Plume(dim=3, side=24, h_over_dx=2.9, kernel=inputs.WENDLAND_C4, jitter=0.3, seed=6)
    xq, C = plume.initial_state()
    D = orc.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
    tau = 0.5 * orc.dt_rule(D, plume.h)
    sim = lib.Simulation(lib.params_for(plume, tau=tau), xq, C)
    assert sim.info.dt == tau
    Q0 = np.zeros(plume.n, dtype=np.float32)
    sim.set_flux(Q0)
    sim.step(4)
    xq4, C4 = sim.state()
    xo, Co, Qo, _ = _oracle(orc, plume, xq, C, Q0.astype(np.float64), sim.info.dt, tau, 4)
    _check(plume, C, xq4, C4, sim.flux().cpu().numpy(), xo, Co, Qo, 4)


def test_cattaneo_graph_replay_mass_and_state_checks(lib):
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    p = lib.params_for(plume, tau=1e-3)
    a = lib.Simulation(p, xq, C)
    b = lib.Simulation(p, xq, C)
    with pytest.raises(lib.AdeError) as e:       # no flux yet
        a.step(1)
    assert e.value.code == -6
    a.set_flux()
    b.set_flux()
    m0 = a.stats().mass
    a.step(10)
    st = b.run(10)
    xa, Ca = a.state()
    xb, Cb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ca.view(np.uint32), Cb.view(np.uint32))
    assert np.array_equal(a.flux().cpu().numpy().view(np.uint32), b.flux().cpu().numpy().view(np.uint32))
    assert st.status == 0 and abs(st.mass - m0) <= 1e-6 * m0       # sum Q(0) = 0 conserves mass
    assert st.c_min == Cb.astype(np.float64).min() and st.c_max == Cb.astype(np.float64).max()


def test_cattaneo_small_tau_approaches_fick(lib):
    """Over a fixed time with Q(0) = R(C(0)), Cattaneo's C approaches the Fickian run as tau
    shrinks (both on the GPU with the same dt)."""
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    fick = lib.Simulation(lib.params_for(plume, flags=lib.FLAG_DIRECT), xq, C)
    dt = fick.info.dt / 8
    fick.close()
    fick = lib.Simulation(lib.params_for(plume, dt=dt, flags=lib.FLAG_DIRECT), xq, C)
    fick.step(64)
    _, Cf = fick.state()
    diffs = []
    for tau in (4 * dt, dt):
        sim = lib.Simulation(lib.params_for(plume, dt=dt, tau=tau, flags=lib.FLAG_DIRECT), xq, C)
        sim.set_flux()
        sim.step(64)
        _, Cc = sim.state()
        diffs.append(np.max(np.abs(Cc.astype(np.float64) - Cf)) / np.max(np.abs(Cf.astype(np.float64) - C)))
    assert diffs[1] < diffs[0] < 0.2
    assert 2.5 < diffs[0] / diffs[1] < 5.5
