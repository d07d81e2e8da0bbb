"""Velocity-field mode (per-particle velocities, Eq. 1 and 3-5 with both terms of Eq. 4) through
the C ABI against the FP64 oracle on the same seeded inputs.

Bars: dC/dt and the step increment max |gpu - oracle| / max |oracle| <= 1e-5 (FP32 pair
arithmetic with compensated row sums, as for the uniform case); in-support pair counts exact;
positions within the fixed-point rounding of one increment per step (2^-32 of the box per step).
"""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu

RATE_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def lib(adelib, torch_cuda):
    return adelib


def _smooth(plume, xq, speed=0.1, amplitude=0.5, seed=2108):
    return inputs.velocity_field(inputs.from_fixed(xq, plume.boxv), plume.boxv, speed=speed,
                                 amplitude=amplitude, seed=seed)


def _shear(plume, xq, vmax, waves=4):
    """Divergence-free shear flow v = (0.999 vmax sin(2 pi waves y / L), 0): neighbours drift
    apart at up to ~vmax while C stays smooth (no compression term)."""
    y = inputs.from_fixed(xq, plume.boxv)[:, 1]
    v = np.zeros((plume.dim, plume.n))
    v[0] = 0.999 * vmax * np.sin(2.0 * np.pi * waves * y / plume.box)
    return np.ascontiguousarray(v.astype(np.float32))


def _mirror(plume, xq, speed=0.05):
    """Checkerboard of mirrored velocities (speed, +-speed): neighbours' off-diagonal D_xy are
    exact negatives, so the harmonic mean of Eq. 5 meets a zero denominator (K_xy = 0)."""
    n1 = plume.side
    i = np.arange(plume.n)
    sign = np.where(((i % n1) + (i // n1)) % 2 == 0, 1.0, -1.0)
    v = np.stack([np.full(plume.n, speed), sign * speed])
    return np.ascontiguousarray(v.astype(np.float32))


CASES = {
    # (plume, velocity generator, vmax)
    "2d-96-c2-smooth": (lambda: inputs.Plume(dim=2, side=96, h_over_dx=1.9, jitter=0.3, seed=11),
                        lambda p, xq: _smooth(p, xq), 0.2),
    "2d-100-c4-smooth": (lambda: inputs.Plume(dim=2, side=100, h_over_dx=4.245,
                                              kernel=inputs.WENDLAND_C4, jitter=0.2, seed=4),
                         lambda p, xq: _smooth(p, xq, amplitude=0.8, seed=5), 0.25),
    "3d-24-c2-smooth": (lambda: inputs.Plume(dim=3, side=24, h_over_dx=1.7, jitter=0.4, seed=5),
                        lambda p, xq: _smooth(p, xq, seed=9), 0.2),
    "2d-80-c2-noise": (lambda: inputs.Plume(dim=2, side=80, h_over_dx=1.6, jitter=0.25, seed=2,
                                            alpha_L=2e-3, alpha_T=1e-3),
                       lambda p, xq: inputs.velocity_noise(p.n, 2, 0.05, seed=3), 0.05),
    "2d-80-c2-shear": (lambda: inputs.Plume(dim=2, side=80, h_over_dx=1.6, jitter=0.25, seed=2,
                                            alpha_L=2e-3, alpha_T=1e-3),
                       lambda p, xq: _shear(p, xq, 0.05), 0.05),
    "2d-64-c2-mirror": (lambda: inputs.Plume(dim=2, side=64, h_over_dx=1.3),
                        lambda p, xq: _mirror(p, xq), 0.071),
}
CONVECTIVE = ("2d-96-c2-smooth", "2d-100-c4-smooth", "3d-24-c2-smooth", "2d-80-c2-noise")


def _setup(lib, name, **over):
    mk, vel, vmax = CASES[name]
    plume = mk()
    xq, C = plume.initial_state()
    v = vel(plume, xq)
    sim = lib.Simulation(lib.params_for(plume, vmax=vmax, **over), xq, C)
    sim.set_velocity_field(v)
    return plume, xq, C, v, sim


def _oracle_args(plume, v, C):
    return (np.ascontiguousarray(v.T, dtype=np.float64), np.asarray(C, dtype=np.float64),
            plume.mass, plume.rho, plume.boxv, plume.kernel, plume.support, plume.dim + 2.0,
            plume.alpha_L, plume.alpha_T, plume.D_m)


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_field_rate_parity(lib, orc, name):
    """Eq. 4 with per-particle D (harmonic means of Eq. 5) and the convective term."""
    plume, xq, C, v, sim = _setup(lib, name)
    x = inputs.from_fixed(xq, plume.boxv)
    r, rd, rc, pairs = orc.rate(x, *_oracle_args(plume, v, C), split=True)
    if name in CONVECTIVE:
        assert np.max(np.abs(rc)) > 0.02 * np.max(np.abs(r))  # the convective term is exercised
    assert _rel(sim.rate().cpu().numpy(), r) <= RATE_TOL
    assert sim.count_pairs() == pairs


@pytest.mark.parametrize("name", sorted(CASES))
def test_field_one_step_parity(lib, orc, name):
    """Eq. 8-9 with per-particle drift: the increment C^1 - C^0 and the positions."""
    plume, xq, C, v, sim = _setup(lib, name)
    dt = sim.info.dt
    sim.step(1)
    xq1, C1 = sim.state()
    x = inputs.from_fixed(xq, plume.boxv)
    xo, Co, _ = orc.step(x, *_oracle_args(plume, v, C), dt)
    dC_gpu = C1.astype(np.float64) - C
    dC_orc = Co - C
    tol = RATE_TOL * np.max(np.abs(dC_orc)) + np.max(np.abs(Co)) * 2.0 ** -24
    assert np.max(np.abs(dC_gpu - dC_orc)) <= tol
    d = np.abs(inputs.from_fixed(xq1, plume.boxv) - xo)
    d = np.minimum(d, 1.0 - d)
    assert d.max() <= 2.0 ** -32


def test_field_skin_covers_relative_drift(lib, orc):
    """A strong shear flow with dt vmax about half the support radius: pairs that come within H
    only at the half step (outside H at the cell build) exist, and the GPU steps still match the
    oracle, whose neighbour search runs at the evaluation positions."""
    name = "2d-80-c2-shear"
    plume, xq, C, v, sim = _setup(lib, name)
    info = sim.info
    assert info.skin > 0.4 * info.support
    x = inputs.from_fixed(xq, plume.boxv)
    xh = (x + 0.5 * info.dt * v.T.astype(np.float64)) % 1.0
    p0, i0 = orc.neighbours(x, plume.boxv, plume.support)
    ph, ih = orc.neighbours(xh, plume.boxv, plume.support)
    s0 = {(a, b) for a in range(plume.n) for b in i0[p0[a]:p0[a + 1]]}
    new = sum((a, b) not in s0 for a in range(plume.n) for b in ih[ph[a]:ph[a + 1]])
    assert new > 1000
    nsteps = 3
    sim.step(nsteps)
    xq3, C3 = sim.state()
    xo, Co, _ = orc.step(x, *_oracle_args(plume, v, C), info.dt, nsteps=nsteps)
    assert _rel(C3.astype(np.float64) - C, Co - C) <= 3 * RATE_TOL
    d = np.abs(inputs.from_fixed(xq3, plume.boxv) - xo)
    d = np.minimum(d, 1.0 - d)
    assert d.max() <= nsteps * 2.0 ** -32


def test_field_constant_velocity_matches_uniform_mode(lib):
    """A field with the same velocity everywhere: the convective term vanishes and the harmonic
    mean of equal tensors is 2D, so field mode reproduces the uniform-velocity kernel."""
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    v = np.ascontiguousarray(np.repeat(plume.velocity.astype(np.float32)[:, None], plume.n, 1))
    vmax = float(np.linalg.norm(plume.velocity.astype(np.float32).astype(np.float64))) * (1 + 1e-6)
    uni = lib.Simulation(lib.params_for(plume, cell_subdiv=3, flags=lib.FLAG_DIRECT), xq, C)
    fld = lib.Simulation(lib.params_for(plume, vmax=vmax, dt=uni.info.dt, cell_subdiv=3), xq, C)
    fld.set_velocity_field(v)
    r_u = uni.rate().cpu().numpy().astype(np.float64)
    assert _rel(fld.rate().cpu().numpy(), r_u) <= RATE_TOL
    assert fld.count_pairs() == uni.count_pairs()


def test_field_run_graph_equals_step_bitwise(lib):
    a = _setup(lib, "2d-96-c2-smooth")[4]
    b = _setup(lib, "2d-96-c2-smooth")[4]
    a.step(5)
    st = b.run(5)
    xa, Ca = a.state()
    xb, Cb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ca.view(np.uint32), Cb.view(np.uint32))
    assert st.step == 5 and st.status == 0
    # the statistics are the field corrector's folded per-warp partials
    C64 = Cb.astype(np.float64)
    assert st.c_min == C64.min() and st.c_max == C64.max()
    assert st.mass == pytest.approx(b.stats().mass, rel=1e-12)


def test_field_autotune_keeps_state_and_parity(lib, orc):
    plume, xq, C, v, sim = _setup(lib, "3d-24-c2-smooth")
    assert sim.autotune() > 0.0
    x1, C1 = sim.state()
    assert np.array_equal(x1, xq) and np.array_equal(C1.view(np.uint32), C.view(np.uint32))
    r, pairs = orc.rate(inputs.from_fixed(xq, plume.boxv), *_oracle_args(plume, v, C))
    assert _rel(sim.rate().cpu().numpy(), r) <= RATE_TOL
    assert sim.count_pairs() == pairs


def test_field_set_dispersivity_reforms_tensors(lib, orc):
    """ade_set_dispersivity in field mode: the per-particle tensors are re-formed before the next
    evaluation, for single calls and for a run whose graph is captured afterwards."""
    import dataclasses
    plume, xq, C, v, sim = _setup(lib, "3d-24-c2-smooth")
    sim.run(1)
    new = dataclasses.replace(plume, alpha_L=3e-2, alpha_T=2e-3, D_m=1e-5)
    sim.set_dispersivity(new.alpha_L, new.alpha_T, new.D_m)
    xq1, C1 = sim.state()
    r, _ = orc.rate(inputs.from_fixed(xq1, plume.boxv), *_oracle_args(new, v, C1))
    assert _rel(sim.rate().cpu().numpy(), r) <= RATE_TOL
    ref = _setup(lib, "3d-24-c2-smooth")[4]
    ref.run(1)
    ref.set_dispersivity(new.alpha_L, new.alpha_T, new.D_m)
    ref.step(2)
    sim.run(2)
    xa, Ca = sim.state()
    xb, Cb = ref.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ca.view(np.uint32), Cb.view(np.uint32))


def test_field_rejects_fast_or_nonfinite_velocities(lib):
    plume, xq, C, v, sim = _setup(lib, "2d-96-c2-smooth")
    fast = v.copy()
    fast[0, 17] = 0.25                            # |v| > vmax = 0.2
    with pytest.raises(lib.AdeError) as e:
        sim.set_velocity_field(fast)
    assert e.value.code == -1
    with pytest.raises(lib.AdeError) as e:       # no field any more
        sim.step(1)
    assert e.value.code == -6
    bad = v.copy()
    bad[1, 5] = np.nan
    with pytest.raises(lib.AdeError) as e:
        sim.set_velocity_field(bad)
    assert e.value.code == -1
    sim.set_velocity_field(v)
    sim.step(1)
    assert sim.stats().status == 0


def test_field_empty_particle_set(lib):
    plume = inputs.Plume(dim=2, side=64, h_over_dx=1.3)
    sim = lib.Simulation(lib.params_for(plume, vmax=0.2), np.zeros((2, 0), np.uint32),
                         np.zeros(0, np.float32))
    sim.set_velocity_field(np.zeros((2, 0), np.float32))
    sim.step(2)
    assert sim.count_pairs() == 0


def test_field_full_size_sampled(lib, orc):
    """The 1024^2 ladder rung (120 neighbours) under the smooth field: sampled particles against
    the oracle, exact pair count at the lattice positions."""
    plume = inputs.ladder_2d(1024, 10)
    xq, C = plume.initial_state()
    v = _smooth(plume, xq)
    sim = lib.Simulation(lib.params_for(plume, vmax=0.2), xq, C)
    sim.set_velocity_field(v)
    sim.autotune()
    r = sim.rate().cpu().numpy()
    sel = np.random.default_rng(1).choice(plume.n, 3000, replace=False).astype(np.int32)
    r_orc, pairs = orc.rate_at(sel, inputs.from_fixed(xq, plume.boxv), *_oracle_args(plume, v, C))
    assert np.max(np.abs(r[sel] - r_orc)) <= RATE_TOL * np.max(np.abs(r))
    assert pairs == 3000 * 120
    assert sim.count_pairs() == plume.n * 120

