"""GPU parity: libade_sph.so (through its C ABI) against the FP64 oracle on the same seeded inputs.

Bars (written in each test):
  * cell lists (permutation and cell start table): bit-exact;
  * dC/dt and one step: max |gpu - oracle| / max |oracle| <= 1e-5 (FP32 pair arithmetic with
    compensated accumulation against FP64);
  * in-support pair counts: exact;
  * FP64 reductions and closed-form norms on the device: <= 1e-12 relative to numpy / the oracle.
"""
import math

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


def _sim(lib, plume, xq=None, C=None, **over):
    if xq is None:
        xq, C = plume.initial_state()
    return lib.Simulation(lib.params_for(plume, **over), xq, C)


def _oracle_rate(orc, plume, xq, C, sel=None):
    x = inputs.from_fixed(xq, plume.boxv)
    args = (plume.velocity, np.asarray(C, dtype=np.float64), plume.mass, plume.rho, plume.boxv,
            plume.kernel, plume.support, plume.dim + 2.0, plume.alpha_L, plume.alpha_T, plume.D_m)
    if sel is None:
        return orc.rate(x, *args)
    return orc.rate_at(sel, x, *args)


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / np.max(np.abs(b)))


def _plume(dim=2, side=64, h_dx=1.3, **kw):
    return inputs.Plume(dim=dim, side=side, h_over_dx=h_dx, **kw)


CASES = {
    "64sq-h1.3": lambda: inputs.lattice_2d_64(),
    "256sq-n28-r1": lambda: inputs.ladder_2d(256, 1),
    "256sq-n28-r100": lambda: inputs.ladder_2d(256, 100),
    "512sq-n60-r10": lambda: inputs.ladder_2d(512, 10),
    "3d-32cube-h2": lambda: inputs.cube_3d_128(side=32),
    "c4-96sq": lambda: _plume(side=96, h_dx=4.245, kernel=inputs.WENDLAND_C4),
    "jitter-100sq": lambda: _plume(side=100, h_dx=1.9, jitter=0.45, seed=3, angle=2.1),
    "3d-jitter-24": lambda: _plume(dim=3, side=24, h_dx=1.7, jitter=0.4, seed=5),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_cells_bit_exact(lib, orc, name):
    plume = CASES[name]()
    sim = _sim(lib, plume)
    sim.build_cells()
    perm, cs = sim.cells()
    xq, _ = plume.initial_state()
    nc = np.array(sim.info.nc)
    key = orc.cell_keys(xq, nc)
    perm_o, cs_o = orc.sort_cells(key, sim.info.ncells)
    assert np.array_equal(perm, perm_o)
    assert np.array_equal(cs, cs_o)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_cells_bit_exact_every_subdivision(lib, orc, k):
    """Random positions, n not a multiple of the sort tile (ragged tail), every grid choice."""
    rng = np.random.default_rng(k)
    n = 3 * 4096 + 777
    plume = _plume(side=128, h_dx=2.0)
    xq = rng.integers(0, 2 ** 32, size=(2, n), dtype=np.uint64).astype(np.uint32)
    C = rng.uniform(size=n).astype(np.float32)
    sim = _sim(lib, plume, xq, C, cell_subdiv=k)
    sim.build_cells()
    perm, cs = sim.cells()
    key = orc.cell_keys(xq, np.array(sim.info.nc))
    perm_o, cs_o = orc.sort_cells(key, sim.info.ncells)
    assert np.array_equal(perm, perm_o) and np.array_equal(cs, cs_o)


@pytest.mark.parametrize("order", ["lattice", "shuffled"])
def test_cells_bit_exact_many_scan_tiles(lib, orc, order):
    """A sparse 3D grid of 240^3 = 13.8 M cells (thousands of one-pass scan tiles) over 512,000
    particles, in lattice order (a block's particles in one or two tiles) and in a seeded shuffled
    order (every warp's particles spread over many tiles), bit-exact against the oracle's counting
    sort; built twice, so the second build runs on the counts and tile totals the first one
    cleared."""
    plume = _plume(dim=3, side=80, h_dx=1.0)
    xq, C = plume.initial_state()
    if order == "shuffled":
        p = np.random.default_rng(11).permutation(xq.shape[1])
        xq, C = np.ascontiguousarray(xq[:, p]), np.ascontiguousarray(C[p])
    sim = _sim(lib, plume, xq, C, cell_subdiv=6)
    assert sim.info.ncells == 240 ** 3
    key = orc.cell_keys(xq, np.array(sim.info.nc))
    perm_o, cs_o = orc.sort_cells(key, sim.info.ncells)
    for _ in range(2):
        sim.build_cells()
        perm, cs = sim.cells()
        assert np.array_equal(perm, perm_o) and np.array_equal(cs, cs_o)


# ADE_FLAG_TILED, _DIRECT, _BRANCHED, the two direct walks with _TRIMMED rows, and the _PAIRED
# branch-free walk (full and trimmed rows)
VARIANTS = {"tiled": 2, "direct": 1, "branched": 4, "direct-trimmed": 9, "branched-trimmed": 12,
            "paired": 17, "paired-trimmed": 25, "paired-branched": 20, "paired-branched-trimmed": 28}


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_rate_parity(lib, orc, name, variant):
    plume = CASES[name]()
    xq, C = plume.initial_state()
    sim = _sim(lib, plume, flags=VARIANTS[variant])
    if variant == "direct":
        assert sim.info.variant == 0
    if variant == "branched":
        assert sim.info.variant == 2
    if variant.startswith("paired"):
        assert sim.info.variant == {"paired": 5, "paired-trimmed": 6, "paired-branched": 7,
                                    "paired-branched-trimmed": 8}[variant]
    r_gpu = sim.rate().cpu().numpy()
    r_orc, pairs = _oracle_rate(orc, plume, xq, C)
    assert _rel(r_gpu, r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs


def test_tiled_variant_is_used_and_deterministic(lib):
    plume = inputs.ladder_2d(512, 10)
    a = _sim(lib, plume, flags=lib.FLAG_TILED)
    assert a.info.variant == 1 and a.info.tile_capacity > 0
    r1 = a.rate().cpu().numpy()
    r2 = a.rate().cpu().numpy()
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))


@pytest.mark.parametrize("name", ["256sq-n28-r100", "jitter-100sq", "c4-96sq", "3d-jitter-24"])
def test_trimmed_direct_walk_equals_full_stencil_bitwise(lib, name):
    """With trimmed rows the direct walks visit, per particle, only the stencil cells within
    (1 + 2^-12) H of the particle; without, and in the shared-memory tiled walk, every cell of the
    stencil.  The skipped candidates contribute exactly 0, so all give the same bits (same row
    order, same pair arithmetic), for the rate and for a step."""
    plume = CASES[name]()
    xq, C = plume.initial_state()
    for k in (2, 4):
        f = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_DIRECT)
        d = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_DIRECT | lib.FLAG_TRIMMED)
        assert d.info.variant == 3
        rf = f.rate().cpu().numpy()
        rd = d.rate().cpu().numpy()
        assert np.array_equal(rd.view(np.uint32), rf.view(np.uint32)), k
        t = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_TILED)
        if t.info.variant == 1:
            rt = t.rate().cpu().numpy()
            assert np.array_equal(rd.view(np.uint32), rt.view(np.uint32)), k
        b = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_BRANCHED)
        bt = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_BRANCHED | lib.FLAG_TRIMMED)
        assert bt.info.variant == 4
        assert np.array_equal(b.rate().cpu().numpy().view(np.uint32), bt.rate().cpu().numpy().view(np.uint32))
        # the paired walks (two targets per thread over the union of their ranges) add only
        # exact zeros to each target's sums
        pf = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_PAIRED)
        pt = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_PAIRED | lib.FLAG_TRIMMED)
        assert pf.info.variant == 5 and pt.info.variant == 6
        assert np.array_equal(pf.rate().cpu().numpy().view(np.uint32), rf.view(np.uint32)), k
        assert np.array_equal(pt.rate().cpu().numpy().view(np.uint32), rf.view(np.uint32)), k
        # the paired branched walks against the one-target branched walk
        pb = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_PAIRED | lib.FLAG_BRANCHED)
        pbt = _sim(lib, plume, xq, C, cell_subdiv=k, flags=lib.FLAG_PAIRED | lib.FLAG_BRANCHED | lib.FLAG_TRIMMED)
        assert pb.info.variant == 7 and pbt.info.variant == 8
        rb = b.rate().cpu().numpy()
        assert np.array_equal(pb.rate().cpu().numpy().view(np.uint32), rb.view(np.uint32)), k
        assert np.array_equal(pbt.rate().cpu().numpy().view(np.uint32), rb.view(np.uint32)), k
        # one step with trimmed rows, or paired, equals one with the full stencil
        f.step(1)
        d.step(1)
        pf.step(1)
        pt.step(1)
        assert np.array_equal(f.state()[1].view(np.uint32), d.state()[1].view(np.uint32))
        assert np.array_equal(f.state()[1].view(np.uint32), pf.state()[1].view(np.uint32))
        assert np.array_equal(f.state()[1].view(np.uint32), pt.state()[1].view(np.uint32))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_paired_walk_clustered_odd_count_bitwise(lib, orc, k):
    """A dense cluster on a lattice with an odd particle count: the paired walk meets pairs in
    different cell rows or several cells apart (each target then walks alone) and a last thread
    with one target; every rate and a step equal the one-target walk bit for bit, and the oracle."""
    rng = np.random.default_rng(10 + k)
    base = inputs.lattice_positions(2, 97)
    blob = np.mod(rng.normal(0.3, 0.03, size=(3000, 2)), 1.0)
    x = np.concatenate([base, blob])
    n = x.shape[0]
    assert n % 2 == 1
    box = np.ones(2)
    xq = inputs.to_fixed(x, box)
    xo = inputs.from_fixed(xq, box)
    C = inputs.gaussian_plume(xo, box, (0.35, 0.4), 0.1).astype(np.float32)
    plume = _plume(side=97, h_dx=2.0)

    def sim(flags):
        p = lib.params(2, plume.h, plume.alpha_L, plume.alpha_T, plume.D_m, plume.velocity, mass=1.0 / n,
                       flags=flags, cell_subdiv=k)
        return lib.Simulation(p, xq, C)

    one, two, two_t = sim(lib.FLAG_DIRECT), sim(lib.FLAG_PAIRED), sim(lib.FLAG_PAIRED | lib.FLAG_TRIMMED)
    r1 = one.rate().cpu().numpy()
    assert np.array_equal(r1.view(np.uint32), two.rate().cpu().numpy().view(np.uint32))
    assert np.array_equal(r1.view(np.uint32), two_t.rate().cpu().numpy().view(np.uint32))
    ob = sim(lib.FLAG_BRANCHED)
    rb = ob.rate().cpu().numpy()
    for fl in (lib.FLAG_PAIRED | lib.FLAG_BRANCHED, lib.FLAG_PAIRED | lib.FLAG_BRANCHED | lib.FLAG_TRIMMED):
        assert np.array_equal(rb.view(np.uint32), sim(fl).rate().cpu().numpy().view(np.uint32))
    r_orc, _ = orc.rate(xo, plume.velocity, C.astype(np.float64), 1.0 / n, 1.0, box, 0,
                        plume.support, 4.0, plume.alpha_L, plume.alpha_T, plume.D_m)
    assert _rel(r1, r_orc) <= RATE_TOL
    for s_ in (one, two, two_t):
        s_.step(2)
    for s_ in (two, two_t):
        assert np.array_equal(one.state()[1].view(np.uint32), s_.state()[1].view(np.uint32))
        assert np.array_equal(one.state()[0], s_.state()[0])


def test_rate_parity_clustered_overflow(lib, orc):
    """A dense cluster on top of a lattice overfills some tiles' staging buffers; those tiles
    take the direct walk, and the result still matches the oracle."""
    rng = np.random.default_rng(4)
    base = inputs.lattice_positions(2, 96)
    blob = np.mod(rng.normal(0.5, 0.02, size=(6000, 2)), 1.0)
    x = np.concatenate([base, blob])
    n = x.shape[0]
    box = np.ones(2)
    xq = inputs.to_fixed(x, box)
    xo = inputs.from_fixed(xq, box)
    C = inputs.gaussian_plume(xo, box, (0.45, 0.5), 0.1).astype(np.float32)
    plume = _plume(side=96, h_dx=2.0)
    p = lib.params(2, plume.h, plume.alpha_L, plume.alpha_T, plume.D_m, plume.velocity, mass=1.0 / n,
                   flags=lib.FLAG_TILED)
    sim = lib.Simulation(p, xq, C)
    assert sim.info.variant == 1
    r_orc, pairs = orc.rate(xo, plume.velocity, C.astype(np.float64), 1.0 / n, 1.0, box, 0,
                            plume.support, 4.0, plume.alpha_L, plume.alpha_T, plume.D_m)
    assert _rel(sim.rate().cpu().numpy(), r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_rate_parity_every_subdivision(lib, orc, k):
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    sim = _sim(lib, plume, cell_subdiv=k)
    r_orc, pairs = _oracle_rate(orc, plume, xq, C)
    assert _rel(sim.rate().cpu().numpy(), r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs == plume.n * 28


def test_rate_parity_nonsquare_box(lib, orc):
    rng = np.random.default_rng(9)
    n = 9000
    box = np.array([1.0, 0.55])
    x = rng.uniform(size=(n, 2)) * box
    plume = _plume(side=95, h_dx=1.8)
    xq = inputs.to_fixed(x, box)
    C = inputs.gaussian_plume(inputs.from_fixed(xq, box), box, (0.4, 0.3), 0.08).astype(np.float32)
    p = lib.params(2, plume.h, plume.alpha_L, plume.alpha_T, plume.D_m, plume.velocity,
                   mass=box.prod() / n, box=box)
    sim = lib.Simulation(p, xq, C)
    xo = inputs.from_fixed(xq, box)
    r_orc, pairs = orc.rate(xo, plume.velocity, C.astype(np.float64), box.prod() / n, 1.0, box, 0,
                            plume.support, 4.0, plume.alpha_L, plume.alpha_T, plume.D_m)
    assert _rel(sim.rate().cpu().numpy(), r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("name", ["64sq-h1.3", "256sq-n28-r100", "3d-32cube-h2", "jitter-100sq"])
def test_one_step_parity(lib, orc, name, variant):
    """Eq. 8-9: the increment C^{l+1} - C^l and the drift after one step."""
    plume = CASES[name]()
    xq, C = plume.initial_state()
    sim = _sim(lib, plume, flags=VARIANTS[variant])
    dt = sim.info.dt
    sim.step(1)
    xq1, C1 = sim.state()
    x = inputs.from_fixed(xq, plume.boxv)
    xo, Co, _ = orc.step(x, plume.velocity, C.astype(np.float64), plume.mass, plume.rho, plume.boxv,
                         plume.kernel, plume.support, plume.dim + 2.0, plume.alpha_L, plume.alpha_T,
                         plume.D_m, dt)
    dC_gpu = C1.astype(np.float64) - C
    dC_orc = Co - C
    # C1 is rounded to FP32: allow that rounding on top of the rate tolerance
    tol = RATE_TOL * np.max(np.abs(dC_orc)) + np.max(np.abs(Co)) * 2.0 ** -24
    assert np.max(np.abs(dC_gpu - dC_orc)) <= tol
    d = np.abs(inputs.from_fixed(xq1, plume.boxv) - xo)
    d = np.minimum(d, 1.0 - d)
    assert d.max() <= 2.0 ** -32


def test_run_graph_equals_step_bitwise(lib):
    plume = inputs.ladder_2d(256, 10)
    a = _sim(lib, plume)
    b = _sim(lib, plume)
    a.step(7)
    st = b.run(7)
    xa, Ca = a.state()
    xb, Cb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(Ca.view(np.uint32), Cb.view(np.uint32))
    assert st.step == 7 and st.status == 0


def test_multi_step_drift_and_conservation(lib, orc):
    """40 steps on the 64^2 plume: drift against the FP64 oracle and sum m C."""
    plume = inputs.lattice_2d_64()
    xq, C = plume.initial_state()
    sim = _sim(lib, plume)
    m0 = sim.stats().mass
    st = sim.run(40)
    _, C40 = sim.state()
    x = inputs.from_fixed(xq, plume.boxv)
    _, Co, _ = orc.step(x, plume.velocity, C.astype(np.float64), plume.mass, plume.rho, plume.boxv,
                        plume.kernel, plume.support, 4.0, plume.alpha_L, plume.alpha_T, plume.D_m,
                        sim.info.dt, nsteps=40)
    assert _rel(C40, Co) <= 2e-5
    assert abs(st.mass - m0) <= 1e-6 * abs(m0)
    assert st.mass == pytest.approx(plume.mass * np.sum(C40.astype(np.float64)), rel=1e-12)


def test_stats_and_closed_form_norms(lib, orc):
    plume = inputs.ladder_2d(256, 10)
    sim = _sim(lib, plume)
    sim.run(30)
    xq, C = sim.state()
    st = sim.stats()
    C64 = C.astype(np.float64)
    assert st.mass == pytest.approx(plume.mass * C64.sum(), rel=1e-12)
    assert st.c_min == C64.min() and st.c_max == C64.max()
    t = 30 * sim.info.dt
    assert st.t == pytest.approx(t, rel=1e-12)
    D = orc.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
    x = inputs.from_fixed(xq, plume.boxv)
    Ca = orc.closed_form(x, plume.boxv, plume.x0[:2], plume.velocity, D, plume.w, 1.0, t, nimg=2)
    e = C64 - Ca
    got = sim.closed_form_error(plume.x0[:2], plume.w, 1.0, nimg=2)
    assert got["linf"] == pytest.approx(np.max(np.abs(e)), rel=1e-9)
    assert got["l2"] == pytest.approx(math.sqrt(np.sum(plume.mass * e * e)), rel=1e-9)
    assert got["rmse"] == pytest.approx(math.sqrt(np.mean(e * e)), rel=1e-9)
    assert got["c_an_max"] == pytest.approx(Ca.max(), rel=1e-12)


def test_empty_and_single_particle(lib):
    plume = inputs.lattice_2d_64()
    e = _sim(lib, plume, np.zeros((2, 0), np.uint32), np.zeros(0, np.float32))
    assert e.rate().numel() == 0
    e.step(2)
    assert e.count_pairs() == 0
    one = _sim(lib, plume, np.array([[123456], [987654]], np.uint32), np.array([0.5], np.float32))
    assert one.rate().cpu().numpy()[0] == 0.0
    one.step(3)
    assert one.state()[1][0] == np.float32(0.5)


def test_nonfinite_concentration_sets_status(lib):
    """A NaN planted in the input (host side) is reported by the status word, not a fault."""
    plume = inputs.lattice_2d_64()
    xq, C = plume.initial_state()
    C = C.copy()
    C[100] = np.nan
    sim = _sim(lib, plume, xq, C)
    sim.step(1)
    st = sim.stats()
    assert st.status == -3


def _check_run_stats(st, plume, C):
    """Statistics of ade_run against the returned state: sum m C within 1e-12 (FP32 two-sum warp
    partials folded in FP64), min and max exact."""
    C64 = C.astype(np.float64)
    assert st.status == 0
    assert st.mass == pytest.approx(plume.mass * C64.sum(), rel=1e-12)
    assert st.c_min == C64.min() and st.c_max == C64.max()


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("side", [64, 256])
def test_run_stats_are_the_folded_corrector_partials(lib, variant, side):
    """ade_run's statistics are the corrector's per-warp partials folded on the device (one fold
    block at 64^2, two at 256^2), for every interaction variant; a fresh ade_get_stats over the
    state agrees."""
    plume = inputs.ladder_2d(side, 10) if side > 64 else inputs.lattice_2d_64()
    sim = _sim(lib, plume, flags=VARIANTS[variant])
    st = sim.run(3)
    _, C = sim.state()
    _check_run_stats(st, plume, C)
    ref = sim.stats()
    assert ref.mass == pytest.approx(st.mass, rel=1e-12)
    assert (ref.c_min, ref.c_max) == (st.c_min, st.c_max)


def test_run_stats_fold_capped_block_count(lib):
    """4.41 M particles (137,813 warp partials): the fold uses its maximum of 8 CTAs, so each
    thread folds several passes of eight partials."""
    plume = _plume(side=2100, h_dx=1.3, jitter=0.2, seed=4)
    sim = _sim(lib, plume)
    st = sim.run(1)
    _, C = sim.state()
    _check_run_stats(st, plume, C)


def test_full_size_ladder_top_rung(lib, orc):
    """The benchmark workload (1024^2, 120 neighbours, ratio 10) in the bench's launch
    configuration: full rate parity, pair count and one step."""
    plume = inputs.ladder_2d(1024, 10)
    xq, C = plume.initial_state()
    sim = _sim(lib, plume)
    r_orc, pairs = _oracle_rate(orc, plume, xq, C)
    assert _rel(sim.rate().cpu().numpy(), r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs == plume.n * 120


def test_full_size_3d_sampled(lib, orc):
    """128^3 with h = 2 dx: sampled particles against the oracle, exact pair count."""
    plume = inputs.cube_3d_128()
    xq, C = plume.initial_state()
    sim = _sim(lib, plume)
    r = sim.rate().cpu().numpy()
    sel = np.random.default_rng(0).choice(plume.n, 3000, replace=False).astype(np.int32)
    r_orc, pairs = _oracle_rate(orc, plume, xq, C, sel=sel)
    assert np.max(np.abs(r[sel] - r_orc)) <= RATE_TOL * np.max(np.abs(r))
    assert pairs == 3000 * 250
    assert sim.count_pairs() == plume.n * 250


@pytest.mark.parametrize("name", ["256sq-n28-r100", "3d-32cube-h2", "jitter-100sq"])
def test_autotune_keeps_state_and_parity(lib, orc, name):
    plume = CASES[name]()
    xq, C = plume.initial_state()
    sim = _sim(lib, plume)
    ms = sim.autotune()
    assert ms > 0.0
    x1, C1 = sim.state()
    assert np.array_equal(x1, xq) and np.array_equal(C1.view(np.uint32), C.view(np.uint32))
    r_orc, pairs = _oracle_rate(orc, plume, xq, C)
    assert _rel(sim.rate().cpu().numpy(), r_orc) <= RATE_TOL
    assert sim.count_pairs() == pairs
    sim.step(2)
    st = sim.stats()
    assert st.status == 0 and np.isfinite(st.mass)
