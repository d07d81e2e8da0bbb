"""Batched plumes (ade_batch_*) on the GPU: each plume of a batch is bit-identical to the same plume
stepped alone with the same cell subdivision; graph replay equals plain launches; the autotuner
leaves the state unchanged; per-plume FP64 stats and pair counts match the single-plume path and
the oracle."""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(adelib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return adelib


def _batch(lib, plumes):
    states = [p.initial_state() for p in plumes]
    plist = [lib.params_for(p) for p in plumes]
    return lib.Batch(plist, [s[0] for s in states], [s[1] for s in states]), states


def _single(lib, plume, subdiv, state):
    return lib.Simulation(lib.params_for(plume, cell_subdiv=subdiv, flags=lib.FLAG_DIRECT), *state)


def _same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


SMALL = dict(nplumes=7, side_lo=20, side_hi=90, seed=7)


def test_batch_bitwise_equals_single_plumes(lib):
    plumes = inputs.batched_2d(**SMALL)
    b, states = _batch(lib, plumes)
    b.step(3)
    for i, p in enumerate(plumes):
        s = _single(lib, p, b.plume_info(i).cell_subdiv, states[i])
        assert s.info.dt == b.plume_info(i).dt
        s.step(3)
        xs, Cs = s.state()
        xb, Cb = b.state(i)
        assert _same(xs, xb) and _same(Cs, Cb), f"plume {i}"


def test_batch_graph_replay_equals_step(lib):
    plumes = inputs.batched_2d(**SMALL)
    a, _ = _batch(lib, plumes)
    g, _ = _batch(lib, plumes)
    a.step(4)
    g.run(4)
    for i in range(len(plumes)):
        xa, Ca = a.state(i)
        xg, Cg = g.state(i)
        assert _same(xa, xg) and _same(Ca, Cg)


def test_batch_autotune_keeps_state_and_identity(lib):
    plumes = inputs.batched_2d(**SMALL)
    b, states = _batch(lib, plumes)
    before = [b.state(i) for i in range(len(plumes))]
    ms = b.autotune()
    assert ms > 0.0
    for i in range(len(plumes)):
        x, C = b.state(i)
        assert _same(x, before[i][0]) and _same(C, before[i][1])
    b.step(2)
    for i, p in enumerate(plumes):
        s = _single(lib, p, b.plume_info(i).cell_subdiv, states[i])
        s.step(2)
        assert _same(s.state()[1], b.state(i)[1])


def test_batch_stats_pairs_and_oracle(lib, orc):
    plumes = inputs.batched_2d(**SMALL)
    b, states = _batch(lib, plumes)
    total = 0
    for i, p in enumerate(plumes):
        x = inputs.from_fixed(states[i][0], p.boxv)
        _, pairs = orc.rate(x, p.velocity, states[i][1].astype(np.float64), p.mass, p.rho, p.boxv,
                            p.kernel, p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)
        total += pairs
    assert b.count_pairs() == total
    b.step(2)
    st = b.stats()
    for i, p in enumerate(plumes):
        C = b.state(i)[1].astype(np.float64)
        assert st[i].mass == pytest.approx(p.mass * C.sum(), rel=1e-12)
        assert st[i].c_min == C.min() and st[i].c_max == C.max()
        assert st[i].t == pytest.approx(2 * b.plume_info(i).dt, rel=1e-14)
    # one plume against the FP64 oracle step (increment within 1e-5)
    i = int(np.argmax([p.n for p in plumes]))
    p = plumes[i]
    c, _ = _batch(lib, [p])
    c.step(1)
    xo, Co, _ = orc.step(inputs.from_fixed(states[i][0], p.boxv), p.velocity,
                         states[i][1].astype(np.float64), p.mass, p.rho, p.boxv, p.kernel, p.support,
                         4.0, p.alpha_L, p.alpha_T, p.D_m, c.plume_info(0).dt)
    dg = c.state(0)[1].astype(np.float64) - states[i][1]
    do = Co - states[i][1]
    assert np.max(np.abs(dg - do)) <= 1e-5 * np.max(np.abs(do)) + np.max(np.abs(Co)) * 2.0 ** -24


def test_full_batch_64_plumes_sampled_identity(lib):
    """The 64-plume workload (about 3M particles): one step, four plumes checked bit for bit."""
    plumes = inputs.batched_2d()
    b, states = _batch(lib, plumes)
    b.step(1)
    for i in (0, 17, 40, 63):
        s = _single(lib, plumes[i], b.plume_info(i).cell_subdiv, states[i])
        s.step(1)
        assert _same(s.state()[1], b.state(i)[1]) and _same(s.state()[0], b.state(i)[0])


def test_batch_config_copy_gives_identical_steps(lib):
    """ade_batch_get_config / ade_batch_set_config: a second batch of the same plumes given the
    first one's autotuned configuration steps bit for bit like it; out-of-range configurations
    are refused and leave the batch unchanged."""
    plumes = inputs.batched_2d(**SMALL)
    a, _ = _batch(lib, plumes)
    b, _ = _batch(lib, plumes)
    a.autotune()
    cfg = a.config()
    b.set_config(cfg)
    assert b.config() == cfg
    for i in range(len(plumes)):
        assert b.plume_info(i).tile[0] == a.plume_info(i).tile[0]
        assert b.plume_info(i).cell_subdiv == a.plume_info(i).cell_subdiv
    a.run(3)
    b.run(3)
    for i in range(len(plumes)):
        xa, Ca = a.state(i)
        xb, Cb = b.state(i)
        assert _same(xa, xb) and _same(Ca, Cb)
    for bad in ((7, 256, 100, 0), (0, 16, 100, 0), (0, 256, 0, 0), (0, 256, 100, 2)):
        with pytest.raises(lib.AdeError) as e:
            b.set_config(bad)
        assert e.value.code == -1
    assert b.config() == cfg


def test_batch_paired_walk_is_bitwise_the_single_walk(lib):
    """The batched rate kernel with two particles per thread (paired walk) steps every plume bit
    for bit like the one-particle-per-thread walk of the same configuration."""
    plumes = inputs.batched_2d(**SMALL)
    a, _ = _batch(lib, plumes)
    b, _ = _batch(lib, plumes)
    m, t, g, _ = a.config()
    a.set_config((m, t, g, 0))
    b.set_config((m, t, g, 1))
    assert b.config()[3] == 1
    a.run(3)
    b.run(3)
    for i in range(len(plumes)):
        xa, Ca = a.state(i)
        xb, Cb = b.state(i)
        assert _same(xa, xb) and _same(Ca, Cb)
