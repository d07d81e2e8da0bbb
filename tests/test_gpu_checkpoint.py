"""Checkpoint and resume (ade_checkpoint_*): stepping on from a restored context gives the same
bits as the uninterrupted run, for the uniform-velocity, velocity-field and Cattaneo modes."""
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


def _same(a, b):
    return all(np.array_equal(np.asarray(x).view(np.uint32), np.asarray(y).view(np.uint32))
               for x, y in zip(a, b))


def _resume_check(lib, make, prepare):
    """make() -> a fresh Simulation; prepare(sim) sets any field or flux.  Run 4 steps, snapshot,
    4 more; a second context restored from the snapshot runs the same 4 and must match bitwise."""
    a = make()
    prepare(a)
    a.run(4)
    blob = a.checkpoint()
    a.step(4)
    b = make()                       # fresh state: the snapshot replaces it
    b.restore(blob)
    b.step(4)
    assert _same(a.state(), b.state())
    sa, sb = a.stats(), b.stats()
    assert sa.step == sb.step == 8 and sa.t == sb.t and sa.mass == sb.mass
    return a, b


def test_resume_uniform(lib):
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    _resume_check(lib, lambda: lib.Simulation(lib.params_for(plume), xq, C), lambda s: None)


def test_resume_velocity_field_3d(lib):
    plume = inputs.Plume(dim=3, side=24, h_over_dx=1.7, jitter=0.4, seed=5)
    xq, C = plume.initial_state()
    v = inputs.velocity_field(inputs.from_fixed(xq, plume.boxv), plume.boxv, seed=9)
    p = lib.params_for(plume, vmax=0.2)

    def make():
        return lib.Simulation(p, xq, C)

    a = make()
    a.set_velocity_field(v)
    a.run(3)
    blob = a.checkpoint()
    a.step(3)
    b = make()                       # no field set: the snapshot carries it
    b.restore(blob)
    b.step(3)
    assert _same(a.state(), b.state())


def test_resume_cattaneo(lib):
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    p = lib.params_for(plume, tau=1e-3)
    a, b = _resume_check(lib, lambda: lib.Simulation(p, xq, C), lambda s: s.set_flux())
    assert _same([a.flux().cpu().numpy()], [b.flux().cpu().numpy()])


def test_restore_refuses_other_particle_counts(lib):
    plume = inputs.ladder_2d(256, 10)
    xq, C = plume.initial_state()
    a = lib.Simulation(lib.params_for(plume), xq, C)
    blob = a.checkpoint()
    small = inputs.Plume(dim=2, side=128, h_over_dx=plume.h_over_dx * 0.5)
    xs, Cs = small.initial_state()
    b = lib.Simulation(lib.params_for(plume), xs, Cs)
    with pytest.raises(lib.AdeError) as e:
        b.restore(blob)
    assert e.value.code == -1
