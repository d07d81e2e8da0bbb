"""Host-side checks of libade_sph.so that need no GPU: the library loads, exports every entry
point declared in include/ade_sph.h, validates arguments, and derives the time step, grid and
stencil from the parameters (no device work is issued by these calls)."""
import math
import os
import re

import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ade_sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ade_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(adelib):
    lib = adelib.load()
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(adelib.EXPORTS)


FAKE = 1 << 40          # 256-aligned placeholder device addresses; never dereferenced here


def _ctx(adelib, p, n):
    nbytes = adelib.workspace_bytes(p, n)
    return adelib.init_particles(p, n, FAKE, FAKE + (1 << 30), FAKE + (2 << 30), nbytes), nbytes


def test_info_matches_oracle_time_step_and_grid(adelib, orc):
    plume = inputs.lattice_2d_64()
    p = adelib.params_for(plume)
    ctx, nbytes = _ctx(adelib, p, plume.n)
    try:
        info = adelib.get_info(ctx)
        D = orc.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
        assert info.dt == pytest.approx(orc.dt_rule(D, plume.h), rel=1e-14)
        assert np.allclose(np.array(info.D[:4]).reshape(2, 2), D, rtol=1e-14, atol=0)
        assert info.support == pytest.approx(2 * plume.h)
        k = info.cell_subdiv
        assert info.nc[0] == math.floor(1.0 * k / (2 * plume.h))
        assert info.ncells == info.nc[0] * info.nc[1]
        assert info.workspace_bytes == nbytes
    finally:
        adelib.destroy(ctx)
    # Eq. 10 trace rule
    p2 = adelib.params_for(plume, dt_rule=adelib.DT_TRACE)
    ctx, _ = _ctx(adelib, p2, plume.n)
    try:
        assert adelib.get_info(ctx).dt == pytest.approx(orc.dt_rule(D, plume.h, "trace"), rel=1e-14)
    finally:
        adelib.destroy(ctx)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_stencil_covers_support(adelib, k):
    """Every cell offset that can hold a neighbour is inside the stencil (checked by sampling
    point pairs in a fine sub-grid of the centre cell and its neighbours)."""
    plume = inputs.ladder_2d(256, 10)
    p = adelib.params_for(plume, cell_subdiv=k)
    ctx, _ = _ctx(adelib, p, plume.n)
    try:
        info = adelib.get_info(ctx)
        assert info.cell_subdiv == k
        s = 1.0 / info.nc[0]
        H = info.support
        assert s >= H / k
        # offsets reachable within H from the centre cell
        need = set()
        g = np.linspace(0, s, 9)[:-1] + s / 16
        for o in range(-k - 1, k + 2):
            for q in range(-k - 1, k + 2):
                for ax in g:
                    for ay in g:
                        bx = o * s + g[:, None]
                        by = q * s + g[None, :]
                        if np.any((bx - ax) ** 2 + (by - ay) ** 2 < H * H):
                            need.add((o, q))
        assert all(abs(o) <= k and abs(q) <= k for o, q in need)
        assert info.stencil_rows >= len({q for _, q in need})
    finally:
        adelib.destroy(ctx)


@pytest.mark.parametrize("bad,code", [
    (dict(dim=4), -1), (dict(h=0.0), -1), (dict(h=0.3), -1), (dict(alpha_L=-1.0), -1),
    (dict(mass=0.0), -1), (dict(cell_subdiv=7), -1), (dict(kernel=5), -1),
    (dict(alpha_L=0.0, alpha_T=0.0, D_m=0.0), -1)])
def test_invalid_arguments(adelib, bad, code):
    plume = inputs.lattice_2d_64()
    p = adelib.params_for(plume, **bad)
    with pytest.raises(adelib.AdeError) as e:
        nbytes = adelib.workspace_bytes(p, plume.n)
        adelib.init_particles(p, plume.n, FAKE, FAKE, FAKE, nbytes)
    assert e.value.code == code


def test_workspace_too_small_and_misaligned(adelib):
    plume = inputs.lattice_2d_64()
    p = adelib.params_for(plume)
    nbytes = adelib.workspace_bytes(p, plume.n)
    with pytest.raises(adelib.AdeError) as e:
        adelib.init_particles(p, plume.n, FAKE, FAKE, FAKE, nbytes - 1)
    assert e.value.code == -5
    with pytest.raises(adelib.AdeError) as e:
        adelib.init_particles(p, plume.n, FAKE, FAKE, FAKE + 8, nbytes)
    assert e.value.code == -1


def test_empty_particle_set_is_valid(adelib):
    plume = inputs.lattice_2d_64()
    p = adelib.params_for(plume)
    ctx, nbytes = _ctx(adelib, p, 0)
    assert nbytes > 0
    adelib.destroy(ctx)


def test_batch_workspace_and_validation(adelib):
    plumes = inputs.batched_2d(nplumes=5, side_lo=16, side_hi=64)
    plist = [adelib.params_for(p) for p in plumes]
    ns = [p.n for p in plumes]
    assert adelib.batch_workspace_bytes(plist, ns) > 16 * sum(ns)
    bad = list(plist)
    bad[2] = adelib.params_for(inputs.cube_3d_128(side=16))
    with pytest.raises(adelib.AdeError) as e:
        adelib.batch_workspace_bytes(bad, ns[:2] + [16 ** 3] + ns[3:])
    assert e.value.code == -1


def test_batch_config_null_arguments(adelib):
    """ade_batch_get_config / ade_batch_set_config refuse a NULL batch or NULL outputs before any
    device work."""
    import ctypes
    lib = adelib.load()
    m, t, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    assert lib.ade_batch_get_config(None, ctypes.byref(m), ctypes.byref(t), ctypes.byref(g), ctypes.byref(g)) == -1
    assert lib.ade_batch_set_config(None, 0, 256, 1216, 0, None) == -1


def _field_plume():
    return inputs.Plume(dim=2, side=96, h_over_dx=1.9, jitter=0.3, seed=11)


@pytest.mark.parametrize("rule", ["lambda_max", "trace"])
def test_velocity_field_mode_time_step_skin_and_grid(adelib, orc, rule):
    """vmax > 0: the dt rule takes the largest tensor any |v| <= vmax gives (the oracle's rule on
    D(v) for |v| = vmax), and the grid is built for H + dt vmax (+ 4 fixed-point units)."""
    plume = _field_plume()
    vmax = 0.25
    code = adelib.DT_LAMBDA_MAX if rule == "lambda_max" else adelib.DT_TRACE
    p = adelib.params_for(plume, vmax=vmax, dt_rule=code)
    ctx, nbytes = _ctx(adelib, p, plume.n)
    try:
        info = adelib.get_info(ctx)
        D = orc.dispersion_tensor([vmax, 0.0], plume.alpha_L, plume.alpha_T, plume.D_m)
        dt = orc.dt_rule(D, plume.h, rule)
        assert info.dt == pytest.approx(dt, rel=1e-14)
        assert info.skin == pytest.approx(vmax * dt + 4.0 / 2 ** 32, rel=1e-14)
        k = info.cell_subdiv
        assert info.nc[0] == math.floor(k / (info.support + info.skin))
        assert info.variant == 0
        # count, the one-pass scan, place, order, field gather, predictor, corrector, statistics fold
        assert adelib.launches_per_step(ctx) == 3 + 1 + 4
        assert nbytes >= (64 + 32) * plume.n   # caller-order and sorted V, D records + 2 sorted states
    finally:
        adelib.destroy(ctx)


@pytest.mark.parametrize("flags,variant", [(16, 5), (17, 5), (24, 6), (25, 6), (20, 7), (28, 8)])
def test_paired_walk_flags(adelib, flags, variant):
    """ADE_FLAG_PAIRED alone or with DIRECT selects the paired branch-free walk (5), with TRIMMED
    its trimmed form (6); with BRANCHED the paired branched walk (7) and its trimmed form (8)."""
    plume = inputs.ladder_2d(256, 10)
    ctx, _ = _ctx(adelib, adelib.params_for(plume, flags=flags), plume.n)
    try:
        assert adelib.get_info(ctx).variant == variant
    finally:
        adelib.destroy(ctx)


@pytest.mark.parametrize("flags", [16 | 2, 16 | 4 | 1, 16 | 4 | 8 | 1, 32])
def test_paired_walk_conflicting_flags(adelib, flags):
    """PAIRED with the tiled walk or with both DIRECT and BRANCHED, and unknown bits, are
    rejected."""
    plume = inputs.ladder_2d(256, 10)
    with pytest.raises(adelib.AdeError) as e:
        adelib.workspace_bytes(adelib.params_for(plume, flags=flags), plume.n)
    assert e.value.code == -1


@pytest.mark.parametrize("bad", [dict(vmax=-1.0), dict(vmax=float("inf")), dict(vmax=0.2, flags=2),
                                 dict(vmax=0.2, flags=4), dict(vmax=0.2, flags=16),
                                 dict(vmax=0.2, dt=3.0)])
def test_velocity_field_mode_invalid(adelib, bad):
    """Negative or infinite vmax, the tiled or branched kernels, and a skin so wide that the grid
    cannot hold the stencil are rejected before any device work."""
    plume = _field_plume()
    with pytest.raises(adelib.AdeError) as e:
        adelib.workspace_bytes(adelib.params_for(plume, **bad), plume.n)
    assert e.value.code == -1


def test_velocity_field_mode_call_order(adelib):
    """Calls that need a field fail with ADE_ERR_STATE until one is set; the uniform-only calls
    (closed form, adjoint, batches) refuse field mode; a uniform context refuses a field."""
    import ctypes
    plume = _field_plume()
    lib = adelib.load()
    ctx, _ = _ctx(adelib, adelib.params_for(plume, vmax=0.2), plume.n)
    try:
        for call in (lambda: adelib.build_cells(ctx), lambda: adelib.dispersion_rate(ctx, FAKE),
                     lambda: adelib.count_pairs(ctx), lambda: adelib.step(ctx, 1),
                     lambda: adelib.closed_form_error(ctx, [0.3, 0.3], 0.05)):
            with pytest.raises(adelib.AdeError) as e:
                call()
            assert e.value.code == -6
        g = (ctypes.c_double * 3)()
        J = ctypes.c_double(0.0)
        rc = lib.ade_adjoint(ctx, FAKE, 4, 2, FAKE, 1 << 40, None, g, ctypes.byref(J), None, None)
        assert rc == -6
    finally:
        adelib.destroy(ctx)
    ctx, _ = _ctx(adelib, adelib.params_for(plume), plume.n)
    try:
        assert lib.ade_set_velocity_field(ctx, FAKE, None) == -6
    finally:
        adelib.destroy(ctx)
    plumes = inputs.batched_2d(nplumes=2, side_lo=16, side_hi=32)
    with pytest.raises(adelib.AdeError) as e:
        adelib.batch_workspace_bytes([adelib.params_for(q, vmax=0.2) for q in plumes],
                                     [q.n for q in plumes])
    assert e.value.code == -1


def test_sweep_host_validation_and_info(adelib, orc):
    """Sweep set-up without device work: argument checks, the common time step (the smallest of
    the oracle's rule over the sets) and the grouping of sets into launches."""
    import ctypes
    plume = inputs.ladder_2d(256, 10)
    p = adelib.params_for(plume)
    for bad_n in (0, 65):
        with pytest.raises(adelib.AdeError):
            adelib.sweep_workspace_bytes(p, plume.n, bad_n)
    with pytest.raises(adelib.AdeError):
        adelib.sweep_workspace_bytes(adelib.params_for(plume, vmax=0.2), plume.n, 3)
    with pytest.raises(adelib.AdeError):
        adelib.sweep_workspace_bytes(adelib.params_for(plume, flags=2), plume.n, 3)
    theta = np.array([[1e-2, 1e-3, 1e-6], [5e-2, 1e-3, 1e-6], [1e-3, 1e-3, 0.0]] * 4)   # 12 sets
    nbytes = adelib.sweep_workspace_bytes(p, plume.n, len(theta))
    assert nbytes >= 2 * 4 * 12 * plume.n
    lib = adelib.load()
    ctx = ctypes.c_void_p()
    th = (ctypes.c_double * theta.size)(*theta.ravel().tolist())
    assert lib.ade_sweep_init(ctypes.byref(ctx), ctypes.byref(p), plume.n, len(theta), th, FAKE,
                              FAKE + (1 << 30), FAKE + (2 << 30), nbytes) == 0
    try:
        info = adelib.Info()
        assert lib.ade_sweep_get_info(ctx, ctypes.byref(info)) == 0
        dts = [orc.dt_rule(orc.dispersion_tensor(plume.velocity, *t), plume.h) for t in theta]
        assert info.dt == pytest.approx(min(dts), rel=1e-14)
        assert info.tile[0] == 2                      # 12 sets = one group of 8 + one of 4
        v = ctypes.c_int(0)
        # count, the one-pass scan, place, order; the sets' gather; 2 per group (4 here)
        assert lib.ade_sweep_launches_per_step(ctx, ctypes.byref(v)) == 0 and v.value == 4 + 1 + 4
    finally:
        lib.ade_sweep_destroy(ctx)
    bad = theta.copy()
    bad[3, 1] = -1.0
    th = (ctypes.c_double * bad.size)(*bad.ravel().tolist())
    assert lib.ade_sweep_init(ctypes.byref(ctx), ctypes.byref(p), plume.n, len(bad), th, FAKE,
                              FAKE + (1 << 30), FAKE + (2 << 30), nbytes) == -1


def test_cattaneo_host_validation(adelib, orc):
    """tau: finite and >= 0; the dt rule is capped at tau; the flux needs a Cattaneo context and
    steps wait for one; field mode, batches and sweeps refuse tau > 0 (all before device work)."""
    import ctypes
    plume = inputs.lattice_2d_64()
    for bad in (-1.0, float("nan")):
        with pytest.raises(adelib.AdeError) as e:
            adelib.workspace_bytes(adelib.params_for(plume, tau=bad), plume.n)
        assert e.value.code == -1
    with pytest.raises(adelib.AdeError):
        adelib.workspace_bytes(adelib.params_for(plume, tau=1.0, vmax=0.2), plume.n)
    D = orc.dispersion_tensor(plume.velocity, plume.alpha_L, plume.alpha_T, plume.D_m)
    dt_rule = orc.dt_rule(D, plume.h)
    lib = adelib.load()
    for tau, want in ((0.25 * dt_rule, 0.25 * dt_rule), (4 * dt_rule, dt_rule)):
        p = adelib.params_for(plume, tau=tau)
        ctx, nbytes = _ctx(adelib, p, plume.n)
        try:
            assert adelib.get_info(ctx).dt == pytest.approx(want, rel=1e-14)
            assert nbytes >= adelib.workspace_bytes(adelib.params_for(plume), plume.n) + 8 * plume.n
            with pytest.raises(adelib.AdeError) as e:
                adelib.step(ctx, 1)
            assert e.value.code == -6
        finally:
            adelib.destroy(ctx)
    ctx, _ = _ctx(adelib, adelib.params_for(plume), plume.n)
    try:
        assert lib.ade_set_flux(ctx, None, None) == -6
        assert lib.ade_get_flux(ctx, FAKE, None) == -6
    finally:
        adelib.destroy(ctx)
    plumes = inputs.batched_2d(nplumes=2, side_lo=16, side_hi=32)
    with pytest.raises(adelib.AdeError):
        adelib.batch_workspace_bytes([adelib.params_for(q, tau=1.0) for q in plumes], [q.n for q in plumes])
    with pytest.raises(adelib.AdeError):
        adelib.sweep_workspace_bytes(adelib.params_for(plume, tau=1.0), plume.n, 2)


def test_checkpoint_format_and_validation(adelib):
    """Snapshots of an empty context need no device: the trailing CRC-32 equals zlib's over header
    and payload; a flipped byte, a truncated buffer, a foreign buffer and other parameters are
    refused (ADE_ERR_ARG) before any copy."""
    import zlib
    plume = inputs.lattice_2d_64()
    p = adelib.params_for(plume)
    ctx, _ = _ctx(adelib, p, 0)
    try:
        blob = adelib.checkpoint_save(ctx)
        assert blob[:8] == b"ADECKPT1"
        assert int.from_bytes(blob[-4:], "little") == zlib.crc32(blob[:-4])
        adelib.checkpoint_load(ctx, blob)
        bad = bytearray(blob)
        bad[40] ^= 0x01
        for b in (bytes(bad), blob[:-1], b"x" * len(blob)):
            with pytest.raises(adelib.AdeError) as e:
                adelib.checkpoint_load(ctx, b)
            assert e.value.code == -1
    finally:
        adelib.destroy(ctx)
    other, _ = _ctx(adelib, adelib.params_for(plume, alpha_L=2e-2), 0)
    try:
        with pytest.raises(adelib.AdeError) as e:
            adelib.checkpoint_load(other, blob)
        assert e.value.code == -1 and "parameters" in str(e.value)
    finally:
        adelib.destroy(other)


@pytest.mark.parametrize("which", ["sorted", "perm", "cell_start", "xq", "C"])
def test_noalloc_rejects_misaligned_buffers(adelib, which):
    """ade_build_cells_noalloc refuses a misaligned buffer before any GPU work: the sorted records
    are stored as 16-byte words, the other buffers as 4-byte words."""
    ptrs = {"xq": FAKE, "C": FAKE + (1 << 30), "perm": FAKE + (2 << 30),
            "cell_start": FAKE + (3 << 30), "sorted": FAKE + (4 << 30)}
    ptrs[which] += 8 if which == "sorted" else 2
    with pytest.raises(adelib.AdeError) as e:
        adelib.build_cells_noalloc(2, 100, ptrs["xq"], ptrs["C"], [8, 8], ptrs["perm"],
                                   ptrs["cell_start"], ptrs["sorted"])
    assert e.value.code == -1 and "aligned" in str(e.value)
