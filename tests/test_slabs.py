"""Slab decomposition of one plume (paper_2108_09488_gb300/slabs.py) on CPU ranks with gloo: the
FP64 oracle evaluates each rank's owned + halo particles, and the distributed rate and steps
(halo exchange before both evaluations, migration after the corrector) must reproduce the serial
oracle run -- positions exactly, concentrations to FP64 summation order -- with particles crossing
slab faces, for two and three ranks."""
import math
import os
import socket

import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs, slabs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _plume():
    return inputs.Plume(dim=2, side=36, h_over_dx=1.6, jitter=0.3, seed=8, speed=0.1, angle=0.3)


def _args(p):
    return (p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)


def _worker(rank, world, port, dt, nsteps, q):
    import torch.distributed as dist

    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _plume()
    x = p.positions()
    C = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.12)
    v = p.velocity
    dec = slabs.SlabDecomposition(p.boxv, p.support + 0.5 * dt * np.linalg.norm(v), world, rank)
    mine = np.nonzero(dec.owner(x) == rank)[0]
    ids, xr, Cr = mine.astype(np.int64), x[mine], C[mine]

    def rate_fn(xl, Cl, n_own):
        r, _ = orc.rate(xl, v, Cl, *_args(p))
        return r[:n_own]

    # one distributed rate evaluation
    hx, hC = dec.halo(xr, Cr)
    r_dist = rate_fn(np.concatenate([xr, hx]), np.concatenate([Cr, hC]), xr.shape[0])
    start = (ids.copy(), r_dist)
    moved = 0
    for _ in range(nsteps):
        before = set(ids.tolist())
        ids, xr, Cr = slabs.distributed_step(dec, rate_fn, ids, xr, v, Cr, dt)
        moved += len(set(ids.tolist()) ^ before)
    stats = slabs.global_stats(Cr, p.mass)
    q.put((rank, start, ids, xr, Cr, moved, stats))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_matches_serial_oracle(orc, world):
    torch = pytest.importorskip("torch")
    p = _plume()
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    dt = 4.0 * orc.dt_rule(D, p.h)
    nsteps = 3
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, world, port, dt, nsteps, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    x = p.positions()
    C = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.12)
    r_ser, _ = orc.rate(x, p.velocity, C, *_args(p))
    xs, Cs, _ = orc.step(x, p.velocity, C, *_args(p), dt, nsteps=nsteps)
    # the first evaluation: every particle's rate, owned by exactly one rank
    ids0 = np.concatenate([r[1][0] for r in res])
    r0 = np.concatenate([r[1][1] for r in res])
    assert np.array_equal(np.sort(ids0), np.arange(p.n))
    assert np.max(np.abs(r0 - r_ser[ids0])) <= 1e-12 * np.max(np.abs(r_ser))
    # after the steps: particles migrated, and the state equals the serial run
    ids = np.concatenate([r[2] for r in res])
    assert np.array_equal(np.sort(ids), np.arange(p.n))
    xd = np.concatenate([r[3] for r in res])
    Cd = np.concatenate([r[4] for r in res])
    assert sum(r[5] for r in res) > 0
    assert np.max(np.abs(xd - xs[ids])) == 0.0
    assert np.max(np.abs(Cd - Cs[ids])) <= 1e-12 * np.max(np.abs(Cs))
    mass, lo, hi = res[0][6]
    assert all(r[6] == res[0][6] for r in res)
    assert mass == pytest.approx(p.mass * Cs.sum(), rel=1e-12)
    assert lo == Cd.min() and hi == Cd.max()          # the all-reduces of the ranks' own values


def test_slab_ownership_and_reach_checks():
    dec = slabs.SlabDecomposition([1.0, 1.0], 0.1, 4, 1)
    x = np.array([[0.0, 0.5], [0.26, 0.1], [0.999, 0.2], [0.5, 0.5]])
    assert dec.owner(x).tolist() == [0, 1, 3, 2]
    assert (dec.left, dec.right) == (0, 2)
    with pytest.raises(ValueError):
        slabs.SlabDecomposition([1.0, 1.0], 0.3, 4, 0)
    with pytest.raises(ValueError):
        slabs.SlabDecomposition([1.0, 1.0], 0.3, 2, 0)


# ---- the fixed-point path (the library's state format, device-agnostic exchange) ---------------

def _fixed_setup(p, dt):
    import torch
    xq_np = p.fixed_positions()
    x = inputs.from_fixed(xq_np, p.boxv)
    C = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.12).astype(np.float32)
    v = p.velocity
    inc_h = [slabs.fixed_increment(v[i], 0.5 * dt, p.boxv[i]) for i in range(p.dim)]
    inc_f = [slabs.fixed_increment(v[i], dt, p.boxv[i]) for i in range(p.dim)]
    reach = p.support + 0.5 * dt * float(np.linalg.norm(v))
    return torch.from_numpy(xq_np.view(np.int32).copy()), torch.from_numpy(C), inc_h, inc_f, reach


def _oracle_rate_fn(orc, p):
    import torch

    def rate_fn(xq, C, n_own):
        x = inputs.from_fixed(xq.numpy().view(np.uint32), p.boxv)
        r, _ = orc.rate(x, p.velocity, C.numpy().astype(np.float64), *_args(p))
        return torch.from_numpy(r[:n_own].astype(np.float32))
    return rate_fn


def _fixed_worker(rank, world, port, dt, nsteps, q):
    import torch
    import torch.distributed as dist

    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _plume()
    xq, C, inc_h, inc_f, reach = _fixed_setup(p, dt)
    dec = slabs.FixedSlabs(reach, p.boxv[0], world, rank)
    mine = torch.nonzero(dec.owner(xq) == rank).flatten()
    ids, xr, Cr = mine.to(torch.int32), xq[:, mine].contiguous(), C[mine].contiguous()
    rate_fn = _oracle_rate_fn(orc, p)
    hx, hC = dec.halo(xr, Cr)
    r0 = rate_fn(torch.cat([xr, hx], dim=1), torch.cat([Cr, hC]), Cr.shape[0])
    start = (ids.numpy().copy(), r0.numpy().copy(), int(hC.shape[0]))
    moved = 0
    for _ in range(nsteps):
        before = set(ids.tolist())
        ids, xr, Cr = slabs.fixed_step(dec, rate_fn, ids, xr, Cr, inc_h, inc_f, dt)
        moved += len(set(ids.tolist()) ^ before)
    q.put((rank, start, ids.numpy(), xr.numpy(), Cr.numpy(), moved))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_fixed_point_slabs_match_serial_oracle_run(orc, world):
    """Halo and migration records in the library's format (uint32 position words + float32 C bits)
    over gloo: the first distributed evaluation and three steps equal the serial run of the same
    fixed-point step with the FP64 oracle as the rate (positions bit for bit, C to float32
    rounding of the oracle's summation order)."""
    torch = pytest.importorskip("torch")
    p = _plume()
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    dt = 4.0 * orc.dt_rule(D, p.h)
    nsteps = 3
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_fixed_worker, args=(r, world, port, dt, nsteps, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    # the serial run: one slab, no exchange
    xq, C, inc_h, inc_f, reach = _fixed_setup(p, dt)
    ser = slabs.FixedSlabs(reach, p.boxv[0], 1, 0)
    rate_fn = _oracle_rate_fn(orc, p)
    r_ser = rate_fn(xq, C, p.n).numpy()
    ids_s = torch.arange(p.n, dtype=torch.int32)
    xs, Cs = xq, C
    for _ in range(nsteps):
        ids_s, xs, Cs = slabs.fixed_step(ser, rate_fn, ids_s, xs, Cs, inc_h, inc_f, dt)
    xs, Cs = xs.numpy(), Cs.numpy()
    ids0 = np.concatenate([r[1][0] for r in res])
    r0 = np.concatenate([r[1][1] for r in res])
    assert np.array_equal(np.sort(ids0), np.arange(p.n))
    assert all(r[1][2] > 0 for r in res)                   # every rank received a halo
    assert np.max(np.abs(r0 - r_ser[ids0])) <= 1e-6 * np.max(np.abs(r_ser))
    ids = np.concatenate([r[2] for r in res]).astype(np.int64)
    assert np.array_equal(np.sort(ids), np.arange(p.n))
    assert sum(r[5] for r in res) > 0                      # particles crossed slab faces
    xd = np.concatenate([r[3] for r in res], axis=1)
    Cd = np.concatenate([r[4] for r in res])
    assert np.array_equal(xd, xs[:, ids])
    assert np.max(np.abs(Cd - Cs[ids])) <= 1e-6 * np.max(np.abs(Cs))


def test_fixed_slabs_ownership_faces_and_reach():
    torch = pytest.importorskip("torch")
    dec = slabs.FixedSlabs(0.05, 1.0, 4, 1)
    words = np.array([0, 1 << 30, (1 << 30) - 1, (3 << 30) + 5, 0xFFFFFFFF], dtype=np.uint32)
    xq = torch.from_numpy(np.stack([words, words]).view(np.int32))
    assert dec.owner(xq).tolist() == [0, 1, 0, 3, 3]
    dl, dr = dec._faces(xq)
    assert int(dl[1]) == 0 and int(dr[1]) == (1 << 30)       # rank 1 starts at word 2^30
    assert int(dl[2]) == -1                                  # one word left of it
    rec = dec.records(xq, torch.arange(5, dtype=torch.float32))
    x2, C2 = dec.unpack(rec)
    assert torch.equal(x2, xq) and C2.tolist() == [0.0, 1.0, 2.0, 3.0, 4.0]
    assert slabs.drift(xq, [1, 1])[0].numpy().view(np.uint32).tolist() == [1, (1 << 30) + 1, 1 << 30, (3 << 30) + 6, 0]
    assert slabs.fixed_increment(-0.1, 0.5, 1.0) == (1 << 32) - slabs.fixed_increment(0.1, 0.5, 1.0)
    with pytest.raises(ValueError):
        slabs.FixedSlabs(0.3, 1.0, 4, 0)
    with pytest.raises(ValueError):
        slabs.FixedSlabs(0.3, 1.0, 2, 0)
