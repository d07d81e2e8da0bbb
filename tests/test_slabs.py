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
