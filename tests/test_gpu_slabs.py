"""The fixed-point slab path (paper_2108_09488_gb300/slabs.py) through the library on one GPU.

W ranks are emulated in lockstep in one process: every rank's outgoing halo records (the library's
uint32 position words + float32 C bits, selected on the device) are handed to its neighbours
directly instead of over NCCL (the exchange itself is covered by the gloo tests on CPU ranks), and
each rank's owned + received set goes to ``ade_dispersion_rate`` through ``slabs.LibraryRate``.
The owned rates must match the library's evaluation of the whole plume and the FP64 oracle, and
one predictor-corrector step assembled from the ranks must match the library's own step (migration
across faces is covered by the multi-step gloo tests)."""
import numpy as np
import pytest

from paper_2108_09488_gb300 import ade, inputs, slabs

pytestmark = pytest.mark.gpu


def _plume():
    return inputs.Plume(dim=2, side=96, h_over_dx=1.6, jitter=0.3, seed=5, speed=0.1, angle=0.7)


def _ranks_rates(p, params, xq, C, own, world, reach):
    """Rates of all particles, each evaluated by its owning rank over owned + received particles."""
    import torch
    decs = [slabs.FixedSlabs(reach, p.boxv[0], world, r, device="cuda") for r in range(world)]
    parts = []
    for r in range(world):
        idx = torch.nonzero(own == r).flatten()
        parts.append((idx, xq[:, idx].contiguous(), C[idx].contiguous()))
    out = [decs[r].outgoing(parts[r][1], parts[r][2]) for r in range(world)]   # (to left, to right)
    rate_fn = slabs.LibraryRate(params)
    rates = torch.full_like(C, float("nan"))
    halo_sizes = []
    for r in range(world):
        d = decs[r]
        # from the left neighbour what it sends right, from the right neighbour what it sends left
        hx, hC = d.unpack(torch.cat([out[d.left][1], out[d.right][0]], dim=0))
        idx, xr, Cr = parts[r]
        rates[idx] = rate_fn(torch.cat([xr, hx], dim=1), torch.cat([Cr, hC]), Cr.shape[0])
        halo_sizes.append(int(hC.shape[0]))
    return rates, halo_sizes


@pytest.mark.parametrize("world", [2, 3])
def test_library_rate_on_slabs_matches_whole_plume(orc, world):
    import torch
    p = _plume()
    params = ade.params_for(p)
    xq_np = p.fixed_positions()
    x = inputs.from_fixed(xq_np, p.boxv)
    C_np = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.12).astype(np.float32)
    sim = ade.Simulation(params, xq_np, C_np)
    full = sim.rate().cpu().numpy()
    xq = torch.from_numpy(xq_np.view(np.int32).copy()).cuda()
    C = torch.from_numpy(C_np).cuda()
    dec0 = slabs.FixedSlabs(p.support, p.boxv[0], world, 0, device="cuda")
    rates, halos = _ranks_rates(p, params, xq, C, dec0.owner(xq), world, p.support)
    r = rates.cpu().numpy()
    assert np.all(np.isfinite(r)) and min(halos) > 0
    scale = np.max(np.abs(full))
    assert np.max(np.abs(r - full)) <= 1e-5 * scale
    r_orc, _ = orc.rate(x, p.velocity, C_np.astype(np.float64), p.mass, p.rho, p.boxv, p.kernel,
                        p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)
    assert np.max(np.abs(r - r_orc)) <= 1e-5 * np.max(np.abs(r_orc))


@pytest.mark.parametrize("world", [2, 3])
def test_slab_step_matches_library_step(world):
    import torch
    p = _plume()
    params = ade.params_for(p)
    xq_np = p.fixed_positions()
    x = inputs.from_fixed(xq_np, p.boxv)
    C_np = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.12).astype(np.float32)
    sim = ade.Simulation(params, xq_np, C_np)
    dt = sim.info.dt
    v = p.velocity
    inc_h = [slabs.fixed_increment(v[i], 0.5 * dt, p.boxv[i]) for i in range(p.dim)]
    inc_f = [slabs.fixed_increment(v[i], dt, p.boxv[i]) for i in range(p.dim)]
    reach = p.support + 0.5 * dt * float(np.linalg.norm(v))
    xq = torch.from_numpy(xq_np.view(np.int32).copy()).cuda()
    C = torch.from_numpy(C_np).cuda()
    own = slabs.FixedSlabs(reach, p.boxv[0], world, 0, device="cuda").owner(xq)   # fixed for the step
    r0, _ = _ranks_rates(p, params, xq, C, own, world, reach)
    Ch = C + (0.5 * dt) * r0
    xh = slabs.drift(xq, inc_h)
    r1, _ = _ranks_rates(p, params, xh, Ch, own, world, reach)
    C1 = (C + dt * r1).cpu().numpy()
    x1 = slabs.drift(xq, inc_f).cpu().numpy()
    sim.step(1)
    torch.cuda.synchronize()
    assert np.array_equal(x1, sim.xq.cpu().numpy())           # the same drift words
    C_lib = sim.C.cpu().numpy()
    assert np.max(np.abs(C1 - C_lib)) <= 1e-5 * np.max(np.abs(C_lib))
