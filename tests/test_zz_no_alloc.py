"""The allocation-free cell build, ade_build_cells_noalloc, against the workspace-based one.

Callers that cannot allocate device memory (or hand the library a workspace) use this entry
point; its scratch lives in a static device array shared by every call.  These tests call it
through the C ABI several times in a row on different problems, so every call after the first
runs on scratch an earlier call left behind (with fewer cells, then more cells, than the call
before), and compare each result bit for bit (the outputs are integers and bit patterns) with
ade_build_cells or, where no context fits the grid, with the oracle's cell list.  The file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc_cells(lib, torch, sim):
    n, dim = sim.n, sim.dim
    ncells = sim.info.ncells
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    srt = torch.zeros((max(n, 1), 4), dtype=torch.int32, device="cuda")
    lib.build_cells_noalloc(dim, n, sim.xq.data_ptr(), sim.C.data_ptr(), list(sim.info.nc),
                            perm.data_ptr(), cs.data_ptr(), srt.data_ptr(), sim.stream)
    torch.cuda.synchronize()
    return (perm.cpu().numpy().view(np.uint32)[:n], cs.cpu().numpy().view(np.uint32),
            srt.cpu().numpy().view(np.uint32)[:n])


def test_noalloc_matches_workspace_build_two_calls(adelib, torch_cuda):
    plumes = [inputs.ladder_2d(256, 10),
              inputs.Plume(dim=3, side=24, h_over_dx=1.7, jitter=0.4, seed=5)]
    for plume in plumes:                      # two calls in a row on the shared scratch
        xq, C = plume.initial_state()
        sim = adelib.Simulation(adelib.params_for(plume), xq, C)
        sim.build_cells()
        perm_ref, cs_ref = sim.cells()
        perm, cs, srt = _noalloc_cells(adelib, torch_cuda, sim)
        assert np.array_equal(perm, perm_ref)
        assert np.array_equal(cs, cs_ref)
        for d in range(plume.dim):
            assert np.array_equal(srt[:, d], xq[d][perm_ref])
        assert np.array_equal(srt[:, 3], C.view(np.uint32)[perm_ref])
        sim.close()


def _noalloc_raw(lib, torch, dim, xq, C, nc):
    n = xq.shape[1]
    ncells = int(np.prod(nc[:dim]))
    xq_d = torch.from_numpy(np.ascontiguousarray(xq).view(np.int32)).cuda()
    C_d = torch.from_numpy(np.ascontiguousarray(C)).cuda()
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    srt = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    lib.build_cells_noalloc(dim, n, xq_d.data_ptr(), C_d.data_ptr(), list(nc), perm.data_ptr(),
                            cs.data_ptr(), srt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return (perm.cpu().numpy().view(np.uint32), cs.cpu().numpy().view(np.uint32),
            srt.cpu().numpy().view(np.uint32))


def _check_against_oracle(orc, dim, xq, C, nc, perm, cs, srt):
    key = orc.cell_keys(xq, nc)
    perm_ref, cs_ref = orc.sort_cells(key, int(np.prod(nc[:dim])))
    assert np.array_equal(perm, perm_ref)
    assert np.array_equal(cs, cs_ref)
    for d in range(dim):
        assert np.array_equal(srt[:, d], xq[d][perm_ref])
    assert np.array_equal(srt[:, 3], C.view(np.uint32)[perm_ref])


def test_noalloc_capacity_limits_then_coarse_grid(adelib, orc, torch_cuda):
    """Two more calls in a row on the shared scratch: one at exactly ADE_NOALLOC_MAX_PARTICLES
    particles and ADE_NOALLOC_MAX_CELLS cells (more cells than any call before it, so its scratch
    offsets reach the end of the array), then one with about 64 particles per cell, which takes
    the one-block-per-cell ordering path; both bit for bit against the oracle's cell list."""
    torch = torch_cuda
    n = adelib.NOALLOC_MAX_PARTICLES
    rng = np.random.default_rng(11)
    xq = rng.integers(0, 2 ** 32, size=(2, n), dtype=np.uint64).astype(np.uint32)
    C = rng.random(n, dtype=np.float32)
    nc = [1024, adelib.NOALLOC_MAX_CELLS // 1024]
    _check_against_oracle(orc, 2, xq, C, nc, *_noalloc_raw(adelib, torch, 2, xq, C, nc))
    plume = inputs.Plume(dim=2, side=512, h_over_dx=1.3, jitter=0.3, seed=3)
    xq2, C2 = plume.initial_state()
    nc2 = [64, 64]                      # 262144 particles in 4096 cells
    _check_against_oracle(orc, 2, xq2, C2, nc2, *_noalloc_raw(adelib, torch, 2, xq2, C2, nc2))


def test_noalloc_rejects_oversize(adelib, torch_cuda):
    big = adelib.NOALLOC_MAX_PARTICLES + 1
    with pytest.raises(adelib.AdeError) as e:
        adelib.build_cells_noalloc(2, big, 0, 0, [64, 64], 0, 0, 0)
    assert e.value.code == -5 and "ADE_NOALLOC_MAX_PARTICLES" in str(e.value)
    with pytest.raises(adelib.AdeError) as e:
        adelib.build_cells_noalloc(2, 10, 0, 0, [2048, 1024], 0, 0, 0)
    assert e.value.code == -5 and "ADE_NOALLOC_MAX_CELLS" in str(e.value)
