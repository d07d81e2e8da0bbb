"""The allocation-free cell build, ade_build_cells_noalloc, against the workspace-based one.

Callers that cannot allocate device memory (or hand the library a workspace) use this entry
point; its scratch lives in a static device array shared by every call.  These tests call it
through the C ABI twice in a row on different problems, so the second call runs on scratch the
first call left behind, and compare each result with ade_build_cells bit for bit (the outputs are
integers and bit patterns).  The file is collected last on purpose.
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


def test_noalloc_rejects_oversize(adelib, torch_cuda):
    big = adelib.NOALLOC_MAX_PARTICLES + 1
    with pytest.raises(adelib.AdeError) as e:
        adelib.build_cells_noalloc(2, big, 0, 0, [64, 64], 0, 0, 0)
    assert e.value.code == -5 and "ADE_NOALLOC_MAX_PARTICLES" in str(e.value)
    with pytest.raises(adelib.AdeError) as e:
        adelib.build_cells_noalloc(2, 10, 0, 0, [2048, 1024], 0, 0, 0)
    assert e.value.code == -5 and "ADE_NOALLOC_MAX_CELLS" in str(e.value)
