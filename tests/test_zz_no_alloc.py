"""The allocation-free cell-list build (hamls_cells_noalloc), for callers that
cannot allocate device memory, must give exactly what the plan's own build
gives (hamls_debug_cells) for the same nodes and key shape, on consecutive
calls that reuse its static scratch. This file is collected last."""
import numpy as np
import pytest
import torch

from hamls_synth import track_hole_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


def _reference(h, x):
    with h.Plan(x, 8, 2) as p:
        keys, perm, start, B, P = p.debug_cells()
        p.sync(60000)
    return keys.cpu(), perm.cpu(), start.cpu(), B, P


@pytest.mark.parametrize("M,seed", [(200_000, 71), (1 << 20, 72)])
def test_noalloc_cells_match_plan_on_two_calls(h, M, seed):
    x = torch.tensor(track_hole_nodes(seed, M)[0], device="cuda")
    keys_ref, perm_ref, start_ref, B, P = _reference(h, x)
    # a smaller node set in between leaves different contents in the shared scratch
    y = torch.tensor(track_hole_nodes(seed + 100, 5000)[0], device="cuda")
    for nodes, want in ((x, (keys_ref, perm_ref, start_ref)), (y, None), (x, (keys_ref, perm_ref, start_ref))):
        n = nodes.shape[0]
        keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        start = torch.full((B * P + 1,), -1, dtype=torch.int32, device="cuda")
        h.cells_noalloc(nodes, B, P, keys, perm, start)
        torch.cuda.synchronize()
        if want is not None:
            assert torch.equal(keys.cpu(), want[0])
            assert torch.equal(perm.cpu(), want[1])
            assert torch.equal(start.cpu(), want[2])


def test_noalloc_rejects_oversize_and_host_memory(h):
    import ctypes
    L = h.lib()
    x = torch.zeros(((1 << 20) + 1, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    assert L.hamls_cells_noalloc(x.data_ptr(), x.shape[0], 64, 128, out.data_ptr(), out.data_ptr(),
                                 out.data_ptr(), None) == 8
    xh = np.zeros((100, 3))
    assert L.hamls_cells_noalloc(xh.ctypes.data, 100, 64, 128, out.data_ptr(), out.data_ptr(),
                                 out.data_ptr(), None) == 1
    assert L.hamls_cells_noalloc(x.data_ptr(), 100, 63, 128, out.data_ptr(), out.data_ptr(),
                                 out.data_ptr(), None) == 1
