"""The allocation-free cell-list build (hamls_cells_noalloc), for callers that
cannot allocate device memory, must give exactly what the plan's own build
gives (hamls_debug_cells) and what the oracle's key definition and stable
sort give, for the same nodes and key shape, on consecutive calls that reuse
its static scratch, and it must not change the device's free memory. This
file is collected last."""
import numpy as np
import pytest
import torch

import oracle as O
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


def _call(h, nodes, B, P):
    n = nodes.shape[0]
    keys = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    start = torch.full((B * P + 1,), -1, dtype=torch.int32, device="cuda")
    h.cells_noalloc(nodes, B, P, keys, perm, start)
    torch.cuda.synchronize()
    return keys.cpu(), perm.cpu(), start.cpu()


# 200,000 and 2^20 nodes give 1024 x 2048 and 512 x 1024 cells (21 and 19 key
# bits: three radix passes); 10,000 nodes give 64 x 128 cells (13 bits: two
# passes, the sort then starts in the caller's arrays)
@pytest.mark.parametrize("M,seed", [(200_000, 71), (1 << 20, 72), (10_000, 73)])
def test_noalloc_cells_match_plan_on_two_calls(h, M, seed):
    x = torch.tensor(track_hole_nodes(seed, M)[0], device="cuda")
    keys_ref, perm_ref, start_ref, B, P = _reference(h, x)
    # a smaller node set in between leaves different contents in the shared scratch
    y = torch.tensor(track_hole_nodes(seed + 100, 5000)[0], device="cuda")
    for nodes, want in ((x, (keys_ref, perm_ref, start_ref)), (y, None), (x, (keys_ref, perm_ref, start_ref))):
        got = _call(h, nodes, B, P)
        if want is not None:
            for g, w in zip(got, want):
                assert torch.equal(g, w)


@pytest.mark.parametrize("B,P", [(64, 128), (16, 32)])
def test_noalloc_two_pass_shapes_match_oracle(h, B, P):
    """Two-pass key shapes on a large node set, against the oracle's key
    definition and its stable sort (independent of the plan's build)."""
    xn = track_hole_nodes(74, 300_000)[0]
    x = torch.tensor(xn, device="cuda")
    k = O.cell_keys(xn, B, P)
    operm, sk, ostart = O.cell_sort(k, B * P)
    for _ in range(2):
        keys, perm, start = _call(h, x, B, P)
        assert np.array_equal(keys.numpy().astype(np.int64), sk)
        assert np.array_equal(perm.numpy().astype(np.int64), operm)
        assert np.array_equal(start.numpy().astype(np.int64), ostart)


def test_noalloc_leaves_free_device_memory_unchanged(h):
    """After one warm-up call (which loads the library's device code and
    looks up the scratch address), further calls of every size up to the
    limit leave the device's free memory exactly as it was."""
    sizes = (1 << 20, 10_000, 300_000, 1 << 20)
    nodes = [torch.tensor(track_hole_nodes(80 + i, n)[0], device="cuda") for i, n in enumerate(sizes)]
    B, P = 512, 1024
    outs = [(torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
             torch.empty(B * P + 1, dtype=torch.int32, device="cuda")) for n in sizes]
    h.cells_noalloc(nodes[0], B, P, *outs[0])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for x, o in zip(nodes, outs):
        h.cells_noalloc(x, B, P, *o)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversize_and_host_memory(h):
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
