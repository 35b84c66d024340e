"""The tensor-core product (tcgen05, 3xTF32 with FP32 accumulation) behind
the batched Legendre contraction, against an FP64 product on the host:
elementwise within (3 2^-20 + K 2^-24) of the |A| |B|^T bound (the split
drops lo*lo and rounds each lo part to TF32, 2^-20 relative each, and the
products are accumulated in FP32), exactly on small integers (every partial
sum exact), on full, ragged and single tiles."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


@pytest.mark.parametrize("M,N,K", [(128, 32, 32), (128, 256, 256), (300, 70, 100), (64, 513, 260),
                                   (256, 96, 4), (129, 33, 36)])
def test_tc_gemm_matches_fp64(h, M, N, K):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C = h.debug_tc_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    tol = 3 * 2.0 ** -20 + K * 2.0 ** -24
    assert np.all(np.abs(C - exact) <= tol * bound + 1e-30)


def test_tc_gemm_exact_on_small_integers(h):
    rng = np.random.default_rng(5)
    A = rng.integers(-8, 9, size=(128, 64)).astype(np.float32)
    B = rng.integers(-8, 9, size=(64, 64)).astype(np.float32)
    C = h.debug_tc_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")).cpu().numpy()
    assert np.array_equal(C, (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float32))
