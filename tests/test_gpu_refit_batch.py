"""Refits of many value sets at fixed nodes (hamls_refit_batch): the stored
operator applied to every set in one pass, then the batched step 3 on the
tensor cores. Every set equals its own single refit (hamls_refit) to FP32
rounding for mixed plans (the sums run in another order), exactly for FP64
plans (the same kernels, set by set), including batches of more than 256
sets (done in passes) and a set whose values are not finite (reported by
hamls_sync)."""
import numpy as np
import pytest
import torch

from hamls_synth import SplitMix64, random_field_coeffs, synth_field, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def value_sets(x, B, L=48, seed=0):
    xt = torch.tensor(x, device="cuda")
    return torch.stack([synth_field(random_field_coeffs(seed + b, L), xt, torch) for b in range(B)]).contiguous()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_refit_batch_equals_single_refits(h, precision):
    w = workload("s2_n128_k3_m200k", xp=torch, device="cuda")
    Y = value_sets(w.nodes, 12, seed=40)
    with h.Plan(torch.tensor(w.nodes, device="cuda"), w.N, w.K, precision=precision) as p:
        p.refit_prepare()
        batch = p.refit_batch(Y)
        singles = [p.refit(Y[b].contiguous()).clone() for b in range(Y.shape[0])]
        p.sync(120000)
    for b in range(Y.shape[0]):
        if precision == "fp64":
            assert torch.equal(batch[b], singles[b])
        else:
            assert relerr(h.to_complex(batch[b]), h.to_complex(singles[b])) < 2e-5


def test_refit_batch_in_passes_and_nonfinite(h):
    w = workload("s2_n16_k2_m5k")
    B = 300
    Y = value_sets(w.nodes, B, L=16, seed=500)
    with h.Plan(torch.tensor(w.nodes, device="cuda"), w.N, w.K, precision="mixed") as p:
        p.refit_prepare()
        batch = p.refit_batch(Y)
        picks = (0, 255, 256, 299)
        singles = {b: p.refit(Y[b].contiguous()).clone() for b in picks}
        p.sync(60000)
        for b in picks:
            assert relerr(h.to_complex(batch[b]), h.to_complex(singles[b])) < 2e-5
        Y[7, 11] = float("nan")
        p.refit_batch(Y[:10].contiguous())
        with pytest.raises(h.HamlsError) as e:
            p.sync(60000)
        assert e.value.code == 7
