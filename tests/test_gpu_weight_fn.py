"""The weight function phi of eq. weight_function_radial (Sec. 2.2 leaves the
Wendland function open; hamls_params.weight_fn): with phi_{3,1} the whole fit
(support radius through the Shepard weights, the local MLS weights, the
refit operator) matches the oracle run with the same phi, to the FP64 and
mixed bars of the default phi_{3,2}; an unknown weight_fn is rejected."""
import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import random_field_coeffs, synth_field, workload

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def small31():
    w = workload("s2_n16_k2_m5k")
    r = O.hamls(w.nodes, w.values, w.N, w.K, O.Params(weight_fn=1))
    r0 = O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    return w, r, r0


def test_fit_fp64_phi31_matches_oracle(h, small31):
    w, r, r0 = small31
    with h.Plan(dev(w.nodes), w.N, w.K, weight_fn=1) as p:
        c = p.fit(dev(w.values))
        g = p.debug_grid()
        p.sync(60000)
    f = g["f"].cpu().numpy()
    fo = r.fgrid.astype(float)
    assert np.max(np.abs(f - fo)) < 1e-10 * np.max(np.abs(fo))
    assert np.allclose(g["delta"].cpu().numpy(), r.support.delta.astype(float), rtol=1e-12)
    assert np.array_equal(g["count"].cpu().numpy(), r.support.count)
    assert np.allclose(g["chi"].cpu().numpy(), r.chi.astype(float), rtol=1e-8)
    assert np.allclose(g["tau"].cpu().numpy(), r.tau_tilde.astype(float), rtol=1e-8, atol=1e-14)
    assert relerr(h.to_complex(c), r.coeffs) < FP64_TOL
    # the choice matters: the default phi gives another fit
    assert relerr(r.coeffs, r0.coeffs) > 1e3 * FP64_TOL


def test_fit_mixed_phi31_matches_oracle(h, small31):
    w, r, _ = small31
    with h.Plan(dev(w.nodes), w.N, w.K, precision="mixed", weight_fn=1) as p:
        c = p.fit(dev(w.values))
        p.sync(60000)
    assert relerr(h.to_complex(c), r.coeffs) < MIXED_TOL


def test_refit_phi31_equals_fit(h, small31):
    w, r, _ = small31
    y2 = synth_field(random_field_coeffs(7, 12), w.nodes)
    with h.Plan(dev(w.nodes), w.N, w.K, weight_fn=1) as p:
        p.refit_prepare()
        a = h.to_complex(p.refit(dev(w.values)))
        b = h.to_complex(p.refit(dev(y2)))
        c = h.to_complex(p.fit(dev(y2)))
        p.sync(60000)
    assert relerr(a, r.coeffs) < FP64_TOL
    assert relerr(b, c) < FP64_TOL


def test_unknown_weight_fn_rejected(h, small31):
    w, _, _ = small31
    with pytest.raises(h.HamlsError) as e:
        h.Plan(dev(w.nodes), w.N, w.K, weight_fn=2)
    assert e.value.code == 1
