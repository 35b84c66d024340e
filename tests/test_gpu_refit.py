"""Values-only refits (new values at fixed nodes) through the C ABI, against
the CPU oracle and against a full fit (GPU only).

For fixed nodes every grid value is linear in the data (Sec. 2.3: the Gram
matrix, chi and tau~ depend on the nodes only), so hamls_refit_prepare keeps
the fit as a sparse operator and hamls_refit applies it. Bars as for
hamls_fit: FP64 relative coefficient error <= 1e-10; the mixed form within
the mixed fit's tolerances and error bar."""
import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import random_field_coeffs, remove_caps, synth_field, uniform_sphere, SplitMix64, workload

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
def small():
    w = workload("s2_n16_k2_m5k")
    y2 = synth_field(random_field_coeffs(7, 12), w.nodes)
    r1 = O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    r2 = O.hamls(w.nodes, y2, w.N, w.K, O.Params())
    return w, y2, r1, r2


def test_refit_fp64_equals_fit_and_oracle(h, small):
    w, y2, r1, r2 = small
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        p.refit_prepare()
        a = h.to_complex(p.refit(dev(w.values)))
        b = h.to_complex(p.refit(dev(y2)))
        c = h.to_complex(p.fit(dev(y2)))          # a fit leaves the operator in place
        d = h.to_complex(p.refit(dev(y2)))
        p.sync(60000)
    assert relerr(a, r1.coeffs) < FP64_TOL
    assert relerr(b, r2.coeffs) < FP64_TOL
    assert relerr(b, c) < FP64_TOL
    assert np.array_equal(b, d)


def test_refit_with_node_weights(h, small):
    w, y2, _, _ = small
    v = 0.5 + np.random.default_rng(3).random(w.M)      # per-node weights v_i > 0
    exp = O.hamls(w.nodes, y2, w.N, w.K, O.Params(), v=v).coeffs
    with h.Plan(dev(w.nodes), w.N, w.K, weights=dev(v)) as p:
        p.refit_prepare()
        got = h.to_complex(p.refit(dev(y2)))
        p.sync(60000)
    assert relerr(got, exp) < FP64_TOL


def test_refit_mixed_small(h, small):
    w, y2, r1, r2 = small
    with h.Plan(dev(w.nodes), w.N, w.K, precision="mixed") as p:
        p.refit_prepare()
        a = h.to_complex(p.refit(dev(w.values)))
        b = h.to_complex(p.refit(dev(y2)))
        p.sync(60000)
    assert relerr(a, r1.coeffs) < MIXED_TOL
    assert relerr(b, r2.coeffs) < MIXED_TOL


def test_refit_guard_path(h):
    # a coarse auxiliary grid with a wide Shepard radius triggers the guard
    x = remove_caps(uniform_sphere(SplitMix64(22), 4000), np.array([[0.0, 0.6, 0.8]]), np.array([0.45]))
    y = x[:, 1] ** 2 + x[:, 2]
    prm = dict(aux_points=200, aux_radius=6.0)
    r = O.hamls(x, y, 8, 2, O.Params(**prm))
    assert r.support.guarded.any()
    with h.Plan(dev(x), 8, 2, **prm) as p:
        p.refit_prepare()
        got = h.to_complex(p.refit(dev(y)))
        p.sync(60000)
        st = p.stats()
    assert st["n_guarded"] == int(r.support.guarded.sum())
    assert relerr(got, r.coeffs) < FP64_TOL


def test_refit_needs_an_operator_for_the_current_nodes(h, small):
    w, y2, r1, _ = small
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        with pytest.raises(h.HamlsError) as e:
            p.refit(dev(w.values))
        assert e.value.code == 1
        p.refit_prepare()
        p.refit(dev(w.values))
        p.replan(dev(w.nodes))
        with pytest.raises(h.HamlsError) as e:
            p.refit(dev(w.values))
        assert e.value.code == 1
        p.refit_prepare()
        got = h.to_complex(p.refit(dev(w.values)))
        p.sync(60000)
    assert relerr(got, r1.coeffs) < FP64_TOL


def test_refit_host_buffers(h, small):
    w, y2, _, _ = small
    with h.Plan(w.nodes, w.N, w.K) as p:
        p.refit_prepare()
        out = torch.empty((O.n_coeffs(w.N), 2), dtype=torch.float64).pin_memory()
        p.refit(y2, out=out)
        p.sync(60000)
        a = h.to_complex(out)
        b = h.to_complex(p.refit(dev(y2)))
        p.sync(60000)
    assert np.array_equal(a, b)


def test_refit_n128_both_forms(h):
    w = workload("s2_n128_k3_m200k", xp=torch, device="cuda")
    r = O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        p.refit_prepare()
        c64 = h.to_complex(p.refit(dev(w.values)))
        p.sync(120000)
    with h.Plan(dev(w.nodes), w.N, w.K, precision="mixed") as p:
        p.refit_prepare()
        cmx = h.to_complex(p.refit(dev(w.values)))
        fmx = h.to_complex(p.fit(dev(w.values)))
        p.sync(120000)
    assert relerr(c64, r.coeffs) < FP64_TOL
    assert relerr(cmx, r.coeffs) < 1e-3
    # the mixed refit is at least as close to the oracle as the mixed fit, to within 10 %
    assert relerr(cmx, r.coeffs) <= 1.1 * relerr(fmx, r.coeffs) + 1e-12
