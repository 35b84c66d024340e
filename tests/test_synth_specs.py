"""The seeded recipes for many fits (CPU): a batch of independent fits of
mixed sizes, and a serving trace of Poisson arrivals with a size mix. They
draw only random numbers (no HAMLS arithmetic) and must be reproducible and
follow their stated distributions."""
import dataclasses
import math

import numpy as np

from hamls_synth import batch_specs, fit_workload, serving_trace


def test_batch_is_reproducible_and_in_range():
    a, b = batch_specs(), batch_specs()
    assert a == b and len(a) == 256
    assert {s.N for s in a} == {32, 64, 128, 256}
    assert all(1e4 <= s.M <= 1e6 for s in a)
    assert {s.K for s in a} == {2, 3}
    assert {s.holes_deg for s in a} == {(), (10.0,), (10.0, 20.0), (10.0, 20.0, 35.0)}
    assert len({s.seed for s in a}) == 256


def test_batch_distributions():
    a = batch_specs(4096)
    for N in (32, 64, 128, 256):
        assert abs(sum(s.N == N for s in a) / 4096 - 0.25) < 0.03
    lm = np.log10([s.M for s in a])
    assert abs(lm.mean() - 5.0) < 0.05 and abs(lm.std() - 2 / math.sqrt(12)) < 0.03
    assert abs(sum(s.K == 3 for s in a) / 4096 - 0.5) < 0.03


def test_serving_trace_is_poisson_with_the_size_mix():
    r = serving_trace(20.0, 20000)
    t = np.array([s.arrival_s for s in r])
    gaps = np.diff(np.r_[0.0, t])
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 20.0 - 1) < 0.03                    # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05              # exponential: cv = 1
    for N, p in zip((64, 128, 256, 512, 1024), (0.30, 0.30, 0.20, 0.15, 0.05)):
        assert abs(sum(s.N == N for s in r) / 20000 - p) < 0.015
    lm = np.log10([s.M for s in r])
    assert lm.min() >= math.log10(5e4) - 1e-9 and lm.max() <= math.log10(1.6e7) + 1e-9
    assert all(s.K == 3 and s.holes_deg == (10.0, 20.0, 35.0) for s in r)


def test_one_fit_has_its_size_and_holes():
    spec = dataclasses.replace(batch_specs()[2], M=6000)          # two holes
    w = fit_workload(spec, L_field=20)
    assert w.nodes.shape == (6000, 3) and np.all(np.isfinite(w.values))
    np.testing.assert_allclose(np.linalg.norm(w.nodes, axis=1), 1.0, atol=1e-14)
    for c, r in zip(w.meta["cap_centres"], w.meta["cap_radii"]):
        assert np.all(w.nodes @ c <= math.cos(r))
    assert len(w.meta["cap_radii"]) == len(spec.holes_deg)
    assert np.array_equal(fit_workload(spec, L_field=20).values, w.values)
