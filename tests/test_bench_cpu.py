"""The benchmark's CPU-oracle estimate (bench.OracleBaseline) against the
oracle's directly timed whole fit, on the workload small enough to time in
full (N = 16, M = 5,000). The estimate times each part on its own and
scales it to a whole fit; it must land near the real time."""
import importlib.util
import os
import time

import oracle as O
from hamls_synth import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sampled_estimate_matches_a_whole_fit():
    bench = load_bench()
    w = workload("s2_n16_k2_m5k")
    est = bench.OracleBaseline(w, 96).estimate()
    assert est["value"] > 0
    t0 = time.perf_counter()
    O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    whole = time.perf_counter() - t0
    ratio = (1.0 / est["value"]) / whole
    assert 0.5 < ratio < 2.0, (ratio, est["sample"], whole)
