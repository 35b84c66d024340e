"""Scheduling of many fits (paper_2609_39200_b300.batch) on the CPU with a
stand-in plan: plans are reused per (N, K, stream), created once per group
for a batch, never shared between streams, replaced when a request needs
more nodes, and results come back in input order."""
import dataclasses

import numpy as np

from hamls_synth import batch_specs, serving_trace


class FakePlan:
    log = []

    def __init__(self, nodes, N, K, precision, stream):
        self.N, self.K, self.cap, self.stream = N, K, len(nodes), stream
        self.streams = {stream}
        self.closed = False
        FakePlan.log.append(("create", N, K, len(nodes), stream))

    def replan(self, nodes, stream=None):
        assert not self.closed and len(nodes) <= self.cap
        self.streams.add(stream)

    def fit(self, values, out=None, stream=None):
        assert not self.closed
        self.streams.add(stream)
        return float(np.sum(values)) + 1000.0 * self.N + self.K

    def sync(self):
        pass

    def close(self):
        self.closed = True


def make_pool():
    from paper_2609_39200_b300.batch import PlanPool
    FakePlan.log = []
    made = []

    def factory(nodes, N, K, precision, stream):
        p = FakePlan(nodes, N, K, precision, stream)
        made.append(p)
        return p
    return PlanPool(factory), made


def load(s):
    rng = np.random.default_rng(s.seed % (2 ** 32))
    return np.zeros((s.M, 3)), rng.normal(size=s.M)


def small(specs):
    return [dataclasses.replace(s, M=max(3, s.M // 1000)) for s in specs]


def test_batch_plans_once_per_group_and_stream_in_order():
    from paper_2609_39200_b300.batch import run_batch
    fits = small(batch_specs(64))
    pool, made = make_pool()
    out = run_batch(fits, load, pool, n_streams=2)
    exp = [float(np.sum(load(s)[1])) + 1000.0 * s.N + s.K for s in fits]
    assert out == exp
    groups = {(s.N, s.K) for s in fits}
    per_group = {g: sum(1 for s in fits if (s.N, s.K) == g) for g in groups}
    assert pool.created == sum(min(2, c) for c in per_group.values())
    for p in made:
        assert len(p.streams) == 1                      # a plan never meets a second stream


def test_serving_replaces_plans_for_larger_requests():
    from paper_2609_39200_b300.batch import serve
    trace = small(serving_trace(50.0, 40))
    pool, made = make_pool()
    now = [0.0]

    def clock():
        now[0] += 1e-4
        return now[0]

    def wait(dt):
        now[0] += dt

    lat = serve(trace, load, pool, n_streams=2, clock=clock, wait=wait)
    assert lat.shape == (40,) and np.all(lat >= 0)
    for p in made:
        assert len(p.streams) == 1
    # a plan is created for the first request of its (N, K, stream slot) and
    # replaced exactly when a later request of that key needs more nodes
    cap, expected = {}, 0
    for i, r in enumerate(trace):
        key = (r.N, r.K, i % 2)
        if r.M > cap.get(key, 0):
            expected += 1
            cap[key] = r.M
    assert pool.created == expected
    assert sum(not p.closed for p in made) == len(cap)
