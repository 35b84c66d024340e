"""Scheduling of many fits (paper_2609_39200_b300.batch) on the CPU with a
stand-in plan: plans are reserved per (N, K, slot) and capacity class, never
shared between slots, reused for smaller fits, evicted least recently used
when the memory budget needs room; every fit reports its own status (also
when it is not the last fit of its plan); results come back in input order;
requests are issued no earlier than their arrival."""
import dataclasses

import numpy as np
import pytest

from hamls_synth import batch_specs, serving_trace


class FakePlan:
    def __init__(self, capacity, N, K, precision, stream, fail_values=None):
        self.N, self.K, self.cap, self.stream = N, K, capacity, stream
        self.streams = {stream}
        self.closed = False
        self.M = 0
        self.flags = 0
        self.fail_values = fail_values

    def replan(self, nodes, stream=None):
        assert not self.closed and len(nodes) <= self.cap
        self.streams.add(stream)
        self.M = len(nodes)
        self.flags = 0

    def fit(self, values, out=None, stream=None):
        assert not self.closed and len(values) == self.M
        self.streams.add(stream)
        if self.fail_values is not None and np.any(values == self.fail_values):
            self.flags |= 4                     # the device would raise the non-finite flag
        return float(np.sum(values)) + 1000.0 * self.N + self.K

    def status_async(self, flags, stream=None):
        flags[0] = self.flags
        self.flags = 0

    def close(self):
        self.closed = True


def status_fn(f):
    return 7 if f & 4 else 0


def make_pool(budget=None, fail_values=None):
    from paper_2609_39200_b300.batch import PlanPool
    made = []

    def factory(capacity, N, K, precision, stream):
        p = FakePlan(capacity, N, K, precision, stream, fail_values)
        made.append(p)
        return p

    def footprint(capacity, N, K, precision):
        return capacity * 100 + N * N * 10

    return PlanPool(factory, footprint, budget_bytes=budget, min_capacity=1024, status_fn=status_fn), made


def load(s):
    rng = np.random.default_rng(s.seed % (2 ** 32))
    return np.zeros((s.M, 3)), rng.normal(size=s.M)


def small(specs):
    return [dataclasses.replace(s, M=max(50, s.M // 100)) for s in specs]


def test_capacity_class():
    from paper_2609_39200_b300.batch import capacity_class
    assert capacity_class(1, 1024) == 1024
    assert capacity_class(1024, 1024) == 1024
    assert capacity_class(1025, 1024) == 2048
    assert capacity_class(5_000_000, 1 << 16) == 1 << 23


def test_batch_reserves_once_per_slot_group_in_order():
    from paper_2609_39200_b300.batch import assign_slots, capacity_class, run_batch
    fits = small(batch_specs(64))
    pool, made = make_pool()
    res = run_batch(fits, load, pool, n_slots=3)
    exp = [float(np.sum(load(s)[1])) + 1000.0 * s.N + s.K for s in fits]
    assert res.outputs == exp
    assert res.status == [0] * len(fits)
    slots = assign_slots(fits, 3)
    assert res.slots == slots
    # one plan per (slot, N, K), holding the slot's largest fit of that group
    need = {}
    for s, j in zip(fits, slots):
        need[(s.N, s.K, j)] = max(need.get((s.N, s.K, j), 0), s.M)
    assert pool.created == len(need)
    for p in made:
        assert len(p.streams) == 1                      # a plan never meets a second stream
    caps = sorted((p.N, p.K, p.cap) for p in made)
    assert caps == sorted((N, K, capacity_class(M, 1024)) for (N, K, j), M in need.items())


def test_slots_are_balanced():
    from paper_2609_39200_b300.batch import assign_slots
    fits = batch_specs(256)
    for n in (2, 4, 8):
        slots = assign_slots(fits, n)
        load_ = np.zeros(n)
        for s, j in zip(fits, slots):
            load_[j] += s.M + 2 * (s.N + 1) * (2 * s.N + 2)
        assert load_.max() / load_.mean() < 1.05


def test_error_of_a_fit_that_is_not_the_last_on_its_plan_is_reported():
    from paper_2609_39200_b300.batch import run_batch
    fits = small(batch_specs(24))
    poison = 12.5
    bad = {3, 10}
    inputs = {}

    def load_bad(s):
        x, y = load(s)
        if s.index in bad:
            y = y.copy()
            y[0] = poison
        inputs[s.index] = y
        return x, y
    pool, made = make_pool(fail_values=poison)
    res = run_batch(fits, load_bad, pool, n_slots=2)
    assert [i for i, st in enumerate(res.status) if st] == sorted(bad)
    # the failing fits shared their plan with later fits
    for i in bad:
        later = [k for k in range(len(fits)) if res.slots[k] == res.slots[i] and
                 (fits[k].N, fits[k].K) == (fits[i].N, fits[i].K) and k != i]
        assert later


def test_serving_issues_after_arrival_and_reuses_plans():
    from paper_2609_39200_b300.batch import capacity_class, serve
    trace = small(serving_trace(50.0, 40))
    pool, made = make_pool()
    now = [0.0]

    def clock():
        now[0] += 1e-5
        return now[0]

    def wait(dt):
        now[0] += dt

    res = serve(trace, load, pool, n_slots=2, clock=clock, wait=wait)
    assert res.latency_s.shape == (40,) and np.all(res.latency_s >= 0)
    assert np.all(res.queue_s >= 0)
    assert res.issued_order == list(range(40))      # arrival order
    for p in made:
        assert len(p.streams) == 1
    # one plan per (N, K, slot) and capacity class actually needed
    classes = {(r.N, r.K, res.slots[i], capacity_class(r.M, 1024)) for i, r in enumerate(trace)}
    assert pool.created <= len(classes)
    exp = [float(np.sum(load(s)[1])) + 1000.0 * s.N + s.K for s in trace]
    assert res.outputs == exp


def test_budget_evicts_least_recently_used_idle_plans():
    from paper_2609_39200_b300.batch import PlanPool
    pool, made = make_pool(budget=10 * (1024 * 100 + 64 * 64 * 10))
    # fill with plans of slot 0 for ten different N
    for i, N in enumerate(range(10, 20)):
        assert pool.reserve(N, 3, "mixed", 0, 100) is not None
    assert pool.evicted == 0
    used = pool.used_bytes
    # a large plan needs room: the oldest idle plans go first
    assert pool.reserve(64, 3, "mixed", 1, 5000) is not None
    assert pool.evicted > 0 and pool.used_bytes <= pool.budget
    assert made[0].closed and not made[9].closed
    # plans of busy slots are never evicted; if nothing idle is left, no room
    big = pool.budget
    assert pool.reserve(128, 3, "mixed", 2, big, busy_slots={0, 1}) is None
    assert not made[9].closed
    assert used > 0
