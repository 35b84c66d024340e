"""Many fits on one GPU: pools of plans reused across fits, and fits spread
over several CUDA streams.

A plan belongs to one bandwidth N, degree K and precision, and holds buffers
for up to the number of nodes it was created with. A later fit with that many
nodes or fewer reuses it through hamls_replan, which allocates nothing; a fit
with more nodes replaces it. A plan must not be used from two streams at
once, so every stream has plans of its own: fit i runs on stream i mod S with
that stream's plan for its (N, K), and the copies and host work of one fit
overlap the kernels of fits on the other streams.

For a known batch, run_batch orders each (N, K) group largest first, so each
stream's plan for it is created once; serve takes requests in arrival order
and replaces plans as larger requests come. Every fit is computed by the CUDA
library through the C ABI; this module only schedules.
"""
from __future__ import annotations

import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch


class PlanPool:
    """Plans keyed by (N, K, precision, stream slot). `factory(nodes, N, K,
    precision, stream)` makes a plan (the binding's Plan by default)."""

    def __init__(self, factory: Optional[Callable] = None):
        if factory is None:
            from . import Plan

            def factory(nodes, N, K, precision, stream):
                return Plan(nodes, N, K, precision=precision, stream=stream)
        self._factory = factory
        self._plans: Dict[Tuple[int, int, str, int], Tuple[object, int]] = {}
        self.created = 0

    def fit(self, nodes, values, N: int, K: int, precision: str = "mixed", slot: int = 0, stream=None, out=None):
        """Coefficients of one fit, asynchronous on `stream`; `slot` names the
        stream, and only fits of the same slot share a plan."""
        key = (int(N), int(K), precision, int(slot))
        M = int(nodes.shape[0])
        entry = self._plans.get(key)
        if entry is not None and M <= entry[1]:
            plan = entry[0]
            plan.replan(nodes, stream=stream)
        else:
            if entry is not None:
                entry[0].close()              # waits for the plan's own stream
            plan = self._factory(nodes, N, K, precision, stream)
            self._plans[key] = (plan, M)
            self.created += 1
        return plan.fit(values, out=out, stream=stream)

    def sync(self):
        for plan, _ in self._plans.values():
            plan.sync()

    def close(self):
        for plan, _ in self._plans.values():
            plan.close()
        self._plans.clear()


def _streams(n: int, device):
    if device is None:
        return [None] * n
    return [torch.cuda.Stream(device) for _ in range(n)]


def run_batch(fits: Sequence, load: Callable, pool: PlanPool, n_streams: int = 2, precision: str = "mixed",
              device=None) -> List:
    """Fit every spec of `fits` (objects with N, K, M); `load(spec)` returns
    (nodes, values). Each (N, K) group runs largest first, so every stream
    creates its plan for the group once. Returns the coefficient tensors in
    the order of `fits`."""
    groups: Dict[Tuple[int, int], list] = {}
    for pos, s in enumerate(fits):
        groups.setdefault((s.N, s.K), []).append(pos)
    order = []
    for key in sorted(groups):
        order += sorted(groups[key], key=lambda p: -fits[p].M)
    streams = _streams(n_streams, device)
    results: List = [None] * len(fits)
    for i, pos in enumerate(order):
        s = fits[pos]
        nodes, values = load(s)
        slot = i % n_streams
        results[pos] = pool.fit(nodes, values, s.N, s.K, precision, slot=slot, stream=streams[slot])
    pool.sync()
    return results


def serve(trace: Sequence, load: Callable, pool: PlanPool, n_streams: int = 2, precision: str = "mixed",
          device=None, clock: Callable[[], float] = time.perf_counter,
          wait: Callable[[float], None] = time.sleep) -> np.ndarray:
    """Serve requests (objects with arrival_s, N, K) in arrival order. A
    request is issued no earlier than its arrival (relative to the start);
    its latency runs from its arrival to the end of its fit on the GPU, taken
    from CUDA events on its stream (from the host clock after a wait when no
    device is given). Returns the latencies in seconds, in trace order."""
    streams = _streams(n_streams, device)
    use_events = device is not None
    if use_events:
        torch.cuda.synchronize(device)
        start = torch.cuda.Event(enable_timing=True)
        start.record(streams[0])
    t0 = clock()
    ends = [None] * len(trace)
    lat = np.zeros(len(trace))
    for i, s in enumerate(trace):
        now = clock() - t0
        if now < s.arrival_s:
            wait(s.arrival_s - now)
        nodes, values = load(s)
        slot = i % n_streams
        pool.fit(nodes, values, s.N, s.K, precision, slot=slot, stream=streams[slot])
        if use_events:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(streams[slot])
            ends[i] = ev
        else:
            pool.sync()
            lat[i] = (clock() - t0) - s.arrival_s
    if use_events:
        for i, ev in enumerate(ends):
            ev.synchronize()
            lat[i] = start.elapsed_time(ev) / 1000.0 - trace[i].arrival_s
    pool.sync()
    return lat
