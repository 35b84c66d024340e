"""Many fits on one GPU: device-resident plans reused across fits, fits spread
over CUDA streams ("slots"), and admission by device-memory footprint.

A plan belongs to one bandwidth N, degree K and precision and holds buffers
for up to its capacity of nodes. Plans are reserved per capacity class (the
next power of two of the node count, at least ``min_capacity``) and reused
through hamls_replan, which allocates nothing; the library chooses the cell
structure from the node count alone, so a fit gives the same coefficients in
every plan that can hold it. A plan must not be used from two streams at
once, so every slot has plans of its own.

``serve`` is continuous batching: a request is issued as soon as it has
arrived, a slot is free and its plan fits the memory budget (idle plans are
evicted, least recently used first, to make room); requests on different
slots run concurrently on the device, and a slot takes its next request as
soon as its previous fit has completed. ``run_batch`` issues a known batch
over all slots at once, optionally captured in one CUDA graph and replayed.

Every fit gets its own device status word (hamls_status_async, copied back
without a host wait), so an error of one fit is reported with that fit even
when its plan is replanned for the next. Every fit is computed by the CUDA
library through the C ABI; this module only schedules.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

try:
    import torch
except ImportError:        # the scheduling logic itself needs no torch
    torch = None


def capacity_class(M: int, min_capacity: int = 1 << 16) -> int:
    """Smallest power of two >= max(M, min_capacity)."""
    c = max(int(min_capacity), 1)
    c = 1 << (c - 1).bit_length()
    while c < M:
        c <<= 1
    return c


@dataclass
class FitHandle:
    """One issued fit: its output, status slot and completion event."""
    index: int
    slot: int
    key: tuple
    out: object = None
    flags: object = None            # int32 element (pinned host) receiving the status word
    event: object = None            # CUDA event recorded after the fit (None: already complete)
    issued_s: float = 0.0
    status_fn: Optional[Callable] = None

    def done(self) -> bool:
        return self.event is None or bool(self.event.query())

    def status(self) -> int:
        """hamls_status of this fit (0 = ok); valid once done()."""
        if self.flags is None or self.status_fn is None:
            return 0
        if self.event is not None:
            self.event.synchronize()
        return int(self.status_fn(int(self.flags.reshape(-1)[0])))


@dataclass
class _Entry:
    plan: object
    capacity: int
    nbytes: int
    last_use: int = 0


class PlanPool:
    """Plans keyed by (N, K, precision, slot), each list sorted by capacity.

    factory(capacity, N, K, precision, stream) -> a plan without nodes
        (default: the binding's reserved Plan, hamls_plan_reserve);
    footprint(capacity, N, K, precision) -> its device bytes
        (default: hamls_plan_footprint);
    budget_bytes: device memory the pool may hold (None: unlimited);
    status_fn(flags) -> hamls_status of a status word (default: the
        binding's status_from_flags)."""

    def __init__(self, factory: Optional[Callable] = None, footprint: Optional[Callable] = None,
                 budget_bytes: Optional[int] = None, min_capacity: int = 1 << 16, device=None,
                 status_fn: Optional[Callable] = None):
        if factory is None or footprint is None:
            from . import Plan, plan_footprint

            def _factory(capacity, N, K, precision, stream):
                return Plan(None, N, K, capacity=capacity, precision=precision, stream=stream)

            def _footprint(capacity, N, K, precision):
                return plan_footprint(capacity, N, K, precision=precision)
            factory = factory or _factory
            footprint = footprint or _footprint
        self._factory, self._footprint = factory, footprint
        self.budget = budget_bytes
        self.min_capacity = int(min_capacity)
        self.device = device
        self._plans: Dict[Tuple[int, int, str, int], List[_Entry]] = {}
        self.used_bytes = 0
        self.created = 0
        self.evicted = 0
        self._tick = 0
        if status_fn is None:
            from . import status_from_flags as status_fn
        self._status_fn = status_fn

    # ------------------------------------------------------------- plans
    def _find(self, key, M) -> Optional[_Entry]:
        for e in self._plans.get(key, []):
            if e.capacity >= M:
                return e
        return None

    def _evict_for(self, need: int, busy_slots) -> bool:
        """Evict idle plans (slots not in busy_slots), least recently used
        first, until need more bytes fit the budget."""
        if self.budget is None or self.used_bytes + need <= self.budget:
            return True
        idle = [(e.last_use, key, e) for key, lst in self._plans.items() if key[3] not in busy_slots for e in lst]
        idle.sort(key=lambda t: t[0])
        for _, key, e in idle:
            if self.used_bytes + need <= self.budget:
                break
            self._plans[key].remove(e)
            e.plan.close()
            self.used_bytes -= e.nbytes
            self.evicted += 1
        return self.used_bytes + need <= self.budget

    def admissible(self, N, K, precision, slot, M, busy_slots=()) -> bool:
        """True if a fit of M nodes can run on `slot` now: a plan exists, or
        one fits the budget once idle plans are evicted."""
        key = (int(N), int(K), precision, int(slot))
        if self._find(key, M) is not None:
            return True
        cap = capacity_class(M, self.min_capacity)
        return self._evict_for(self._footprint(cap, N, K, precision), set(busy_slots) - {slot})

    def reserve(self, N, K, precision, slot, M, stream=None, busy_slots=()):
        """The plan of `slot` for a fit of M nodes, created (capacity class of
        M) if needed; None if the budget cannot hold it."""
        key = (int(N), int(K), precision, int(slot))
        e = self._find(key, M)
        if e is None:
            cap = capacity_class(M, self.min_capacity)
            nb = self._footprint(cap, N, K, precision)
            if not self._evict_for(nb, set(busy_slots) - {slot}):
                return None
            e = _Entry(self._factory(cap, N, K, precision, stream), cap, nb)
            lst = self._plans.setdefault(key, [])
            lst.append(e)
            lst.sort(key=lambda x: x.capacity)
            self.used_bytes += nb
            self.created += 1
        self._tick += 1
        e.last_use = self._tick
        return e.plan

    def plans(self):
        return [e.plan for lst in self._plans.values() for e in lst]

    # ------------------------------------------------------------- fits
    def issue(self, nodes, values, N, K, precision, slot, stream=None, index=0, out=None, flags=None,
              busy_slots=()) -> FitHandle:
        """replan + fit + status copy on `stream` (the slot's stream);
        returns at once. Inputs written on the caller's current stream are
        waited for; the slot stream owns the output's memory."""
        plan = self.reserve(N, K, precision, slot, int(nodes.shape[0]), stream, busy_slots)
        if plan is None:
            raise MemoryError(f"fit {index}: no room for a plan of {int(nodes.shape[0])} nodes")
        key = (int(N), int(K), precision, int(slot))
        h = FitHandle(index, slot, key, issued_s=time.perf_counter(), status_fn=self._status_fn)
        if self.device is None or stream is None:
            plan.replan(nodes, stream=stream)
            h.out = plan.fit(values, out=out, stream=stream)
            h.flags = flags if flags is not None else np.zeros(1, dtype=np.int32)
            plan.status_async(h.flags, stream=stream)
            return h
        caller = torch.cuda.current_stream(self.device)
        stream.wait_stream(caller)
        if not torch.cuda.is_current_stream_capturing():
            for t in (nodes, values):
                if isinstance(t, torch.Tensor) and t.is_cuda:
                    t.record_stream(stream)
        with torch.cuda.stream(stream):
            if out is None:
                out = torch.empty(((N + 1) * (N + 2) // 2, 2), dtype=torch.float64, device=self.device)
            plan.replan(nodes, stream=stream)
            h.out = plan.fit(values, out=out, stream=stream)
            if flags is None:
                flags = torch.zeros(1, dtype=torch.int32, pin_memory=True)
            plan.status_async(flags, stream=stream)
            h.flags = flags
            h.event = torch.cuda.Event(enable_timing=True)
            h.event.record(stream)
        return h

    def close(self):
        for lst in self._plans.values():
            for e in lst:
                e.plan.close()
        self._plans.clear()
        self.used_bytes = 0


def _streams(n: int, device):
    if device is None:
        return [None] * n
    return [torch.cuda.Stream(device) for _ in range(n)]


def assign_slots(fits: Sequence, n_slots: int, cost: Optional[Callable] = None) -> List[int]:
    """Slot of every fit: fits sorted by (N, K), then by falling cost, each
    given to the slot with the least work so far (longest processing time
    first), so each slot meets each (N, K) group in one run of fits and the
    slots finish together. cost(spec) defaults to M + 2 M_Q."""
    if cost is None:
        def cost(s):
            return s.M + 2 * (s.N + 1) * (2 * s.N + 2)
    order = sorted(range(len(fits)), key=lambda i: (fits[i].N, fits[i].K, -cost(fits[i])))
    load = [0.0] * n_slots
    slot = [0] * len(fits)
    for i in order:
        j = int(np.argmin(load))
        slot[i] = j
        load[j] += cost(fits[i])
    return slot


@dataclass
class BatchResult:
    outputs: list
    status: list
    slots: list
    graph: bool = False
    seconds: float = 0.0


def run_batch(fits: Sequence, load: Callable, pool: PlanPool, n_slots: int = 4, precision: str = "mixed",
              device=None, graph: bool = False, replays: int = 1) -> BatchResult:
    """Fit every spec of `fits` (objects with N, K, M); `load(spec)` returns
    (nodes, values) (device tensors for a graph). Plans are reserved for
    every (slot, N, K) first; the fits of each slot then run in order on that
    slot's stream, all slots concurrently. With graph=True the whole batch is
    captured in one CUDA graph (every replan, fit and status copy) and
    replayed `replays` times. Returns outputs and statuses in input order."""
    slots = assign_slots(fits, n_slots)
    inputs = [load(s) for s in fits]
    streams = _streams(n_slots, device)
    # reserve, for each slot and (N, K), a plan for the largest fit it gets
    need: Dict[tuple, int] = {}
    for s, j in zip(fits, slots):
        k = (s.N, s.K, j)
        need[k] = max(need.get(k, 0), s.M)
    for (N, K, j), M in need.items():
        if pool.reserve(N, K, precision, j, M, streams[j]) is None:
            raise MemoryError(f"no room for the plans of slot {j}, N={N}, K={K}")
    order = sorted(range(len(fits)), key=lambda i: (slots[i], fits[i].N, fits[i].K, -fits[i].M))
    outs: list = [None] * len(fits)
    flags = None
    if device is not None:
        torch.cuda.synchronize(device)
        flags = torch.zeros(len(fits), dtype=torch.int32, pin_memory=True)
        for i, s in enumerate(fits):
            outs[i] = torch.empty(((s.N + 1) * (s.N + 2) // 2, 2), dtype=torch.float64, device=device)

    def issue_all():
        hs = []
        for i in order:
            nodes, values = inputs[i]
            s = fits[i]
            hs.append(pool.issue(nodes, values, s.N, s.K, precision, slots[i], streams[slots[i]], index=i,
                                 out=outs[i], flags=None if flags is None else flags[i:i + 1]))
        return hs

    t0 = time.perf_counter()
    if graph and device is not None:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device)
        cap.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.graph(g, stream=cap):
            for st in streams:
                st.wait_stream(cap)
            handles = issue_all()
            for st in streams:
                cap.wait_stream(st)
        t0 = time.perf_counter()
        for _ in range(replays):
            g.replay()
        torch.cuda.synchronize(device)
        for h in handles:
            h.event = None          # events inside a graph are not queried: the replay is complete
    else:
        handles = issue_all()
        if device is not None:
            torch.cuda.synchronize(device)
    secs = time.perf_counter() - t0
    res_out: list = [None] * len(fits)
    res_st: list = [0] * len(fits)
    for h in handles:
        res_out[h.index] = h.out
        res_st[h.index] = h.status()
    return BatchResult(res_out, res_st, slots, graph=bool(graph and device is not None), seconds=secs)


@dataclass
class ServeResult:
    latency_s: np.ndarray           # arrival -> fit complete on the device
    queue_s: np.ndarray             # arrival -> issued
    outputs: list
    status: list
    slots: list
    makespan_s: float = 0.0
    issued_order: list = field(default_factory=list)


def serve(trace: Sequence, load: Callable, pool: PlanPool, n_slots: int = 4, precision: str = "mixed",
          device=None, clock: Callable[[], float] = time.perf_counter,
          wait: Callable[[float], None] = time.sleep, keep_outputs: bool = True, poll_s: float = 2e-5) -> ServeResult:
    """Serve requests (objects with arrival_s, N, K, M; in arrival order) by
    continuous batching over `n_slots` streams. A request is issued no
    earlier than its arrival (relative to the start), on a free slot
    (preferring one that already holds a plan for it), once its plan fits
    the pool's memory budget; a slot is free again as soon as its fit has
    completed on the device. Latency runs from arrival to the end of the fit
    on the device (CUDA events; host clock without a device)."""
    n = len(trace)
    streams = _streams(n_slots, device)
    use_events = device is not None
    if use_events:
        torch.cuda.synchronize(device)
        start = torch.cuda.Event(enable_timing=True)
        start.record(streams[0])
    t0 = clock()
    pending = list(range(n))
    free = list(range(n_slots))
    running: Dict[int, FitHandle] = {}
    lat = np.zeros(n)
    queue = np.zeros(n)
    outs: list = [None] * n
    stat: list = [0] * n
    slot_of: list = [0] * n
    handles: Dict[int, FitHandle] = {}
    issued = []
    done_host = np.zeros(n)

    def retire(h: FitHandle):
        stat[h.index] = h.status()
        if keep_outputs:
            outs[h.index] = h.out
        if not use_events:
            done_host[h.index] = clock() - t0

    while pending or running:
        progressed = False
        for j, h in list(running.items()):
            if h.done():
                retire(h)
                del running[j]
                free.append(j)
                progressed = True
        now = clock() - t0
        while pending and free and trace[pending[0]].arrival_s <= now:
            r = trace[pending[0]]
            # a free slot that already holds a plan for the request, else any
            pick = next((j for j in free if pool._find((r.N, r.K, precision, j), r.M) is not None), free[0])
            if not pool.admissible(r.N, r.K, precision, pick, r.M, busy_slots=running.keys()):
                break                               # wait for memory to free up
            i = pending.pop(0)
            free.remove(pick)
            nodes, values = load(r)
            queue[i] = (clock() - t0) - r.arrival_s
            h = pool.issue(nodes, values, r.N, r.K, precision, pick, streams[pick], index=i,
                           busy_slots=running.keys())
            slot_of[i] = pick
            handles[i] = h
            issued.append(i)
            if h.event is None:                     # no device: complete at once
                retire(h)
                free.append(pick)
            else:
                running[pick] = h
            progressed = True
        if not progressed:
            now = clock() - t0
            if not running and pending:
                wait(max(0.0, trace[pending[0]].arrival_s - now))
            else:
                nxt = trace[pending[0]].arrival_s - now if pending else poll_s
                wait(max(0.0, min(poll_s, nxt)))
    makespan = clock() - t0
    for i in range(n):
        if use_events:
            lat[i] = start.elapsed_time(handles[i].event) / 1000.0 - trace[i].arrival_s
        else:
            lat[i] = done_host[i] - trace[i].arrival_s
    return ServeResult(lat, queue, outs, stat, slot_of, makespan, issued)


class SlotTuner:
    """Autotuner of the batched form's launch configuration: the number of
    concurrent streams (slots) a batch is spread over. For each batch shape
    (the multiset of (N, K) and the capacity classes) it times one graph
    replay per candidate the first time the shape is seen and keeps the
    fastest; later batches of the same shape reuse the choice."""

    def __init__(self, candidates=(2, 4, 8)):
        self.candidates = tuple(candidates)
        self.cache: Dict[tuple, int] = {}
        self.trials: Dict[tuple, Dict[int, float]] = {}

    @staticmethod
    def shape(fits, min_capacity=1 << 16) -> tuple:
        return tuple(sorted((s.N, s.K, capacity_class(s.M, min_capacity)) for s in fits))

    def choose(self, fits, load, pool: PlanPool, precision="mixed", device=None) -> int:
        key = self.shape(fits, pool.min_capacity)
        if key in self.cache:
            return self.cache[key]
        times = {}
        for n in self.candidates:
            r = run_batch(fits, load, pool, n_slots=n, precision=precision, device=device, graph=device is not None)
            times[n] = r.seconds
        best = min(times, key=times.get)
        self.cache[key] = best
        self.trials[key] = times
        return best
