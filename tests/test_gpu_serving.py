"""Many fits on the GPU (batched and serving forms, through the C ABI):

* a fit gives the same coefficients in a plan of any capacity that holds it
  (the cell structure follows the node count), so plans can be pooled;
* every request of a serving mix (continuous batching over several streams,
  plans reused, fits overlapping on the device) equals the same request
  fitted alone, including an N = 1024 request;
* a batch captured in one CUDA graph equals its fits run alone, replayed
  twice on plans that ran other fits before the capture;
* a fit with a non-finite value reports its own status in the batch while
  the fits around it (on the same plan) report none;
* the FP64 form of a batch matches the oracle's fits to 1e-10 on a subset.
"""
import dataclasses

import numpy as np
import pytest
import torch

from hamls_synth import FitSpec, fit_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


def _spec(i, N, K, M, holes=(10.0, 20.0), t=0.0):
    return FitSpec(i, N, K, M, holes, 0x5E57 ^ (i * 7919 + M), t)


_CACHE = {}


def _load(s):
    key = (s.seed, s.M)
    if key not in _CACHE:
        w = fit_workload(s, xp=torch, device="cuda", L_field=64)
        _CACHE[key] = (torch.tensor(w.nodes, device="cuda"), torch.tensor(w.values, device="cuda"))
    return _CACHE[key]


def _alone(h, s, precision):
    x, y = _load(s)
    with h.Plan(x, s.N, s.K, precision=precision) as p:
        c = p.fit(y)
        p.sync(120000)
        return c.clone()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fit_is_the_same_in_any_plan_that_holds_it(h, precision):
    s = _spec(1, 32, 3, 30_000)
    x, y = _load(s)
    ref = _alone(h, s, precision)
    with h.Plan(None, s.N, s.K, capacity=1 << 19, precision=precision) as p:
        big = _spec(2, 32, 3, 400_000)
        xb, yb = _load(big)
        p.replan(xb)
        p.fit(yb)
        p.replan(x)
        c = p.fit(y)
        p.sync(120000)
    assert torch.equal(c, ref)


def test_reserved_plan_rejects_fit_before_nodes(h):
    with h.Plan(None, 16, 2, capacity=10_000) as p:
        y = torch.zeros(100, dtype=torch.float64, device="cuda")
        with pytest.raises(h.HamlsError):
            p.fit(y)


def test_serving_mix_equals_alone(h):
    from paper_2609_39200_b300.batch import PlanPool, serve
    sizes = [(64, 60_000), (32, 150_000), (64, 20_000), (128, 90_000), (32, 40_000), (64, 200_000),
             (1024, 50_000), (128, 30_000), (32, 120_000), (64, 70_000)]
    # arrivals 1 ms apart: fits overlap on the device over four slots
    trace = [_spec(10 + i, N, 3, M, t=0.001 * i) for i, (N, M) in enumerate(sizes)]
    alone = [_alone(h, s, "mixed") for s in trace]
    pool = PlanPool(device=torch.device("cuda"), budget_bytes=24 << 30, min_capacity=1 << 15)
    try:
        res = serve(trace, _load, pool, n_slots=4, precision="mixed", device=torch.device("cuda"))
    finally:
        torch.cuda.synchronize()
    assert res.status == [0] * len(trace)
    assert len(set(res.slots)) > 1
    for i, s in enumerate(trace):
        assert torch.equal(res.outputs[i], alone[i]), f"request {i} (N={s.N}, M={s.M}) differs in the mix"
    assert np.all(res.latency_s > 0)
    pool.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_alone_and_reports_per_fit_status(h, graph):
    from paper_2609_39200_b300.batch import PlanPool, run_batch
    specs = [_spec(40 + i, N, K, M) for i, (N, K, M) in enumerate(
        [(32, 2, 20_000), (32, 3, 60_000), (64, 3, 40_000), (32, 2, 50_000), (64, 3, 15_000), (32, 3, 25_000),
         (64, 2, 80_000), (32, 2, 10_000)])]
    bad = 3                                            # a NaN value in the 4th fit
    alone = [_alone(h, s, "mixed") for s in specs]

    def load(s):
        x, y = _load(s)
        if s.index == specs[bad].index:
            y = y.clone()
            y[5] = float("nan")
        return x, y
    pool = PlanPool(device=torch.device("cuda"), min_capacity=1 << 15)
    if graph:
        # plans that have run other fits first, then a captured batch replayed
        # twice: a slot's fits change cell structure from one fit to the next,
        # and every replay must give the same as the fits alone
        run_batch(specs[::-1], load, pool, n_slots=3, precision="mixed", device=torch.device("cuda"))
    res = run_batch(specs, load, pool, n_slots=3, precision="mixed", device=torch.device("cuda"), graph=graph,
                    replays=2 if graph else 1)
    assert res.graph == graph
    st = np.array(res.status)
    assert st[bad] == 7 and np.all(np.delete(st, bad) == 0)
    for i in range(len(specs)):
        if i != bad:
            assert torch.equal(res.outputs[i], alone[i])
    pool.close()


def test_batch_fp64_matches_oracle(h):
    """A batch in the FP64 form (plans reused across fits of different node
    counts on two slots) against the oracle's whole fits."""
    import oracle as O
    from paper_2609_39200_b300.batch import PlanPool, run_batch
    specs = [_spec(60 + i, N, K, M, holes=holes) for i, (N, K, M, holes) in enumerate(
        [(16, 2, 4000, (10.0,)), (16, 3, 6000, ()), (32, 2, 5000, (20.0,)), (16, 2, 3000, ())])]
    pool = PlanPool(device=torch.device("cuda"), min_capacity=1 << 13)
    res = run_batch(specs, _load, pool, n_slots=2, precision="fp64", device=torch.device("cuda"))
    assert res.status == [0] * len(specs)
    for i, s in enumerate(specs):
        x, y = _load(s)
        r = O.hamls(x.cpu().numpy(), y.cpu().numpy(), s.N, s.K, O.Params())
        got = h.to_complex(res.outputs[i])
        assert np.linalg.norm(got - r.coeffs) / np.linalg.norm(r.coeffs) < 1e-10, f"fit {i} (N={s.N}, M={s.M})"
    pool.close()
