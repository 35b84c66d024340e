"""The forward transform F (Sec. 1, eq. LSQR-Problem_Regularized; hamls_forward)
against the oracle's forward() (oracle/forward.py, extended precision):

* N = 16 and N = 128 at random points, N = 512 at sampled points (the
  benchmark bandwidth), each with points exactly at both poles and 1e-3 rad
  from them (where the FP32 seed Pbar_m^m leaves the FP32 range long before
  Pbar_l^m is negligible);
* FP64 plans to 1e-11 of the field's largest value; mixed plans within the
  FP32 error bound of the sum, 2 (N + 3) 2^-24 times the sum of the terms'
  absolute values at each point (FP32 recurrence, carried exponent), and a
  median error below 1e-6 of the field's scale;
* at the plan's own nodes (sorted evaluation order, written back in node
  order) the same values as at the same points given explicitly, to device
  and to host buffers; applied to a fit's coefficients, the residual at the
  nodes;
* invalid arguments are rejected.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import SplitMix64, random_field_coeffs, uniform_sphere

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_39200_b300 as h
    h.lib()
    return h


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def packed(N, seed):
    c = random_field_coeffs(seed, N)
    return O.pack_coeffs(np.tril(c), N)


def as_pairs(cp):
    return np.ascontiguousarray(np.stack([cp.real, cp.imag], axis=1))


def special_points(seed, n):
    """n random points, both poles, and points 1e-3 rad from each pole."""
    x = uniform_sphere(SplitMix64(seed), n)
    extra = []
    for sgn in (1.0, -1.0):
        extra.append([0.0, 0.0, sgn])
        for a in (0.3, 2.1, 4.0):
            th = 1e-3
            extra.append([math.sin(th) * math.cos(a), math.sin(th) * math.sin(a), sgn * math.cos(th)])
    return np.concatenate([x, np.array(extra)])


@pytest.mark.parametrize("N,n", [(16, 300), (128, 200), (512, 24)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_matches_oracle(h, N, n, precision):
    cp = packed(N, 500 + N)
    pts = special_points(600 + N, n)
    exp = O.forward(cp, N, pts)
    nodes = dev(uniform_sphere(SplitMix64(1), 2000))
    with h.Plan(nodes, N, 1, precision=precision) as p:
        got = p.forward(dev(as_pairs(cp)), points=dev(pts))
        p.sync(120000)
    got = got.cpu().numpy()
    scale = np.max(np.abs(exp))
    err = np.abs(got - exp)
    if precision == "fp64":
        assert np.max(err) < 1e-11 * scale, (float(np.max(err) / scale), int(np.argmax(err)))
        return
    # FP32: the sum of (N + 1)(N + 2)/2 terms f_l^m Pbar_l^m(t) e^{i m phi},
    # each term's Pbar from a stable three-term recurrence (relative error
    # growing about linearly in l) and added in FP32, errs by at most about
    # 2 (N + 3) u sum |terms| (u = 2^-24); the absolute sum from the oracle's
    # Legendre values at each point. Near the poles the m = 0 order alone adds
    # N + 1 terms of size |f_l^0| sqrt((2 l + 1) / (4 pi)), so its bound is the
    # one that matters there.
    t = np.clip(pts[:, 2], -1.0, 1.0).astype(O.LD)
    absum = np.zeros(len(pts))
    for m in range(N + 1):
        P = np.abs(O.legendre_m(N, m, t)).astype(np.float64)
        o = O.coeff_offset(N, m)
        am = np.abs(cp[o:o + N + 1 - m])
        absum += (1.0 if m == 0 else 2.0) * (am @ P)
    tol = 2 * (N + 3) * 2.0 ** -24 * absum
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (float((err / tol)[worst]), worst, float(err[worst] / scale))
    # and away from the poles, a few FP32 roundings of the field's scale
    assert np.median(err) < 1e-6 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forward_at_plan_nodes(h, precision):
    N = 64
    x = uniform_sphere(SplitMix64(7), 30_000)
    cp = packed(N, 77)
    c = dev(as_pairs(cp))
    xd = dev(x)
    with h.Plan(xd, N, 2, precision=precision) as p:
        at_nodes = p.forward(c)
        at_points = p.forward(c, points=xd)
        host = torch.empty(len(x), dtype=torch.float64).pin_memory()
        p.forward(c.cpu().numpy(), out=host)
        p.sync(60000)
    assert torch.equal(at_nodes, at_points)
    assert torch.equal(at_nodes.cpu(), host)
    sel = np.arange(0, len(x), 997)
    exp = O.forward(cp, N, x[sel])
    tol = 1e-11 if precision == "fp64" else 3e-6
    assert np.max(np.abs(at_nodes.cpu().numpy()[sel] - exp)) < tol * np.max(np.abs(exp))


def test_forward_of_a_fit_is_its_residual(h):
    """F applied to a fit's coefficients at the nodes; the residual against
    the data is what the paper's least-squares problem measures."""
    from hamls_synth import workload
    w = workload("s2_n16_k2_m5k")
    r = O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        c = p.fit(dev(w.values))
        fx = p.forward(c)
        p.sync(60000)
    exp = O.forward(r.coeffs, w.N, w.nodes)
    assert np.max(np.abs(fx.cpu().numpy() - exp)) < 1e-9 * np.max(np.abs(exp))
    res = fx.cpu().numpy() - w.values
    assert np.sqrt(np.mean(res ** 2)) < 0.05 * np.sqrt(np.mean(w.values ** 2))


def test_forward_rejects_invalid_arguments(h):
    x = dev(uniform_sphere(SplitMix64(3), 1000))
    c = torch.zeros((O.n_coeffs(8), 2), dtype=torch.float64, device="cuda")
    with h.Plan(x, 8, 1) as p:
        host_pts = np.ascontiguousarray(uniform_sphere(SplitMix64(4), 10))
        with pytest.raises(h.HamlsError) as e:
            p.forward(c, points=host_pts, out=torch.empty(10, dtype=torch.float64, device="cuda"))
        assert e.value.code == 1
        with pytest.raises(h.HamlsError) as e:
            h.lib().hamls_forward  # noqa: B018
            from paper_2609_39200_b300 import _check, _ptr, _stream
            out = torch.empty(5, dtype=torch.float64, device="cuda")
            _check(h.lib().hamls_forward(p.h, _ptr(c), None, 5, _ptr(out), _stream(None)), "hamls_forward")
        assert e.value.code == 1
    with h.Plan(None, 8, 1, capacity=1000) as p:
        with pytest.raises(h.HamlsError):
            p.forward(c)
