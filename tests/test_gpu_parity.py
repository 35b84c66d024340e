"""Parity of the CUDA library with the CPU oracle, stage by stage and end to
end, on seeded inputs (GPU only).

Bars: bit-exact for cell keys, sort permutation, CSR runs, k-NN radii and
local node sets; relative coefficient error <= 1e-10 for the FP64 form; the
mixed form within a tolerance that follows from its FP32 moments (about
1e-6 relative per moment, amplified by the conditioned local solves: <= 1e-4
relative on the coefficients here) and within 1.05x of the oracle's error
against the known truth."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import SplitMix64, random_field_coeffs, synth_field, uniform_sphere, workload, remove_caps

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
    r = O.hamls(w.nodes, w.values, w.N, w.K, O.Params())
    return w, r


# ------------------------------------------------------------------ step 1
@pytest.mark.parametrize("N", [1, 2, 16, 63, 128, 512])
def test_gauss_legendre_nodes(h, N):
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1) as p:
        t, w = p.debug_gl()
        p.sync(60000)
    to, wo = O.gauss_legendre(N + 1)
    assert np.max(np.abs(t.cpu().numpy() - to.astype(float))) < 2e-16 * (N + 1)
    assert np.max(np.abs(w.cpu().numpy() / wo.astype(float) - 1)) < 5e-14


# --------------------------------------------------------- neighbour structure
@pytest.mark.parametrize("M,seed", [(5000, 1), (77777, 2), (200_000, 3)])
def test_cell_keys_sort_and_runs_bit_exact(h, M, seed):
    x, _ = __import__("hamls_synth").track_hole_nodes(seed, M)
    x[:3] = [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [-1.0, 0.0, 0.0]]     # poles and the phi = pi seam
    with h.Plan(dev(x), 8, 2) as p:
        keys, perm, start, B, P = p.debug_cells()
        p.sync(60000)
    k = O.cell_keys(x, B, P)
    operm, sk, ostart = O.cell_sort(k, B * P)
    assert np.array_equal(keys.cpu().numpy().astype(np.int64), sk)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)
    assert np.array_equal(start.cpu().numpy().astype(np.int64), ostart)


def _edge_points(B, P, k, seed):
    """Unit vectors on and next to band edges (zeta = -1 + 2b/B) and cell
    edges (|y|/(|x|+|y|) = w/(P/4)), where the key's integer part is decided
    by the last bits of the FP64 arithmetic."""
    rng = np.random.default_rng(seed)
    # a third of the edges moved by 0.0021..0.01 of a band or cell: just
    # outside the FP32 fast path's guard band, where that path must agree
    near = np.where(rng.random(k) < 1 / 3, rng.choice([-1.0, 1.0], k) * rng.uniform(0.0021, 0.01, k), 0.0)
    b = rng.integers(1, B, k)
    zeta = -1.0 + 2.0 * (b + near) / B
    z = np.where(zeta >= 0, 1.0 - (1.0 - zeta) ** 2, (1.0 + zeta) ** 2 - 1.0)
    z = z + rng.choice([-1.0, 0.0, 1.0], k) * np.spacing(np.abs(z) + 1e-300) * rng.integers(0, 3, k)
    qc = P // 4
    w = np.clip(rng.integers(0, qc + 1, k) + near, 0, qc)
    ay, ax = w / qc, 1.0 - w / qc
    sx, sy = rng.choice([-1.0, 1.0], k), rng.choice([-1.0, 1.0], k)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    nrm = np.hypot(ax, ay)
    x = np.stack([sx * ax / nrm * rho, sy * ay / nrm * rho, z], axis=1)
    # half of them with only the band edge, at a random longitude
    phi = rng.uniform(0, 2 * np.pi, k)
    half = rng.random(k) < 0.5
    x[half, 0], x[half, 1] = rho[half] * np.cos(phi[half]), rho[half] * np.sin(phi[half])
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def test_cell_keys_on_edges_bit_exact(h):
    # 20000 nodes give 128 bands of 256 cells
    x = _edge_points(128, 256, 20000, 9)
    with h.Plan(dev(x), 8, 2) as p:
        keys, perm, start, B, P = p.debug_cells()
        p.sync(60000)
    assert (B, P) == (128, 256)
    operm, sk, ostart = O.cell_sort(O.cell_keys(x, B, P), B * P)
    assert np.array_equal(keys.cpu().numpy().astype(np.int64), sk)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm)


@pytest.mark.parametrize("n", [1, 6, 24, 40, 128])
def test_knn_bit_exact(h, n):
    x, _ = __import__("hamls_synth").track_hole_nodes(11, 30000)
    q = np.concatenate([uniform_sphere(SplitMix64(12), 3000), O.fibonacci_points(500),
                        [[0, 0, 1.0], [0, 0, -1.0]]])
    with h.Plan(dev(x), 8, 2) as p:
        got = p.debug_knn(dev(q), n)
        p.sync(120000)
    exp = O.NodeSet(x).knn_chord2(q, n)
    assert np.array_equal(got.cpu().numpy(), exp)


def test_knn_inside_large_hole(h):
    # queries deep inside a 60 degree hole: the search must grow far
    x = remove_caps(uniform_sphere(SplitMix64(5), 20000), np.array([[0.0, 0.0, 1.0]]), np.array([math.radians(60)]))
    q = uniform_sphere(SplitMix64(6), 400)
    q = q[q[:, 2] > 0.6]
    with h.Plan(dev(x), 8, 2) as p:
        got = p.debug_knn(dev(q), 40)
        p.sync(120000)
    assert np.array_equal(got.cpu().numpy(), O.NodeSet(x).knn_chord2(q, 40))


def test_local_node_sets_bit_exact(h):
    x, _ = __import__("hamls_synth").track_hole_nodes(21, 50000)
    rng = SplitMix64(22)
    q = np.concatenate([uniform_sphere(rng, 2000), [[0, 0, 1.0], [0, 0, -1.0]]])
    r = np.concatenate([0.002 + 0.1 * rng.uniform(2000) ** 3, [0.05, 0.3]])
    rho2 = (2 * np.sin(r / 2)) ** 2
    ns = O.NodeSet(x)
    with h.Plan(dev(x), 8, 2) as p:
        cnt, ids, hx = p.debug_ball(dev(q), dev(rho2))
        p.sync(120000)
    cnt, ids, hx = cnt.cpu().numpy(), ids.cpu().numpy(), hx.cpu().numpy().view(np.uint64)
    for j in range(len(q)):
        idx = ns.ball(q[j], rho2[j])
        assert cnt[j] == len(idx)
        assert ids[j] == int(idx.sum())
        from hamls_synth.gen import _mix64
        hh = np.bitwise_xor.reduce(_mix64(idx.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))) if len(idx) else 0
        assert hx[j] == np.uint64(hh)


# ------------------------------------------------------------ support radius
def test_aux_grid_and_dn(h, small):
    w, r = small
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        xyz, dn = p.debug_aux()
        p.sync(60000)
    xyz = xyz.cpu().numpy()
    aux = O.fibonacci_points(len(xyz))
    assert np.max(np.abs(xyz - aux)) < 4e-15
    # d_n at the GPU's own auxiliary points, exactly (chords) and to rounding (geodesic)
    exp = O.geodesic_from_chord2(O.NodeSet(w.nodes).knn_chord2(xyz, O.Params().n_for(w.K)))
    assert np.max(np.abs(dn.cpu().numpy() / exp - 1)) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_support_radius_and_counts(h, small, prec):
    w, r = small
    with h.Plan(dev(w.nodes), w.N, w.K, precision=prec) as p:
        p.fit(dev(w.values))
        g = p.debug_grid()
        p.sync(60000)
        st = p.stats()
    delta = g["delta"].cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.max(np.abs(delta / r.support.delta.astype(float) - 1)) < tol
    if prec == "fp64":
        assert np.array_equal(g["count"].cpu().numpy(), r.support.count)
    assert st["sum_n"] == int(g["count"].cpu().numpy().sum())
    assert st["min_n"] >= O.dim_tan(w.K)


# ---------------------------------------------------------------- step 3
@pytest.mark.parametrize("N", [1, 2, 7, 16, 36, 64])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quadrature_matches_oracle(h, N, prec):
    rng = SplitMix64(100 + N)
    g = O.quad_grid(N)
    f = rng.normal(g.MQ)
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1, precision=prec) as p:
        c = p.debug_quadrature(dev(f))
        p.sync(60000)
    got = h.to_complex(c)
    exp = O.quadrature(f, g)
    assert relerr(got, exp) < (1e-13 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("N", [16, 128, 256, 512])
def test_quadrature_exact_on_bandlimited(h, N):
    # Alg. 1 step 3 reproduces f in Pi_N (quadrature exact on Pi_2N)
    c = random_field_coeffs(7 + N, N)
    g_t, _ = O.gauss_legendre(N + 1)
    L = 2 * N + 2
    t = g_t.astype(float)
    phi = 2 * np.pi * np.arange(L) / L
    st = np.sqrt((1 - t) * (1 + t))
    xyz = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                    np.repeat(t, L)], axis=1)
    f = synth_field(c, torch.tensor(xyz, device="cuda"), torch).contiguous()
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1) as p:
        got = h.to_complex(p.debug_quadrature(f))
        p.sync(120000)
    exp = O.pack_coeffs(np.tril(c), N)
    assert relerr(got, exp) < 1e-12


# ------------------------------------------------------------- end to end
def test_fit_fp64_small(h, small):
    w, r = small
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        c = p.fit(dev(w.values))
        g = p.debug_grid()
        p.sync(60000)
        st = p.stats()
    f = g["f"].cpu().numpy()
    fo = r.fgrid.astype(float)
    assert np.max(np.abs(f - fo)) < 1e-10 * np.max(np.abs(fo))
    assert np.allclose(g["chi"].cpu().numpy(), r.chi.astype(float), rtol=1e-8)
    assert np.allclose(g["tau"].cpu().numpy(), r.tau_tilde.astype(float), rtol=1e-8, atol=1e-14)
    assert relerr(h.to_complex(c), r.coeffs) < FP64_TOL
    assert st["n_regularized"] == int((r.tau_tilde > 0).sum())


def test_fit_mixed_small(h, small):
    w, r = small
    with h.Plan(dev(w.nodes), w.N, w.K, precision="mixed") as p:
        c = p.fit(dev(w.values))
        p.sync(60000)
    assert relerr(h.to_complex(c), r.coeffs) < MIXED_TOL


def test_host_buffers_equal_device_buffers(h, small):
    w, r = small
    with h.Plan(w.nodes, w.N, w.K) as p:                       # host numpy nodes
        out = torch.empty((O.n_coeffs(w.N), 2), dtype=torch.float64).pin_memory()
        p.fit(w.values, out=out)                                # host values, pinned host output
        p.sync(60000)
        a = h.to_complex(out)
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        b = h.to_complex(p.fit(dev(w.values)))
        p.sync(60000)
    assert np.array_equal(a, b)


def test_replan_smaller_node_set(h, small):
    w, r = small
    x2 = w.nodes[:3000].copy()
    y2 = w.values[:3000].copy()
    exp = O.hamls(x2, y2, w.N, w.K, O.Params()).coeffs
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        p.replan(dev(x2))
        c = p.fit(dev(y2))
        p.sync(60000)
        assert relerr(h.to_complex(c), exp) < FP64_TOL
        with pytest.raises(h.HamlsError):
            p.replan(dev(np.concatenate([w.nodes, w.nodes])))


@pytest.mark.parametrize("K", [1, 3, 4])
def test_fit_other_degrees(h, K):
    x, _ = __import__("hamls_synth").track_hole_nodes(40 + K, 8000, n_tracks=8, hole_deg=(25.0,))
    c = random_field_coeffs(41, 10)
    y = synth_field(c, x)
    N = 12
    exp = O.hamls(x, y, N, K, O.Params()).coeffs
    with h.Plan(dev(x), N, K) as p:
        got = h.to_complex(p.fit(dev(y)))
        p.sync(60000)
    assert relerr(got, exp) < FP64_TOL


def test_few_nodes(h):
    # M = 4n nodes: supports span a large part of the sphere but stay below pi/2
    K = 1
    n = 4 * O.dim_tan(K)
    x = O.fibonacci_points(4 * n)
    y = x[:, 0] + 0.5 * x[:, 2]
    N = 3
    exp = O.hamls(x, y, N, K, O.Params()).coeffs
    with h.Plan(dev(x), N, K) as p:
        got = h.to_complex(p.fit(dev(y)))
        p.sync(60000)
    assert relerr(got, exp) < FP64_TOL


def test_guard_path_matches_oracle(h):
    # a coarse auxiliary grid with a wide Shepard radius triggers the guard
    x = remove_caps(uniform_sphere(SplitMix64(22), 4000), np.array([[0.0, 0.6, 0.8]]), np.array([0.45]))
    y = x[:, 1] ** 2 + x[:, 2]
    prm = dict(aux_points=200, aux_radius=6.0)
    r = O.hamls(x, y, 8, 2, O.Params(**prm))
    assert r.support.guarded.any()
    with h.Plan(dev(x), 8, 2, **prm) as p:
        got = h.to_complex(p.fit(dev(y)))
        p.sync(60000)
        st = p.stats()
    assert st["n_guarded"] == int(r.support.guarded.sum())
    assert relerr(got, r.coeffs) < FP64_TOL


def test_device_errors_reported(h):
    x = uniform_sphere(SplitMix64(3), 2000)
    bad = x.copy()
    bad[10] *= 1.5                               # not on the unit sphere
    p = h.Plan(dev(bad), 8, 2)
    with pytest.raises(h.HamlsError) as e:
        p.sync(60000)
    assert e.value.code == 1
    p.close()
    with h.Plan(dev(x), 8, 2) as p:
        y = np.ones(2000)
        y[5] = np.nan
        p.fit(dev(y))
        with pytest.raises(h.HamlsError) as e:
            p.sync(60000)
        assert e.value.code == 7
        p.fit(dev(np.ones(2000)))                # the plan stays usable
        p.sync(60000)


def test_support_too_large_reported(h):
    # 40 nodes clustered at one pole, K=2 needs n=24: supports elsewhere exceed pi/2
    x = O.fibonacci_points(4000)
    x = x[x[:, 2] > 0.97][:60]
    with pytest.raises(h.HamlsError) as e:
        p = h.Plan(dev(x), 4, 2)
        p.sync(60000)
    assert e.value.code == 5
