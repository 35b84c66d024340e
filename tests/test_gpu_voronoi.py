"""Spherical Voronoi areas through the C ABI against the CPU oracle (GPU only).

The cells V_i = {p : p.x_i >= p.x_j for all j} give the weights that rescale
the local MLS weights (Sec. 2.2, the remark after Theorem 2.1). Bars: FP64
plans within 1e-10 relative per cell; mixed plans (FP32 geometry on FP64
differences, about 1e-7 relative per vertex) within 1e-4 per cell and 1e-6 on
the total 4 pi."""
import itertools
import math

import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

import oracle as O
from hamls_synth import SplitMix64, uniform_sphere, workload

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


def gpu_areas(h, x, mixed=False, tiny=False):
    kw = dict(precision="mixed" if mixed else "fp64")
    if tiny:
        kw["n_target"] = 3
    with h.Plan(dev(x), 8, 1 if tiny else 2, **kw) as p:
        try:
            p.sync(60000)        # a tiny node set may leave support flags from the plan itself
        except h.HamlsError:
            pass
        a = p.voronoi_areas()
        p.sync(120000)
        return a.cpu().numpy()


def unit(a):
    a = np.asarray(a, dtype=np.float64)
    return a / np.linalg.norm(a, axis=1)[:, None]


def rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


PHI = (1 + 5 ** 0.5) / 2
SIGNS = lambda v: [list(s) for s in itertools.product(*[(-a, a) if a else (0.0,) for a in v])]
CYC = lambda rows: [r2 for r in rows for r2 in (r, [r[1], r[2], r[0]], [r[2], r[0], r[1]])]
SOLIDS = {
    "tetrahedron": [[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]],
    "octahedron": [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
    "cube": SIGNS([1, 1, 1]),
    "icosahedron": CYC(SIGNS([0, 1, PHI])),
    "dodecahedron": SIGNS([1, 1, 1]) + CYC(SIGNS([0, 1 / PHI, PHI])),
}


@pytest.mark.parametrize("mixed", [False, True])
def test_platonic_solids(h, mixed):
    for name, v in SOLIDS.items():
        x = unit(v) @ rotation(len(v)).T
        a = gpu_areas(h, x, mixed=mixed, tiny=True)
        np.testing.assert_allclose(a, 4 * np.pi / len(x), rtol=MIXED_TOL if mixed else 1e-12, err_msg=name)


def test_regular_polygon_around_a_pole(h):
    # the pole's cell among k nodes at colatitude alpha is the regular k-gon
    # with apothem alpha/2 (Napier's rule for its 2k right triangles)
    k, alpha = 7, 0.3
    ring = [[math.sin(alpha) * math.cos(2 * math.pi * j / k), math.sin(alpha) * math.sin(2 * math.pi * j / k),
             math.cos(alpha)] for j in range(k)]
    rest = uniform_sphere(SplitMix64(k), 4000)
    rest = rest[rest[:, 2] < math.cos(1.0)][:300]
    x = np.vstack([[[0.0, 0.0, 1.0]], ring, rest]) @ rotation(1).T
    B = math.acos(math.cos(alpha / 2) * math.sin(math.pi / k))
    exact = 2 * math.pi + 2 * k * B - k * math.pi          # 1e-14 relative in double here
    assert abs(gpu_areas(h, x)[0] / exact - 1) < 1e-11


@pytest.mark.parametrize("name", ["s2_n16_k2_m5k", "s2_n128_k3_m200k"])
def test_matches_oracle_on_the_workloads(h, name):
    w = workload(name, xp=torch, device="cuda")
    ref = O.voronoi_areas(w.nodes)
    a64 = gpu_areas(h, w.nodes)
    amx = gpu_areas(h, w.nodes, mixed=True)
    assert np.max(np.abs(a64 / ref - 1)) < FP64_TOL
    assert np.max(np.abs(amx / ref - 1)) < MIXED_TOL
    assert abs(a64.sum() / (4 * np.pi) - 1) < 1e-12
    assert abs(amx.sum() / (4 * np.pi) - 1) < 1e-6


def test_duplicates_share_their_cell(h):
    x = uniform_sphere(SplitMix64(5), 2000)
    y = np.vstack([x, x[[7, 7]], x[[30]]])
    ref = O.voronoi_areas(y)
    a = gpu_areas(h, y)
    np.testing.assert_allclose(a, ref, rtol=FP64_TOL)
    assert a[7] == a[2000] == a[2001]


def test_host_output_buffer(h):
    w = workload("s2_n16_k2_m5k")
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        host = torch.empty(w.M, dtype=torch.float64).pin_memory()
        p.voronoi_areas(out=host)
        d = p.voronoi_areas()
        p.sync(60000)
        np.testing.assert_array_equal(host.numpy(), d.cpu().numpy())


def test_nodes_in_a_small_cap_are_rejected(h):
    # cells of nodes confined to a cap of 0.5 rad reach far beyond 1.5 rad
    x = uniform_sphere(SplitMix64(8), 3000)
    x = x[x[:, 2] > math.cos(0.5)]
    with h.Plan(dev(x), 8, 1, n_target=3) as p:
        try:
            p.sync(60000)
        except h.HamlsError:
            pass
        a = p.voronoi_areas()
        with pytest.raises(h.HamlsError) as e:
            p.sync(60000)
        assert e.value.code == 9
        assert torch.isnan(a).any()


def test_fit_with_voronoi_weights(h):
    # the fit of Sec. 3: MLS weights rescaled by the Voronoi areas
    w = workload("s2_n16_k2_m5k")
    v = O.voronoi_areas(w.nodes)
    exp = O.hamls(w.nodes, w.values, w.N, w.K, O.Params(), v=v).coeffs
    with h.Plan(dev(w.nodes), w.N, w.K) as p:
        p.voronoi_weights()
        got = h.to_complex(p.fit(dev(w.values)))
        p.sync(60000)
    rel = np.linalg.norm(got - exp) / np.linalg.norm(exp)
    assert rel < FP64_TOL
    with h.Plan(dev(w.nodes), w.N, w.K, precision="mixed") as p:
        p.voronoi_weights()
        gm = h.to_complex(p.fit(dev(w.values)))
        p.sync(60000)
    assert np.linalg.norm(gm - exp) / np.linalg.norm(exp) < 1e-4


def test_full_size_workload(h):
    # N = 512, M = 4,000,000: the total and sampled cells against the oracle
    # computed one cell at a time
    w = workload("s2_n512_k3_m4m", xp=torch, device="cuda")
    x = w.nodes
    tree = cKDTree(x)
    rng = np.random.default_rng(11)
    idx = rng.choice(len(x), 40, replace=False)
    ref = np.array([O.voronoi_area_at(x, int(i), tree) for i in idx])
    for mixed in (False, True):
        with h.Plan(dev(x), w.N, w.K, precision="mixed" if mixed else "fp64") as p:
            a = p.voronoi_areas()
            p.sync(120000)
            a = a.cpu().numpy()
        tol = MIXED_TOL if mixed else FP64_TOL
        assert np.all(np.isfinite(a)) and np.all(a > 0)
        assert abs(a.sum() / (4 * np.pi) - 1) < (1e-6 if mixed else 1e-11)
        assert np.max(np.abs(a[idx] / ref - 1)) < tol
