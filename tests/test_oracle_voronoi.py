"""Pins of the spherical Voronoi-area oracle (CPU).

The cells V_i = {p : p.x_i >= p.x_j for all j} (the areas that rescale the
MLS weights, Sec. 2.2 after Theorem 2.1; used throughout Sec. 3) are checked
against closed forms, a brute-force construction with a different area
formula, an independent library routine and the invariants of a partition
of S^2."""
import itertools
import math

import mpmath
import numpy as np
import pytest
from scipy.spatial import SphericalVoronoi, cKDTree

import oracle as O
from hamls_synth import workload, uniform_sphere, SplitMix64

PHI = (1 + 5 ** 0.5) / 2


def unit(a):
    a = np.asarray(a, dtype=np.float64)
    return a / np.linalg.norm(a, axis=1)[:, None]


def rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def cyclic(rows):
    out = []
    for r in rows:
        out += [r, [r[1], r[2], r[0]], [r[2], r[0], r[1]]]
    return out


def signs(v):
    return [list(s) for s in itertools.product(*[(-a, a) if a else (0.0,) for a in v])]


SOLIDS = {
    "tetrahedron": [[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]],
    "octahedron": [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
    "cube": signs([1, 1, 1]),
    "icosahedron": cyclic(signs([0, 1, PHI])),
    "dodecahedron": signs([1, 1, 1]) + cyclic(signs([0, 1 / PHI, PHI])),
}


@pytest.mark.parametrize("name", sorted(SOLIDS))
def test_platonic_solids_have_equal_cells(name):
    # vertex-transitive sets: every cell is 4 pi / M, in any orientation
    x = unit(SOLIDS[name])
    for seed in range(3):
        a = O.voronoi_areas(x @ rotation(seed).T)
        np.testing.assert_allclose(a, 4 * np.pi / len(x), rtol=1e-13, atol=0)


def regular_polygon_area(k, apothem):
    # a regular spherical k-gon is 2k right triangles with angle pi/k at the
    # centre and the apothem as adjacent leg; Napier's rule gives the angle at
    # the vertex, cos B = cos(apothem) sin(pi/k), and the excess sums to this
    # (in 40 digits: the three terms nearly cancel for small polygons)
    with mpmath.workdps(40):
        a = mpmath.mpf(apothem)
        B = mpmath.acos(mpmath.cos(a) * mpmath.sin(mpmath.pi / k))
        return float(2 * mpmath.pi + 2 * k * B - k * mpmath.pi)


@pytest.mark.parametrize("k,alpha", [(5, 0.4), (7, 0.3), (12, 0.1)])
def test_pole_with_a_ring_is_a_regular_polygon(k, alpha):
    # the north pole with k nodes equally spaced at colatitude alpha: its cell
    # is the regular k-gon with apothem alpha / 2; the other nodes lie beyond
    # colatitude 1 rad and cannot reach it
    ring = [[math.sin(alpha) * math.cos(2 * math.pi * j / k), math.sin(alpha) * math.sin(2 * math.pi * j / k),
             math.cos(alpha)] for j in range(k)]
    rest = uniform_sphere(SplitMix64(k), 4000)
    rest = rest[rest[:, 2] < math.cos(1.0)][:300]
    x = np.vstack([[[0.0, 0.0, 1.0]], ring, rest])
    R = rotation(k)
    a = O.voronoi_areas(x @ R.T)
    assert abs(a[0] / regular_polygon_area(k, alpha / 2) - 1) < 1e-13


def lhuilier(a, b, c):
    # spherical excess from the three sides (L'Huilier's theorem)
    ang = lambda p, q: 2 * math.asin(min(1.0, np.linalg.norm(p - q) / 2))
    sa, sb, sc = ang(b, c), ang(a, c), ang(a, b)
    s = (sa + sb + sc) / 2
    t = math.tan(s / 2) * math.tan((s - sa) / 2) * math.tan((s - sb) / 2) * math.tan((s - sc) / 2)
    return 4 * math.atan(math.sqrt(max(t, 0.0)))


def brute_force_areas(x):
    # every cell vertex is the point equidistant from x_i and two others that
    # is no farther from x_i than from any node: enumerate all pairs, keep the
    # valid ones, order them around x_i and sum the fan by L'Huilier
    M = len(x)
    out = np.zeros(M)
    for i in range(M):
        verts = []
        for j, k in itertools.combinations([t for t in range(M) if t != i], 2):
            n = np.cross(x[i] - x[j], x[i] - x[k])
            if np.linalg.norm(n) < 1e-12:
                continue
            n /= np.linalg.norm(n)
            for v in (n, -n):
                if v @ x[i] >= np.max(x @ v) - 1e-12:
                    verts.append(v)
        verts = np.array(verts)
        e1 = np.cross([0.0, 0.0, 1.0], x[i])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(x[i], e1)
        verts = verts[np.argsort(np.arctan2(verts @ e2, verts @ e1))]
        out[i] = sum(lhuilier(x[i], verts[t], verts[(t + 1) % len(verts)]) for t in range(len(verts)))
    return out


def test_brute_force_on_tiny_inputs():
    for seed in (3, 4):
        x = uniform_sphere(SplitMix64(seed), 14)
        np.testing.assert_allclose(O.voronoi_areas(x), brute_force_areas(x), rtol=1e-10)


def test_matches_scipy_spherical_voronoi():
    w = workload("s2_n16_k2_m5k")
    ref = SphericalVoronoi(w.nodes).calculate_areas()
    np.testing.assert_allclose(O.voronoi_areas(w.nodes), ref, rtol=1e-9)


def test_cells_partition_the_sphere():
    for x in (uniform_sphere(SplitMix64(9), 20000), workload("s2_n16_k2_m5k").nodes):
        a = O.voronoi_areas(x)
        assert np.all(a > 0)
        assert abs(a.sum() / (4 * np.pi) - 1) < 1e-13


def test_duplicates_share_their_cell():
    x = uniform_sphere(SplitMix64(5), 500)
    base = O.voronoi_areas(x)
    y = np.vstack([x, x[[7, 7]], x[[30]]])
    a = O.voronoi_areas(y)
    np.testing.assert_array_equal(a[[7, 500, 501]], base[7] / 3)
    np.testing.assert_array_equal(a[[30, 502]], base[30] / 2)
    others = np.setdiff1d(np.arange(500), [7, 30])
    np.testing.assert_allclose(a[others], base[others], rtol=1e-14)


def test_nodes_in_a_hemisphere_are_rejected():
    x = uniform_sphere(SplitMix64(6), 200)
    x[:, 2] = np.abs(x[:, 2]) + 0.01
    with pytest.raises(ValueError):
        O.voronoi_areas(unit(x))


def test_single_cell_equals_the_whole_diagram():
    w = workload("s2_n16_k2_m5k")
    a = O.voronoi_areas(w.nodes)
    tree = cKDTree(w.nodes)
    idx = np.r_[np.arange(0, w.M, 251), np.argsort(a)[-5:]]      # includes the cells at the hole's rim
    got = np.array([O.voronoi_area_at(w.nodes, i, tree) for i in idx])
    np.testing.assert_allclose(got, a[idx], rtol=1e-13)
