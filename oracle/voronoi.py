"""Spherical Voronoi cell areas: a plain CPU oracle (test infrastructure).

The paper rescales each node's local MLS weight by the area of its Voronoi
cell (Sec. 2.2, the remark after Theorem 2.1 on ill-distributed nodes), and
every experiment of Sec. 3 uses these areas. The cell of node x_i is the set
of points of S^2 that are at least as close, in angle, to x_i as to any
other node:

    V_i = { p in S^2 : p . x_i >= p . x_j for every node x_j }.

This oracle reaches the cells through their dual. For points on the sphere
the facets of the convex hull are the spherical Delaunay triangles, and the
unit outer normal of a facet is the point of S^2 equidistant from its three
nodes, the common vertex of their three cells (Brown, "Voronoi diagrams from
convex hulls", 1979). The hull is taken from scipy (Qhull), a library
primitive; everything after it is written out here:

  1. the circumcentre of every facet, from the cross product of two of its
     edges in extended precision, oriented away from the origin;
  2. for every node, the circumcentres of its incident facets sorted by
     their angle around the node in a tangent frame: the vertices of V_i
     in order;
  3. the area of V_i as the sum of the solid angles of the fan triangles
     (x_i, c_k, c_k+1), each by the formula of van Oosterom and Strackee
     (IEEE Trans. Biomed. Eng. 30, 1983):
        tan(E/2) = det[a, b, c] / (1 + a.b + b.c + c.a)   (unit vectors).

Exact duplicates share their common cell equally. The construction needs the
origin strictly inside the hull (no closed hemisphere holds all nodes);
otherwise a ValueError is raised.

Test infrastructure only: tests, the smoke check and the benchmark's CPU
baseline leg may use this module; the CUDA library never does. Pins
(tests/test_oracle_voronoi.py): the five Platonic solids in random rotations
(equal cells of 4 pi / M), the total 4 pi, a brute-force vertex enumeration
with L'Huilier's triangle formula on tiny inputs, scipy's SphericalVoronoi
areas, and the duplicate rule.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import ConvexHull, cKDTree

LD = np.longdouble


def _cross(a, b):
    return np.stack([a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1],
                     a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2],
                     a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]], axis=1)


def _dot(a, b):
    return (a * b).sum(axis=1)


def _frame(x):
    """An orthonormal tangent frame (e1, e2) at every row of x (extended)."""
    t = np.zeros_like(x)
    use_z = np.abs(x[:, 2]) < LD("0.9")
    t[use_z, 2] = 1
    t[~use_z, 0] = 1
    e1 = _cross(t, x)
    e1 /= np.sqrt(_dot(e1, e1))[:, None]
    e2 = _cross(x, e1)
    return e1, e2


def _unique_cells(u: np.ndarray, with_radius: bool = False):
    """Areas of the Voronoi cells of distinct unit vectors u (K x 3); with
    with_radius also the largest chord from each node to its cell's vertices."""
    K = len(u)
    if K < 4:
        raise ValueError("need at least 4 distinct nodes")
    hull = ConvexHull(u)
    if not np.all(hull.equations[:, 3] < 0):
        raise ValueError("the origin is not strictly inside the hull: the nodes lie in a closed hemisphere")
    tri = hull.simplices
    P = u.astype(LD)
    a, b, c = P[tri[:, 0]], P[tri[:, 1]], P[tri[:, 2]]
    n = _cross(b - a, c - a)
    n /= np.sqrt(_dot(n, n))[:, None]
    n *= np.sign(_dot(n, a))[:, None]                 # away from the origin
    # incidences (node, facet), sorted by node, then by angle around the node
    node = tri.reshape(-1)
    fac = np.repeat(np.arange(len(tri)), 3)
    x = P[node]
    e1, e2 = _frame(P)
    cv = n[fac]
    ang = np.arctan2(_dot(cv, e2[node]).astype(np.float64), _dot(cv, e1[node]).astype(np.float64))
    o = np.lexsort((ang, node))
    node, fac, x = node[o], fac[o], x[o]
    cv = n[fac]
    # the next vertex of the same cell, cyclically
    first = np.r_[0, np.flatnonzero(np.diff(node)) + 1]
    cnt = np.diff(np.r_[first, len(node)])
    nxt = np.arange(len(node)) + 1
    nxt[first + cnt - 1] = first
    cn = cv[nxt]
    # solid angle of (x, c_k, c_k+1); det via differences to the node
    det = _dot(x, _cross(cv - x, cn - x))
    den = 1 + _dot(x, cv) + _dot(cv, cn) + _dot(cn, x)
    E = 2 * np.arctan2(det, den)
    area = np.zeros(K, dtype=LD)
    np.add.at(area, node, E)
    if not with_radius:
        return area
    rad = np.zeros(K, dtype=LD)
    np.maximum.at(rad, node, np.sqrt(_dot(cv - x, cv - x)))
    return area, rad


def voronoi_areas(x: np.ndarray) -> np.ndarray:
    """Area of the spherical Voronoi cell of every node (M x 3 unit vectors),
    in float64; exact duplicates split their cell equally."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    u, inv, mult = np.unique(x, axis=0, return_inverse=True, return_counts=True)
    area = _unique_cells(u)
    return (area[inv.reshape(-1)] / mult[inv.reshape(-1)]).astype(np.float64)


def voronoi_area_at(x: np.ndarray, i: int, tree: cKDTree = None, k0: int = 48) -> float:
    """Area of the Voronoi cell of node i alone, for node sets too large for
    voronoi_areas. A cell depends only on the nodes closer than twice its
    largest vertex chord rho: a node x_j can cut off a vertex c only if
    |x_j - c| < |x_i - c| <= rho, hence |x_j - x_i| < 2 rho. The k nearest
    nodes S (k doubling from k0, all within angle R of x_i) together with
    their antipodes -S form a set whose hull holds the origin. While the cell
    lies within angle psi of x_i and R + 2 psi < pi, every antipode is farther
    than x_i from every point of the cell and cuts nothing, so the cell of x_i
    in S u -S is the global one as soon as all nodes within 2 rho are in S.
    Exact duplicates of x_i share the cell."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if tree is None:
        tree = cKDTree(x)
    M = len(x)
    k = min(k0, M)
    while k < M:
        d, idx = tree.query(x[i], k=k)
        sel = x[idx]
        mult = int(np.sum(np.all(sel == x[i], axis=1)))
        S = np.unique(sel, axis=0)
        U = np.unique(np.vstack([S, -S]), axis=0)
        area, rad = _unique_cells(U, with_radius=True)
        j = int(np.flatnonzero(np.all(U == x[i], axis=1))[0])
        R = 2 * np.arcsin(min(d[-1] / 2, 1.0))
        psi = 2 * np.arcsin(min(float(rad[j]) / 2, 1.0))
        if 2 * rad[j] * (1 + 1e-12) < d[-1] and R + 2 * psi < np.pi:
            return float(area[j] / mult)
        k = min(2 * k, M)
    return float(voronoi_areas(x)[i])
