"""HAMLS on S^2: a plain CPU oracle (test infrastructure).

This module restates Algorithm 1 of the paper ("Harmonic Approximation via
Moving Least Squares") for the sphere, step by step, in numpy/scipy. It is slow
on purpose and written to be read against the paper:

* Step 1, the quadrature grid (Sec. 2.1): Gauss-Legendre nodes in cos(theta)
  times an equispaced trapezoidal rule in longitude, exact on Pi_{2N}.
* Step 2, MLS evaluation at every grid node (Sec. 2.2, 2.3): adaptive support
  radius delta = (1 + eps) * d_n smoothed by a degree-zero MLS over a Fibonacci
  auxiliary grid (eq. adaptive_support_radius and the paragraph after it),
  weighted local least squares in the tangent-plane ansatz space, centre
  amplification chi (eq. chi via coupling), degree-adapted regularisation with
  bisection for tau (eq. regularized MLS problem, eq. regularized MLS
  amplification) and the smoothed strength tau~.
* Step 3, the adjoint transform (Alg. 1 step 3, eq.
  quadrature_based_approximation): a direct DFT over every ring, then the
  associated-Legendre quadrature.

Local problems are solved in numpy ``longdouble`` (x86 80-bit extended) so
that the oracle's own rounding sits far below the CUDA library's FP64 error.
Neighbour selection and the k-nearest-neighbour radius are computed in plain
IEEE float64 with a fixed operation order, so that they are bit-comparable
with any other implementation that uses the same formula.

Test infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the CUDA library never does. Every function
here is pinned by a test in ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force; none is "parity unpinned".

Readings of points the paper leaves open (all shared with the CUDA library):
  n = 4 m (Sec. 3.2 uses n = 4 dim Pi_K^tan), eps = 0.05, chi_T = 16,
  chi_full = 32, s = 1, Wendland phi_{3,2}, Fibonacci auxiliary grid with
  2 M_Q points and Shepard radius 3 sqrt(4 pi / M_aux), the C^3 smoothstep
  tau~ = S(t) tau with t = (chi - chi_T)/(chi_full - chi_T), bisection on
  [0, r0 / (mu_min r*)], a pivot floor that drops numerically dependent
  basis directions, and a guard that falls back to delta = (1 + eps) d_n(q)
  computed exactly at q when fewer than m nodes fall in the smoothed support.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
from scipy.spatial import cKDTree

LD = np.longdouble
PI_LD = LD("3.14159265358979323846264338327950288")


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Method parameters (Sec. 2.2 adaptive radius, Sec. 2.3 regularisation)."""
    n_target: int = 0          # target neighbour count n; 0 -> 4 m
    eps: float = 0.05          # delta = (1 + eps) d_n
    chi_target: float = 16.0   # chi_T
    chi_full: float = 32.0     # chi_full > chi_T
    sobolev_s: float = 1.0     # mu = (l (l + 1))^s
    aux_points: int = 0        # Fibonacci auxiliary grid size; 0 -> 2 M_Q
    aux_radius: float = 3.0    # Shepard radius / sqrt(4 pi / M_aux)
    pivot_floor: float = 1e-12  # Cholesky pivot (squared) below which a direction is dropped
    bisect_iters: int = 200
    weight_fn: int = 0         # phi of eq. weight_function_radial: 0 Wendland phi_{3,2}, 1 phi_{3,1}

    def n_for(self, K: int) -> int:
        return self.n_target if self.n_target > 0 else 4 * dim_tan(K)


def dim_tan(K: int) -> int:
    """m = dim Pi_K^tan(S^2; x): bivariate polynomials of degree <= K."""
    return (K + 1) * (K + 2) // 2


def monomial_exponents(K: int):
    """Basis order of Sec. 2.3: ascending degree; inside one degree k the
    monomials u^a v^(k-a) with a descending. Returns [(a, b, degree)]."""
    out = []
    for k in range(K + 1):
        for a in range(k, -1, -1):
            out.append((a, k - a, k))
    return out


# --------------------------------------------------------------------------
# step 1: quadrature grid (Sec. 2.1, S^2 bullet)
# --------------------------------------------------------------------------
def gauss_legendre(npts: int):
    """Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on
    P_npts with the three-term recurrence (Golub-Welsch is not used). Nodes
    are returned in descending order (north pole first). Extended precision."""
    n = npts
    k = np.arange(n, dtype=LD)
    t = np.cos(PI_LD * (k + LD(0.75)) / (LD(n) + LD(0.5)))   # initial guesses, descending
    for _ in range(100):
        p0 = np.ones_like(t)
        p1 = t.copy()
        for j in range(2, n + 1):
            p0, p1 = p1, ((2 * j - 1) * t * p1 - (j - 1) * p0) / LD(j)
        if n == 1:
            p0 = np.ones_like(t)
        dp = n * (t * p1 - p0) / (t * t - 1)
        dt = p1 / dp
        t = t - dt
        if np.max(np.abs(dt)) < LD(1e-19):
            break
    p0 = np.ones_like(t)
    p1 = t.copy()
    for j in range(2, n + 1):
        p0, p1 = p1, ((2 * j - 1) * t * p1 - (j - 1) * p0) / LD(j)
    if n == 1:
        p0 = np.ones_like(t)
    dp = n * (t * p1 - p0) / (t * t - 1)
    w = 2 / ((1 - t * t) * dp * dp)
    return t, w


@dataclass
class Grid:
    N: int
    t: np.ndarray        # cos(theta_k), k = 0..N, descending (longdouble)
    w: np.ndarray        # Gauss-Legendre weights (longdouble)
    phi: np.ndarray      # 2 pi j / (2N + 2), j = 0..2N+1 (longdouble)
    xyz: np.ndarray      # M_Q x 3 float64, ring-major: index k (2N+2) + j
    xyz_ld: np.ndarray   # same, longdouble

    @property
    def MQ(self) -> int:
        return (self.N + 1) * (2 * self.N + 2)


def quad_grid(N: int) -> Grid:
    """Product grid: Gauss-Legendre in t = cos(theta) with N+1 nodes, trapezoid
    in phi with 2N+2 nodes, M_Q = (2N+2)(N+1), exact on Pi_{2N} (Sec. 2.1)."""
    t, w = gauss_legendre(N + 1)
    L = 2 * N + 2
    phi = 2 * PI_LD * np.arange(L, dtype=LD) / LD(L)
    st = np.sqrt(1 - t * t)
    X = st[:, None] * np.cos(phi)[None, :]
    Y = st[:, None] * np.sin(phi)[None, :]
    Z = np.broadcast_to(t[:, None], X.shape)
    xyz_ld = np.stack([X.ravel(), Y.ravel(), np.ascontiguousarray(Z).ravel()], axis=1)
    return Grid(N, t, w, phi, xyz_ld.astype(np.float64), xyz_ld)


GOLDEN_FRAC_Q64 = 0x61C8864680B583EA   # floor(2^64 (3 - sqrt 5)/2), i.e. 1 - 1/Phi in 0.64 fixed point


def fibonacci_points(M_aux: int) -> np.ndarray:
    """Fibonacci (golden-angle spiral) grid, approximately uniform on S^2
    (Sec. 2.2 names it for the auxiliary grid): z_i = 1 - (2i+1)/M_aux,
    phi_i = 2 pi {i (1 - 1/Phi)}. The fractional part is taken in 64-bit
    fixed point and truncated to 53 bits, so that it is exact for any i."""
    i = np.arange(M_aux, dtype=np.uint64)
    with np.errstate(over="ignore"):
        fr = (i * np.uint64(GOLDEN_FRAC_Q64)) >> np.uint64(11)
    frac = fr.astype(LD) / LD(2.0 ** 53)
    z = 1 - (2 * i.astype(LD) + 1) / LD(M_aux)
    ph = 2 * PI_LD * frac
    s = np.sqrt(1 - z * z)
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1).astype(np.float64)


# --------------------------------------------------------------------------
# distances and weights (Sec. 2.2, eq. weight_function_radial)
# --------------------------------------------------------------------------
def chord2(q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Squared chord |x - q|^2 in float64 with the fixed order
    ((dx*dx + dy*dy) + dz*dz) and no fused multiply-add."""
    dx = x[..., 0] - q[..., 0]
    dy = x[..., 1] - q[..., 1]
    dz = x[..., 2] - q[..., 2]
    return (dx * dx + dy * dy) + dz * dz


def geodesic_from_chord2(c2):
    """Geodesic distance 2 asin(|x - q| / 2) (well conditioned for small d)."""
    c2 = np.asarray(c2)
    if c2.dtype == LD:
        return 2 * np.arcsin(np.sqrt(c2) / 2)
    return 2.0 * np.arcsin(np.sqrt(c2) / 2.0)


def chord_radius2(delta):
    """Squared chord of the geodesic radius delta: (2 sin(delta/2))^2."""
    s = 2.0 * np.sin(np.asarray(delta, dtype=np.float64) / 2.0)
    return s * s


def wendland(r):
    """Wendland function phi_{3,2}(r) = (1-r)^6 (35 r^2 + 18 r + 3) on [0,1),
    0 beyond: continuous, nonincreasing, supp = [0, 1], C^4 (Sec. 2.2 asks for
    a Wendland function; Sec. 2.3 for a weight at least C^3)."""
    r = np.asarray(r)
    one = r.dtype.type(1)
    om = np.where(r < one, one - r, r.dtype.type(0))
    return om ** 6 * (35 * r * r + 18 * r + 3)


def wendland31(r):
    """Wendland function phi_{3,1}(r) = (1-r)^4 (4 r + 1) on [0,1), 0 beyond:
    continuous, nonincreasing, supp = [0, 1], C^2 as a radial function (the
    other Wendland choice that Sec. 2.2 leaves open; below the C^3 that
    Sec. 2.3 names for a C^3 smoothed tau)."""
    r = np.asarray(r)
    one = r.dtype.type(1)
    om = np.where(r < one, one - r, r.dtype.type(0))
    return om ** 4 * (4 * r + 1)


def weight_phi(r, fn: int = 0):
    """phi of eq. weight_function_radial: 0 -> phi_{3,2}, 1 -> phi_{3,1}."""
    if fn == 0:
        return wendland(r)
    if fn == 1:
        return wendland31(r)
    raise ValueError(f"weight_fn {fn}: 0 (phi_3,2) or 1 (phi_3,1)")


# --------------------------------------------------------------------------
# k nearest neighbours and the adaptive support radius (eq. adaptive_support_radius)
# --------------------------------------------------------------------------
class NodeSet:
    """Scattered nodes with a k-d tree (scipy) used only to find candidates;
    every distance that decides anything is recomputed with ``chord2``."""

    def __init__(self, x: np.ndarray):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.tree = cKDTree(self.x)

    def knn_chord2(self, q: np.ndarray, n: int, slack: int = 6) -> np.ndarray:
        """Exact n-th smallest squared chord from each query to the nodes."""
        k = min(n + slack, len(self.x))
        _, idx = self.tree.query(q, k=k)
        idx = np.asarray(idx).reshape(len(q), k)
        c2 = chord2(q[:, None, :], self.x[idx])
        c2.sort(axis=1)
        return c2[:, n - 1]

    def ball(self, q: np.ndarray, rho2: float) -> np.ndarray:
        """Indices i with chord2(q, x_i) < rho2 (open geodesic ball)."""
        r = math.sqrt(rho2) * (1.0 + 1e-9) + 1e-300
        cand = np.asarray(self.tree.query_ball_point(q, r), dtype=np.int64)
        if len(cand) == 0:
            return cand
        c2 = chord2(q[None, :], self.x[cand])
        return np.sort(cand[c2 < rho2])


def shepard(q: np.ndarray, aux: np.ndarray, aux_tree: cKDTree, values: np.ndarray, rho: float, weight_fn: int = 0):
    """Degree-zero MLS (Shepard) of values given at aux points, with constant
    geodesic support radius rho and the weight phi of eq.
    weight_function_radial (Sec. 2.2, last paragraph). Extended precision."""
    rho2 = float(chord_radius2(rho))
    out = np.empty(len(q), dtype=LD)
    cands = aux_tree.query_ball_point(q, math.sqrt(rho2) * (1 + 1e-9))
    for j, c in enumerate(cands):
        c = np.asarray(c, dtype=np.int64)
        c2 = chord2(q[j][None, :], aux[c])
        c = c[c2 < rho2]
        d = geodesic_from_chord2(chord2(q[j][None, :].astype(LD), aux[c].astype(LD)))
        wt = weight_phi(d / LD(rho), weight_fn)
        out[j] = np.sum(wt * values[c].astype(LD)) / np.sum(wt)
    return out


@dataclass
class Support:
    delta: np.ndarray          # geodesic support radius per grid node (longdouble)
    rho2: np.ndarray           # float64 squared chord radius per grid node
    count: np.ndarray          # #X(q)
    guarded: np.ndarray        # bool: guard fallback used
    dn_aux: np.ndarray         # d_n at the auxiliary points (longdouble)
    aux: np.ndarray


def support_radius(nodes: NodeSet, q: np.ndarray, K: int, p: Params, subset=None) -> Support:
    """delta(q) = (1 + eps) d~_n(q) (eq. adaptive_support_radius) with d_n
    smoothed over the Fibonacci auxiliary grid; guard: if fewer than m nodes
    fall inside, use (1 + eps) d_n(q) computed exactly at q."""
    m = dim_tan(K)
    n = p.n_for(K)
    MQ = len(q)
    M_aux = p.aux_points if p.aux_points > 0 else 2 * MQ
    aux = fibonacci_points(M_aux)
    h_aux = math.sqrt(4.0 * math.pi / M_aux)
    rho = p.aux_radius * h_aux
    aux_tree = cKDTree(aux)
    sel = np.arange(MQ) if subset is None else np.asarray(subset)
    qs = q[sel]
    # only the auxiliary points that some selected grid node can see
    need = np.unique(np.concatenate(
        [np.asarray(c, dtype=np.int64) for c in aux_tree.query_ball_point(qs, math.sqrt(float(chord_radius2(rho))) * (1 + 1e-6))]
        + [np.zeros(0, dtype=np.int64)]))
    dn_aux = np.full(M_aux, np.nan, dtype=LD)
    if len(need):
        dn_aux[need] = geodesic_from_chord2(nodes.knn_chord2(aux[need], n).astype(LD))
    dtil = shepard(qs, aux, aux_tree, dn_aux, rho, p.weight_fn)
    delta = (1 + LD(p.eps)) * dtil
    rho2 = chord_radius2(delta.astype(np.float64))
    count = np.array([len(nodes.ball(qs[j], rho2[j])) for j in range(len(qs))], dtype=np.int64)
    guarded = count < m
    for j in np.nonzero(guarded)[0]:
        dn = geodesic_from_chord2(LD(nodes.knn_chord2(qs[j][None, :], n)[0]))
        delta[j] = (1 + LD(p.eps)) * dn
        rho2[j] = chord_radius2(float(delta[j]))
        count[j] = len(nodes.ball(qs[j], rho2[j]))
    return Support(delta, rho2, count, guarded, dn_aux, aux)


# --------------------------------------------------------------------------
# the local regularised MLS problem (Sec. 2.3)
# --------------------------------------------------------------------------
def tangent_frame(q_ld: np.ndarray):
    """Orthonormal tangent frame at q: e1 = d/dtheta, e2 = d/dphi (unit)."""
    x, y, z = q_ld
    s = np.sqrt(x * x + y * y)
    cph, sph = x / s, y / s
    e1 = np.array([z * cph, z * sph, -s], dtype=LD)
    e2 = np.array([-sph, cph, LD(0)], dtype=LD)
    return e1, e2


def smoothstep3(t):
    """C^3 smoothstep S(t) = 35 t^4 - 84 t^5 + 70 t^6 - 20 t^7, S(0)=0, S(1)=1."""
    return t ** 4 * (35 - 84 * t + 70 * t * t - 20 * t ** 3)


def cholesky_floor(C: np.ndarray, floor: float):
    """Cholesky C = L L^T (eq. mls local Cholesky factor). A pivot whose
    squared value falls to ``floor`` or below (C has unit diagonal) marks a
    numerically dependent direction: its column of L is set to zero and the
    direction is dropped from the ansatz."""
    n = C.shape[0]
    L = np.zeros_like(C)
    dropped = np.zeros(n, dtype=bool)
    for j in range(n):
        s = C[j, j] - np.dot(L[j, :j], L[j, :j])
        if s <= floor:
            dropped[j] = True
            continue
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (C[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L, dropped


def forward_subst(L: np.ndarray, dropped: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = L^{-1} b with dropped directions set to zero."""
    x = np.zeros_like(b)
    for j in range(len(b)):
        if dropped[j]:
            continue
        x[j] = (b[j] - np.dot(L[j, :j], x[:j])) / L[j, j]
    return x


@dataclass
class LocalResult:
    c1: LD
    chi: LD
    tau: LD
    tau_tilde: LD
    n: int
    n_dropped: int
    d: np.ndarray = field(repr=False, default=None)
    e: np.ndarray = field(repr=False, default=None)
    beta: LD = None
    L: np.ndarray = field(repr=False, default=None)
    B: np.ndarray = field(repr=False, default=None)
    yw: np.ndarray = field(repr=False, default=None)
    mu: np.ndarray = field(repr=False, default=None)
    wn: np.ndarray = field(repr=False, default=None)


def local_design(q_ld, xs, delta, vs, K, frame=None, weight_fn: int = 0):
    """Normalised weights and the scaled design B of eq. (mls local vectors).

    Weights w_i = v_i phi(d_i / delta) (phi by weight_fn), normalised to sum 1; basis g_j =
    monomials of the tangent coordinates (u, v) = (e1 . x_i, e2 . x_i) of the
    orthogonal projection onto T_q S^2, centred at q (g_j(q) = 0 for j >= 2),
    each column scaled to unit discrete norm sum_i w_i g_j(x_i)^2 = 1."""
    xs_ld = xs.astype(LD)
    d = geodesic_from_chord2(chord2(q_ld[None, :], xs_ld))
    w = weight_phi(d / LD(delta), weight_fn) * (np.ones(len(xs), dtype=LD) if vs is None else vs.astype(LD))
    wn = w / np.sum(w)
    e1, e2 = tangent_frame(q_ld) if frame is None else frame
    u = (xs_ld @ e1) / LD(delta)
    v = (xs_ld @ e2) / LD(delta)
    ex = monomial_exponents(K)
    G = np.stack([u ** a * v ** b for (a, b, _) in ex], axis=1)
    scale = np.sqrt(np.sum(wn[:, None] * G * G, axis=0))
    inv = np.where(scale > 0, 1 / np.where(scale > 0, scale, 1), 0)   # a zero column stays zero (dropped)
    B = np.sqrt(wn)[:, None] * G * inv[None, :]
    degrees = np.array([k for (_, _, k) in ex])
    return B, wn, degrees


def solve_local(B: np.ndarray, yw: np.ndarray, degrees: np.ndarray, p: Params,
                tau_override: Optional[float] = None) -> LocalResult:
    """Centre value c_1 of the regularised local problem (eq. regularized MLS
    problem), following Sec. 2.3 in the paper's order:
    H = B^T B split as [[1, b^T], [b, C]]; C = L L^T; d = L^{-1} b;
    r_0 = |d|^2, chi = 1/(1 - r_0) (eq. chi via coupling); if chi > chi_T,
    bisection for tau with chi_tau = chi_T (eq. regularized MLS
    amplification); tau~ smoothed between chi_T and chi_full; then c_1 from
    the regularised normal equations, written in closed form through
    d, e = L^{-1} V^T y_w and beta = v_1^T y_w:
        c_1 = (beta - sum_j d_j e_j/(1 + tau~ mu_j)) / (1 - sum_j d_j^2/(1 + tau~ mu_j)).
    """
    H = B.T @ B
    v1 = B[:, 0]
    V = B[:, 1:]
    b = H[1:, 0]
    C = H[1:, 1:]
    z = V.T @ yw
    beta = v1 @ yw
    L, dropped = cholesky_floor(C, p.pivot_floor)
    d = forward_subst(L, dropped, b)
    e = forward_subst(L, dropped, z)
    ell = degrees[1:].astype(LD)
    mu = (ell * (ell + 1)) ** LD(p.sobolev_s)        # eq. mls degree multipliers, d = 2
    r0 = np.sum(d * d)
    chi = LD(np.inf) if r0 >= 1 else 1 / (1 - r0)
    chiT, chiF = LD(p.chi_target), LD(p.chi_full)
    tau = LD(0)
    tau_t = LD(0)
    if tau_override is not None:
        tau = tau_t = LD(tau_override)
    elif chi > chiT:
        rstar = 1 - 1 / chiT
        lo, hi = LD(0), r0 / (np.min(mu) * rstar)      # r_hi <= r0 / (hi mu_min) = r*
        for _ in range(p.bisect_iters):
            mid = (lo + hi) / 2
            if np.sum(d * d / (1 + mid * mu)) > rstar:
                lo = mid
            else:
                hi = mid
            if hi - lo <= LD(1e-18) * hi:
                break
        tau = (lo + hi) / 2
        tt = LD(1) if not np.isfinite(chi) else min(LD(1), (chi - chiT) / (chiF - chiT))
        tau_t = smoothstep3(tt) * tau
    den = 1 - np.sum(d * d / (1 + tau_t * mu))
    num = beta - np.sum(d * e / (1 + tau_t * mu))
    return LocalResult(num / den, chi, tau, tau_t, B.shape[0], int(dropped.sum()), d, e, beta, L, B, yw, mu)


def solve_local_literal(res: LocalResult) -> LD:
    """Form A: solve the regularised normal equations
    [[1, b^T], [b, L (I + tau~ D) L^T]] c = B^T y_w and return c_1 (used to
    pin the closed form; needs no dropped direction)."""
    B, yw, L, mu = res.B, res.yw, res.L, res.mu
    H = B.T @ B
    Ht = H.copy()
    Ht[1:, 1:] = L @ np.diag(1 + res.tau_tilde * mu) @ L.T
    rhs = B.T @ yw
    return gauss_solve(Ht, rhs)[0]


def gauss_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense solve by Gaussian elimination with partial pivoting, in the
    dtype of A (extended precision here; numpy.linalg has no longdouble)."""
    A = A.copy()
    b = b.copy()
    n = len(b)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            b[[k, p]] = b[[p, k]]
        f = A[k + 1:, k] / A[k, k]
        A[k + 1:, k:] -= f[:, None] * A[k, k:][None, :]
        b[k + 1:] -= f * b[k]
    x = np.zeros_like(b)
    for k in range(n - 1, -1, -1):
        x[k] = (b[k] - np.dot(A[k, k + 1:], x[k + 1:])) / A[k, k]
    return x


def mls_at(q_ld, xs, ys, delta, K, p: Params, vs=None, frame=None, tau_override=None) -> LocalResult:
    """Regularised MLS value at one centre q from its local nodes."""
    B, wn, degrees = local_design(q_ld, xs, delta, vs, K, frame, p.weight_fn)
    yw = np.sqrt(wn) * ys.astype(LD)
    res = solve_local(B, yw, degrees, p, tau_override)
    res.wn = wn
    return res


# --------------------------------------------------------------------------
# step 3: adjoint transform by quadrature (Alg. 1 step 3)
# --------------------------------------------------------------------------
def ring_dft(fgrid: np.ndarray, N: int) -> np.ndarray:
    """F[k, m] = sum_j f[k, j] exp(-i m phi_j), m = 0..N, by a direct DFT
    (extended precision, no FFT). Returns (re, im) longdouble arrays."""
    L = 2 * N + 2
    f = np.asarray(fgrid, dtype=LD).reshape(N + 1, L)
    j = np.arange(L, dtype=LD)
    mm = np.arange(N + 1, dtype=LD)
    ang = 2 * PI_LD * np.outer(j, mm) / LD(L)
    return f @ np.cos(ang), -(f @ np.sin(ang))


def legendre_m(N: int, m: int, t: np.ndarray) -> np.ndarray:
    """Pbar_l^m(t) for l = m..N (rows), orthonormal on the sphere with the
    Condon-Shortley phase, by the standard three-term recurrence in l at fixed
    m started from Pbar_m^m. Extended precision."""
    t = np.asarray(t, dtype=LD)
    s = np.sqrt(1 - t * t)
    pmm = np.full_like(t, 1 / np.sqrt(4 * PI_LD))
    for k in range(1, m + 1):
        pmm = -np.sqrt(LD(2 * k + 1) / LD(2 * k)) * s * pmm
    out = np.zeros((N + 1 - m, len(t)), dtype=LD)
    out[0] = pmm
    if m < N:
        out[1] = np.sqrt(LD(2 * m + 3)) * t * pmm
    for l in range(m + 2, N + 1):
        a = np.sqrt(LD(4 * l * l - 1) / LD(l * l - m * m))
        b = np.sqrt(LD((l - 1) ** 2 - m * m) / LD(4 * (l - 1) ** 2 - 1))
        out[l - m] = a * (t * out[l - m - 1] - b * out[l - m - 2])
    return out


def coeff_offset(N: int, m: int) -> int:
    """Start of order m in the packed m-major layout (l = m..N)."""
    return m * (N + 1) - m * (m - 1) // 2


def n_coeffs(N: int) -> int:
    return (N + 1) * (N + 2) // 2


def quadrature(fgrid: np.ndarray, grid: Grid) -> np.ndarray:
    """fhat_l^m = sum_j omega_j f(q_j) conj(Y_l^m(q_j)) (Alg. 1 step 3) on the
    product grid: (2 pi / (2N+2)) sum_k w_k Pbar_l^m(t_k) F_k(m).
    Returns packed complex128, m-major, l = m..N."""
    N = grid.N
    Fr, Fi = ring_dft(fgrid, N)
    h = 2 * PI_LD / LD(2 * N + 2)
    out = np.zeros(n_coeffs(N), dtype=np.complex128)
    for m in range(N + 1):
        P = legendre_m(N, m, grid.t) * (h * grid.w)[None, :]
        re = P @ Fr[:, m]
        im = P @ Fi[:, m]
        o = coeff_offset(N, m)
        out[o:o + N + 1 - m] = re.astype(np.float64) + 1j * im.astype(np.float64)
    return out


def unpack_coeffs(c: np.ndarray, N: int) -> np.ndarray:
    """Packed m-major -> array [l, m] (m <= l)."""
    out = np.zeros((N + 1, N + 1), dtype=c.dtype)
    for m in range(N + 1):
        o = coeff_offset(N, m)
        out[m:, m] = c[o:o + N + 1 - m]
    return out


def pack_coeffs(a: np.ndarray, N: int) -> np.ndarray:
    out = np.zeros(n_coeffs(N), dtype=a.dtype)
    for m in range(N + 1):
        o = coeff_offset(N, m)
        out[o:o + N + 1 - m] = a[m:N + 1, m]
    return out


def real_coeff_norm2(c_packed: np.ndarray, N: int) -> float:
    """sum over m = -l..l of |fhat_l^m|^2 for a real field stored with m >= 0."""
    a = unpack_coeffs(c_packed, N)
    return float(np.sum(np.abs(a[:, 0]) ** 2) + 2.0 * np.sum(np.abs(a[:, 1:]) ** 2))


# --------------------------------------------------------------------------
# Algorithm 1, end to end
# --------------------------------------------------------------------------
@dataclass
class HamlsResult:
    coeffs: Optional[np.ndarray]   # packed complex128 (None when only a subset was evaluated)
    fgrid: np.ndarray              # MLS values at the evaluated grid nodes (longdouble)
    subset: np.ndarray             # evaluated grid-node indices
    support: Support
    chi: np.ndarray
    tau_tilde: np.ndarray
    n_dropped: np.ndarray
    grid: Grid


class UnderdeterminedError(RuntimeError):
    pass


class SupportTooLargeError(RuntimeError):
    pass


def mls_grid_values(x: np.ndarray, y: np.ndarray, N: int, K: int, p: Params = Params(),
                    v: Optional[np.ndarray] = None, subset=None, grid: Optional[Grid] = None):
    """Alg. 1 step 2: f_j = M_y(q_j) at the grid nodes (or a subset of them)."""
    grid = grid or quad_grid(N)
    nodes = NodeSet(x)
    sel = np.arange(grid.MQ) if subset is None else np.asarray(subset, dtype=np.int64)
    sup = support_radius(nodes, grid.xyz, K, p, subset=sel)
    m = dim_tan(K)
    if np.any(sup.count < m):
        raise UnderdeterminedError("fewer than m nodes in the support of a grid node")
    if np.any(sup.delta >= PI_LD / 2):
        raise SupportTooLargeError("support radius reaches pi/2")
    f = np.zeros(len(sel), dtype=LD)
    chi = np.zeros(len(sel), dtype=LD)
    taut = np.zeros(len(sel), dtype=LD)
    ndrop = np.zeros(len(sel), dtype=np.int64)
    for jj, j in enumerate(sel):
        idx = nodes.ball(grid.xyz[j], sup.rho2[jj])
        res = mls_at(grid.xyz_ld[j], x[idx], y[idx], sup.delta[jj], K, p,
                     None if v is None else v[idx])
        f[jj], chi[jj], taut[jj], ndrop[jj] = res.c1, res.chi, res.tau_tilde, res.n_dropped
    return f, sel, sup, chi, taut, ndrop, grid


def hamls(x: np.ndarray, y: np.ndarray, N: int, K: int, p: Params = Params(),
          v: Optional[np.ndarray] = None, subset=None) -> HamlsResult:
    """Algorithm 1 on S^2: grid (step 1), MLS values (step 2), quadrature
    (step 3). With ``subset`` only those grid nodes are evaluated and no
    coefficients are returned."""
    f, sel, sup, chi, taut, ndrop, grid = mls_grid_values(x, y, N, K, p, v, subset)
    coeffs = quadrature(f, grid) if subset is None else None
    return HamlsResult(coeffs, f, sel, sup, chi, taut, ndrop, grid)


# --------------------------------------------------------------------------
# the neighbour-structure keys (bit-comparable definition)
# --------------------------------------------------------------------------
def cell_keys(x: np.ndarray, bands: int, cells: int) -> np.ndarray:
    """Integer cell key of each node: band from zeta = sign(z)(1 - sqrt(1-|z|))
    on ``bands`` equal steps of [-1, 1]; longitude cell from the diamond
    parameter of (x, y): quadrant q in 0..3 plus a fraction in [0, 1] given by
    one IEEE division, on ``cells`` equal steps of [0, 4).
    key = band * cells + cell. Plain float64, no fused operations."""
    X, Y, Z = (np.asarray(x[:, i], dtype=np.float64) for i in range(3))
    az = np.abs(Z)
    s = np.sqrt(1.0 - az)
    zeta = np.where(Z < 0, -(1.0 - s), 1.0 - s)
    band = np.floor((zeta + 1.0) * (bands / 2)).astype(np.int64)
    band = np.clip(band, 0, bands - 1)
    ax, ay = np.abs(X), np.abs(Y)
    den = ax + ay
    q = np.zeros(len(X), dtype=np.int64)
    num = np.zeros(len(X))
    c0 = (X > 0) & (Y >= 0)
    c1 = (X <= 0) & (Y > 0)
    c2 = (X < 0) & (Y <= 0)
    c3 = (X >= 0) & (Y < 0)
    q[c1], q[c2], q[c3] = 1, 2, 3
    num = np.where(c0 | c2, ay, np.where(c1 | c3, ax, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        frac = np.where(den > 0, num / den, 0.0)
    qc = cells // 4
    within = np.minimum(np.floor(frac * qc).astype(np.int64), qc - 1)
    return band * cells + q * qc + within


def cell_sort(keys: np.ndarray, n_cells: int):
    """Stable sort of (key, index) and the CSR cell start array of size
    n_cells + 1 (start[c] = first sorted position with key >= c)."""
    perm = np.argsort(keys, kind="stable")
    sk = keys[perm]
    start = np.searchsorted(sk, np.arange(n_cells + 1), side="left")
    return perm, sk, start

