"""Seeded generators: scattered nodes on S^2 and synthetic fields sampled at them.

Every random number comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream s is mix(seed_s + (i+1) * 0x9E3779B97F4A7C15).
Uniform doubles take the top 53 bits; normal variates use Box-Muller.

The node sets mirror the shape of the paper's sphere experiments (Sec. 3.1,
3.2): dense clusters, sparse regions and large gaps. Three families:

* ``uniform_minus_cap_nodes``: uniform nodes with one spherical cap removed.
* ``track_hole_nodes``: a fraction of the nodes along random great-circle
  tracks with Gaussian cross-track jitter, the rest uniform, and several caps
  ("holes") with no nodes at all.

Fields:

* ``bump_field``: sum of Gaussian bumps exp(-|x - c|^2 / s) (closed-form SH
  expansion, used by the small workload).
* ``random_field_coeffs`` + ``synth_field``: a random band-limited real field
  with a prescribed degree spectrum; ``synth_field`` evaluates
  sum_{l,m} fhat_l^m Y_l^m(x) with fully normalised complex spherical
  harmonics (Condon-Shortley phase), for numpy arrays on the CPU or torch
  tensors on any device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class SplitMix64:
    """Counter-based SplitMix64 streams.

    ``stream(tag)`` derives an independent stream from the base seed; each
    stream hands out consecutive counters, so draws are reproducible in any
    batch size.
    """

    def __init__(self, seed: int, tag: int = 0):
        with np.errstate(over="ignore"):
            base = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^
                                    np.uint64((tag * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF)],
                                   dtype=np.uint64))[0]
        self.base = np.uint64(base)
        self.counter = 0

    def stream(self, tag: int) -> "SplitMix64":
        return SplitMix64(int(self.base), tag + 1)

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + i * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normal variates (Box-Muller, both branches)."""
        h = (n + 1) // 2
        u1 = 1.0 - self.uniform(h)          # (0, 1]
        u2 = self.uniform(h)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * h)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:n]


def uniform_sphere(rng: SplitMix64, n: int) -> np.ndarray:
    """n points uniform on S^2 (z uniform in [-1, 1], longitude uniform)."""
    z = 2.0 * rng.uniform(n) - 1.0
    ph = 2.0 * np.pi * rng.uniform(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


def _in_caps(x: np.ndarray, centres: np.ndarray, radii_rad: np.ndarray) -> np.ndarray:
    inside = np.zeros(len(x), dtype=bool)
    for c, r in zip(centres, radii_rad):
        inside |= (x @ c) > math.cos(r)
    return inside


def remove_caps(x: np.ndarray, centres: np.ndarray, radii_rad: np.ndarray) -> np.ndarray:
    return x[~_in_caps(x, centres, radii_rad)]


def _orthonormal_pair(nrm: np.ndarray):
    """Two unit vectors a, b with (a, b, nrm) orthonormal."""
    helper = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    a = np.cross(helper, nrm)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(nrm, a)
    return a, b


def _track_points(rng: SplitMix64, n: int, normals: np.ndarray, sigma_rad: float) -> np.ndarray:
    t = np.minimum((rng.uniform(n) * len(normals)).astype(np.int64), len(normals) - 1)
    s = 2.0 * np.pi * rng.uniform(n)
    g = sigma_rad * rng.normal(n)
    nrm = normals[t]
    a, b = _orthonormal_pair(nrm)
    p = np.cos(s)[:, None] * a + np.sin(s)[:, None] * b
    x = np.cos(g)[:, None] * p + np.sin(g)[:, None] * nrm
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def _fill_outside(gen_batch, n: int, centres, radii) -> np.ndarray:
    """Rejection sampling until exactly n points lie outside every cap."""
    out, have = [], 0
    while have < n:
        need = n - have
        cand = gen_batch(int(need * 1.25) + 64)
        cand = cand[~_in_caps(cand, centres, radii)] if len(centres) else cand
        out.append(cand[:need])
        have += len(out[-1])
    return np.concatenate(out, axis=0)


def uniform_minus_cap_nodes(seed: int, M: int, cap_deg: float = 30.0):
    """M uniform nodes with every node inside one random cap removed."""
    rng = SplitMix64(seed)
    c = uniform_sphere(rng.stream(1), 1)
    radii = np.array([math.radians(cap_deg)])
    u = rng.stream(2)
    x = _fill_outside(lambda k: uniform_sphere(u, k), M, c, radii)
    return x, dict(cap_centres=c, cap_radii=radii)


def track_hole_nodes(seed: int, M: int, n_tracks: int = 40, track_frac: float = 0.6,
                     sigma_deg: float = 0.5, hole_deg=(10.0, 20.0, 35.0)):
    """Ill-distributed nodes: tracks along random great circles plus uniform
    background, with random caps removed (rejection until exactly M remain)."""
    rng = SplitMix64(seed)
    normals = uniform_sphere(rng.stream(1), n_tracks)
    hole_deg = tuple(hole_deg)
    centres = uniform_sphere(rng.stream(2), len(hole_deg)) if hole_deg else np.zeros((0, 3))
    radii = np.radians(np.array(hole_deg, dtype=np.float64))
    n_track = int(round(track_frac * M))
    tr, un = rng.stream(3), rng.stream(4)
    xt = _fill_outside(lambda k: _track_points(tr, k, normals, math.radians(sigma_deg)), n_track,
                       centres, radii)
    xu = _fill_outside(lambda k: uniform_sphere(un, k), M - n_track, centres, radii)
    x = np.concatenate([xt, xu], axis=0)
    perm = np.argsort(rng.stream(5).u64(M), kind="stable")   # interleave: no order leaks into tests
    return x[perm], dict(track_normals=normals, cap_centres=centres, cap_radii=radii)


def bump_field(seed: int, x: np.ndarray, n_bumps: int = 5, width: float = 0.1):
    """f(x) = sum_i exp(-|x - c_i|^2 / width) with random unit centres c_i."""
    c = uniform_sphere(SplitMix64(seed).stream(7), n_bumps)
    f = np.zeros(len(x))
    for ci in c:
        d2 = np.sum((x - ci) ** 2, axis=1)
        f += np.exp(-d2 / width)
    return f, c


def random_field_coeffs(seed: int, L: int, power: float = -3.0):
    """Random real band-limited field up to degree L.

    Degree-l total power is proportional to (1+l)^power, spread evenly over the
    2l+1 orders, and the field is scaled to unit RMS over the sphere. Returns a
    complex array c[l, m] for m = 0..l (m > l unused), with the real-field
    symmetry fhat_l^{-m} = (-1)^m conj(fhat_l^m) implied.
    """
    rng = SplitMix64(seed).stream(11)
    c = np.zeros((L + 1, L + 1), dtype=np.complex128)
    for l in range(L + 1):
        var = (1.0 + l) ** power / (2 * l + 1)
        g = rng.normal(2 * l + 1)
        c[l, 0] = math.sqrt(var) * g[0]
        if l:
            c[l, 1:l + 1] = math.sqrt(var / 2.0) * (g[1:l + 1] + 1j * g[l + 1:2 * l + 1])
    # RMS over the sphere = ||fhat||_2 / sqrt(4 pi)
    nrm2 = np.sum(np.abs(c[:, 0]) ** 2) + 2.0 * np.sum(np.abs(c[:, 1:]) ** 2)
    c *= math.sqrt(4.0 * math.pi / nrm2)
    return c


def coeff_norm2(c: np.ndarray) -> float:
    """sum over all (l, m), m = -l..l, of |fhat_l^m|^2 for a real field stored m >= 0."""
    return float(np.sum(np.abs(c[:, 0]) ** 2) + 2.0 * np.sum(np.abs(c[:, 1:]) ** 2))


def synth_field(coeffs: np.ndarray, x, xp=np, chunk: Optional[int] = None):
    """Evaluate sum_{l,m} fhat_l^m Y_l^m at unit vectors x (real field).

    Y_l^m(theta, phi) = Pbar_l^m(cos theta) e^{i m phi}, Pbar orthonormal on the
    sphere with the Condon-Shortley phase. Works for numpy arrays (xp=np) and
    torch tensors (xp=torch, on any device). The recurrence over l at fixed m is
    the standard three-term one for fully normalised functions.
    """
    L = coeffs.shape[0] - 1
    n = x.shape[0]
    if chunk is not None and n > chunk:
        parts = [synth_field(coeffs, x[i:i + chunk], xp) for i in range(0, n, chunk)]
        return xp.cat(parts) if xp is not np else np.concatenate(parts)
    t = x[:, 2]
    rxy = xp.sqrt(x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1])
    s = rxy                                  # sin(theta)
    safe = xp.where(rxy > 0, rxy, 1.0)
    ce = xp.where(rxy > 0, x[:, 0] / safe, 1.0)     # cos(phi)
    se = xp.where(rxy > 0, x[:, 1] / safe, 0.0)     # sin(phi)
    out = xp.zeros_like(t)
    pmm = xp.ones_like(t) * (1.0 / math.sqrt(4.0 * math.pi))
    cm, sm = xp.ones_like(t), xp.zeros_like(t)      # cos(m phi), sin(m phi)
    for m in range(L + 1):
        if m > 0:
            pmm = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
            cm, sm = cm * ce - sm * se, sm * ce + cm * se
        # sum_l fhat_l^m Pbar_l^m(t), real and imaginary parts
        ar = float(coeffs[m, m].real) * pmm
        ai = float(coeffs[m, m].imag) * pmm
        p2, p1 = pmm, None
        if m < L:
            p1 = math.sqrt(2.0 * m + 3.0) * t * pmm
            ar = ar + float(coeffs[m + 1, m].real) * p1
            ai = ai + float(coeffs[m + 1, m].imag) * p1
        for l in range(m + 2, L + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            p = a * (t * p1 - b * p2)
            cr, ci = coeffs[l, m].real, coeffs[l, m].imag
            ar = ar + float(cr) * p
            ai = ai + float(ci) * p
            p2, p1 = p1, p
        if m == 0:
            out = out + ar
        else:
            out = out + 2.0 * (ar * cm - ai * sm)
    return out


@dataclass
class Workload:
    name: str
    N: int
    K: int
    M: int
    nodes: np.ndarray
    values: np.ndarray
    truth: Optional[np.ndarray] = None        # fhat[l, m], m >= 0, complex (None if not band-limited)
    meta: dict = field(default_factory=dict)


WORKLOADS = {
    # N=16, K=2, M=5000 uniform minus one 30 degree cap, 5 Gaussian bumps, noise sigma 1e-3
    "s2_n16_k2_m5k": dict(N=16, K=2, M=5000, nodes="cap", field="bumps", noise=1e-3),
    # N=128, K=3, M=200k tracks + holes, random field to degree 200, noise 1e-4
    "s2_n128_k3_m200k": dict(N=128, K=3, M=200_000, nodes="tracks", field="random", L_field=200, noise=1e-4),
    # N=512, K=3, M=4M tracks + holes, random field to degree 200, noise 1e-4
    "s2_n512_k3_m4m": dict(N=512, K=3, M=4_000_000, nodes="tracks", field="random", L_field=200, noise=1e-4),
}

SEED_BASE = 0x48414D4C53


def workload(name: str, fit_index: int = 0, M: Optional[int] = None, xp=np, device=None,
             L_field: Optional[int] = None) -> Workload:
    """Build one seeded workload. ``xp=torch`` evaluates the random field with
    torch on ``device`` (used for multi-million-node inputs); the result is
    always returned as numpy float64 arrays."""
    spec = dict(WORKLOADS[name])
    idx = list(WORKLOADS).index(name)
    seed = SEED_BASE ^ (idx << 32) ^ fit_index
    if M is not None:
        spec["M"] = M
    if L_field is not None:
        spec["L_field"] = L_field
    if spec["nodes"] == "cap":
        x, meta = uniform_minus_cap_nodes(seed, spec["M"])
    else:
        x, meta = track_hole_nodes(seed, spec["M"])
    truth = None
    if spec["field"] == "bumps":
        f, c = bump_field(seed, x)
        meta["bump_centres"] = c
    else:
        truth = random_field_coeffs(seed, spec["L_field"])
        if xp is np:
            f = synth_field(truth, x, np, chunk=1 << 16)
        else:
            tx = xp.as_tensor(x, dtype=xp.float64, device=device)
            f = synth_field(truth, tx, xp, chunk=1 << 22).cpu().numpy()
    noise = SplitMix64(seed).stream(13).normal(len(f)) * spec["noise"]
    return Workload(name, spec["N"], spec["K"], spec["M"], x, f + noise, truth, meta)


# ---------------------------------------------------------------- many fits
@dataclass
class FitSpec:
    """One fit of a batch or of a serving trace: sizes, holes and its seed."""
    index: int
    N: int
    K: int
    M: int
    holes_deg: tuple
    seed: int
    arrival_s: float = 0.0      # serving traces: arrival time of the request


BATCH_N = (32, 64, 128, 256)
HOLES_DEG = (10.0, 20.0, 35.0)
SERVE_N = (64, 128, 256, 512, 1024)
SERVE_P = (0.30, 0.30, 0.20, 0.15, 0.05)


def batch_specs(n_fits: int = 256, seed: int = SEED_BASE ^ (3 << 32)) -> list:
    """A batch of independent fits: N uniform over {32, 64, 128, 256}, M
    log-uniform in [1e4, 1e6], K uniform over {2, 3}, and 0 to 3 holes (the
    first h of 10, 20 and 35 degrees), each fit with its own seed."""
    u = SplitMix64(seed).stream(1).uniform(4 * n_fits).reshape(n_fits, 4)
    specs = []
    for i in range(n_fits):
        N = BATCH_N[min(int(u[i, 0] * 4), 3)]
        M = int(round(10.0 ** (4.0 + 2.0 * u[i, 1])))
        K = 2 + min(int(u[i, 2] * 2), 1)
        h = min(int(u[i, 3] * 4), 3)
        specs.append(FitSpec(i, N, K, M, HOLES_DEG[:h], (seed ^ (i + 1)) & 0xFFFFFFFFFFFFFFFF))
    return specs


def serving_trace(rate_per_s: float, n_requests: int, seed: int = SEED_BASE ^ (4 << 32)) -> list:
    """Requests arriving as a Poisson process of rate rate_per_s (exponential
    gaps): N from {64, 128, 256, 512, 1024} with probabilities
    {0.30, 0.30, 0.20, 0.15, 0.05}, M log-uniform in [5e4, 1.6e7], K = 3, the
    three holes of the benchmark workload."""
    rng = SplitMix64(seed)
    gaps = -np.log(1.0 - rng.stream(1).uniform(n_requests)) / rate_per_s
    t = np.cumsum(gaps)
    un = rng.stream(2).uniform(n_requests)
    um = rng.stream(3).uniform(n_requests)
    cum = np.cumsum(SERVE_P)
    specs = []
    for i in range(n_requests):
        N = SERVE_N[min(int(np.searchsorted(cum, un[i], side="right")), len(SERVE_N) - 1)]
        M = int(round(5e4 * (1.6e7 / 5e4) ** um[i]))
        specs.append(FitSpec(i, N, 3, M, HOLES_DEG, (seed ^ (i + 1)) & 0xFFFFFFFFFFFFFFFF, float(t[i])))
    return specs


def fit_workload(spec: FitSpec, xp=np, device=None, L_field: int = 200, noise: float = 1e-4) -> Workload:
    """The nodes and values of one fit: track/hole nodes with the spec's holes
    and a random field to degree L_field (degree power (1+l)^-3), noise sigma."""
    x, meta = track_hole_nodes(spec.seed, spec.M, hole_deg=spec.holes_deg)
    truth = random_field_coeffs(spec.seed, L_field)
    if xp is np:
        f = synth_field(truth, x, np, chunk=1 << 16)
    else:
        tx = xp.as_tensor(x, dtype=xp.float64, device=device)
        f = synth_field(truth, tx, xp, chunk=1 << 22).cpu().numpy()
    f = f + SplitMix64(spec.seed).stream(13).normal(len(f)) * noise
    return Workload(f"fit{spec.index}_n{spec.N}_k{spec.K}_m{spec.M}", spec.N, spec.K, spec.M, x, f, truth, meta)
