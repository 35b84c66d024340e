"""The FP32 geodesic distance of the CUDA library's MLS weights and k-NN
bounds (`geodesic_series_f` in csrc/common.cuh) is the Maclaurin series of
arcsin. This pins the constants shipped in that source against the series'
exact coefficients (2k)! / (4^k (k!)^2 (2k+1)), and the same Horner scheme,
evaluated in FP32 with NumPy, against the FP64 arcsin over the range where
the library uses it (half-chord s <= 1/4)."""
import math
import os
import re
from fractions import Fraction

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2609_39200_b300", "csrc", "common.cuh")


def _series_constants():
    text = open(SRC).read()
    body = text[text.index("float geodesic_series_f(float c2)"):]
    body = body[:body.index("\n}\n")]
    # the Horner scheme: p = c5; p = fma(p, t, c4); ... p = fma(p, t, 1)
    first = re.search(r"float p = (\d+)\.f / (\d+)\.f;", body)
    rest = re.findall(r"__fmaf_rn\(p, t, (\d+)\.f(?: / (\d+)\.f)?\)", body)
    coeffs = [Fraction(int(first.group(1)), int(first.group(2)))]
    coeffs += [Fraction(int(a), int(b) if b else 1) for a, b in rest]
    return coeffs[::-1]          # ascending powers of t = s^2


def test_constants_are_the_arcsin_series():
    c = _series_constants()
    assert len(c) == 6
    for k, ck in enumerate(c):
        exact = Fraction(math.factorial(2 * k), 4 ** k * math.factorial(k) ** 2 * (2 * k + 1))
        assert ck == exact, (k, ck, exact)


def test_fp32_horner_matches_arcsin():
    c = [np.float32(float(x)) for x in _series_constants()]
    rng = np.random.default_rng(7)
    s64 = np.concatenate([rng.uniform(0, 0.25, 200_000), np.linspace(0, 0.25, 1001)])
    c2 = (4.0 * s64 * s64).astype(np.float32)
    s = np.float32(0.5) * np.sqrt(c2)
    t = s * s
    p = np.full_like(t, c[5])
    for k in (4, 3, 2, 1, 0):
        p = (p * t + c[k]).astype(np.float32)       # FP32 products and sums (bounds the fused form too)
    got = (np.float32(2.0) * s * p).astype(np.float64)
    ref = 2.0 * np.arcsin(0.5 * np.sqrt(c2.astype(np.float64)))
    nz = ref > 0
    rel = np.abs(got[nz] / ref[nz] - 1.0)
    # a few FP32 roundings; the truncation after s^11 is below 1.1e-9 of the sum
    assert rel.max() < 4e-7
    # the first omitted term at s = 1/4, relative to the sum
    s_max = 0.25
    omitted = float(Fraction(math.factorial(12), 4 ** 6 * math.factorial(6) ** 2 * 13)) * s_max ** 13
    assert omitted / math.asin(s_max) < 1.1e-9
