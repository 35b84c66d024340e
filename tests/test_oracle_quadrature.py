"""Pins for the oracle's step 1 and step 3 (grid, ring DFT, Legendre quadrature).

Each test checks the oracle against something other than itself: exact
integrals of monomials, the addition theorem, closed-form low-degree
functions, scipy's independent spherical harmonics, band-limited fields
synthesised by the independent generator, and the closed-form expansion of a
Gaussian bump (modified spherical Bessel functions)."""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y, spherical_in

import oracle as O
from hamls_synth import random_field_coeffs, synth_field


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 65])
def test_gauss_legendre_integrates_monomials(n):
    # Sec. 2.1: the Gauss-Legendre rule with n nodes is exact up to degree 2n-1
    t, w = O.gauss_legendre(n)
    assert np.all(np.diff(t.astype(float)) < 0)          # descending: north first
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(float(np.sum(w * t ** p)) - exact) < 1e-15 * max(1, n / 8)


def test_gauss_legendre_not_exact_beyond():
    t, w = O.gauss_legendre(5)
    assert abs(float(np.sum(w * t ** 10)) - 2.0 / 11) > 1e-6


def test_legendre_addition_theorem():
    # sum_m |Y_l^m|^2 = (2l+1)/(4 pi) for every t
    N = 40
    t = np.array([-0.999, -0.3, 0.0, 0.51, 0.97], dtype=O.LD)
    acc = np.zeros((N + 1, len(t)), dtype=O.LD)
    for m in range(N + 1):
        P = O.legendre_m(N, m, t)
        acc[m:] += (1 if m == 0 else 2) * P * P
    for l in range(N + 1):
        assert np.allclose(acc[l].astype(float), (2 * l + 1) / (4 * math.pi), rtol=1e-14, atol=0)


def test_legendre_closed_forms():
    t = np.array([-0.7, 0.2, 0.9], dtype=O.LD)
    s = np.sqrt(1 - t * t)
    c = 1 / np.sqrt(4 * O.PI_LD)
    expect = {
        (0, 0): c * np.ones_like(t),
        (1, 0): np.sqrt(O.LD(3)) * c * t,
        (1, 1): -np.sqrt(O.LD(3) / 2) * c * s,            # Condon-Shortley phase
        (2, 0): np.sqrt(O.LD(5)) * c * (3 * t * t - 1) / 2,
        (2, 1): -np.sqrt(O.LD(15) / 2) * c * t * s,
        (2, 2): np.sqrt(O.LD(15) / 8) * c * s * s,
    }
    for (l, m), v in expect.items():
        P = O.legendre_m(3, m, t)[l - m]
        assert np.allclose(P.astype(float), v.astype(float), rtol=1e-15, atol=1e-17)


def test_legendre_matches_scipy_sph_harm():
    th = np.array([0.3, 1.1, 2.9])
    ph = np.array([0.0, 2.0, 5.0])
    for l, m in [(3, 2), (10, 7), (25, 0), (40, 40), (60, 13)]:
        ours = O.legendre_m(60, m, np.cos(th).astype(O.LD))[l - m].astype(float) * np.exp(1j * m * ph)
        ref = sph_harm_y(l, m, th, ph)
        assert np.allclose(ours, ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("N", [4, 16, 31])
def test_quadrature_reproduces_bandlimited(N):
    # Alg. 1 step 3 on a grid exact on Pi_{2N}: f in Pi_N is reproduced exactly
    # (f_Q = f for f in Pi_L, eq. quadrature_based_approximation)
    c = random_field_coeffs(1234 + N, N)
    g = O.quad_grid(N)
    f = synth_field(c, g.xyz)
    got = O.unpack_coeffs(O.quadrature(f, g), N)
    assert np.max(np.abs(got - np.tril(c))) < 1e-13


def test_quadrature_parseval():
    # F^H W F = I on Pi_N: sum_j omega_j f_j^2 = ||fhat||^2
    N = 20
    c = random_field_coeffs(7, N)
    g = O.quad_grid(N)
    f = synth_field(c, g.xyz)
    wq = np.repeat((g.w * 2 * O.PI_LD / (2 * N + 2)).astype(float), 2 * N + 2)
    assert abs(np.sum(wq * f * f) - O.real_coeff_norm2(O.pack_coeffs(c, N), N)) < 1e-12


def test_quadrature_grid_weights_sum_to_area():
    g = O.quad_grid(12)
    total = np.sum(g.w) * (2 * O.PI_LD / (2 * 12 + 2)) * (2 * 12 + 2)
    assert abs(float(total) - 4 * math.pi) < 1e-14


def test_quadrature_bump_closed_form():
    # exp(kappa x.c) = sum_l 4 pi i_l(kappa) sum_m Y_l^m(x) conj(Y_l^m(c)), so the
    # Gaussian bump exp(-|x-c|^2/0.1) = e^{-20} e^{20 x.c} has coefficients
    # e^{-20} 4 pi i_l(20) conj(Y_l^m(c)); aliasing beyond degree 2N+1-l is
    # below 1e-15 relative at N = 40.
    N = 40
    c = np.array([0.3, -0.5, 0.8])
    c /= np.linalg.norm(c)
    g = O.quad_grid(N)
    f = np.exp(-np.sum((g.xyz - c) ** 2, axis=1) / 0.1)
    got = O.unpack_coeffs(O.quadrature(f, g), N)
    th, ph = math.acos(c[2]), math.atan2(c[1], c[0])
    exp = np.zeros_like(got)
    for l in range(N + 1):
        for m in range(l + 1):
            exp[l, m] = math.exp(-20) * 4 * math.pi * spherical_in(l, 20.0) * np.conj(sph_harm_y(l, m, th, ph))
    assert np.max(np.abs(got - exp)) < 1e-13 * np.max(np.abs(exp))


def test_ring_dft_against_fft():
    N = 9
    rng = np.random.default_rng(0)
    f = rng.standard_normal((N + 1) * (2 * N + 2))
    Fr, Fi = O.ring_dft(f, N)
    ref = np.fft.fft(f.reshape(N + 1, 2 * N + 2), axis=1)[:, :N + 1]
    assert np.allclose(Fr.astype(float), ref.real, atol=1e-13)
    assert np.allclose(Fi.astype(float), ref.imag, atol=1e-13)


def test_packing_layout():
    N = 6
    assert O.n_coeffs(N) == 28
    assert [O.coeff_offset(N, m) for m in range(N + 1)] == [0, 7, 13, 18, 22, 25, 27]
    a = np.arange(49).reshape(7, 7).astype(complex)
    assert np.array_equal(O.unpack_coeffs(O.pack_coeffs(a, N), N), np.tril(a))


def test_paper_printed_values():
    # tests/golden/paper_values.txt holds the values the paper prints
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = v
    assert O.dim_tan(2) == int(vals["dim_tan_K2"])
    assert O.dim_tan(4) == int(vals["dim_tan_K4"])
    assert O.Params().n_for(4) == int(vals["n_target_K4"])
    for N in (3, 16):
        assert O.quad_grid(N).MQ == (2 * N + 2) * (N + 1)
