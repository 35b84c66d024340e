"""Pins of the forward transform and the dense least-squares comparator (CPU).

forward() evaluates sum fhat_l^m Y_l^m at scattered nodes (the sampling matrix
F of the problem statement, eq. LSQR-Problem_Regularized); global_lsq() solves
that weighted, regularised least-squares problem densely for tiny sizes."""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y, spherical_in

import oracle as O
from oracle.forward import complex_coeffs, forward, forward_full, global_lsq
from hamls_synth import SplitMix64, uniform_sphere


def angles(x):
    return np.arccos(np.clip(x[:, 2], -1, 1)), np.arctan2(x[:, 1], x[:, 0])


def random_real_coeffs(N, seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=O.n_coeffs(N)) + 1j * rng.normal(size=O.n_coeffs(N))
    for l in range(N + 1):
        c[O.coeff_offset(N, 0) + l] = c[O.coeff_offset(N, 0) + l].real      # m = 0 is real for a real field
    return c


@pytest.mark.parametrize("l,m", [(0, 0), (3, 0), (5, 2), (12, 7), (20, 20)])
def test_single_harmonic_matches_scipy(l, m):
    N = 20
    x = uniform_sphere(SplitMix64(l * 31 + m), 200)
    th, ph = angles(x)
    c = np.zeros(O.n_coeffs(N), dtype=np.complex128)
    coef = 0.7 - 0.4j if m > 0 else 0.7
    c[O.coeff_offset(N, m) + (l - m)] = coef
    Y = sph_harm_y(l, m, th, ph)
    exp = (coef * Y).real if m == 0 else 2 * (coef * Y).real
    np.testing.assert_allclose(forward(c, N, x), exp, rtol=0, atol=1e-13)


def test_round_trip_with_the_grid_quadrature():
    # the grid rule is exact on Pi_2N, so quadrature() inverts forward() on Pi_N
    N = 14
    c = random_real_coeffs(N, 1)
    g = O.quad_grid(N)
    f = forward(c, N, g.xyz)
    back = O.quadrature(f.reshape(N + 1, 2 * N + 2), g)
    np.testing.assert_allclose(back, c, rtol=0, atol=1e-12)


def test_gaussian_bump_closed_form():
    # exp(-|x - c|^2 / 0.1) = e^{-20} e^{20 x.c} has fhat_l^m = 4 pi e^{-20} i_l(20) conj(Y_l^m(c))
    N = 48
    cen = np.array([0.3, -0.5, 0.81])
    cen /= np.linalg.norm(cen)
    thc, phc = angles(cen[None, :])
    c = np.zeros(O.n_coeffs(N), dtype=np.complex128)
    for m in range(N + 1):
        for l in range(m, N + 1):
            c[O.coeff_offset(N, m) + l - m] = 4 * np.pi * np.exp(-20) * spherical_in(l, 20.0) * np.conj(
                sph_harm_y(l, m, thc, phc)[0])
    x = uniform_sphere(SplitMix64(4), 500)
    exact = np.exp(-np.sum((x - cen) ** 2, axis=1) / 0.1)
    assert np.max(np.abs(forward(c, N, x) - exact)) < 1e-10


def test_complex_data_as_two_real_fields():
    N = 10
    cu, cv = random_real_coeffs(N, 2), random_real_coeffs(N, 3)
    x = uniform_sphere(SplitMix64(5), 300)
    f = forward_full(complex_coeffs(cu, cv, N), N, x)
    np.testing.assert_allclose(f.real, forward(cu, N, x), atol=1e-12)
    np.testing.assert_allclose(f.imag, forward(cv, N, x), atol=1e-12)


def test_lsq_with_an_exact_quadrature_rule_is_the_adjoint():
    # nodes and weights of an exact rule give F^H W F = I: with alpha = 0 the
    # least-squares solution is F^H W y, the quadrature of the data
    N = 8
    g = O.quad_grid(N)
    w = np.repeat(np.asarray(g.w, dtype=np.float64), 2 * N + 2) * (2 * np.pi / (2 * N + 2))
    y = np.random.default_rng(6).normal(size=len(w))
    lsq = global_lsq(g.xyz, y, N, w=w)
    adj = O.quadrature(y.reshape(N + 1, 2 * N + 2), g)
    np.testing.assert_allclose(lsq, adj, rtol=0, atol=1e-12)


def test_lsq_recovers_band_limited_data():
    N = 6
    c = random_real_coeffs(N, 7)
    x = uniform_sphere(SplitMix64(8), 400)
    np.testing.assert_allclose(global_lsq(x, forward(c, N, x), N), c, rtol=0, atol=1e-10)


def test_lsq_regularisation_damps_high_degrees():
    # with alpha > 0 the Sobolev penalty (1 + l(l+1))^s shrinks every degree,
    # the high ones most
    N = 6
    c = random_real_coeffs(N, 9)
    x = uniform_sphere(SplitMix64(10), 400)
    y = forward(c, N, x)
    r = global_lsq(x, y, N, alpha=1e-3)
    ratio = np.abs(O.unpack_coeffs(r, N)) / np.maximum(np.abs(O.unpack_coeffs(c, N)), 1e-300)
    per_degree = [np.mean(ratio[l, :l + 1]) for l in range(N + 1)]
    assert all(p < 1 + 1e-12 for p in per_degree)
    assert per_degree[-1] < per_degree[1]


def test_hamls_close_to_the_global_least_squares_fit():
    # well-distributed nodes (Fibonacci), a smooth bump, Voronoi weights for
    # both: the dense least-squares fit reaches the L2 projection's error, and
    # HAMLS stays within 5 % of it (the paper compares the two in Sec. 3)
    N, NT = 12, 60
    x = O.fibonacci_points(3000)
    cen = np.array([0.3, -0.5, 0.81])
    cen /= np.linalg.norm(cen)
    y = np.exp(-np.sum((x - cen) ** 2, axis=1) / 0.1)
    thc, phc = np.arccos(cen[2]), np.arctan2(cen[1], cen[0])

    def truth(n):
        c = np.zeros(O.n_coeffs(n), dtype=np.complex128)
        for m in range(n + 1):
            for l in range(m, n + 1):
                c[O.coeff_offset(n, m) + l - m] = 4 * np.pi * np.exp(-20) * spherical_in(l, 20.0) * np.conj(
                    sph_harm_y(l, m, thc, phc))
        return c

    ct, full = truth(N), O.real_coeff_norm2(truth(NT), NT)
    tail2 = full - O.real_coeff_norm2(ct, N)
    err = lambda c: math.sqrt((O.real_coeff_norm2(c - ct, N) + tail2) / full)
    v = O.voronoi_areas(x)
    e_lsq = err(global_lsq(x, y, N, w=v))
    e_ham = err(O.hamls(x, y, N, 3, O.Params(), v=v).coeffs)
    assert e_lsq < 1.0001 * math.sqrt(tail2 / full)
    assert e_ham < 1.05 * e_lsq
