"""Forward transform and dense least-squares comparator on S^2 (test
infrastructure).

forward: the sampling matrix F of the paper's problem statement (Sec. 1,
eq. LSQR-Problem_Regularized) applied to a coefficient vector,
    f(x) = sum_{l=0}^{N} sum_{m=-l}^{l} fhat_l^m Y_l^m(x),
    Y_l^m(theta, phi) = Pbar_l^m(cos theta) e^{i m phi}
(fully normalised, Condon-Shortley phase: the convention of quadrature(), the
adjoint F^H W on the grid). A real field stores m >= 0 only, with
fhat_l^{-m} = (-1)^m conj(fhat_l^m), so
    f(x) = sum_l fhat_l^0 Pbar_l^0 + 2 Re sum_{m>=1} e^{i m phi} sum_l fhat_l^m Pbar_l^m.
Complex data y = u + i v (the problem statement allows complex values) is
fitted as two real fields; complex_coeffs() combines their coefficients into
the full set over m = -l..l, and forward_full() evaluates such a set.

global_lsq: the weighted, regularised least-squares problem itself,
    min || W^{1/2} (F fhat - y) ||^2 + alpha || R^{1/2} fhat ||^2,
    R_kk = (1 + l(l+1))^s,
for real data, by an SVD of the stacked system in the real parametrisation
(Re and Im of fhat_l^m for m >= 1 count twice in both norms). The paper solves
it with LSQR at large sizes; this dense solve is a comparator for tiny N and M.

Pins (tests/test_oracle_forward.py): scipy's sph_harm_y for single
coefficients, the exact round trip with the grid quadrature, the closed-form
expansion of a Gaussian bump, the combination of two real fields into a
complex one, and, for global_lsq, the paper's remark that an exact quadrature
rule makes the solution the adjoint F^H W y, and exact recovery of
band-limited data.
"""
from __future__ import annotations

import numpy as np

from .hamls_oracle import LD, coeff_offset, legendre_m, n_coeffs


def _angles(x):
    x = np.asarray(x, dtype=np.float64)
    t = np.clip(x[:, 2], -1.0, 1.0).astype(LD)
    phi = np.arctan2(x[:, 1], x[:, 0]).astype(LD)
    return t, phi


def forward(c_packed: np.ndarray, N: int, x: np.ndarray) -> np.ndarray:
    """Values at the nodes x (M x 3) of the real field with packed m >= 0
    coefficients c_packed (m-major, l = m..N). Extended precision."""
    t, phi = _angles(x)
    c = np.asarray(c_packed, dtype=np.complex128)
    f = np.zeros(len(t), dtype=LD)
    for m in range(N + 1):
        P = legendre_m(N, m, t)                              # (N+1-m) x M
        o = coeff_offset(N, m)
        cm = c[o:o + N + 1 - m]
        gr = cm.real.astype(LD) @ P
        gi = cm.imag.astype(LD) @ P
        if m == 0:
            f += gr
        else:
            f += 2 * (gr * np.cos(m * phi) - gi * np.sin(m * phi))
    return f.astype(np.float64)


def complex_coeffs(cu: np.ndarray, cv: np.ndarray, N: int) -> np.ndarray:
    """Full coefficients a[l, m + N] (m = -l..l) of u + i v from the packed
    m >= 0 coefficients of the real fields u and v."""
    a = np.zeros((N + 1, 2 * N + 1), dtype=np.complex128)
    for m in range(N + 1):
        o = coeff_offset(N, m)
        u = cu[o:o + N + 1 - m]
        v = cv[o:o + N + 1 - m]
        a[m:, N + m] = u + 1j * v
        if m > 0:
            a[m:, N - m] = (-1) ** m * (np.conj(u) + 1j * np.conj(v))
    return a


def forward_full(a: np.ndarray, N: int, x: np.ndarray) -> np.ndarray:
    """Complex values at x of the field with full coefficients a[l, m + N]."""
    t, phi = _angles(x)
    f = np.zeros(len(t), dtype=np.complex128)
    for m in range(N + 1):
        P = legendre_m(N, m, t).astype(np.float64)           # Pbar_l^m, m >= 0
        e = np.exp(1j * m * phi.astype(np.float64))
        f += (a[m:, N + m] @ P) * e
        if m > 0:
            # Y_l^{-m} = (-1)^m conj(Y_l^m)
            f += (a[m:, N - m] @ P) * (-1) ** m * np.conj(e)
    return f


def _real_design(N: int, x: np.ndarray):
    """Columns of F for the real parametrisation: Re fhat_l^0, and for m >= 1
    Re and Im of fhat_l^m (with their factor 2); the degree of each column."""
    t, phi = _angles(x)
    cols, deg = [], []
    for m in range(N + 1):
        P = legendre_m(N, m, t).astype(np.float64)
        if m == 0:
            for r in range(N + 1):
                cols.append(P[r]); deg.append(r)
        else:
            cm = np.cos(m * phi.astype(np.float64))
            sm = np.sin(m * phi.astype(np.float64))
            for r in range(N + 1 - m):
                cols.append(2 * P[r] * cm); deg.append(m + r)
                cols.append(-2 * P[r] * sm); deg.append(m + r)
    return np.stack(cols, axis=1), np.array(deg)


def global_lsq(x: np.ndarray, y: np.ndarray, N: int, w: np.ndarray = None, alpha: float = 0.0,
               s: float = 2.0) -> np.ndarray:
    """Packed coefficients (m >= 0) of the weighted, regularised least-squares
    fit of real data y at the nodes x, solved densely by SVD."""
    A, deg = _real_design(N, x)
    M = len(y)
    w = np.ones(M) if w is None else np.asarray(w, dtype=np.float64)
    sw = np.sqrt(w)
    # the coefficient norm counts Re/Im of m >= 1 twice (m and -m)
    mult = np.ones(A.shape[1])
    k = 0
    for m in range(N + 1):
        cnt = (N + 1 - m) * (1 if m == 0 else 2)
        if m > 0:
            mult[k:k + cnt] = 2.0
        k += cnt
    rows = [sw[:, None] * A]
    rhs = [sw * np.asarray(y, dtype=np.float64)]
    if alpha > 0:
        R = (1.0 + deg * (deg + 1.0)) ** s
        rows.append(np.diag(np.sqrt(alpha * R * mult)))
        rhs.append(np.zeros(A.shape[1]))
    z = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
    out = np.zeros(n_coeffs(N), dtype=np.complex128)
    k = 0
    for m in range(N + 1):
        o = coeff_offset(N, m)
        if m == 0:
            out[o:o + N + 1] = z[k:k + N + 1]
            k += N + 1
        else:
            for r in range(N + 1 - m):
                out[o + r] = z[k] + 1j * z[k + 1]
                k += 2
    return out
