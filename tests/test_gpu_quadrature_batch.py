"""Step 3 (eq. quadrature_based_approximation) for many sets of grid values
at once (hamls_quadrature_batch): ring FFTs of every set, the folded spectra,
and the Legendre contraction of all sets as one tensor-core product per
order and parity (tcgen05, 3xTF32, FP32 accumulation) for mixed plans.

* every set of a batch equals the single-set FP32 path (hamls_debug_quadrature)
  to FP32 rounding, and the oracle's quadrature on its first and last sets,
  per coefficient, at N = 128 and 512 for B = 1, 8, 64 and 256 (one to four
  128-row tiles of value-set parts), and at N = 16 and 256 (B = 17: a ragged
  tile);
* the batch reproduces band-limited fields (the quadrature is exact on
  Pi_N) to FP32 accuracy;
* FP64 plans take the FP64 contraction set by set: identical to hamls_fit's;
* the FP64 form at N = 1024 (the largest bandwidth; its FFT needs more than
  48 KB of shared memory) is exact on band-limited fields.

Tolerances: an FP32 contraction of hc = N/2 + 1 terms has relative error up
to about hc 2^-24 on a coefficient whose terms do not cancel; the product's
own error is 3 2^-20 per term (tests/test_gpu_tcgemm.py)."""
import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import SplitMix64, random_field_coeffs, synth_field, uniform_sphere

pytestmark = pytest.mark.gpu


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


def fp32_tol(N):
    return 2e-6 + (N // 2 + 1) * 2.0 ** -24 * 4


def grid_xyz(N):
    t, _ = O.gauss_legendre(N + 1)
    t = t.astype(float)
    L = 2 * N + 2
    phi = 2 * np.pi * np.arange(L) / L
    st = np.sqrt((1 - t) * (1 + t))
    return np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(), np.repeat(t, L)], axis=1)


@pytest.mark.parametrize("N,B,oracle_sets", [(16, 1, (0,)), (16, 8, (0, 3, 7)), (256, 17, (16,))] +
                         [(N, B, (0, B - 1) if B > 1 else (0,)) for N in (128, 512) for B in (1, 8, 64, 256)])
def test_batch_matches_single_sets_and_oracle(h, N, B, oracle_sets):
    g = O.quad_grid(N)
    f = SplitMix64(300 + N + B).normal(B * g.MQ).reshape(B, g.MQ)
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1, precision="mixed") as p:
        fb = dev(f)
        batch = p.quadrature_batch(fb)
        singles = [p.debug_quadrature(fb[b].contiguous()) for b in range(B)]
        p.sync(120000)
        got = [h.to_complex(batch[b]) for b in range(B)]
        one = [h.to_complex(c) for c in singles]
    tol = fp32_tol(N)
    for b in range(B):
        assert relerr(got[b], one[b]) < 2 * tol, f"set {b}"
    for b in oracle_sets:
        exp = O.quadrature(f[b], g)
        assert relerr(got[b], exp) < tol, f"set {b} vs oracle"
        assert relerr(one[b], exp) < tol, f"set {b}: single-set path vs oracle"
        # per coefficient, against the largest
        assert np.max(np.abs(got[b] - exp)) < 4 * tol * np.max(np.abs(exp))


@pytest.mark.parametrize("N", [128, 512])
def test_batch_exact_on_bandlimited(h, N):
    B = 4
    xyz = torch.tensor(grid_xyz(N), device="cuda")
    cs = [random_field_coeffs(70 + N + b, N) for b in range(B)]
    f = torch.stack([synth_field(c, xyz, torch) for c in cs]).contiguous()
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1, precision="mixed") as p:
        out = p.quadrature_batch(f)
        p.sync(120000)
    for b in range(B):
        assert relerr(h.to_complex(out[b]), O.pack_coeffs(np.tril(cs[b]), N)) < fp32_tol(N)


def test_batch_fp64_is_the_fp64_contraction(h):
    N, B = 64, 5
    g = O.quad_grid(N)
    f = dev(SplitMix64(9).normal(B * g.MQ).reshape(B, g.MQ))
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1) as p:
        batch = p.quadrature_batch(f)
        singles = [p.debug_quadrature(f[b].contiguous()) for b in range(B)]
        p.sync(60000)
    for b in range(B):
        assert torch.equal(batch[b], singles[b])


def test_fp64_quadrature_exact_at_n1024(h):
    N = 1024
    c = random_field_coeffs(1024, 400)                # degree 400 < N: exact
    f = synth_field(c, torch.tensor(grid_xyz(N), device="cuda"), torch).contiguous()
    x = dev(uniform_sphere(SplitMix64(1), 500))
    with h.Plan(x, N, 1) as p:
        got = h.to_complex(p.debug_quadrature(f))
        p.sync(120000)
    full = np.zeros((N + 1, N + 1), complex)
    full[:401, :401] = np.tril(c)
    assert relerr(got, O.pack_coeffs(full, N)) < 1e-12


def test_plans_share_their_tables(h):
    """Plans of the same bandwidth and form share one copy of the grid and
    quadrature tables; the copy lives until its last plan is destroyed."""
    x = dev(uniform_sphere(SplitMix64(1), 2000))
    free0 = torch.cuda.mem_get_info()[0]
    with h.Plan(x, 384, 1, precision="mixed") as a:
        a.sync(60000)
        free1 = torch.cuda.mem_get_info()[0]
        with h.Plan(x, 384, 1, precision="mixed") as b:
            b.sync(60000)
            free2 = torch.cuda.mem_get_info()[0]
            # the second plan does not hold another FP32 matrix (about 38 MB at N = 384)
            assert (free1 - free2) < (free0 - free1) - 30e6
            ca = a.fit(dev(np.ones(2000)))
            cb = b.fit(dev(np.ones(2000)))
            a.sync(60000)
            b.sync(60000)
            assert torch.equal(ca, cb)
