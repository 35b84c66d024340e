"""d_n at every auxiliary point (eq. adaptive_support_radius, Sec. 2.2) from
the plan's chained search, against the oracle's exact k-NN (a k-d tree for
candidates, every distance recomputed in FP64), on whole auxiliary grids:

* the track/hole workloads at N = 128 (66,564 points) and N = 512 (1,052,676
  points): every d_n of an FP64 plan equals the oracle's to rounding of the
  final arcsine (the squared chords are bit-exact), and so does a mixed
  plan's (its search is the same; checked here to FP32 accuracy, which is
  all the mixed form's support radius uses);
* edge cases: the smallest node set (M = n, every d_n is the farthest
  node), nodes confined to one small cap (almost every point lies far
  outside it), exact duplicate nodes, and an auxiliary grid whose size is
  not a multiple of the work chunk (32 points).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from hamls_synth import SplitMix64, uniform_sphere, workload

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


def aux_dn(h, x, N, K, wide=False, **kw):
    """d_n at the plan's auxiliary points. wide: the node set leaves supports
    of pi/2 or more (reported by hamls_sync, expected here)."""
    with h.Plan(dev(x), N, K, **kw) as p:
        xyz, dn = p.debug_aux()
        try:
            p.sync(300000)
        except h.HamlsError as e:
            if not (wide and e.code == 5):
                raise
        st = p.stats()
    return xyz.cpu().numpy(), dn.cpu().numpy(), st


def check(x, xyz, dn, n, mixed=False):
    c2 = O.NodeSet(x).knn_chord2(xyz, n)
    exp = np.asarray(O.geodesic_from_chord2(c2.astype(O.LD)), dtype=np.float64)
    if mixed:
        # the FP32 geodesic of the exact chord (FP32 arcsine: a few ulp)
        assert np.max(np.abs(dn / exp - 1)) < 1e-6
    else:
        assert np.max(np.abs(dn / exp - 1)) < 1e-14


@pytest.mark.parametrize("name", ["s2_n128_k3_m200k", "s2_n512_k3_m4m"])
def test_dn_whole_aux_grid_fp64(h, name):
    w = workload(name, xp=torch, device="cuda")
    n = O.Params().n_for(w.K)
    xyz, dn, st = aux_dn(h, w.nodes, w.N, w.K)
    assert st["aux_points"] == len(xyz)
    check(w.nodes, xyz, dn, n)


def test_dn_mixed(h):
    w = workload("s2_n128_k3_m200k", xp=torch, device="cuda")
    n = O.Params().n_for(w.K)
    xyz, dn, _ = aux_dn(h, w.nodes, w.N, w.K, precision="mixed")
    check(w.nodes, xyz, dn, n, mixed=True)


def test_dn_edge_cases(h):
    rng = SplitMix64(901)
    # M = n: every d_n is the distance to the farthest node
    x = uniform_sphere(rng, 40)
    xyz, dn, st = aux_dn(h, x, 4, 3, wide=True)
    check(x, xyz, dn, 40)
    # nodes confined to a 5 degree cap: nearly every point searches alone
    u = uniform_sphere(SplitMix64(902), 2_000_000)
    c = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    x = u[u @ c > math.cos(math.radians(5.0))][:3000]
    xyz, dn, st = aux_dn(h, x, 8, 2, wide=True)
    check(x, xyz, dn, 24)
    # exact duplicates (every node three times) and a ragged auxiliary grid
    base = uniform_sphere(SplitMix64(903), 4000)
    x = np.concatenate([base, base, base])
    xyz, dn, st = aux_dn(h, x, 16, 2, aux_points=1003)
    assert len(xyz) == 1003
    check(x, xyz, dn, 24)
