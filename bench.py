#!/usr/bin/env python
"""Benchmark of the HAMLS hot path on S^2: fits/s at N=512, K=3, M=4,000,000.

One step = one whole fit of one synthetic input: the node-dependent plan
stage (cell keys, counting sort by cell, runs, auxiliary k-NN, Shepard support radius,
work ordering; hamls_replan) and the value-dependent stage (value staging,
MLS with n(q) at all 526,338 grid nodes, ring FFT, Legendre quadrature;
hamls_fit). Inputs are resident in device memory when a step starts; a
256 MiB buffer is written between timed steps to flush the 126 MB L2. Each
step is timed with CUDA events on the plan's stream. The e2e leg passes
pinned host buffers through the same calls (copies in every step), two
plans on two streams taking alternate steps, timed on the host clock.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "S^2 N=512 M=4M fits/s & p99 latency, mixed vs FP64 GPU at equal L2 error"
WORKLOAD = "s2_n512_k3_m4m"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each
# stage's dominant kernel from an ncu capture (see profiles/); a stage whose
# kernel changed after that capture has no entry and reports null.
TRAFFIC = {
    # profiles/aux_knn_kernel_s2_n512_k3_m4m.md: 199.7 MB read + 21.7 MB written
    "aux_knn": 221_427_200,
    # profiles/mls_gather_kernel_s2_n512_k3_m4m.md (the MLS stage's main kernel): 80.6 + 49.2 MB
    "mls": 129_811_200,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=48, help="grid nodes the oracle evaluates for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frac", type=float, default=0.01, help="fraction of the grid nodes the oracle evaluates on "
                    "all host cores for the CPU baseline")
    ap.add_argument("--clocks-csv", default=None, help="also write the clock samples here ({rank} = the rank)")
    ap.add_argument("--quick", action="store_true", help="skip the FP64 form, e2e and CPU baseline (profiling)")
    ap.add_argument("--cache", default=None, help="directory to keep/reuse the generated workload (profiling runs)")
    ap.add_argument("--nodes", type=int, default=None, help="profiling runs: the benchmark workload generated with "
                    "this many nodes instead of its 4M (the line's config names the smaller workload)")
    ap.add_argument("--fp64-pivot", type=float, default=None, help="mixed form: squared FP32 pivot below which a "
                    "local solve is redone in FP64 (library default if omitted)")
    ap.add_argument("--batch-sets", type=int, default=64, help="value sets of the many-sets leg (0: skip)")
    ap.add_argument("--batch-fits", type=int, default=256, help="fits of the batched leg (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per arrival rate of the serving leg "
                    "(0: skip)")
    ap.add_argument("--serve-rates", default="40,80,160", help="arrival rates (requests/s) of the serving leg")
    return ap.parse_args()


# ------------------------------------------------------------------ oracle
class OracleBaseline:
    """Times the CPU oracle, as it stands, on a bounded sample of the workload
    and extrapolates to one whole fit. Every part is timed on its own (no part
    is inferred by subtracting one timing from another). Once per fit, timed
    once: the node tree and the grid, the auxiliary grid and its tree, the
    full quadrature step. Sampled, timed per estimate: d_n at seeded auxiliary
    points (all 2 M_Q per fit) and, at seeded grid nodes, the Shepard
    smoothing, the ball and the local problem (all M_Q per fit), with the
    supports the oracle's support_radius gives them (computed once, untimed)."""

    def __init__(self, w, sample: int, seed: int = 7):
        import oracle as O
        from hamls_synth import SplitMix64

        self.O, self.w = O, w
        self.MQ = (w.N + 1) * (2 * w.N + 2)
        self.M_aux = 2 * self.MQ
        self.p = O.Params()
        self.n = self.p.n_for(w.K)
        self.sel = np.unique((SplitMix64(seed).uniform(sample) * self.MQ).astype(np.int64))
        self.asel = np.unique((SplitMix64(seed + 1).uniform(8 * len(self.sel)) * self.M_aux).astype(np.int64))
        t0 = time.perf_counter()
        self.nodes = O.NodeSet(w.nodes)
        self.grid = O.quad_grid(w.N)
        self.t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.aux = O.fibonacci_points(self.M_aux)
        self.aux_tree = O.cKDTree(self.aux)
        self.t_aux = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.quadrature(np.zeros(self.MQ), self.grid)
        self.t_quad = time.perf_counter() - t0
        self.sup = O.support_radius(self.nodes, self.grid.xyz, w.K, self.p, subset=self.sel)

    def estimate_all_cores(self, frac=0.01, pool=None) -> dict:
        """The same estimate with the per-node work on all host cores: a
        seeded sample of frac of the grid nodes with twice as many auxiliary
        points (a fit has 2 M_Q of them per M_Q grid nodes), so the sample's
        parallel wall time scales to the whole fit by M_Q / sample."""
        r = oracle_all_cores(self.w, frac, pool=pool)
        per_fit = self.t_build + self.t_aux + r["wall_s"] * self.MQ / r["grid_nodes"] + self.t_quad
        one = self.estimate()
        return {"value": 1.0 / per_fit, "unit": "fits/s", "cores": r["cores"], "kind": "oracle",
                "value_1core": one["value"],
                "sample": (f"all {r['cores']} host cores (nproc): the per-node work of {r['grid_nodes']} seeded grid "
                           f"nodes ({100.0 * r['grid_nodes'] / self.MQ:.2f} % of {self.MQ}) and {r['aux_points']} "
                           f"auxiliary points in {r['wall_s']:.2f} s of wall clock from a common start, scaled to the "
                           f"whole fit; the tree, grid and quadrature parts once per fit ({self.t_build:.2f} + "
                           f"{self.t_aux:.2f} + {self.t_quad:.2f} s, one thread). One core: {one['value']:.6f} fits/s "
                           f"({one['sample']})")}

    def estimate(self) -> dict:
        O, w, sel = self.O, self.w, self.sel
        t0 = time.perf_counter()
        O.geodesic_from_chord2(self.nodes.knn_chord2(self.aux[self.asel], self.n).astype(O.LD))
        t_knn = (time.perf_counter() - t0) / len(self.asel)
        rho = self.p.aux_radius * math.sqrt(4.0 * math.pi / self.M_aux)
        t0 = time.perf_counter()
        O.shepard(self.grid.xyz[sel], self.aux, self.aux_tree, self.sup.dn_aux, rho)
        for jj, j in enumerate(sel):
            idx = self.nodes.ball(self.grid.xyz[j], self.sup.rho2[jj])
            O.mls_at(self.grid.xyz_ld[j], w.nodes[idx], w.values[idx], self.sup.delta[jj], w.K, self.p)
        t_node = (time.perf_counter() - t0) / len(sel)
        per_fit = self.t_build + self.t_aux + t_knn * self.M_aux + t_node * self.MQ + self.t_quad
        return {"value": 1.0 / per_fit, "unit": "fits/s", "cores": 1, "kind": "oracle",
                "t_knn_s": t_knn, "t_node_s": t_node,
                "sample": (f"k-d tree over all {w.M} nodes and the grid ({self.t_build:.2f} s) and the auxiliary "
                           f"grid ({self.t_aux:.2f} s), once; d_n at {len(self.asel)} seeded auxiliary points "
                           f"({t_knn * 1e3:.3f} ms each, scaled to all {self.M_aux}); Shepard smoothing, ball and "
                           f"local problem at {len(sel)} seeded grid nodes ({t_node * 1e3:.3f} ms each, scaled to "
                           f"all {self.MQ}); full quadrature step ({self.t_quad:.2f} s); numpy/scipy, one host "
                           f"thread")}


# ------------------------------------------------------- all host cores
_W = {}


def _oracle_worker_init(nodes, values, N, K):
    """A spawned worker's copy of the oracle's node tree and grids."""
    import oracle as O
    _W["O"] = O
    _W["nodes"] = O.NodeSet(nodes)
    _W["values"] = values
    _W["grid"] = O.quad_grid(N)
    _W["K"] = K
    _W["p"] = O.Params()
    MQ = (N + 1) * (2 * N + 2)
    _W["aux"] = O.fibonacci_points(2 * MQ)
    _W["aux_tree"] = O.cKDTree(_W["aux"])


def _oracle_worker_task(sel, asel, barrier):
    """The sampled grid nodes sel (support radius set up untimed) and
    auxiliary points asel of this worker, timed between wall-clock stamps
    that start once every worker is ready."""
    O, nodes, grid, K, p = _W["O"], _W["nodes"], _W["grid"], _W["K"], _W["p"]
    sup = O.support_radius(nodes, grid.xyz, K, p, subset=sel)
    n = p.n_for(K)
    rho = p.aux_radius * math.sqrt(4.0 * math.pi / len(_W["aux"]))
    barrier.wait()
    t0 = time.time()
    O.geodesic_from_chord2(nodes.knn_chord2(_W["aux"][asel], n).astype(O.LD))
    O.shepard(grid.xyz[sel], _W["aux"], _W["aux_tree"], sup.dn_aux, rho)
    for jj, j in enumerate(sel):
        idx = nodes.ball(grid.xyz[j], sup.rho2[jj])
        O.mls_at(grid.xyz_ld[j], nodes.x[idx], _W["values"][idx], sup.delta[jj], K, p)
    return t0, time.time()


class AllCoresPool:
    """Spawned worker processes, one per host core, each holding the oracle's
    node tree and grids for one workload; reused for every timed sample."""

    def __init__(self, w, workers=None):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor

        self.w = w
        self.cores = workers or len(os.sched_getaffinity(0))
        ctx = mp.get_context("spawn")
        self.man = ctx.Manager()
        self.barrier = self.man.Barrier(self.cores)
        self.ex = ProcessPoolExecutor(max_workers=self.cores, mp_context=ctx, initializer=_oracle_worker_init,
                                      initargs=(w.nodes, w.values, w.N, w.K))

    def run(self, frac=0.01, seed=11):
        """The oracle's per-node work (d_n at auxiliary points, the Shepard
        smoothing, ball and local problem at grid nodes) on a seeded sample of
        frac of the grid nodes and twice as many auxiliary points, split over
        the workers, wall-clock timed from a common start."""
        from hamls_synth import SplitMix64

        w, cores = self.w, self.cores
        MQ = (w.N + 1) * (2 * w.N + 2)
        n_sel = max(cores, int(frac * MQ))
        sel = np.unique((SplitMix64(seed).uniform(n_sel) * MQ).astype(np.int64))
        asel = np.unique((SplitMix64(seed + 1).uniform(2 * len(sel)) * 2 * MQ).astype(np.int64))
        futs = [self.ex.submit(_oracle_worker_task, sel[i::cores], asel[i::cores], self.barrier)
                for i in range(cores)]
        stamps = [f.result() for f in futs]
        wall = max(t1 for _, t1 in stamps) - min(t0 for t0, _ in stamps)
        return {"cores": cores, "grid_nodes": len(sel), "aux_points": len(asel), "wall_s": wall}

    def close(self):
        self.ex.shutdown()
        self.man.shutdown()


def oracle_all_cores(w, frac=0.01, seed=11, workers=None, pool=None):
    """AllCoresPool.run on a given pool, or on a pool made for this call."""
    if pool is not None:
        return pool.run(frac, seed)
    pool = AllCoresPool(w, workers)
    try:
        return pool.run(frac, seed)
    finally:
        pool.close()


def run_reference(args):
    from hamls_synth import workload

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    # input generation (a random field of degree 200 at 4M nodes) is not part
    # of the timed oracle; on the GPU it takes seconds instead of minutes
    w = workload(WORKLOAD, xp=torch, device="cuda" if torch.cuda.is_available() else None)
    ob = OracleBaseline(w, max(8, args.cpu_sample // 4))
    # each step: the per-node work of the main line's sample (args.cpu_frac of
    # the grid nodes) on all host cores, the workers spawned once
    pool = AllCoresPool(w)
    try:
        steps = [ob.estimate_all_cores(args.cpu_frac, pool=pool) for _ in range(args.warmup + args.steps)]
    finally:
        pool.close()
    timed = steps[args.warmup:]
    v = float(np.mean([s["value"] for s in timed]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": w.N, "K": w.K, "M": w.M},
            "cpu_baseline": {"value": v, "unit": "fits/s", "cores": timed[-1]["cores"], "kind": "oracle",
                             "value_1core": float(np.mean([s["value_1core"] for s in timed])),
                             "sample": timed[-1]["sample"]},
            "e2e": {"value": v, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- replicas
def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself on one process)."""
    if not dist:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_fits_per_s(steps_per_rank: int, local_seconds: float, world: int, dist, device) -> float:
    """Whole-job throughput of independent replicas: every rank fits its own
    steps_per_rank inputs; the job ends with the slowest rank."""
    return world * steps_per_rank / max_over_ranks(local_seconds, dist, device)


# -------------------------------------------------------------------- clocks
class Clocks:
    """SM clock and throttle reasons sampled during the timed region: NVML
    polled every 10 ms from a thread (nvidia-smi at 50 ms if NVML is
    unavailable); with a path, the samples are also written there as CSV."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, index: int, path=None):
        self.index = index
        self.p = None
        self.thread = None
        self.rows = []
        self.nvml_error = None
        self.path = path.replace("{rank}", str(index)) if path else None

    def _poll(self, nv, h):
        while not self.stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
                rs = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                pw = nv.nvmlDeviceGetPowerUsage(h) / 1000.0
                self.rows.append((sm, mx, rs, pw))
            except Exception:
                pass
            self.stop.wait(0.01)

    def __enter__(self):
        import threading
        if self.path and os.path.dirname(self.path):
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            import pynvml as nv
            nv.nvmlInit()
            h = nv.nvmlDeviceGetHandleByIndex(self.index)
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(nv, h), daemon=True)
            self.thread.start()
            return self
        except Exception as e:
            self.thread = None
            self.nvml_error = f"{type(e).__name__}: {e}"[:120]
        import tempfile
        self.smi_path = self.path or os.path.join(tempfile.gettempdir(), f"hamls_clocks_{os.getpid()}_{self.index}.csv")
        try:
            self.fh = open(self.smi_path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv",
                                       "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
            if self.path:
                with open(self.path, "w") as fh:
                    fh.write("sm_mhz,max_sm_mhz,event_reasons,power_w\n")
                    for r in self.rows:
                        fh.write(f"{r[0]},{r[1]},{r[2]:#x},{r[3]:.1f}\n")
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.fh.close()

    def summary(self):
        if self.thread is not None:
            if not self.rows:
                return None
            reasons = sorted({n for r in self.rows for n, bit in self.REASONS if r[2] & bit})
            return {"sm_mhz": float(np.median([r[0] for r in self.rows])), "sm_max_mhz": max(r[1] for r in self.rows),
                    "reasons": reasons, "samples": len(self.rows), "source": "nvml, 10 ms"}
        if self.p is None or not os.path.exists(self.smi_path):
            return None
        rows = [l.strip().split(", ") for l in open(self.smi_path) if l.strip() and not l.startswith("index")]
        if not rows:
            return None
        mhz = [float(r[1].split()[0]) for r in rows if len(r) > 2]
        mx = [float(r[2].split()[0]) for r in rows if len(r) > 2]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": max(mx), "reasons": reasons, "samples": len(rows),
                "source": "nvidia-smi, 50 ms", "nvml_error": self.nvml_error}



# --------------------------------------------------------------------- ours
def workload_name(nodes):
    """The benchmark workload's name, or that of its reduced form (--nodes)."""
    if not nodes:
        return WORKLOAD
    tag = f"m{nodes // 1_000_000}m" if nodes % 1_000_000 == 0 else f"m{nodes // 1000}k"
    return WORKLOAD.rsplit("_", 1)[0] + "_" + tag


def load_workload(cache, rank, torch, dev, nodes=None):
    """The seeded benchmark workload (with nodes: generated with that many
    nodes, for profiling runs); with a cache directory, generated once and
    reused."""
    from hamls_synth import workload
    from hamls_synth.gen import Workload

    name = workload_name(nodes)
    path = os.path.join(cache, f"{name}_{rank}.npz") if cache else None
    if path and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return Workload(name, int(z["N"]), int(z["K"]), int(z["M"]), z["nodes"], z["values"], z["truth"], {})
    w = workload(WORKLOAD, fit_index=rank, xp=torch, device=dev, M=nodes)
    if path:
        os.makedirs(cache, exist_ok=True)
        np.savez(path, N=w.N, K=w.K, M=w.M, nodes=w.nodes, values=w.values, truth=w.truth)
    return w


def many_sets_leg(h, plan, w, y, flush, stream, B, steps, warmup, peaks, truth_err):
    """Refits of B value sets at the plan's (prepared) nodes with
    hamls_refit_batch, and step 3 of B grids with hamls_quadrature_batch; the
    tensor-core contraction's own roofline from its stage events."""
    import torch

    dev = y.device
    N = w.N
    ncoef = (N + 1) * (N + 2) // 2
    MQ = (N + 1) * (2 * N + 2)
    hc = N // 2 + 1
    hcp = (hc + 7) // 8 * 8
    scales = torch.linspace(1.0, 2.0, B, dtype=torch.float64, device=dev)
    Y = (scales[:, None] * y[None, :]).contiguous()         # set 0: the workload's values
    out = torch.empty((B, ncoef, 2), dtype=torch.float64, device=dev)

    def timed(fn):
        plan.set_timing(True)
        ts, st = [], []
        for i in range(warmup + steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ts.append(e0.elapsed_time(e1))
                st.append(plan.stage_times())
        plan.set_timing(False)
        plan.sync(600000)
        return np.array(ts), {k: float(np.mean([d[k] for d in st])) for k in st[0]}

    ts, st = timed(lambda: plan.refit_batch(Y, out=out))
    c0 = h.to_complex(out[0])
    lin = float(np.linalg.norm(h.to_complex(out[B - 1]) - 2.0 * c0) / np.linalg.norm(2.0 * c0))
    refit = {"sets": B, "value": B * len(ts) / (float(ts.sum()) / 1000.0), "unit": "fits/s",
             "ms_per_call": float(ts.mean()), "l2_error_set0": truth_err(c0),
             "linearity_rel_err": lin, "stage_ms": {k: round(v, 4) for k, v in st.items() if v >= 0}}
    # step 3 alone for B grids (the last refit's grid values, scaled)
    g = plan.debug_grid()["f"]
    F = (scales[:, None] * g[None, :]).contiguous()
    ts, st = timed(lambda: plan.quadrature_batch(F, out=out))
    t_tc = st["legendre"] / 1000.0
    # executed tensor work: 3 products per term, K padded to 32, value-set parts
    # padded to 128 rows, degrees of each (order, parity) block padded to 32
    rows_pad = 0
    for m in range(N + 1):
        for cnt in ((N - m) // 2 + 1, (N - m + 1) // 2):
            rows_pad += -(-cnt // 32) * 32 if cnt else 0
    kp = -(-hc // 32) * 32
    mt = -(-2 * B // 128) * 128
    flops_exec = 3 * 2 * rows_pad * kp * mt
    flops_alg = 2 * ncoef * hc * 2 * B
    # algorithmic bytes: the FP32 matrix and folded spectra once each (the
    # kernel splits them for 3xTF32 in shared memory), the coefficients out
    bytes_alg = ncoef * hcp * 4 + (2 * (N + 1)) * (2 * B) * hcp * 4 + B * ncoef * 16
    tf32_peak = float(peaks.get("bf16_tflops", 1800.0)) * 0.5
    quad = {"sets": B, "value": B * len(ts) / (float(ts.sum()) / 1000.0), "unit": "grids/s",
            "ms_per_call": float(ts.mean()), "spectra_ms": st["fft"], "tensor_ms": st["legendre"],
            "roofline": {"bound": "hbm", "kernel": "tc_gemm_kernel<EpiLegendre> (tcgen05 kind::tf32, 3xTF32)",
                         "achieved": bytes_alg / t_tc / 1e9, "peak": float(peaks.get("hbm_gbs", 6400.0)),
                         "unit": "GB/s", "frac": bytes_alg / t_tc / 1e9 / float(peaks.get("hbm_gbs", 6400.0)),
                         "traffic": None, "algorithmic_bytes_per_launch": int(bytes_alg)},
            "tensor": {"achieved_tflops_executed": flops_exec / t_tc / 1e12,
                       "achieved_tflops_fp32_equivalent": flops_alg / t_tc / 1e12,
                       "peak_tf32_tflops": tf32_peak, "peak_source": "measured bf16 x 0.5 (nominal tf32/bf16)",
                       "frac_executed": flops_exec / t_tc / 1e12 / tf32_peak}}
    del Y, F
    return {"refit_batch": refit, "quadrature_batch": quad}


def batched_leg(h, dev, n_fits, precision="mixed"):
    """Config 4: n_fits independent fits (N over {32, 64, 128, 256}, M
    log-uniform in [1e4, 1e6], K over {2, 3}, 0-3 holes) replanned and fitted
    from reserved plans, the whole batch captured in one CUDA graph and
    replayed; the stream concurrency is chosen by the slot autotuner. Node sets
    are seeded; values come from a degree-32 field (their content does not
    change the work)."""
    import torch

    from hamls_synth import batch_specs, fit_workload
    from paper_2609_39200_b300.batch import PlanPool, SlotTuner, run_batch

    specs = batch_specs(n_fits)
    t0 = time.perf_counter()
    inputs = {}
    for s in specs:
        wl = fit_workload(s, xp=torch, device=dev, L_field=32)
        inputs[s.index] = (torch.tensor(wl.nodes, device=dev), torch.tensor(wl.values, device=dev))
    gen_s = time.perf_counter() - t0

    def load(s):
        return inputs[s.index]

    pool = PlanPool(device=dev, min_capacity=1 << 14)
    tuner = SlotTuner((2, 4, 8))
    slots = tuner.choose(specs, load, pool, precision=precision, device=dev)
    reps = 3
    r = run_batch(specs, load, pool, n_slots=slots, precision=precision, device=dev, graph=True, replays=reps)
    bad = [{"index": s.index, "N": s.N, "K": s.K, "M": s.M, "holes": len(s.holes_deg), "status": int(x)}
           for s, x in zip(specs, r.status) if x]
    res = {"fits": n_fits, "value": n_fits * reps / r.seconds, "unit": "fits/s", "ms_per_batch": 1000 * r.seconds / reps,
           "slots": slots, "autotune_s_per_batch": {str(k): round(v, 4) for k, v in
                                                     tuner.trials[tuner.shape(specs, pool.min_capacity)].items()},
           "graph": r.graph, "plans": pool.created, "plan_bytes": pool.used_bytes, "failed_fits": len(bad),
           "failures": bad[:16],
           "grid_nodes": int(sum((s.N + 1) * (2 * s.N + 2) for s in specs)), "input_generation_s": round(gen_s, 1),
           "note": "one CUDA graph replay runs every replan, fit and status copy of the batch"}
    res["grid_nodes_per_s"] = res["grid_nodes"] * res["value"] / n_fits
    pool.close()
    del inputs
    return res


def serving_leg(h, dev, n_req, rates, precision="mixed"):
    """Config 5: Poisson arrivals of fit requests (N over {64..1024} with
    probabilities {.3, .3, .2, .15, .05}, M log-uniform in [5e4, 1.6e7], K = 3,
    three holes) served by continuous batching over 4 slots, plans kept on the
    device and admitted by their memory footprint. A request's nodes are the
    first M of one seeded 16M-node track/hole set (the same distribution), its
    values a degree-32 field. The trace is served once to create the plans,
    then at each rate; latency runs from arrival to the end of the fit."""
    import torch

    from hamls_synth import random_field_coeffs, serving_trace, synth_field, track_hole_nodes
    from paper_2609_39200_b300.batch import PlanPool, serve

    t0 = time.perf_counter()
    Mmax = 16_000_000
    xn = track_hole_nodes(0x48414D4C53 ^ (5 << 32), Mmax)[0]
    X = torch.tensor(xn, device=dev)
    Yv = synth_field(random_field_coeffs(55, 32), X, torch).contiguous()
    gen_s = time.perf_counter() - t0

    def load(r):
        return X[:r.M], Yv[:r.M]

    free, _ = torch.cuda.mem_get_info(dev)
    pool = PlanPool(device=dev, budget_bytes=int(0.6 * free), min_capacity=1 << 16)
    out = {"requests_per_rate": n_req, "slots": 4, "input_generation_s": round(gen_s, 1), "rates": {}}
    warm = serving_trace(1e6, n_req)
    serve(warm, load, pool, n_slots=4, precision=precision, device=dev, keep_outputs=False)
    for lam in rates:
        tr = serving_trace(lam, n_req)
        r = serve(tr, load, pool, n_slots=4, precision=precision, device=dev, keep_outputs=False)
        lat = r.latency_s * 1000.0
        out["rates"][str(lam)] = {"fits_per_s": n_req / r.makespan_s, "p50_ms": float(np.percentile(lat, 50)),
                                  "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                                  "queue_p99_ms": float(np.percentile(r.queue_s * 1000.0, 99)),
                                  "failed": int(sum(1 for x in r.status if x))}
    out["plans"] = pool.created
    out["evicted"] = pool.evicted
    out["plan_bytes"] = pool.used_bytes
    pool.close()
    del X, Yv
    return out


def run_ours(args):
    import torch

    import paper_2609_39200_b300 as h
    from hamls_synth import workload
    from hamls_synth.gen import coeff_norm2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    h.lib()

    # CPU baseline first (rank 0, N=1), before any GPU work
    w = load_workload(args.cache, rank, torch, dev, args.nodes)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        try:
            cpu = OracleBaseline(w, args.cpu_sample).estimate_all_cores(args.cpu_frac)
        except Exception as e:                  # reported, never fatal to the headline line
            cpu = {"value": None, "unit": "fits/s", "cores": 1, "kind": "oracle", "error": f"{type(e).__name__}: {e}"}

    x = torch.tensor(w.nodes, device=dev)
    y = torch.tensor(w.values, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)    # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)
    ncoef = (w.N + 1) * (w.N + 2) // 2

    def timed_steps(plan, nodes, values, out, steps, warmup, collect=False):
        plan.set_timing(True)
        times, mls, stage_sum = [], [], {}
        for i in range(warmup + steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if i == warmup:
                plan.launch_count(reset=True)
            e0.record(stream)
            plan.replan(nodes)
            plan.fit(values, out=out)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                times.append(e0.elapsed_time(e1))
                st = plan.stage_times()
                mls.append(st["mls"])
                for k, v in st.items():
                    if v >= 0:                  # stages the step did not run report -1
                        stage_sum[k] = stage_sum.get(k, 0.0) + v
        launches = plan.launch_count()
        plan.sync(600000)
        return np.array(times), np.array(mls), {k: v / steps for k, v in stage_sum.items()}, launches

    # ---- mixed form (the headline)
    out = torch.empty((ncoef, 2), dtype=torch.float64, device=dev)
    kw = {} if args.fp64_pivot is None else {"fp64_pivot": args.fp64_pivot}
    plan = h.Plan(x, w.N, w.K, precision="mixed", **kw)
    plan.sync(600000)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local, args.clocks_csv) as clk:
        times, mls, stages, launches = timed_steps(plan, x, y, out, args.steps, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stats = plan.stats()
    c_mixed = h.to_complex(out)
    value = aggregate_fits_per_s(args.steps, float(times.sum()) / 1000.0, world, dist, dev)
    total_ms = 1000.0 * world * args.steps / value           # the slowest rank's timed region

    # ---- values-only refits at the same nodes: hamls_refit_prepare once
    # (untimed), then hamls_refit per step (sparse operator + step 3)
    refit, c_refit = None, None
    if not args.quick:
        plan.set_timing(False)
        tp = time.perf_counter()
        plan.refit_prepare()
        plan.sync(600000)
        prep_s = time.perf_counter() - tp
        nnz = plan.stats()["sum_n"]
        plan.set_timing(True)
        # the steps are enqueued back to back (each after its L2 flush, between
        # its own pair of events) and synchronised once: a refit is short
        # (~0.4 ms), so a host synchronisation per step would put the host's
        # launch latency inside every timed interval
        pairs = []
        for i in range(args.warmup + args.steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.refit(y, out=out)
            e1.record(stream)
            if i >= args.warmup:
                pairs.append((e0, e1))
        torch.cuda.synchronize()
        rts = np.array([e0.elapsed_time(e1) for e0, e1 in pairs])
        a_ms = float(plan.stage_times()["mls"])          # the last step's operator product
        plan.set_timing(False)
        plan.sync(600000)
        c_refit = h.to_complex(out)
        # operator entry (FP32 value + column) and a 4 B gathered value each, per grid node the row
        # start and the FP64 result, per node the FP64 value read and its FP32 copy written and read
        op_bytes = nnz * (4 + 4 + 4) + (w.N + 1) * (2 * w.N + 2) * (4 + 8) + w.M * (8 + 4 + 4)
        refit = {"value": world * len(rts) / (float(rts.sum()) / 1000.0), "unit": "fits/s",
                 "ms_per_step": float(rts.mean()), "prepare_s": prep_s, "operator_entries": int(nnz),
                 "roofline": {"bound": "hbm", "kernel": "op_apply_kernel<float> (+ to_float_kernel)",
                              "achieved": op_bytes / (a_ms / 1000.0) / 1e9, "peak": None, "unit": "GB/s",
                              "frac": None, "traffic": TRAFFIC.get("refit"),
                              "algorithmic_bytes_per_launch": int(op_bytes), "ms_per_launch": a_ms},
                 "note": "new values at the plan's nodes: the stored operator, then ring FFT and Legendre"}

    # ---- many value sets at the plan's nodes (tensor-core step 3); the
    # batched form (config 4) and the serving trace (config 5)
    def truth_err_fn(c):
        import oracle as O   # packing helpers only
        N = w.N
        Lt = w.truth.shape[0] - 1
        t = np.zeros((max(N, Lt) + 1,) * 2, complex)
        t[:Lt + 1, :Lt + 1] = np.tril(w.truth)
        t[:N + 1, :N + 1] -= O.unpack_coeffs(c, N)
        d2 = np.sum(np.abs(t[:, 0]) ** 2) + 2 * np.sum(np.abs(t[:, 1:]) ** 2)
        return float(math.sqrt(d2 / coeff_norm2(w.truth)))

    peaks0 = {}
    try:
        peaks0 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    many = batched = serving = None
    if not args.quick and refit is not None and args.batch_sets > 0:
        try:
            many = many_sets_leg(h, plan, w, y, flush, stream, args.batch_sets, max(3, args.steps // 10), 2, peaks0,
                                 truth_err_fn)
        except Exception as e:                  # reported, never fatal to the headline line
            many = {"error": f"{type(e).__name__}: {e}"[:300]}

    # ---- Voronoi areas of the nodes (the weights v_i of Sec. 2.2, computed once
    # per node set): CUDA events around hamls_voronoi_areas, L2 flushed between calls
    def voronoi_leg(pl, reps):
        try:
            pl.set_timing(False)
            area = torch.empty(w.M, dtype=torch.float64, device=dev)
            for _ in range(2):
                pl.voronoi_areas(out=area)
            pl.sync(600000)
            ts = []
            for i in range(reps):
                flush.fill_(float(i))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.voronoi_areas(out=area)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            pl.sync(600000)
            ms = float(np.mean(ts))
            return {"ms": ms, "cells_per_s": w.M / (ms / 1000.0), "reps": reps,
                    "area_sum_minus_4pi": float(area.sum()) - 4.0 * np.pi,
                    "kernels": "vor_split_kernel + voronoi_kernel"}
        except Exception as e:                  # reported, never fatal to the headline line
            return {"error": f"{type(e).__name__}: {e}"}

    voronoi = None
    if not args.quick:
        voronoi = {"mixed": voronoi_leg(plan, 10)}

    # ---- the forward transform F (hamls_forward) of the fit's coefficients at
    # the 4M nodes: CUDA events, L2 flushed between calls. FP32 ALU-bound: per
    # node the (N+1)(N+2)/2 recurrence terms of 8 FP32 flops each (the
    # three-term step: two products, a difference and the factor; two FMAs
    # into the order's sum); peak = 148 SMs x 128 FP32 lanes x 2 flops x the
    # SM clock seen during the run.
    def forward_leg(pl, coeffs, reps):
        try:
            pl.set_timing(False)
            vals = torch.empty(w.M, dtype=torch.float64, device=dev)
            for _ in range(2):
                pl.forward(coeffs, out=vals)
            pl.sync(600000)
            ts = []
            for i in range(reps):
                flush.fill_(float(i))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pl.forward(coeffs, out=vals)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            pl.sync(600000)
            ms = float(np.mean(ts))
            terms = (w.N + 1) * (w.N + 2) // 2
            flops = 8.0 * terms * w.M
            res = vals.cpu().numpy() - (w.values if isinstance(w.values, np.ndarray) else w.values.cpu().numpy())
            return {"ms": ms, "points_per_s": w.M / (ms / 1000.0), "reps": reps,
                    "kernel": "forward_kernel<float> (+ coefficient and factor conversion)",
                    "roofline": {"bound": "alu", "achieved": flops / (ms / 1000.0) / 1e12, "unit": "TFLOP/s",
                                 "flops_per_point": 8.0 * terms, "peak_note": "148 SMs x 128 FP32 lanes x 2 x SM clock"},
                    "residual_rms_over_data_rms": float(np.sqrt(np.mean(res ** 2)) /
                                                        np.sqrt(np.mean(np.asarray(w.values) ** 2)))}
        except Exception as e:                  # reported, never fatal to the headline line
            return {"error": f"{type(e).__name__}: {e}"}

    forward = None
    if not args.quick:
        forward = {"mixed": forward_leg(plan, out, 5)}

    # ---- e2e: host buffers through the C ABI, copies inside the timed region.
    # Two plans on two streams take the steps in turn, as a caller with a
    # stream of fits would: one step's host-to-device copy overlaps the other
    # plan's kernels. Every step copies its inputs in and its result out.
    e2e = None
    if not args.quick:
        xh = torch.tensor(w.nodes).pin_memory()
        yh = torch.tensor(w.values).pin_memory()
        oh = [torch.empty((ncoef, 2), dtype=torch.float64).pin_memory() for _ in range(2)]
        plan.set_timing(False)
        plan_b = h.Plan(x, w.N, w.K, precision="mixed", **kw)
        plan_b.sync(600000)
        plans = (plan, plan_b)
        streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))

        def e2e_step(i):
            p, st = plans[i % 2], streams[i % 2]
            p.replan(xh, stream=st)
            p.fit(yh, out=oh[i % 2], stream=st)

        for i in range(max(4, args.warmup)):
            e2e_step(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        n_e2e = max(4, args.steps // 2)
        t0 = time.perf_counter()
        for i in range(n_e2e):
            e2e_step(i)
        for st in streams:
            st.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist, dev)
        for p in plans:
            p.sync(600000)
        plan_b.close()
        e2e = {"value": world * n_e2e / el, "unit": "fits/s",
               "h2d_bytes_per_step": int(xh.numel() * 8 + yh.numel() * 8), "d2h_bytes_per_step": int(oh[0].numel() * 8),
               "ms_per_step": 1000.0 * el / n_e2e, "steps": n_e2e,
               "timing": "host wall clock over all steps, both streams synchronised at the end",
               "pipelining": "two plans on two streams take alternate steps"}
    plan.close()

    if not args.quick and args.batch_fits > 0 and world == 1:
        try:
            batched = batched_leg(h, dev, args.batch_fits)
        except Exception as e:
            batched = {"error": f"{type(e).__name__}: {e}"[:300]}
    if not args.quick and args.serve_requests > 0 and world == 1:
        try:
            serving = serving_leg(h, dev, args.serve_requests, [float(r) for r in args.serve_rates.split(",")])
        except Exception as e:
            serving = {"error": f"{type(e).__name__}: {e}"[:300]}

    # ---- FP64 form (the comparison)
    fp64 = None
    c64 = None
    if not args.quick and args.fp64_steps > 0:
        out64 = torch.empty((ncoef, 2), dtype=torch.float64, device=dev)
        p64 = h.Plan(x, w.N, w.K, precision="fp64")
        t64, m64, st64, _ = timed_steps(p64, x, y, out64, args.fp64_steps, 1)
        c64 = h.to_complex(out64)
        fp64 = {"value": world * len(t64) / (float(t64.sum()) / 1000.0), "unit": "fits/s",
                "ms_per_step": float(t64.mean()), "mls_ms": float(m64.mean()),
                "stage_ms": {k: round(v, 4) for k, v in st64.items()}}
        if voronoi is not None:
            voronoi["fp64"] = voronoi_leg(p64, 5)
        p64.close()

    # ---- accuracy against the known truth (eq. relative_error_S2, by Parseval)
    def truth_err(c):
        import oracle as O   # packing helpers only
        N = w.N
        Lt = w.truth.shape[0] - 1
        t = np.zeros((max(N, Lt) + 1,) * 2, complex)
        t[:Lt + 1, :Lt + 1] = np.tril(w.truth)
        t[:N + 1, :N + 1] -= O.unpack_coeffs(c, N)
        d2 = np.sum(np.abs(t[:, 0]) ** 2) + 2 * np.sum(np.abs(t[:, 1:]) ** 2)
        return float(math.sqrt(d2 / coeff_norm2(w.truth)))

    l2 = {"mixed": truth_err(c_mixed)}
    if c_refit is not None:
        l2["mixed_refit"] = truth_err(c_refit)
    if c64 is not None:
        l2["fp64"] = truth_err(c64)
        l2["ratio_mixed_over_fp64"] = l2["mixed"] / l2["fp64"]
        l2["mixed_vs_fp64_coeff_rel"] = float(np.linalg.norm(c_mixed - c64) / np.linalg.norm(c64))

    # ---- roofline: per stage, algorithmic bytes over the stage's CUDA-event time;
    # the dominant stage's figure is the headline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    MQ = stats["grid_nodes"]
    m_dim = (w.K + 1) * (w.K + 2) // 2
    n_nb = 4 * m_dim
    hc = (w.N + 2) // 2
    B_cells = 16
    while B_cells * B_cells * 4 < w.M and B_cells < 4096:
        B_cells *= 2
    alg = {
        # per node: keys pass xyz in (24 B), key and arrival rank out (8 B); scatter key and rank in
        # (8 B), position out (4 B); ordering pass position and key in (8 B), xyz in (24 B), order and
        # sorted key out (8 B), FP64 + FP32 copies out (40 B). Per cell: count cleared, scanned in
        # place (12 B)
        "cells": ("cell_count_kernel + cell_scatter_kernel + cell_order_kernel (+ scan of the counts)",
                  w.M * (24 + 8 + 8 + 4 + 8 + 24 + 8 + 40) + 12 * (B_cells * 2 * B_cells + 1)),
        # n nearest FP32 node records (x, y, z, y) per auxiliary point + its FP64 coordinates + d_n out
        "aux_knn": ("aux_knn_kernel", stats["aux_points"] * (16 * n_nb + 24 + 8)),
        # gathered FP32 node records + per grid node delta, rho2 (in), f (out), order key
        "mls": ("mls_gather_kernel + mls_solve_kernel + reg_kernel + redo_kernel", stats["sum_n"] * 16 + MQ * (8 + 8 + 8 + 4)),
        # grid values in, ring spectra out
        "fft": ("ring_fft_kernel", MQ * 8 + (w.N + 1) ** 2 * 8),
        # the folded FP32 Legendre matrix + spectra in, coefficients out
        "legendre": ("legendre_kernel", (w.N + 1) * (w.N + 2) // 2 * hc * 4 + (w.N + 1) ** 2 * 8
                     + (w.N + 1) * (w.N + 2) * 8),
    }
    stage_roof = {}
    for st_name, (kname, nbytes) in alg.items():
        ms = stages.get(st_name, 0.0)
        if ms > 0:
            ach = nbytes / (ms / 1000.0) / 1e9
            stage_roof[st_name] = {"kernel": kname, "ms": round(ms, 4), "algorithmic_bytes": int(nbytes),
                                   "achieved_gbs": round(ach, 1), "frac": round(ach / hbm_peak, 4),
                                   "traffic": TRAFFIC.get(st_name)}
    if refit is not None:
        refit["roofline"]["peak"] = hbm_peak
        refit["roofline"]["frac"] = refit["roofline"]["achieved"] / hbm_peak
    # the MLS stage as a whole (auxiliary k-NN, Shepard support radius, work
    # order, gather + local solves): its stages' bytes over their summed time.
    # Shepard: about pi aux_radius^2 = 28 auxiliary members per grid node
    # (column, weight, d_n: 12 B each in the mixed form) + 41 B of per-node
    # inputs and outputs; work order: a key/value sort of M_Q entries (16 B)
    shep_nnz = MQ * math.pi * 3.0 ** 2
    extra = {"shepard": shep_nnz * 12 + MQ * 41, "order": MQ * 16}
    mls_parts = ("aux_knn", "shepard", "order", "mls")
    if all(stages.get(k, 0.0) > 0 for k in mls_parts):
        ms_sum = sum(stages[k] for k in mls_parts)
        b_sum = alg["aux_knn"][1] + alg["mls"][1] + extra["shepard"] + extra["order"]
        ach = b_sum / (ms_sum / 1000.0) / 1e9
        stage_roof["mls_stage"] = {"kernel": "aux_knn_kernel + shepard_apply_kernel + work-order sort + "
                                   "mls_gather_kernel + mls_solve_kernel + reg_kernel + redo_kernel", "ms": round(ms_sum, 4),
                                   "algorithmic_bytes": int(b_sum), "achieved_gbs": round(ach, 1),
                                   "frac": round(ach / hbm_peak, 4), "traffic": None}
    dom = max(alg, key=lambda k: stages.get(k, 0.0))      # the slowest stage with a byte count
    dr = stage_roof.get(dom)
    roof = {"bound": "hbm", "kernel": dr["kernel"] if dr else dom, "achieved": dr["achieved_gbs"] if dr else None,
            "peak": hbm_peak, "unit": "GB/s", "frac": dr["frac"] if dr else None,
            "traffic": TRAFFIC.get(dom), "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_launch": dr["algorithmic_bytes"] if dr else None,
            "ms_per_launch": dr["ms"] if dr else None, "stages": stage_roof}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": workload_name(args.nodes), "N": w.N, "K": w.K, "M": w.M, "grid_nodes": MQ,
                           "precision": "mixed", "parallelism": f"replicas x{world}" if world > 1 else "single",
                           "l2": "256 MiB write between timed steps"},
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                "grid_nodes_per_s": value * MQ,
                "stage_ms": {k: round(v, 4) for k, v in stages.items()},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk.summary(), "fp64_form": fp64, "refit": refit, "many_sets": many,
                "batched": batched, "serving": serving, "voronoi": voronoi, "forward": forward, "l2_error": l2,
                "mls_stats": {k: stats[k] for k in ("sum_n", "min_n", "max_n", "n_regularized", "n_guarded",
                                                    "n_fp64_redo", "n_dropped")},
                "knn_stats": {k: stats[k] for k in stats if k.startswith("knn_") or k == "aux_points"}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
