"""Benchmark of the GB300 small-scale power-spectrum path (arXiv:2005.01739, Sec. 3).

One step = one complete hip_power call on a device-resident catalog: cell-list
build, the FP32 pair pass (Legendre moments of the separation, with the FP64
projection of the bin-edge functions and the FP64 contraction), FP64 finalize
(W~^a, reduction, normalisation) and the download of P and DD.  Metric:
unordered pairs with 0 < r < R0, times the number of k bins, per second
(pairs x k-bins / s).  The same line also reports, each with its own event
timing: the plain FP64 path on the same catalog; the bispectrum workload
(5e5 particles, 1.5e6 randoms: rate, stage times, the rooflines of the a_lm
pass and of the tensor-core contraction, parity of a primary sample against the
oracle, and the random-free variant); the 64-catalog batch (graph replays of
the mixed plan, the FP64 plan, their ratio and the mixed-vs-FP64 parity of
every catalog, and B of 16 catalogs); the 5e4-particle plain configuration in
both precisions with parity against the oracle; the parity of the timed
workload on the oracle's sample (floored, unfloored and plain errors); the
subsample selection, the clocks seen and the oracle's own rate on the host
cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank measures its own catalog of
the same size (different seed): weak scaling, no data-path collective; only the
step times are max-reduced.  ``--impl reference`` times the FP64 CPU oracle on
the host cores over a bounded primary sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs×k-bins/s for P_ℓ(k), B_ℓ; mixed-prec batched vs FP64 GPU at stated err"
UNIT = "pairs*kbins/s"
WORKLOAD = "pk_mixed_n2e6"
FLOPS_PER_PAIR_BIN = 12.0  # nominal algorithmic FP32 flops per (unordered pair, k bin)
# DRAM bytes (read + write) of one pair-pass launch on the 2e6-particle workload: ncu measured
# 5.464 MB for the moment pass (5.18 MB for the direct pass) on the same workload shrunk to 2.5e5
# particles; the traffic is the particle data read once, so it scales with N: x 8.
PAIR_KERNEL_DRAM_BYTES = {1: 5.464e6 * 8, 0: 5.18e6 * 8}
PAIR_KERNEL_NAME = {1: "k_power_moments<float,21,8>", 0: "k_power_pairs<float,4,21>"}
# kernels one FP32 hip_power call launches: cell build 3, pair pass (moments: coefficients, sum |w|,
# pairs, contraction) 4 or 1, finalize 2
PAIR_PASS_LAUNCHES = {1: 9, 0: 6}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_peak_tflops(pk) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(rank: int, scale: float = 1.0):
    """The timed workload; `scale` < 1 shrinks the box volume (and N, parents)
    by that factor at fixed density, R0 and bins, for profiler captures."""
    from paper_2005_01739_gb300 import catalogs
    wl = catalogs.workload(WORKLOAD)
    if rank > 0 or scale != 1.0:  # weak scaling: same density and settings, another seed
        L = 1000.0 * scale ** (1.0 / 3.0)
        pos, w = catalogs.thomas(int(2_000_000 * scale), L, int(50_000 * scale), 1.5, 1001 + 97 * rank,
                                 weights="u05_15")
        wl = dict(wl, pos=pos, w=w, L=L)
    return wl


def _config(wl, nranks, shard=False):
    return {"workload": WORKLOAD, "N": int(len(wl["pos"])), "L": wl["L"], "R0": wl["R0"],
            "n_k": int(len(wl["edges"]) - 1), "k_range": [float(wl["edges"][0]), float(wl["edges"][-1])],
            "ell": [0, 2, 4], "weights": "U(0.5,1.5)", "catalog": "Thomas process, 5e4 parents, sigma 1.5",
            "l2": "flushed between timed steps (512 MB write)",
            "parallelism": f"{'shard' if shard else 'replicas'}{nranks}"}


def combine_ranks(ms: float, work: float, device: str):
    """Whole-job timing over ranks: the slowest rank's time and the sum of the
    work all ranks did (no data-path collective; one scalar each)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(work)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def shard_range(rank: int, world: int, n: int):
    """Primary range [p0, p1) of one rank when a catalog is sharded by primaries."""
    return rank * n // world, (rank + 1) * n // world


def combine_shards(DD, device: str):
    """Sum over ranks of the partial ordered pair sums DD [n_ell, n_k] of disjoint
    primary ranges (one FP64 all-reduce); their sum is the catalog's full DD."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(DD, dtype=np.float64), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def oracle_sample(wl, seconds: float):
    """Time the FP64 oracle on a primary subset sized for ~`seconds` of work."""
    import oracle
    pos = wl["pos"].astype(np.float64)
    w = wl["w"].astype(np.float64)
    m = 32
    while True:
        t0 = time.perf_counter()
        DD, npairs = oracle.power_pair_sum(pos, w, wl["L"], wl["R0"], wl["edges"], 4, 2, primaries=np.arange(m))
        dt = time.perf_counter() - t0
        if dt > 0.5 * seconds or m >= len(pos):
            break
        m = min(len(pos), max(2 * m, int(m * seconds / max(dt, 1e-3))))
    nk = len(wl["edges"]) - 1
    return {"value": npairs * nk / dt, "seconds": dt, "primaries": m, "ordered_pairs": npairs,
            "cores": oracle.num_threads(), "DD": DD}


def sample_parity(binding, dpos, dw, wl, cpu):
    """Error of the GPU paths on the oracle's sample (the same primaries), per
    multipole: max over bins of |DD - DD_ref| / max(|DD_ref,l|, |DD_ref,0|,
    1e-2 max |DD_ref,0|), the metric of the parity tests."""
    ref = cpu["DD"]
    floor = 1e-2 * np.max(np.abs(ref[0]))
    scale = np.maximum(np.maximum(np.abs(ref), np.abs(ref[0])[None, :]), floor)
    out, unf = {}, {}
    for prec in ("mixed", "fp64"):
        _, DD, _ = binding.hip_power(dpos, dw, wl["L"], wl["R0"], wl["edges"], 4, 2, prec,
                                     prim_range=(0, cpu["primaries"]))
        out[prec] = [float(x) for x in np.max(np.abs(DD - ref) / scale, axis=1)]
        unf[prec] = _pk_metrics(DD, ref)
    return {"metric": "max over k bins of |DD_l - DD_l,oracle| / max(|DD_l|, |DD_0|, 1e-2 max|DD_0|)",
            "ell": [0, 2, 4], "mixed_max_rel_err": out["mixed"], "fp64_max_rel_err": out["fp64"],
            "mixed_all_metrics": unf["mixed"], "fp64_all_metrics": unf["fp64"],
            "all_metrics_note": ("floored: the asserted metric; survey: the same without the 1e-2 max|DD_0| "
                                 "floor; plain: |dDD| / |DD| per bin"),
            "tolerance": {"mixed": 1e-5, "fp64": 1e-10},
            "sample": f"the cpu_baseline sample: pair sums of the first {cpu['primaries']} primaries"}


def _bk_metrics(B, Bref):
    """Per-bin errors of the B parity: floored (the asserted metric of the tests),
    the same without the floor, and the plain relative error."""
    B, Bref = np.asarray(B, float), np.asarray(Bref, float)
    d = np.abs(B - Bref)
    scale = np.maximum(np.abs(Bref), np.abs(Bref[0])[None])
    floor = 1e-2 * np.max(np.abs(Bref), axis=(1, 2))[:, None, None]
    nz = scale > 0
    plain = np.abs(Bref) > 0
    return {"floored": float(np.max(d / np.maximum(scale, floor))),
            "survey": float(np.max(d[nz] / scale[nz])) if np.any(nz) else 0.0,
            "plain": float(np.max(d[plain] / np.abs(Bref[plain]))) if np.any(plain) else 0.0}


def bispectrum_rate(binding, stream, reps: int = 2, scale: float = 1.0, parity: bool = True):
    """B_l (l = 0..4) of the 5e5-particle workload with 1.5e6 randoms: ordered
    (primary, data) pairs, random primaries included, times bins, per second;
    stage times, the rooflines of the a_lm pass and of the tensor-core
    contraction, and the primary sums of a sample of data and random primaries
    against the oracle (hip_bispectrum_partial vs oracle.bispectrum_primary_sum).
    `scale` < 1 shrinks the volume at fixed density (profiler captures only)."""
    import torch
    from paper_2005_01739_gb300 import catalogs
    wl = catalogs.workload("bk_n5e5")
    if scale != 1.0:
        L = 1000.0 * scale ** (1.0 / 3.0)
        pos, _ = catalogs.thomas(int(500_000 * scale), L, int(12_500 * scale), 1.5, 1002)
        wl = dict(wl, pos=pos, rand=catalogs.uniform(int(1_500_000 * scale), L, 1002 + 7919), L=L)
    dpos = torch.from_numpy(wl["pos"]).cuda()
    drnd = torch.from_numpy(wl["rand"]).cuda()
    nk = len(wl["edges"]) - 1
    binding.set_profiling(True)
    with torch.cuda.stream(stream):
        binding.hip_bispectrum(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], 4, "mixed", stream=stream)
    ts, stages = [], []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                _, (nd, nr) = binding.hip_bispectrum(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], 4, "mixed",
                                                     stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
            stages.append(binding.bispectrum_stage_times())
    ms = float(np.mean(ts))
    st = np.mean(np.array(stages), axis=0)
    n_prim = len(wl["pos"]) + len(wl["rand"])
    pk = _peaks()
    fp32 = fp32_peak_tflops(pk)
    bf16 = float(pk.get("bf16_tflops", 1906.9))
    alm_flops = 60.0 * (nd + nr) * nk              # 25 harmonic FMAs + 5 jbar per (p, j)-bin
    con_alg = 2.0 * 25 * nk * nk * n_prim          # sum_l (2l+1) n_k^2 MACs per primary
    P = 8 if 128 // nk >= 5 else 4
    K = ((9 * P + 15) // 16) * 16
    tiles = (5 + min(5, 128 // nk) - 1) // min(5, 128 // nk)
    con_exec = 2.0 * 128 * 128 * K * 6 * tiles * np.ceil(n_prim / P)  # 6 slice products per K step
    out = {"workload": "bk_n5e5" if scale == 1.0 else f"bk_n5e5 x{scale}", "value": (nd + nr) * nk / (ms / 1e3),
           "unit": UNIT, "ms_per_call": ms, "pairs_data_primaries": nd, "pairs_random_primaries": nr, "n_k": nk,
           "ell": [0, 1, 2, 3, 4], "clocks": clk.summary(),
           "stage_ms": {"alm_pass": float(st[0]), "contraction": float(st[1]), "c_term": float(st[2]),
                        "chunks": int(st[3]), "rest": ms - float(st[0] + st[1] + st[2])},
           "roofline_alm": {"bound": "alu", "kernel": "k_bk_alm<float,1>", "achieved": alm_flops / (st[0] / 1e3) / 1e12,
                            "peak": fp32, "unit": "TFLOP/s", "frac": alm_flops / (st[0] / 1e3) / 1e12 / fp32,
                            "flops_per_pair_bin": 60.0, "peak_note": "derived FP32 FMA peak"},
           "roofline_contraction": {"bound": "tensor", "kernel": "k_bk_contract_tc", "unit": "TFLOP/s",
                                    "achieved": con_alg / (st[1] / 1e3) / 1e12, "peak": bf16,
                                    "frac": con_alg / (st[1] / 1e3) / 1e12 / bf16,
                                    "executed_tflops": con_exec / (st[1] / 1e3) / 1e12,
                                    "flops_per_primary": 2.0 * 25 * nk * nk,
                                    "note": ("achieved = algorithmic 2 sum_l (2l+1) n_k^2 flops per primary; "
                                             "executed counts the padded 128-row tiles and the 6 exact-split "
                                             "products (BF16 MMAs); peak = measured BF16 burst")}}
    if parity:
        import oracle
        p64, r64 = wl["pos"].astype(np.float64), wl["rand"].astype(np.float64)
        dS, rS = (1000, 1064), (3000, 3064)
        T, _ = binding.hip_bispectrum_partial(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], 4, "mixed",
                                              data_range=dS, rand_range=rS)
        Td, _ = oracle.bispectrum_primary_sum(p64[dS[0]:dS[1]], np.ones(dS[1] - dS[0]), np.arange(*dS), p64, None,
                                              wl["L"], wl["R0"], wl["edges"], 4)
        Tr, _ = oracle.bispectrum_primary_sum(r64[rS[0]:rS[1]], np.ones(rS[1] - rS[0]), None, p64, None,
                                              wl["L"], wl["R0"], wl["edges"], 4)
        Tref = Td - (len(wl["pos"]) / len(wl["rand"])) * Tr
        out["parity"] = dict(_bk_metrics(T, Tref), tolerance=1e-4,
                             sample=(f"primary sums of data primaries {dS[0]}..{dS[1]} and random primaries "
                                     f"{rS[0]}..{rS[1]} (input order) against the FP64 oracle"))
    # the same estimator without randoms: the DDR^II term from the E^II kernel (App. A)
    with torch.cuda.stream(stream):
        binding.hip_bispectrum_analytic(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, "mixed", stream=stream)
    ta = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            binding.hip_bispectrum_analytic(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, "mixed", stream=stream)
        b.record(stream)
        b.synchronize()
        ta.append(a.elapsed_time(b))
    out["analytic_ddr2"] = {"ms_per_call": float(np.mean(ta)),
                            "note": "same B without the random catalog (E^II kernel, App. A)"}
    # the anisotropic bispectrum about zhat (18 (l1, l2, L) combinations) on the same catalogs
    with torch.cuda.stream(stream):
        Bi, _ = binding.hip_bispectrum(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], 4, "mixed", stream=stream)
        Ba, _ = binding.hip_bispectrum_aniso(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], stream=stream)
    tb = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            Ba, _ = binding.hip_bispectrum_aniso(dpos, None, drnd, wl["L"], wl["R0"], wl["edges"], stream=stream)
        b.record(stream)
        b.synchronize()
        tb.append(a.elapsed_time(b))
    l0 = max(float(np.max(np.abs(Ba[binding.ANISO_COMBOS.index((l, l, 0))]
                                 - (-1) ** l * np.sqrt(2 * l + 1) * Bi[l])) / np.max(np.abs(Bi[l]))) for l in range(5))
    out["anisotropic"] = {"ms_per_call": float(np.mean(tb)), "combinations": len(binding.ANISO_COMBOS),
                          "value": (nd + nr) * nk / (float(np.mean(tb)) / 1e3), "unit": UNIT,
                          "l_l_0_vs_isotropic_max_rel": l0,
                          "note": "B_{l1 l2 L} about zhat (tripolar projection; the conclusions' extension); "
                                  "(l, l, 0) = (-1)^l sqrt(2l+1) B_l checked against hip_bispectrum at full size"}
    return out


def _pk_metrics(P, Pref):
    """Per-bin errors of a P (or DD) array [n_ell][n_k]: floored (the asserted
    metric of the tests), the same without the floor, and the plain relative error."""
    P, Pref = np.asarray(P, float), np.asarray(Pref, float)
    d = np.abs(P - Pref)
    scale = np.maximum(np.abs(Pref), np.abs(Pref[0])[None, :])
    floor = 1e-2 * np.max(np.abs(Pref[0]))
    nz, plain = scale > 0, np.abs(Pref) > 0
    return {"floored": float(np.max(d / np.maximum(scale, floor))),
            "survey": float(np.max(d[nz] / scale[nz])) if np.any(nz) else 0.0,
            "plain": float(np.max(d[plain] / np.abs(Pref[plain]))) if np.any(plain) else 0.0}


def batched_summary(binding, stream, steps: int = 2, fp64: bool = True, bispectrum: bool = True):
    """The 64-catalog batch: graph replays of the mixed plan (timed), one replay of
    the same plan in FP64 (the plain baseline, and the parity reference of every
    catalog's P), and B of the first 16 catalogs in one hip_bispectrum_batched call."""
    import torch
    from paper_2005_01739_gb300 import catalogs
    cats = catalogs.workload("batched64")["catalogs"]
    for c in cats:
        c["pos"] = torch.from_numpy(c["pos"]).cuda()
        c["w"] = torch.from_numpy(c["w"]).cuda()
    plan = binding.BatchPlan(cats, "mixed", stream=stream)

    def replays():
        ts = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = plan.run(stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return r, float(np.mean(ts))

    res = plan.run(stream)
    default_shape = plan.shape()
    _, ms_default = replays()
    # the autotuner's second stage (warps per CTA, fold period) on this batch, then the tuned plan is timed
    chosen, cand = plan.tune_kernel(stream)
    plan.run(stream)
    with ClockSampler(torch.cuda.current_device()) as clk:
        res, ms = replays()
    work = sum((n // 2) * (len(c["edges"]) - 1) for c, (_, _, n) in zip(cats, res))
    out = {"workload": "batched64", "catalogs": len(cats),
           "particles": int(sum(int(c["pos"].shape[0]) for c in cats)), "pair_bins": int(work),
           "value": work / (ms / 1e3), "unit": UNIT, "ms_per_replay": ms, "launches_per_replay": plan.launches,
           "clocks": clk.summary(),
           "autotune": {"shape": dict(zip(("particles_per_cell", "warps_per_cta", "fold_pairs"), plan.shape())),
                        "default_shape": dict(zip(("particles_per_cell", "warps_per_cta", "fold_pairs"),
                                                  default_shape)),
                        "default_ms_per_replay": ms_default,
                        "candidates_ms": {f"warps{w}_fold{f}": v for (w, f), v in cand.items()},
                        "note": "ms_per_replay is the tuned plan (hip_batch_plan_tune_kernel at the default 64 "
                                "particles per cell); warps 0 / fold 0 = the defaults (by occupancy / 16384)"}}
    mixed = [(np.array(P), np.array(DD)) for P, DD, _ in res]
    plan.close()
    if fp64:
        plan64 = binding.BatchPlan(cats, "fp64", stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res64 = plan64.run(stream)
        b.record(stream)
        b.synchronize()
        ms64 = a.elapsed_time(b)
        plan64.close()
        errs = [_pk_metrics(Pm, np.array(P64)) for (Pm, _), (P64, _, _) in zip(mixed, res64)]
        out["fp64_plain"] = {"value": work / (ms64 / 1e3), "unit": UNIT, "ms_per_replay": ms64,
                             "mixed_over_fp64": ms64 / ms}
        out["parity_vs_fp64"] = {k: max(e[k] for e in errs) for k in ("floored", "survey", "plain")}
        out["parity_vs_fp64"]["note"] = ("max over the 64 catalogs and their bins of the mixed P against the same "
                                         "plan in FP64 (which the tests hold to the oracle at 1e-10)")
    if bispectrum:
        bc = []
        for i, c in enumerate(cats[:16]):
            N = int(c["pos"].shape[0])
            rnd = torch.from_numpy(catalogs.uniform(3 * N, c["L"], 2000 + i + 7919)).cuda()
            bc.append(dict(pos=c["pos"], w=c["w"], rand=rnd, L=c["L"], R0=c["R0"], edges=c["edges"][:26], lmax=4))
        with torch.cuda.stream(stream):
            binding.hip_bispectrum_batched(bc, "mixed", stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            resb = binding.hip_bispectrum_batched(bc, "mixed", stream=stream)
        b.record(stream)
        b.synchronize()
        msb = a.elapsed_time(b)
        wb = sum((nd + nr) * 25 for _, (nd, nr) in resb)
        out["bispectrum_batched"] = {"workload": "first 16 catalogs of batched64, first 25 bins, 3N randoms, l = 0..4",
                                     "value": wb / (msb / 1e3), "unit": UNIT, "ms": msb, "pair_bins": int(wb)}
    return out


def plain_config_summary(binding, stream, cpu_seconds: float = 4.0, reps: int = 3):
    """The 5e4-particle catalog (plain FP64 configuration): both precisions timed
    (event-timed calls), and their pair sums on a primary sample against the oracle."""
    import torch
    import oracle
    from paper_2005_01739_gb300 import catalogs
    wl = catalogs.workload("pk_plain_n5e4")
    dpos = torch.from_numpy(wl["pos"]).cuda()
    nk = len(wl["edges"]) - 1
    out = {"workload": "pk_plain_n5e4", "N": int(len(wl["pos"])), "L": wl["L"], "R0": wl["R0"], "n_k": nk}
    ref_n = None
    for prec in ("fp64", "mixed"):
        with torch.cuda.stream(stream):
            binding.hip_power(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, 2, prec, stream=stream)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                _, _, n = binding.hip_power(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, 2, prec, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.mean(ts))
        out[prec] = {"value": (n // 2) * nk / (ms / 1e3), "unit": UNIT, "ms_per_call": ms}
        ref_n = n
    out["mixed_over_fp64"] = out["fp64"]["ms_per_call"] / out["mixed"]["ms_per_call"]
    m = 4000
    DD, _ = oracle.power_pair_sum(wl["pos"].astype(np.float64), None, wl["L"], wl["R0"], wl["edges"], 4, 2,
                                  primaries=np.arange(m))
    for prec in ("fp64", "mixed"):
        _, DDg, _ = binding.hip_power(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, 2, prec, prim_range=(0, m))
        out[prec]["parity_DD"] = _pk_metrics(DDg, DD)
    out["parity_sample"] = f"DD of the first {m} primaries against the FP64 oracle"
    out["unordered_pairs"] = int(ref_n // 2)
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = _workload(0)
    for _ in range(args.warmup):
        oracle_sample(wl, 2.0)
    times, rates, last = [], [], None
    for _ in range(args.steps):
        last = oracle_sample(wl, args.ref_seconds)
        rates.append(last["value"])
        times.append(last["seconds"])
    v = float(np.mean(rates))
    sample = (f"ordered pair sums of the first {last['primaries']} primaries against all "
              f"{len(wl['pos'])} particles, all {len(wl['edges']) - 1} bins, l=0,2,4 (FP64 brute force)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(wl, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def subsample_rate(binding, dpos, dw, stream, flush, fraction=0.01, reps=10):
    """hip_subsample on the device-resident catalog (the 1/f_sub selection of
    Sec. 9 at f_sub = 100): event-timed calls, L2 flushed before each; algorithmic
    bytes = 16 read per particle (positions and weights) + 16 written per kept one."""
    import torch
    n = int(dpos.shape[0])
    ts, kept = [], 0
    for i in range(reps + 2):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ps, _ = binding.hip_subsample(dpos, dw, fraction, 1234 + i, stream=stream)
        b.record(stream)
        b.synchronize()
        kept = int(ps.shape[0])
        if i >= 2:
            ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    nbytes = 16.0 * n + 16.0 * kept
    return {"fraction": fraction, "particles": n, "kept": kept, "ms_per_call": ms,
            "achieved_GBps": nbytes / (ms / 1e3) / 1e9,
            "note": "call includes the count read-back and its host synchronisation"}


def run_batched(args):
    """The 64-catalog batch alone (batched_summary), optionally after autotuning
    the plan's cell shape."""
    import torch

    from paper_2005_01739_gb300 import binding, build, catalogs
    build.build()
    binding.load()
    stream = torch.cuda.Stream()
    tuned = None
    if args.tune:  # pick the cell shape by timing each candidate once
        cats = catalogs.workload("batched64")["catalogs"]
        for c in cats:
            c["pos"] = torch.from_numpy(c["pos"]).cuda()
            c["w"] = torch.from_numpy(c["w"]).cuda()
        plan = binding.BatchPlan(cats, "mixed", stream=stream)
        chosen, tms = plan.tune(stream)
        plan.close()
        tuned = {"chosen_particles_per_cell": chosen, "replay_ms": {str(k): v for k, v in tms.items()}}
    out = batched_summary(binding, stream, steps=args.steps, fp64=not args.skip_fp64,
                          bispectrum=not args.skip_bispectrum)
    out["autotune"] = tuned
    print(json.dumps({"batched": out}), flush=True)
    return 0


def run_large(args):
    """The 256^3 Zel'dovich lattice: P (R0 = 20, 200 bins to k = 10, l = 0,2,4) and
    B (R0 = 15, 40 bins, l = 0..4, 3x randoms), mixed path, one timed call each
    after one warm-up."""
    import torch

    from paper_2005_01739_gb300 import binding, build, catalogs
    build.build()
    binding.load()
    wl = catalogs.workload("large_zeldovich")
    stream = torch.cuda.Stream()
    dpos = torch.from_numpy(wl["pos"]).cuda()

    def timed(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return out, a.elapsed_time(b)

    def pk():
        with torch.cuda.stream(stream):
            return binding.hip_power(dpos, None, wl["L"], wl["R0"], wl["edges"], 4, 2, "mixed", stream=stream)

    (_, _, npairs), ms_p = timed(pk)
    nk = len(wl["edges"]) - 1
    out = {"workload": "large_zeldovich", "N": int(len(wl["pos"])),
           "power": {"value": (npairs // 2) * nk / (ms_p / 1e3), "unit": UNIT, "ms": ms_p,
                     "unordered_pairs": int(npairs // 2), "n_k": nk, "R0": wl["R0"]}}
    if not args.skip_bispectrum:
        rnd = catalogs.uniform(3 * len(wl["pos"]), wl["L"], 1004 + 7919)
        drnd = torch.from_numpy(rnd).cuda()
        nkb = len(wl["edges_b"]) - 1

        def bk():
            with torch.cuda.stream(stream):
                return binding.hip_bispectrum(dpos, None, drnd, wl["L"], wl["R0_b"], wl["edges_b"], 4, "mixed",
                                              stream=stream)

        (_, (nd, nr)), ms_b = timed(bk)
        out["bispectrum"] = {"value": (nd + nr) * nkb / (ms_b / 1e3), "unit": UNIT, "ms": ms_b,
                             "pairs_data_primaries": int(nd), "pairs_random_primaries": int(nr), "n_k": nkb,
                             "R0": wl["R0_b"], "randoms": int(len(rnd))}
    print(json.dumps(out), flush=True)
    return 0


def run_bispectrum_only(args):
    import torch

    from paper_2005_01739_gb300 import binding, build
    build.build()
    binding.load()
    stream = torch.cuda.Stream()
    print(json.dumps({"bispectrum": bispectrum_rate(binding, stream, reps=args.steps, scale=args.scale)}),
          flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2005_01739_gb300 import binding, build

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    binding.load()
    shard = ws > 1 and args.multi == "shard"
    # sharded: every rank holds the one catalog and takes a primary range; replicas:
    # every rank its own catalog of the same size (another seed)
    wl = _workload(0 if shard else rank, args.scale)
    L, R0, edges = wl["L"], wl["R0"], wl["edges"]
    nk = len(edges) - 1
    stream = torch.cuda.Stream()
    dpos = torch.from_numpy(wl["pos"]).cuda()
    dw = torch.from_numpy(wl["w"]).cuda()
    prim = shard_range(rank, ws, len(wl["pos"])) if shard else None
    S1 = float(np.sum(wl["w"], dtype=np.float64))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    binding.set_profiling(True)

    def call(pos, w):
        with torch.cuda.stream(stream):
            P, DD, npairs = binding.hip_power(pos, w, L, R0, edges, 4, 2, "mixed", prim_range=prim, stream=stream)
        if shard:  # the one exchange of the path: the FP64 sum of the partial DD, then P on rank 0
            DD = combine_shards(DD, "cuda")
            P = binding.hip_power_from_pairs(DD, L, R0, edges, S1, stream=stream) if rank == 0 else None
        return P, DD, npairs

    def step():
        return call(dpos, dw)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_ms, pair_ms = [], []
    npairs = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[i][0].record(stream)
            _, _, npairs = step()
            ev[i][1].record(stream)
            st_i = binding.stage_times()
            pair_ms.append(float(st_i[2]))
            stage_rec = [float(x) for x in st_i]
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    pairs = npairs // 2  # unordered pairs with 0 < r < R0
    work = float(pairs) * nk
    ms_max, work_sum = combine_ranks(ms, work, "cuda")
    value = work_sum / (ms_max / 1e3)

    # end to end through the public call with pinned host inputs (H2D and result D2H inside)
    hpos = torch.from_numpy(wl["pos"]).pin_memory()
    hw = torch.from_numpy(wl["w"]).pin_memory()
    e2e_t = []
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call(hpos, hw)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    e2e_max, _ = combine_ranks(e2e_ms, 0.0, "cuda")
    e2e_value = work_sum / (e2e_max / 1e3)
    n = len(wl["pos"])
    h2d = 12 * n + 4 * n
    d2h = 2 * 3 * nk * 8 + 8 + 4
    subs = subsample_rate(binding, dpos, dw, stream, flush)

    # the plain FP64 kernel on the same catalog (one step), for the mixed/FP64 ratio
    fp64 = None
    if not args.skip_fp64:
        with torch.cuda.stream(stream):
            binding.hip_power(dpos, dw, L, R0, edges, 4, 2, "fp64", stream=stream)
        st = binding.stage_times()
        fp64_kernel_ms = float(st[2])
        fp64 = {"value": work / (float(sum(st[1:4])) / 1e3), "unit": UNIT, "pair_kernel_ms": fp64_kernel_ms,
                "speedup_mixed_vs_fp64_kernel": fp64_kernel_ms / float(np.mean(pair_ms))}

    bisp = None
    if not args.skip_bispectrum:
        bisp = bispectrum_rate(binding, stream)
    batched = None
    plain = None
    if rank == 0 and not args.skip_batched:
        batched = batched_summary(binding, stream, fp64=not args.skip_fp64, bispectrum=not args.skip_bispectrum)
    if rank == 0 and not args.skip_cpu:
        plain = plain_config_summary(binding, stream)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    pk = _peaks()
    peak = fp32_peak_tflops(pk)
    kern_ms = float(np.mean(pair_ms))
    achieved = FLOPS_PER_PAIR_BIN * work / (kern_ms / 1e3) / 1e12
    pair_pass = binding.power_pair_pass(wl["R0"], float(wl["edges"][-1]), "mixed")
    cpu = oracle_sample(wl, args.ref_seconds) if not args.skip_cpu else None
    cpu1 = None
    if cpu:  # the same oracle on one core, a shorter sample
        import oracle
        nthr = oracle.num_threads()
        oracle.set_threads(1)
        cpu1 = oracle_sample(wl, 3.0)
        oracle.set_threads(nthr)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": _config(wl, ws, shard),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_max},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": PAIR_KERNEL_DRAM_BYTES[pair_pass], "kernel": PAIR_KERNEL_NAME[pair_pass],
                     "kernel_ms": kern_ms, "flops_per_pair_bin": FLOPS_PER_PAIR_BIN,
                     "peak_note": "derived FP32 FMA peak: 152 SM x 128 lanes x 2 x max SM clock"},
        "gpu_launches": PAIR_PASS_LAUNCHES[pair_pass] * args.steps,
        "clocks": clk.summary(),
        "pairs": int(pairs),
        "stage_ms": dict(zip(["upload", "cells", "pairs", "finalize", "download"], stage_rec)),
        "fp64_plain": fp64,
        "bispectrum": bisp,
        "batched": batched,
        "plain_n5e4": plain,
        "subsample": subs,
    }
    # after stage_ms is read: these calls replace the recorded stage times
    line["parity"] = sample_parity(binding, dpos, dw, wl, cpu) if cpu else None
    if cpu:
        line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                                "sample": (f"FP64 brute force, ordered pair sums of the first {cpu['primaries']} "
                                           f"primaries against all {n} particles, {nk} bins, l=0,2,4 "
                                           f"({cpu['seconds']:.1f} s)"),
                                "single_core_value": cpu1["value"],
                                "single_core_sample": f"first {cpu1['primaries']} primaries ({cpu1['seconds']:.1f} s)"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--multi", choices=["shard", "replicas"], default="shard",
                    help="N > 1: shard the catalog's primaries over the ranks (one FP64 all-reduce of DD) "
                         "or run one catalog per rank")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-bispectrum", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--bk-only", action="store_true", help="time only the bispectrum workload")
    ap.add_argument("--batched", action="store_true", help="time the 64-catalog batched workload")
    ap.add_argument("--large", action="store_true", help="time P and B on the 256^3 Zel'dovich lattice")
    ap.add_argument("--tune", action="store_true", help="--batched: autotune the plan's cell shape first")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the catalog volume at fixed density (profiler captures only)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.bk_only:
        return run_bispectrum_only(args)
    if args.large:
        return run_large(args)
    if args.batched:
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
