"""Batched power spectra (many catalogs, one persistent pair launch inside a CUDA
graph) and batched bispectra (one persistent launch over all catalogs'
primaries) against the FP64 oracle and against single-catalog calls."""
import numpy as np
import pytest

import parity_metrics

import oracle
from paper_2005_01739_gb300 import binding, catalogs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_01739_gb300 import build
    build.build()
    binding.load()


def _err(P, Pref, what=""):
    # the asserted metric and its two companions are printed (run with -s)
    return parity_metrics.report("P", P, Pref, what)["floored"]


def _batch(device):
    """Eight catalogs of uneven N, box, R0, bins (uniform and not), l_max and line of sight."""
    import torch
    rng = np.random.default_rng(9)
    cats = []
    for i in range(8):
        N = int(np.exp(rng.uniform(np.log(300), np.log(5000))))
        L = float(rng.uniform(40, 90))
        R0 = float([6.0, 9.0, 13.0][i % 3])
        nk = [8, 40, 70][i % 3]
        edges = catalogs.linear_edges(25.0 / R0 / 10, 25.0 / R0 / 10 + 3.0 * nk / R0 / 3, nk)
        if i == 5:
            edges = np.concatenate([[0.0], np.geomspace(0.05, 3.0, nk)])
        pos, w = catalogs.thomas(N, L, max(4, N // 30), 1.2, seed=500 + i, background_frac=0.3,
                                 los_sigma=1.0, weights="u05_15" if i % 2 else "unit")
        c = dict(pos=pos, w=w, L=L, R0=R0, edges=edges, ell_max=[4, 2, 4, 0][i % 4], los_axis=i % 3)
        if device:
            c["pos"] = torch.from_numpy(pos).cuda()
            c["w"] = None if w is None else torch.from_numpy(w).cuda()
        cats.append((c, pos, w))
    return cats


def test_batched_matches_oracle_and_single_calls():
    cats = _batch(device=True)
    plan = binding.BatchPlan([c for c, _, _ in cats], "mixed")
    # cell builds (3 per catalog), the pair pass (sum |w|, moment pass and contraction, or the direct pass),
    # finalize (2)
    pm = all(binding.power_pair_pass(c["R0"], c["edges"][-1]) == 1 for c, _, _ in cats)
    assert pm
    assert plan.launches == 3 * len(cats) + (5 if pm else 3)
    res1 = plan.run()
    res2 = plan.run()  # replay of the same graph
    for (c, pos, w), (P, DD, n), (P2, _, n2) in zip(cats, res1, res2):
        w64 = None if w is None else w.astype(np.float64)
        DDr, nr = oracle.power_pair_sum(pos.astype(np.float64), w64, c["L"], c["R0"], c["edges"], c["ell_max"],
                                        c["los_axis"])
        S1 = len(pos) if w is None else float(np.sum(w64))
        Pr = oracle.power_from_pairs(DDr, S1, c["L"], oracle.window_transform_binned(c["edges"], c["R0"]))
        assert abs(n - nr) <= 2 and n2 == n
        assert _err(P, Pr) < 1e-5
        assert _err(P2, P) < 1e-5  # FP32 sums in a different order (dynamic scheduling)
        Ps, _, ns = binding.hip_power(c["pos"], c["w"], c["L"], c["R0"], c["edges"], c["ell_max"], c["los_axis"],
                                      "mixed")
        assert _err(P, Ps) < 1e-5
    plan.close()


def test_batched_fp64_host_inputs_and_nonfinite():
    cats = _batch(device=False)[:4]
    res = binding.hip_power_batched([c for c, _, _ in cats], "fp64")
    for (c, pos, w), (P, DD, n) in zip(cats, res):
        Ps, _, ns = binding.hip_power(pos, w, c["L"], c["R0"], c["edges"], c["ell_max"], c["los_axis"], "fp64")
        assert n == ns
        assert _err(P, Ps) < 1e-10
    bad = [dict(c) for c, _, _ in cats]
    p = bad[2]["pos"].copy()
    p[3, 2] = np.nan
    bad[2]["pos"] = p
    with pytest.raises(binding.HipError) as ei:
        binding.hip_power_batched(bad, "mixed")
    assert ei.value.status == binding.HIP_ERR_NONFINITE


def test_batched_direct_pass_beyond_moment_range():
    # one catalog with R0 k_max = 1080 (> 1024) sends the whole plan to the direct
    # pass; both catalogs must equal their single FP64 calls
    cats = []
    for i, (N, L, R0, kmax, nk) in enumerate([(1200, 60.0, 12.0, 90.0, 255), (900, 50.0, 10.0, 3.0, 20)]):
        pos, w = catalogs.thomas(N, L, 40, 1.5, seed=610 + i, background_frac=0.3, weights="u05_15")
        cats.append((dict(pos=pos, w=w, L=L, R0=R0, edges=catalogs.linear_edges(0.5, kmax, nk), ell_max=4,
                          los_axis=2), pos, w))
    assert binding.power_pair_pass(12.0, 90.0, "fp64") == 0
    plan = binding.BatchPlan([c for c, _, _ in cats], "fp64")
    assert plan.launches == 3 * len(cats) + 3
    for (c, pos, w), (P, DD, n) in zip(cats, plan.run()):
        Ps, _, ns = binding.hip_power(pos, w, c["L"], c["R0"], c["edges"], 4, 2, "fp64")
        assert n == ns
        assert _err(P, Ps) < 1e-10
    plan.close()


def test_bispectrum_batched_matches_single_calls_and_oracle():
    # three catalogs of different N, L, R0 and bins through ONE batched launch;
    # each must equal its own hip_bispectrum call (same estimator, other
    # summation order) and, for one of them, the FP64 oracle
    import torch
    specs = [(1200, 60.0, 12.0, (0.3, 2.4, 12), 71), (900, 50.0, 10.0, (0.4, 3.0, 9), 72),
             (1500, 70.0, 14.0, (0.25, 2.0, 14), 73)]
    cats = []
    for N, L, R0, (k0, k1, nk), seed in specs:
        pos, w = catalogs.thomas(N, L, N // 25, 1.5, seed=seed, background_frac=0.2, weights="u05_15")
        rnd = catalogs.uniform(3 * N, L, seed=seed + 1)
        cats.append(dict(pos=torch.from_numpy(pos).cuda(), w=torch.from_numpy(w).cuda(), rand=rnd, L=L, R0=R0,
                         edges=catalogs.linear_edges(k0, k1, nk), lmax=4, hpos=pos, hw=w))
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        res = binding.hip_bispectrum_batched(cats, prec)
        for c, (B, (nd, nr)) in zip(cats, res):
            Bs, (nds, nrs) = binding.hip_bispectrum(c["pos"], c["w"], c["rand"], c["L"], c["R0"], c["edges"], 4, prec)
            assert (nd, nr) == (nds, nrs)
            assert _berr(B, Bs) < tol, prec
    c = cats[1]
    Bref, _ = oracle.bispectrum(c["hpos"].astype(np.float64), c["hw"].astype(np.float64),
                                c["rand"].astype(np.float64), c["L"], c["R0"], c["edges"], 4)
    res = binding.hip_bispectrum_batched(cats, "mixed")
    assert _berr(res[1][0], Bref) < 1e-4


def _berr(B, Bref):
    floor = 1e-2 * np.max(np.abs(Bref), axis=(1, 2))[:, None, None]
    scale = np.maximum(np.maximum(np.abs(Bref), np.abs(Bref[0])[None]), floor)
    return float(np.max(np.abs(B - Bref) / scale))


def test_plan_autotune_keeps_results():
    # the autotuner only changes the cell shape and the moment pass's CTA shape and
    # fold period; every candidate gives the same estimator, so the tuned plan's
    # output matches the untuned one
    cats = [c for c, _, _ in _batch(True)]
    plan = binding.BatchPlan(cats, "mixed")
    try:
        before = [(P, n) for P, _, n in plan.run()]
        chosen, ms = plan.tune()
        assert chosen in (4, 8, 16, 32, 64, 128, 256, 0) and len(ms) == 8 and all(v > 0 for v in ms.values())
        assert plan.shape()[0] == chosen
        # second stage: warps per CTA and fold period of the moment pass
        (w, f), kms = plan.tune_kernel()
        assert (w, f) in kms and len(kms) == 6 and all(v > 0 for v in kms.values())
        assert plan.shape() == (chosen, w, f)
        after = plan.run()
        for (P0, n0), (P1, _, n1) in zip(before, after):
            assert _err(P1, P0) < 1e-5
            assert abs(n1 - n0) <= max(2, int(2e-6 * n0))
    finally:
        plan.close()
