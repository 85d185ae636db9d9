"""Full-size checks in the benchmark's launch configuration, on primary subsets
the oracle can sum directly: the 256^3-particle Zel'dovich lattice (P with 200
bins to k = 10, B with 40 bins) and the bispectrum workload, plus the sharding
identity of the bispectrum's primary sums."""
import numpy as np
import pytest

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


def _rel(X, Xref):
    """Per-bin error with the floors of the P and B metrics (1 % of the largest |X_0|)."""
    if Xref.ndim == 2:
        floor = 1e-2 * np.max(np.abs(Xref[0]))
        scale = np.maximum(np.maximum(np.abs(Xref), np.abs(Xref[0])[None, :]), floor)
    else:
        floor = 1e-2 * np.max(np.abs(Xref), axis=(1, 2))[:, None, None]
        scale = np.maximum(np.maximum(np.abs(Xref), np.abs(Xref[0])[None]), floor)
    return float(np.max(np.abs(X - Xref) / scale))


@pytest.fixture(scope="module")
def large():
    import torch
    wl = catalogs.workload("large_zeldovich")
    wl["dpos"] = torch.from_numpy(wl["pos"]).cuda()
    return wl


def test_large_power_sampled(large):
    wl = large
    S = (5000, 5160)
    DDref, nref = oracle.power_pair_sum(wl["pos"].astype(np.float64), None, wl["L"], wl["R0"], wl["edges"], 4, 2,
                                        primaries=np.arange(*S))
    for prec, tol in (("mixed", 1e-5), ("fp64", 1e-10)):
        _, DD, n = binding.hip_power(wl["dpos"], None, wl["L"], wl["R0"], wl["edges"], 4, 2, prec, prim_range=S)
        assert abs(n - nref) <= (0 if prec == "fp64" else 2)
        assert _rel(DD, DDref) < tol


def test_large_bispectrum_sampled(large):
    import torch
    wl = large
    rnd = catalogs.uniform(3 * len(wl["pos"]) // 8, wl["L"], 1004 + 7919)  # a random subset is enough here
    drnd = torch.from_numpy(rnd).cuda()
    S1 = float(len(wl["pos"]))
    p64 = wl["pos"].astype(np.float64)
    dS, rS = (2000, 2040), (7000, 7040)
    T, (nd, nr) = binding.hip_bispectrum_partial(wl["dpos"], None, drnd, wl["L"], wl["R0_b"], wl["edges_b"], 4,
                                                 "mixed", data_range=dS, rand_range=rS)
    Td, npd = oracle.bispectrum_primary_sum(p64[dS[0]:dS[1]], np.ones(dS[1] - dS[0]), np.arange(*dS), p64, None,
                                            wl["L"], wl["R0_b"], wl["edges_b"], 4)
    Tr, npr = oracle.bispectrum_primary_sum(rnd[rS[0]:rS[1]].astype(np.float64), np.ones(rS[1] - rS[0]), None, p64,
                                            None, wl["L"], wl["R0_b"], wl["edges_b"], 4)
    Tref = Td - (S1 / len(rnd)) * Tr
    assert abs(nd - npd) <= 2 and abs(nr - npr) <= 2
    assert _rel(T, Tref) < 1e-4


def test_bispectrum_partial_sums_add_up():
    import torch
    L, R0 = 60.0, 12.0
    pos, _ = catalogs.thomas(1500, L, 60, 1.5, seed=61, background_frac=0.2)
    rnd = catalogs.uniform(4500, L, seed=62)
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    dpos, drnd = torch.from_numpy(pos).cuda(), torch.from_numpy(rnd).cuda()
    Tfull, (nd, nr) = binding.hip_bispectrum_partial(dpos, None, drnd, L, R0, edges, 4, "fp64")
    parts = [((0, 700), (0, 0)), ((700, 1500), (0, 2000)), ((0, 0), (2000, 4500))]
    Tsum = 0
    for dr, rr in parts:
        Tp, _ = binding.hip_bispectrum_partial(dpos, None, drnd, L, R0, edges, 4, "fp64", data_range=dr, rand_range=rr)
        Tsum = Tsum + Tp
    assert _rel(Tsum, Tfull) < 1e-12
    # against the oracle on the data primaries alone
    Td, _ = oracle.bispectrum_primary_sum(pos.astype(np.float64), np.ones(1500), np.arange(1500),
                                          pos.astype(np.float64), None, L, R0, edges, 4)
    Tg, _ = binding.hip_bispectrum_partial(dpos, None, drnd, L, R0, edges, 4, "mixed", rand_range=(0, 0))
    assert _rel(Tg, Td) < 1e-4
