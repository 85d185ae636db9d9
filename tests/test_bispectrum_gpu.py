"""GPU parity of the bispectrum path (Sec. 4, summary of Sec. 4.5) against the
FP64 oracle, through the C ABI.

Per-bin metric (the multipoles cross zero, so the scale of a bin is set by its
own value, the monopole of the same (a, b), and 1 % of the largest |B_l| of
the multipole):

    |B_gpu - B_ref| / max(|B_ref,l^ab|, |B_ref,0^ab|, 1e-2 max_a'b' |B_ref,l^a'b'|)

Tolerances: plain FP64 path 1e-10, mixed path 1e-4.
"""
import numpy as np
import pytest

import parity_metrics

import oracle
from paper_2005_01739_gb300 import binding, catalogs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_01739_gb300 import build
    build.build()
    binding.load()


def _dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _err(B, Bref, what=""):
    # the asserted metric and its two companions are printed (run with -s)
    return parity_metrics.report("B", B, Bref, what)["floored"]


_cache = {}


def _oracle_B(key, pos, w, rnd, L, R0, edges, lmax=4):
    if key not in _cache:
        w64 = None if w is None else w.astype(np.float64)
        B, info = oracle.bispectrum(pos.astype(np.float64), w64, rnd.astype(np.float64), L, R0, edges, lmax)
        _cache[key] = (B, info)
    return _cache[key]


def _case(seed=41, N=1500, weights="unit"):
    L, R0 = 60.0, 12.0
    pos, w = catalogs.thomas(N, L, N // 25, 1.5, seed=seed, background_frac=0.2, weights=weights)
    rnd = catalogs.uniform(3 * N, L, seed=seed + 1)
    return pos, w, rnd, L, R0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bispectrum_parity_small(prec):
    pos, w, rnd, L, R0 = _case()
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    Bref, info = _oracle_B("small", pos, w, rnd, L, R0, edges)
    B, (nd, nr) = binding.hip_bispectrum(_dev(pos), None, _dev(rnd), L, R0, edges, 4, prec)
    slack = 0 if prec == "fp64" else max(2, int(2e-6 * info["npairs_data"]))
    assert abs(nd - info["npairs_data"]) <= slack and abs(nr - info["npairs_rand"]) <= slack
    assert _err(B, Bref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bispectrum_parity_weighted(prec):
    pos, w, rnd, L, R0 = _case(seed=43, N=1200, weights="u05_15")
    edges = catalogs.linear_edges(0.2, 2.0, 9)
    Bref, _ = _oracle_B("weighted", pos, w, rnd, L, R0, edges)
    B, _ = binding.hip_bispectrum(pos, w, rnd, L, R0, edges, 4, prec)  # host inputs
    assert _err(B, Bref) < TOL[prec]


def test_bispectrum_parity_two_chunks():
    # 40 bins: 41 edges, two 32-edge chunks per lane (mixed path only)
    pos, w, rnd, L, R0 = _case(seed=45, N=800)
    edges = catalogs.linear_edges(0.3, 4.3, 40)
    Bref, _ = _oracle_B("chunks", pos, w, rnd, L, R0, edges, lmax=2)
    B, _ = binding.hip_bispectrum(_dev(pos), None, _dev(rnd), L, R0, edges, 2, "mixed")
    assert _err(B, Bref) < TOL["mixed"]


def test_bispectrum_sixty_bins():
    # 60 bins: 61 edges (two 32-edge chunks per lane in the a_lm pass) and three
    # 128-row tiles of (l, a) rows in the tensor-core contraction
    pos, w, rnd, L, R0 = _case(seed=55, N=500)
    edges = catalogs.linear_edges(0.3, 6.3, 60)
    Bref, _ = _oracle_B("sixty", pos, w, rnd, L, R0, edges, lmax=4)
    B, _ = binding.hip_bispectrum(_dev(pos), None, _dev(rnd), L, R0, edges, 4, "mixed")
    assert _err(B, Bref) < TOL["mixed"]


def test_bispectrum_one_cta_many_primaries():
    # a single contraction CTA takes all 3000 data and 9000 random primaries: the
    # FP32 accumulators in tensor memory are folded into FP64 every 64 primaries,
    # so the error must not grow with the number of primaries a CTA accumulates
    pos, w, rnd, L, R0 = _case(seed=51, N=3000)
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    Bref, _ = _oracle_B("one_cta", pos, w, rnd, L, R0, edges)
    binding.debug_bk_caps(tc_grid_cap=1)
    try:
        B, _ = binding.hip_bispectrum(_dev(pos), None, _dev(rnd), L, R0, edges, 4, "mixed")
    finally:
        binding.debug_bk_caps(0, 0)
    assert _err(B, Bref) < TOL["mixed"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bispectrum_chunks_and_both_signs(prec):
    # the primaries pass in chunks of 1000 (several a_lm / contraction launches),
    # and every seventh data weight is negative, so tensor-core stages hold
    # primaries of both signs (issued once per sign)
    pos, w, rnd, L, R0 = _case(seed=53, N=1000, weights="u05_15")
    w = w.copy()
    w[::7] = -0.4
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    Bref, _ = _oracle_B("signs", pos, w, rnd, L, R0, edges)
    binding.debug_bk_caps(chunk_cap=1000)
    try:
        B, _ = binding.hip_bispectrum(_dev(pos), _dev(w), _dev(rnd), L, R0, edges, 4, prec)
    finally:
        binding.debug_bk_caps(0, 0)
    assert _err(B, Bref) < TOL[prec]


def test_bispectrum_symmetric_and_translation_invariant():
    pos, w, rnd, L, R0 = _case(seed=47, N=1500)
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    B, _ = binding.hip_bispectrum(_dev(pos), None, _dev(rnd), L, R0, edges, 4, "mixed")
    assert _err(np.transpose(B, (0, 2, 1)), B) < 1e-5
    sh = np.array([11.1, 23.7, 41.3])
    p2 = np.mod(pos.astype(np.float64) + sh, L).astype(np.float32)
    r2 = np.mod(rnd.astype(np.float64) + sh, L).astype(np.float32)
    B2, _ = binding.hip_bispectrum(_dev(p2), None, _dev(r2), L, R0, edges, 4, "mixed")
    assert _err(B2, B) < 2e-4


def test_bispectrum_argument_checks():
    pos, w, rnd, L, R0 = _case(N=100)
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    with pytest.raises(binding.HipError):
        binding.hip_bispectrum(pos, None, rnd, L, R0, edges, 5, "mixed")
    with pytest.raises(binding.HipError):
        binding.hip_bispectrum(pos, None, rnd, L, 31.0, edges, 4, "mixed")
    with pytest.raises(binding.HipError):
        binding.hip_bispectrum(pos, None, rnd, L, R0, catalogs.linear_edges(0.3, 2.4, 40), 4, "fp64")
    bad = rnd.copy()
    bad[5, 0] = np.inf
    with pytest.raises(binding.HipError) as ei:
        binding.hip_bispectrum(pos, None, bad, L, R0, edges, 4, "mixed")
    assert ei.value.status == binding.HIP_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bispectrum_analytic_ddr2_matches_oracle(prec):
    # the random-free estimator (App. A): data primaries plus the E^II pair sum to
    # 2 R0; the oracle takes the pair sum inside the p integral over exact pair
    # distances, the library over a 16384-bin moment histogram (third-order in the
    # bin width) with coarser (still converged) quadrature
    L, R0 = 60.0, 12.0
    pos, w = catalogs.thomas(600, L, 24, 1.5, seed=49, background_frac=0.3, weights="u05_15")
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    key = "analytic"
    if key not in _cache:
        _cache[key] = oracle.bispectrum_analytic(pos.astype(np.float64), w.astype(np.float64), L, R0, edges, 4)
    Bref, info = _cache[key]
    B, nd = binding.hip_bispectrum_analytic(_dev(pos), _dev(w), L, R0, edges, 4, prec)
    slack = 0 if prec == "fp64" else max(2, int(2e-6 * info["npairs_data"]))
    assert abs(nd - info["npairs_data"]) <= slack
    assert _err(B, Bref) < {"fp64": 1e-7, "mixed": 1e-4}[prec], _err(B, Bref)


def test_bispectrum_analytic_rejects_large_R0():
    pos, w, rnd, L, R0 = _case(N=200)
    edges = catalogs.linear_edges(0.3, 2.4, 12)
    with pytest.raises(binding.HipError) as ei:
        binding.hip_bispectrum_analytic(pos, None, L, 0.26 * L, edges, 4, "mixed")
    assert ei.value.status == binding.HIP_ERR_RANGE


# ------------------------------------------------ anisotropic bispectrum ----
def _aniso_case():
    # z-displaced clustering: the L > 0 components about zhat are far from zero
    L, R0 = 50.0, 10.0
    pos, w = catalogs.thomas(800, L, 32, 1.5, seed=71, background_frac=0.2, los_sigma=2.5, weights="u05_15")
    rnd = catalogs.uniform(2400, L, seed=72)
    return pos, w, rnd, L, R0


def test_bispectrum_aniso_parity():
    # every (l1, l2, L) combination against the oracle's per-primary Wigner-3j form
    pos, w, rnd, L, R0 = _aniso_case()
    edges = catalogs.linear_edges(0.3, 2.0, 9)  # 9 bins: the Gram's 4 x 4 tiles have a ragged edge
    Bref, info = oracle.bispectrum_aniso(pos.astype(np.float64), w.astype(np.float64), rnd.astype(np.float64),
                                         L, R0, edges)
    assert tuple(binding.ANISO_COMBOS) == tuple(oracle.ANISO_COMBOS)
    B, (nd, nr) = binding.hip_bispectrum_aniso(_dev(pos), _dev(w), _dev(rnd), L, R0, edges)
    slack = max(2, int(2e-6 * info["npairs_data"]))
    assert abs(nd - info["npairs_data"]) <= slack and abs(nr - info["npairs_rand"]) <= slack
    # the L > 0 components carry signal (relative to the monopole) in this catalog
    big = max(np.max(np.abs(Bref[c])) for c, (_, _, Lc) in enumerate(oracle.ANISO_COMBOS) if Lc > 0)
    assert big > 1e-2 * np.max(np.abs(Bref[0]))
    assert _err(B, Bref, "aniso") < TOL["mixed"]


def test_bispectrum_aniso_l0_matches_isotropic_path():
    # (l, l, 0) = (-1)^l sqrt(2l+1) B_l: the matching-m Gram and the tensor-core contraction of
    # the isotropic path give the same primary sums
    pos, w, rnd, L, R0 = _case(seed=43, N=2000, weights="u05_15")
    edges = catalogs.linear_edges(0.3, 2.4, 15)
    dpos, dw, drnd = _dev(pos), _dev(w), _dev(rnd)
    Bi, _ = binding.hip_bispectrum(dpos, dw, drnd, L, R0, edges, 4, "mixed")
    Ba, _ = binding.hip_bispectrum_aniso(dpos, dw, drnd, L, R0, edges)
    for l in range(5):
        c = binding.ANISO_COMBOS.index((l, l, 0))
        ref = (-1) ** l * np.sqrt(2 * l + 1) * Bi[l]
        assert np.max(np.abs(Ba[c] - ref)) < 1e-5 * np.max(np.abs(ref)), l
