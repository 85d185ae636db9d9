"""The random subsample of Sec. 9 (hip_subsample) against the oracle's SplitMix64
selection: the kept set must be bit-exact, and the power spectrum of the
subsample must equal the oracle's on the oracle-selected subsample.  The seeded
random catalog (hip_uniform_randoms, hip_bispectrum_seeded) against the oracle's
generator: bit-exact positions, and the seeded bispectrum equal to the one with
the same randoms passed in."""
import numpy as np
import pytest

import oracle
import parity_metrics
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


@pytest.mark.parametrize("N,fraction,seed", [(1, 1.0, 3), (4095, 0.5, 11), (4096 * 3 + 17, 0.1, 2 ** 63 + 5),
                                             (250_000, 0.01, 42), (100_000, 0.0, 1), (70_001, 1.0, 9)])
def test_selection_is_bit_exact(N, fraction, seed):
    import torch
    rng = np.random.default_rng(N)
    pos = rng.uniform(0, 100, (N, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, N).astype(np.float32)
    mask = oracle.subsample_mask(N, fraction, seed)
    # device inputs with weights
    ps, ws = binding.hip_subsample(torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda(), fraction, seed)
    assert ps.shape[0] == int(mask.sum())
    assert np.array_equal(ps.cpu().numpy(), pos[mask]) and np.array_equal(ws.cpu().numpy(), w[mask])
    # host inputs, no weights
    ph, wh = binding.hip_subsample(pos, None, fraction, seed)
    assert wh is None and np.array_equal(ph, pos[mask])


def test_subsampled_power_spectrum_matches_oracle():
    # the f_sub workflow: subsample on the device, then the estimator on the subsample
    import torch
    pos, w = catalogs.thomas(20000, 60.0, 400, 1.0, seed=77, background_frac=0.2, weights="u05_15")
    L, R0, edges = 60.0, 10.0, catalogs.linear_edges(0.3, 3.0, 20)
    ps, ws = binding.hip_subsample(torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda(), 0.2, 2020)
    P, _, n = binding.hip_power(ps, ws, L, R0, edges, 4, 2, "mixed")
    mask = oracle.subsample_mask(len(pos), 0.2, 2020)
    p64, w64 = pos[mask].astype(np.float64), w[mask].astype(np.float64)
    DD, nref = oracle.power_pair_sum(p64, w64, L, R0, edges, 4, 2)
    Pref = oracle.power_from_pairs(DD, float(w64.sum()), L, oracle.window_transform_binned(edges, R0))
    assert abs(n - nref) <= 2
    floor = 1e-2 * np.max(np.abs(Pref[0]))
    scale = np.maximum(np.maximum(np.abs(Pref), np.abs(Pref[0])[None, :]), floor)
    assert float(np.max(np.abs(P - Pref) / scale)) < 1e-5


def test_bad_fraction():
    pos = np.zeros((10, 3), np.float32)
    for f in (-0.1, 1.5, float("nan")):
        with pytest.raises(binding.HipError) as ei:
            binding.hip_subsample(pos, None, f, 1)
        assert ei.value.status == binding.HIP_ERR_RANGE


@pytest.mark.parametrize("n_r,L,seed", [(1, 1.0, 0), (5, 1000.0, 7), (100_003, 777.77, 2 ** 64 - 1)])
def test_uniform_randoms_bit_exact(n_r, L, seed):
    import torch
    ref = oracle.uniform_randoms(n_r, L, seed)
    d = binding.hip_uniform_randoms(n_r, L, seed, device="cuda")
    h = binding.hip_uniform_randoms(n_r, L, seed)
    assert np.array_equal(d.cpu().numpy(), ref) and np.array_equal(h, ref)


def test_uniform_randoms_rejects():
    import ctypes
    lib = binding.load()
    buf = np.empty(3, np.float32)
    for n_r, L, status in ((1, 0.0, binding.HIP_ERR_RANGE), (1, float("inf"), binding.HIP_ERR_RANGE),
                           (1, float("nan"), binding.HIP_ERR_RANGE), (-1, 1.0, binding.HIP_ERR_ARG)):
        assert lib.hip_uniform_randoms(buf.ctypes.data_as(ctypes.c_void_p), n_r, L, 1, None) == status
    assert lib.hip_uniform_randoms(None, 1, 1.0, 1, None) == binding.HIP_ERR_ARG


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_bispectrum_seeded_equals_explicit_randoms(prec):
    # the seeded entry point is hip_bispectrum on hip_uniform_randoms' catalog; against the oracle too
    import torch
    pos, w = catalogs.thomas(2500, 70.0, 60, 1.0, seed=515, background_frac=0.3, weights="u05_15")
    L, R0, edges, n_r, seed = 70.0, 14.0, catalogs.linear_edges(0.3, 2.0, 10), 7500, 99
    dpos, dw = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda()
    Bs, (nds, nrs) = binding.hip_bispectrum_seeded(dpos, dw, n_r, seed, L, R0, edges, 4, prec)
    rnd = oracle.uniform_randoms(n_r, L, seed)
    Be, (nde, nre) = binding.hip_bispectrum(dpos, dw, torch.from_numpy(rnd).cuda(), L, R0, edges, 4, prec)
    assert (nds, nrs) == (nde, nre)
    # the same inputs through the same kernels: equal up to the order of the atomic adds
    # (FP32 sums in the mixed path, FP64 in the plain one)
    assert np.max(np.abs(Bs - Be)) <= {"mixed": 1e-6, "fp64": 1e-12}[prec] * np.max(np.abs(Be))
    Bref, _ = oracle.bispectrum(pos.astype(np.float64), w.astype(np.float64), rnd.astype(np.float64), L, R0, edges, 4)
    err = parity_metrics.report("B", Bs, Bref, "seeded " + prec)["floored"]
    assert err < {"mixed": 1e-4, "fp64": 1e-10}[prec]
