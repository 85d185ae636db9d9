"""The random subsample of Sec. 9 (hip_subsample) against the oracle's SplitMix64
selection: the kept set must be bit-exact, and the power spectrum of the
subsample must equal the oracle's on the oracle-selected subsample."""
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
