"""The binned window kernel omega^a_l(p) (Eq. omega-ell-a-def) through the C ABI
(hip_window_omega) against the oracle's own quadrature of the same integral."""
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


@pytest.mark.parametrize("R0,edges", [(40.0, catalogs.linear_edges(0.3, 3.0, 25)),
                                      (12.0, np.concatenate([[0.0], np.geomspace(0.05, 4.0, 17)]))])
def test_omega_matches_oracle(R0, edges):
    # p from 0 through the bins to beyond k_max, including the bin edges themselves
    p = np.unique(np.concatenate([[0.0, 1e-3], np.linspace(0.0, 1.5 * edges[-1], 61), edges]))
    om = binding.hip_window_omega(edges, R0, 4, p)
    assert om.shape == (5, len(edges) - 1, len(p))
    for l in range(5):
        ref = oracle.omega_binned(l, edges, R0, p)
        err = float(np.max(np.abs(om[l] - ref)) / np.max(np.abs(ref)))
        assert err < 1e-10, (l, err)
