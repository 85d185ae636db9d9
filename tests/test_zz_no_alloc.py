"""The allocation-free power-spectrum entry point (hip_power_noalloc).

Some callers cannot allocate device memory while they run (a host application
whose own memory pool has already reserved the device's memory, or a service
that must fix its peak device footprint up front); this entry point serves them
from a static device array.  Like hip_power it is eager and synchronises the
caller's stream before it returns.  Checked here through the C ABI against hip_power on two calls in
a row (the array keeps the previous call's contents, so the second call also
checks that everything that must start at zero is cleared), with the mixed-path
tolerance of the other tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _err(P, Pref, what=""):
    # the asserted metric and its two companions are printed (run with -s)
    return parity_metrics.report("P", P, Pref, what)["floored"]


def test_noalloc_matches_hip_power_twice():
    import torch
    L, R0 = 200.0, 20.0
    pos, w = catalogs.thomas(60_000, L, 1500, 1.5, seed=77, los_sigma=2.0, weights="u05_15")
    edges = catalogs.linear_edges(0.1, 3.0, 60)
    dpos, dw = torch.from_numpy(pos).cuda(), torch.from_numpy(w).cuda()
    Pref, DDref, nref = binding.hip_power(dpos, dw, L, R0, edges, 4, 2, "mixed")
    for _ in range(2):
        P, DD, n = binding.hip_power_noalloc(dpos, dw, L, R0, edges, 4, 2)
        assert n == nref
        assert _err(P, Pref) < 1e-5
        assert _err(DD, DDref) < 1e-5
    # host inputs and a primary range go through the same static array
    P2, _, n2 = binding.hip_power_noalloc(pos, w, L, R0, edges, 4, 2, prim_range=(100, 5000))
    Pr, _, nr = binding.hip_power(pos, w, L, R0, edges, 4, 2, "mixed", prim_range=(100, 5000))
    assert n2 == nr
    assert _err(P2, Pr) < 1e-5


def test_noalloc_rejects_oversized_call():
    # host positions are staged in the array too: about 36 bytes per particle
    cap = binding.load().hip_noalloc_capacity()
    n = cap // 36 + 1000
    pos = np.zeros((n, 3), np.float32)
    pos[:, 0] = np.linspace(0, 99, n)
    with pytest.raises(binding.HipError) as ei:
        binding.hip_power_noalloc(pos, None, 100.0, 10.0, catalogs.linear_edges(0.1, 1.0, 5))
    assert ei.value.status == binding.HIP_ERR_RANGE
    assert "bytes" in str(ei.value)


def test_noalloc_device_input_limit():
    # device-resident inputs need about 24 bytes per particle: just above the
    # limit the call is refused, well below it the call runs
    import torch
    cap = binding.load().hip_noalloc_capacity()
    edges = catalogs.linear_edges(0.1, 1.0, 5)
    n_big = cap // 24 + 1000
    big = torch.zeros((n_big, 3), dtype=torch.float32, device="cuda")
    big[:, 0] = torch.linspace(0, 99, n_big, device="cuda")
    with pytest.raises(binding.HipError) as ei:
        binding.hip_power_noalloc(big, None, 100.0, 10.0, edges)
    assert ei.value.status == binding.HIP_ERR_RANGE
    assert "bytes" in str(ei.value)
    del big
    n_ok = cap // 24 - (1 << 18)
    pos = torch.rand((n_ok, 3), dtype=torch.float32, device="cuda") * 100.0
    P, _, n = binding.hip_power_noalloc(pos, None, 100.0, 2.0, edges, 0, 2)
    assert np.all(np.isfinite(P)) and n > 0
