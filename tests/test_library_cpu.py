"""CPU checks of the CUDA library: it builds, loads without a GPU, exports every
symbol its header declares, validates arguments on the host, and its per-pair
special-function code (compiled for the host from the same source) agrees with
the oracle's D_l (App. C) -- no kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2005_01739_gb300 import binding, build, catalogs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hip_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "hip_power" in names and "hip_status_string" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in range(0, -7, -1):
        assert lib.hip_status_string(code).decode() != "unknown status"


def _call(lib, **kw):
    a = dict(pos=np.zeros((4, 3), np.float32), w=None, N=4, L=100.0, R0=10.0, edges=np.array([0.1, 0.2]),
             n_k=1, ell_max=4, los=2, prec=1, p0=0, p1=4)
    a.update(kw)
    P = np.zeros(3 * max(1, a["n_k"]))
    vp = ctypes.c_void_p
    pos = None if a["pos"] is None else a["pos"].ctypes.data_as(vp)
    return lib.hip_power(pos, None, a["N"], a["L"], a["R0"], 0, a["edges"].ctypes.data_as(vp), a["n_k"],
                         a["ell_max"], a["los"], a["prec"], a["p0"], a["p1"], P.ctypes.data_as(vp), None, None, None)


@pytest.mark.parametrize("kw,code", [
    (dict(N=0), binding.HIP_ERR_ARG),
    (dict(pos=None), binding.HIP_ERR_ARG),
    (dict(ell_max=3), binding.HIP_ERR_ARG),
    (dict(los=3), binding.HIP_ERR_ARG),
    (dict(prec=7), binding.HIP_ERR_ARG),
    (dict(R0=50.0), binding.HIP_ERR_RANGE),
    (dict(R0=-1.0), binding.HIP_ERR_RANGE),
    (dict(L=0.0), binding.HIP_ERR_RANGE),
    (dict(edges=np.array([0.2, 0.1])), binding.HIP_ERR_RANGE),
    (dict(edges=np.array([-0.1, 0.1])), binding.HIP_ERR_RANGE),
    (dict(edges=np.array([0.1, np.nan])), binding.HIP_ERR_RANGE),
    (dict(n_k=300, edges=np.linspace(0.1, 1, 301)), binding.HIP_ERR_RANGE),
    (dict(p0=3, p1=2), binding.HIP_ERR_RANGE),
    (dict(p1=5), binding.HIP_ERR_RANGE),
])
def test_argument_validation_on_host(lib, kw, code):
    assert _call(lib, **kw) == code


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_kernel_F_fp64_matches_oracle(lib, l):
    # F_l(u) = D_l(u)/u^3 as the FP64 kernels evaluate it, across every branch
    # (series below 2.5, Si series to 12, fitted auxiliaries above).
    us = np.concatenate([np.geomspace(1e-4, 2.5, 60), np.linspace(2.5, 12, 80), np.linspace(12, 2000, 200)])
    for u in us:
        ref = oracle.dhat(l, u) / u ** 3
        env = 1.0 / 3.0 if u < 1 else 1.0 / u ** 2
        assert abs(binding.debug_F("fp64", l, u) - ref) < 5e-12 * env, (l, u)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_kernel_F_fp32_error_budget(lib, l):
    # FP32 path: series below u = 6, closed forms with fitted Si auxiliaries
    # above.  The bound is a few FP32 ulps of the envelope plus the rounding of
    # the argument u itself (phase error ~ u * 2^-24).
    us = np.concatenate([np.geomspace(1e-4, 6, 80), np.linspace(6, 60, 200), np.linspace(60, 1500, 200)])
    for u in us:
        ref = oracle.dhat(l, u) / u ** 3
        env = 1.0 / 3.0 if u < 1 else 1.0 / u ** 2
        bound = env * (4e-6 + 1.2e-7 * u)
        assert abs(binding.debug_F("mixed", l, u) - ref) < bound, (l, u)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_kernel_F_bispectrum_error_budget(lib, l):
    # The bispectrum pass's FP32 F_l: a degree-6 polynomial in u^2 below u = 4,
    # closed forms with degree-10 Si auxiliaries above (host build of the same
    # code), against the oracle's D_l.  Same envelope as the power path, with the
    # bispectrum's looser constant (its tolerance is 1e-4, not 1e-5).
    us = np.concatenate([np.geomspace(1e-4, 4, 80), np.linspace(4, 60, 200), np.linspace(60, 1500, 200)])
    worst = 0.0
    for u in us:
        ref = oracle.dhat(l, u) / u ** 3
        env = 1.0 / 3.0 if u < 1 else 1.0 / u ** 2
        err = abs(binding.debug_Fb(l, u) - ref)
        assert err < env * (2e-6 + 1.2e-7 * u), (l, u, err / env)
        worst = max(worst, err / env / (1.0 + u))
    assert worst > 0.0  # the FP32 path is not secretly exact


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("variant,lo,hi", [("series", 1e-4, 6.0), ("fit", 6.0, 3000.0), ("asym", 24.0, 3000.0)])
def test_kernel_D_fp32_branches(lib, variant, lo, hi, l):
    # D_l(u) = u^3 F_l(u) as the FP32 pair kernels accumulate it, each branch on
    # its whole domain: the series below 6, the closed form with fitted Si
    # auxiliaries (any u >= 6: the kernel uses it whenever a warp straddles
    # u = 24) and with the four-term asymptotic auxiliaries (u >= 24).  sin and
    # cos are correctly rounded here, so the bound is on the D-form arithmetic:
    # a few FP32 ulps of the envelope u^3 (1/3 if u < 1 else 1/u^2), more for the
    # alternating series near its upper end.
    us = np.geomspace(lo, hi, 400) if variant == "series" else np.linspace(lo, hi, 600)
    bound = 3e-6 if variant == "series" else 5e-7
    for u in us:
        uf = float(np.float32(u))
        env = uf ** 3 * (1.0 / 3.0 if uf < 1 else 1.0 / uf ** 2)
        assert abs(binding.debug_D(variant, l, uf) - oracle.dhat(l, uf)) < bound * env, (variant, l, uf)


def test_power_pair_pass_choice():
    # moment pass while n_c = max(8, ceil(R0 k_max / 4)) <= 256, the direct pass beyond
    assert binding.power_pair_pass(50.0, 5.0) == 1
    assert binding.power_pair_pass(50.0, 5.0, "fp64") == 1
    assert binding.power_pair_pass(20.0, 51.2) == 1  # R0 k_max = 1024: n_c = 256
    assert binding.power_pair_pass(20.0, 51.3) == 0
    assert binding.power_pair_pass(17.3, 14.0) == 1
    with pytest.raises(ValueError):
        binding.power_pair_pass(-1.0, 5.0)
    with pytest.raises(ValueError):
        binding.power_pair_pass(10.0, 0.0)


def test_subsample_argument_checks(lib):
    # rejected before any device work
    vp = ctypes.c_void_p
    pos = np.zeros((4, 3), np.float32)
    out = np.zeros((4, 3), np.float32)
    n = ctypes.c_int64(0)
    args = lambda f: (pos.ctypes.data_as(vp), None, 4, f, 1, out.ctypes.data_as(vp), None, ctypes.byref(n), None)
    assert lib.hip_subsample(*args(1.5)) == binding.HIP_ERR_RANGE
    assert lib.hip_subsample(*args(float("nan"))) == binding.HIP_ERR_RANGE
    assert lib.hip_subsample(None, None, 4, 0.5, 1, out.ctypes.data_as(vp), None, ctypes.byref(n), None) == \
        binding.HIP_ERR_ARG
    assert lib.hip_subsample(pos.ctypes.data_as(vp), None, -1, 0.5, 1, out.ctypes.data_as(vp), None,
                             ctypes.byref(n), None) == binding.HIP_ERR_ARG


def test_window_omega_argument_checks(lib):
    # rejected on the host, before any device work
    edges = catalogs.linear_edges(0.3, 3.0, 5)
    for args, code in [((edges, -1.0, 4, [0.1]), binding.HIP_ERR_RANGE),
                       ((edges, 10.0, 5, [0.1]), binding.HIP_ERR_ARG),
                       ((edges, 10.0, 4, [-0.1]), binding.HIP_ERR_RANGE),
                       ((edges, 10.0, 4, [float("nan")]), binding.HIP_ERR_RANGE),
                       ((edges[::-1], 10.0, 4, [0.1]), binding.HIP_ERR_RANGE)]:
        with pytest.raises(binding.HipError) as ei:
            binding.hip_window_omega(*args)
        assert ei.value.status == code
