"""Thin ctypes binding of libhipster_gb300.so (argument marshalling only).

Every computation happens in the CUDA library; this module converts arrays to
pointers, checks the returned status and raises on failure.  There is no CPU
fallback: if the library is missing or fails to load, calls raise RuntimeError.

Inputs may be numpy arrays (host memory) or CUDA torch tensors (device memory,
float32, contiguous); the library detects which per pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HIP_OK, HIP_ERR_ARG, HIP_ERR_RANGE, HIP_ERR_NONFINITE, HIP_ERR_CUDA, HIP_ERR_NOMEM, HIP_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "mixed": 1}
HIP_MAX_BINS = 255

_lock = threading.Lock()
_lib = None


class HipCatalog(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("w", ctypes.c_void_p), ("N", ctypes.c_int64), ("L", ctypes.c_double),
                ("R0", ctypes.c_double), ("k_edges", ctypes.c_void_p), ("n_k", ctypes.c_int),
                ("ell_max", ctypes.c_int), ("los_axis", ctypes.c_int), ("prim_begin", ctypes.c_int64),
                ("prim_end", ctypes.c_int64), ("P_out", ctypes.c_void_p), ("DD_out", ctypes.c_void_p),
                ("npairs_out", ctypes.c_void_p)]


class HipBCatalog(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("w", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("rand_pos", ctypes.c_void_p), ("N_r", ctypes.c_int64), ("L", ctypes.c_double),
                ("R0", ctypes.c_double), ("k_edges", ctypes.c_void_p), ("n_k", ctypes.c_int), ("lmax", ctypes.c_int),
                ("B_out", ctypes.c_void_p), ("npairs_out", ctypes.c_void_p)]


class HipError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the CUDA library (built by ``build.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
        L = ctypes.CDLL(p)
        i64, d, i, P = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.hip_power.restype = i
        L.hip_power.argtypes = [P, P, i64, d, d, i, P, i, i, i, i, i64, i64, P, P, P, P]
        L.hip_bispectrum.restype = i
        L.hip_bispectrum.argtypes = [P, P, i64, P, i64, d, d, i, P, i, i, i, P, P, P]
        L.hip_bispectrum_aniso.restype = i
        L.hip_bispectrum_aniso.argtypes = [P, P, i64, P, i64, d, d, i, P, i, P, P, P]
        L.hip_power_noalloc.restype = i
        L.hip_power_noalloc.argtypes = [P, P, i64, d, d, i, P, i, i, i, i64, i64, P, P, P, P]
        L.hip_power_from_pairs.restype = i
        L.hip_power_from_pairs.argtypes = [P, i, i, d, d, i, P, d, P, P]
        L.hip_window_omega.restype = i
        L.hip_window_omega.argtypes = [P, i, d, i, P, i, P, P]
        L.hip_subsample.restype = i
        L.hip_subsample.argtypes = [P, P, i64, d, ctypes.c_uint64, P, P, P, P]
        L.hip_uniform_randoms.restype = i
        L.hip_uniform_randoms.argtypes = [P, i64, d, ctypes.c_uint64, P]
        L.hip_bispectrum_seeded.restype = i
        L.hip_bispectrum_seeded.argtypes = [P, P, i64, i64, ctypes.c_uint64, d, d, i, P, i, i, i, P, P, P]
        L.hip_noalloc_capacity.restype = ctypes.c_size_t
        L.hip_noalloc_capacity.argtypes = []
        L.hip_noalloc_message.restype = ctypes.c_char_p
        L.hip_noalloc_message.argtypes = []
        L.hip_batch_plan_create.restype = i
        L.hip_batch_plan_create.argtypes = [P, i, i, ctypes.POINTER(ctypes.c_void_p), P]
        L.hip_batch_plan_run.restype = i
        L.hip_batch_plan_run.argtypes = [P, P]
        L.hip_batch_plan_destroy.restype = None
        L.hip_batch_plan_destroy.argtypes = [P]
        L.hip_batch_plan_launches.restype = i
        L.hip_batch_plan_launches.argtypes = [P]
        L.hip_power_batched.restype = i
        L.hip_power_batched.argtypes = [P, i, i, P]
        L.hip_batch_message.restype = ctypes.c_char_p
        L.hip_batch_message.argtypes = []
        L.hip_batch_plan_tune.restype = i
        L.hip_batch_plan_tune.argtypes = [P, P, P, P]
        L.hip_batch_plan_tune_kernel.restype = i
        L.hip_batch_plan_tune_kernel.argtypes = [P, P, P, P, P]
        L.hip_batch_plan_shape.restype = None
        L.hip_batch_plan_shape.argtypes = [P, P, P, P]
        L.hip_bispectrum_analytic.restype = i
        L.hip_bispectrum_analytic.argtypes = [P, P, i64, d, d, i, P, i, i, i, P, P, P]
        L.hip_bispectrum_batched.restype = i
        L.hip_bispectrum_batched.argtypes = [P, i, i, P]
        L.hip_bispectrum_partial.restype = i
        L.hip_bispectrum_partial.argtypes = [P, P, i64, P, i64, d, d, i, P, i, i, i, P, P, P, P]
        L.hip_status_string.restype = ctypes.c_char_p
        L.hip_status_string.argtypes = [i]
        L.hip_last_error.restype = ctypes.c_char_p
        L.hip_last_error.argtypes = []
        L.hip_debug_F.restype = d
        L.hip_power_pair_pass.argtypes = [d, d, i]
        L.hip_power_pair_pass.restype = i
        L.hip_debug_F.argtypes = [i, i, d]
        L.hip_debug_D.restype = d
        L.hip_debug_D.argtypes = [i, i, d]
        L.hip_debug_Fb.restype = d
        L.hip_debug_Fb.argtypes = [i, d]
        L.hip_debug_F_array.restype = None
        L.hip_debug_F_array.argtypes = [i, i, P, P, i64]
        L.hip_debug_bk_caps.restype = None
        L.hip_debug_bk_caps.argtypes = [i, i]
        L.hip_debug_bk_mode.restype = None
        L.hip_debug_bk_mode.argtypes = [i, i]
        L.hip_bispectrum_stage_times.restype = i
        L.hip_bispectrum_stage_times.argtypes = [P, i]
        L.hip_set_profiling.restype = None
        L.hip_set_profiling.argtypes = [i]
        L.hip_stage_times.restype = i
        L.hip_stage_times.argtypes = [P, i]
        _lib = L
        return L


def _check(L, rc: int, what: str):
    if rc != HIP_OK:
        msg = L.hip_status_string(rc).decode()
        extra = L.hip_last_error().decode()
        raise HipError(rc, f"{what}: {msg}" + (f" ({extra})" if extra else ""))


def _ptr(x):
    """(pointer, keepalive) for a numpy array or a torch tensor (host or CUDA)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):  # torch tensor
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("tensor inputs must be contiguous float32")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    return a.ctypes.data_as(ctypes.c_void_p), a


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def hip_power(pos, w, L, R0, k_edges, ell_max=4, los_axis=2, prec="mixed", prim_range=None, stream=None):
    """P^a_l (Sec. 3 binned estimator) of one periodic catalog.

    Returns (P [n_ell, n_k], DD [n_ell, n_k], npairs) as float64 numpy arrays and
    the number of ordered pairs counted."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    n_ell = ell_max // 2 + 1
    P = np.zeros((n_ell, n_k))
    DD = np.zeros((n_ell, n_k))
    npairs = ctypes.c_int64(0)
    p0, p1 = (0, n) if prim_range is None else (int(prim_range[0]), int(prim_range[1]))
    rc = lib.hip_power(pp, wp, n, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p), n_k,
                       int(ell_max), int(los_axis), PREC[prec], p0, p1, P.ctypes.data_as(ctypes.c_void_p),
                       DD.ctypes.data_as(ctypes.c_void_p), ctypes.byref(npairs), _stream_handle(stream))
    _check(lib, rc, "hip_power")
    del keep_p, keep_w
    return P, DD, int(npairs.value)


def hip_power_from_pairs(DD, L, R0, k_edges, S1, stream=None):
    """P^a_l from summed ordered pair sums DD [n_ell, n_k] (e.g. the DD of
    hip_power calls over disjoint primary ranges, added up); S1 = the sum of the
    whole catalog's weights.  Returns P [n_ell, n_k] float64."""
    lib = load()
    DD = np.ascontiguousarray(np.asarray(DD, dtype=np.float64))
    n_ell, n_k = DD.shape
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    P = np.zeros((n_ell, n_k))
    rc = lib.hip_power_from_pairs(DD.ctypes.data_as(ctypes.c_void_p), n_k, 2 * (n_ell - 1), float(L), float(R0), 0,
                                  edges.ctypes.data_as(ctypes.c_void_p), float(S1), P.ctypes.data_as(ctypes.c_void_p),
                                  _stream_handle(stream))
    _check(lib, rc, "hip_power_from_pairs")
    return P


def hip_window_omega(k_edges, R0, lmax, p, stream=None):
    """omega^a_l(p) (Eq. omega-ell-a-def) for l = 0..lmax: [lmax+1, n_k, len(p)] float64."""
    lib = load()
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    pp = np.ascontiguousarray(np.atleast_1d(np.asarray(p, dtype=np.float64)))
    n_k = len(edges) - 1
    out = np.zeros((int(lmax) + 1, n_k, len(pp)))
    rc = lib.hip_window_omega(edges.ctypes.data_as(ctypes.c_void_p), n_k, float(R0), int(lmax),
                              pp.ctypes.data_as(ctypes.c_void_p), len(pp), out.ctypes.data_as(ctypes.c_void_p),
                              _stream_handle(stream))
    _check(lib, rc, "hip_window_omega")
    return out


def hip_subsample(pos, w, fraction, seed, stream=None):
    """Random subsample of a catalog (hip_subsample): keeps particle i iff its
    SplitMix64 variate is below `fraction`, in input order.  Outputs are of the
    inputs' kind (torch tensors on the same device, else numpy): (pos [n, 3],
    w [n] or None)."""
    lib = load()
    n = int(pos.shape[0])
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    if hasattr(pos, "data_ptr"):
        import torch
        pos_out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        w_out = None if w is None else torch.empty((n,), dtype=torch.float32, device=pos.device)
    else:
        pos_out = np.empty((n, 3), dtype=np.float32)
        w_out = None if w is None else np.empty((n,), dtype=np.float32)
    po, _ = _ptr(pos_out)
    wo = None if w_out is None else _ptr(w_out)[0]
    n_out = ctypes.c_int64(0)
    rc = lib.hip_subsample(pp, wp, n, float(fraction), int(seed) & 0xFFFFFFFFFFFFFFFF, po, wo, ctypes.byref(n_out),
                           _stream_handle(stream))
    _check(lib, rc, "hip_subsample")
    del keep_p, keep_w
    m = int(n_out.value)
    return pos_out[:m], (None if w_out is None else w_out[:m])


def hip_power_noalloc(pos, w, L, R0, k_edges, ell_max=4, los_axis=2, prim_range=None, stream=None):
    """hip_power (mixed precision) with its scratch in the library's static device
    array instead of allocated memory.  Same returns as hip_power."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    n_ell = ell_max // 2 + 1
    P = np.zeros((n_ell, n_k))
    DD = np.zeros((n_ell, n_k))
    npairs = ctypes.c_int64(0)
    p0, p1 = (0, n) if prim_range is None else (int(prim_range[0]), int(prim_range[1]))
    rc = lib.hip_power_noalloc(pp, wp, n, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p), n_k,
                               int(ell_max), int(los_axis), p0, p1, P.ctypes.data_as(ctypes.c_void_p),
                               DD.ctypes.data_as(ctypes.c_void_p), ctypes.byref(npairs), _stream_handle(stream))
    if rc != HIP_OK:
        raise HipError(rc, f"hip_power_noalloc: {lib.hip_status_string(rc).decode()} "
                           f"({lib.hip_noalloc_message().decode()})")
    del keep_p, keep_w
    return P, DD, int(npairs.value)


class BatchPlan:
    """Batched power spectra of many catalogs (hip_batch_plan_*): the cell builds,
    one persistent pair-kernel launch over all catalogs and the FP64 finalize,
    recorded once into a CUDA graph and replayed by run().

    `catalogs` is a list of dicts with keys pos, w (or None), L, R0, edges and
    optionally ell_max (4), los_axis (2), prim_range.  After run(), .results[i] is
    (P, DD, npairs) of catalog i."""

    def __init__(self, catalogs, prec="mixed", stream=None):
        self._lib = load()
        self._keep = []
        n = len(catalogs)
        self._cats = (HipCatalog * n)()
        self.results = []
        for i, c in enumerate(catalogs):
            pp, kp = _ptr(c["pos"])
            wp, kw = _ptr(c.get("w"))
            edges = np.ascontiguousarray(np.asarray(c["edges"], dtype=np.float64))
            N = int(c["pos"].shape[0])
            ell_max = int(c.get("ell_max", 4))
            n_k = len(edges) - 1
            P = np.zeros((ell_max // 2 + 1, n_k))
            DD = np.zeros_like(P)
            npairs = np.zeros(1, dtype=np.int64)
            p0, p1 = c.get("prim_range", (0, N))
            self._keep += [kp, kw, edges, P, DD, npairs]
            self._cats[i] = HipCatalog(pp.value if pp is not None else None, wp.value if wp is not None else None,
                                       N, float(c["L"]), float(c["R0"]), edges.ctypes.data, n_k, ell_max,
                                       int(c.get("los_axis", 2)), int(p0), int(p1), P.ctypes.data, DD.ctypes.data,
                                       npairs.ctypes.data)
            self.results.append((P, DD, npairs))
        self._plan = ctypes.c_void_p()
        rc = self._lib.hip_batch_plan_create(ctypes.cast(self._cats, ctypes.c_void_p), n, PREC[prec],
                                             ctypes.byref(self._plan), _stream_handle(stream))
        if rc != HIP_OK:
            raise HipError(rc, f"hip_batch_plan_create: {self._lib.hip_status_string(rc).decode()} "
                               f"({self._lib.hip_batch_message().decode()})")

    @property
    def launches(self) -> int:
        return int(self._lib.hip_batch_plan_launches(self._plan))

    def run(self, stream=None):
        rc = self._lib.hip_batch_plan_run(self._plan, _stream_handle(stream))
        if rc != HIP_OK:
            raise HipError(rc, f"hip_batch_plan_run: {self._lib.hip_status_string(rc).decode()} "
                               f"({self._lib.hip_batch_message().decode()})")
        return [(P.copy(), DD.copy(), int(n[0])) for P, DD, n in self.results]

    def tune(self, stream=None):
        """Autotune the plan's cell shape (hip_batch_plan_tune): returns (chosen
        target particles per cell, 0 = cells R0 wide; {candidate: replay ms})."""
        chosen = ctypes.c_int(0)
        ms = (ctypes.c_float * 8)()
        rc = self._lib.hip_batch_plan_tune(self._plan, _stream_handle(stream), ctypes.byref(chosen), ms)
        if rc != 0:
            raise HipError(rc, f"hip_batch_plan_tune: {self._lib.hip_status_string(rc).decode()} "
                               f"({self._lib.hip_batch_message().decode()})")
        return int(chosen.value), dict(zip((4, 8, 16, 32, 64, 128, 256, 0), (float(x) for x in ms)))

    def tune_kernel(self, stream=None):
        """Autotune the moment pass's warps per CTA and fold period at the plan's cell
        occupancy (hip_batch_plan_tune_kernel): returns ((warps, fold) chosen,
        {(warps, fold): replay ms})."""
        w, f = ctypes.c_int(0), ctypes.c_int(0)
        ms = (ctypes.c_float * 6)()
        rc = self._lib.hip_batch_plan_tune_kernel(self._plan, _stream_handle(stream), ctypes.byref(w), ctypes.byref(f),
                                                  ms)
        if rc != 0:
            raise HipError(rc, f"hip_batch_plan_tune_kernel: {self._lib.hip_status_string(rc).decode()} "
                               f"({self._lib.hip_batch_message().decode()})")
        shapes = [(a, b) for a in (4, 8) for b in (4096, 8192, 16384)]
        return (int(w.value), int(f.value)), dict(zip(shapes, (float(x) for x in ms)))

    def shape(self):
        """(occ, warps, fold) of the plan (warps 0 = by occupancy, fold 0 = 16384)."""
        o, w, f = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._lib.hip_batch_plan_shape(self._plan, ctypes.byref(o), ctypes.byref(w), ctypes.byref(f))
        return int(o.value), int(w.value), int(f.value)

    def close(self):
        if self._plan:
            self._lib.hip_batch_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hip_power_batched(catalogs, prec="mixed", stream=None):
    """One-shot batched power spectra (plan, run, destroy)."""
    plan = BatchPlan(catalogs, prec, stream)
    try:
        return plan.run(stream)
    finally:
        plan.close()


def hip_bispectrum(pos, w, rand_pos, L, R0, k_edges, lmax=4, prec="mixed", stream=None):
    """B^ab_l (Sec. 4.5 summary estimator) of one periodic catalog with a random
    catalog for the DDR^II term.  Returns (B [lmax+1, n_k, n_k], (pairs from data
    primaries, pairs from random primaries))."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    nr = int(rand_pos.shape[0]) if hasattr(rand_pos, "shape") else len(rand_pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    rp, keep_r = _ptr(rand_pos)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    B = np.zeros((lmax + 1, n_k, n_k))
    npairs = (ctypes.c_int64 * 2)()
    rc = lib.hip_bispectrum(pp, wp, n, rp, nr, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p), n_k,
                            int(lmax), PREC[prec], B.ctypes.data_as(ctypes.c_void_p), npairs,
                            _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum")
    del keep_p, keep_w, keep_r
    return B, (int(npairs[0]), int(npairs[1]))


def hip_uniform_randoms(n_r, L, seed, device=None, stream=None):
    """Uniform random catalog [n_r, 3] float32 from SplitMix64 (hip_uniform_randoms):
    a torch tensor on `device` when given, else numpy."""
    lib = load()
    if device is not None:
        import torch
        out = torch.empty((int(n_r), 3), dtype=torch.float32, device=device)
    else:
        out = np.empty((int(n_r), 3), dtype=np.float32)
    po, keep = _ptr(out)
    rc = lib.hip_uniform_randoms(po, int(n_r), float(L), int(seed) & 0xFFFFFFFFFFFFFFFF, _stream_handle(stream))
    _check(lib, rc, "hip_uniform_randoms")
    del keep
    return out


def hip_bispectrum_seeded(pos, w, n_r, rand_seed, L, R0, k_edges, lmax=4, prec="mixed", stream=None):
    """hip_bispectrum with the random catalog hip_uniform_randoms(n_r, L, rand_seed)
    generated on the device.  Same returns as hip_bispectrum."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    B = np.zeros((lmax + 1, n_k, n_k))
    npairs = (ctypes.c_int64 * 2)()
    rc = lib.hip_bispectrum_seeded(pp, wp, n, int(n_r), int(rand_seed) & 0xFFFFFFFFFFFFFFFF, float(L), float(R0), 0,
                                   edges.ctypes.data_as(ctypes.c_void_p), n_k, int(lmax), PREC[prec],
                                   B.ctypes.data_as(ctypes.c_void_p), npairs, _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum_seeded")
    del keep_p, keep_w
    return B, (int(npairs[0]), int(npairs[1]))


ANISO_COMBOS = ((0, 0, 0), (0, 2, 2), (0, 4, 4), (1, 1, 0), (1, 1, 2), (1, 3, 2), (1, 3, 4), (2, 2, 0), (2, 2, 2),
                (2, 2, 4), (2, 4, 2), (2, 4, 4), (3, 3, 0), (3, 3, 2), (3, 3, 4), (4, 4, 0), (4, 4, 2), (4, 4, 4))


def hip_bispectrum_aniso(pos, w, rand_pos, L, R0, k_edges, stream=None):
    """Anisotropic B^ab_{l1 l2 L} about zhat (the 18 combinations of ANISO_COMBOS),
    mixed precision.  Returns (B [18, n_k, n_k], (data-primary pairs,
    random-primary pairs))."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    nr = int(rand_pos.shape[0]) if hasattr(rand_pos, "shape") else len(rand_pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    rp, keep_r = _ptr(rand_pos)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    B = np.zeros((len(ANISO_COMBOS), n_k, n_k))
    npairs = (ctypes.c_int64 * 2)()
    rc = lib.hip_bispectrum_aniso(pp, wp, n, rp, nr, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p),
                                  n_k, B.ctypes.data_as(ctypes.c_void_p), npairs, _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum_aniso")
    del keep_p, keep_w, keep_r
    return B, (int(npairs[0]), int(npairs[1]))


def hip_bispectrum_analytic(pos, w, L, R0, k_edges, lmax=4, prec="mixed", stream=None):
    """B^ab_l with the random-free DDR^II term (App. A; no random catalog).
    Returns (B [lmax+1, n_k, n_k], ordered (primary, data) pairs within R0)."""
    lib = load()
    n = int(pos.shape[0]) if hasattr(pos, "shape") else len(pos)
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    B = np.zeros((lmax + 1, n_k, n_k))
    npairs = (ctypes.c_int64 * 1)()
    rc = lib.hip_bispectrum_analytic(pp, wp, n, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p), n_k,
                                     int(lmax), PREC[prec], B.ctypes.data_as(ctypes.c_void_p), npairs,
                                     _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum_analytic")
    del keep_p, keep_w
    return B, int(npairs[0])


def hip_bispectrum_batched(catalogs, prec="mixed", stream=None):
    """Bispectra of many catalogs with one persistent kernel launch over all
    their primaries.  `catalogs`: dicts with pos, w (or None), rand, L, R0, edges
    and optionally lmax (default 4).  Returns a list of (B, (pairs from data
    primaries, pairs from random primaries)) in catalog order."""
    lib = load()
    n = len(catalogs)
    arr = (HipBCatalog * n)()
    keep, outs = [], []
    for i, c in enumerate(catalogs):
        pp, k1 = _ptr(c["pos"])
        wp, k2 = _ptr(c.get("w"))
        rp, k3 = _ptr(c["rand"])
        edges = np.ascontiguousarray(np.asarray(c["edges"], dtype=np.float64))
        n_k = len(edges) - 1
        lmax = int(c.get("lmax", 4))
        B = np.zeros((lmax + 1, n_k, n_k))
        npairs = np.zeros(2, dtype=np.int64)
        keep += [k1, k2, k3, edges]
        outs.append((B, npairs))
        arr[i] = HipBCatalog(pp.value, wp.value if wp is not None else None, int(c["pos"].shape[0]), rp.value,
                             int(c["rand"].shape[0]), float(c["L"]),
                             float(c["R0"]), edges.ctypes.data, n_k, lmax, B.ctypes.data, npairs.ctypes.data)
    rc = lib.hip_bispectrum_batched(ctypes.cast(arr, ctypes.c_void_p), n, PREC[prec], _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum_batched")
    del keep
    return [(B, (int(np_[0]), int(np_[1]))) for B, np_ in outs]


def hip_bispectrum_partial(pos, w, rand_pos, L, R0, k_edges, lmax=4, prec="mixed", data_range=None,
                           rand_range=None, stream=None):
    """T^ab_l summed over data primaries in data_range and random primaries in
    rand_range (input order), before normalisation.  Returns (T, (pairs, pairs))."""
    lib = load()
    n = int(pos.shape[0])
    nr = int(rand_pos.shape[0])
    pp, keep_p = _ptr(pos)
    wp, keep_w = _ptr(w)
    rp, keep_r = _ptr(rand_pos)
    edges = np.ascontiguousarray(np.asarray(k_edges, dtype=np.float64))
    n_k = len(edges) - 1
    T = np.zeros((lmax + 1, n_k, n_k))
    d0, d1 = (0, n) if data_range is None else data_range
    r0, r1 = (0, nr) if rand_range is None else rand_range
    rng = np.array([d0, d1, r0, r1], dtype=np.int64)
    npairs = (ctypes.c_int64 * 2)()
    rc = lib.hip_bispectrum_partial(pp, wp, n, rp, nr, float(L), float(R0), 0, edges.ctypes.data_as(ctypes.c_void_p),
                                    n_k, int(lmax), PREC[prec], rng.ctypes.data_as(ctypes.c_void_p),
                                    T.ctypes.data_as(ctypes.c_void_p), npairs, _stream_handle(stream))
    _check(lib, rc, "hip_bispectrum_partial")
    del keep_p, keep_w, keep_r
    return T, (int(npairs[0]), int(npairs[1]))


def debug_F(prec: str, l: int, u: float) -> float:
    """Host evaluation of the kernels' F_l(u) = D_l(u)/u^3 (same source and tables)."""
    return load().hip_debug_F(PREC[prec], int(l), float(u))


def debug_D(variant: str, l: int, u: float) -> float:
    """D_l(u) = u^3 F_l(u) as the FP32 pair kernels evaluate it (host build of the same
    code); variant "series", "fit" (closed form, fitted Si auxiliaries) or "asym"
    (closed form, asymptotic auxiliaries).  sin u and cos u are passed in correctly
    rounded, so the result isolates the D-form arithmetic."""
    return load().hip_debug_D({"series": 0, "fit": 1, "asym": 2}[variant], int(l), float(u))


def debug_Fb(l: int, u: float) -> float:
    """F_l(u) = D_l(u)/u^3 as the bispectrum's FP32 a_lm pass evaluates it (host
    build of the same source)."""
    return load().hip_debug_Fb(int(l), float(u))


def debug_bk_caps(tc_grid_cap: int = 0, chunk_cap: int = 0) -> None:
    """Test hook: cap the CTAs of the bispectrum's tensor-core contraction and the
    primaries per chunk of the bispectrum pass (0 = the library's own choice)."""
    load().hip_debug_bk_caps(int(tc_grid_cap), int(chunk_cap))


def debug_bk_mode(contract_on_cores: bool = False, fold_prims: int = 0) -> None:
    """Test hook: contract the mixed path's accumulators on the CUDA cores in FP64
    instead of the tensor cores, and/or set the primaries between the tensor-core
    contraction's FP64 folds (0 = the library's default)."""
    load().hip_debug_bk_mode(int(bool(contract_on_cores)), int(fold_prims))


def debug_F_array(prec: str, l: int, u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    out = np.zeros_like(u)
    load().hip_debug_F_array(PREC[prec], int(l), u.ctypes.data_as(ctypes.c_void_p),
                             out.ctypes.data_as(ctypes.c_void_p), u.size)
    return out


def set_profiling(on: bool) -> None:
    """Record CUDA events around the stages of each call (see hip_stage_times)."""
    load().hip_set_profiling(1 if on else 0)


def power_pair_pass(R0, k_max, prec="mixed"):
    """0: the direct pair pass, 1: the Legendre-moment pass (see hip_power_pair_pass)."""
    r = load().hip_power_pair_pass(float(R0), float(k_max), PREC[prec])
    if r < 0:
        raise ValueError("hip_power_pair_pass: invalid arguments")
    return r


def bispectrum_stage_times():
    """Stage times (ms) of the last bispectrum primary sum with profiling on:
    the a_lm passes, the contractions, the C terms (summed over chunks), and the
    number of chunks."""
    out = np.zeros(4)
    n = load().hip_bispectrum_stage_times(out.ctypes.data_as(ctypes.c_void_p), 4)
    return out[:n]


def stage_times():
    """Stage times (ms) of the last call: upload, cells, pairs, finalize, download."""
    out = np.zeros(5)
    n = load().hip_stage_times(out.ctypes.data_as(ctypes.c_void_p), 5)
    return out[:n]
