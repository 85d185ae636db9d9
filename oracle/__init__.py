"""FP64 CPU oracle for the small-scale spectrum estimators of Philcox (arXiv:2005.01739).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  The product path (``paper_2005_01739_gb300``) never imports it, and the
two share no code: not the kernels, the tables, the quadrature, nor the
finalisation.  The only module both sides use is the seeded input generator
``paper_2005_01739_gb300.catalogs`` (random numbers only, none of the method's
arithmetic), and this package does not import even that.

What is computed, and where each piece comes from:

* ``hip_oracle.c`` -- brute-force ordered pair sums in double precision:
  the window W (Eq. window_defn), the bin-averaged Bessel function jbar (Eq.
  jla-def with D_l from App. C), the power-spectrum pair sum (Sec. 3) and the
  per-primary A_lm / C_l accumulators contracted into the bispectrum sum (Eq.
  AC-def, binned form of Sec. 4.4).
* this module -- the analytic random-pair terms and the final estimators:
  the binned window transform W~^a (Eq. wka-def) by composite Gauss-Legendre
  quadrature, P^a_l (binned estimator of Sec. 3) and B^ab_l (summary, Sec. 4.5);
  and the random-free DDR^II term of App. A: omega^a_l (Eq. omega-ell-a-def),
  the kernel E^{II,ab}_l(r) = int p^2 dp/(2 pi^2) j_0(p r) omega^a_l omega^b_l and
  the pair sum over it, with the bipolar form of App. B for cross-checks;
  the random subsample of Sec. 9 (a fraction 1/f_sub of the tracers) and a
  seeded uniform random catalog, both drawn with SplitMix64 written here from
  its published definition; and the
  anisotropic bispectrum the conclusions propose (two harmonics of different
  order about the line of sight), in the reading written out above
  `ANISO_COMBOS`: per-primary a_lm in complex harmonics coupled by Wigner 3j
  symbols (Racah's formula), the random-neighbour terms and the normalisation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hip_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhip_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc + OpenMP (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            L.orc_window.restype = d
            L.orc_window.argtypes = [d]
            L.orc_si.restype = d
            L.orc_si.argtypes = [d]
            L.orc_sph_jn.restype = d
            L.orc_sph_jn.argtypes = [i, d]
            L.orc_dhat.restype = d
            L.orc_dhat.argtypes = [i, d]
            L.orc_jbar.restype = d
            L.orc_jbar.argtypes = [i, d, d, d]
            L.orc_legendre.restype = d
            L.orc_legendre.argtypes = [i, d]
            L.orc_ylm_export.restype = None
            L.orc_ylm_export.argtypes = [d, d, d, P, P]
            L.orc_num_threads.restype = i
            L.orc_set_threads.argtypes = [i]
            L.orc_power_pairs.restype = i
            L.orc_power_pairs.argtypes = [P, P, i64, d, d, P, i, i, i, P, i64, P, P]
            L.orc_bispec_primaries.restype = i
            L.orc_bispec_primaries.argtypes = [P, P, P, i64, P, P, i64, d, d, P, i, i, P, P]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ----------------------------------------------------------- scalar pieces ---
def window(x: float) -> float:
    """W(x) of Eq. window_defn, x = r / R0."""
    return lib().orc_window(float(x))


def sine_integral(u: float) -> float:
    return lib().orc_si(float(u))


def sph_jn(n: int, x: float) -> float:
    return lib().orc_sph_jn(int(n), float(x))


def dhat(l: int, u: float) -> float:
    """D_l(u) = int_0^u t^2 j_l(t) dt (App. C, definite from 0)."""
    return lib().orc_dhat(int(l), float(u))


def jbar(l: int, r: float, klo: float, khi: float) -> float:
    """Bin-averaged spherical Bessel function, Eq. jla-def."""
    return lib().orc_jbar(int(l), float(r), float(klo), float(khi))


def legendre(l: int, mu: float) -> float:
    return lib().orc_legendre(int(l), float(mu))


def ylm(u) -> np.ndarray:
    """Complex Y_lm(u) for l <= 4, index l*l + l + m (Condon-Shortley phase)."""
    re = np.zeros(25)
    im = np.zeros(25)
    lib().orc_ylm_export(float(u[0]), float(u[1]), float(u[2]), _ptr(re), _ptr(im))
    return re + 1j * im


# --------------------------------------------------------- window transform ---
def _gl_panels(a: float, b: float, hmax: float, order: int = 16):
    n = max(1, int(np.ceil((b - a) / hmax)))
    x, wq = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, n + 1)
    lo, hi = edges[:-1, None], edges[1:, None]
    pts = 0.5 * (hi - lo) * x[None, :] + 0.5 * (hi + lo)
    wts = 0.5 * (hi - lo) * wq[None, :]
    return pts.ravel(), wts.ravel()


def window_transform_binned(edges, R0: float) -> np.ndarray:
    """W~^a(R0) = 4 pi int_0^R0 r^2 jbar^a_0(r) W(r/R0) dr (Eq. wka-def).

    Composite Gauss-Legendre on the three polynomial pieces of W, [0, R0/2],
    [R0/2, 3R0/4], [3R0/4, R0], each cut into panels no wider than pi/(4 k_hi).
    jbar^a_0 = 3 [D_0(r k_hi) - D_0(r k_lo)] / (r^3 (k_hi^3 - k_lo^3)).
    """
    edges = np.asarray(edges, dtype=np.float64)
    out = np.zeros(len(edges) - 1)
    for a in range(len(edges) - 1):
        klo, khi = edges[a], edges[a + 1]
        hmax = np.pi / (4.0 * khi)
        tot = 0.0
        for lo, hi in ((0.0, 0.5 * R0), (0.5 * R0, 0.75 * R0), (0.75 * R0, R0)):
            pts, wts = _gl_panels(lo, hi, hmax)
            for r, wq in zip(pts, wts):
                tot += wq * r * r * jbar(0, r, klo, khi) * window(r / R0)
        out[a] = 4.0 * np.pi * tot
    return out


# ------------------------------------------------------------ pair sums ------
def power_pair_sum(pos, w, L, R0, edges, ell_max=4, los=2, primaries=None):
    """Ordered-pair sum DD[l/2][a] = sum_{i in S} sum_{j != i} w_i w_j W jbar^a_l L_l(mu).

    Returns (DD [n_ell, nk], number of ordered pairs counted)."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    N = pos.shape[0]
    wv = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    nk = len(edges) - 1
    n_ell = ell_max // 2 + 1
    prim = np.arange(N, dtype=np.int64) if primaries is None else np.ascontiguousarray(
        np.asarray(primaries, dtype=np.int64))
    DD = np.zeros((n_ell, nk))
    npairs = ctypes.c_int64(0)
    rc = lib().orc_power_pairs(_ptr(pos), _ptr(wv), N, float(L), float(R0), _ptr(edges), nk, n_ell,
                               int(los), _ptr(prim), len(prim), _ptr(DD), ctypes.byref(npairs))
    if rc != 0:
        raise ValueError(f"orc_power_pairs failed ({rc})")
    return DD, int(npairs.value)


def bispectrum_primary_sum(prim_pos, prim_w, prim_self, data_pos, data_w, L, R0, edges, lmax=4):
    """T[l][a][b] = sum_p prim_w[p] [4pi/(2l+1) Re sum_m A^a_lm A^b*_lm - C^ab_l](p)."""
    pp = np.ascontiguousarray(np.asarray(prim_pos, dtype=np.float64).reshape(-1, 3))
    pw = np.ascontiguousarray(np.asarray(prim_w, dtype=np.float64))
    ps = None if prim_self is None else np.ascontiguousarray(np.asarray(prim_self, dtype=np.int64))
    dp = np.ascontiguousarray(np.asarray(data_pos, dtype=np.float64).reshape(-1, 3))
    dw = None if data_w is None else np.ascontiguousarray(np.asarray(data_w, dtype=np.float64))
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    nk = len(edges) - 1
    T = np.zeros((lmax + 1, nk, nk))
    npairs = ctypes.c_int64(0)
    rc = lib().orc_bispec_primaries(_ptr(pp), _ptr(pw), _ptr(ps), pp.shape[0], _ptr(dp), _ptr(dw),
                                    dp.shape[0], float(L), float(R0), _ptr(edges), nk, int(lmax),
                                    _ptr(T), ctypes.byref(npairs))
    if rc != 0:
        raise ValueError(f"orc_bispec_primaries failed ({rc})")
    return T, int(npairs.value)


# ------------------------------------------------------------- estimators ----
def power_from_pairs(DD, S1, L, Wt):
    """P^a_l = (-1)^(l/2) (2l+1) DD^a_l / (n_w^2 V) - delta_l0 W~^a (Sec. 3).

    (-i)^l = (-1)^(l/2) for even l.  n_w = S1 / V with S1 = sum of weights
    (= N for unit weights, the paper's n)."""
    V = float(L) ** 3
    n_w = float(S1) / V
    P = np.zeros_like(DD)
    for il in range(DD.shape[0]):
        l = 2 * il
        P[il] = ((-1.0) ** (l // 2)) * (2 * l + 1) * DD[il] / (n_w * n_w * V)
    P[0] -= Wt
    return P


def power_spectrum(pos, w, L, R0, edges, ell_max=4, los=2):
    """Full brute-force P^a_l for ell = 0, 2, ..., ell_max (binned estimator, Sec. 3)."""
    DD, npairs = power_pair_sum(pos, w, L, R0, edges, ell_max, los)
    N = np.asarray(pos).reshape(-1, 3).shape[0]
    S1 = float(N) if w is None else float(np.sum(np.asarray(w, dtype=np.float64)))
    Wt = window_transform_binned(edges, R0)
    return power_from_pairs(DD, S1, L, Wt), DD, npairs


def bispectrum_from_sums(Tdata, Trand, S, S1, N_r, L, Wt):
    """B^ab_l from the summary of Sec. 4.5.

    B = (-1)^l (2l+1) [Tdata - (S1/N_r) Trand] / (V n_w^3)
        - delta_l0 (W~^a S^b + W~^b S^a) / (V n_w^2) + 2 delta_l0 W~^a W~^b,
    S^a = sum_{i != j} w_i w_j jbar^a_0 W (the ordered DD_0 pair sum), and each
    random primary carries weight S1/N_r (= 1/f_rand for unit weights)."""
    V = float(L) ** 3
    n_w = float(S1) / V
    nl = Tdata.shape[0]
    B = np.zeros_like(Tdata)
    for l in range(nl):
        B[l] = ((-1.0) ** l) * (2 * l + 1) * (Tdata[l] - (float(S1) / float(N_r)) * Trand[l]) / (V * n_w ** 3)
    B[0] -= (np.outer(Wt, S) + np.outer(S, Wt)) / (V * n_w * n_w)
    B[0] += 2.0 * np.outer(Wt, Wt)
    return B


def bispectrum(pos, w, rand_pos, L, R0, edges, lmax=4, data_primaries=None, rand_primaries=None):
    """Brute-force B^ab_l.  Optional primary subsets restrict the A/C sums (used for
    sampled parity at large N); S^a is always the full pair sum when no subset is
    given, else the same subset's ordered sum (callers compare like with like)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    rp = np.asarray(rand_pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    wv = np.ones(N) if w is None else np.asarray(w, dtype=np.float64)
    dsel = np.arange(N) if data_primaries is None else np.asarray(data_primaries, dtype=np.int64)
    rsel = np.arange(rp.shape[0]) if rand_primaries is None else np.asarray(rand_primaries, dtype=np.int64)
    Td, npd = bispectrum_primary_sum(pos[dsel], wv[dsel], dsel, pos, w, L, R0, edges, lmax)
    Tr, npr = bispectrum_primary_sum(rp[rsel], np.ones(len(rsel)), None, pos, w, L, R0, edges, lmax)
    DD, _ = power_pair_sum(pos, w, L, R0, edges, 0, 2, primaries=dsel)
    Wt = window_transform_binned(edges, R0)
    S1 = float(np.sum(wv))
    B = bispectrum_from_sums(Td, Tr, DD[0], S1, rp.shape[0], L, Wt)
    return B, dict(Tdata=Td, Trand=Tr, S=DD[0], Wt=Wt, npairs_data=npd, npairs_rand=npr)


# ------------------------------------------------ random-free DDR^II (App. A) --
def _sph_jn_vec(l: int, z):
    """Spherical Bessel j_l (library routine, vectorised)."""
    from scipy.special import spherical_jn
    return spherical_jn(l, z)


def _jbar_table(l: int, edges, rs) -> np.ndarray:
    """jbar^a_l(r) for every bin a at the nodes rs: [n_k][len(rs)]."""
    edges = np.asarray(edges, dtype=np.float64)
    return np.array([[jbar(l, r, edges[a], edges[a + 1]) for r in rs] for a in range(len(edges) - 1)])


def _r_nodes(R0: float, hmax: float):
    """Composite Gauss-Legendre nodes on the three polynomial pieces of W."""
    pts, wts = [], []
    for lo, hi in ((0.0, 0.5 * R0), (0.5 * R0, 0.75 * R0), (0.75 * R0, R0)):
        x, wq = _gl_panels(lo, hi, hmax)
        pts.append(x)
        wts.append(wq)
    return np.concatenate(pts), np.concatenate(wts)


def e2_p_nodes(edges, R0: float, pmax_factor: float = 1.0):
    """The p quadrature of the E^II integrals: composite Gauss-Legendre on
    [0, p_max], p_max = k_hi + 120/R0 (times pmax_factor), panels no wider than
    pi/(8 R0) (j_0(p r) with r < 2 R0 oscillates at most once per 2 pi/(2 R0))."""
    k_hi = float(np.max(edges))
    pmax = pmax_factor * (k_hi + 120.0 / R0)
    return _gl_panels(0.0, pmax, np.pi / (8.0 * R0))


def omega_binned(l: int, edges, R0: float, p) -> np.ndarray:
    """omega^a_l(p) = 4 pi int_0^R0 r^2 j_l(p r) jbar^a_l(r) W(r/R0) dr
    (Eq. omega-ell-a-def): [n_k][len(p)], composite Gauss-Legendre in r."""
    p = np.atleast_1d(np.asarray(p, dtype=np.float64))
    kmax = max(float(np.max(edges)), float(np.max(p)) if p.size else 0.0)
    rs, rw = _r_nodes(R0, np.pi / (4.0 * max(kmax, 1.0 / R0)))
    Wr = np.array([window(r / R0) for r in rs])
    JB = _jbar_table(l, edges, rs)
    jl = _sph_jn_vec(l, np.outer(p, rs))  # [p][r]
    return 4.0 * np.pi * np.einsum("pr,ar,r->ap", jl, JB * (Wr * rs * rs)[None, :], rw)


def e2_kernel(l: int, edges, R0: float, x, pmax_factor: float = 1.0) -> np.ndarray:
    """E^{II,ab}_l(x) = int p^2 dp/(2 pi^2) j_0(p x) omega^a_l(p) omega^b_l(p)
    (binned kernel of App. A): [len(x)][n_k][n_k]."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    ps, pw = e2_p_nodes(edges, R0, pmax_factor)
    om = omega_binned(l, edges, R0, ps)
    j0 = np.sinc(np.outer(x, ps) / np.pi)  # j_0(p x)
    return np.einsum("xp,p,ap,bp->xab", j0, pw * ps * ps / (2.0 * np.pi ** 2), om, om)


def e2_kernel_bipolar(l: int, edges, R0: float, x: float, n_panel: int = 24) -> np.ndarray:
    """The same kernel from the bipolar double integral of App. B:
    2 pi int int dr1 dr2 (r1 r2 / x) jbar^a_l(r1) jbar^b_l(r2) W(r1) W(r2) L_l(Delta),
    Delta = (r1^2 + r2^2 - x^2)/(2 r1 r2), over |r1 - r2| <= x <= r1 + r2
    (cross-check only; slow)."""
    edges = np.asarray(edges, dtype=np.float64)
    nk = len(edges) - 1
    out = np.zeros((nk, nk))
    lo1 = max(0.0, x - R0)
    r1s, w1s = _gl_panels(lo1, R0, (R0 - lo1) / n_panel)
    for r1, w1 in zip(r1s, w1s):
        lo, hi = abs(x - r1), min(R0, x + r1)
        if hi <= lo:
            continue
        r2s, w2s = _gl_panels(lo, hi, (hi - lo) / max(2, n_panel // 2))
        f1 = np.array([jbar(l, r1, edges[a], edges[a + 1]) for a in range(nk)]) * window(r1 / R0)
        f2 = _jbar_table(l, edges, r2s) * np.array([window(r / R0) for r in r2s])[None, :]
        D = np.clip((r1 * r1 + r2s ** 2 - x * x) / (2.0 * r1 * r2s), -1.0, 1.0)
        Ll = np.array([legendre(l, d) for d in D])
        out += w1 * np.outer(f1, f2 @ (w2s * r1 * r2s / x * Ll))
    return 2.0 * np.pi * out


def ddr2_pair_sum(pos, w, L, R0, edges, lmax=4, pmax_factor: float = 1.0) -> np.ndarray:
    """sum over ordered pairs i != j of w_i w_j E^{II,ab}_l(|x_i - x_j|) (minimum
    image; E^II vanishes beyond 2 R0, so only pairs closer than 2 R0 enter):
    [lmax+1][n_k][n_k].  The sum over pairs is taken inside the p integral:
    sum_ij w_i w_j E(r_ij) = int p^2 dp/(2 pi^2) S(p) omega^a omega^b with
    S(p) = sum_ij w_i w_j j_0(p r_ij).  Brute force over all pairs (small N)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    wv = np.ones(N) if w is None else np.asarray(w, dtype=np.float64)
    rr, ww = [], []
    for i in range(N):
        d = pos[i + 1:] - pos[i]
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        m = (r < 2.0 * R0) & (r > 0.0)
        rr.append(r[m])
        ww.append(2.0 * wv[i] * wv[i + 1:][m])  # both orders
    rr = np.concatenate(rr)
    ww = np.concatenate(ww)
    ps, pw = e2_p_nodes(edges, R0, pmax_factor)
    S = np.array([np.sum(ww * np.sinc(p * rr / np.pi)) for p in ps])
    nk = len(edges) - 1
    out = np.zeros((lmax + 1, nk, nk))
    for l in range(lmax + 1):
        om = omega_binned(l, edges, R0, ps)
        out[l] = np.einsum("p,ap,bp->ab", pw * ps * ps / (2.0 * np.pi ** 2) * S, om, om)
    return out


def bispectrum_analytic(pos, w, L, R0, edges, lmax=4):
    """B^ab_l with the DDR^II term from the E^II kernel instead of a random
    catalog (App. A): the random primaries' sum (S1/N_r) sum_r G(x_r) -> its
    expectation (S1/V) sum_{i != j} w_i w_j E^{II,ab}_l(r_ij)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    wv = np.ones(N) if w is None else np.asarray(w, dtype=np.float64)
    Td, npd = bispectrum_primary_sum(pos, wv, np.arange(N), pos, w, L, R0, edges, lmax)
    E2 = ddr2_pair_sum(pos, w, L, R0, edges, lmax)
    DD, _ = power_pair_sum(pos, w, L, R0, edges, 0, 2)
    Wt = window_transform_binned(edges, R0)
    S1 = float(np.sum(wv))
    V = float(L) ** 3
    # bispectrum_from_sums subtracts (S1/N_r) Trand; pass Trand = E2 N_r / V with N_r = 1
    B = bispectrum_from_sums(Td, E2 / V, DD[0], S1, 1.0, L, Wt)
    return B, dict(Tdata=Td, E2=E2, S=DD[0], Wt=Wt, npairs_data=npd)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """Outputs 1..n of SplitMix64 seeded with `seed` (Steele, Lea & Flood 2014):
    z = seed + i * 0x9E3779B97F4A7C15, z = (z ^ z>>30) * 0xBF58476D1CE4E5B9,
    z = (z ^ z>>27) * 0x94D049BB133111EB, output z ^ z>>31 (all mod 2^64)."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def subsample_mask(n: int, fraction: float, seed: int) -> np.ndarray:
    """The random subsample of Sec. 9: particle i (0-based) is kept iff its
    uniform variate u_i = (z_{i+1} >> 11) 2^-53 is below `fraction`, compared
    exactly in integers as (z >> 11) < floor(fraction 2^53)."""
    import math
    thr = np.uint64(math.floor(math.ldexp(float(fraction), 53)))
    return (splitmix64(seed, n) >> np.uint64(11)) < thr


def uniform_randoms(n: int, L: float, seed: int) -> np.ndarray:
    """A seeded uniform random catalog for the DDR^II term's random catalog
    (Sec. 4.3): coordinate d of random j is fl32(u * fl32(L)) with
    u = (z >> 40) 2^-24, z output 3j + d + 1 of SplitMix64; u is exact in
    float32 and the product is one IEEE float32 multiplication."""
    z = splitmix64(seed, 3 * int(n))
    u = (z >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
    return (u * np.float32(L)).astype(np.float32).reshape(int(n), 3)


# ------------------------------------ anisotropic bispectrum (Sec. 10 extension) --
# The conclusions propose the anisotropic (redshift-space) bispectrum as an
# extension: the sum over spherical harmonics of the isotropic estimator becomes
# a product of two harmonics of different order.  The paper fixes no estimator;
# the reading written out here (and in the design notes) projects the triangle
# onto the tripolar basis about the fixed line of sight zhat,
#     S_{l1 l2 L}(u, v) = sum_m (l1 l2 L; m, -m, 0) y_{l1 m}(u) y_{l2 -m}(v),
# y_lm = sqrt(4 pi / (2l + 1)) Y_lm (so y_{L0}(zhat) = 1), for l1, l2 <= 4,
# l1 + l2 and L even, |l1 - l2| <= L <= min(l1 + l2, 4).  S_{l l 0} =
# (-1)^l L_l(u.v) / sqrt(2l + 1), so L = 0 holds the isotropic multipoles.
ANISO_COMBOS = tuple((l1, l2, Lc) for l1 in range(5) for l2 in range(l1, 5) for Lc in range(0, 5, 2)
                     if (l1 + l2) % 2 == 0 and abs(l1 - l2) <= Lc <= l1 + l2)


def wigner3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """Wigner 3j symbol (j1 j2 j3; m1 m2 m3) of integer arguments, Racah's formula."""
    from math import factorial as fac, sqrt
    if m1 + m2 + m3 != 0 or abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    t1, t2 = j2 - m1 - j3, j1 + m2 - j3
    t3, t4, t5 = j1 + j2 - j3, j1 - m1, j2 + m2
    s = 0.0
    for t in range(max(0, t1, t2), min(t3, t4, t5) + 1):
        s += (-1.0) ** t / (fac(t) * fac(t - t1) * fac(t - t2) * fac(t3 - t) * fac(t4 - t) * fac(t5 - t))
    tri = fac(j1 + j2 - j3) * fac(j1 - j2 + j3) * fac(-j1 + j2 + j3) / fac(j1 + j2 + j3 + 1)
    return ((-1.0) ** (j1 - j2 - m3)) * sqrt(tri * fac(j1 + m1) * fac(j1 - m1) * fac(j2 + m2) * fac(j2 - m2)
                                              * fac(j3 + m3) * fac(j3 - m3)) * s


_GL_CACHE = {}


def jbar_vec(l: int, edges, r, order: int = 32) -> np.ndarray:
    """jbar^a_l(r) of Eq. jla-def for every bin a at the separations r: [n_k][len(r)],
    the k-shell average 3 / (k_b^3 - k_a^3) int k^2 j_l(k r) dk by Gauss-Legendre
    (library Bessel function; a vectorised restatement of `jbar`)."""
    edges = np.asarray(edges, dtype=np.float64)
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    if order not in _GL_CACHE:
        _GL_CACHE[order] = np.polynomial.legendre.leggauss(order)
    x, wq = _GL_CACHE[order]
    lo, hi = edges[:-1, None], edges[1:, None]
    k = 0.5 * (hi - lo) * x[None, :] + 0.5 * (hi + lo)  # [n_k][order]
    wk = 0.5 * (hi - lo) * wq[None, :] * k * k * 3.0 / (hi ** 3 - lo ** 3)
    jl = _sph_jn_vec(l, k.reshape(-1, 1) * r[None, :]).reshape(k.shape[0], k.shape[1], len(r))
    return np.einsum("aq,aqr->ar", wk, jl)


def _ylm_vec(u) -> np.ndarray:
    """Complex Y_lm (Condon-Shortley phase, polar axis z) of unit vectors u [n][3]
    for l <= 4, index l*l + l + m: the library's harmonics, vectorised."""
    from scipy.special import sph_harm_y
    th = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    ph = np.arctan2(u[:, 1], u[:, 0])
    out = np.zeros((u.shape[0], 25), dtype=complex)
    for l in range(5):
        for m in range(-l, l + 1):
            out[:, l * l + l + m] = sph_harm_y(l, m, th, ph)
    return out


def _aniso_coeffs():
    """For each combination, the m range and (l1 l2 L; m, -m, 0)."""
    out = []
    for l1, l2, Lc in ANISO_COMBOS:
        mm = np.arange(-min(l1, l2), min(l1, l2) + 1)
        out.append((mm, np.array([wigner3j(l1, l2, Lc, int(m), int(-m), 0) for m in mm])))
    return out


def bispectrum_aniso_primary_sum(prim_pos, prim_w, prim_self, data_pos, data_w, L, R0, edges):
    """T[c][a][b] = sum_p s_p sum_{j != k} w_j w_k W_j W_k jbar^a_{l1}(r_j) jbar^b_{l2}(r_k)
    S_{l1 l2 L}(rhat_j, rhat_k) for the combinations c of ANISO_COMBOS (r_j the
    minimum-image separation of neighbour j from primary p, 0 < r_j < R0, j not p
    itself), formed per primary as sum_m (l1 l2 L; m, -m, 0) A^a_{l1 m} A^b_{l2, -m}
    minus the j = k terms, A^a_{lm} = sum_j w_j W_j jbar^a_l(r_j) y_lm(rhat_j)."""
    pp = np.asarray(prim_pos, dtype=np.float64).reshape(-1, 3)
    pw = np.asarray(prim_w, dtype=np.float64)
    dp = np.asarray(data_pos, dtype=np.float64).reshape(-1, 3)
    dw = np.ones(dp.shape[0]) if data_w is None else np.asarray(data_w, dtype=np.float64)
    nk = len(edges) - 1
    coeffs = _aniso_coeffs()
    ynorm = np.array([np.sqrt(4 * np.pi / (2 * l + 1)) for l in range(5) for _ in range(2 * l + 1)])
    T = np.zeros((len(ANISO_COMBOS), nk, nk))
    npairs = 0
    for p in range(pp.shape[0]):
        d = dp - pp[p]
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        ok = (r > 0) & (r < R0)
        if prim_self is not None and prim_self[p] >= 0:
            ok[prim_self[p]] = False
        sel = np.where(ok)[0]
        if len(sel) == 0:
            continue
        npairs += len(sel)
        rs = r[sel]
        wv = dw[sel] * np.array([window(x / R0) for x in rs])
        Y = _ylm_vec(d[sel] / rs[:, None]) * ynorm  # [nnb][25], y_lm
        J = [jbar_vec(l, edges, rs) for l in range(5)]  # [l][a][j]
        for ci, ((l1, l2, _), (mm, cm)) in enumerate(zip(ANISO_COMBOS, coeffs)):
            full = np.zeros((nk, nk), dtype=complex)
            diag = np.zeros(nk, dtype=complex)
            sdiag = np.zeros(len(sel), dtype=complex)
            for m, c in zip(mm, cm):
                y1 = Y[:, l1 * l1 + l1 + m]
                y2 = Y[:, l2 * l2 + l2 - m]
                A1 = J[l1] @ (wv * y1)
                A2 = J[l2] @ (wv * y2)
                full += c * np.outer(A1, A2)
                sdiag += c * y1 * y2
            diag = (J[l1] * (wv * wv * sdiag)) @ J[l2].T
            T[ci] += pw[p] * np.real(full - diag)
    return T, npairs


def bispectrum_aniso_from_sums(Tdata, Trand, DD, S1, N_r, L, Wt):
    """B^ab_{l1 l2 L} of the reading: with N = D - R expanded as in Sec. 4.5 (the
    random primaries enter T; the analytic terms are those with a random
    neighbour, where the angular average of y_{l m} leaves l = 0),
        B = (2 l1 + 1)(2 l2 + 1)(-1)^((l1 + l2)/2) [ (Tdata - (S1/N_r) Trand) / (V n^3)
            - d_{l2 0} d_{L l1} k_{l1} DD^a_{l1} W~^b / (V n^2)
            - d_{l1 0} d_{L l2} k_{l2} W~^a DD^b_{l2} / (V n^2) + 2 d_{l1 0} d_{l2 0} W~^a W~^b ],
    k_l = (l 0 l; 0 0 0) = (-1)^l / sqrt(2l + 1), DD^a_l the ordered power pair sum
    with L_l(mu) about zhat (DD[l/2]), n = S1 / V.  (0, 0, 0) is the isotropic B_0."""
    V = float(L) ** 3
    n = float(S1) / V
    B = np.zeros_like(Tdata)
    for ci, (l1, l2, Lc) in enumerate(ANISO_COMBOS):
        t = (Tdata[ci] - (float(S1) / float(N_r)) * Trand[ci]) / (V * n ** 3)
        if l2 == 0 and Lc == l1:
            t -= ((-1.0) ** l1 / np.sqrt(2 * l1 + 1)) * np.outer(DD[l1 // 2], Wt) / (V * n * n)
        if l1 == 0 and Lc == l2:
            t -= ((-1.0) ** l2 / np.sqrt(2 * l2 + 1)) * np.outer(Wt, DD[l2 // 2]) / (V * n * n)
        if l1 == 0 and l2 == 0:
            t += 2.0 * np.outer(Wt, Wt)
        B[ci] = (2 * l1 + 1) * (2 * l2 + 1) * ((-1.0) ** ((l1 + l2) // 2)) * t
    return B


def bispectrum_aniso(pos, w, rand_pos, L, R0, edges):
    """Brute-force B^ab_{l1 l2 L} (all of ANISO_COMBOS) of a periodic catalog with a
    random catalog for the random primaries; line of sight zhat."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    rp = np.asarray(rand_pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    wv = np.ones(N) if w is None else np.asarray(w, dtype=np.float64)
    Td, npd = bispectrum_aniso_primary_sum(pos, wv, np.arange(N), pos, wv, L, R0, edges)
    Tr, npr = bispectrum_aniso_primary_sum(rp, np.ones(rp.shape[0]), None, pos, wv, L, R0, edges)
    DD, _ = power_pair_sum(pos, wv, L, R0, edges, 4, 2)
    Wt = window_transform_binned(edges, R0)
    S1 = float(np.sum(wv))
    B = bispectrum_aniso_from_sums(Td, Tr, DD, S1, rp.shape[0], L, Wt)
    return B, dict(Tdata=Td, Trand=Tr, DD=DD, Wt=Wt, npairs_data=npd, npairs_rand=npr)
