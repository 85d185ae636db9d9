"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one piece of ``oracle/`` against something other than itself:
exact values of the window, library special functions and quadrature, the
plane-wave definitions the estimators are derived from (Eq. discrete-xy for P,
Eq. general-XYZ-counts for B), brute-force triple sums (the DDD reformulation of
Sec. 4.2), Monte Carlo nulls and symmetries.  A plausible slip anywhere in the
oracle -- a dropped term, a wrong sign or index, a transposed operand -- fails
at least one of these.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import sici, spherical_jn, eval_legendre

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _minimage(d, L):
    return d - L * np.round(d / L)


# ------------------------------------------------------------------ window ---
def test_window_values_and_smoothness():
    # Eq. window_defn: W = 1 on [0,1/2), 1/2 at x = 3/4, 0 from x = 1.
    assert oracle.window(0.0) == 1.0
    assert oracle.window(0.49) == 1.0
    assert oracle.window(0.5) == pytest.approx(1.0, abs=1e-15)
    assert oracle.window(0.75) == pytest.approx(0.5, abs=1e-15)
    assert oracle.window(1.0) == 0.0
    assert oracle.window(1.2) == 0.0
    # continuity and C^1 at the joins (slopes 0, -4, 0)
    h = 1e-7
    for x0, slope in ((0.5, 0.0), (0.75, -4.0), (1.0, 0.0)):
        left = (oracle.window(x0 - h) - oracle.window(x0 - 2 * h)) / h
        right = (oracle.window(x0 + 2 * h) - oracle.window(x0 + h)) / h
        assert left == pytest.approx(slope, abs=1e-5)
        assert right == pytest.approx(slope, abs=1e-5)
        assert abs(oracle.window(x0 - 1e-12) - oracle.window(x0 + 1e-12)) < 1e-9


def test_window_moments_exact_rationals():
    # int_0^1 x^2 W dx = 47/320 and int_0^1 x^2 W^2 dx = 3713/31680, exact
    # rationals from integrating the piecewise polynomial of Eq. window_defn.
    m1 = integrate.quad(lambda x: x * x * oracle.window(x), 0, 1, points=[0.5, 0.75], epsabs=1e-15)[0]
    m2 = integrate.quad(lambda x: x * x * oracle.window(x) ** 2, 0, 1, points=[0.5, 0.75], epsabs=1e-15)[0]
    assert m1 == pytest.approx(47 / 320, rel=1e-13)
    assert m2 == pytest.approx(3713 / 31680, rel=1e-13)


# ------------------------------------------------------- special functions ---
def test_sine_integral_matches_library():
    u = np.concatenate([np.linspace(0, 10, 2001), np.linspace(10, 1500, 3001)])
    ours = np.array([oracle.sine_integral(x) for x in u])
    assert np.max(np.abs(ours - sici(u)[0])) < 5e-15
    assert oracle.sine_integral(-3.0) == pytest.approx(-sici(3.0)[0], abs=1e-15)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_dhat_matches_quadrature(l):
    # D_l(u) = int_0^u t^2 j_l(t) dt (App. C, definite from 0), across the
    # series / recursion switch at u = 4 and up to u = 400.
    for u in [1e-3, 0.05, 0.3, 1.5, 3.9, 3.999, 4.0, 4.1, 6.0, 11.0, 25.0, 137.0, 400.0]:
        ref = integrate.quad(lambda t: t * t * spherical_jn(l, t), 0, u, limit=5000,
                             epsabs=1e-16, epsrel=1e-14)[0]
        got = oracle.dhat(l, u)
        scale = max(abs(ref), u ** (l + 3) / 1e6 if u < 1 else 1e-300)
        assert abs(got - ref) <= 5e-12 * max(abs(ref), 1e-300) + 1e-14 * scale, (l, u, got, ref)


def test_dhat_closed_forms_and_constants():
    # D_0 = sin u - u cos u exactly; odd-l constants of integration: the App. C
    # closed form is -2 (l=1) and -8 (l=3) at u = 0, so the definite integral
    # adds them back.
    for u in [4.5, 9.0, 33.0]:
        assert oracle.dhat(0, u) == pytest.approx(np.sin(u) - u * np.cos(u), rel=1e-13, abs=1e-13)
        j = [spherical_jn(n, u) for n in range(6)]
        I1 = -j[0]
        I3 = (2 * I1 - 5 * j[2]) / 3
        assert oracle.dhat(1, u) == pytest.approx(u * u * j[2] - u * j[1] + 2 * I1 + 2.0, rel=1e-12)
        assert oracle.dhat(3, u) == pytest.approx(u * u * j[4] - 3 * u * j[3] + 12 * I3 + 8.0, rel=1e-12)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_jbar_is_shell_average(l):
    # Eq. jla-def: jbar^a_l(r) = (4 pi / v_a) int k^2 j_l(k r) dk over the bin.
    for klo, khi in [(0.0, 0.05), (0.2, 0.26), (1.9, 2.0), (4.95, 5.0)]:
        norm = 3.0 / (khi ** 3 - klo ** 3)
        for r in [1e-3, 0.7, 3.3, 19.9, 49.0]:
            ref = norm * integrate.quad(lambda k: k * k * spherical_jn(l, k * r), klo, khi,
                                        epsabs=1e-16, epsrel=1e-13, limit=200)[0]
            got = oracle.jbar(l, r, klo, khi)
            assert abs(got - ref) < 1e-10 * max(1.0, abs(ref)) + 1e-12, (l, klo, khi, r, got, ref)


def test_jbar_limits():
    assert oracle.jbar(0, 0.0, 0.1, 0.2) == 1.0
    for l in range(1, 5):
        assert oracle.jbar(l, 0.0, 0.1, 0.2) == 0.0
    assert oracle.jbar(0, 1e-6, 0.1, 0.2) == pytest.approx(1.0, abs=1e-11)
    # narrow bin -> j_l(k_c r)
    for l in range(5):
        kc, r = 1.3, 7.7
        assert oracle.jbar(l, r, kc - 1e-6, kc + 1e-6) == pytest.approx(spherical_jn(l, kc * r), abs=1e-9)


def test_ylm_addition_theorem_and_norm():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        b = rng.normal(size=3)
        b /= np.linalg.norm(b)
        Ya, Yb = oracle.ylm(a), oracle.ylm(b)
        for l in range(5):
            sl = slice(l * l, l * l + 2 * l + 1)
            lhs = np.sum(Ya[sl] * np.conj(Yb[sl]))
            assert lhs.real == pytest.approx((2 * l + 1) / (4 * np.pi) * eval_legendre(l, a @ b), abs=1e-13)
            assert abs(lhs.imag) < 1e-13
    # orthonormality on the sphere (Gauss-Legendre x trapezoid)
    ct, wt = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * 2 * np.pi / 32
    G = np.zeros((25, 25), dtype=complex)
    for c, wc in zip(ct, wt):
        s = np.sqrt(1 - c * c)
        for p in phis:
            Y = oracle.ylm((s * np.cos(p), s * np.sin(p), c))
            G += wc * (2 * np.pi / 32) * np.outer(Y, np.conj(Y))
    assert np.max(np.abs(G - np.eye(25))) < 1e-12


# ------------------------------------------------------- window transform ---
def test_window_transform_low_k_limit():
    # W~^a -> 4 pi R0^3 int x^2 W dx = 4 pi R0^3 47/320 as the bin shrinks to k = 0.
    R0 = 37.0
    Wt = oracle.window_transform_binned([0.0, 1e-5], R0)
    assert Wt[0] == pytest.approx(4 * np.pi * R0 ** 3 * 47 / 320, rel=1e-8)


def test_window_transform_matches_double_integral():
    # Eq. wka-def: W~^a = (4 pi / v_a) int k^2 W~(k R0) dk with
    # W~(k R0) = 4 pi int r^2 j_0(k r) W dr (RR term of Sec. 3), done here in the
    # opposite order with library quadrature.
    R0 = 20.0
    edges = [0.05, 0.25, 0.9, 1.0]

    def Wk(k):
        return 4 * np.pi * integrate.quad(lambda r: r * r * spherical_jn(0, k * r) * oracle.window(r / R0),
                                          0, R0, points=[R0 / 2, 0.75 * R0], limit=400,
                                          epsabs=1e-13, epsrel=1e-13)[0]

    got = oracle.window_transform_binned(edges, R0)
    for a in range(3):
        klo, khi = edges[a], edges[a + 1]
        ref = 3 / (khi ** 3 - klo ** 3) * integrate.quad(lambda k: k * k * Wk(k), klo, khi,
                                                       epsabs=1e-13, epsrel=1e-12, limit=200)[0]
        assert got[a] == pytest.approx(ref, rel=1e-9, abs=1e-9 * abs(got[0]))


# ------------------------------------------------------- power spectrum -----
def _tiny_catalog(N, L, seed, spread):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, L, size=3)
    return np.mod(c + rng.normal(0, spread, size=(N, 3)), L)


def test_power_pair_sum_equals_plane_wave_definition():
    # Eq. discrete-xy with the window, projected on L_l(khat.z) and averaged
    # over the k shell (Eq. pk-binned), equals (-i)^l (2l+1) DD^a_l: this pins the
    # Bessel/Legendre expansion of Eq. general-XY-counts, its sign and the binning.
    L, R0 = 60.0, 20.0
    pos = _tiny_catalog(8, L, 11, 6.0)
    edges = np.array([0.05, 0.2, 0.35])
    DD, npairs = oracle.power_pair_sum(pos, None, L, R0, edges, ell_max=4)
    assert npairs > 20
    d = _minimage(pos[:, None, :] - pos[None, :, :], L)
    r = np.linalg.norm(d, axis=-1)
    mask = (r > 0) & (r < R0)
    dv = d[mask]
    Wv = np.array([oracle.window(x / R0) for x in r[mask]])
    ct, wct = np.polynomial.legendre.leggauss(40)
    nphi = 80
    phi = np.arange(nphi) * 2 * np.pi / nphi
    C, PH = np.meshgrid(ct, phi, indexing="ij")
    S = np.sqrt(1 - C * C)
    khat = np.stack([S * np.cos(PH), S * np.sin(PH), C], axis=-1).reshape(-1, 3)
    wang = (np.outer(wct, np.full(nphi, 2 * np.pi / nphi)) / (4 * np.pi)).ravel()
    xk, wk = np.polynomial.legendre.leggauss(24)
    for a in range(2):
        klo, khi = edges[a], edges[a + 1]
        ks = 0.5 * (khi - klo) * xk + 0.5 * (khi + klo)
        wks = 0.5 * (khi - klo) * wk * 3 * ks * ks / (khi ** 3 - klo ** 3)
        for l in (0, 2, 4):
            Ll = eval_legendre(l, khat[:, 2])
            tot = 0.0 + 0.0j
            for k, wkk in zip(ks, wks):
                phase = np.exp(-1j * k * (khat @ dv.T))  # [ndir, npairs]
                tot += wkk * (2 * l + 1) * np.sum(wang * Ll * (phase @ Wv))
            expect = ((-1) ** (l // 2)) * (2 * l + 1) * DD[l // 2, a]
            assert abs(tot.imag) < 1e-10 * max(1.0, abs(expect))
            assert tot.real == pytest.approx(expect, rel=1e-9, abs=1e-9 * np.max(np.abs(DD)))


def test_power_two_particle_ordered_pair():
    # two particles across the periodic boundary: one pair in each order, the
    # minimum-image separation 3 along x (mu = 0) and weights w_i w_j.
    L, R0 = 50.0, 10.0
    pos = np.array([[0.5, 10.0, 10.0], [47.5, 10.0, 10.0]])
    w = np.array([2.0, 0.5])
    edges = np.array([0.1, 0.4, 1.2])
    DD, npairs = oracle.power_pair_sum(pos, w, L, R0, edges, ell_max=4)
    assert npairs == 2
    for a in range(2):
        for l in (0, 2, 4):
            jb = oracle.jbar(l, 3.0, edges[a], edges[a + 1])
            assert DD[l // 2, a] == pytest.approx(2 * 1.0 * oracle.window(0.3) * jb * eval_legendre(l, 0.0),
                                                  rel=1e-14, abs=1e-16)


def test_power_poisson_null_and_rr_term():
    # Fixed-N uniform catalogs: E[DD_0^a] / (n^2 V) = W~^a (N-1)/N, so
    # E[P_0^a] = -W~^a / N and E[P_2], E[P_4] = 0 (RR term of Sec. 3 and the
    # translation-invariance argument DR = RR).
    N, L, R0 = 300, 100.0, 20.0
    edges = np.linspace(0.1, 0.5, 5)
    Wt = oracle.window_transform_binned(edges, R0)
    Ps = []
    rng = np.random.default_rng(123)
    for s in range(60):
        pos = rng.uniform(0, L, size=(N, 3))
        DD, _ = oracle.power_pair_sum(pos, None, L, R0, edges, ell_max=4)
        Ps.append(oracle.power_from_pairs(DD, N, L, Wt))
    Ps = np.array(Ps)
    mean = Ps.mean(axis=0)
    se = Ps.std(axis=0, ddof=1) / np.sqrt(len(Ps))
    assert np.all(np.abs(mean[0] + Wt / N) < 4 * se[0] + 1e-12)
    assert np.all(np.abs(mean[1:]) < 4 * se[1:] + 1e-12)
    # and the signal is not trivially zero: the spread is resolved
    assert np.all(se[0] > 0)


def test_power_invariances():
    L, R0 = 200.0, 20.0
    rng = np.random.default_rng(7)
    parents = rng.uniform(0, L, size=(60, 3))
    pos = np.mod(parents[rng.integers(0, 60, 1500)] + rng.normal(0, 3.0, size=(1500, 3)), L)
    w = rng.uniform(0.5, 1.5, 1500)
    edges = np.linspace(0.2, 1.2, 6)
    base, _ = oracle.power_pair_sum(pos, w, L, R0, edges, ell_max=4)
    scale = np.max(np.abs(base))
    shift = np.mod(pos + rng.uniform(0, L, 3), L)
    perm = rng.permutation(len(pos))
    swap = pos[:, [1, 0, 2]]
    flip = np.mod(-pos * np.array([1, 1, -1]) + np.array([0, 0, L]), L)
    for p2, w2 in ((shift, w), (pos[perm], w[perm]), (swap, w), (flip, w)):
        got, _ = oracle.power_pair_sum(p2, w2, L, R0, edges, ell_max=4)
        assert np.max(np.abs(got - base)) < 1e-10 * scale


# ------------------------------------------------------------- bispectrum ---
def test_bispectrum_primary_sum_equals_triple_sum():
    # Sec. 4.2: sum_i w_i [4pi/(2l+1) sum_m A^a_lm A^b*_lm - C^ab_l](x_i) equals the
    # triple sum over i, j != i, k != i, k != j of
    # w_i w_j w_k jbar^a_l(r_ij) jbar^b_l(r_ik) W W L_l(rhat_ij . rhat_ik).
    L, R0 = 40.0, 15.0
    rng = np.random.default_rng(3)
    pos = _tiny_catalog(25, L, 5, 5.0)
    w = rng.uniform(0.5, 1.5, 25)
    edges = np.array([0.1, 0.3, 0.5, 0.7])
    T, _ = oracle.bispectrum_primary_sum(pos, w, np.arange(25), pos, w, L, R0, edges, lmax=4)
    nk = 3
    ref = np.zeros((5, nk, nk))
    for i in range(25):
        d = _minimage(pos[i] - pos, L)
        r = np.linalg.norm(d, axis=1)
        sel = np.where((r > 0) & (r < R0))[0]
        if len(sel) < 2:
            continue
        rh = d[sel] / r[sel, None]
        Wv = np.array([oracle.window(x / R0) for x in r[sel]])
        cosm = rh @ rh.T
        for l in range(5):
            jb = np.array([[oracle.jbar(l, x, edges[a], edges[a + 1]) for x in r[sel]] for a in range(nk)])
            Lm = eval_legendre(l, np.clip(cosm, -1, 1))
            np.fill_diagonal(Lm, 0.0)  # k != j
            y = jb * (w[sel] * Wv)[None, :]
            ref[l] += w[i] * (y @ Lm @ y.T)
    assert np.max(np.abs(T - ref)) < 1e-10 * np.max(np.abs(ref))


def test_bispectrum_plane_wave_definition():
    # Eq. general-XYZ-counts / general-Bkl-exp: averaging
    # e^{-i k1.x_ij} e^{-i k2.x_ik} against (2l+1) L_l(k1hat.k2hat) over both k
    # directions and both k shells gives (-1)^l (2l+1) times the triple sum,
    # i.e. the oracle's primary sum T.  This pins the (-1)^l (2l+1) convention.
    L, R0 = 60.0, 20.0
    pos = _tiny_catalog(6, L, 17, 5.0)
    edges = np.array([0.05, 0.2, 0.35])
    T, _ = oracle.bispectrum_primary_sum(pos, np.ones(6), np.arange(6), pos, None, L, R0, edges, lmax=4)
    ct, wct = np.polynomial.legendre.leggauss(20)
    nphi = 40
    phi = np.arange(nphi) * 2 * np.pi / nphi
    C, PH = np.meshgrid(ct, phi, indexing="ij")
    S = np.sqrt(1 - C * C)
    khat = np.stack([S * np.cos(PH), S * np.sin(PH), C], axis=-1).reshape(-1, 3)
    wang = (np.outer(wct, np.full(nphi, 2 * np.pi / nphi)) / (4 * np.pi)).ravel()
    cosk = np.clip(khat @ khat.T, -1, 1)
    xk, wk = np.polynomial.legendre.leggauss(8)
    N = 6
    dvec, Wm = {}, {}
    for i in range(N):
        d = _minimage(pos[i] - pos, L)
        r = np.linalg.norm(d, axis=1)
        sel = np.where((r > 0) & (r < R0))[0]
        dvec[i] = d[sel]
        Wm[i] = np.array([oracle.window(x / R0) for x in r[sel]])
    for l in range(5):
        Lmat = eval_legendre(l, cosk) * wang[:, None] * wang[None, :]
        for a in range(2):
            for b in range(2):
                ka = 0.5 * (edges[a + 1] - edges[a]) * xk + 0.5 * (edges[a + 1] + edges[a])
                wa = 0.5 * (edges[a + 1] - edges[a]) * wk * 3 * ka ** 2 / (edges[a + 1] ** 3 - edges[a] ** 3)
                kb = 0.5 * (edges[b + 1] - edges[b]) * xk + 0.5 * (edges[b + 1] + edges[b])
                wb = 0.5 * (edges[b + 1] - edges[b]) * wk * 3 * kb ** 2 / (edges[b + 1] ** 3 - edges[b] ** 3)
                tot = 0.0 + 0.0j
                for i in range(N):
                    dv, Wv = dvec[i], Wm[i]
                    if len(Wv) == 0:
                        continue
                    proj = khat @ dv.T  # [ndir, nnb]
                    E1 = np.einsum("q,qdn->dn", wa, np.exp(-1j * ka[:, None, None] * proj[None]) * Wv)
                    E2 = np.einsum("q,qdn->dn", wb, np.exp(-1j * kb[:, None, None] * proj[None]) * Wv)
                    full = np.sum(E1.sum(1) * (Lmat @ E2.sum(1)))
                    diag = np.sum(E1 * (Lmat @ E2))  # j == k terms
                    tot += (2 * l + 1) * (full - diag)
                expect = ((-1) ** l) * (2 * l + 1) * T[l, a, b]
                assert abs(tot.imag) < 1e-8 * max(1.0, np.max(np.abs(T)))
                assert tot.real == pytest.approx(expect, rel=1e-8, abs=1e-8 * np.max(np.abs(T)))


def _cluster(N, L, seed):
    rng = np.random.default_rng(seed)
    parents = rng.uniform(0, L, size=(N // 10, 3))
    return np.mod(parents[rng.integers(0, len(parents), N)] + rng.normal(0, 2.0, size=(N, 3)), L)


def test_bispectrum_symmetries():
    # B^ab_l = B^ba_l; invariance under translations, relabelling and the
    # rotations/reflections of the cube (the isotropic bispectrum, Sec. 2).
    L, R0 = 100.0, 20.0
    pos = _cluster(200, L, 9)
    rnd = np.random.default_rng(10).uniform(0, L, size=(600, 3))
    edges = np.linspace(0.2, 0.8, 4)
    B, _ = oracle.bispectrum(pos, None, rnd, L, R0, edges, lmax=4)
    scale = np.max(np.abs(B))
    assert np.max(np.abs(B - np.transpose(B, (0, 2, 1)))) < 1e-12 * scale
    rng = np.random.default_rng(1)
    sh = rng.uniform(0, L, 3)
    perm = rng.permutation(200)
    rot = lambda p: np.mod(np.stack([p[:, 1], -p[:, 0], p[:, 2]], 1) + np.array([0, L, 0]), L)
    refl = lambda p: np.mod(np.stack([p[:, 2], p[:, 1], -p[:, 0]], 1) + np.array([0, 0, L]), L)
    for p2, r2 in ((np.mod(pos + sh, L), np.mod(rnd + sh, L)), (pos[perm], rnd),
                   (rot(pos), rot(rnd)), (refl(pos), refl(rnd))):
        B2, _ = oracle.bispectrum(p2, None, r2, L, R0, edges, lmax=4)
        assert np.max(np.abs(B2 - B)) < 1e-10 * scale


def test_bispectrum_null_mean():
    # Unclustered data: the four l = 0 terms of the summary (Sec. 4.5) cancel in
    # expectation, so the seed-mean of B_0 (and of the l > 0 multipoles) is zero
    # up to O(1/N) and the Monte Carlo noise of the random catalog.
    N, L, R0 = 250, 80.0, 20.0
    edges = np.linspace(0.15, 0.45, 3)
    rng = np.random.default_rng(77)
    Bs = []
    for s in range(16):
        pos = rng.uniform(0, L, size=(N, 3))
        rnd = rng.uniform(0, L, size=(3 * N, 3))
        B, info = oracle.bispectrum(pos, None, rnd, L, R0, edges, lmax=2)
        Bs.append(B)
    Bs = np.array(Bs)
    mean = Bs.mean(0)
    se = Bs.std(0, ddof=1) / np.sqrt(len(Bs))
    Wt = info["Wt"]
    # O(1/N) bias bound: a few W~^a W~^b / N
    bias = 5.0 * np.abs(np.outer(Wt, Wt)) / N
    assert np.all(np.abs(mean[0]) < 4 * se[0] + bias)
    assert np.all(np.abs(mean[1:]) < 4 * se[1:] + 1e-12 * np.max(np.abs(Bs)))


# ------------------------------------------- random-free DDR^II (App. A / B) --
_E2_EDGES = np.linspace(0.4, 2.0, 7)


def test_e2_kernel_fourier_matches_bipolar_and_origin():
    # App. A (p integral over omega^a omega^b) and App. B (bipolar double integral)
    # are two derivations of the same kernel; at x = 0 both reduce to
    # 4 pi int r^2 jbar^a jbar^b W^2 dr (L_l(1) = 1).
    R0 = 8.0
    for l, x in ((0, 2.0), (2, 7.5), (4, 12.0)):
        Ef = oracle.e2_kernel(l, _E2_EDGES, R0, [x])[0]
        Eb = oracle.e2_kernel_bipolar(l, _E2_EDGES, R0, x)
        assert np.max(np.abs(Ef - Eb)) < 1e-7 * np.max(np.abs(Ef)), (l, x)
    for l in (0, 3):
        E0 = oracle.e2_kernel(l, _E2_EDGES, R0, [0.0])[0]
        rs, wq = oracle._gl_panels(0.0, R0, R0 / 64)
        f = np.array([[oracle.jbar(l, r, _E2_EDGES[a], _E2_EDGES[a + 1]) * oracle.window(r / R0) for r in rs]
                      for a in range(6)])
        direct = 4.0 * np.pi * np.einsum("ar,br,r->ab", f, f, wq * rs * rs)
        assert np.max(np.abs(E0 - direct)) < 1e-8 * np.max(np.abs(direct)), l


def test_e2_kernel_vanishes_beyond_two_R0_and_converges_in_p():
    R0 = 8.0
    E0 = np.max(np.abs(oracle.e2_kernel(0, _E2_EDGES, R0, [0.0])[0]))
    far = oracle.e2_kernel(2, _E2_EDGES, R0, [2.05 * R0, 2.5 * R0])
    assert np.max(np.abs(far)) < 1e-7 * E0
    a = oracle.e2_kernel(4, _E2_EDGES, R0, [3.0, 9.0])
    b = oracle.e2_kernel(4, _E2_EDGES, R0, [3.0, 9.0], pmax_factor=2.0)
    assert np.max(np.abs(a - b)) < 1e-9 * E0


def test_ddr2_pair_sum_is_the_kernel_summed_over_pairs():
    rng = np.random.default_rng(3)
    L, R0 = 30.0, 6.0
    pos = rng.uniform(0, L, (25, 3))
    w = rng.uniform(0.5, 1.5, 25)
    S = oracle.ddr2_pair_sum(pos, w, L, R0, _E2_EDGES, lmax=2)
    rs, ws = [], []
    for i in range(25):
        for j in range(25):
            d = pos[i] - pos[j]
            d -= L * np.round(d / L)
            r = float(np.sqrt(d @ d))
            if i != j and r < 2 * R0:
                rs.append(r)
                ws.append(w[i] * w[j])
    direct = np.array([np.einsum("x,xab->ab", np.array(ws), oracle.e2_kernel(l, _E2_EDGES, R0, rs))
                       for l in range(3)])
    assert np.max(np.abs(S - direct)) < 1e-10 * np.max(np.abs(direct))


def test_ddr2_is_the_expectation_of_the_random_catalog_term():
    # the random primaries' sum (1/N_r) sum_r G(x_r) is a Monte Carlo estimate of
    # (1/V) sum_{i != j} w_i w_j E^II(r_ij): they must agree within the sampling
    # error (estimated from independent batches of randoms)
    L, R0 = 30.0, 6.0
    rng = np.random.default_rng(11)
    parents = rng.uniform(0, L, (8, 3))
    pos = np.mod(parents[rng.integers(0, 8, 70)] + rng.normal(0, 1.5, (70, 3)), L)
    w = rng.uniform(0.5, 1.5, 70)
    edges = np.linspace(0.4, 2.0, 5)
    E2 = oracle.ddr2_pair_sum(pos, w, L, R0, edges, lmax=4) / L ** 3
    batches = []
    for b in range(6):
        rnd = rng.uniform(0, L, (40000, 3))
        T, _ = oracle.bispectrum_primary_sum(rnd, np.ones(len(rnd)), None, pos, w, L, R0, edges, 4)
        batches.append(T / len(rnd))
    batches = np.array(batches)
    mean, err = batches.mean(axis=0), batches.std(axis=0, ddof=1) / np.sqrt(len(batches))
    z = np.abs(mean - E2) / np.maximum(err, 1e-12 * np.max(np.abs(E2)))
    assert np.max(z) < 5.0, float(np.max(z))
    assert np.max(np.abs(mean - E2)) < 0.05 * np.max(np.abs(E2))


# --------------------------------------------------------------- subsample ----
def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 0, as printed by its reference implementation
    z = oracle.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_subsample_fraction_and_limits():
    n = 400_000
    for f in (0.01, 0.3, 0.77):
        k = int(oracle.subsample_mask(n, f, seed=12345).sum())
        assert abs(k - f * n) < 6.0 * np.sqrt(n * f * (1 - f)), (f, k)
    assert not oracle.subsample_mask(n, 0.0, 7).any()
    assert oracle.subsample_mask(n, 1.0, 7).all()
    # different seeds give (nearly) independent selections; nested fractions nest
    a, b = oracle.subsample_mask(n, 0.5, 1), oracle.subsample_mask(n, 0.5, 2)
    assert abs((a & b).sum() - 0.25 * n) < 6.0 * np.sqrt(n * 0.25 * 0.75)
    small, big = oracle.subsample_mask(n, 0.2, 9), oracle.subsample_mask(n, 0.6, 9)
    assert not (small & ~big).any()


def test_uniform_randoms_generator():
    # the seeded random catalog: each coordinate is the top 24 bits of one SplitMix64
    # output (published first outputs for seed 0 above) scaled by L in one float32 product
    r = oracle.uniform_randoms(1, 1.0, 0)
    assert [float(x) for x in r[0]] == [(0xE220A8397B1DCDAF >> 40) / 2.0 ** 24, (0x6E789E6AA1B965F4 >> 40) / 2.0 ** 24,
                                      (0x06C45D188009454F >> 40) / 2.0 ** 24]
    n, L = 300_000, 1000.0
    x = oracle.uniform_randoms(n, L, 2024).astype(np.float64)
    assert x.shape == (n, 3) and x.min() >= 0.0 and x.max() < L
    # uniform in the box: means, variances and the occupation of 10^3 sub-cells
    assert np.all(np.abs(x.mean(axis=0) - L / 2) < 6.0 * L / np.sqrt(12 * n))
    assert np.all(np.abs(x.var(axis=0) / L ** 2 - 1 / 12) < 6.0 * np.sqrt(1 / 180 / n))
    counts = np.bincount((np.floor(x / (L / 10)).astype(int) @ np.array([100, 10, 1])), minlength=1000)
    chi2 = float(np.sum((counts - n / 1000) ** 2 / (n / 1000)))
    assert 800 < chi2 < 1200
    # the largest variate times L stays below L for L a power of two and otherwise
    top = np.float32(1.0 - 2.0 ** -24)
    for Lt in (1.0, 1000.0, 1024.0, 777.77, 3.0e5):
        assert top * np.float32(Lt) < np.float32(Lt)
    # seeds give different catalogs
    assert not np.array_equal(oracle.uniform_randoms(10, L, 1), oracle.uniform_randoms(10, L, 2))


# ------------------------------------------- estimator assembly (l > 0) -------
# The pins above check the raw pair and primary sums; these run the oracle's
# finalize functions (power_from_pairs, bispectrum_from_sums via bispectrum) and
# compare whole estimates, every multipole, with the defining plane-wave forms
# normalised as the paper does: P by n^2 V (Eq. general-Pk-ell with the
# windowed counts of Eq. general-XY-counts, the RR term of Sec. 3), B by 6 n^3 V
# with the six identical permutations of Eq. general-XYZ-counts, the DDR^I / DDR^II
# split of Sec. 4.3 and the RRR term of Sec. 4.1.  A wrong phase ((-1)^l for
# (-1)^(l/2) in P), a dropped (2l+1) or a wrong normaliser fails here.
def _sphere_and_shell(n_ct, n_phi, n_k):
    ct, wct = np.polynomial.legendre.leggauss(n_ct)
    phi = np.arange(n_phi) * 2 * np.pi / n_phi
    C, PH = np.meshgrid(ct, phi, indexing="ij")
    S = np.sqrt(1 - C * C)
    khat = np.stack([S * np.cos(PH), S * np.sin(PH), C], axis=-1).reshape(-1, 3)
    wang = (np.outer(wct, np.full(n_phi, 2 * np.pi / n_phi)) / (4 * np.pi)).ravel()
    xk, wk = np.polynomial.legendre.leggauss(n_k)
    return khat, wang, xk, wk


def _shell(edges, a, xk, wk):
    # nodes and weights of (4 pi / v_a) int k^2 dk over bin a
    klo, khi = edges[a], edges[a + 1]
    ks = 0.5 * (khi - klo) * xk + 0.5 * (khi + klo)
    return ks, 0.5 * (khi - klo) * wk * 3 * ks * ks / (khi ** 3 - klo ** 3)


def test_power_estimate_equals_plane_wave_estimator():
    L, R0 = 60.0, 20.0
    pos = _tiny_catalog(9, L, 23, 6.0)
    w = np.random.default_rng(24).uniform(0.5, 1.5, len(pos))
    edges = np.array([0.05, 0.2, 0.35])
    DD, _ = oracle.power_pair_sum(pos, w, L, R0, edges, ell_max=4)
    Wt = oracle.window_transform_binned(edges, R0)
    S1 = float(np.sum(w))
    P = oracle.power_from_pairs(DD, S1, L, Wt)
    V, n_w = L ** 3, S1 / L ** 3
    d = _minimage(pos[:, None, :] - pos[None, :, :], L)
    r = np.linalg.norm(d, axis=-1)
    mask = (r > 0) & (r < R0)
    ww = (w[:, None] * w[None, :])[mask] * np.array([oracle.window(x / R0) for x in r[mask]])
    khat, wang, xk, wk = _sphere_and_shell(40, 80, 24)
    for a in range(2):
        ks, wks = _shell(edges, a, xk, wk)
        for l in (0, 2, 4):
            Ll = eval_legendre(l, khat[:, 2])  # line of sight z
            dd = 0.0 + 0.0j
            for k, wkk in zip(ks, wks):
                dd += wkk * (2 * l + 1) * np.sum(wang * Ll * (np.exp(-1j * k * (khat @ d[mask].T)) @ ww))
            expect = dd.real / (n_w * n_w * V) - (Wt[a] if l == 0 else 0.0)
            assert abs(dd.imag) < 1e-9 * abs(dd)
            assert P[l // 2, a] == pytest.approx(expect, rel=1e-8, abs=1e-9 * np.max(np.abs(P)))


def _triple_plane_wave(prim_pos, prim_w, prim_is_data, pos, w, L, R0, edges, l, a, b, khat, wang, xk, wk):
    """(2l+1) <L_l(k1hat.k2hat)> sum_p s_p sum_{j != k, both != p} w_j w_k
    e^{-i k1.x_pj} e^{-i k2.x_pk} W(x_pj) W(x_pk), averaged over both k directions
    and the shells a, b (one of the six identical permutations)."""
    ka, wa = _shell(edges, a, xk, wk)
    kb, wb = _shell(edges, b, xk, wk)
    Lmat = eval_legendre(l, np.clip(khat @ khat.T, -1, 1)) * wang[:, None] * wang[None, :]
    tot = 0.0 + 0.0j
    for p in range(len(prim_pos)):
        dv = _minimage(prim_pos[p] - pos, L)
        r = np.linalg.norm(dv, axis=1)
        sel = (r > 0) & (r < R0)
        if prim_is_data:
            sel[p] = False
        dv, r = dv[sel], r[sel]
        if len(r) == 0:
            continue
        f = w[sel] * np.array([oracle.window(x / R0) for x in r])
        proj = khat @ dv.T
        E1 = np.einsum("q,qdn->dn", wa, np.exp(-1j * ka[:, None, None] * proj[None]) * f)
        E2 = np.einsum("q,qdn->dn", wb, np.exp(-1j * kb[:, None, None] * proj[None]) * f)
        tot += prim_w[p] * (2 * l + 1) * (np.sum(E1.sum(1) * (Lmat @ E2.sum(1))) - np.sum(E1 * (Lmat @ E2)))
    return tot


def test_bispectrum_estimate_equals_plane_wave_estimator():
    L, R0 = 60.0, 20.0
    pos = _tiny_catalog(7, L, 29, 5.0)
    w = np.random.default_rng(30).uniform(0.5, 1.5, len(pos))
    rnd = np.mod(pos[:4] + np.random.default_rng(31).normal(0, 4.0, size=(4, 3)), L)
    edges = np.array([0.05, 0.2, 0.35])
    B, info = oracle.bispectrum(pos, w, rnd, L, R0, edges, lmax=4)
    Wt = oracle.window_transform_binned(edges, R0)
    S1 = float(np.sum(w))
    V, n_w = L ** 3, S1 / L ** 3
    khat, wang, xk, wk = _sphere_and_shell(16, 32, 8)
    # S^a = sum_{i != j} w_i w_j jbar^a_0 W from its own plane waves (l = 0 of Eq. general-XY-counts)
    d = _minimage(pos[:, None, :] - pos[None, :, :], L)
    r = np.linalg.norm(d, axis=-1)
    mask = (r > 0) & (r < R0)
    ww = (w[:, None] * w[None, :])[mask] * np.array([oracle.window(x / R0) for x in r[mask]])
    S = np.zeros(2)
    for a in range(2):
        ks, wks = _shell(edges, a, xk, wk)
        S[a] = sum(wkk * np.sum(wang * (np.exp(-1j * k * (khat @ d[mask].T)) @ ww)).real for k, wkk in zip(ks, wks))
    for l in range(5):
        for a in range(2):
            for b in range(2):
                ddd = _triple_plane_wave(pos, w, True, pos, w, L, R0, edges, l, a, b, khat, wang, xk, wk)
                ddr2 = _triple_plane_wave(rnd, np.ones(len(rnd)), False, pos, w, L, R0, edges, l, a, b,
                                          khat, wang, xk, wk)
                # 1/(6 n^3 V) [6 DDD - 3 (4 DDR^I + 2 DDR^II)] + 2 delta W~W~, DDR^II from the randoms
                # with weight S1 / N_r each (1/f_rand for unit weights)
                expect = (ddd - (S1 / len(rnd)) * ddr2).real / (V * n_w ** 3)
                if l == 0:
                    expect += -(Wt[a] * S[b] + Wt[b] * S[a]) / (V * n_w ** 2) + 2 * Wt[a] * Wt[b]
                scale = max(np.max(np.abs(B[l])), np.max(np.abs(B[0])))
                assert B[l, a, b] == pytest.approx(expect, rel=1e-7, abs=1e-8 * scale)
