"""Pins of the oracle's anisotropic bispectrum (the extension proposed in the
paper's conclusions: two harmonics of different order about the line of sight).

The reading is fixed by the tripolar projection of the plane-wave bispectrum
about zhat; these tests check the oracle's per-primary form against things other
than itself: the Wigner symbols' orthogonality and tabulated values, the
library's Bessel quadrature, the direction-averaged plane-wave definition on a
tiny catalog, the isotropic estimator (L = 0), the random-neighbour terms
estimated with an explicit random catalog, and symmetries.
"""
import numpy as np
import pytest
from scipy.special import sph_harm_y

import oracle

COMBOS = oracle.ANISO_COMBOS


def _minimage(d, L):
    return d - L * np.round(d / L)


def test_wigner3j_values_and_orthogonality():
    w3 = oracle.wigner3j
    # tabulated values
    assert w3(1, 1, 0, 1, -1, 0) == pytest.approx(1 / np.sqrt(3), rel=1e-14)
    assert w3(1, 1, 1, 1, -1, 0) == pytest.approx(1 / np.sqrt(6), rel=1e-14)
    assert w3(2, 2, 2, 0, 0, 0) == pytest.approx(-np.sqrt(2 / 35), rel=1e-14)
    assert w3(1, 1, 2, 0, 0, 0) == pytest.approx(np.sqrt(2 / 15), rel=1e-14)
    assert w3(2, 1, 1, 0, 0, 0) == pytest.approx(np.sqrt(2 / 15), rel=1e-14)
    assert w3(1, 2, 2, 0, 0, 0) == 0.0  # odd j1 + j2 + j3 with all m = 0
    # orthogonality: sum_{m1 m2} (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3) = delta_{j3 j3'} / (2 j3 + 1)
    for j1 in range(4):
        for j2 in range(4):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for j3p in range(abs(j1 - j2), j1 + j2 + 1):
                    for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                        s = sum(w3(j1, j2, j3, m1, -m1 - m3, m3) * w3(j1, j2, j3p, m1, -m1 - m3, m3)
                                for m1 in range(-j1, j1 + 1))
                        assert s == pytest.approx((j3 == j3p) / (2 * j3 + 1), abs=1e-13)
    # the standard form: sum over m1, m2, m3 of the squares is 1 for a valid triple
    for j1, j2, j3 in ((1, 1, 2), (2, 2, 2), (3, 4, 5), (4, 4, 4)):
        s = sum(w3(j1, j2, j3, m1, m2, -m1 - m2) ** 2 for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1))
        assert s == pytest.approx(1.0, abs=1e-13)
    # column exchange symmetry (-1)^(j1+j2+j3)
    assert w3(2, 3, 4, 1, -2, 1) == pytest.approx(-w3(3, 2, 4, -2, 1, 1), abs=1e-15)
    assert w3(2, 3, 3, 1, -2, 1) == pytest.approx(w3(3, 2, 3, -2, 1, 1), abs=1e-15)
    assert abs(w3(2, 3, 4, 1, -2, 1)) > 0.05


def test_jbar_vec_matches_scalar_jbar():
    edges = np.array([0.05, 0.3, 0.8, 2.0])
    r = np.array([0.01, 0.7, 3.3, 11.9, 24.0])
    for l in range(5):
        J = oracle.jbar_vec(l, edges, r)
        for a in range(3):
            for i, rr in enumerate(r):
                assert J[a, i] == pytest.approx(oracle.jbar(l, rr, edges[a], edges[a + 1]), rel=1e-11, abs=1e-14)


def test_l0_components_are_the_isotropic_multipoles():
    # S_{l l 0}(u, v) = (-1)^l L_l(u.v) / sqrt(2l + 1): B_{l l 0} = (-1)^l sqrt(2l + 1) B_l of Sec. 4.5
    rng = np.random.default_rng(3)
    L, R0 = 40.0, 8.0
    pos = rng.uniform(0, L, (120, 3))
    rnd = rng.uniform(0, L, (360, 3))
    w = rng.uniform(0.5, 1.5, 120)
    edges = np.array([0.3, 0.6, 1.0])
    B, _ = oracle.bispectrum_aniso(pos, w, rnd, L, R0, edges)
    Bi, _ = oracle.bispectrum(pos, w, rnd, L, R0, edges, 4)
    for l in range(5):
        c = COMBOS.index((l, l, 0))
        np.testing.assert_allclose(B[c], (-1) ** l * np.sqrt(2 * l + 1) * Bi[l], rtol=1e-12,
                                   atol=1e-12 * np.max(np.abs(Bi[l])))


def _tiny(N, L, seed, spread, zstretch=1.0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, L, size=3)
    d = rng.normal(0, spread, size=(N, 3))
    d[:, 2] *= zstretch
    return np.mod(c + d, L)


def _y(l, m, khat):
    # y_lm = sqrt(4 pi / (2l+1)) Y_lm (library harmonics, polar axis z)
    th = np.arccos(np.clip(khat[:, 2], -1, 1))
    ph = np.arctan2(khat[:, 1], khat[:, 0])
    return np.sqrt(4 * np.pi / (2 * l + 1)) * sph_harm_y(l, m, th, ph)


@pytest.mark.parametrize("combo", [(0, 2, 2), (1, 1, 2), (1, 3, 4), (2, 2, 2), (2, 4, 4), (4, 4, 2)])
def test_primary_sum_equals_plane_wave_definition(combo):
    # The reading's definition: B_{l1 l2 L}(k1, k2) = (2l1+1)(2l2+1) <S*_{l1 l2 L}(k1hat, k2hat)
    # Bhat(k1, k2)> over both k directions and both k shells, Bhat the DDD sum of
    # e^{-i k1.x_ij} e^{-i k2.x_ik} (j != k, windowed, i the primary) -- equals
    # (2l1+1)(2l2+1)(-1)^((l1+l2)/2) T, the oracle's per-primary form.  Library
    # harmonics and quadrature on the k side; this pins the 3j coupling, the m
    # pairing, the y normalisation and the phase.
    l1, l2, Lc = combo
    L, R0 = 60.0, 20.0
    pos = _tiny(6, L, 17, 5.0, zstretch=1.7)
    edges = np.array([0.05, 0.2, 0.35])
    T, _ = oracle.bispectrum_aniso_primary_sum(pos, np.ones(6), np.arange(6), pos, None, L, R0, edges)
    ci = COMBOS.index(combo)
    ct, wct = np.polynomial.legendre.leggauss(20)
    nphi = 40
    phi = np.arange(nphi) * 2 * np.pi / nphi
    C, PH = np.meshgrid(ct, phi, indexing="ij")
    Sn = np.sqrt(1 - C * C)
    khat = np.stack([Sn * np.cos(PH), Sn * np.sin(PH), C], axis=-1).reshape(-1, 3)
    wang = (np.outer(wct, np.full(nphi, 2 * np.pi / nphi)) / (4 * np.pi)).ravel()
    # S*(k1hat, k2hat) as a matrix over the direction grid
    Smat = np.zeros((len(khat), len(khat)), dtype=complex)
    for m in range(-min(l1, l2), min(l1, l2) + 1):
        c = oracle.wigner3j(l1, l2, Lc, m, -m, 0)
        Smat += c * np.outer(_y(l1, m, khat), _y(l2, -m, khat))
    Smat = np.conj(Smat) * wang[:, None] * wang[None, :]
    xk, wk = np.polynomial.legendre.leggauss(8)
    dvec, Wm = {}, {}
    for i in range(6):
        d = _minimage(pos - pos[i], L)
        r = np.linalg.norm(d, axis=1)
        sel = np.where((r > 0) & (r < R0))[0]
        dvec[i] = d[sel]
        Wm[i] = np.array([oracle.window(x / R0) for x in r[sel]])
    scale = max(1.0, np.max(np.abs(T[ci])))
    for a in range(2):
        for b in range(2):
            ka = 0.5 * (edges[a + 1] - edges[a]) * xk + 0.5 * (edges[a + 1] + edges[a])
            wa = 0.5 * (edges[a + 1] - edges[a]) * wk * 3 * ka ** 2 / (edges[a + 1] ** 3 - edges[a] ** 3)
            kb = 0.5 * (edges[b + 1] - edges[b]) * xk + 0.5 * (edges[b + 1] + edges[b])
            wb = 0.5 * (edges[b + 1] - edges[b]) * wk * 3 * kb ** 2 / (edges[b + 1] ** 3 - edges[b] ** 3)
            tot = 0.0 + 0.0j
            for i in range(6):
                dv, Wv = dvec[i], Wm[i]
                if len(Wv) == 0:
                    continue
                proj = khat @ dv.T  # [ndir, nnb]
                E1 = np.einsum("q,qdn->dn", wa, np.exp(-1j * ka[:, None, None] * proj[None]) * Wv)
                E2 = np.einsum("q,qdn->dn", wb, np.exp(-1j * kb[:, None, None] * proj[None]) * Wv)
                full = np.sum(E1.sum(1) * (Smat @ E2.sum(1)))
                diag = np.sum(E1 * (Smat @ E2))  # j == k terms
                tot += (2 * l1 + 1) * (2 * l2 + 1) * (full - diag)
            expect = (2 * l1 + 1) * (2 * l2 + 1) * ((-1) ** ((l1 + l2) // 2)) * T[ci, a, b]
            assert abs(tot.imag) < 1e-8 * scale * 100
            assert tot.real == pytest.approx(expect, rel=1e-7, abs=1e-8 * scale * 100)


def test_self_coupling_is_a_legendre_polynomial_of_mu():
    # S_{l1 l2 L}(u, u) = (l1 l2 L; 0 0 0) L_L(u_z): the j = k terms of a primary
    # depend on the neighbour's direction only through mu (library harmonics)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(50, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    from scipy.special import eval_legendre
    for l1, l2, Lc in COMBOS:
        s = sum(oracle.wigner3j(l1, l2, Lc, m, -m, 0) * _y(l1, m, u) * _y(l2, -m, u)
                for m in range(-min(l1, l2), min(l1, l2) + 1))
        np.testing.assert_allclose(s.real, oracle.wigner3j(l1, l2, Lc, 0, 0, 0) * eval_legendre(Lc, u[:, 2]),
                                   atol=1e-13)
        assert np.max(np.abs(s.imag)) < 1e-13


def test_random_neighbour_terms_against_an_explicit_random_catalog():
    # The analytic terms of the reading: a random neighbour on the l1 = 0 leg
    # averages y_{l1 m} to delta_{l1 0}, leaving (0 l2 L; 0 0 0) y_{l2 0} =
    # d_{L l2} (-1)^l2 / sqrt(2 l2 + 1) L_l2(mu) on the other leg, so that term of
    # T is k_l2 n W~^a DD^b_l2.  Here the continuum is a dense random catalog:
    # sum over data primaries of sum_m (0 l2 l2; 0 m -m)-weighted A^a from random
    # neighbours (scaled by n / n_R) times A^b from data neighbours, for a
    # z-elongated clustered catalog (DD_2, DD_4 far from 0), within its sampling error.
    rng = np.random.default_rng(11)
    L, R0 = 50.0, 10.0
    parents = rng.uniform(0, L, (40, 3))
    d = rng.normal(0, 1.2, (400, 3))
    d[:, 2] *= 3.0
    pos = np.mod(parents[rng.integers(0, 40, 400)] + d, L)
    rnd = rng.uniform(0, L, (60000, 3))
    edges = np.array([0.15, 0.35, 0.6])
    n = 400 / L ** 3
    nR = 60000 / L ** 3
    DD, _ = oracle.power_pair_sum(pos, None, L, R0, edges, 4, 2)
    Wt = oracle.window_transform_binned(edges, R0)
    ynorm = {l: np.sqrt(4 * np.pi / (2 * l + 1)) for l in range(5)}
    for l2 in (2,):  # (l = 4 is too weak in this catalog to resolve against the sampling error)
        tot = np.zeros((2, 2))
        for p in range(400):
            out = []
            for cat in (rnd, pos):
                dv = _minimage(cat - pos[p], L)
                r = np.linalg.norm(dv, axis=1)
                sel = (r > 0) & (r < R0)
                rs, uv = r[sel], dv[sel] / r[sel][:, None]
                Wv = np.array([oracle.window(x / R0) for x in rs])
                out.append((rs, uv, Wv))
            (rr, ur, Wr), (rd, ud, Wd) = out
            A1 = oracle.jbar_vec(0, edges, rr) @ Wr * (n / nR)  # y_00 = 1
            A2 = oracle.jbar_vec(l2, edges, rd) @ (Wd * ynorm[l2] * np.real(
                np.array([oracle.ylm(v)[l2 * l2 + l2] for v in ud])))  # m = 0 survives
            tot += oracle.wigner3j(0, l2, l2, 0, 0, 0) * np.outer(A1, A2)
        expect = ((-1.0) ** l2 / np.sqrt(2 * l2 + 1)) * n * np.outer(Wt, DD[l2 // 2])
        assert np.max(np.abs(DD[l2 // 2])) > 0.05 * np.max(np.abs(DD[0]))  # really anisotropic
        np.testing.assert_allclose(tot, expect, rtol=0.04, atol=0.04 * np.max(np.abs(expect)))


def test_symmetries():
    # rotations about the line of sight and the reflection z -> -z leave every
    # component unchanged; B^ab_{l l L} = B^ba_{l l L}; tilting the catalog
    # against the line of sight changes the L > 0 components but not L = 0
    rng = np.random.default_rng(7)
    L, R0 = 40.0, 9.0
    parents = rng.uniform(0, L, (12, 3))
    d = rng.normal(0, 1.5, (150, 3))
    d[:, 2] *= 2.5
    pos = np.mod(parents[rng.integers(0, 12, 150)] + d, L)
    edges = np.array([0.2, 0.5, 0.9])
    T0, _ = oracle.bispectrum_aniso_primary_sum(pos, np.ones(150), np.arange(150), pos, None, L, R0, edges)
    scale = np.max(np.abs(T0))
    # a quarter turn about z and the reflection z -> -z map the periodic box onto itself
    rot = np.mod(np.stack([-pos[:, 1], pos[:, 0], pos[:, 2]], axis=1), L)
    ref = np.mod(np.stack([pos[:, 0], pos[:, 1], -pos[:, 2]], axis=1), L)
    for q in (rot, ref):
        T1, _ = oracle.bispectrum_aniso_primary_sum(q, np.ones(150), np.arange(150), q, None, L, R0, edges)
        np.testing.assert_allclose(T1, T0, atol=1e-10 * scale)
    for ci, (l1, l2, _) in enumerate(COMBOS):
        if l1 == l2:
            np.testing.assert_allclose(T0[ci], T0[ci].T, atol=1e-10 * scale)
    # swapping x and z tilts the elongation onto the other axis
    tilt = np.stack([pos[:, 2], pos[:, 1], pos[:, 0]], axis=1)
    T2, _ = oracle.bispectrum_aniso_primary_sum(tilt, np.ones(150), np.arange(150), tilt, None, L, R0, edges)
    for ci, (_, _, Lc) in enumerate(COMBOS):
        if Lc == 0:
            np.testing.assert_allclose(T2[ci], T0[ci], atol=1e-10 * scale)
    moved = max(np.max(np.abs(T2[ci] - T0[ci])) for ci, (_, _, Lc) in enumerate(COMBOS) if Lc > 0)
    assert moved > 1e-3 * scale


def test_vectorised_harmonics_match_the_oracle_ylm():
    rng = np.random.default_rng(9)
    u = rng.normal(size=(20, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    np.testing.assert_allclose(oracle._ylm_vec(u), np.array([oracle.ylm(v) for v in u]), atol=1e-13)
