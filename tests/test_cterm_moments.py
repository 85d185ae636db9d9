"""The approximation the bispectrum's C term rests on, checked on the CPU.

Summed over primaries, the C term of Eq. AC-def (binned as in Sec. 4.4) is a
pair sum of a function of the separation alone:

    sum_p s_p C^ab_l(x_p) = sum_(p,j) s_p w_j^2 W(r_pj)^2 f(r_pj),
    f(r) = jbar^a_l(r) jbar^b_l(r),

so the bispectrum pass only accumulates, per interval of width R0/n_cc,
n_cc = ceil(R0 k_max / 8), the 32 Legendre moments of s_p w_j^2 W^2 in the
interval coordinate t; the products f are projected on the same polynomials in
FP64 afterwards.  f is band-limited to 2 k_max (a product of two functions of
bandwidth <= k_max), so on an interval of half-width h its Legendre coefficients
fall like (2m+1)(2 k_max h)^m/(2m+1)!! with 2 k_max h <= 8: 32 terms must
reproduce f to ~1e-12 of max|f|.  Checked with the oracle's jbar (no CUDA code),
and the whole decomposition against a brute-force pair sum.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle

M = 32


def _n_cc(R0, kmax):
    return max(1, int(np.ceil(R0 * kmax / 8.0)))


def _f(l, edges, a, b, r):
    return np.array([oracle.jbar(l, x, edges[a], edges[a + 1]) * oracle.jbar(l, x, edges[b], edges[b + 1])
                     for x in r])


def _max_trunc_err(l, edges, a, b, r0, h2):
    gx, gw = Lg.leggauss(64)
    V = Lg.legvander(gx, M - 1)
    coef = (V * gw[:, None]).T @ _f(l, edges, a, b, r0 + 0.5 * h2 * (1 + gx)) * (2 * np.arange(M) + 1) / 2
    t = np.linspace(-1, 1, 301)
    exact = _f(l, edges, a, b, r0 + 0.5 * h2 * (1 + t))
    return float(np.max(np.abs(Lg.legval(t, coef) - exact)))


@pytest.mark.parametrize("l", [0, 2, 4])
@pytest.mark.parametrize("R0,kmax,nk", [(40.0, 3.0, 25), (15.0, 9.67, 40), (12.0, 40.0, 20)])
def test_thirty_two_legendre_terms_reproduce_the_product(l, R0, kmax, nk):
    edges = np.linspace(kmax / 10.0, kmax, nk + 1)
    n_cc = _n_cc(R0, kmax)
    h2 = R0 / n_cc
    assert 2 * kmax * h2 / 2 <= 8.0 + 1e-12
    # the top bins (the hardest) and a low one, on the first, a middle and the last interval
    for a, b in ((nk - 1, nk - 1), (nk - 2, nk - 1), (0, nk - 1)):
        fmax = 1.0  # |jbar| <= 1
        for c in (0, n_cc // 2, n_cc - 1):
            err = _max_trunc_err(l, edges, a, b, c * h2, h2)
            assert err < 1e-12 * fmax, (l, a, b, c, err)


def test_wider_intervals_fail_the_bound():
    # the bound is not vacuous: at 2 k_max h = 24 thirty-two terms no longer suffice
    kmax = 10.0
    edges = np.linspace(1.0, kmax, 10)
    h2 = 24.0 / kmax
    assert _max_trunc_err(0, edges, 8, 8, 0.0, h2) > 1e-7


def test_cterm_moment_decomposition_reproduces_the_pair_sum():
    # moments of s_p w_j^2 W^2 P_m(t) per interval, each interval's density rebuilt from its 32
    # moments and integrated against jbar^a_l jbar^b_l by Gauss-Legendre, against the direct pair
    # sum of the same products (FP64 numpy; no CUDA code)
    rng = np.random.default_rng(8)
    N, L, R0 = 200, 40.0, 10.0
    pos = rng.uniform(0, L, (N, 3))
    w = rng.uniform(0.5, 1.5, N)
    s = np.where(rng.uniform(size=N) < 0.5, w, -0.7)  # data-like and random-like primary weights
    edges = np.linspace(0.3, 4.0, 9)
    nk = len(edges) - 1
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    pi, pj = np.nonzero((r > 0) & (r < R0))
    rr = r[pi, pj]
    wgt = s[pi] * w[pj] ** 2 * np.array([oracle.window(x / R0) for x in rr]) ** 2
    n_cc = _n_cc(R0, edges[-1])
    h2 = R0 / n_cc
    c = np.minimum((rr / h2).astype(int), n_cc - 1)
    t = (rr - c * h2) / (0.5 * h2) - 1.0
    mom = np.zeros((n_cc, M))
    np.add.at(mom, c, wgt[:, None] * Lg.legvander(t, M - 1))
    gx, gw = Lg.leggauss(48)
    V = Lg.legvander(gx, M - 1)
    rho = mom @ (V * (2 * np.arange(M) + 1) / 2).T  # [n_cc][node]
    for l in (0, 1, 3, 4):
        jb = np.array([[oracle.jbar(l, x, edges[a], edges[a + 1]) for x in rr] for a in range(nk)])
        ref = (jb * wgt[None, :]) @ jb.T
        got = np.zeros((nk, nk))
        for cc in range(n_cc):
            rn = cc * h2 + 0.5 * h2 * (1 + gx)
            jn = np.array([[oracle.jbar(l, x, edges[a], edges[a + 1]) for x in rn] for a in range(nk)])
            got += (jn * (gw * rho[cc])[None, :]) @ jn.T
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)), l
