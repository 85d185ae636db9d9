"""The approximation the power spectrum's moment pass rests on, checked on the CPU.

The pair pass of Sec. 3 needs, per bin edge k and multipole l, the edge
function f(r) = k^3 F_l(r k) with F_l(u) = D_l(u)/u^3 (App. C).  The moment pass
expands f on every interval of width h2 = R0/n_c, n_c = max(8, ceil(R0 k_max/4)),
in 16 Legendre polynomials of the interval coordinate.  f is band-limited
(F_l(u) is the average of j_l(u y) over y in [0, 1], its spectrum in r lies in
[-k, k]), so its Legendre coefficients on an interval of half-width h fall like
(2m+1)(k h)^m/(2m+1)!!; with k h <= 2 the 16-term expansion must reproduce f to
~1e-12 of max|f|.  These tests evaluate that claim with the oracle's own D_l (no
code of the CUDA path is involved): 24-point Gauss-Legendre projection, as the
library does, then the truncated series on a dense grid.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle

M = 16


def _f(l, k, r):
    u = r * k
    return np.array([k ** 3 * oracle.dhat(l, x) / x ** 3 if x > 0 else (k ** 3 / 3.0 if l == 0 else 0.0)
                     for x in u])


def _max_trunc_err(l, k, r0, h2):
    gx, gw = Lg.leggauss(24)
    V = Lg.legvander(gx, M - 1)
    a = (V * gw[:, None]).T @ _f(l, k, r0 + 0.5 * h2 * (1 + gx)) * (2 * np.arange(M) + 1) / 2
    t = np.linspace(-1, 1, 401)
    exact = _f(l, k, r0 + 0.5 * h2 * (1 + t))
    return float(np.max(np.abs(Lg.legval(t, a) - exact)))


@pytest.mark.parametrize("l", [0, 2, 4])
@pytest.mark.parametrize("R0,kmax", [(50.0, 5.0), (12.0, 10.0), (17.3, 14.0), (20.0, 51.2)])
def test_sixteen_legendre_terms_reproduce_the_edge_function(l, R0, kmax):
    n_c = max(8, int(np.ceil(R0 * kmax / 4.0)))
    h2 = R0 / n_c
    assert kmax * h2 / 2 <= 2.0 + 1e-12
    fmax = kmax ** 3 / 3.0  # |k^3 F_l| <= k^3 F_0(0) = k^3 / 3
    # the largest edge (the hardest) and a mid edge, on the first, a middle and the last interval
    for k in (kmax, 0.37 * kmax):
        for c in (0, n_c // 2, n_c - 1):
            err = _max_trunc_err(l, k, c * h2, h2)
            assert err < 1e-12 * fmax, (l, k, c, err / fmax)


def test_wider_intervals_fail_the_bound():
    # the bound is not vacuous: at k h = 8 sixteen terms no longer suffice
    R0, kmax = 20.0, 10.0
    h2 = 16.0 / kmax
    err = _max_trunc_err(0, kmax, 5 * h2, h2)
    assert err > 1e-9 * kmax ** 3 / 3.0


def test_moment_decomposition_reproduces_the_pair_sum():
    # the whole decomposition in FP64 numpy: moments of omega L_l P_m(t) per interval, contracted with the
    # edge functions' Legendre coefficients, differenced over the bin edges -> DD, against the oracle's
    # brute-force pair sum (Sec. 3).  No CUDA code is involved.
    rng = np.random.default_rng(5)
    N, L, R0 = 300, 40.0, 10.0
    pos = rng.uniform(0, L, (N, 3))
    w = rng.uniform(0.5, 1.5, N)
    edges = np.linspace(0.2, 3.0, 15)
    DDref, _ = oracle.power_pair_sum(pos, w, L, R0, edges, 4, 2)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(N, 1)
    rr, dz = r[iu], d[..., 2][iu]
    ww = (w[:, None] * w[None, :])[iu]
    keep = (rr > 0) & (rr < R0)
    rr, mu, ww = rr[keep], dz[keep] / rr[keep], ww[keep]
    om = 2.0 * ww * np.array([oracle.window(x) for x in rr / R0])  # both orders of each pair
    Lw = [np.ones_like(mu), 0.5 * (3 * mu ** 2 - 1), (35 * mu ** 4 - 30 * mu ** 2 + 3) / 8]
    n_c = max(8, int(np.ceil(R0 * edges[-1] / 4.0)))
    h2 = R0 / n_c
    c = np.minimum((rr / h2).astype(int), n_c - 1)
    t = (rr - c * h2) / (0.5 * h2) - 1.0
    P = Lg.legvander(t, M - 1)
    gx, gw = Lg.leggauss(24)
    V = Lg.legvander(gx, M - 1)
    S = np.zeros((3, len(edges)))
    for il, l in enumerate((0, 2, 4)):
        mom = np.zeros((n_c, M))
        np.add.at(mom, c, (om * Lw[il])[:, None] * P)
        for e, k in enumerate(edges):
            for cc in range(n_c):
                f = _f(l, k, cc * h2 + 0.5 * h2 * (1 + gx))
                a = (V * gw[:, None]).T @ f * (2 * np.arange(M) + 1) / 2
                S[il, e] += a @ mom[cc]
    k3 = edges ** 3
    DD = 3 * (S[:, 1:] - S[:, :-1]) / (k3[1:] - k3[:-1])
    assert np.max(np.abs(DD - DDref)) < 1e-11 * np.max(np.abs(DDref))
