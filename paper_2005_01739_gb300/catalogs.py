"""Seeded synthetic catalogs (inputs only; none of the estimator's arithmetic).

These stand in for the N-body halo and matter catalogs the paper measures
(Quijote halos and matter particles, Sec. 9), which are not available here:

* ``thomas`` -- a Thomas (Neyman-Scott) cluster process: uniform parents, each
  with Gaussian-displaced children, optional uniform background and an optional
  Gaussian line-of-sight displacement (a stand-in for redshift-space distortion);
* ``zeldovich_lattice`` -- a lattice displaced by the Zel'dovich field of a
  Gaussian random field with P(k) ~ k^-2 (a stand-in for matter particles);
* ``uniform`` -- uniform random points (Poisson nulls and bispectrum randoms).

All positions are generated in float64, wrapped into [0, L) and rounded to
float32, the precision the kernels read.  This module is shared by the tests,
the benchmark and the oracle checks; it imports nothing from the estimator.
"""
from __future__ import annotations

import numpy as np


def _wrap32(x: np.ndarray, L: float) -> np.ndarray:
    x = np.mod(x, L)
    out = x.astype(np.float32)
    out[out >= np.float32(L)] = 0.0  # float32 rounding can land exactly on L
    return out


def uniform(N: int, L: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _wrap32(rng.uniform(0.0, L, size=(N, 3)), L)


def thomas(N: int, L: float, n_parents: int, sigma: float, seed: int,
           background_frac: float = 0.0, los_sigma: float = 0.0,
           weights: str = "unit"):
    """Thomas process with exactly N points.

    ``round(background_frac * N)`` points are uniform; the rest are children,
    assigned to the ``n_parents`` uniform parents multinomially (equal
    probabilities, i.e. Poisson counts conditioned on the total) and offset by
    N(0, sigma^2 I).  If ``los_sigma`` > 0 every point's z is shifted by
    N(0, los_sigma^2).  ``weights``: "unit" -> None, "u05_15" -> U(0.5, 1.5)."""
    rng = np.random.default_rng(seed)
    nb = int(round(background_frac * N))
    nc = N - nb
    parents = rng.uniform(0.0, L, size=(n_parents, 3))
    counts = rng.multinomial(nc, np.full(n_parents, 1.0 / n_parents))
    owner = np.repeat(np.arange(n_parents), counts)
    kids = parents[owner] + rng.normal(0.0, sigma, size=(nc, 3))
    bg = rng.uniform(0.0, L, size=(nb, 3))
    pos = np.concatenate([kids, bg], axis=0)
    if los_sigma > 0:
        pos[:, 2] += rng.normal(0.0, los_sigma, size=N)
    perm = rng.permutation(N)
    pos = _wrap32(pos[perm], L)
    if weights == "unit":
        w = None
    elif weights == "u05_15":
        w = rng.uniform(0.5, 1.5, size=N).astype(np.float32)
    else:
        raise ValueError(weights)
    return pos, w


def zeldovich_lattice(n_side: int, L: float, seed: int, rms_disp: float = 2.0,
                      spectral_index: float = -2.0) -> np.ndarray:
    """n_side^3 particles on a lattice displaced by psi(k) = i k delta(k) / k^2.

    delta is a Gaussian random field on the n_side^3 grid with P(k) ~ k^n
    (n = spectral_index, zero mode removed); the displacement amplitude is
    scaled so that the rms 1-D displacement equals ``rms_disp``."""
    rng = np.random.default_rng(seed)
    g = n_side
    white = rng.normal(size=(g, g, g))
    dk = np.fft.rfftn(white)
    kf = 2.0 * np.pi / L
    kx = np.fft.fftfreq(g, d=1.0 / g) * kf
    kz = np.fft.rfftfreq(g, d=1.0 / g) * kf
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k2[0, 0, 0] = 1.0
    amp = np.power(np.sqrt(k2), 0.5 * spectral_index)
    amp[0, 0, 0] = 0.0
    dk *= amp
    disp = []
    for K in (KX, KY, KZ):
        psi_k = 1j * K * dk / k2
        psi_k[0, 0, 0] = 0.0
        disp.append(np.fft.irfftn(psi_k, s=(g, g, g), axes=(0, 1, 2)))
    disp = np.stack(disp, axis=-1).reshape(-1, 3)
    rms = np.sqrt(np.mean(disp * disp))
    disp *= rms_disp / rms
    q = (np.arange(g) + 0.5) * (L / g)
    QX, QY, QZ = np.meshgrid(q, q, q, indexing="ij")
    lattice = np.stack([QX, QY, QZ], axis=-1).reshape(-1, 3)
    return _wrap32(lattice + disp, L)


# ----------------------------------------------------------- named workloads --
def linear_edges(k_lo: float, k_hi: float, n: int) -> np.ndarray:
    return np.linspace(k_lo, k_hi, n + 1)


def workload(name: str):
    """The benchmark workloads (seed = 1000 + index).  Returns a dict with the
    catalog and the estimator settings."""
    if name == "pk_plain_n5e4":  # index 0
        pos, w = thomas(50_000, 500.0, 2000, 2.0, 1000, background_frac=0.1, los_sigma=3.0)
        return dict(pos=pos, w=w, L=500.0, R0=20.0, edges=linear_edges(0.2, 2.0, 30), ell_max=4)
    if name == "pk_mixed_n2e6":  # index 1
        pos, w = thomas(2_000_000, 1000.0, 50_000, 1.5, 1001, weights="u05_15")
        return dict(pos=pos, w=w, L=1000.0, R0=50.0, edges=linear_edges(0.1, 5.0, 100), ell_max=4)
    if name == "bk_n5e5":  # index 2
        pos, w = thomas(500_000, 1000.0, 12_500, 1.5, 1002)
        rand = uniform(1_500_000, 1000.0, 1002 + 7919)
        return dict(pos=pos, w=w, rand=rand, L=1000.0, R0=40.0, edges=linear_edges(0.3, 3.0, 25), lmax=4)
    if name == "batched64":  # index 3
        return dict(catalogs=[batched_catalog(c) for c in range(64)])
    if name == "large_zeldovich":  # index 4
        pos = zeldovich_lattice(256, 1000.0, 1004)
        edges_p = linear_edges(1.25, 10.0, 200)            # R0 = 20: k_min = 25/R0
        edges_b = linear_edges(25.0 / 15.0, 25.0 / 15.0 + 40 * 3.0 / 15.0, 40)  # R0 = 15, dk = 3/R0
        return dict(pos=pos, w=None, L=1000.0, R0=20.0, edges=edges_p, ell_max=4, R0_b=15.0, edges_b=edges_b,
                    lmax=4)
    raise KeyError(name)


def batched_catalog(c: int):
    """Catalog c of the 64-catalog batch (seed 2000 + c): N log-uniform in
    [1e5, 4e6], L uniform in [500, 2000], R0 drawn from {10, 20, 40}; bins of
    width 3/R0 from k = 25/R0 up to 10 h/Mpc (the R0 ~ 1/k_min and dk >~ 3/R0
    rules of Sec. 9.1); Thomas process as the 2e6 workload (sigma 1.5, 40
    children per parent, weights U(0.5, 1.5))."""
    rng = np.random.default_rng(2000 + c)
    N = int(np.exp(rng.uniform(np.log(1e5), np.log(4e6))))
    L = float(rng.uniform(500.0, 2000.0))
    R0 = float(rng.choice([10.0, 20.0, 40.0]))
    nk = int((10.0 * R0 - 25.0) // 3.0)
    edges = np.linspace(25.0 / R0, 25.0 / R0 + nk * 3.0 / R0, nk + 1)
    pos, w = thomas(N, L, max(1, N // 40), 1.5, 2000 + c, weights="u05_15")
    return dict(pos=pos, w=w, L=L, R0=R0, edges=edges, ell_max=4, los_axis=2)
