"""Per-bin error metrics of the parity tests (imported by the test modules).

P (power spectrum multipoles, rows l = 0, 2, 4 of a [n_ell, n_k] array):
  survey   |dP| / max(|P_l^a|, |P_0^a|)            -- the monopole of the bin sets
           the scale of all its multipoles, which cross zero;
  floored  the same with the scale floored at 1e-2 max_a' |P_0^a'|;
  plain    |dP| / |P_l^a| over the bins where P_l^a != 0.
B (bispectrum multipoles [l, a, b]):
  floored  |dB| / max(|B_l^ab|, |B_0^ab|, 1e-2 max_a'b' |B_l^a'b'|);
  survey   the same without the floor; plain as for P.
Every call prints one line "PARITY <test> <what> floored=.. survey=.. plain=..",
so a run with -s records all three beside the asserted one.
"""
import os

import numpy as np


def _plain(X, Xref):
    nz = Xref != 0
    return float(np.max(np.abs(X - Xref)[nz] / np.abs(Xref[nz]))) if np.any(nz) else 0.0


def power_metrics(P, Pref):
    P, Pref = np.asarray(P, float), np.asarray(Pref, float)
    d = np.abs(P - Pref)
    scale = np.maximum(np.abs(Pref), np.abs(Pref[0])[None, :])
    floor = 1e-2 * np.max(np.abs(Pref[0]))
    with np.errstate(divide="ignore", invalid="ignore"):
        survey = float(np.max(np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))))
    return dict(floored=float(np.max(d / np.maximum(scale, floor))), survey=survey, plain=_plain(P, Pref))


def bispec_metrics(B, Bref):
    B, Bref = np.asarray(B, float), np.asarray(Bref, float)
    d = np.abs(B - Bref)
    scale = np.maximum(np.abs(Bref), np.abs(Bref[0])[None])
    floor = 1e-2 * np.max(np.abs(Bref), axis=(1, 2))[:, None, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        survey = float(np.max(np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))))
    return dict(floored=float(np.max(d / np.maximum(scale, floor))), survey=survey, plain=_plain(B, Bref))


def report(kind, X, Xref, what=""):
    m = power_metrics(X, Xref) if kind == "P" else bispec_metrics(X, Xref)
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    print(f"PARITY {test} {what} floored={m['floored']:.3e} survey={m['survey']:.3e} plain={m['plain']:.3e}")
    return m
