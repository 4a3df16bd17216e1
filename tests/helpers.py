"""Shared test helpers: conversions between the oracle's and the library's layouts."""
import math

import numpy as np

import oracle.dbfft_oracle as o

MANDEL_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def e9_to_oracle(prob, e9):
    """Library macro vector [9] (Mandel 0..5 or 3i+j) -> oracle's active vector."""
    idx = np.nonzero(prob.active)[0]
    return np.asarray(e9, dtype=np.float64)[idx]


def e_oracle_to9(prob, e):
    out = np.zeros(9)
    out[np.nonzero(prob.active)[0]] = e
    return out


def iso_tangent(phase, E, nu, scale=None):
    lam, mu = o.lame(np.asarray(E)[phase], np.asarray(nu)[phase])
    if scale is not None:
        lam, mu = lam * scale, mu * scale
    return o.IsoTangent(lam, mu)


def mask9(pairs):
    m = np.zeros((3, 3), bool)
    for i, j in pairs:
        m[i, j] = m[j, i] = True
    return m.reshape(-1)
