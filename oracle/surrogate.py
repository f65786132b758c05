"""Features and targets of the warm-rain surrogate -- TEST INFRASTRUCTURE.

The surrogate replaces the four warm-rain rates of the scheme
(autoconversion, accretion, cloud and rain self-collection) at a point.  Its
12 inputs are taken from the state the rates see (after saturation
adjustment and activation); its 4 outputs are the natural logarithms of the
rates.  A rate is defined (mask 1) where the scheme computes it: cloud
present for autoconversion and cloud self-collection, cloud and rain for
accretion, rain with a positive number for rain self-collection.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

QMIN = 1e-14
# state indices
T, QV, QC, QR, NC, NR, NA, P, RHO, W = 0, 1, 2, 3, 7, 8, 12, 13, 14, 15


def features(st: np.ndarray) -> np.ndarray:
    """12 features of one post-activation state (FP64)."""
    return np.array([
        math.log(max(st[QC], QMIN)),
        math.log(max(st[QR], QMIN)),
        math.log(max(st[NC], 1.0)),
        math.log(max(st[NR], 1e-3)),
        math.log(st[RHO]),
        st[T] - 273.15,
        math.log(st[P]),
        math.log(max(st[QV], 1e-10)),
        st[W],
        math.log(max(st[NA], 1.0)),
        1.0 if st[QC] > QMIN else 0.0,
        1.0 if st[QR] > QMIN else 0.0,
    ])


def targets(st: np.ndarray, dt: float = 1.0):
    """(log-rates[4], mask[4]) of one post-activation state from the oracle's rates."""
    r = O.rates(st, dt)
    vals = (r["aut"], r["acc"], r["scc"], r["scr"])
    hc, hr = st[QC] > QMIN, st[QR] > QMIN
    defined = (hc, hc and hr, hc, hr and vals[3] > 0.0)
    y = np.array([math.log(v) if d and v > 0.0 else 0.0 for v, d in zip(vals, defined)])
    m = np.array([1.0 if d and v > 0.0 else 0.0 for v, d in zip(vals, defined)])
    return y, m


def warm(st: np.ndarray) -> bool:
    """Points the surrogate serves: cloud or rain present after adjustment."""
    return st[QC] > QMIN or st[QR] > QMIN
