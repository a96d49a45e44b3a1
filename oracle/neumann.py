"""Analytical Stefan / Neumann solutions of the paper's 1D conduction cases.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Each function restates the
closed form the paper prints:

* melting of a half-space initially at T_m, Sec. 3.1.1, Eq. 60-61;
* solidification of a half-space initially above T_m, Sec. 3.1.2, Eq. 62-63.

Roots of the transcendental equations are bracketed and found with
``scipy.optimize.brentq``; ``scipy.special.erf / erfc`` are the special functions.
Positions are measured from the wall, which the lattice places half a cell
outside the first node (node i sits at i + 1/2).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import erf, erfc


def melting_k(ste_l: float) -> float:
    """Root k of Ste_l / (exp(k^2) erf(k)) = k sqrt(pi)   (Eq. 61)."""
    fn = lambda k: ste_l / (math.exp(k * k) * math.erf(k)) - k * math.sqrt(math.pi)
    return brentq(fn, 1e-12, 10.0, xtol=1e-15, rtol=1e-15, maxiter=500)


def melting_front(t, chi_l: float, k: float):
    """X(t) = 2 k sqrt(t chi_l)   (Eq. 61)."""
    return 2.0 * k * np.sqrt(np.asarray(t, dtype=np.float64) * chi_l)


def melting_temperature(x, t, chi_l, k, Th=1.0, Tm=0.0):
    """T(x, t) of Eq. 60: erf profile in the liquid (x <= X), T_m in the solid."""
    x = np.asarray(x, dtype=np.float64)
    X = melting_front(t, chi_l, k)
    liquid = Th - (Th - Tm) / math.erf(k) * erf(x / (2.0 * np.sqrt(t * chi_l)))
    return np.where(x <= X, liquid, Tm)


def solidification_k(ste_s: float, ste_l: float, chi_s: float, chi_l: float) -> float:
    """Root k of Eq. 63:
    Ste_s / (exp(k^2) erf k) - Ste_l sqrt(chi_l/chi_s) / (exp(k^2 chi_s/chi_l)
    erfc(k sqrt(chi_s/chi_l))) = k sqrt(pi)."""
    r = math.sqrt(chi_s / chi_l)

    def fn(k):
        return (ste_s / (math.exp(k * k) * math.erf(k))
                - ste_l * math.sqrt(chi_l / chi_s) / (math.exp(k * k * chi_s / chi_l)
                                                      * math.erfc(k * r))
                - k * math.sqrt(math.pi))

    return brentq(fn, 1e-12, 5.0, xtol=1e-15, rtol=1e-15, maxiter=500)


def solidification_front(t, chi_s: float, k: float):
    """X(t) = 2 k sqrt(t chi_s)   (Eq. 63)."""
    return 2.0 * k * np.sqrt(np.asarray(t, dtype=np.float64) * chi_s)


def solidification_temperature(x, t, chi_s, chi_l, k, T0=1.0, T1=-1.0, Tm=0.0):
    """T(x, t) of Eq. 62: erf profile in the solid (x <= X), erfc profile in the liquid."""
    x = np.asarray(x, dtype=np.float64)
    X = solidification_front(t, chi_s, k)
    solid = T1 + (Tm - T1) * erf(x / (2.0 * np.sqrt(chi_s * t))) / math.erf(k)
    liquid = T0 + (Tm - T0) * erfc(x / (2.0 * np.sqrt(chi_l * t))) / math.erfc(
        k * math.sqrt(chi_s / chi_l))
    return np.where(x <= X, solid, liquid)
