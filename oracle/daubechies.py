"""Daubechies filter taps for the oracle, from Daubechies' construction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper uses periodic orthonormal Daubechies-3 wavelets (Sec. 3, after
Eq. fewha).  The reading taken here is the extremal-phase filter with N = 3
vanishing moments (6 taps).  The taps are built, not typed in:

  |H(w)|^2 = 2 cos^{2N}(w/2) P_N(sin^2(w/2)),  P_N(y) = sum_{k<N} C(N-1+k, k) y^k.

Each root y_k of P_N gives, through y = (2 - z - 1/z)/4, a reciprocal pair of
roots z; the one inside the unit circle is kept (minimum phase).  Then
h(z) = c (1 + z^{-1})^N prod_k (1 - z_k z^{-1}), normalised to sum h = sqrt(2).
numpy's polynomial root finder is the one library step.
"""
from math import comb, sqrt

import numpy as np


def daubechies_taps(N: int) -> np.ndarray:
    """Low-pass taps h_0..h_{2N-1} of the extremal-phase Daubechies-N filter."""
    if N < 1:
        raise ValueError("N >= 1")
    # P_N coefficients, highest power first for numpy.roots
    pc = [comb(N - 1 + k, k) for k in range(N)][::-1]
    yroots = np.roots(pc) if N > 1 else np.array([])
    poly = np.array([1.0 + 0j])
    for y in yroots:
        a = 1.0 - 2.0 * y
        disc = np.sqrt(a * a - 1.0 + 0j)
        z1, z2 = a + disc, a - disc
        z = z1 if abs(z1) < 1.0 else z2
        poly = np.convolve(poly, np.array([1.0, -z]))
    for _ in range(N):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    h = np.real(poly)
    h = h * (sqrt(2.0) / h.sum())
    return h.astype(np.float64)
