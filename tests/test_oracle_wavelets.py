"""Pins for the oracle's Daubechies filter and periodic DWT (Sec. 3, Eq. fewha).

What fixes these values independently of the oracle:
  * orthonormality and vanishing moments of a Daubechies filter (definition);
  * Daubechies-1 is Haar and Daubechies-2 has the closed form
    (1+sqrt3, 3+sqrt3, 3-sqrt3, 1-sqrt3)/(4 sqrt2);
  * the multi-level 2-D Haar pyramid has block-sum closed forms;
  * an orthonormal transform preserves norms and is inverted by its transpose;
  * a constant layer has zero detail coefficients and approximation
    coefficients const * 2^J (2-D, J levels).
"""
import math

import numpy as np
import pytest

from oracle import daubechies_taps
from oracle import oracle as orc


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_taps_orthonormal_and_moments(N):
    h = daubechies_taps(N)
    assert len(h) == 2 * N
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    for m in range(N):
        s = sum(h[k] * h[k + 2 * m] for k in range(2 * N - 2 * m))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 1e-14, (m, s)
    n = np.arange(2 * N)
    for p in range(N):
        assert abs(np.sum((-1.0) ** n * n ** p * h)) < 1e-12 * max(1, (2 * N) ** p)


def test_taps_closed_forms():
    assert np.allclose(daubechies_taps(1), [1 / math.sqrt(2)] * 2, atol=1e-15)
    r3 = math.sqrt(3)
    d4 = np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * math.sqrt(2))
    assert np.allclose(daubechies_taps(2), d4, atol=1e-15)


def test_dwt1_haar_closed_form():
    x = np.random.default_rng(0).standard_normal(16)
    out = orc.dwt1_fwd(x, daubechies_taps(1))
    a = (x[0::2] + x[1::2]) / math.sqrt(2)
    d = (x[0::2] - x[1::2]) / math.sqrt(2)
    assert np.allclose(out, np.concatenate([a, d]), atol=1e-14)


def test_dwt2_haar_pyramid_closed_form():
    rng = np.random.default_rng(1)
    n, J = 16, 3
    x = rng.standard_normal((n, n))
    c = orc.dwt2_fwd(x, J, daubechies_taps(1))
    # coarsest approximation: block sums over 2^J x 2^J blocks divided by 2^J
    b = 2 ** J
    for r in range(n // b):
        for q in range(n // b):
            blk = x[r * b:(r + 1) * b, q * b:(q + 1) * b]
            assert abs(c[r, q] - blk.sum() / b) < 1e-12
    # finest level bands: the top-right quadrant is low-pass in y (rows) and
    # high-pass in x (columns); bottom-left the opposite; bottom-right both.
    h = n // 2
    for r in range(h):
        for q in range(h):
            x00, x01 = x[2 * r, 2 * q], x[2 * r, 2 * q + 1]
            x10, x11 = x[2 * r + 1, 2 * q], x[2 * r + 1, 2 * q + 1]
            assert abs(c[r, h + q] - (x00 - x01 + x10 - x11) / 2) < 1e-12
            assert abs(c[h + r, q] - (x00 + x01 - x10 - x11) / 2) < 1e-12
            assert abs(c[h + r, h + q] - (x00 - x01 - x10 + x11) / 2) < 1e-12


@pytest.mark.parametrize("n,J", [(8, 1), (8, 2), (16, 2), (16, 4), (32, 3), (32, 4), (64, 4),
                                 (64, 5), (128, 5), (128, 6)])
def test_dwt2_perfect_reconstruction_and_isometry(n, J):
    h = daubechies_taps(3)
    x = np.random.default_rng(n * 10 + J).standard_normal((n, n))
    c = orc.dwt2_fwd(x, J, h)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    y = orc.dwt2_inv(c, J, h)
    assert np.max(np.abs(y - x)) < 1e-12 * np.max(np.abs(x))


@pytest.mark.parametrize("n,J", [(8, 2), (16, 2)])
def test_dwt2_explicit_matrix_orthogonal(n, J):
    """W assembled column by column is orthogonal and W^{-1} is its transpose,
    including the folds where a line is shorter than the 6-tap filter."""
    h = daubechies_taps(3)
    E = np.eye(n * n)
    W = np.stack([orc.dwt2_fwd(E[i].reshape(n, n), J, h).ravel() for i in range(n * n)], axis=1)
    assert np.max(np.abs(W @ W.T - np.eye(n * n))) < 1e-13
    Winv = np.stack([orc.dwt2_inv(E[i].reshape(n, n), J, h).ravel() for i in range(n * n)], axis=1)
    assert np.max(np.abs(Winv - W.T)) < 1e-13


def test_dwt2_constant_layer():
    h = daubechies_taps(3)
    n, J = 32, 3
    c = orc.dwt2_fwd(np.full((n, n), 2.5), J, h)
    a = n >> J
    assert np.allclose(c[:a, :a], 2.5 * 2 ** J, atol=1e-12)
    det = c.copy()
    det[:a, :a] = 0
    assert np.max(np.abs(det)) < 1e-12


def test_dwt1_vanishing_moments_interior():
    """A quadratic line has zero detail coefficients wherever the 6-tap window
    does not wrap around the periodic boundary (3 vanishing moments)."""
    h = daubechies_taps(3)
    N = 32
    t = np.arange(N, dtype=float)
    x = 0.3 + 0.1 * t - 0.02 * t * t
    out = orc.dwt1_fwd(x, h)
    d = out[N // 2:]
    for k in range(N // 2):
        if 2 * k + 5 < N:
            assert abs(d[k]) < 1e-11, (k, d[k])
    assert np.max(np.abs(d)) > 1e-3  # the wrapped windows do see the jump


def test_band_of_matches_mallat_blocks():
    n, J = 32, 3
    a = n >> J
    for r in range(n):
        for q in range(n):
            s, quad = orc.band_of(n, J, r, q)
            if r < a and q < a:
                assert (s, quad) == (0, 0)
                continue
            # the band is the smallest dyadic block 2^k * a containing (r, q)
            size = a
            lev = 0
            while not (r < size and q < size):
                size *= 2
                lev += 1
            half = size // 2
            assert s == lev
            exp_quad = 1 if (r < half and q >= half) else (2 if (r >= half and q < half) else 3)
            assert quad == exp_quad
