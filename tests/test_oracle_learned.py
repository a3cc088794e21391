"""Pins of the learned-warm-start oracle (oracle/learned.py) against facts
outside it: an independent convolution routine, the adjoint identity, finite
differences, Adam's closed-form first steps, and the Galerkin conditions of
the deflated warm start."""
import numpy as np
import pytest

from oracle import learned as L

signal = pytest.importorskip("scipy.signal")


def rand(*shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_scipy_correlate2d():
    x, w, b = rand(2, 3, 7, 9, seed=1), rand(4, 3, 3, 3, seed=2), rand(4, seed=3)
    y = L.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for bi in range(2):
        for co in range(4):
            ref[bi, co] = b[co] + sum(signal.correlate2d(x[bi, ci], w[co, ci], mode="same", boundary="fill")
                                      for ci in range(3))
    assert np.max(np.abs(y - ref)) < 1e-12
    assert np.max(np.abs(L.conv3x3(x, w, b, relu=True) - np.maximum(ref, 0.0))) < 1e-12


def test_conv_single_tap_is_a_shift():
    # w with one non-zero tap at (ky, kx) = (0, 2): out[y, x] = in[y - 1, x + 1]
    x = rand(1, 1, 5, 6, seed=4)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 0, 2] = 1.0
    y = L.conv3x3(x, w)
    assert np.all(y[0, 0, 0, :] == 0.0) and np.all(y[0, 0, :, -1] == 0.0)
    assert np.array_equal(y[0, 0, 1:, :-1], x[0, 0, :-1, 1:])


def test_conv_data_gradient_is_the_adjoint():
    x, w, g = rand(3, 5, 8, 6, seed=5), rand(7, 5, 3, 3, seed=6), rand(3, 7, 8, 6, seed=7)
    lhs = np.sum(L.conv3x3(x, w) * g)
    rhs = np.sum(x * L.conv3x3_bwd_data(g, w))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_conv_weight_gradient_by_finite_differences():
    x, w, b, g = rand(2, 3, 6, 5, seed=8), rand(4, 3, 3, 3, seed=9), rand(4, seed=10), rand(2, 4, 6, 5, seed=11)
    gw, gb = L.conv3x3_bwd_weight(x, g)
    f = lambda w_, b_: np.sum(L.conv3x3(x, w_, b_) * g)  # noqa: E731
    h = 1e-3  # f is linear in (w, b): central differences are exact up to rounding
    for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 0), (2, 0, 1, 1)]:
        e = np.zeros_like(w)
        e[idx] = h
        fd = (f(w + e, b) - f(w - e, b)) / (2 * h)
        assert abs(fd - gw[idx]) < 1e-9 * max(1.0, abs(fd))
    for co in range(4):
        e = np.zeros(4)
        e[co] = h
        assert abs((f(w, b + e) - f(w, b - e)) / (2 * h) - gb[co]) < 1e-9 * max(1.0, abs(gb[co]))


def test_network_gradient_by_finite_differences():
    rng = np.random.default_rng(12)
    p = {"w1": rng.standard_normal((6, 4, 3, 3)) * 0.4, "b1": rng.standard_normal(6) * 0.1,
         "w2": rng.standard_normal((6, 6, 3, 3)) * 0.3, "b2": rng.standard_normal(6) * 0.1,
         "w3": rng.standard_normal((5, 6, 3, 3)) * 0.3, "b3": rng.standard_normal(5) * 0.1}
    x, t = rng.standard_normal((2, 4, 7, 5)), rng.standard_normal((2, 5, 7, 5))

    def loss(pp):
        y, _ = L.net_forward(x, pp)
        return L.mse(y, t)[0]

    y, hid = L.net_forward(x, p)
    _, gy = L.mse(y, t)
    g = L.net_backward(x, p, hid, gy)
    h = 1e-6
    checked = 0
    for name in p:
        flat = p[name].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[i] += h
            lp = loss(q)
            q[name].reshape(-1)[i] -= 2 * h
            lm = loss(q)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[i]) < 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, i)
            checked += 1
    assert checked >= 30


def test_mse_and_relu_backward():
    p, t = rand(3, 4, seed=13), rand(3, 4, seed=14)
    loss, g = L.mse(p, t)
    assert abs(loss - np.sum((p - t) ** 2) / 12) < 1e-15
    assert np.allclose(g, (p - t) / 6, rtol=0, atol=1e-15)
    act = np.array([0.0, 1.0, -0.0, 2.0])
    assert np.array_equal(L.relu_bwd(act, np.array([5.0, 6.0, 7.0, 8.0])), np.array([0.0, 6.0, 0.0, 8.0]))


def test_adam_first_steps_closed_form():
    p0, g = np.array([1.0, -2.0, 0.5]), np.array([0.3, -4.0, 1e-3])
    lr, eps = 0.01, 1e-8
    p1, m, v = L.adam(p0, g, np.zeros(3), np.zeros(3), 1, lr, eps=eps)
    # step 1: bias-corrected moments are g and g^2, so the step is lr g / (|g| + eps)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # step 2 with the same gradient: still g and g^2 after correction
    p2, _, _ = L.adam(p1, g, m, v, 2, lr, eps=eps)
    assert np.allclose(p2, p1 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)


def test_targets_split_the_increment():
    rng = np.random.default_rng(15)
    n = 50
    cn, cc, s = rng.standard_normal(n), rng.standard_normal(n), rng.uniform(0.5, 2.0, n)
    grp = rng.integers(1, 5, n)
    T = L.targets(cn, cc, s, grp)
    assert T.shape == (5, n)
    assert np.allclose(T[1:].sum(axis=0), T[0], rtol=0, atol=1e-15)
    assert np.allclose(T[0], (cn - cc) * np.sqrt(s), rtol=0, atol=1e-15)


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def test_deflation_galerkin_condition_and_optimality():
    n, k = 40, 5
    M = _spd(n, 16)
    rng = np.random.default_rng(17)
    c_true = rng.standard_normal(n)
    b = M @ c_true
    c = c_true + 0.3 * rng.standard_normal(n)           # a warm start
    b_prev = rng.standard_normal(n)
    r_prev = (b_prev - M @ c)                            # consistent previous residual
    D = rng.standard_normal((k, n))
    Q = D @ M                                            # rows: M d_j (M symmetric)
    taken, c1, bp1, rp1, w, n1, n0 = L.deflate_warm_start(b, D, Q, c, b_prev, r_prev)
    r0 = b - M @ c
    assert abs(n0 - np.linalg.norm(r0)) < 1e-12 * n0
    assert taken and n1 < n0
    # Galerkin condition: the new residual is orthogonal to the directions
    assert np.max(np.abs(D @ rp1)) < 1e-10 * np.linalg.norm(r0) * np.linalg.norm(D)
    assert np.allclose(rp1, b - M @ c1, rtol=0, atol=1e-10 * n0)
    assert np.array_equal(bp1, b)
    # energy-norm optimality: w minimises ||c_true - (c + D^T w)||_M
    Lc = np.linalg.cholesky(M)
    w_ls, *_ = np.linalg.lstsq(Lc.T @ D.T, Lc.T @ (c_true - c), rcond=None)
    assert np.allclose(w, w_ls, rtol=1e-9, atol=1e-12)


def test_deflation_gate_keeps_the_plain_warm_start():
    n = 30
    M = _spd(n, 18)
    rng = np.random.default_rng(19)
    c = rng.standard_normal(n)
    b = M @ c                                            # the warm start is already exact
    D = rng.standard_normal((2, n))
    taken, c1, bp1, rp1, w, n1, n0 = L.deflate_warm_start(b, D, D @ M, c, b, np.zeros(n))
    assert not taken and n0 == 0.0
    assert np.array_equal(c1, c) and np.array_equal(rp1, np.zeros(n))
    # not taken: with d = e_0 and q = e_0 + 10 e_1, r0 = e_0 gives w = 1 and
    # ||r0 - q w|| = 10 > ||r0||, so the plain warm restart r0 = (b - b_prev)
    # + r_prev is folded into the state unchanged
    e0, e1 = np.eye(n)[0], np.eye(n)[1]
    b2 = b + e0
    taken, c1, bp1, rp1, w, n1, n0 = L.deflate_warm_start(b2, e0[None, :], (e0 + 10 * e1)[None, :], c, b,
                                                          np.zeros(n))
    assert not taken and abs(w[0] - 1.0) < 1e-15 and abs(n1 - 10.0) < 1e-12
    assert np.array_equal(c1, c) and np.array_equal(bp1, b2) and np.array_equal(rp1, (b2 - b) + np.zeros(n))
