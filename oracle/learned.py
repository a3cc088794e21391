"""FP64 oracle of the learned warm start (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): only the tests and the
CPU-baseline leg of the benchmark may use it; it shares no code with the CUDA
library.

The paper has no learned component.  The reconstructor loop it describes
(Algorithm 3) starts every time step from the previous solution; this module
states, plainly and in FP64, what the library's learned variant computes
around that loop:

- a small convolutional network (3x3 cross-correlations with zero padding,
  ReLU) over image-shaped arrays of layer coefficients, its gradients with
  respect to its inputs and parameters, the mean-squared-error loss, and
  Adam (Kingma & Ba, 2015, Algorithm 1, with bias correction);
- the prior whitening x * sqrt(s) used to scale its inputs and outputs, and
  its training targets (whitened solution increment, split by wavelet scale
  group);
- the deflated warm start: the Galerkin projection of the new time step's
  error onto predicted directions D, i.e. the initial projection of the
  augmented PCG (Algorithm 2) with D in place of the recycled basis,
  c0 = c + D w, w = (D^T M D)^{-1} D^T r0, r0 the warm-restart residual of
  Algorithm 3; it is kept only if it lowers ||r0||.

Pins (tests/test_oracle_learned.py): the convolution against
scipy.signal.correlate2d, the data gradient by the adjoint identity, the
parameter gradients by central finite differences, Adam's first steps in
closed form, the projection by the Galerkin condition D^T r = 0 and by its
energy-norm optimality against a least-squares solve.
"""
import numpy as np


# --- convolution ---------------------------------------------------------------

def _pad(x):
    """Zero padding of one pixel on both spatial axes of (B, C, H, W)."""
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


def conv3x3(x, w, b=None, relu=False):
    """out[b, co, y, x] = b[co] + sum_{ci, ky, kx} w[co, ci, ky, kx] x[b, ci, y+ky-1, x+kx-1].

    x: (B, Cin, H, W); w: (Cout, Cin, 3, 3); zero outside the image."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, Cin, H, W = x.shape
    Cout = w.shape[0]
    xp = _pad(x)
    out = np.zeros((B, Cout, H, W))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + H, kx:kx + W]          # (B, Cin, H, W)
            out += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], patch)
    if b is not None:
        out += np.asarray(b, dtype=np.float64)[None, :, None, None]
    if relu:
        out = np.maximum(out, 0.0)
    return out


def conv3x3_bwd_data(gout, w):
    """Adjoint of x -> conv3x3(x, w) (no bias, no ReLU) applied to gout (B, Cout, H, W):
    gin[b, ci, y, x] = sum_{co, ky, kx} w[co, ci, ky, kx] gout[b, co, y-ky+1, x-kx+1]."""
    gout = np.asarray(gout, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, Cout, H, W = gout.shape
    Cin = w.shape[1]
    gp = _pad(gout)
    gin = np.zeros((B, Cin, H, W))
    for ky in range(3):
        for kx in range(3):
            # gout at (y - ky + 1, x - kx + 1) = gp at (y - ky + 2, x - kx + 2)
            patch = gp[:, :, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W]
            gin += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], patch)
    return gin


def conv3x3_bwd_weight(x, gout):
    """Gradients of sum(gout * conv3x3(x, w, b)) with respect to w and b."""
    x = np.asarray(x, dtype=np.float64)
    gout = np.asarray(gout, dtype=np.float64)
    B, Cin, H, W = x.shape
    xp = _pad(x)
    gw = np.zeros((gout.shape[1], Cin, 3, 3))
    for ky in range(3):
        for kx in range(3):
            gw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gout, xp[:, :, ky:ky + H, kx:kx + W])
    return gw, gout.sum(axis=(0, 2, 3))


def relu_bwd(act, g):
    """Gradient through ReLU given its output act: zero where act <= 0."""
    return np.where(np.asarray(act) > 0.0, g, 0.0)


def mse(pred, target):
    """Loss mean((pred - target)^2) and its gradient 2 (pred - target) / n."""
    d = np.asarray(pred, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --- the network -------------------------------------------------------------------

def net_forward(x, params):
    """Three 3x3 convolutions, ReLU after the first two.  params: w1, b1, w2, b2, w3, b3.
    Returns the output and the hidden activations (h1, h2)."""
    h1 = conv3x3(x, params["w1"], params["b1"], relu=True)
    h2 = conv3x3(h1, params["w2"], params["b2"], relu=True)
    return conv3x3(h2, params["w3"], params["b3"]), (h1, h2)


def net_backward(x, params, hidden, gy):
    """Parameter gradients of sum(gy * net_forward(x)) (chain rule, layer by layer)."""
    h1, h2 = hidden
    g = {}
    g["w3"], g["b3"] = conv3x3_bwd_weight(h2, gy)
    gh2 = relu_bwd(h2, conv3x3_bwd_data(gy, params["w3"]))
    g["w2"], g["b2"] = conv3x3_bwd_weight(h1, gh2)
    gh1 = relu_bwd(h1, conv3x3_bwd_data(gh2, params["w2"]))
    g["w1"], g["b1"] = conv3x3_bwd_weight(x, gh1)
    return g


# --- whitening, targets and the deflated warm start ------------------------------

def whiten(x, s):
    """x * sqrt(s) elementwise."""
    return np.asarray(x, dtype=np.float64) * np.sqrt(np.asarray(s, dtype=np.float64))


def targets(c_next, c_cur, s, group):
    """Five target channels: t0 = (c_next - c_cur) sqrt(s); t_k = t0 on the
    coefficients of scale group k (k = 1..4), zero elsewhere."""
    t0 = whiten(np.asarray(c_next, np.float64) - np.asarray(c_cur, np.float64), s)
    out = [t0]
    for k in range(1, 5):
        out.append(np.where(np.asarray(group) == k, t0, 0.0))
    return np.stack(out)


def deflate_warm_start(b, D, Q, c, b_prev, r_prev):
    """Galerkin correction of the warm start over the rows of D (Q = M D).

    r0 = (b - b_prev) + r_prev; w solves sym(D^T Q) w = D^T r0; the correction
    c + D w with residual r0 - Q w is taken if ||r0 - Q w|| < ||r0||.  Either
    way this time step's right-hand side is folded into the state: b_prev <- b
    and r_prev <- the warm-restart residual (r0 - Q w if taken, else r0, the
    plain warm start of Algorithm 3), so that the solve that follows need not
    form the right-hand side again.
    Returns (taken, c_new, b_prev_new, r_prev_new, w, ||r0 - Q w||, ||r0||).
    Directions are assumed linearly independent (no pivot is dropped)."""
    b, D, Q = (np.asarray(a, dtype=np.float64) for a in (b, D, Q))
    c, b_prev, r_prev = (np.asarray(a, dtype=np.float64) for a in (c, b_prev, r_prev))
    r0 = (b - b_prev) + r_prev
    G = D @ Q.T
    G = 0.5 * (G + G.T)
    w = np.linalg.solve(G, D @ r0)
    r1 = r0 - Q.T @ w
    n1, n0 = float(np.linalg.norm(r1)), float(np.linalg.norm(r0))
    if n1 < n0:
        return True, c + D.T @ w, b.copy(), r1, w, n1, n0
    return False, c.copy(), b.copy(), r0, w, n1, n0
