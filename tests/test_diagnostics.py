"""The Lanczos condition-number diagnostic on CPU (dense SPD matrices): the
Ritz extremes equal numpy's eigenvalues when Lanczos runs to the dimension, and
the deflated operator S H^T M H S has the nonzero spectrum of the same matrix
built densely; deflation by M-conjugate directions does not raise cond(M)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2011_06842_gb300.diagnostics import deflated_operator, lanczos_extremes  # noqa: E402


def spd(n, seed, spread=1e3):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, spread, n)
    return (Qm * lam) @ Qm.T


def test_lanczos_full_run_matches_eigvalsh():
    n = 60
    A = spd(n, 1)
    At = torch.tensor(A)
    lo, hi, ritz = lanczos_extremes(lambda x: At @ x, torch.randn(n, dtype=torch.float64), n)
    ev = np.linalg.eigvalsh(A)
    assert abs(lo - ev[0]) < 1e-8 * ev[-1] and abs(hi - ev[-1]) < 1e-10 * ev[-1]


def test_deflated_operator_spectrum():
    n, k = 50, 4
    A = spd(n, 2, spread=1e4)
    At = torch.tensor(A)
    rng = np.random.default_rng(3)
    P = rng.standard_normal((k, n))
    Q = P @ A
    sj = torch.tensor(rng.uniform(0.5, 2.0, n))
    op, start = deflated_operator(lambda x: At @ x, torch.tensor(P), torch.tensor(Q), sj)
    lo, hi, _ = lanczos_extremes(op, start(torch.randn(n, dtype=torch.float64)), n, null_tol=1e-11)
    # dense: S H^T A H S with H = I - P^T G^{-1} Q
    G = P @ Q.T
    H = np.eye(n) - P.T @ np.linalg.inv(0.5 * (G + G.T)) @ Q
    S = np.diag(sj.numpy())
    B = S @ H.T @ A @ H @ S
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    nz = ev[ev > 1e-9 * ev[-1]]
    assert len(nz) == n - k
    assert abs(hi - nz[-1]) < 1e-9 * nz[-1] and abs(lo - nz[0]) < 1e-7 * nz[0]
    # with S = I the deflated condition number does not exceed cond(A)
    op1, start1 = deflated_operator(lambda x: At @ x, torch.tensor(P), torch.tensor(Q), torch.ones(n, dtype=torch.float64))
    lo1, hi1, _ = lanczos_extremes(op1, start1(torch.randn(n, dtype=torch.float64)), n, null_tol=1e-11)
    evA = np.linalg.eigvalsh(A)
    assert hi1 / lo1 <= evA[-1] / evA[0] * (1 + 1e-9)
