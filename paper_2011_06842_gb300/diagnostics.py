"""Condition-number diagnostics of the FEWHA system (Sec. 6.2).

kappa_0 = cond(M), kappa_1 = cond(J^{-1/2} M J^{-1/2}) and
kappa_2 = cond(J^{-1/2} H^T M H J^{-1/2}), with H = I - P G^{-1} Q^T the
M-orthogonal projection away from the recycled directions P (Q = M P,
G = P^T M P; Eq. H, where G is the diagonal D_m for exactly conjugate P).
H^T M H vanishes on span(P); its condition number is taken over the rest of the
spectrum: the Lanczos start vector is placed in the operator's range, and Ritz
values below 1e-11 lambda_max (the null space, reached through rounding in long
runs) are not counted.

This is a diagnostic, not part of the time step: every operator application is
the library's M on the GPU (fewha_apply_op); the Lanczos recurrence around it
(inner products, axpys, full reorthogonalisation, the small tridiagonal
eigenproblem) uses plain tensor operations.  Lanczos finds the largest
eigenvalue quickly; its smallest Ritz value approaches lambda_min from above,
so with fewer steps than unknowns the returned kappa is a lower bound.
"""
import numpy as np


def lanczos_extremes(apply, v0, steps, null_tol=0.0):
    """Ritz values of the symmetric operator `apply` from `steps` Lanczos steps
    with full reorthogonalisation (v0 a tensor, apply(tensor) -> tensor).
    Returns (lambda_min, lambda_max, ritz_values); with null_tol > 0, Ritz
    values below null_tol * lambda_max count as the operator's null space
    (which rounding lets a long run reach even from a start in the range)."""
    import torch
    n = v0.numel()
    steps = min(steps, n)
    V = torch.zeros((steps, n), dtype=v0.dtype, device=v0.device)
    v = v0 / torch.linalg.norm(v0)
    alphas, betas = [], []
    for j in range(steps):
        V[j] = v
        w = apply(v)
        alpha = float(torch.dot(w, v))
        w = w - alpha * v
        if j > 0:
            w = w - betas[-1] * V[j - 1]
        # full reorthogonalisation (twice is enough)
        for _ in range(2):
            w = w - V[:j + 1].T @ (V[:j + 1] @ w)
        alphas.append(alpha)
        beta = float(torch.linalg.norm(w))
        if j == steps - 1 or beta <= 1e-14 * max(abs(a) for a in alphas):
            break
        betas.append(beta)
        v = w / beta
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    ritz = np.linalg.eigvalsh(T)
    kept = ritz[ritz > null_tol * ritz[-1]] if null_tol > 0 else ritz
    return float(kept[0]), float(ritz[-1]), ritz


def deflated_operator(M, P, Q, sj):
    """x -> S H^T M H S x with S = diag(sj), H = I - P^T G^{-1} Q (rows of P
    and Q are the directions p_j and M p_j, G = sym(P Q^T)); and a map taking
    any vector into the operator's range (where Lanczos must start)."""
    import torch
    P = P.to(dtype=torch.float64, device=sj.device)
    Q = Q.to(dtype=torch.float64, device=sj.device)
    G = P @ Q.T
    Gi = torch.linalg.inv(0.5 * (G + G.T))

    def H(x):
        return x - P.T @ (Gi @ (Q @ x))

    def HT(y):
        return y - Q.T @ (Gi @ (P @ y))

    def op(x):
        return sj * HT(M((H(sj * x)).contiguous()))

    return op, (lambda v: sj * HT(v))


def condition_numbers(f, basis=None, steps=200, seed=0):
    """kappa_0, kappa_1 and (if `basis` = (P, Q) rows of recycled directions and
    M times them is given) kappa_2 of an FP64 Fewha instance."""
    import torch
    if f.precision != "f64":
        raise ValueError("condition numbers need the FP64 operator")
    dev = f.device
    g = torch.Generator(device="cpu").manual_seed(seed)
    v0 = torch.randn(f.n, generator=g, dtype=torch.float64).to(dev)
    sj = torch.sqrt(torch.tensor(f.precond(), dtype=torch.float64, device=dev))  # J^{-1/2}
    M = f.apply_op
    out = {}
    lo, hi, _ = lanczos_extremes(M, v0, steps)
    out["kappa0"], out["lambda0"] = hi / lo, (lo, hi)
    lo, hi, _ = lanczos_extremes(lambda x: sj * M((sj * x).contiguous()), v0, steps)
    out["kappa1"], out["lambda1"] = hi / lo, (lo, hi)
    if basis is not None:
        op, start = deflated_operator(M, basis[0], basis[1], sj)
        lo, hi, _ = lanczos_extremes(op, start(v0), steps, null_tol=1e-11)
        out["kappa2"], out["lambda2"] = hi / lo, (lo, hi)
        out["k"] = int(basis[0].shape[0])
    out["steps"] = steps
    return out
