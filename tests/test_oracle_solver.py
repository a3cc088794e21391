"""Pins for the oracle's PCG (Algorithm 1) and augmented PCG (Algorithm 2).

Independent facts used (Sec. 4, Sec. 6.2):
  * preconditioned CG on an SPD system of size n reaches the exact solution
    c* = M^{-1} b (dense Cholesky) in at most n steps;
  * residuals are J^{-1}-orthogonal, (r_i, z_j) = 0 for i != j, and the search
    directions are M-conjugate: P^T M P is diagonal (Eq. PD);
  * after the initial projection of Algorithm 2, P^T r_0 = 0 and the first
    direction is M-conjugate to every recycled direction; each new direction
    is M-conjugate to the newest recycled one (the reading mu = (z,q_m)/(p_m,q_m));
  * augmented PCG converges to the same c* as PCG and is PCG when nothing is
    recycled;
  * the energy-norm error bound of Sec. 6.2 with kappa from dense eigenvalues.
"""
import numpy as np
import pytest

from oracle import Oracle
from synth import FrozenFlowSensors, configs


@pytest.fixture(scope="module")
def micro():
    geom = configs.micro()
    sim = FrozenFlowSensors(geom, seed=3)
    s, w = sim.sequence(6, seed=4)
    o = Oracle(geom, w, with_precond=True)
    M = o.dense_M()
    return geom, o, M, s.numpy()


@pytest.fixture(scope="module")
def micro20():
    """The micro system with alpha = 20 (kappa ~ 1e3): finite termination and
    convergence to c* are exact-arithmetic properties that FP64 rounding hides
    at the paper's alpha = 2 (kappa ~ 2e4 on this grid)."""
    geom = configs.micro()
    geom.alpha = 20.0
    sim = FrozenFlowSensors(geom, seed=3)
    s, w = sim.sequence(6, seed=4)
    o = Oracle(geom, w, with_precond=True)
    M = o.dense_M()
    return geom, o, M, s.numpy()


def _exact(o, M, s):
    return np.linalg.solve(M, o.rhs(s))


def _mnorm(M, e):
    return np.sqrt(e @ M @ e)


def test_pcg_exact_in_n_steps(micro20):
    geom, o, M, s = micro20
    cstar = _exact(o, M, s[0])
    st = o.new_state(4)
    res = o.solve(s[0], st, max_iter=o.n, augmented=False, rtol=1e-13)
    assert res["status"] == 0 and res["iterations"] <= o.n
    assert np.linalg.norm(st["c"] - cstar) <= 1e-10 * np.linalg.norm(cstar)


def test_pcg_orthogonality_and_conjugacy(micro):
    geom, o, M, s = micro
    st = o.new_state(4)
    K = 8
    res = o.solve(s[0], st, max_iter=K, augmented=False, history=True)
    H = res["history"]
    R, Z, P = H["r"][:K], H["z"][:K], H["p"][:K]
    RZ = R @ Z.T
    off = RZ - np.diag(np.diag(RZ))
    assert np.max(np.abs(off)) < 1e-10 * np.max(np.abs(np.diag(RZ)))
    D = P @ M @ P.T
    off = D - np.diag(np.diag(D))
    assert np.max(np.abs(off)) < 1e-9 * np.max(np.abs(np.diag(D)))
    # q_k = M p_k
    assert np.allclose(H["q"][:K], P @ M.T, rtol=0, atol=1e-11 * np.max(np.abs(H["q"][:K])))
    # the p_0 = z_0 reading: the first direction is the preconditioned residual
    assert np.allclose(P[0], o.invJ() * R[0])


def test_pcg_error_bound(micro):
    geom, o, M, s = micro
    cstar = _exact(o, M, s[0])
    invJ = o.invJ()
    Js = np.sqrt(invJ)
    ev = np.linalg.eigvalsh((Js[:, None] * M) * Js[None, :])
    kappa = ev[-1] / ev[0]
    rate = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    e0 = _mnorm(M, cstar)
    for k in (1, 3, 6, 12):
        st = o.new_state(4)
        o.solve(s[0], st, max_iter=k, augmented=False)
        assert _mnorm(M, st["c"] - cstar) <= 2 * e0 * rate ** k * (1 + 1e-9)


def _run(o, frames, kcap, max_iter, augmented, **kw):
    st = o.new_state(kcap)
    out = []
    for f in frames:
        out.append(o.solve(f, st, max_iter=max_iter, augmented=augmented, **kw))
    return st, out


def test_augmented_equals_pcg_without_basis(micro):
    geom, o, M, s = micro
    st_a = o.new_state(8)
    st_p = o.new_state(8)
    o.solve(s[0], st_a, max_iter=5, augmented=True)
    o.solve(s[0], st_p, max_iter=5, augmented=False)
    assert np.array_equal(st_a["c"], st_p["c"])
    assert np.array_equal(st_a["r_prev"], st_p["r_prev"])


def test_augmented_projection_conditions(micro):
    geom, o, M, s = micro
    st, _ = _run(o, s[:2], kcap=6, max_iter=6, augmented=True)
    kv = st["k_valid"]
    assert kv == 6
    P, Q, pq = st["P"][:kv].copy(), st["Q"][:kv].copy(), st["pq"][:kv].copy()
    # stored q = M p and pq = (p, q)
    assert np.allclose(Q, P @ M.T, atol=1e-10 * np.max(np.abs(Q)))
    assert np.allclose(pq, np.einsum("ij,ij->i", P, Q))
    res = o.solve(s[2], st, max_iter=6, augmented=True, history=True)
    H = res["history"]
    r0, p0 = H["r"][0], H["p"][0]
    # condition: P^T r_0 = 0 after the initial-guess projection
    assert np.max(np.abs(P @ r0)) < 1e-9 * np.linalg.norm(P, axis=1).max() * np.linalg.norm(r0)
    # condition 1: p_0 is M-conjugate to every recycled direction
    assert np.max(np.abs(Q @ p0)) < 1e-9 * np.linalg.norm(Q, axis=1).max() * np.linalg.norm(p0)
    # every new direction is M-conjugate to the newest recycled direction p_m
    qm = Q[kv - 1]
    for k in range(6):
        pk = H["p"][k]
        assert abs(qm @ pk) < 1e-8 * np.linalg.norm(qm) * np.linalg.norm(pk)


def test_augmented_reaches_pcg_solution(micro20):
    geom, o, M, s = micro20
    st, _ = _run(o, s[:2], kcap=8, max_iter=8, augmented=True)
    o.solve(s[2], st, max_iter=3 * o.n, augmented=True, rtol=1e-13)
    cstar = _exact(o, M, s[2])
    # the warm-restart residual has drifted slightly; compare the solution of
    # the system the recurrence actually solves, then the true one loosely
    assert np.linalg.norm(st["c"] - cstar) <= 1e-7 * np.linalg.norm(cstar)
    st2, _ = _run(o, s[:2], kcap=8, max_iter=8, augmented=True)
    o.solve(s[2], st2, max_iter=3 * o.n, augmented=True, rtol=1e-13, true_residual_init=True)
    assert np.linalg.norm(st2["c"] - cstar) <= 1e-10 * np.linalg.norm(cstar)


def test_paper_sequential_init_equals_gram_init(micro):
    """With an M-conjugate basis the paper's sequential sigma_j and the Gram
    form sigma = G^{-1} P^T r coincide (G is diagonal)."""
    geom, o, M, s = micro
    st_g, _ = _run(o, s[:2], kcap=5, max_iter=5, augmented=True)
    st_p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st_g.items()}
    o.solve(s[2], st_g, max_iter=4, augmented=True, init_mode=Oracle.INIT_GRAM)
    o.solve(s[2], st_p, max_iter=4, augmented=True, init_mode=Oracle.INIT_PAPER)
    assert np.linalg.norm(st_g["c"] - st_p["c"]) < 1e-9 * np.linalg.norm(st_g["c"])


def test_loop_all_projection_keeps_full_conjugacy(micro):
    geom, o, M, s = micro
    st, _ = _run(o, s[:2], kcap=6, max_iter=6, augmented=True)
    kv = st["k_valid"]
    Q = st["Q"][:kv].copy()
    res = o.solve(s[2], st, max_iter=5, augmented=True, loop_mode=Oracle.LOOP_ALL, history=True)
    for k in range(5):
        pk = res["history"]["p"][k]
        assert np.max(np.abs(Q @ pk)) < 1e-8 * np.linalg.norm(Q, axis=1).max() * np.linalg.norm(pk)


def test_warm_restart_residual_tracks_true_residual(micro):
    """Algorithm 3: r_0 = (b - b_prev) + r_prev equals b - M c_prev while the
    recurrence residual stays exact (few iterations, FP64)."""
    geom, o, M, s = micro
    st, _ = _run(o, s[:3], kcap=4, max_iter=4, augmented=True)
    true_r = st["b_prev"] - M @ st["c"]
    assert np.linalg.norm(st["r_prev"] - true_r) < 1e-9 * np.linalg.norm(st["b_prev"])


def test_rtol_stopping(micro):
    geom, o, M, s = micro
    st = o.new_state(4)
    res = o.solve(s[0], st, max_iter=200, augmented=False, rtol=1e-4)
    assert res["rel_res"] <= 1e-4
    st2 = o.new_state(4)
    res2 = o.solve(s[0], st2, max_iter=res["iterations"] - 1, augmented=False)
    assert res2["rel_res"] > 1e-4


def test_recycling_lowers_residual_on_frozen_flow():
    """The qualitative claim of Sec. 5: at equal iterations the augmented
    method reaches a lower residual than PCG on a slowly changing sequence."""
    geom = configs.tiny()
    sim = FrozenFlowSensors(geom, seed=11)
    s, w = sim.sequence(12, seed=12)
    s = s.numpy()
    o = Oracle(geom, w)
    _, plain = _run(o, s, kcap=4, max_iter=4, augmented=False)
    _, aug = _run(o, s, kcap=4, max_iter=4, augmented=True)
    rp = np.mean([r["rel_res"] for r in plain[4:]])
    ra = np.mean([r["rel_res"] for r in aug[4:]])
    assert ra < rp


# --- residual replacement (true residual every N iterations) ----------------
# In exact arithmetic the recurrence residual of CG equals b - M c, so
# replacing it changes nothing; with an inconsistent warm start (c changed
# between time steps while r_prev was not) the recurrence carries the
# inconsistency forever and the replacement removes it.  The dense M below is
# the independently pinned assembly (dense M = product of explicit matrices).

def test_true_residual_every_iteration_is_b_minus_Mc(micro20):
    geom, o, M, s = micro20
    st = o.new_state(4)
    res = o.solve(s[0], st, max_iter=6, augmented=False, true_res_every=1)
    b = o.rhs(s[0])
    assert res["status"] == 0 and res["iterations"] == 6
    assert np.linalg.norm(st["r_prev"] - (b - M @ st["c"])) <= 1e-13 * np.linalg.norm(b)


def test_true_residual_same_iterates_as_recurrence(micro20):
    """Same iterates as plain and augmented PCG up to rounding (N = 1, 2)."""
    geom, o, M, s = micro20
    for aug in (False, True):
        for N in (1, 2):
            st0, st1 = o.new_state(4), o.new_state(4)
            for t in range(3):
                r0 = o.solve(s[t], st0, max_iter=5, augmented=aug)
                r1 = o.solve(s[t], st1, max_iter=5, augmented=aug, true_res_every=N)
                assert r0["iterations"] == r1["iterations"]
                assert np.linalg.norm(st1["c"] - st0["c"]) <= 1e-10 * np.linalg.norm(st0["c"]), (aug, N, t)


def test_true_residual_beyond_max_iter_changes_nothing(micro):
    geom, o, M, s = micro
    st0, st1 = o.new_state(4), o.new_state(4)
    for t in range(2):
        o.solve(s[t], st0, max_iter=4)
        o.solve(s[t], st1, max_iter=4, true_res_every=5)
        assert np.array_equal(st0["c"], st1["c"]) and np.array_equal(st0["r_prev"], st1["r_prev"])


def test_true_residual_repairs_an_inconsistent_warm_start(micro20):
    """c is moved (1e-6 relative) between time steps without touching r_prev:
    the recurrence keeps that inconsistency in every later residual; with a
    replacement after iteration 2 or 4 of 6 the final residual is b - M c to
    rounding (the recurrence after a replacement stays consistent)."""
    geom, o, M, s = micro20
    b = o.rhs(s[1])
    gap = {}
    for N in (0, 2, 4, 7):
        rng = np.random.default_rng(9)
        st = o.new_state(4)
        o.solve(s[0], st, max_iter=30, augmented=False)
        st["c"] = st["c"] + 1e-6 * np.linalg.norm(st["c"]) / np.sqrt(o.n) * rng.standard_normal(o.n)
        o.solve(s[1], st, max_iter=6, augmented=True, true_res_every=N)
        gap[N] = np.linalg.norm(st["r_prev"] - (b - M @ st["c"])) / np.linalg.norm(b)
    assert gap[2] < 1e-13 and gap[4] < 1e-13, gap
    assert gap[0] > 1e-9 and gap[7] > 1e-9, gap
