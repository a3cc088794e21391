"""Condition-number diagnostics on the GPU operator (Sec. 6.2): Lanczos over
fewha_apply_op against the eigenvalues of the oracle's dense M on the micro
geometry (kappa_0, kappa_1, and kappa_2 with the recycled basis of a real
solve), and the paper's statement cond(H^T M H) <= cond(M) on tiny."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


def solved_state(f, s, frames, kcap):
    st = f.new_state(kcap)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    for t in range(frames):
        f.solve(s[t].cuda(), c, st, 6)
    return st


def test_micro_against_dense_eigenvalues(lib):
    from paper_2011_06842_gb300.diagnostics import condition_numbers
    geom = configs.get("micro")
    s, w = FrozenFlowSensors(geom, seed=71).sequence(3, seed=72)
    o = Oracle(geom, w)
    f = lib.Fewha(geom, w, "f64")
    st = solved_state(f, s, 3, 4)
    P, Q, _ = st.basis()
    res = condition_numbers(f, basis=(P, Q), steps=o.n)
    M = o.dense_M()
    ev0 = np.linalg.eigvalsh(M)
    sj = np.sqrt(o.invJ())
    ev1 = np.linalg.eigvalsh(sj[:, None] * M * sj[None, :])
    assert abs(res["kappa0"] / (ev0[-1] / ev0[0]) - 1) < 1e-6
    assert abs(res["kappa1"] / (ev1[-1] / ev1[0]) - 1) < 1e-6
    Pn, Qn = P.cpu().numpy(), Q.cpu().numpy()
    G = Pn @ Qn.T
    H = np.eye(o.n) - Pn.T @ np.linalg.inv(0.5 * (G + G.T)) @ Qn
    B = sj[:, None] * (H.T @ M @ H) * sj[None, :]
    ev2 = np.linalg.eigvalsh(0.5 * (B + B.T))
    nz = ev2[ev2 > 1e-11 * ev2[-1]]
    assert len(nz) == o.n - Pn.shape[0]
    assert abs(res["kappa2"] / (nz[-1] / nz[0]) - 1) < 1e-6
    f.close()


def test_deflation_does_not_raise_the_condition_number(lib):
    from paper_2011_06842_gb300.diagnostics import deflated_operator, lanczos_extremes
    geom = configs.get("tiny")
    s, w = FrozenFlowSensors(geom, seed=73).sequence(3, seed=74)
    f = lib.Fewha(geom, w, "f64")
    st = solved_state(f, s, 3, 8)
    P, Q, _ = st.basis()
    v0 = torch.randn(f.n, dtype=torch.float64, device="cuda")
    lo0, hi0, _ = lanczos_extremes(f.apply_op, v0, f.n)
    op, start = deflated_operator(f.apply_op, P, Q, torch.ones(f.n, dtype=torch.float64, device="cuda"))
    lo, hi, _ = lanczos_extremes(op, start(v0), f.n, null_tol=1e-11)
    print("tiny: cond(M) %.3e, cond(H^T M H) %.3e (k = %d)" % (hi0 / lo0, hi / lo, P.shape[0]))
    assert hi / lo <= (hi0 / lo0) * (1 + 1e-6)
    f.close()
