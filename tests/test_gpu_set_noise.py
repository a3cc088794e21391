"""fewha_set_noise: new noise weights C_eta^{-1} (Sec. 3, Eq. M) on an
existing handle.  After the call the operator, the right-hand side and a
time step equal the oracle built with the new weights (FP64 1e-10, FP32
1e-5); the modified Jacobi preconditioner (Sec. 4) equals the new oracle's
when refreshed and the old one's otherwise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402

TOL = {"f64": 1e-10, "f32": 1e-5}
DT = {"f64": torch.float64, "f32": torch.float32}


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


@pytest.mark.parametrize("refresh", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", ["mixed", "elt"])
def test_set_noise_matches_new_oracle(lib, name, prec, refresh):
    geom = configs.get(name)
    s, w1 = FrozenFlowSensors(geom, seed=44).sequence(3, seed=45)
    s = s.numpy()
    w2 = np.asarray(w1) * np.linspace(0.3, 3.0, len(w1))  # every sensor's noise level changes
    o1, o2 = Oracle(geom, w1), Oracle(geom, w2)
    f = lib.Fewha(geom, w1, prec)
    f.set_noise(w2, refresh_precond=refresh)
    # J^{-1} is computed in FP64 and stored in the working precision
    assert rel(f.precond(), (o2 if refresh else o1).invJ()) < (1e-11 if prec == "f64" else 2.0 ** -24)
    if not refresh:
        o2.set_invJ(o1.invJ())  # the same (kept) preconditioner on both sides
    x = random_vector(o2.n, 3)
    assert rel(f.apply_op(torch.tensor(x, dtype=DT[prec], device="cuda")).cpu().numpy(), o2.apply_op(x)) < TOL[prec]
    assert rel(f.rhs(torch.tensor(s[0], dtype=DT[prec], device="cuda")).cpu().numpy(), o2.rhs(s[0])) < TOL[prec]
    st_o, st_g = o2.new_state(4), f.new_state(4)
    c = torch.zeros(o2.n, dtype=DT[prec], device="cuda")
    for t in range(3):
        o2.solve(s[t], st_o, max_iter=4)
        rg = f.read_stats(f.solve(torch.tensor(s[t], dtype=DT[prec], device="cuda"), c, st_g, 4))
        assert rg["status"] == 0
        assert rel(c.cpu().numpy(), st_o["c"]) < TOL[prec]
    f.close()


def test_set_noise_rejects_bad_weights(lib):
    geom = configs.get("tiny")
    f = lib.Fewha(geom, np.ones(len(geom.gs)), "f64")
    for bad in ([1.0, -1.0, 1.0, 1.0], [1.0, np.nan, 1.0, 1.0], [np.inf, 1.0, 1.0, 1.0]):
        with pytest.raises(lib.FewhaError) as e:
            f.set_noise(bad)
        assert e.value.status == -1
    f.close()
