"""MCAO fitting on the GPU (fewha_mcao_fit) against the FP64 oracle
(oracle/mcao.py): the same mirror shapes after 0, 1 and 4 CG iterations from a
random start, on the tiny, mixed and ELT geometries (ELT with the paper's
three mirrors).  Tolerances (relative L2): FP64 1e-10, FP32 1e-5, BF16
storage 2e-2 (the layers are read in bfloat16)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from oracle.mcao import McaoFit as OracleMcao, fitting_directions, paper_mirrors  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


def mirrors_for(geom):
    if geom.D > 30:
        return paper_mirrors()
    return [(geom.n_sub + 3, geom.D / geom.n_sub, 0.0), (int(geom.D) + 5, 1.0, 4000.0),
            (int(geom.D) + 9, 1.0, 12700.0)]


@pytest.mark.parametrize("name", ["tiny", "mixed", "elt"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16s", 2e-2)])
def test_mcao_fit_matches_oracle(lib, name, prec, tol):
    geom = configs.get(name)
    _, w = FrozenFlowSensors(geom, seed=71).sequence(1, seed=72)
    o = Oracle(geom, w, with_precond=False)
    dms, dirs = mirrors_for(geom), fitting_directions(0.25, 6)
    of = OracleMcao(o, geom, dms, dirs)
    f = lib.Fewha(geom, w, prec)
    g = lib.McaoFit(f, dms, dirs)
    assert g.n_actuators == of.n_actuators
    c = random_vector(o.n, 73)
    a0 = 0.1 * random_vector(of.n_actuators, 74)
    cd = torch.tensor(c, dtype=f.dtype, device="cuda")
    for iters in (0, 1, 4):
        a = torch.tensor(a0, dtype=f.dtype, device="cuda")
        g.fit(cd, a, iters)
        got = a.double().cpu().numpy()
        if iters == 0:
            assert np.array_equal(got, torch.tensor(a0, dtype=f.dtype).double().numpy())
        else:
            assert rel(got, of.fit(c, a0, iters)) < tol, (iters, rel(got, of.fit(c, a0, iters)))
    g.close()
    f.close()


def test_mcao_rejects_a_mirror_that_does_not_cover_the_pupil(lib):
    geom = configs.get("tiny")
    _, w = FrozenFlowSensors(geom, seed=75).sequence(1, seed=76)
    f = lib.Fewha(geom, w, "f64")
    with pytest.raises(lib.FewhaError):
        lib.McaoFit(f, [(5, 0.5, 0.0)], fitting_directions(0.25, 6))
    f.close()
