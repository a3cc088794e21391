"""Mixed precision (BF16 storage of the operator's intermediates, FP32
arithmetic, FP64 scalars) and FP32 against the FP64 oracle.

Bound for the BF16-storage operator: bfloat16 keeps 8 significant bits, unit
roundoff u = 2^-9 ~ 1.95e-3.  One application of M stores the nodal layers and
the adjoint wavefronts in bfloat16 and uses bfloat16-rounded interpolation
weights (a perturbed P); each is a relative perturbation <= u of a linear map, and
M composes about six of them, so ||M_bf16 x - M x|| <= 6 u ||M x|| ~ 1.2e-2 in the
worst case.  The test allows 1.5e-2.  For a time step (a few CG iterations)
the same per-application perturbation enters every iteration; the sequence
test chains 500 time steps, so each run follows its own trajectory (CG
amplifies every difference over the frames): it reports per frame the relative
L2 error of the layer coefficients, the relative error in the energy norm
||e||_M / ||c||_M (the data-fit norm the solver minimises), and the relative
error of ||r||, and guards them with regression bounds set with margin over
the values measured on a GB300 (FP32: layer L2 median 2e-4, max 5e-3;
BF16S: layer L2 median 0.11, max 0.24, dominated by weakly observed modes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402

U_BF16 = 2.0 ** -9


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


@pytest.mark.parametrize("name", ["tiny", "mixed", "elt"])
def test_bf16_operator_and_rhs(lib, name):
    geom = configs.get(name)
    sim = FrozenFlowSensors(geom, seed=21)
    s, w = sim.sequence(1, seed=22)
    o = Oracle(geom, w, with_precond=False)
    f = lib.Fewha(geom, w, "bf16s")
    x = random_vector(o.n, 4)
    y = f.apply_op(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    err = rel(y, o.apply_op(x))
    assert err < 1.5e-2, err
    assert err > 1e-5  # the intermediates really are stored in bfloat16
    b = f.rhs(s[0].to(torch.bfloat16).cuda()).cpu().numpy()
    assert rel(b, o.rhs(s[0].numpy())) < 1.5e-2


def test_mixed_precision_sequence_500_frames(lib):
    """The mixed-precision workload: tiny geometry, 500 frozen-flow frames,
    4 augmented PCG iterations per frame; BF16S and FP32 against the FP64
    oracle, relative L2 error of the layer coefficients and of ||r|| per frame."""
    geom = configs.tiny()
    nf = 500
    sim = FrozenFlowSensors(geom, seed=31)
    s, w = sim.sequence(nf, seed=32)
    s64 = s.numpy()
    o = Oracle(geom, w)
    st_o = o.new_state(8)
    runs = {}
    for prec in ("bf16s", "f32"):
        f = lib.Fewha(geom, w, prec)
        runs[prec] = (f, f.new_state(8), torch.zeros(o.n, dtype=torch.float32, device="cuda"),
                      s.to(f.slope_dtype).cuda())
    errs = {p: [] for p in runs}
    enrg = {p: [] for p in runs}
    rres = {p: [] for p in runs}
    for t in range(nf):
        ro = o.solve(s64[t], st_o, max_iter=4, augmented=True)
        cm = o.apply_op(st_o["c"]) @ st_o["c"]
        for p, (f, st, c, sd) in runs.items():
            rg = f.read_stats(f.solve(sd[t], c, st, 4))
            assert rg["status"] == 0
            cg = c.double().cpu().numpy()
            e = cg - st_o["c"]
            errs[p].append(rel(cg, st_o["c"]))
            if t % 10 == 0:
                enrg[p].append(np.sqrt(max(o.apply_op(e) @ e, 0.0) / cm))
            rres[p].append(abs(rg["rel_res"] - ro["rel_res"]) / ro["rel_res"])
    for p in runs:
        e = np.array(errs[p])
        print("%s vs FP64 oracle over %d frames: layer L2 error median %.2e max %.2e; "
              "energy-norm error median %.2e max %.2e; ||r|| relative error median %.2e max %.2e"
              % (p, nf, np.median(e), e.max(), np.median(enrg[p]), np.max(enrg[p]),
                 np.median(rres[p]), np.max(rres[p])))
    assert np.median(errs["f32"]) < 1e-3 and max(errs["f32"]) < 2e-2
    assert np.median(rres["f32"]) < 1e-3
    assert np.median(errs["bf16s"]) < 0.3 and max(errs["bf16s"]) < 0.6
    assert np.median(rres["bf16s"]) < 2e-2
