"""Mirror side of Algorithm 3 on the GPU against the FP64 oracle: fitting
a~ = F W^{-1} c, pseudo-open-loop slopes s + Gamma a, gain control, and a
closed-loop sequence of whole time steps (POL slopes -> augmented PCG ->
fitting -> control).  Tolerances: FP64 1e-10, FP32 1e-5 (relative L2), BF16
storage 1.5e-2 (the fitting reads the bfloat16 nodal layers)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


@pytest.mark.parametrize("name", ["tiny", "mixed", "elt"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5), ("bf16s", 1.5e-2)])
def test_fit_pol_control(lib, name, prec, tol):
    geom = configs.get(name)
    s, w = FrozenFlowSensors(geom, seed=41).sequence(1, seed=42)
    o = Oracle(geom, w, with_precond=False)
    f = lib.Fewha(geom, w, prec)
    assert f.n_actuators == o.n_actuators == (geom.n_sub + 1) ** 2
    c = random_vector(o.n, 43)
    a = f.fit(torch.tensor(c, dtype=f.dtype, device="cuda")).cpu().numpy()
    assert rel(a, o.fit(c)) < tol
    ap = random_vector(o.n_actuators, 44)
    sd = s[0].to(f.slope_dtype).cuda()
    sp = f.pol_slopes(sd, torch.tensor(ap, dtype=f.dtype, device="cuda")).double().cpu().numpy()
    assert rel(sp, o.pol_slopes(sd.double().cpu().numpy(), ap)) < (tol if prec != "bf16s" else 1.5e-2)
    am1, ai, af = (random_vector(o.n_actuators, 45 + i) for i in range(3))
    t = [torch.tensor(v, dtype=f.dtype, device="cuda") for v in (am1, ai, af)]
    for closed in (True, False):
        an = f.control(closed, 0.3, *t).cpu().numpy()
        assert rel(an, o.control(closed, 0.3, am1, ai, af)) < (1e-15 if prec == "f64" else 1e-6)
    f.close()


def test_pol_slopes_in_place(lib):
    geom = configs.get("tiny")
    s, w = FrozenFlowSensors(geom, seed=51).sequence(1, seed=52)
    f = lib.Fewha(geom, w, "f64")
    a = torch.tensor(random_vector(f.n_actuators, 53), dtype=torch.float64, device="cuda")
    sd = s[0].cuda().clone()
    ref = f.pol_slopes(sd, a).cpu().numpy()
    f.pol_slopes(sd, a, out=sd)
    assert np.array_equal(sd.cpu().numpy(), ref)
    f.close()


@pytest.mark.parametrize("closed", [True, False])
def test_closed_loop_sequence_f64(lib, closed):
    """Whole time steps of Algorithm 3 on the tiny geometry, 8 frames, 4
    augmented PCG iterations each: mirror shapes and layers equal the oracle's."""
    geom = configs.get("tiny")
    nf = 8
    s, w = FrozenFlowSensors(geom, seed=61).sequence(nf, seed=62)
    s64 = s.numpy()
    o = Oracle(geom, w)
    f = lib.Fewha(geom, w, "f64")
    st_o, st_g = o.new_state(8), f.new_state(8)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    na = o.n_actuators
    ao = [np.zeros(na), np.zeros(na)]
    ag = [f.new_mirror(), f.new_mirror()]
    gain = 0.4
    for t in range(nf):
        so = o.pol_slopes(s64[t], ao[0]) if closed else s64[t]
        o.solve(so, st_o, max_iter=4, augmented=True)
        ao = [ao[1], o.control(closed, gain, ao[0], ao[1], o.fit(st_o["c"]))]
        sg = f.pol_slopes(s[t].cuda(), ag[0]) if closed else s[t].cuda()
        r = f.read_stats(f.solve(sg, c, st_g, 4))
        assert r["status"] == 0
        ag = [ag[1], f.control(closed, gain, ag[0], ag[1], f.fit(c))]
        assert rel(c.cpu().numpy(), st_o["c"]) < 1e-10
        assert rel(ag[1].cpu().numpy(), ao[1]) < 1e-10
    f.close()
