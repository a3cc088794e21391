"""Asterisms whose guide stars carry Shack-Hartmann sensors of different
sizes (fewha_gs.n_sub): the paper's MCAO asterism (Sec. 5.1 system-settings
table: 6 LGS with 84x84 sensors, NGS with one 2x2 and two 1x1 sensors) at ELT
size, and a small geometry with 16x16, 12x12, 2x2 and 1x1 sensors.  GPU parity
with the FP64 oracle through the C ABI: operator and right-hand side (Eq. M),
time steps of augmented PCG (Algorithm 2 in Algorithm 3) in the persistent and
per-phase launches and in a batch, the allocation-free operator; FP64 1e-10,
FP32 1e-5, BF16 storage 1.5e-2 (the bound derived in
test_gpu_mixed_precision)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402

TOL = {"f64": 1e-10, "f32": 1e-5, "bf16s": 1.5e-2}
DT = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.float32}
SDT = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.bfloat16}


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


_cache = {}


def setup(name):
    if name not in _cache:
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=61).sequence(4, seed=62)
        _cache[name] = (geom, s.numpy(), w, Oracle(geom, w))
    return _cache[name]


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16s"])
@pytest.mark.parametrize("name", ["sizes", "mcao"])
def test_operator_rhs_noalloc(lib, name, prec):
    geom, s, w, o = setup(name)
    f = lib.Fewha(geom, w, prec)
    assert f.n_slopes == o.n_slopes == geom.n_slopes
    x = random_vector(o.n, 9)
    y0 = o.apply_op(x)
    xd = torch.tensor(x, dtype=DT[prec], device="cuda")
    assert rel(f.apply_op(xd).cpu().numpy(), y0) < TOL[prec]
    assert rel(f.apply_op_noalloc(xd).cpu().numpy(), y0) < TOL[prec]
    sl = torch.tensor(s[0], dtype=SDT[prec], device="cuda")
    assert rel(f.rhs(sl).cpu().numpy(), o.rhs(sl.double().cpu().numpy())) < TOL[prec]
    f.close()


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", ["sizes", "mcao"])
def test_augmented_sequence(lib, name, prec, persistent):
    geom, s, w, o = setup(name)
    f = lib.Fewha(geom, w, prec)
    st_o, st_g = o.new_state(8), f.new_state(8)
    c = torch.zeros(o.n, dtype=DT[prec], device="cuda")
    for t in range(3):
        ro = o.solve(s[t], st_o, max_iter=4, augmented=True)
        rg = f.read_stats(f.solve(torch.tensor(s[t], dtype=DT[prec], device="cuda"), c, st_g, 4,
                                  persistent=persistent))
        assert rg["status"] == 0 and rg["iterations"] == ro["iterations"]
        assert rel(c.cpu().numpy(), st_o["c"]) < TOL[prec], t
    f.close()


def test_batched_with_sensor_sizes(lib):
    """A batch of a mixed-size asterism (split and whole-layer forms) beside
    a uniform one equals the oracle."""
    inst = []
    for i, name in enumerate(["sizes", "tiny", "sizes"]):
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=130 + i).sequence(3, seed=140 + i)
        o = Oracle(geom, w)
        f = lib.Fewha(geom, w, "f64")
        inst.append((o, o.new_state(4), f, f.new_state(4), torch.zeros(f.n, dtype=torch.float64, device="cuda"),
                     s.cuda(), s.numpy()))
    b = lib.FewhaBatch([x[2] for x in inst], [8, 5, 2])
    for t in range(3):
        stats = b.solve([x[5][t] for x in inst], [x[4] for x in inst], [x[3] for x in inst], max_iter=4)
        for (o, st_o, f, st_g, c, sd, s64), rg in zip(inst, b.read_stats(stats)):
            o.solve(s64[t], st_o, max_iter=4, augmented=True)
            assert rg["status"] == 0 and rel(c.cpu().numpy(), st_o["c"]) < 1e-10
    b.close()


def test_pol_slopes_need_the_mirror_grid(lib):
    """Pseudo-open-loop slopes add Gamma of the ground mirror, whose actuators
    sit on the geometry's pupil grid: refused when a sensor has another size."""
    geom, s, w, o = setup("sizes")
    f = lib.Fewha(geom, w, "f64")
    with pytest.raises(lib.FewhaError) as e:
        f.pol_slopes(torch.tensor(s[0], device="cuda"), f.new_mirror())
    assert e.value.status == -2
    f.close()
