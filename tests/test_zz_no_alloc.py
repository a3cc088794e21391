"""fewha_apply_op_noalloc: the operator application for callers that cannot
allocate device memory where they apply it (a real-time loop that must not
stall on the allocator, plug-ins whose host owns all device memory).  It must
give the same y = M x as fewha_apply_op, call after call, while its
intermediates live in the library's fixed static scratch, and the device's
free memory must not change across its calls; problems too large for that
scratch are refused.  Collected last on purpose (file name), so a failing run
has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import configs, random_vector  # noqa: E402

# FP64 / FP32 parity tolerances of the other GPU tests; BF16 storage: both
# entry points round the same intermediates the same way, so they agree to
# FP32 arithmetic except for the order of the partial sums of (p, Mp) (not
# part of y): the FP32 bound applies.
TOL = {"f64": 1e-10, "f32": 1e-5, "bf16s": 1e-5}


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    return P


@pytest.mark.parametrize("name,prec", [("tiny", "f64"), ("tiny", "bf16s"), ("elt", "f32"), ("elt", "f64")])
def test_noalloc_matches_apply_op_twice(lib, name, prec):
    geom = configs.get(name)
    f = lib.Fewha(geom, np.linspace(0.5, 2.0, len(geom.gs)), prec)
    dt = f.dtype
    xs = [torch.tensor(random_vector(f.n, seed), dtype=dt, device="cuda") for seed in (11, 12)]
    ys = [torch.empty(f.n, dtype=dt, device="cuda") for _ in xs]
    f.apply_op_noalloc(xs[0], out=ys[0])  # warm-up: kernels loaded, launch resources sized
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for x, y in zip(xs, ys):  # two calls in a row share the static scratch
        f.apply_op_noalloc(x, out=y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the allocation-free entry point changed free device memory"
    for x, y in zip(xs, ys):
        assert _rel(y, f.apply_op(x)) < TOL[prec], (name, prec)
    f.close()


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    """16 layers of 128^2 and 16 sensors of 100 x 100 subapertures in FP64 need
    more intermediate storage than the fixed scratch holds."""
    big = configs.Geometry("big", D=20.0, obstruction=0.0, n_sub=100,
                           gs=[configs.GuideStar(1e-5 * (i % 4), 1e-5 * (i // 4), 0.0) for i in range(16)],
                           layers=[configs.Layer(500.0 * i, 1.0 / 16, 128, 1) for i in range(16)], r0=0.15)
    f = lib.Fewha(big, np.ones(16), "f64")
    x = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.FewhaError) as e:
        f.apply_op_noalloc(x)
    assert e.value.status == -8
    f.close()
