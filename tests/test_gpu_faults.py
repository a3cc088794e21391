"""Failure detection without a GPU fault: every failure is made on the host
(NaN slopes, a corrupted recycled basis, a zero time limit on the device-side
waits) and must come back as a status, with the context still usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import FrozenFlowSensors, configs  # noqa: E402


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    geom = configs.tiny()
    s, w = FrozenFlowSensors(geom, seed=5).sequence(4, seed=6)
    return P, geom, s.to("cuda"), w


def _healthy_solve(P, f, s):
    st = f.new_state(4)
    c = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    r = f.read_stats(f.solve(s[0], c, st, 4))
    assert r["status"] == 0 and r["iterations"] == 4
    return r


def test_barrier_timeout_is_reported(env):
    P, geom, s, w = env
    f = P.Fewha(geom, w, "f64")
    f.set_timeout(0)  # every grid-barrier wait gives up at once
    st = f.new_state(4)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    r = f.read_stats(f.solve(s[0], c, st, 4))
    assert r["status"] == -4  # FEWHA_ERR_TIMEOUT
    assert int(st.meta[1]) == 0  # no basis was recorded
    f.set_timeout(1_000_000_000)
    _healthy_solve(P, f, s)  # the context and the handle still work


@pytest.mark.parametrize("persistent", [True, False])
def test_nan_slopes_give_breakdown(env, persistent):
    P, geom, s, w = env
    f = P.Fewha(geom, w, "f64")
    st = f.new_state(4)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    bad = s[0].clone()
    bad[3] = float("nan")
    r = f.read_stats(f.solve(bad, c, st, 4, persistent=persistent))
    assert r["status"] == -5  # FEWHA_ERR_BREAKDOWN
    _healthy_solve(P, f, s)


def test_corrupted_basis_is_not_spd(env):
    P, geom, s, w = env
    f = P.Fewha(geom, w, "f64")
    st = f.new_state(4)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    assert f.read_stats(f.solve(s[0], c, st, 4))["status"] == 0
    bank = int(st.meta[0])
    st.Q[bank] = -st.P[bank]  # G = P^T Q is now negative definite
    r = f.read_stats(f.solve(s[1], c, st, 4))
    assert r["status"] == -6  # FEWHA_ERR_NOT_SPD
    _healthy_solve(P, f, s)


def test_device_status_codes_have_text(env):
    P = env[0]
    lib = P.load_library()
    for code in range(-8, 1):
        assert lib.fewha_strerror(code)
