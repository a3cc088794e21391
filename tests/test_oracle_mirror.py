"""Pins of the oracle's mirror side of Algorithm 3 (fitting, pseudo-open-loop
slopes, gain control) against closed forms: bilinear interpolation of planar
layers is exact, the Shack-Hartmann operator maps a planar mirror to constant
slopes, and the closed loop on a static atmosphere settles on the fitted
mirror with the open-loop measurements recovered exactly."""
import numpy as np
import pytest

from oracle import Oracle
from oracle.oracle import dwt2_fwd
from synth import FrozenFlowSensors, configs


@pytest.fixture(scope="module", params=["mixed", "tiny"])
def setup(request):
    geom = configs.get(request.param)
    _, w = FrozenFlowSensors(geom, seed=3).sequence(1, seed=4)
    return geom, Oracle(geom, w, with_precond=False)


def pupil_xy(geom):
    m = geom.n_sub + 1
    x = -geom.D / 2 + np.arange(m) * geom.D / geom.n_sub
    return x[None, :], x[:, None]  # (x_j, y_i)


def test_fit_of_planar_layers_is_exact(setup):
    geom, o = setup
    rng = np.random.default_rng(5)
    coef, expect = [], 0.0
    X, Y = pupil_xy(geom)
    for l, lay in enumerate(geom.layers):
        n, d = lay.n, o.layer_spacing(l)
        k = (np.arange(n) - n / 2) * d
        a0, bx, by = rng.standard_normal(3)
        nodal = a0 + bx * k[None, :] + by * k[:, None]          # planar layer, row = y
        coef.append((lay.delta * dwt2_fwd(nodal, lay.J, o.taps)).reshape(-1))  # W nodal
        expect = expect + a0 + bx * X + by * Y
    a = o.fit(np.concatenate(coef))
    assert np.max(np.abs(a - expect.reshape(-1))) < 1e-11 * (1 + np.max(np.abs(expect)))


def test_pol_slopes_of_a_planar_mirror(setup):
    geom, o = setup
    X, Y = pupil_xy(geom)
    beta, gamma = 0.7, -1.3
    a = (0.2 + beta * X + gamma * Y).reshape(-1)
    s = np.random.default_rng(6).standard_normal(o.n_slopes)
    d = o.pol_slopes(s, a) - s
    ns2, ds = geom.n_sub ** 2, geom.D / geom.n_sub
    for g in range(len(geom.gs)):
        blk = d[2 * ns2 * g: 2 * ns2 * (g + 1)]
        assert np.allclose(blk[:ns2], beta * ds, rtol=0, atol=1e-12)
        assert np.allclose(blk[ns2:], gamma * ds, rtol=0, atol=1e-12)


def test_control_closed_forms(setup):
    _, o = setup
    rng = np.random.default_rng(7)
    am1, ai, af = rng.standard_normal((3, 11))
    g = 0.4
    assert np.allclose(o.control(True, g, am1, ai, af), ai + g * (af - am1), rtol=0, atol=1e-15)
    assert np.allclose(o.control(False, g, am1, ai, af), (1 - g) * ai + g * af, rtol=0, atol=1e-15)
    # gain 1 in open loop returns the fitted shape; gain 0 holds the mirror
    assert np.array_equal(o.control(False, 1.0, am1, ai, af), af)
    assert np.array_equal(o.control(True, 0.0, am1, ai, af), ai)


def test_closed_loop_on_a_static_atmosphere():
    """Sensors see the atmosphere minus the mirror applied two steps earlier;
    the pseudo-open-loop slopes recover the open-loop measurements exactly,
    every time step reconstructs the same layers, and the mirror settles on
    the fitted shape (e_{i+1} = e_i - gain e_{i-1}: |z| = sqrt(gain) < 1)."""
    geom = configs.get("micro")
    _, w = FrozenFlowSensors(geom, seed=8).sequence(1, seed=9)
    o = Oracle(geom, w)
    rng = np.random.default_rng(10)
    c_atm = rng.standard_normal(o.n)
    # open-loop slopes of the atmosphere: A W^{-1} c_atm (noise-free)
    nodal = np.concatenate([dwt2_inv_layer(o, lay, l, c_atm) for l, lay in enumerate(geom.layers)])
    s_open = o.apply_A(nodal)
    na = o.n_actuators
    a = [np.zeros(na), np.zeros(na)]  # a^{(i-1)}, a^{(i)}
    st = o.new_state(4)
    gain = 0.5
    fits = []
    for it in range(40):
        ga = np.concatenate([gamma_of(o, a[0])] * len(geom.gs))
        s_cl = s_open - ga                        # what the sensors measure in closed loop
        s_pol = o.pol_slopes(s_cl, a[0])
        assert np.max(np.abs(s_pol - s_open)) < 1e-12 * (1 + np.max(np.abs(s_open)))
        o.solve(s_pol, st, max_iter=200, rtol=1e-12)
        fit = o.fit(st["c"])
        fits.append(fit)
        a = [a[1], o.control(True, gain, a[0], a[1], fit)]
    assert np.max(np.abs(fits[-1] - fits[-2])) < 1e-8 * np.max(np.abs(fits[-1]))
    assert np.max(np.abs(a[1] - fits[-1])) < 1e-4 * np.max(np.abs(fits[-1]))


def dwt2_inv_layer(o, lay, l, c):
    from oracle.oracle import dwt2_inv
    off = sum(x.n * x.n for x in o.geom.layers[:l])
    blk = c[off: off + lay.n * lay.n].reshape(lay.n, lay.n)
    return (dwt2_inv(blk, lay.J, o.taps) / lay.delta).reshape(-1)


def gamma_of(o, a):
    from oracle.oracle import gamma_fwd
    m = o.n_sub + 1
    return gamma_fwd(a.reshape(m, m)).reshape(-1)
