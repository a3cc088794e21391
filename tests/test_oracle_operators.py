"""Pins for the oracle's operators (Sec. 2 and 3, Eq. M).

Independent facts used:
  * Gamma of a planar wavefront a*x + b*y is the constant (a*ds, b*ds) on every
    subaperture; of a constant it is zero (Sec. 2 slope definition);
  * bilinear interpolation reproduces a + b u + c v + e u v exactly, so the
    propagated wavefront of such layers is the closed form evaluated at
    (1 - h/H) x + theta h (Sec. 2, P^NGS and P^LGS);
  * adjoint identities <Ax, y> = <x, A^T y> for P_g, Gamma, A and M;
  * M is symmetric positive definite (Sec. 3); its dense assembly equals the
    product of explicitly built matrices W^{-T} A^T C A W^{-1} + alpha D.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from oracle import oracle as orc
from synth import configs, pupil_mask

RNG = np.random.default_rng(1234)


def _oracle(geom, w=None, precond=False):
    w = np.linspace(0.5, 2.0, len(geom.gs)) if w is None else w
    return Oracle(geom, w, with_precond=precond)


def test_gamma_planar_and_constant():
    ns, ds = 6, 0.7
    a, b, c0 = 0.37, -1.25, 4.0
    x = np.arange(ns + 1) * ds
    phi = a * x[None, :] + b * x[:, None] + c0  # phi[i, j] = a x_j + b y_i
    s = orc.gamma_fwd(phi)
    assert np.allclose(s[:ns * ns], a * ds, atol=1e-13)
    assert np.allclose(s[ns * ns:], b * ds, atol=1e-13)
    assert np.max(np.abs(orc.gamma_fwd(np.full((ns + 1, ns + 1), 3.0)))) == 0.0


def test_gamma_adjoint():
    ns = 7
    wf = RNG.standard_normal((ns + 1, ns + 1))
    s = RNG.standard_normal(2 * ns * ns)
    lhs = orc.gamma_fwd(wf) @ s
    rhs = wf.ravel() @ orc.gamma_adj(s, ns).ravel()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("name", ["micro", "tiny", "mixed"])
def test_layer_grid_reading(name):
    """Layer spacing is the tightest one keeping every projected pupil node one
    cell inside the grid: max |projected coordinate| / d_l = n_l/2 - 2."""
    geom = configs.get(name)
    o = _oracle(geom)
    for l, lay in enumerate(geom.layers):
        d = o.layer_spacing(l)
        R = 0.0
        for g in geom.gs:
            s = (1 - lay.h / g.H) if g.H > 0 else 1.0
            for xs in (-geom.D / 2, geom.D / 2):
                R = max(R, abs(s * xs + g.theta_x * lay.h), abs(s * xs + g.theta_y * lay.h))
        assert abs(R / d - (lay.n / 2 - 2)) < 1e-9


@pytest.mark.parametrize("name", ["micro", "tiny", "mixed", "sizes"])
def test_propagation_reproduces_bilinear_functions(name):
    geom = configs.get(name)
    o = _oracle(geom)
    coeffs = RNG.standard_normal((len(geom.layers), 4))
    nodal = np.zeros(o.n)
    for l, lay in enumerate(geom.layers):
        d = o.layer_spacing(l)
        u = (np.arange(lay.n) - lay.n / 2) * d
        ux, uy = u[None, :], u[:, None]
        a, b, c, e = coeffs[l]
        nodal[o.layer_off[l]:o.layer_off[l + 1]] = (a + b * ux + c * uy + e * ux * uy).ravel()
    for gi, g in enumerate(geom.gs):
        ns = geom.sensor_ns(gi)
        m = ns + 1
        x = -geom.D / 2 + np.arange(m) * geom.D / ns
        X, Y = x[None, :], x[:, None]
        expect = np.zeros((m, m))
        for l, lay in enumerate(geom.layers):
            s = (1 - lay.h / g.H) if g.H > 0 else 1.0
            px, py = s * X + g.theta_x * lay.h, s * Y + g.theta_y * lay.h
            a, b, c, e = coeffs[l]
            expect += a + b * px + c * py + e * px * py
        got = o.prop_fwd(gi, nodal).reshape(m, m)
        assert np.max(np.abs(got - expect)) < 1e-11 * max(1.0, np.max(np.abs(expect)))


@pytest.mark.parametrize("name", ["micro", "mixed", "sizes"])
def test_propagation_adjoint(name):
    geom = configs.get(name)
    o = _oracle(geom)
    for g in range(len(geom.gs)):
        m = geom.sensor_ns(g) + 1
        x = RNG.standard_normal(o.n)
        y = RNG.standard_normal(m * m)
        lhs = o.prop_fwd(g, x) @ y
        rhs = x @ o.prop_adj(g, y)
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("name", ["micro", "tiny", "mixed", "sizes"])
def test_tomography_adjoint_and_M_symmetric(name):
    geom = configs.get(name)
    o = _oracle(geom)
    x, y = RNG.standard_normal(o.n), RNG.standard_normal(o.n)
    s = RNG.standard_normal(o.n_slopes)
    lhs, rhs = o.apply_A(x) @ s, x @ o.apply_AT(s)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs, rhs = o.apply_op(x) @ y, x @ o.apply_op(y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert o.apply_op(x) @ x > 0


@pytest.mark.parametrize("name", ["mixed", "sizes"])
def test_noise_weight_mask(name):
    geom = configs.get(name)
    w = np.arange(1.0, len(geom.gs) + 1.0)
    o = _oracle(geom, w)
    s = np.ones(o.n_slopes)
    cs = o.apply_Cinv(s)
    off = 0
    for g in range(len(geom.gs)):
        ns = geom.sensor_ns(g)
        mask = pupil_mask(geom, ns)
        assert np.array_equal(o.mask(g), mask)
        if ns > 2:
            assert mask.sum() < mask.size  # the obstruction removes subapertures
        if ns == 1:
            assert mask.all()  # a 1x1 sensor sees the whole pupil
        assert o.slope_off[g] == off
        for a in range(2):
            blk = cs[off + a * ns * ns: off + (a + 1) * ns * ns]
            assert np.all(blk[mask] == w[g]) and np.all(blk[~mask] == 0.0)
        off += 2 * ns * ns
    assert off == o.n_slopes == geom.n_slopes


def test_planar_ground_layer_gives_constant_slopes_on_every_sensor_size():
    """A plane a x + b y on the ground layer (no cone, no shift at h = 0)
    seen by sensors of 16, 12, 2 and 1 subapertures across: every subaperture
    of sensor g measures s^x = a D/n_g, s^y = b D/n_g (Sec. 2, Gamma)."""
    geom = configs.get("sizes")
    o = _oracle(geom)
    a, b = 0.37, -1.21
    nodal = np.zeros(o.n)
    lay = geom.layers[0]
    d = o.layer_spacing(0)
    u = (np.arange(lay.n) - lay.n / 2) * d
    nodal[:lay.n * lay.n] = (a * u[None, :] + b * u[:, None]).ravel()
    s = o.apply_A(nodal)
    for g in range(len(geom.gs)):
        ns = geom.sensor_ns(g)
        ds = geom.D / ns
        blk = s[o.slope_off[g]:o.slope_off[g + 1]]
        assert np.allclose(blk[:ns * ns], a * ds, rtol=0, atol=1e-12 * abs(a * ds))
        assert np.allclose(blk[ns * ns:], b * ds, rtol=0, atol=1e-12 * abs(b * ds))


def _explicit_matrices(o, geom, w):
    """W^{-1}, A and C built as explicit matrices from their definitions, by
    means other than the oracle's operator code (hat functions for the
    interpolation, the slope stencil written per entry)."""
    from oracle import daubechies_taps
    h = daubechies_taps(geom.wavelet_N)
    n = o.n
    Winv = np.zeros((n, n))
    for l, lay in enumerate(geom.layers):
        nn = lay.n * lay.n
        E = np.eye(nn)
        blk = np.stack([orc.dwt2_inv(E[i].reshape(lay.n, lay.n), lay.J, h).ravel()
                        for i in range(nn)], axis=1)
        a, b = o.layer_off[l], o.layer_off[l + 1]
        Winv[a:b, a:b] = blk / lay.delta
    def gamma(ns):
        m = ns + 1
        G = np.zeros((2 * ns * ns, m * m))
        for i in range(ns):
            for j in range(ns):
                r = i * ns + j
                G[r, i * m + j + 1] += 0.5
                G[r, i * m + j] -= 0.5
                G[r, (i + 1) * m + j + 1] += 0.5
                G[r, (i + 1) * m + j] -= 0.5
                G[ns * ns + r, (i + 1) * m + j] += 0.5
                G[ns * ns + r, i * m + j] -= 0.5
                G[ns * ns + r, (i + 1) * m + j + 1] += 0.5
                G[ns * ns + r, i * m + j + 1] -= 0.5
        return G
    hat = lambda t: np.maximum(0.0, 1.0 - np.abs(t))  # noqa: E731
    blocks = []
    for gi, g in enumerate(geom.gs):
        ns = geom.sensor_ns(gi)
        m = ns + 1
        x = -geom.D / 2 + np.arange(m) * geom.D / ns
        G = gamma(ns)
        P = np.zeros((m * m, n))
        for l, lay in enumerate(geom.layers):
            d = o.layer_spacing(l)
            s = (1 - lay.h / g.H) if g.H > 0 else 1.0
            fx = (s * x + g.theta_x * lay.h) / d + lay.n / 2  # fractional node index
            fy = (s * x + g.theta_y * lay.h) / d + lay.n / 2
            k = np.arange(lay.n)
            Wx = hat(fx[:, None] - k[None, :])  # (m, n_l)
            Wy = hat(fy[:, None] - k[None, :])
            P[:, o.layer_off[l]:o.layer_off[l + 1]] = np.kron(Wy, Wx)
        blocks.append(G @ P)
    A = np.concatenate(blocks, axis=0)
    masks = [pupil_mask(geom, geom.sensor_ns(g)) for g in range(len(geom.gs))]
    cdiag = np.concatenate([np.concatenate([w[g] * masks[g], w[g] * masks[g]]) for g in range(len(geom.gs))])
    return Winv, A, cdiag


@pytest.mark.parametrize("name", ["micro", "tiny", "sizes"])
def test_dense_M_matches_explicit_product_and_is_spd(name):
    geom = configs.get(name)
    w = np.linspace(0.7, 1.9, len(geom.gs))
    o = _oracle(geom, w)
    M = o.dense_M()
    Winv, A, cdiag = _explicit_matrices(o, geom, w)
    Mx = Winv.T @ A.T @ (cdiag[:, None] * A) @ Winv + geom.alpha * np.diag(o.prior())
    scale = np.max(np.abs(Mx))
    assert np.max(np.abs(M - Mx)) < 1e-11 * scale
    assert np.max(np.abs(M - M.T)) < 1e-12 * scale
    np.linalg.cholesky(M)  # SPD: raises if not
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev[0] > 0
    # right-hand side b = W^{-T} A^T C s
    s = RNG.standard_normal(o.n_slopes)
    assert np.allclose(o.rhs(s), Winv.T @ A.T @ (cdiag * s), rtol=0, atol=1e-11 * np.max(np.abs(Mx)))


def test_prior_levels():
    """D depends only on (layer, level), grows by 2^{11/3} per finer level and
    scales with cn2_l * (d_l / r0)^{5/3}, the Kolmogorov spectrum reading."""
    geom = configs.tiny()
    o = _oracle(geom)
    d = o.prior()
    ratio = 2.0 ** (11.0 / 3.0)
    per_layer = []
    for l, lay in enumerate(geom.layers):
        blk = d[o.layer_off[l]:o.layer_off[l + 1]].reshape(lay.n, lay.n)
        vals = {}
        for r in range(lay.n):
            for q in range(lay.n):
                s, _ = orc.band_of(lay.n, lay.J, r, q)
                vals.setdefault(s, []).append(blk[r, q])
        for v in vals.values():
            assert max(v) - min(v) <= 1e-14 * max(v)
        lev = [vals[s][0] for s in range(lay.J + 1)]
        for s in range(lay.J):
            assert abs(lev[s + 1] / lev[s] - ratio) < 1e-9
        per_layer.append(lev[0])
        # kappa_l * 2^{(11/3) J} * 0.5 * 6.88 * (d_l / r0_l)^{5/3} == 1
        r0l = geom.r0 * lay.cn2 ** (-0.6)
        assert abs(lev[0] * 2 ** (11 / 3 * lay.J) * 0.5 * 6.88 * (o.layer_spacing(l) / r0l) ** (5 / 3) - 1) < 1e-12


def test_preconditioner_is_band_mean_of_exact_diagonal():
    geom = configs.micro()
    w = np.array([1.3, 0.6])
    o = _oracle(geom, w, precond=True)
    M = o.dense_M()
    data_diag = np.diag(M) - geom.alpha * o.prior()
    invJ = o.invJ()
    for l, lay in enumerate(geom.layers):
        n = lay.n
        for s in range(lay.J + 1):
            nb = (n >> lay.J) << max(s - 1, 0)
            for quad in ([0] if s == 0 else [1, 2, 3]):
                r0 = nb if quad in (2, 3) else 0
                q0 = nb if quad in (1, 3) else 0
                offs = sorted({nb // 4, (3 * nb) // 4})
                idx = [o.layer_off[l] + (r0 + a) * n + (q0 + b) for a in offs for b in offs]
                t = np.mean(data_diag[idx])
                band = [o.layer_off[l] + r * n + q for r in range(n) for q in range(n)
                        if orc.band_of(n, lay.J, r, q) == (s, quad)]
                Jexp = geom.alpha * o.prior()[band] + t
                assert np.allclose(1.0 / invJ[band], Jexp, rtol=1e-12)
    # the sampled entries are the exact diagonal of M minus the prior
    for i in (0, 5, 77):
        assert abs(o.data_diag(i) - data_diag[i]) < 1e-10 * np.max(np.abs(data_diag))


def test_cone_effect_changes_footprint():
    """An LGS at height H sees a layer at h through a pupil compressed by
    1 - h/H: a layer function linear in u gives slopes scaled by that factor."""
    base = configs.micro()
    base.gs = [configs.GuideStar(0.0, 0.0, 0.0), configs.GuideStar(0.0, 0.0, 20000.0)]
    base.layers = [configs.Layer(5000.0, 1.0, 16, 2)]
    o = _oracle(base)
    d = o.layer_spacing(0)
    u = (np.arange(16) - 8) * d
    nodal = np.tile(0.8 * u, (16, 1)).ravel()  # phi(u) = 0.8 u_x
    s = o.apply_A(nodal)
    ns2 = base.n_sub ** 2
    ds = base.D / base.n_sub
    assert np.allclose(s[:ns2], 0.8 * ds, atol=1e-12)
    assert np.allclose(s[2 * ns2:3 * ns2], 0.8 * ds * (1 - 5000.0 / 20000.0), atol=1e-12)
    assert math.isclose(np.max(np.abs(s[ns2:2 * ns2])), 0.0, abs_tol=1e-12)
