"""Pins of the MCAO fitting oracle (oracle/mcao.py) against facts outside it:
bilinear interpolation is exact for planes (closed-form projections of planar
mirrors and layers, with the altitude shifts), the adjoint identity, scipy's
CG on the dense normal matrix, and an exactly representable atmosphere whose
fitting residual vanishes."""
import numpy as np
import pytest

from oracle import Oracle
from oracle.mcao import McaoFit, fitting_directions, interp_matrix
from synth import FrozenFlowSensors, configs

sla = pytest.importorskip("scipy.sparse.linalg")


def small_fit(name="tiny"):
    geom = configs.get(name)
    _, w = FrozenFlowSensors(geom, seed=3).sequence(1, seed=4)
    o = Oracle(geom, w, with_precond=False)
    dms = [(geom.n_sub + 3, geom.D / geom.n_sub, 0.0), (int(geom.D) + 5, 1.0, 4000.0),
           (int(geom.D) + 9, 1.0, 12700.0)]
    return geom, o, McaoFit(o, geom, dms, fitting_directions(0.25, 6))


def test_interp_matrix_rows_and_plane():
    M = interp_matrix(np.array([-1.3, 0.0, 1.75]), 0.5, 4.0, 9)
    assert np.allclose(M.sum(axis=1), 1.0)
    nodes = (np.arange(9) - 4.0) * 0.5
    assert np.allclose(M @ (3.0 * nodes - 1.0), 3.0 * np.array([-1.3, 0.0, 1.75]) - 1.0, atol=1e-14)
    with pytest.raises(ValueError):
        interp_matrix(np.array([2.1]), 0.5, 4.0, 9)


def test_planar_mirrors_project_in_closed_form():
    geom, o, f = small_fit()
    coef = [(0.3, -0.7, 0.1), (-1.1, 0.4, 2.0), (0.25, 0.9, -0.5)]
    parts = []
    for (n, pitch, h), (al, be, ga) in zip(f.dms, coef):
        xs = (np.arange(n) - 0.5 * (n - 1)) * pitch
        X, Y = np.meshgrid(xs, xs)  # row index = y
        parts.append((al * X + be * Y + ga).ravel())
    y = f.project_dms(np.concatenate(parts))
    ds = geom.D / geom.n_sub
    x = -0.5 * geom.D + ds * np.arange(f.m)
    X, Y = np.meshgrid(x, x)
    for t, (tx, ty) in enumerate(f.dirs):
        ref = sum(al * (X + h * tx) + be * (Y + h * ty) + ga for (n, p, h), (al, be, ga) in zip(f.dms, coef))
        assert np.max(np.abs(y[t] - ref)) < 1e-12


def test_planar_layers_project_in_closed_form():
    geom, o, f = small_fit("mixed")
    layers = []
    for l, ly in enumerate(geom.layers):
        xs = (np.arange(ly.n) - 0.5 * ly.n) * o.layer_spacing(l)
        X, Y = np.meshgrid(xs, xs)
        layers.append(0.2 * (l + 1) * X - 0.3 * Y + l)
    phi = f.project_layers(layers)
    x = -0.5 * geom.D + geom.D / geom.n_sub * np.arange(f.m)
    X, Y = np.meshgrid(x, x)
    for t, (tx, ty) in enumerate(f.dirs):
        ref = sum(0.2 * (l + 1) * (X + ly.h * tx) - 0.3 * (Y + ly.h * ty) + l for l, ly in enumerate(geom.layers))
        assert np.max(np.abs(phi[t] - ref)) < 1e-12


def test_adjoint_identity():
    _, _, f = small_fit()
    rng = np.random.default_rng(5)
    a = rng.standard_normal(f.n_actuators)
    y = rng.standard_normal((len(f.dirs), f.m, f.m))
    lhs = np.sum(f.project_dms(a) * y)
    assert abs(lhs - a @ f.project_dms_T(y)) < 1e-11 * abs(lhs)


def test_cg_iterations_equal_scipy_cg_on_the_dense_normal_matrix():
    geom, o, f = small_fit()
    rng = np.random.default_rng(6)
    c = rng.standard_normal(o.n)
    a0 = rng.standard_normal(f.n_actuators) * 0.1
    N = np.column_stack([f.normal(e) for e in np.eye(f.n_actuators)])
    b = f.rhs(c)
    for iters in (1, 2, 4):
        ref, _ = sla.cg(N, b, x0=a0.copy(), maxiter=iters, rtol=1e-300, atol=0.0)
        got = f.fit(c, a0, iters)
        assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(ref)
    assert np.array_equal(f.fit(c, a0, 0), a0)


def test_representable_atmosphere_is_fitted_exactly():
    """Only the ground layer is non-zero and holds a plane: the ground mirror
    represents it exactly, so the fitting residual goes to zero."""
    geom, o, f = small_fit()
    ly = geom.layers[0]
    xs = (np.arange(ly.n) - 0.5 * ly.n) * o.layer_spacing(0)
    X, Y = np.meshgrid(xs, xs)
    layers = [0.4 * X - 0.2 * Y + 0.3] + [np.zeros((l.n, l.n)) for l in geom.layers[1:]]
    # c = W nodal, layer by layer: the coefficients whose synthesis is the plane
    from oracle.oracle import dwt2_fwd
    c = np.concatenate([dwt2_fwd(L * l.delta, l.J, o.taps).ravel() for L, l in zip(layers, geom.layers)])
    phi2 = float(np.sum(f.project_layers(f.nodal(c)) ** 2))
    # the plane on the ground mirror (others flat) fits it exactly ...
    n0, p0, _ = f.dms[0]
    xa = (np.arange(n0) - 0.5 * (n0 - 1)) * p0
    Xa, Ya = np.meshgrid(xa, xa)
    exact = np.concatenate([(0.4 * Xa - 0.2 * Ya + 0.3).ravel(), np.zeros(f.n_actuators - n0 * n0)])
    assert f.residual(c, exact) < 1e-24 * phi2
    # ... and the CG iterates approach a zero residual (the normal matrix is
    # singular and ill-conditioned: slow, monotone)
    res = [f.residual(c, f.fit(c, np.zeros(f.n_actuators), k)) for k in (4, 40, 300)]
    assert res[0] > res[1] > res[2] and res[2] < 1e-5 * phi2
