"""Batched time steps: instances of different geometries in one cooperative
launch, each on its own group of CTAs, must match the FP64 oracle like
single-instance solves (1e-10 in FP64 for fixed-iteration solves, 1e-5 in
FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from synth import FrozenFlowSensors, configs  # noqa: E402


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


@pytest.mark.parametrize("prec,tol,ctas,rounds", [("f64", 1e-10, None, None), ("f32", 1e-5, None, None),
                                                 ("f64", 1e-10, [1, 3, 2, 5, 4], None),
                                                 ("f64", 1e-10, [1, 3, 2, 5, 9], [1, 1, 0, 1, 0]),
                                                 ("f32", 1e-5, None, [2, 0, 1, 2, 0]),
                                                 ("f64", 1e-10, [4, 3, 6, 1, 10], None),
                                                 ("f32", 1e-5, [4, 3, 6, 1, 10], None)])
def test_batched_matches_oracle(lib, prec, tol, ctas, rounds):
    """Each instance of a batch equals the oracle.  An instance with at least
    twice as many CTAs as layers splits the finest wavelet level off and tiles
    it over its CTAs; one with fewer runs whole-layer transforms: the
    [4, 3, 6, 1, 10] split covers both kinds in one launch (tiny and mixed
    and medium split, micro and the second tiny whole)."""
    names = ["tiny", "micro", "mixed", "tiny", "medium"]
    frames = 3
    inst = []
    for i, name in enumerate(names):
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=40 + i).sequence(frames, seed=50 + i)
        o = Oracle(geom, w)
        f = lib.Fewha(geom, w, prec)
        inst.append((o, o.new_state(4), f, f.new_state(4), torch.zeros(f.n, dtype=f.dtype, device="cuda"),
                     s.to(f.slope_dtype).cuda(), s.numpy()))
    batch = lib.FewhaBatch([x[2] for x in inst], ctas, rounds)
    if ctas is not None:
        assert batch.ctas() == ctas
    for t in range(frames):
        stats = batch.solve([x[5][t] for x in inst], [x[4] for x in inst], [x[3] for x in inst], max_iter=4)
        for (o, st_o, f, st_g, c, sd, s64), rg in zip(inst, batch.read_stats(stats)):
            ro = o.solve(s64[t], st_o, max_iter=4, augmented=True)
            assert rg["status"] == 0 and rg["iterations"] == ro["iterations"]
            assert rel(c.cpu().numpy(), st_o["c"]) < tol
    batch.close()


def test_batched_rtol_instances_finish_independently(lib):
    """Instances stop at their own residual: each one's iteration count equals
    its single-instance solve's."""
    names = ["tiny", "mixed"]
    inst = []
    for i, name in enumerate(names):
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=60 + i).sequence(2, seed=70 + i)
        f = lib.Fewha(geom, w, "f64")
        g = lib.Fewha(geom, w, "f64")
        inst.append((f, f.new_state(8), torch.zeros(f.n, dtype=torch.float64, device="cuda"),
                     g, g.new_state(8), torch.zeros(g.n, dtype=torch.float64, device="cuda"), s.cuda()))
    batch = lib.FewhaBatch([x[0] for x in inst])
    for t in range(2):
        rb = batch.read_stats(batch.solve([x[6][t] for x in inst], [x[2] for x in inst], [x[1] for x in inst],
                                          max_iter=80, rtol=2e-2))
        for (f, st, c, g, st2, c2, s), r in zip(inst, rb):
            r2 = g.read_stats(g.solve(s[t], c2, st2, 80, rtol=2e-2))
            assert r["iterations"] == r2["iterations"]
            assert rel(c.cpu().numpy(), c2.cpu().numpy()) < 1e-9
    batch.close()


def test_batched_graph_replay_matches_oracle(lib):
    """One batched time step captured once in a CUDA graph over fixed slope
    buffers (fewha_batch_bind / fewha_batch_launch) and replayed every frame
    after the new slopes are copied in: each instance equals the oracle."""
    names = ["tiny", "mixed", "medium"]
    frames = 3
    inst = []
    for i, name in enumerate(names):
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=80 + i).sequence(frames, seed=90 + i)
        o = Oracle(geom, w)
        f = lib.Fewha(geom, w, "f32")
        inst.append((o, o.new_state(8), f, f.new_state(8), torch.zeros(f.n, dtype=f.dtype, device="cuda"),
                     s.to(torch.float32).cuda(), s.numpy(), torch.zeros(f.n_slopes, dtype=torch.float32,
                                                                         device="cuda")))
    batch = lib.FewhaBatch([x[2] for x in inst])
    stats = batch.bind([x[7] for x in inst], [x[4] for x in inst], [x[3] for x in inst], max_iter=4)
    graph = batch.capture_graph()
    torch.cuda.synchronize()
    for x in inst:  # capture does not run the kernels: nothing may have changed
        assert torch.count_nonzero(x[4]).item() == 0
    for t in range(frames):
        for x in inst:
            x[7].copy_(x[5][t])
        graph.replay()
        for (o, st_o, f, st_g, c, sd, s64, buf), rg in zip(inst, batch.read_stats(stats)):
            ro = o.solve(s64[t], st_o, max_iter=4, augmented=True)
            assert rg["status"] == 0 and rg["iterations"] == ro["iterations"]
            assert rel(c.cpu().numpy(), st_o["c"]) < 1e-5
    batch.close()


def test_pt_bands_replan_keeps_the_operator(lib):
    """fewha_set_pt_bands re-plans the P^T gather's work items: the operator
    (ELT geometry, FP64) equals the oracle for every band height tried, and a
    band that does not fit is refused with the earlier plan kept."""
    geom = configs.get("elt")
    s, w = FrozenFlowSensors(geom, seed=71).sequence(1, seed=72)
    o = Oracle(geom, w)
    f = lib.Fewha(geom, w, "f64")
    x = np.random.default_rng(3).standard_normal(f.n)
    y0 = o.apply_op(x)
    planned = 0
    for bl in ((4, 2), (2, 2), (8, 8), (1, 16), (8, 4)):
        before = f.launch_info()
        try:
            f.set_pt_bands(*bl)
            planned += 1
            li = f.launch_info()
            assert (li["pt_rows_large"], li["pt_rows_small"]) == bl
        except lib.FewhaError as e:  # staged rows beyond the shared memory: the plan stays
            assert e.status == -2
            assert f.launch_info() == before
        y = f.apply_op(torch.tensor(x, device="cuda")).cpu().numpy()
        assert rel(y, y0) < 1e-10, bl
    assert planned >= 3
    f.close()


def test_batched_explicit_tiles_and_autotuner(lib):
    """Explicit WFS tiles per instance (fewha_batch_create_ex) and the
    autotuner's chosen launch (CTA split, rounds, tiles, band heights) give
    the oracle's time steps (FP64, 1e-10)."""
    names = ["tiny", "mixed", "micro", "tiny"]
    inst = []
    for i, name in enumerate(names):
        geom = configs.get(name)
        s, w = FrozenFlowSensors(geom, seed=110 + i).sequence(8, seed=120 + i)
        o = Oracle(geom, w)
        f = lib.Fewha(geom, w, "f64")
        inst.append([o, o.new_state(4), f, f.new_state(4), torch.zeros(f.n, dtype=torch.float64, device="cuda"),
                     s.cuda(), s.numpy()])
    fewhas = [x[2] for x in inst]
    b = lib.FewhaBatch(fewhas, [5, 7, 1, 3], None, [(8, 8), (16, 8), (4, 4), (24, 16)])
    assert b.tiles() == [(8, 8), (16, 8), (4, 4), (24, 16)]
    for t in range(2):
        stats = b.solve([x[5][t] for x in inst], [x[4] for x in inst], [x[3] for x in inst], max_iter=4)
        for x, rg in zip(inst, b.read_stats(stats)):
            x[0].solve(x[6][t], x[1], max_iter=4, augmented=True)
            assert rg["status"] == 0 and rel(x[4].cpu().numpy(), x[1]["c"]) < 1e-10
    b.close()
    frame = [2]

    def step(batch):  # the tuning steps run on scratch states
        batch.solve([x[5][frame[0]] for x in inst], [torch.zeros_like(x[4]) for x in inst],
                    [x[2].new_state(4) for x in inst], max_iter=4)

    best, timings = lib.autotune_batch(fewhas, step, reps=1)
    assert len(timings) >= 3 and best["ms"] > 0
    b = lib.FewhaBatch(fewhas, best["ctas"], best["rounds"], best["tiles"])
    for t in range(2, 4):
        stats = b.solve([x[5][t] for x in inst], [x[4] for x in inst], [x[3] for x in inst], max_iter=4)
        for x, rg in zip(inst, b.read_stats(stats)):
            x[0].solve(x[6][t], x[1], max_iter=4, augmented=True)
            assert rg["status"] == 0 and rel(x[4].cpu().numpy(), x[1]["c"]) < 1e-10
    b.close()
