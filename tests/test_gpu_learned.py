"""Learned warm start on the GPU against the FP64 oracle (oracle/learned.py):
the convolution kernels and their gradients, loss, Adam, whitening and
targets, the multi-vector operator, the deflated warm start, the whole
network's gradients, and a small training run that reports what the trained
network gains over the plain warm start.

Tolerances: FP32 kernels against FP64 with relative L2 error 1e-5 (sums of at
most a few thousand FP32 products per output, accumulated in FP32 within a
tile and in FP64 across tiles); the Galerkin weights of the deflated warm
start 1e-4 (they solve a small system whose condition number multiplies the
FP32 rounding of its entries)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle  # noqa: E402
from oracle import learned as OL  # noqa: E402
from synth import FrozenFlowSensors, configs, random_vector  # noqa: E402


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_06842_gb300 import build
    build.build()
    import paper_2011_06842_gb300 as P
    from paper_2011_06842_gb300 import fewha
    return P, fewha.load_library()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def ptr(t, off=0):
    return C.c_void_p(t.data_ptr() + 4 * off)


def S():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("B,Cin,Cout,H,W", [(3, 5, 11, 37, 45), (1, 4, 32, 64, 64), (2, 32, 5, 33, 16)])
def test_conv_forward_and_gradients(lib, B, Cin, Cout, H, W):
    _, L = lib
    rng = np.random.default_rng(B * 100 + Cin)
    x, w, b = rng.standard_normal((B, Cin, H, W)), rng.standard_normal((Cout, Cin, 3, 3)), rng.standard_normal(Cout)
    g = rng.standard_normal((B, Cout, H, W))
    xd, wd, bd, gd = dev(x), dev(w), dev(b), dev(g)
    hw = H * W
    for relu in (0, 1):
        out = torch.empty((B, Cout, H, W), device="cuda")
        assert L.fewha_conv3x3_fwd(ptr(xd), Cin * hw, hw, Cin, ptr(wd), ptr(bd), ptr(out), Cout * hw, hw, Cout,
                                   B, H, W, relu, S()) == 0
        assert rel(out.cpu().numpy(), OL.conv3x3(x, w, b, relu=bool(relu))) < 1e-5
    gin = torch.empty((B, Cin, H, W), device="cuda")
    assert L.fewha_conv3x3_bwd_data(ptr(gd), Cout * hw, hw, Cout, ptr(wd), ptr(gin), Cin * hw, hw, Cin,
                                    B, H, W, S()) == 0
    assert rel(gin.cpu().numpy(), OL.conv3x3_bwd_data(g, w)) < 1e-5
    ws = torch.empty(L.fewha_conv3x3_wgrad_workspace(Cin, Cout, B, H, W), device="cuda")
    gw, gb = torch.full((Cout, Cin, 3, 3), 7.0, device="cuda"), torch.full((Cout,), 7.0, device="cuda")
    assert L.fewha_conv3x3_bwd_weight(ptr(xd), Cin * hw, hw, Cin, ptr(gd), Cout * hw, hw, Cout, B, H, W,
                                      ptr(gw), ptr(gb), 0, ptr(ws), S()) == 0
    rw, rb = OL.conv3x3_bwd_weight(x, g)
    assert rel(gw.cpu().numpy(), rw) < 1e-5 and rel(gb.cpu().numpy(), rb) < 1e-5
    # accumulate: adds to what is stored
    assert L.fewha_conv3x3_bwd_weight(ptr(xd), Cin * hw, hw, Cin, ptr(gd), Cout * hw, hw, Cout, B, H, W,
                                      ptr(gw), ptr(gb), 1, ptr(ws), S()) == 0
    assert rel(gw.cpu().numpy(), 2 * rw) < 1e-5 and rel(gb.cpu().numpy(), 2 * rb) < 1e-5


def test_conv_strided_channels(lib):
    """Channels as whole vectors (stride n, and -n over a ring, newest first)."""
    _, L = lib
    rng = np.random.default_rng(3)
    H = W = 24
    Bt, Cin, Cout, n = 2, 4, 6, 2 * 24 * 24 + 64
    ring = rng.standard_normal((8, n))
    w, b = rng.standard_normal((Cout, Cin, 3, 3)), rng.standard_normal(Cout)
    rd, wd, bd = dev(ring), dev(w), dev(b)
    base = 6  # channel k at ring[6 - k]
    x = np.stack([np.stack([ring[base - k, i * H * W:(i + 1) * H * W].reshape(H, W) for k in range(Cin)])
                  for i in range(Bt)])
    out = torch.zeros((Cout, n), device="cuda")
    assert L.fewha_conv3x3_fwd(ptr(rd, base * n), H * W, -n, Cin, ptr(wd), ptr(bd), ptr(out), H * W, n, Cout,
                               Bt, H, W, 1, S()) == 0
    ref = OL.conv3x3(x, w, b, relu=True)
    got = np.stack([np.stack([out[co, i * H * W:(i + 1) * H * W].cpu().numpy().reshape(H, W)
                              for co in range(Cout)]) for i in range(Bt)])
    assert rel(got, ref) < 1e-5
    assert np.all(out[:, 2 * H * W:].cpu().numpy() == 0.0)  # nothing written past the batch


def test_elementwise_kernels(lib):
    _, L = lib
    rng = np.random.default_rng(4)
    n = 100003
    a, t, s = rng.standard_normal(n), rng.standard_normal(n), rng.uniform(0.1, 3.0, n)
    ad, td, sd = dev(a), dev(t), dev(s)
    g = torch.empty(n, device="cuda")
    part = torch.zeros(512, dtype=torch.float64, device="cuda")
    assert L.fewha_mse_grad(ptr(ad), ptr(td), ptr(g), n, C.c_void_p(part.data_ptr()), S()) == 0
    loss, gref = OL.mse(a.astype(np.float32), t.astype(np.float32))
    assert abs(part.sum().item() / n - loss) < 1e-6 * loss
    assert rel(g.cpu().numpy(), gref) < 1e-6
    act = dev(np.maximum(a, 0.0))
    g2 = td.clone()
    assert L.fewha_relu_bwd(ptr(act), ptr(g2), n, S()) == 0
    assert np.array_equal(g2.cpu().numpy(), OL.relu_bwd(np.maximum(a, 0.0).astype(np.float32),
                                                        t.astype(np.float32)).astype(np.float32))
    for mode in (0, 1, 2):
        y = td.clone()
        assert L.fewha_scale(ptr(ad), ptr(sd), ptr(y), n, mode, S()) == 0
        a32, s32 = a.astype(np.float32).astype(np.float64), s.astype(np.float32).astype(np.float64)
        ref = [a32 * np.sqrt(s32), a32 / np.sqrt(s32), t.astype(np.float32) + a32 / np.sqrt(s32)][mode]
        assert rel(y.cpu().numpy(), ref) < 1e-6
    grp = rng.integers(1, 5, n).astype(np.int8)
    gd = torch.tensor(grp, device="cuda")
    T = torch.empty((5, n), device="cuda")
    assert L.fewha_learned_targets(ptr(ad), ptr(td), ptr(sd), C.c_void_p(gd.data_ptr()), ptr(T), n, S()) == 0
    ref = OL.targets(a.astype(np.float32), t.astype(np.float32), s.astype(np.float32), grp)
    assert rel(T.cpu().numpy(), ref) < 1e-6


def test_adam_steps(lib):
    _, L = lib
    rng = np.random.default_rng(5)
    n = 5000
    p, m, v = rng.standard_normal(n), np.zeros(n), np.zeros(n)
    pd, md, vd = dev(p), dev(m), dev(v)
    for step in range(1, 4):
        g = rng.standard_normal(n)
        assert L.fewha_adam_step(ptr(pd), ptr(dev(g)), ptr(md), ptr(vd), n, 1e-2, 0.9, 0.999, 1e-8, step, S()) == 0
        p, m, v = OL.adam(p, g.astype(np.float32), m, v, step, 1e-2)
    assert rel(pd.cpu().numpy(), p) < 1e-6


def test_apply_op_multi_matches_single_and_oracle(lib):
    P, _ = lib
    geom = configs.get("mixed")
    sim = FrozenFlowSensors(geom, seed=7)
    _, w = sim.sequence(1, seed=8)
    o = Oracle(geom, w, with_precond=False)
    for prec, tol in (("f64", 1e-10), ("f32", 1e-5)):
        f = P.Fewha(geom, w, prec)
        X = np.stack([random_vector(o.n, 40 + v) for v in range(5)])
        Xd = torch.tensor(X, dtype=f.dtype, device="cuda")
        Y = f.apply_op_multi(Xd).cpu().numpy()
        for v in range(5):
            assert rel(Y[v], o.apply_op(X[v])) < tol
            single = f.apply_op(Xd[v].contiguous()).cpu().numpy()
            assert rel(Y[v], single) < (1e-14 if prec == "f64" else 1e-6)
        f.close()


def test_deflate_warm_start_matches_oracle(lib):
    P, L = lib
    geom = configs.get("tiny")
    sim = FrozenFlowSensors(geom, seed=9)
    s, w = sim.sequence(2, seed=10)
    f = P.Fewha(geom, w, "f32")
    n = f.n
    rng = np.random.default_rng(11)
    c = rng.standard_normal(n) * 0.1
    bp, rp = rng.standard_normal(n), rng.standard_normal(n) * 0.1
    D = rng.standard_normal((5, n))
    cd, bpd, rpd, Dd = dev(c), dev(bp), dev(rp), dev(D)
    b = f.rhs(s[1].to(torch.float32).cuda())
    Q = f.apply_op_multi(Dd)
    work = torch.zeros(4096, dtype=torch.float64, device="cuda")
    info = torch.zeros(16, dtype=torch.float64, device="cuda")
    r0 = torch.empty(n, device="cuda")
    assert L.fewha_deflate_warm_start(ptr(b), ptr(Dd), n, ptr(Q), n, 5, ptr(cd), ptr(bpd), ptr(rpd), n, ptr(r0),
                                      C.c_void_p(work.data_ptr()), C.c_void_p(info.data_ptr()), S()) == 0
    taken, c1, bp1, rp1, wv, n1, n0 = OL.deflate_warm_start(b.cpu().numpy(), D.astype(np.float32),
                                                            Q.cpu().numpy(), c.astype(np.float32),
                                                            bp.astype(np.float32), rp.astype(np.float32))
    inf = info.cpu().numpy()
    assert bool(inf[0]) == taken and taken
    assert int(inf[3]) == 5
    assert rel(inf[4:9], wv) < 1e-4
    assert abs(inf[2] - n0) < 1e-5 * n0 and abs(inf[1] - n1) < 1e-4 * n0
    assert rel(cd.cpu().numpy(), c1) < 1e-5
    assert rel(rpd.cpu().numpy(), rp1) < 1e-4
    assert np.array_equal(bpd.cpu().numpy(), b.cpu().numpy())
    # gate: an exact warm start (r0 = 0) is left untouched, bit for bit
    c_before, rz = cd.clone(), torch.zeros(n, device="cuda")
    assert L.fewha_deflate_warm_start(ptr(b), ptr(Dd), n, ptr(Q), n, 5, ptr(cd), ptr(b), ptr(rz), n, ptr(r0),
                                      C.c_void_p(work.data_ptr()), C.c_void_p(info.data_ptr()), S()) == 0
    assert info[0].item() == 0.0
    assert torch.equal(cd, c_before) and torch.count_nonzero(rz).item() == 0
    # invalid arguments
    assert L.fewha_deflate_warm_start(ptr(b), ptr(Dd), n, ptr(Q), n, 7, ptr(cd), ptr(bpd), ptr(rpd), n, ptr(r0),
                                      C.c_void_p(work.data_ptr()), C.c_void_p(info.data_ptr()), S()) != 0
    f.close()


def test_network_gradients_match_oracle(lib):
    """Forward, loss and every parameter gradient of the whole network on the
    mixed geometry (two layer groups: 32x32 and 16x16)."""
    P, _ = lib
    from paper_2011_06842_gb300.learned import ConvNet
    geom = configs.get("mixed")
    net = ConvNet(geom, seed=3)
    n = net.n
    rng = np.random.default_rng(12)
    x, t = rng.standard_normal((4, n)), rng.standard_normal((5, n)) * 0.1
    xd, td = dev(x), dev(t)
    y, gy = torch.empty((5, n), device="cuda"), torch.empty((5, n), device="cuda")
    net.forward(xd.data_ptr(), n, y)
    net.mse(y, td, gy)
    net.backward(xd.data_ptr(), n, gy)
    p = net.params_numpy()
    grads = {k: 0.0 for k in p}
    outs = []
    for off, cnt, nl in net.groups:
        xs = np.stack([np.stack([x[c, off + i * nl * nl: off + (i + 1) * nl * nl].reshape(nl, nl) for c in range(4)])
                       for i in range(cnt)])
        yo, hid = OL.net_forward(xs, p)
        outs.append((off, cnt, nl, xs, yo, hid))
    # loss over all five output vectors (both groups), as the kernel computes it
    Y = np.zeros((5, n))
    for off, cnt, nl, xs, yo, hid in outs:
        for i in range(cnt):
            Y[:, off + i * nl * nl: off + (i + 1) * nl * nl] = yo[i].reshape(5, -1)
    loss_ref, GY = OL.mse(Y, t)
    assert rel(y.cpu().numpy(), Y) < 1e-5
    assert abs(net.loss() - loss_ref) < 1e-5 * loss_ref
    for off, cnt, nl, xs, yo, hid in outs:
        gys = np.stack([GY[:, off + i * nl * nl: off + (i + 1) * nl * nl].reshape(5, nl, nl) for i in range(cnt)])
        g = OL.net_backward(xs, p, hid, gys)
        for k in grads:
            grads[k] = grads[k] + g[k]
    gpu = net.grad.cpu().numpy()
    for name, (o, shp) in net.offsets.items():
        got = gpu[o:o + int(np.prod(shp))].reshape(shp)
        assert rel(got, grads[name]) < 1e-4, name


def test_training_and_gain_tiny(lib):
    """Trains on 400 frames the plain method solves, then runs the plain and the
    learned loop over 60 held-out frames (tiny geometry, SNR 100, rtol 1e-3)
    and reports iterations, time and how often the deflated warm start was
    taken.  Checks: the loss falls, every solve succeeds, a taken correction
    always lowered the warm-restart residual, and the learned loop needs no
    more iterations on average than the plain one."""
    P, _ = lib
    from paper_2011_06842_gb300 import learned
    geom = configs.get("tiny")
    geom.snr = 100.0
    sim = FrozenFlowSensors(geom, seed=13, device="cuda")
    st, w = sim.sequence_chunked(400, seed=14)
    se, _ = sim.sequence_chunked(60, seed=15, first_frame=5000)
    f = P.Fewha(geom, w, "f32")
    res = learned.study(f, geom, st, se, rtol=1e-3, max_iter=1000, epochs=3, lr=2e-3, seed=0)
    res.pop("learner")
    print("learned warm start, tiny SNR 100 rtol 1e-3:", res)
    assert res["status_ok"]
    assert res["loss_last"] < res["loss_first"]
    assert res["learned"]["r0_ratio_taken"] is None or res["learned"]["r0_ratio_taken"] < 1.0
    assert res["learned"]["iterations"] <= res["plain"]["iterations"] + 0.5
    f.close()


@pytest.mark.parametrize("B,Cin,Cout,H,W", [(5, 32, 32, 128, 128), (4, 4, 32, 64, 64), (2, 32, 5, 33, 16),
                                            (1, 7, 13, 9, 21)])
def test_conv_forward_tensor_cores(lib, B, Cin, Cout, H, W):
    """fewha_conv3x3_fwd_tc (tcgen05, BF16 operands, FP32 accumulation)
    against the FP64 oracle convolution, elementwise: rounding x and w to
    bfloat16 perturbs every product by at most 2 u + u^2 (u = 2^-9) of
    |w||x|, and FP32 accumulation of K = 9 Cin products adds at most
    K u_32 of the same, so |y - y_exact| <= (2 u + u^2 + K u_32) (|w| * |x|)
    + u_32 |y| per output (before ReLU; ReLU is 1-Lipschitz).  Shapes: the
    ELT network's 32 -> 32 layer on the 128^2 batch, its 4 -> 32 input layer,
    its 32 -> 5 output layer, and a ragged tile (H W not a multiple of 128)."""
    _, L = lib
    rng = np.random.default_rng(B * 7 + Cin)
    x, w, b = rng.standard_normal((B, Cin, H, W)), rng.standard_normal((Cout, Cin, 3, 3)), rng.standard_normal(Cout)
    hw = H * W
    out = torch.full((B, Cout, H, W), np.nan, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for relu in (0, 1):
        assert L.fewha_conv3x3_fwd_tc(ptr(dev(x)), Cin * hw, hw, Cin, ptr(dev(w)), ptr(dev(b)), ptr(out), Cout * hw,
                                      hw, Cout, B, H, W, relu, ptr(status), S()) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        y = out.double().cpu().numpy()
        exact = OL.conv3x3(x, w, b, relu=bool(relu))
        pre = OL.conv3x3(x, w, b, relu=False)
        mag = OL.conv3x3(np.abs(x), np.abs(w), None, relu=False)
        u, u32 = 2.0 ** -9, 2.0 ** -24
        bound = ((2 * u + u * u + 9 * Cin * u32) * mag + u32 * (np.abs(pre) + np.abs(b)[None, :, None, None])
                 + 1e-30)
        assert np.all(np.isfinite(y))
        assert np.all(np.abs(y - exact) <= bound), np.max(np.abs(y - exact) / bound)
        assert rel(y, exact) < 1e-2  # and the bfloat16 operands are really in use:
        assert rel(y, exact) > 1e-5
