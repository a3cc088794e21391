"""Learned warm start around the reconstructor loop (not part of the paper).

A small convolutional network reads the last four time steps' layer
coefficients and predicts, for the next time step, the increment of the
solution (channel 0) and that increment's parts on four wavelet scale groups
(channels 1-4).  The five predicted directions D enter the next solve through
a deflated warm start: the Galerkin projection onto span(D), which is the
initial projection of the augmented PCG (Algorithm 2) with D in place of the
recycled basis; it needs M D (one multi-vector operator application) and is
kept only if it lowers the warm-restart residual of Algorithm 3.  PCG, with
its own recycled basis, then runs as usual, so the solver still decides when
the time step is solved.

Everything here is argument marshalling around libfewha: the network's
forward and backward passes, the loss, Adam, the whitening, the multi-vector
operator and the projection are CUDA kernels (``csrc/learned.cu``,
``fewha_apply_op_multi``).  Layer coefficients are whitened by the prior
(x sqrt(alpha D)) and by one global scale each for inputs and outputs; the
layers of one grid size form the network's batch, and a network input
channel is a whole coefficient vector (channel stride -n over a ring of past
solutions, newest first).

Network: 4 -> 32 -> 32 -> 5 channels, 3x3 kernels, ReLU after the first two.
"""
import ctypes as C
import math

import numpy as np

from .fewha import FewhaError, _stream_ptr, load_library

CHANNELS = (4, 32, 32, 5)
N_DIR = 5


def layer_groups(geom):
    """Runs of consecutive layers with the same grid size: [(offset, count, n)]."""
    groups, off, i = [], 0, 0
    layers = list(geom.layers)
    while i < len(layers):
        j = i
        while j < len(layers) and layers[j].n == layers[i].n:
            j += 1
        groups.append((off, j - i, layers[i].n))
        off += (j - i) * layers[i].n ** 2
        i = j
    return groups


def scale_groups(geom):
    """Wavelet scale group of every coefficient (int8, length n): in the Mallat
    layout of an n x n layer, coefficient (r, q) with m = max(r, q) belongs to
    group 4 if m >= n/2 (finest details), 3 if m >= n/4, 2 if m >= n/8 and 1
    otherwise (coarser details and the approximation)."""
    out = []
    for lay in geom.layers:
        n = lay.n
        r = np.arange(n)
        m = np.maximum(r[:, None], r[None, :])
        g = np.where(m >= n // 2, 4, np.where(m >= n // 4, 3, np.where(m >= n // 8, 2, 1)))
        out.append(g.reshape(-1))
    return np.concatenate(out).astype(np.int8)


class ConvNet:
    """Parameters, Adam state and activation buffers of the network on the GPU."""

    def __init__(self, geom, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.groups = layer_groups(geom)
        self.n = sum(cnt * nl * nl for _, cnt, nl in self.groups)
        c0, c1, c2, c3 = CHANNELS
        shapes = [("w1", (c1, c0, 3, 3)), ("b1", (c1,)), ("w2", (c2, c1, 3, 3)), ("b2", (c2,)),
                  ("w3", (c3, c2, 3, 3)), ("b3", (c3,))]
        sizes = [int(np.prod(s)) for _, s in shapes]
        self.nparam = sum(sizes)
        rng = np.random.default_rng(seed)
        init = np.zeros(self.nparam, dtype=np.float32)
        self.offsets = {}
        o = 0
        for (name, shp), sz in zip(shapes, sizes):
            self.offsets[name] = (o, shp)
            if name[0] == "w":
                fan_in = shp[1] * 9
                gain = 0.1 if name == "w3" else 1.0  # He initialisation, small last layer
                init[o:o + sz] = rng.standard_normal(sz) * gain * math.sqrt(2.0 / fan_in)
            o += sz
        dev = torch.device(device)
        self.param = torch.tensor(init, device=dev)
        self.grad = torch.zeros_like(self.param)
        self.m = torch.zeros_like(self.param)
        self.v = torch.zeros_like(self.param)
        self.step_count = 0
        self.h1, self.h2, self.ga, self.gb = [], [], [], []
        ws = 0
        for _, cnt, nl in self.groups:
            for buf in (self.h1, self.h2, self.ga, self.gb):
                buf.append(torch.empty((cnt, 32, nl, nl), dtype=torch.float32, device=dev))
            for ci, co in ((c0, c1), (c1, c2), (c2, c3)):
                ws = max(ws, self.lib.fewha_conv3x3_wgrad_workspace(ci, co, cnt, nl, nl))
        self.work = torch.empty(max(ws, 1), dtype=torch.float32, device=dev)
        self.loss_part = torch.zeros(512, dtype=torch.float64, device=dev)

    def _p(self, t, name):
        o, _ = self.offsets[name]
        return C.c_void_p(t.data_ptr() + 4 * o)

    def _ck(self, st, what):
        if st != 0:
            raise FewhaError(st, what)

    def forward(self, x_ptr, x_cs, y, tensor_cores=False):
        """y (5, n) = network(x), x channel k at address x_ptr + 4 * k * x_cs.
        tensor_cores: the convolutions run on the tcgen05 kernel (bfloat16
        operands, FP32 accumulation; inference), else on the FP32 kernel
        (training: its activations feed the backward pass)."""
        for name, _, launch in self.convolutions(x_ptr, x_cs, y, tensor_cores):
            self._ck(launch(), name)
        return y

    def convolutions(self, x_ptr, x_cs, y, tensor_cores=False):
        """The launches of forward(), in order: (name, FLOPs, launch) per 3x3
        convolution of each group of equal-size layers; launch() returns the
        C-ABI status."""
        lib, s = self.lib, _stream_ptr(self.torch)
        c0, c1, c2, c3 = CHANNELS
        if tensor_cores:
            if not hasattr(self, "tc_status"):
                self.tc_status = self.torch.zeros(1, dtype=self.torch.int32, device=self.param.device)
            st = C.c_void_p(self.tc_status.data_ptr())
            conv = lambda *a: lib.fewha_conv3x3_fwd_tc(*a[:-1], st, a[-1])  # noqa: E731
        else:
            conv = lib.fewha_conv3x3_fwd
        out = []
        for gi, (off, cnt, nl) in enumerate(self.groups):
            hw = nl * nl
            h1, h2 = self.h1[gi], self.h2[gi]
            stages = ((C.c_void_p(x_ptr + 4 * off), hw, x_cs, c0, "w1", "b1", C.c_void_p(h1.data_ptr()), 32 * hw,
                       hw, c1, 1),
                      (C.c_void_p(h1.data_ptr()), 32 * hw, hw, c1, "w2", "b2", C.c_void_p(h2.data_ptr()), 32 * hw,
                       hw, c2, 1),
                      (C.c_void_p(h2.data_ptr()), 32 * hw, hw, c2, "w3", "b3", C.c_void_p(y.data_ptr() + 4 * off),
                       hw, y.stride(0), c3, 0))
            for i, (xp, xbs, xcs, ci, wn, bn, yp, ybs, ycs, co, relu) in enumerate(stages):
                args = (xp, xbs, xcs, ci, self._p(self.param, wn), self._p(self.param, bn), yp, ybs, ycs, co, cnt,
                        nl, nl, relu, s)
                out.append(("conv%d %dx%dx%d %d->%d" % (i + 1, cnt, nl, nl, ci, co), 18.0 * cnt * hw * ci * co,
                            (lambda a=args: conv(*a))))
        return out

    def backward(self, x_ptr, x_cs, gy):
        """Parameter gradients (self.grad) of sum(gy * y) after forward() on the same x."""
        lib, s = self.lib, _stream_ptr(self.torch)
        c0, c1, c2, c3 = CHANNELS
        work = C.c_void_p(self.work.data_ptr())
        for gi, (off, cnt, nl) in enumerate(self.groups):
            hw = nl * nl
            acc = 1 if gi > 0 else 0
            h1, h2, ga, gb = self.h1[gi], self.h2[gi], self.ga[gi], self.gb[gi]
            gyp = C.c_void_p(gy.data_ptr() + 4 * off)
            self._ck(lib.fewha_conv3x3_bwd_weight(C.c_void_p(h2.data_ptr()), 32 * hw, hw, c2, gyp, hw, gy.stride(0),
                                                  c3, cnt, nl, nl, self._p(self.grad, "w3"),
                                                  self._p(self.grad, "b3"), acc, work, s), "wgrad3")
            self._ck(lib.fewha_conv3x3_bwd_data(gyp, hw, gy.stride(0), c3, self._p(self.param, "w3"),
                                                C.c_void_p(ga.data_ptr()), 32 * hw, hw, c2, cnt, nl, nl, s), "dgrad3")
            self._ck(lib.fewha_relu_bwd(C.c_void_p(h2.data_ptr()), C.c_void_p(ga.data_ptr()), ga.numel(), s),
                     "relu2")
            self._ck(lib.fewha_conv3x3_bwd_weight(C.c_void_p(h1.data_ptr()), 32 * hw, hw, c1,
                                                  C.c_void_p(ga.data_ptr()), 32 * hw, hw, c2, cnt, nl, nl,
                                                  self._p(self.grad, "w2"), self._p(self.grad, "b2"), acc, work, s),
                     "wgrad2")
            self._ck(lib.fewha_conv3x3_bwd_data(C.c_void_p(ga.data_ptr()), 32 * hw, hw, c2,
                                                self._p(self.param, "w2"), C.c_void_p(gb.data_ptr()), 32 * hw, hw,
                                                c1, cnt, nl, nl, s), "dgrad2")
            self._ck(lib.fewha_relu_bwd(C.c_void_p(h1.data_ptr()), C.c_void_p(gb.data_ptr()), gb.numel(), s),
                     "relu1")
            self._ck(lib.fewha_conv3x3_bwd_weight(C.c_void_p(x_ptr + 4 * off), hw, x_cs, c0,
                                                  C.c_void_p(gb.data_ptr()), 32 * hw, hw, c1, cnt, nl, nl,
                                                  self._p(self.grad, "w1"), self._p(self.grad, "b1"), acc, work, s),
                     "wgrad1")

    def mse(self, y, target, gy):
        """gy = d mean((y - target)^2) / dy; the loss stays on the device (loss())."""
        self._ck(self.lib.fewha_mse_grad(C.c_void_p(y.data_ptr()), C.c_void_p(target.data_ptr()),
                                         C.c_void_p(gy.data_ptr()), y.numel(),
                                         C.c_void_p(self.loss_part.data_ptr()), _stream_ptr(self.torch)), "mse")
        self._n_loss = y.numel()

    def loss(self):
        """Last mse() loss (synchronises)."""
        return float(self.loss_part.sum().item()) / self._n_loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        self._ck(self.lib.fewha_adam_step(C.c_void_p(self.param.data_ptr()), C.c_void_p(self.grad.data_ptr()),
                                          C.c_void_p(self.m.data_ptr()), C.c_void_p(self.v.data_ptr()),
                                          self.nparam, lr, beta1, beta2, eps, self.step_count,
                                          _stream_ptr(self.torch)), "adam")

    def params_numpy(self):
        p = self.param.cpu().numpy().astype(np.float64)
        out = {}
        for name, (o, shp) in self.offsets.items():
            out[name] = p[o:o + int(np.prod(shp))].reshape(shp)
        return out


def _scale(lib, torch, x, s, y, mode):
    st = lib.fewha_scale(C.c_void_p(x.data_ptr()), C.c_void_p(s.data_ptr()), C.c_void_p(y.data_ptr()),
                         x.numel(), mode, _stream_ptr(torch))
    if st != 0:
        raise FewhaError(st, "fewha_scale")


class LearnedWarmStart:
    """Training and online use of the network for one FP32 Fewha instance."""

    def __init__(self, fewha, geom, seed=0, tensor_cores=True):
        import torch
        if fewha.precision != "f32":
            raise ValueError("the learned warm start runs with an FP32 Fewha instance")
        self.torch, self.f, self.lib = torch, fewha, load_library()
        self.tensor_cores = tensor_cores  # online prediction on the tcgen05 convolution
        self.net = ConvNet(geom, seed=seed)
        n = self.n = fewha.n
        dev = fewha.device
        self.alpha_d = torch.tensor(fewha.prior(), dtype=torch.float32, device=dev)
        self.group = torch.tensor(scale_groups(geom), device=dev)
        self.in_scale = self.alpha_d.clone()
        self.out_scale = self.alpha_d.clone()
        self.x = torch.zeros((4, n), dtype=torch.float32, device=dev)
        self.y = torch.zeros((N_DIR, n), dtype=torch.float32, device=dev)
        self.gy = torch.zeros_like(self.y)
        self.t = torch.zeros_like(self.y)
        self.ring = torch.zeros((8, n), dtype=torch.float32, device=dev)
        self.count = 0
        self.D = torch.zeros((N_DIR, n), dtype=torch.float32, device=dev)
        self.Q = torch.zeros_like(self.D)
        self.b = torch.zeros(n, dtype=torch.float32, device=dev)
        self.r0 = torch.zeros(n, dtype=torch.float32, device=dev)
        self.work = torch.zeros(4096, dtype=torch.float64, device=dev)
        self.info = torch.zeros(16, dtype=torch.float64, device=dev)
        self.zero = torch.zeros(N_DIR * n, dtype=torch.float32, device=dev)

    # -- normalisation ------------------------------------------------------------
    def _mean_square(self, v):
        self.net.mse(v, self.zero[:v.numel()], self.gy.view(-1)[:v.numel()])
        return self.net.loss()

    def fit_scales(self, C_frames, sample=64):
        """Global input/output scales from a sample of solutions C_frames (T, n):
        inputs whitened by alpha D have unit mean square, and so do the targets."""
        torch = self.torch
        T = C_frames.shape[0]
        idx = np.linspace(0, T - 2, min(sample, T - 1)).astype(int)
        ms_in, ms_out = 0.0, 0.0
        for t in idx:
            _scale(self.lib, torch, C_frames[t], self.alpha_d, self.x[0], 0)
            ms_in += self._mean_square(self.x[0])
            self._targets(C_frames[t + 1], C_frames[t], self.alpha_d)
            ms_out += self._mean_square(self.t[0])
        ms_in /= len(idx)
        ms_out /= len(idx)
        self.in_scale = self.alpha_d / ms_in
        self.out_scale = self.alpha_d / ms_out
        return ms_in, ms_out

    def _targets(self, c_next, c_cur, scale):
        st = self.lib.fewha_learned_targets(C.c_void_p(c_next.data_ptr()), C.c_void_p(c_cur.data_ptr()),
                                            C.c_void_p(scale.data_ptr()), C.c_void_p(self.group.data_ptr()),
                                            C.c_void_p(self.t.data_ptr()), self.n, _stream_ptr(self.torch))
        if st != 0:
            raise FewhaError(st, "fewha_learned_targets")

    # -- training -------------------------------------------------------------------
    def train_step(self, C_frames, t, lr):
        """One Adam step on the example 'frames t-3..t -> frame t+1' of C_frames (T, n)."""
        torch = self.torch
        for k in range(4):
            _scale(self.lib, torch, C_frames[t - k], self.in_scale, self.x[k], 0)
        x_ptr = self.x.data_ptr()
        self.net.forward(x_ptr, self.n, self.y)
        self._targets(C_frames[t + 1], C_frames[t], self.out_scale)
        self.net.mse(self.y, self.t, self.gy)
        self.net.backward(x_ptr, self.n, self.gy)
        self.net.adam(lr)

    def train(self, C_frames, epochs=2, lr=1e-3, seed=0, log=None):
        """Adam over all examples of C_frames in a seeded random order per epoch;
        the learning rate decays by cosine to lr/20.  Returns the mean loss
        of the first and the last 200 steps."""
        T = C_frames.shape[0]
        rng = np.random.default_rng(seed)
        idx_all = np.arange(3, T - 1)
        total = epochs * len(idx_all)
        first, last, k = [], [], 0
        for ep in range(epochs):
            for t in rng.permutation(idx_all):
                a = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * k / total)))
                self.train_step(C_frames, int(t), a)
                if k < 200 or k >= total - 200 or (log and k % 2000 == 0):
                    L = self.net.loss()
                    if k < 200:
                        first.append(L)
                    if k >= total - 200:
                        last.append(L)
                    if log and k % 2000 == 0:
                        log("step %d/%d loss %.4f" % (k, total, L))
                k += 1
        return float(np.mean(first)), float(np.mean(last))

    def validation_loss(self, C_frames):
        T = C_frames.shape[0]
        tot = 0.0
        for t in range(3, T - 1):
            for k in range(4):
                _scale(self.lib, self.torch, C_frames[t - k], self.in_scale, self.x[k], 0)
            self.net.forward(self.x.data_ptr(), self.n, self.y)
            self._targets(C_frames[t + 1], C_frames[t], self.out_scale)
            self.net.mse(self.y, self.t, self.gy)
            tot += self.net.loss()
        return tot / max(1, T - 4)

    # -- online use -------------------------------------------------------------------
    def reset(self):
        self.count = 0

    def push(self, c):
        """Records the solution of the time step just solved (whitened into the ring)."""
        j = self.count % 4
        _scale(self.lib, self.torch, c, self.in_scale, self.ring[j], 0)
        self.ring[j + 4].copy_(self.ring[j])
        self.count += 1

    def prepare(self, s, c, state):
        """Before solving the time step with slopes s: predict the directions and
        apply the deflated warm start to (c, state).  Returns False (and does
        nothing) until four solutions have been pushed."""
        if self.count < 4:
            return False
        torch, lib, n = self.torch, self.lib, self.n
        self.f.rhs(s, out=self.b)
        j = (self.count - 1) % 4
        self.net.forward(self.ring[j + 4].data_ptr(), -n, self.y, tensor_cores=self.tensor_cores)
        for k in range(N_DIR):
            _scale(lib, torch, self.y[k], self.out_scale, self.D[k], 1)
        self.f.apply_op_multi(self.D, out=self.Q)
        st = lib.fewha_deflate_warm_start(C.c_void_p(self.b.data_ptr()), C.c_void_p(self.D.data_ptr()), n,
                                          C.c_void_p(self.Q.data_ptr()), n, N_DIR, C.c_void_p(c.data_ptr()),
                                          C.c_void_p(state.b_prev.data_ptr()),
                                          C.c_void_p(state.r_prev.data_ptr()), n, C.c_void_p(self.r0.data_ptr()),
                                          C.c_void_p(self.work.data_ptr()), C.c_void_p(self.info.data_ptr()),
                                          _stream_ptr(torch))
        if st != 0:
            raise FewhaError(st, "fewha_deflate_warm_start")
        return True

    def last_info(self):
        """(taken, ||r after||, ||r0||, directions kept) of the last prepare() (synchronises)."""
        i = self.info.cpu().numpy()
        return bool(i[0]), float(i[1]), float(i[2]), int(i[3])


def solve_sequence(f, slopes, rtol, max_iter, kcap=8, augmented=True, learned=None, record=None, flush=None):
    """Runs the reconstructor loop over slopes (T, n_slopes) with fresh state.
    learned: a LearnedWarmStart used for the deflated warm start (None: the
    plain warm start of Algorithm 3).  record: optional (T, n) tensor that
    receives every solution.  Returns per-frame iterations, rel_res, device
    microseconds (CUDA events around prepare + solve) and, for the learned
    loop, the deflation info.  flush: optional tensor larger than L2, zeroed
    before every frame (outside the timed region)."""
    torch = f._torch
    T = slopes.shape[0]
    c = torch.zeros(f.n, dtype=f.dtype, device=f.device)
    st = f.new_state(kcap)
    stats = [f.new_stats() for _ in range(T)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(T)]
    infos = []
    if learned is not None:
        learned.reset()
    for t in range(T):
        if flush is not None:
            flush.zero_()
        ev[t][0].record()
        used = learned.prepare(slopes[t], c, st) if learned is not None else False
        # after prepare() the state holds this step's right-hand side
        f.solve(slopes[t], c, st, max_iter, rtol=rtol, augmented=augmented, stats=stats[t], rhs_in_state=used)
        ev[t][1].record()
        if learned is not None:
            learned.push(c)
            infos.append(learned.info.clone() if used else None)
        if record is not None:
            record[t].copy_(c)
    torch.cuda.synchronize()
    out = {"iterations": [], "rel_res": [], "us": [], "status": []}
    for t in range(T):
        r = f.read_stats(stats[t])
        out["iterations"].append(r["iterations"])
        out["rel_res"].append(r["rel_res"])
        out["status"].append(r["status"])
        out["us"].append(ev[t][0].elapsed_time(ev[t][1]) * 1e3)
    if learned is not None:
        out["taken"] = [None if i is None else bool(i[0].item()) for i in infos]
        out["r_ratio"] = [None if i is None else float(i[1].item() / max(i[2].item(), 1e-300)) for i in infos]
    return out


def study(f, geom, slopes_train, slopes_eval, rtol, max_iter=1000, epochs=2, lr=1e-3, kcap=8, seed=0,
          skip=10, log=None, flush=None):
    """Trains the network on the solutions the plain method produces for
    slopes_train, then runs the plain and the learned loop over slopes_eval.
    Returns a summary dict (means over the evaluation frames after `skip`)."""
    torch = f._torch
    import time
    T = slopes_train.shape[0]
    C_frames = torch.empty((T, f.n), dtype=torch.float32, device=f.device)
    t0 = time.time()
    gen = solve_sequence(f, slopes_train, rtol, max_iter, kcap, record=C_frames)
    t_gen = time.time() - t0
    lw = LearnedWarmStart(f, geom, seed=seed)
    ms_in, ms_out = lw.fit_scales(C_frames[skip:])
    t0 = time.time()
    loss0, loss1 = lw.train(C_frames[skip:], epochs=epochs, lr=lr, seed=seed, log=log)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    plain = solve_sequence(f, slopes_eval, rtol, max_iter, kcap, flush=flush)
    lrn = solve_sequence(f, slopes_eval, rtol, max_iter, kcap, learned=lw, flush=flush)
    # the learned loop's own cost: network, M D and the projection (prepare() alone)
    sl = slice(skip, None)

    def mean(v):
        return float(np.mean(v[sl]))

    taken = [x for x in lrn["taken"][sl] if x is not None]
    ratios = [r for r, k in zip(lrn["r_ratio"][sl], lrn["taken"][sl]) if k]
    return {
        "train_frames": int(T), "eval_frames": int(slopes_eval.shape[0]), "rtol": rtol, "epochs": epochs,
        "gen_s": t_gen, "train_s": t_train, "gen_iterations_mean": float(np.mean(gen["iterations"][skip:])),
        "loss_first": loss0, "loss_last": loss1, "val_loss": lw.validation_loss(C_frames[-min(200, T):]),
        "rms_in": math.sqrt(ms_in), "rms_out": math.sqrt(ms_out),
        "plain": {"iterations": mean(plain["iterations"]), "us": mean(plain["us"]),
                  "rel_res": mean(plain["rel_res"]), "max_iter_hits": int(np.sum(np.array(plain["iterations"][sl]) >= max_iter))},
        "learned": {"iterations": mean(lrn["iterations"]), "us": mean(lrn["us"]),
                    "rel_res": mean(lrn["rel_res"]), "taken_frac": float(np.mean(taken)) if taken else 0.0,
                    "r0_ratio_taken": float(np.mean(ratios)) if ratios else None,
                    "max_iter_hits": int(np.sum(np.array(lrn["iterations"][sl]) >= max_iter))},
        "status_ok": all(s == 0 for s in plain["status"] + lrn["status"]),
        "learner": lw,
    }
