"""Seeded synthetic wavefront-sensor data: von Karman frozen-flow turbulence
seen by Shack-Hartmann sensors.

This is the stand-in for the paper's end-to-end simulator (MOST, Sec. 5.1),
which is not available.  It models the sky, not the reconstructor: each layer
is a periodic von Karman phase screen (FFT method, r0_l = r0 cn2_l^{-3/5},
outer scale L0) on a grid twice as fine as the subapertures, moved by its wind
vector every frame (frozen flow).  A sensor measures, per subaperture, the
difference of the mean phase on opposite edges (three points per edge), with
the phase at a point being the sum over layers of the screens sampled at the
point's position on each layer (cone compression for laser guide stars).
White Gaussian noise with sigma_g = rms(noise-free slopes of g)/SNR is added.
None of the reconstructor's discrete operators (bilinear layer
interpolation, the four-node gradient, wavelets) is used here.
"""
import math

import numpy as np
import torch


def pupil_mask(geom, ns=None) -> np.ndarray:
    """Illuminated subapertures of an ns x ns sensor (default: the geometry's
    n_sub): centre radius within [obstruction*D/2, D/2]; the single
    subaperture of a 1x1 sensor sees the whole pupil and is always lit."""
    ns, D = ns or geom.n_sub, geom.D
    if ns == 1:
        return np.ones(1, dtype=bool)
    c = -D / 2 + (np.arange(ns) + 0.5) * D / ns
    r = np.hypot(c[None, :], c[:, None])
    return ((r >= geom.obstruction * D / 2) & (r <= D / 2)).reshape(-1)


def random_vector(n, seed, dtype=np.float64):
    """Standard normal test vector of length n (seeded)."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype)


class FrozenFlowSensors:
    """Noise-free and noisy Shack-Hartmann slopes for a sequence of frames."""

    def __init__(self, geom, seed=0, device="cpu", oversample=2, frame_rate=500.0):
        self.geom = geom
        self.device = torch.device(device)
        self.dt = 1.0 / frame_rate
        ns, D = geom.n_sub, geom.D
        self.ds = D / ns
        self.step = self.ds / oversample
        rmax = 0.0
        for l in geom.layers:
            for g in geom.gs:
                s = (1.0 - l.h / g.H) if g.H > 0 else 1.0
                rmax = max(rmax, s * D / 2 + max(abs(g.theta_x), abs(g.theta_y)) * l.h)
        M = 64
        while M < 2 * rmax / self.step + 8:
            M *= 2
        self.M = M
        rng = np.random.default_rng(seed)
        f = np.fft.fftfreq(M, self.step)
        fx, fy = np.meshgrid(f, f)
        f2 = fx * fx + fy * fy
        df = 1.0 / (M * self.step)
        screens = []
        for l in geom.layers:
            r0l = geom.r0 * l.cn2 ** (-3.0 / 5.0)
            psd = 0.023 * r0l ** (-5.0 / 3.0) * (f2 + 1.0 / geom.L0 ** 2) ** (-11.0 / 6.0)
            psd[0, 0] = 0.0
            cn = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) * np.sqrt(psd) * df
            screens.append(np.real(np.fft.ifft2(cn)) * M * M)
        self.screens = torch.tensor(np.stack(screens), dtype=torch.float64, device=self.device)
        winds = geom.wind if geom.wind else [(10.0, 0.0)] * len(geom.layers)
        self.wind = [(s * math.cos(d), s * math.sin(d)) for s, d in winds]
        # edge sample points of every sensor size: per size, the vertical
        # edges (x = nodes[j], y = rows[i, e], shape (ns, ns+1, 3)) and the
        # horizontal edges (y = nodes[i], x = rows[j, e], shape (ns+1, ns, 3))
        t = torch.tensor([1.0 / 6, 0.5, 5.0 / 6], dtype=torch.float64, device=self.device)
        self.edges, self.masks = {}, {}
        for g in range(len(geom.gs)):
            nsg = geom.sensor_ns(g)
            if nsg in self.edges:
                continue
            dsg = D / nsg
            nodes = -D / 2 + torch.arange(nsg + 1, dtype=torch.float64, device=self.device) * dsg
            rows = -D / 2 + (torch.arange(nsg, dtype=torch.float64, device=self.device)[:, None] + t) * dsg
            self.edges[nsg] = (nodes[None, :, None].expand(nsg, nsg + 1, 3), rows[:, None, :].expand(nsg, nsg + 1, 3),
                               rows[None, :, :].expand(nsg + 1, nsg, 3), nodes[:, None, None].expand(nsg + 1, nsg, 3))
            self.masks[nsg] = pupil_mask(geom, nsg)
        self.mask = self.masks[geom.sensor_ns(0)]

    def _sample(self, l, px, py):
        M, st = self.M, self.step
        u = px / st + M / 2
        v = py / st + M / 2
        iu = torch.floor(u)
        iv = torch.floor(v)
        fu, fv = u - iu, v - iv
        iu = iu.long() % M
        iv = iv.long() % M
        iu1, iv1 = (iu + 1) % M, (iv + 1) % M
        S = self.screens[l]
        return ((1 - fv) * ((1 - fu) * S[iv, iu] + fu * S[iv, iu1])
                + fv * ((1 - fu) * S[iv1, iu] + fu * S[iv1, iu1]))

    def _phase(self, g, frame, x, y):
        """Phase at points (x, y) seen from guide star g; `frame` is an int or a
        1-D tensor of frame indices (then a leading frame axis is added)."""
        if isinstance(frame, torch.Tensor):
            sh = (-1,) + (1,) * x.dim()
            fr = frame.to(torch.float64).reshape(sh)
            x, y = x.unsqueeze(0), y.unsqueeze(0)
        else:
            fr = frame
        tot = 0.0
        for l, lay in enumerate(self.geom.layers):
            s = (1.0 - lay.h / g.H) if g.H > 0 else 1.0
            wx, wy = self.wind[l]
            ox = g.theta_x * lay.h - wx * fr * self.dt
            oy = g.theta_y * lay.h - wy * fr * self.dt
            tot = tot + self._sample(l, s * x + ox, s * y + oy)
        return tot

    def clean_slopes(self, frame) -> torch.Tensor:
        """Noise-free slopes of all sensors, [x block | y block] per guide star."""
        out = []
        for k, g in enumerate(self.geom.gs):
            vx, vy, hx, hy = self.edges[self.geom.sensor_ns(k)]
            V = self._phase(g, frame, vx, vy).mean(-1)  # (ns, ns+1)
            Hh = self._phase(g, frame, hx, hy).mean(-1)  # (ns+1, ns)
            sx = V[:, 1:] - V[:, :-1]
            sy = Hh[1:, :] - Hh[:-1, :]
            out += [sx.reshape(-1), sy.reshape(-1)]
        return torch.cat(out)

    def clean_slopes_many(self, frames) -> torch.Tensor:
        """clean_slopes for a 1-D tensor of frame indices: (len(frames), n_slopes)."""
        out = []
        for k, g in enumerate(self.geom.gs):
            vx, vy, hx, hy = self.edges[self.geom.sensor_ns(k)]
            V = self._phase(g, frames, vx, vy).mean(-1)
            Hh = self._phase(g, frames, hx, hy).mean(-1)
            sx = V[:, :, 1:] - V[:, :, :-1]
            sy = Hh[:, 1:, :] - Hh[:, :-1, :]
            out += [sx.reshape(len(frames), -1), sy.reshape(len(frames), -1)]
        return torch.cat(out, dim=1)

    def noise_sigma(self) -> np.ndarray:
        """sigma_g = rms of the noise-free slopes of g on lit subapertures / SNR."""
        s0 = self.clean_slopes(0).cpu().numpy()
        sig, off = [], 0
        for g in range(len(self.geom.gs)):
            nsg = self.geom.sensor_ns(g)
            ns2, mk = nsg * nsg, self.masks[nsg]
            blk = s0[off: off + 2 * ns2]
            off += 2 * ns2
            v = np.concatenate([blk[:ns2][mk], blk[ns2:][mk]])
            sig.append(math.sqrt(float(np.mean(v * v))) / self.geom.snr)
        return np.array(sig)

    def _sigma_vector(self, sig):
        """sigma_g repeated over the 2 n_g^2 slopes of every guide star."""
        reps = [2 * self.geom.sensor_ns(g) ** 2 for g in range(len(self.geom.gs))]
        return torch.tensor(np.repeat(sig, reps), dtype=torch.float64, device=self.device)

    def sequence(self, n_frames, seed=1, noise=True, dtype=torch.float64, first_frame=0):
        """Returns (slopes [n_frames, n_slopes] on self.device, noise weights 1/sigma^2)."""
        sig = self.noise_sigma()
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        sig_vec = self._sigma_vector(sig)
        frames = torch.empty((n_frames, self.geom.n_slopes), dtype=dtype, device=self.device)
        for t in range(n_frames):
            s = self.clean_slopes(first_frame + t)
            if noise:
                s = s + sig_vec * torch.randn(s.shape, generator=gen, dtype=torch.float64,
                                              device=self.device)
            frames[t] = s.to(dtype)
        return frames, 1.0 / sig ** 2

    def sequence_chunked(self, n_frames, seed=1, dtype=torch.float32, first_frame=0, chunk=64):
        """Like `sequence` (same sky and noise model) for long runs: frames
        are produced `chunk` at a time and the noise of a chunk is drawn in one
        call, so the noise values differ from `sequence` for the same seed."""
        sig = self.noise_sigma()
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        sig_vec = self._sigma_vector(sig)
        frames = torch.empty((n_frames, self.geom.n_slopes), dtype=dtype, device=self.device)
        for t0 in range(0, n_frames, chunk):
            f = torch.arange(first_frame + t0, first_frame + min(n_frames, t0 + chunk), device=self.device)
            s = self.clean_slopes_many(f)
            s = s + sig_vec * torch.randn(s.shape, generator=gen, dtype=torch.float64, device=self.device)
            frames[t0:t0 + len(f)] = s.to(dtype)
        return frames, 1.0 / sig ** 2
