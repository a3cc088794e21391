#!/usr/bin/env python
"""Benchmark of the augmented FEWHA time step on GB300.

A step is one reconstructor time step (Algorithm 3: right-hand side, warm
restart residual, augmented PCG to a fixed relative residual) on one frame of
the ELT-size workload: 39 m pupil, 6 LGS at 90 km with 84x84 Shack-Hartmann
sensors, 9 layers (5 x 128^2 + 4 x 64^2, n = 98304), Daubechies-3 with 5
levels, recycled basis k = 8.  Inputs are a seeded frozen-flow slope sequence
resident in HBM; L2 is flushed (256 MB written) before every timed frame.

--impl reference runs the FP64 CPU oracle on the same workload (a bounded
sample of frames per step) on the host cores.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ELT-size \u00b5s/frame & frames/s at fixed residual vs plain PCG; L2/HBM % of peak"
UNIT = "frames/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="elt")
    p.add_argument("--precision", default="f32", choices=["f64", "f32", "bf16s"])
    p.add_argument("--rtol", type=float, default=1e-2)
    p.add_argument("--max-iter", type=int, default=200)
    p.add_argument("--k", type=int, default=8)
    p.add_argument("--snr", type=float, default=None)
    p.add_argument("--plain", action="store_true", help="PCG instead of augmented PCG")
    p.add_argument("--launch", default="persistent", choices=["persistent", "phases"])
    p.add_argument("--no-flush", action="store_true")
    p.add_argument("--no-compare", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-frames", type=int, default=3)
    p.add_argument("--tile", type=int, default=0)
    p.add_argument("--grid", type=int, default=0)
    p.add_argument("--no-batched", action="store_true", help="skip the 64-instance batched measurement")
    p.add_argument("--batched-steps", type=int, default=20)
    p.add_argument("--learned", action="store_true",
                   help="learned warm start study instead of the time-step benchmark")
    p.add_argument("--learned-train", type=int, default=20000, help="training frames")
    p.add_argument("--learned-eval", type=int, default=500, help="held-out frames")
    p.add_argument("--epochs", type=int, default=2)
    p.add_argument("--diagnostics", action="store_true",
                   help="condition numbers kappa_0..2 of the configuration (Lanczos on the FP64 operator)")
    p.add_argument("--lanczos-steps", type=int, default=300)
    return p.parse_args()


def workload_name(geom, args):
    return ("%s: D=%.0f m, %d GS (%s), %dx%d SH, %d layers (%s), n=%d, Daubechies-%d, k=%d, "
            "%s PCG to rel. residual %g, %s"
            % (geom.name, geom.D, len(geom.gs), "LGS H=90 km" if geom.gs[0].H > 0 else "NGS",
               geom.n_sub, geom.n_sub, len(geom.layers),
               "+".join("%d^2" % l.n for l in geom.layers), geom.n_unknowns, geom.wavelet_N,
               args.k, "plain" if args.plain else "augmented", args.rtol, args.precision))


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2011_06842_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def max_over_ranks(total_ms, ws, device):
    """The timed region's length as the job sees it: the maximum over ranks
    (all-reduce MAX, then a barrier).  Replicas share no data; this is the only
    collective of the measurement."""
    if ws <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_rate(units_per_rank, ws, max_ms):
    """Units of all ranks per second over the slowest rank's time."""
    return ws * units_per_rank / (max_ms / 1e3)


def make_frames(geom, nframes, seed, device):
    from synth import FrozenFlowSensors
    sim = FrozenFlowSensors(geom, seed=seed, device=device)
    s, w = sim.sequence_chunked(nframes, seed=seed + 1, dtype=torch_float64())
    return s, w


def torch_float64():
    import torch
    return torch.float64


def time_solves(f, frames, dtype, args, nwarm, nsteps, aug, flush_buf, stats_buf, rtol):
    """Per-frame CUDA-event timing; returns (times_ms, stats list)."""
    import torch
    n = f.n
    c = torch.zeros(n, dtype=f.dtype, device="cuda")
    st = f.new_state(args.k)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    sl = frames.to(dtype)
    for t in range(nwarm):
        f.solve(sl[t], c, st, args.max_iter, rtol=rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats_buf[t % len(stats_buf)])
    torch.cuda.synchronize()
    for t in range(nsteps):
        if flush_buf is not None:
            flush_buf.zero_()
        starts[t].record()
        f.solve(sl[nwarm + t], c, st, args.max_iter, rtol=rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats_buf[t])
        ends[t].record()
    torch.cuda.synchronize()
    times = [starts[t].elapsed_time(ends[t]) for t in range(nsteps)]
    stats = [f.read_stats(stats_buf[t]) for t in range(nsteps)]
    return times, stats


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup(args)
    from paper_2011_06842_gb300 import Fewha, build, workload
    build.build()
    from synth import configs
    geom = configs.get(args.config)
    if args.snr:
        geom.snr = args.snr
    geom.k_recycle = args.k
    nframes = args.warmup + args.steps
    frames, w = make_frames(geom, nframes, seed=100 + rank, device="cuda")
    sdt = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.bfloat16}[args.precision]
    f = Fewha(geom, w, args.precision, tile=args.tile, grid=args.grid)
    flush = None if args.no_flush else torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stats_buf = [f.new_stats() for _ in range(max(args.steps, args.warmup, 1))]
    aug = not args.plain

    # timed region: K frames, per-frame events; barrier + sync on both sides
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local) if rank == 0 else None
    times, stats = time_solves(f, frames, sdt, args, args.warmup, args.steps, aug, flush, stats_buf,
                               args.rtol)
    clocks = clk.stop() if clk else None
    total_ms = sum(times)
    total_ms = max_over_ranks(total_ms, ws, "cuda")
    bad = [s for s in stats if s["status"] != 0]
    if bad:
        raise RuntimeError("device-side error in a timed frame: %s" % bad[0])
    iters = [s["iterations"] for s in stats]
    relres = [s["rel_res"] for s in stats]
    fps = whole_job_rate(args.steps, ws, total_ms)
    us_frame = total_ms / args.steps * 1e3

    # roofline of the dominant kernel (the persistent solver kernel; one launch per frame)
    word = 8 if args.precision == "f64" else 4
    mean_it = float(np.mean(iters))
    algo_bytes = workload.solve_bytes(geom, mean_it, min(args.k, max(1, int(round(mean_it)))) if aug else 0,
                                      word)
    achieved = algo_bytes / (us_frame * 1e-6) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        tj = json.load(open(tp))
        key = "%s/%s/%s" % (args.config, args.precision, "aug" if aug else "plain")
        if tj.get("source_hash") == source_hash() and key in tj.get("per_launch", {}):
            traffic = tj["per_launch"][key]

    out = {"metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": us_frame / 1e3, "us_per_frame": us_frame,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision, "data": "synthetic: seeded von Karman frozen-flow screens "
           "(r0=%.3f m, L0=%.0f m, wind 5-20 m/s) seen by SH sensors, SNR %g" % (geom.r0, geom.L0, geom.snr),
           "config": {"workload": workload_name(geom, args), "n_unknowns": geom.n_unknowns,
                      "n_slopes": geom.n_slopes, "rtol": args.rtol, "max_iter": args.max_iter,
                      "k_recycle": args.k, "launch": args.launch, "frames": nframes,
                      "l2": "flushed (256 MB written) before every timed frame" if flush is not None
                      else "not flushed", "parallelism": "replicas" if ws > 1 else "single GPU"},
           "iterations": {"mean": mean_it, "min": min(iters), "max": max(iters)},
           "rel_res": {"mean": float(np.mean(relres)), "max": float(np.max(relres))},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "kernel": "k_solve_persistent" if args.launch == "persistent" else "all phases",
                        "algorithmic_bytes_per_launch": algo_bytes, "peak_source": peak_kind},
           "gpu_launches": args.steps * (1 if args.launch == "persistent" else 6 + 6 * args.max_iter)}
    if clocks:
        out["clocks"] = clocks

    if rank == 0:
        out["e2e"] = run_e2e(f, geom, frames, sdt, args, aug)
        out["algorithm3"] = run_algorithm3(f, frames, sdt, args, aug, flush)
        out["mcao_fit"] = run_mcao(f, geom, frames, sdt, args, aug, flush)
        if not args.no_compare:
            out["compare"] = run_compare(geom, w, frames, args, stats_buf, flush)
        if not args.no_cpu and ws == 1:
            out["cpu_baseline"] = run_cpu_baseline(geom, w, frames, iters, args, aug)
        if not args.no_batched and args.precision == "f32":
            out["batched"] = run_batched(args, flush)
    f.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


def launch_shape(cand):
    """(rounds, CTAs of the launch) of a tuned batch candidate (ctas, rounds)."""
    if not isinstance(cand, tuple):
        return None
    ctas, rounds = cand
    per = {}
    for n, r in zip(ctas, rounds):
        per[r] = per.get(r, 0) + n
    return [len(per), max(per.values())]


def run_batched(args, flush):
    """64 independent instances of uneven size (24 x tiny, 24 x medium, 16 x ELT
    geometry, each with its own seeded frozen-flow sequence), FP32, augmented
    PCG to the same relative residual, in ONE cooperative launch per step with
    an autotuned split of the CTAs between instances (one round, or two or
    three rounds: the ELT instances first on many CTAs each, then the small
    instances on the same CTAs, separated by a barrier over the launch)."""
    import numpy as np
    import torch
    from paper_2011_06842_gb300 import Fewha, FewhaBatch, autotune_batch, workload
    from synth import configs
    kinds = ["tiny"] * 24 + ["medium"] * 24 + ["elt"] * 16
    K, W = args.batched_steps, 3
    inst = []
    for i, kind in enumerate(kinds):
        geom = configs.get(kind)
        frames, w = make_frames(geom, W + K + 4, seed=500 + i, device="cuda")
        f = Fewha(geom, w, "f32")
        inst.append({"geom": geom, "f": f, "s": frames.float(), "c": torch.zeros(f.n, device="cuda"),
                     "st": f.new_state(args.k)})
    fewhas = [x["f"] for x in inst]
    frame = [0]

    def step(b, t=None):
        t = frame[0] if t is None else t
        b.solve([x["s"][t] for x in inst], [x["c"] for x in inst], [x["st"] for x in inst],
                args.max_iter, rtol=args.rtol, augmented=not args.plain)
        frame[0] = (t + 1) % 4  # the autotuner reuses the first frames

    # candidates: one round (the library's work-proportional split); two
    # rounds (the 16 ELT instances on 8-9 CTAs each, then the small ones); three
    # rounds (8 ELT instances at a time on 18-19 CTAs each, enough for the
    # split transforms, then the small ones)
    two = [0 if k == "elt" else 1 for k in kinds]
    elt_ids = [i for i, k in enumerate(kinds) if k == "elt"]
    three = [(0 if elt_ids.index(i) < 8 else 1) if k == "elt" else 2 for i, k in enumerate(kinds)]

    def split(elt, med, tiny):
        return [elt if k == "elt" else med if k == "medium" else tiny for k in kinds]

    cands = [None, (split(9, 4, 1), two), (split(9, 5, 1), two), (split(8, 5, 1), two),
             (split(19, 4, 1), three), (split(18, 5, 1), three)]
    best, timings = autotune_batch(fewhas, step, candidates=cands, reps=2)
    for x in inst:  # fresh states after tuning
        x["st"] = x["f"].new_state(args.k)
        x["c"].zero_()
    batch = FewhaBatch(fewhas, *best)
    stats = [batch.new_stats() for _ in range(K)]
    for t in range(W):
        batch.solve([x["s"][4 + t] for x in inst], [x["c"] for x in inst], [x["st"] for x in inst],
                    args.max_iter, rtol=args.rtol, augmented=not args.plain)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for t in range(K):
        if flush is not None:
            flush.zero_()
        ev[t][0].record()
        batch.solve([x["s"][4 + W + t] for x in inst], [x["c"] for x in inst], [x["st"] for x in inst],
                    args.max_iter, rtol=args.rtol, augmented=not args.plain, stats=stats[t])
        ev[t][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    st = [batch.read_stats(x) for x in stats]
    bad = [r for row in st for r in row if r["status"] != 0]
    its = np.array([[r["iterations"] for r in row] for row in st])
    algo = sum(workload.solve_bytes(x["geom"], float(its[:, i].mean()), args.k, 4) for i, x in enumerate(inst))
    us_step = ms / K * 1e3
    peak, _ = measured_peaks()
    out = {"instances": len(inst), "mix": "24 x tiny (8 m, 16x16, 4 NGS, 2 x 32^2) + 24 x medium (16 m, 40x40, "
           "4 LGS, 5 x 64^2) + 16 x ELT (39 m, 84x84, 6 LGS, 9 layers)", "steps": K, "warmup": W,
           "us_per_step": us_step, "instance_frames_per_s": len(inst) * K / (ms / 1e3),
           "elt_instance_frames_per_s": 16 * K / (ms / 1e3),
           "elt_equivalent_frames_per_s": sum(x["f"].n for x in inst) / inst[-1]["f"].n * K / (ms / 1e3),
           "iterations_mean": float(its.mean()),
           "ctas": batch.ctas(), "rounds": batch.rounds,
           "autotune_ms_per_step": [[launch_shape(c), t] for c, t in timings],
           "status_ok": not bad, "roofline": {"bound": "hbm", "achieved": algo / (us_step * 1e-6) / 1e9,
                                             "peak": peak, "unit": "GB/s",
                                             "frac": algo / (us_step * 1e-6) / 1e9 / peak},
           "gpu_launches_per_step": 2}
    batch.close()
    for x in inst:
        x["f"].close()
    return out


def run_e2e(f, geom, frames, sdt, args, aug):
    """Same metric through the public API with host buffers: per frame the
    slopes are copied from pinned host memory and the solution c is read back."""
    import torch
    K = args.steps
    host = frames[args.warmup:args.warmup + K].to(sdt).cpu().pin_memory()
    out_host = torch.empty((K, f.n), dtype=f.dtype).pin_memory()
    dev_s = torch.empty(f.n_slopes, dtype=sdt, device="cuda")
    c = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    st = f.new_state(args.k)
    stats = f.new_stats()
    for t in range(min(args.warmup, K)):
        dev_s.copy_(host[t], non_blocking=True)
        f.solve(dev_s, c, st, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(K):
        dev_s.copy_(host[t], non_blocking=True)
        f.solve(dev_s, c, st, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
        out_host[t].copy_(c, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    esz = torch.tensor([], dtype=sdt).element_size()
    return {"value": K / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": f.n_slopes * esz,
            "d2h_bytes_per_step": f.n * c.element_size(), "us_per_frame": ms / K * 1e3}


def run_algorithm3(f, frames, sdt, args, aug, flush):
    """Whole closed-loop time steps of Algorithm 3 on the device: pseudo-open-loop
    slopes, the solve, fitting onto the ground mirror and gain control (gain
    0.4), per-frame CUDA events, L2 flushed before every frame.  The frames'
    slopes are open-loop; the closed-loop measurement s - Gamma a^(i-1) is
    formed before each timed step."""
    import torch
    K = min(args.steps, 200)
    sl = frames.to(sdt)
    c = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    st = f.new_state(args.k)
    stats = f.new_stats()
    mir = [f.new_mirror() for _ in range(3)]  # a^(i-1), a^(i), next (rotated, no copies)
    a_f, neg = f.new_mirror(), f.new_mirror()
    s_cl, s_pol = torch.empty_like(sl[0]), torch.empty_like(sl[0])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]

    def plant(t):
        # the sensors see the atmosphere minus the mirror applied two steps
        # earlier (outside the timed region: this is the telescope, not the
        # reconstructor)
        torch.neg(mir[0], out=neg)
        f.pol_slopes(sl[t], neg, out=s_cl)

    def step(t):
        f.pol_slopes(s_cl, mir[0], out=s_pol)
        f.solve(s_pol, c, st, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
        f.fit(c, out=a_f)
        f.control(True, 0.4, mir[0], mir[1], a_f, out=mir[2])
        mir[:] = [mir[1], mir[2], mir[0]]

    for t in range(args.warmup):
        plant(t)
        step(t)
    torch.cuda.synchronize()
    for k in range(K):
        plant(args.warmup + k)
        if flush is not None:
            flush.zero_()
        ev[k][0].record()
        step(args.warmup + k)
        ev[k][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    it = f.read_stats(stats)["iterations"]
    return {"us_per_frame": ms / K * 1e3, "frames_per_s": K / (ms / 1e3), "frames": K, "gain": 0.4,
            "loop": "closed", "iterations_last_frame": it, "gpu_launches_per_frame": 1 + 1 + 2 + 1}


def run_mcao(f, geom, frames, sdt, args, aug, flush):
    """MCAO fitting onto three mirrors after each solve (Sec. 5, 9-layer MCAO:
    4 unpreconditioned CG iterations on the fitting normal equations, warm
    started from the previous frame's mirrors): the paper's mirrors 85x85 /
    0.5 m at 0 m, 47x47 / 1 m at 4 km, 53x53 / 1 m at 12.7 km; fitting
    directions: the axis and 6 on a circle of 0.25 arcmin.  Per-frame CUDA
    events around (a) the fit alone and (b) solve + fit, L2 flushed before
    every frame."""
    import math
    import torch
    from paper_2011_06842_gb300 import McaoFit
    if geom.D > 30:
        dms = [(85, 0.5, 0.0), (47, 1.0, 4000.0), (53, 1.0, 12700.0)]
    else:
        dms = [(geom.n_sub + 3, geom.D / geom.n_sub, 0.0), (int(geom.D) + 5, 1.0, 4000.0),
               (int(geom.D) + 9, 1.0, 12700.0)]
    r = 0.25 * math.pi / (180.0 * 60.0)
    dirs = [(0.0, 0.0)] + [(r * math.cos(2 * math.pi * i / 6), r * math.sin(2 * math.pi * i / 6)) for i in range(6)]
    fit = McaoFit(f, dms, dirs)
    K = min(args.steps, 200)
    sl = frames.to(sdt)
    c = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    st = f.new_state(args.k)
    stats = f.new_stats()
    a = fit.new_mirrors()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for t in range(args.warmup):
        f.solve(sl[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug, stats=stats)
        fit.fit(c, a, 4)
    torch.cuda.synchronize()
    for k in range(K):
        if flush is not None:
            flush.zero_()
        ev[k][0].record()
        f.solve(sl[args.warmup + k], c, st, args.max_iter, rtol=args.rtol, augmented=aug, stats=stats)
        ev[k][1].record()
        fit.fit(c, a, 4)
        ev[k][2].record()
    torch.cuda.synchronize()
    fit_ms = sum(e[1].elapsed_time(e[2]) for e in ev)
    step_ms = sum(e[0].elapsed_time(e[2]) for e in ev)
    n_act = fit.n_actuators
    fit.close()
    return {"us_per_fit": fit_ms / K * 1e3, "us_per_step": step_ms / K * 1e3, "frames_per_s": K / (step_ms / 1e3),
            "frames": K, "cg_iterations": 4, "mirrors": dms, "directions": len(dirs), "actuators": n_act,
            "gpu_launches_per_fit": 2}


def run_compare(geom, w, frames, args, stats_buf, flush):
    """Plain PCG, the FP64 forms and the mixed-precision (BF16 storage) form on
    the same frames and residual target."""
    import numpy as np
    import torch
    from paper_2011_06842_gb300 import Fewha
    K = min(args.steps, 60)
    res = {}
    for prec, aug in (("f32", False), ("f64", False), ("f64", True), ("f32", True), ("bf16s", True)):
        if prec == args.precision and aug == (not args.plain):
            continue
        f = Fewha(geom, w, prec, tile=args.tile, grid=args.grid)
        sdt = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.bfloat16}[prec]
        times, stats = time_solves(f, frames, sdt, args, args.warmup, K, aug, flush, stats_buf, args.rtol)
        f.close()
        it = [s["iterations"] for s in stats]
        res["%s_%s" % ("aug" if aug else "plain", prec)] = {
            "frames_per_s": K / (sum(times) / 1e3), "us_per_frame": sum(times) / K * 1e3,
            "iterations_mean": float(np.mean(it)), "frames": K,
            "status_ok": all(s["status"] == 0 for s in stats)}
    return res


def run_cpu_baseline(geom, w, frames, gpu_iters, args, aug):
    """The FP64 oracle, single-threaded, on the first frames of the same sequence
    with the same per-frame iteration counts as the GPU run."""
    import numpy as np
    from oracle import Oracle
    nf = max(1, min(args.cpu_frames, args.steps))
    s = frames[:args.warmup + nf].double().cpu().numpy()
    o = Oracle(geom, w)
    st = o.new_state(args.k)
    for t in range(args.warmup):
        o.solve(s[t], st, max_iter=args.max_iter, rtol=args.rtol, augmented=aug)
    t0 = time.perf_counter()
    for t in range(nf):
        o.solve(s[args.warmup + t], st, max_iter=gpu_iters[t], rtol=0.0, augmented=aug)
    dt = time.perf_counter() - t0
    return {"value": nf / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d ELT frames after %d warm-up frames, FP64, same iteration counts as the GPU "
                      "frames (%s)" % (nf, args.warmup, ",".join(str(i) for i in gpu_iters[:nf]))}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from oracle import Oracle, build_oracle
    from synth import FrozenFlowSensors, configs
    build_oracle()
    geom = configs.get(args.config)
    if args.snr:
        geom.snr = args.snr
    sim = FrozenFlowSensors(geom, seed=100)
    s, w = sim.sequence_chunked(args.warmup + args.steps, seed=101, dtype=torch_float64())
    s = s.numpy()
    o = Oracle(geom, w)
    st = o.new_state(args.k)
    aug = not args.plain
    for t in range(args.warmup):
        o.solve(s[t], st, max_iter=args.max_iter, rtol=args.rtol, augmented=aug)
    t0 = time.perf_counter()
    its = []
    for t in range(args.steps):
        r = o.solve(s[args.warmup + t], st, max_iter=args.max_iter, rtol=args.rtol, augmented=aug)
        its.append(r["iterations"])
    dt = time.perf_counter() - t0
    v = args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (same seeded frozen-flow workload)",
            "config": {"workload": workload_name(geom, args) + " [FP64 CPU oracle]", "rtol": args.rtol},
            "iterations": {"mean": float(np.mean(its))},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d full frames, one per step, single-threaded" % args.steps},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_learned(args):
    """Learned warm start vs the plain warm start of Algorithm 3 (both with
    augmented PCG, FP32): train on frames the plain method solves, then run
    both loops over held-out frames to the same relative residual."""
    import numpy as np
    import torch
    from paper_2011_06842_gb300 import Fewha, build, learned
    from synth import FrozenFlowSensors, configs
    build.build()
    geom = configs.get(args.config)
    geom.snr = args.snr if args.snr else 100.0
    geom.k_recycle = args.k
    sim = FrozenFlowSensors(geom, seed=300, device="cuda")
    t0 = time.time()
    st, w = sim.sequence_chunked(args.learned_train, seed=301)
    se, _ = sim.sequence_chunked(args.learned_eval, seed=302, first_frame=10 * args.learned_train + 1000)
    t_slopes = time.time() - t0
    f = Fewha(geom, w, "f32")
    flush = None if args.no_flush else torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clk = Clocks(0)
    res = learned.study(f, geom, st, se, rtol=args.rtol, max_iter=args.max_iter, epochs=args.epochs,
                        kcap=args.k, flush=flush, log=lambda m: print(m, file=sys.stderr, flush=True))
    clocks = clk.stop()
    lw = res.pop("learner")

    def ev_us(fn, reps=20):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    x = torch.randn(learned.N_DIR, f.n, device="cuda")
    y = torch.empty_like(x)
    cost = {"rhs_us": ev_us(lambda: f.rhs(se[0], out=y[0])),
            "network_forward_us": ev_us(lambda: lw.net.forward(lw.ring[4].data_ptr(), -f.n, y)),
            "apply_multi5_us": ev_us(lambda: f.apply_op_multi(x, out=y)),
            "apply_single_us": ev_us(lambda: f.apply_op(x[0], out=y[1]))}
    out = {"metric": METRIC, "mode": "learned warm start", "unit": "frames/s",
           "value": 1e6 / res["learned"]["us"], "plain_value": 1e6 / res["plain"]["us"],
           "higher_is_better": True, "n_gpus": 1, "dtype": "f32",
           "data": "synthetic: seeded von Karman frozen-flow screens seen by SH sensors, SNR %g" % geom.snr,
           "config": {"workload": workload_name(geom, args) + ", learned warm start",
                      "rtol": args.rtol, "max_iter": args.max_iter, "k_recycle": args.k,
                      "network": "3x3 conv 4-32-32-5, ReLU", "train_frames": args.learned_train,
                      "eval_frames": args.learned_eval, "epochs": args.epochs,
                      "l2": "flushed before every frame" if flush is not None else "not flushed"},
           "slopes_generation_s": t_slopes, "study": res, "cost_breakdown": cost, "clocks": clocks}
    f.close()
    return out


def run_diagnostics(args):
    """kappa_0 = cond(M), kappa_1 = cond(J^{-1/2} M J^{-1/2}), kappa_2 with the
    recycled basis after 5 time steps (Sec. 6.2); Lanczos lower bounds."""
    import torch
    from paper_2011_06842_gb300 import Fewha, build
    from paper_2011_06842_gb300.diagnostics import condition_numbers
    from synth import configs
    build.build()
    geom = configs.get(args.config)
    if args.snr:
        geom.snr = args.snr
    frames, w = make_frames(geom, 5, seed=100, device="cuda")
    f = Fewha(geom, w, "f64")
    st = f.new_state(args.k)
    c = torch.zeros(f.n, dtype=torch.float64, device="cuda")
    for t in range(5):
        f.solve(frames[t], c, st, args.max_iter, rtol=args.rtol)
    P, Q, _ = st.basis()
    t0 = time.time()
    res = condition_numbers(f, basis=(P, Q), steps=args.lanczos_steps)
    res["seconds"] = time.time() - t0
    res["config"] = workload_name(geom, args)
    res["note"] = "Lanczos with %d steps: kappa values are lower bounds" % args.lanczos_steps
    f.close()
    return res


def main():
    args = parse()
    if args.diagnostics:
        print(json.dumps(run_diagnostics(args)))
        return
    if args.learned:
        print(json.dumps(run_learned(args)))
        return
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
