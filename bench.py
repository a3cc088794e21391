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
    p.add_argument("--cpu-frames", type=int, default=40)
    p.add_argument("--no-cpu-all", action="store_true", help="skip the all-host-cores oracle baseline")
    p.add_argument("--tile", type=int, default=0)
    p.add_argument("--grid", type=int, default=0)
    p.add_argument("--no-batched", action="store_true", help="skip the 64-instance batched measurement")
    p.add_argument("--batched-steps", type=int, default=20)
    p.add_argument("--learned", action="store_true",
                   help="learned warm start study instead of the time-step benchmark")
    p.add_argument("--trace", action="store_true",
                   help="per-phase trace of the time step (plain and augmented PCG)")
    p.add_argument("--conv-layers", action="store_true",
                   help="time each 3x3 convolution of the learned predictor (tensor cores and FP32)")
    p.add_argument("--learned-train", type=int, default=20000, help="training frames")
    p.add_argument("--learned-eval", type=int, default=500, help="held-out frames")
    p.add_argument("--epochs", type=int, default=2)
    p.add_argument("--diagnostics", action="store_true",
                   help="condition numbers kappa_0..2 of the configuration (Lanczos on the FP64 operator)")
    p.add_argument("--lanczos-steps", type=int, default=300)
    return p.parse_args()


def sensors_name(geom):
    """The asterism as text: '6 GS (LGS H=90 km), 84x84 SH' when every guide
    star has the same kind and sensor, else its groups in order."""
    def kind(g):
        return "LGS H=%.0f km" % (g.H / 1e3) if g.H > 0 else "NGS"
    groups = []
    for i, g in enumerate(geom.gs):
        key = (kind(g), geom.sensor_ns(i))
        if groups and groups[-1][0] == key:
            groups[-1][1] += 1
        else:
            groups.append([key, 1])
    if len(groups) == 1:
        (k, ns), cnt = groups[0]
        return "%d GS (%s), %dx%d SH" % (cnt, k, ns, ns)
    return "%d GS (%s) SH" % (len(geom.gs), ", ".join("%d %s %dx%d" % (cnt, k, ns, ns) for (k, ns), cnt in groups))


def workload_name(geom, args):
    return ("%s: D=%.0f m, %s, %d layers (%s), n=%d, Daubechies-%d, k=%d, "
            "%s PCG to rel. residual %g, SNR %g"
            % (geom.name, geom.D, sensors_name(geom), len(geom.layers),
               "+".join("%d^2" % l.n for l in geom.layers), geom.n_unknowns, geom.wavelet_N,
               args.k, "plain" if args.plain else "augmented", args.rtol, geom.snr))


def bench_config(geom, args, flush=True):
    """The `config` object of the JSON line, the same for both arms."""
    return {"workload": workload_name(geom, args), "n_unknowns": geom.n_unknowns, "n_slopes": geom.n_slopes,
            "rtol": args.rtol, "max_iter": args.max_iter, "k_recycle": args.k, "snr": geom.snr,
            "frames": args.warmup + args.steps,
            "l2": "flushed (256 MB written) before every timed frame" if flush else "not flushed",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "single GPU"}


def cpu_model():
    """CPU model name of this host (lscpu or /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# the sources of k_solve_persistent's translation unit and of its launch and
# tables (the ncu traffic in profiles/traffic.json is valid while they are unchanged)
KERNEL_SOURCES = ("api.cu", "device.cuh", "inst_f32.cu", "kernels.cuh", "mcao.cuh", "plan.cpp", "plan.h",
                  "solver.cuh")


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2011_06842_gb300", "csrc")
    for f in KERNEL_SOURCES:
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


def time_solves(f, frames, dtype, args, nwarm, nsteps, aug, flush_buf, stats_buf, rtol, true_res_every=0):
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
                persistent=args.launch == "persistent", stats=stats_buf[t % len(stats_buf)],
                true_res_every=true_res_every)
    torch.cuda.synchronize()
    for t in range(nsteps):
        if flush_buf is not None:
            flush_buf.zero_()
        starts[t].record()
        f.solve(sl[nwarm + t], c, st, args.max_iter, rtol=rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats_buf[t], true_res_every=true_res_every)
        ends[t].record()
    torch.cuda.synchronize()
    times = [starts[t].elapsed_time(ends[t]) for t in range(nsteps)]
    stats = [f.read_stats(stats_buf[t]) for t in range(nsteps)]
    return times, stats


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_setup(args)
    from paper_2011_06842_gb300 import Fewha, build, read_bandwidth, workload
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
    kv = min(args.k, max(1, int(round(mean_it)))) if aug else 0
    algo_bytes = workload.reference_solve_bytes(geom, mean_it, args.k, word, augmented=aug)
    impl_bytes = workload.solve_bytes(geom, mean_it, kv, word)
    achieved = algo_bytes / (us_frame * 1e-6) / 1e9
    peak, peak_kind = measured_peaks()
    l2_peak = read_bandwidth(48 << 20)
    traffic, l2_traffic = None, None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        tj = json.load(open(tp))
        key = "%s/%s/%s" % (args.config, args.precision, "aug" if aug else "plain")
        if tj.get("source_hash") == source_hash():
            traffic = tj.get("per_launch", {}).get(key)
            l2_traffic = tj.get("l2_per_launch", {}).get(key)

    out = {"metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": us_frame / 1e3, "us_per_frame": us_frame,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision, "data": "synthetic: seeded von Karman frozen-flow screens "
           "(r0=%.3f m, L0=%.0f m, wind 5-20 m/s) seen by SH sensors, SNR %g" % (geom.r0, geom.L0, geom.snr),
           "config": bench_config(geom, args, flush is not None),
           "launch": dict(f.launch_info(), mode=args.launch),
           "iterations": {"mean": mean_it, "min": min(iters), "max": max(iters)},
           "rel_res": {"mean": float(np.mean(relres)), "max": float(np.max(relres))},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "kernel": "k_solve_persistent" if args.launch == "persistent" else "all phases",
                        "algorithmic_bytes_per_launch": algo_bytes,
                        "algorithmic_count": "per iteration 14 n solver-vector words + the operator "
                        "intermediates (nodal layers, forward wavefronts, slopes, adjoint wavefronts, adjoint "
                        "layers) written once and read once; per time step + 1.5 operator-equivalents "
                        "(right-hand side, initial projection) + 9 n k basis reads (augmented)",
                        "impl_bytes_per_launch": impl_bytes,
                        "impl_count": "what this kernel must move: the slopes stay in registers inside the "
                        "fused WFS phase and z is never stored",
                        "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs, copy)" % peak_kind,
                        "l2": {"achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
                               "peak_source": "measured: fewha_read_probe, 48 MB L2-resident buffer read 20 times in one launch",
                               "traffic": l2_traffic}},
           "gpu_launches": args.steps * (1 if args.launch == "persistent" else 6 + 6 * args.max_iter)}
    if clocks:
        out["clocks"] = clocks

    if rank == 0:
        out["e2e"] = run_e2e(f, geom, frames, sdt, args, aug, flush)
        if len({geom.sensor_ns(g) for g in range(len(geom.gs))}) == 1:
            out["algorithm3"] = run_algorithm3(f, frames, sdt, args, aug, flush)
        else:
            out["algorithm3"] = {"skipped": "pseudo-open-loop slopes need every sensor on the ground mirror's "
                                            "node grid; this asterism has sensors of different sizes"}
        out["mcao_fit"] = run_mcao(f, geom, frames, sdt, args, aug, flush)
        if not args.no_compare:
            out["compare"] = run_compare(geom, w, frames, args, stats_buf, flush,
                                         (args.precision, aug, us_frame, mean_it))
        if not args.no_cpu and ws == 1:
            out["cpu_baseline"] = run_cpu_baseline(geom, w, frames, iters, args, aug)
        if not args.no_batched and args.precision == "f32":
            out["batched"] = run_batched(args, flush)
    f.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


def run_batched(args, flush):
    """64 independent instances of uneven size (24 x tiny, 24 x medium, 16 x ELT
    geometry, each with its own seeded frozen-flow sequence), FP32, augmented
    PCG to the same relative residual, in ONE cooperative launch per step.
    The launch shape (CTA split, rounds, WFS tile and P^T band height per
    geometry class) is chosen by the library's autotuner (autotune_batch);
    the timed steps replay a CUDA graph of the bound launch (fewha_batch_bind
    + fewha_batch_launch), each step's slopes copied into the bound buffers
    and L2 flushed before it, outside its events."""
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

    def step(b):
        t = frame[0]
        b.solve([x["s"][t] for x in inst], [x["c"] for x in inst], [x["st"] for x in inst],
                args.max_iter, rtol=args.rtol, augmented=not args.plain)
        frame[0] = (t + 1) % 4  # the autotuner reuses the first frames

    best, timings = autotune_batch(fewhas, step, reps=2)
    for x in inst:  # fresh states after tuning
        x["st"] = x["f"].new_state(args.k)
        x["c"].zero_()
    batch = FewhaBatch(fewhas, best["ctas"], best["rounds"], best["tiles"])
    bound_s = [torch.empty_like(x["s"][0]) for x in inst]
    stats = batch.bind(bound_s, [x["c"] for x in inst], [x["st"] for x in inst], args.max_iter, rtol=args.rtol,
                       augmented=not args.plain)

    def load(t):
        for x, b in zip(inst, bound_s):
            b.copy_(x["s"][t])

    for t in range(W):  # warm-up through the bound launch
        load(4 + t)
        batch.launch()
    graph = batch.capture_graph()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    its, ok = [], True
    for t in range(K):
        load(4 + W + t)
        if flush is not None:
            flush.zero_()
        ev[t][0].record()
        graph.replay()
        ev[t][1].record()
        rows = batch.read_stats(stats)  # synchronises, outside the events
        ok = ok and all(r["status"] == 0 for r in rows)
        its.append([r["iterations"] for r in rows])
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    its = np.array(its)
    algo = sum(workload.reference_solve_bytes(x["geom"], float(its[:, i].mean()), args.k, 4)
               for i, x in enumerate(inst))
    us_step = ms / K * 1e3
    peak, _ = measured_peaks()
    by_kind = {}
    for i, k in enumerate(kinds):
        by_kind.setdefault(k, {"ctas": best["ctas"][i], "round": best["rounds"][i] if best["rounds"] else 0,
                               "wfs_tile": list(best["tiles"][i]), "pt_band_rows": list(best["bands"][i])})
    out = {"instances": len(inst), "mix": "24 x tiny (8 m, 16x16, 4 NGS, 2 x 32^2) + 24 x medium (16 m, 40x40, "
           "4 LGS, 5 x 64^2) + 16 x ELT (39 m, 84x84, 6 LGS, 9 layers)", "steps": K, "warmup": W,
           "timed": "CUDA-graph replay of the bound batched launch", "us_per_step": us_step,
           "instance_frames_per_s": len(inst) * K / (ms / 1e3),
           "elt_instance_frames_per_s": 16 * K / (ms / 1e3),
           "elt_equivalent_frames_per_s": sum(x["f"].n for x in inst) / inst[-1]["f"].n * K / (ms / 1e3),
           "iterations_mean": float(its.mean()), "chosen": by_kind, "autotune_best_ms": best["ms"],
           "autotune_candidates": len(timings),
           "status_ok": ok, "roofline": {"bound": "hbm", "achieved": algo / (us_step * 1e-6) / 1e9,
                                         "peak": peak, "unit": "GB/s",
                                         "frac": algo / (us_step * 1e-6) / 1e9 / peak},
           "gpu_launches_per_step": 2}
    batch.close()
    for x in inst:
        x["f"].close()
    return out


def run_e2e(f, geom, frames, sdt, args, aug, flush):
    """Same metric through the public API with host buffers: every frame's
    slopes come from pinned host memory and its solution c goes back to pinned
    host memory inside the frame's timed window.  The solve kernel reads the
    slopes in place (fewha_solve accepts page-locked host slopes) and writes c
    into the host buffer at the end of the step (fewha_solve_opts.c_out), so
    the bytes cross the host link with no transfer on the stream.  L2 is
    flushed before every frame (outside the window), as for `value`."""
    import torch
    K = args.steps
    host = frames[args.warmup:args.warmup + K].to(sdt).cpu().pin_memory()
    warm = frames[:args.warmup].to(sdt).cpu().pin_memory()
    out_host = torch.empty((K, f.n), dtype=f.dtype).pin_memory()
    c = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    st = f.new_state(args.k)
    stats = f.new_stats()
    for t in range(args.warmup):
        f.solve(warm[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for t in range(K):
        if flush is not None:
            flush.zero_()
        ev[t][0].record()
        f.solve(host[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats, c_out=out_host[t])
        ev[t][1].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    esz = torch.tensor([], dtype=sdt).element_size()
    ok = bool(torch.equal(out_host[K - 1], c.cpu()))
    # the same frames again with copy-engine transfers on the stream (for
    # comparison): slopes copied into a device buffer, c copied back
    c2 = torch.zeros(f.n, dtype=f.dtype, device="cuda")
    st2 = f.new_state(args.k)
    dev_s = torch.empty(f.n_slopes, dtype=sdt, device="cuda")
    for t in range(args.warmup):
        dev_s.copy_(warm[t], non_blocking=True)
        f.solve(dev_s, c2, st2, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
    torch.cuda.synchronize()
    for t in range(K):
        if flush is not None:
            flush.zero_()
        ev[t][0].record()
        dev_s.copy_(host[t], non_blocking=True)
        f.solve(dev_s, c2, st2, args.max_iter, rtol=args.rtol, augmented=aug,
                persistent=args.launch == "persistent", stats=stats)
        out_host[t].copy_(c2, non_blocking=True)
        ev[t][1].record()
    torch.cuda.synchronize()
    ms_ce = sum(a.elapsed_time(b) for a, b in ev)
    ok = ok and bool(torch.equal(c2, c))  # the same solution either way
    return {"value": K / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": f.n_slopes * esz,
            "d2h_bytes_per_step": f.n * c.element_size(), "us_per_frame": ms / K * 1e3,
            "transfer": "slopes read by the solve kernel from pinned host memory; c written to pinned host "
                        "memory by the solve kernel (fewha_solve_opts.c_out)",
            "result_check": ok,
            "copy_engine": {"value": K / (ms_ce / 1e3), "us_per_frame": ms_ce / K * 1e3},
            "l2": "flushed before every frame (outside the timed window), as for value"}


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


def run_compare(geom, w, frames, args, stats_buf, flush, main):
    """Plain PCG against augmented PCG on the same frames and residual target,
    at the workload's SNR and at SNR 100 (where recycling saves iterations),
    plus the FP64 forms, the mixed-precision (BF16 storage) form and the
    residual replacement every 5 iterations.  `main` is the timed line's own
    (precision, augmented, us per frame, mean iterations)."""
    import copy
    import numpy as np
    import torch
    from paper_2011_06842_gb300 import Fewha
    K = min(args.steps, 60)
    sdts = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.bfloat16}

    def one(g, wts, fr, prec, aug, tre=0, rtol=None, nframes=None):
        f = Fewha(g, wts, prec, tile=args.tile, grid=args.grid)
        a = copy.copy(args)
        n = nframes or K
        if rtol is not None:
            a.max_iter = 1000  # the largest a solve takes (FEWHA_MAX_ITER)
        times, stats = time_solves(f, fr, sdts[prec], a, args.warmup, n, aug, flush, stats_buf,
                                   args.rtol if rtol is None else rtol, true_res_every=tre)
        f.close()
        it = [x["iterations"] for x in stats]
        return {"us_per_frame": sum(times) / n * 1e3, "frames_per_s": n / (sum(times) / 1e3),
                "iterations_mean": float(np.mean(it)), "frames": n,
                "status_ok": all(x["status"] == 0 for x in stats)}

    res = {}
    snr0 = "snr%g" % geom.snr
    res[snr0] = {}
    for prec, aug, tre in (("f32", False, 0), ("f32", True, 0), ("f32", True, 5), ("f64", False, 0),
                           ("f64", True, 0), ("bf16s", True, 0)):
        key = "%s_%s%s" % ("aug" if aug else "plain", prec, "_true_res5" if tre else "")
        if prec == main[0] and aug == main[1] and tre == 0:
            res[snr0][key] = {"us_per_frame": main[2], "iterations_mean": main[3], "frames": args.steps,
                              "note": "the timed line itself"}
            continue
        res[snr0][key] = one(geom, w, frames, prec, aug, tre)
    g100 = copy.deepcopy(geom)
    g100.snr = 100.0
    fr100, w100 = make_frames(g100, args.warmup + K, seed=200, device="cuda")
    res["snr100"] = {"plain_f32": one(g100, w100, fr100, "f32", False),
                     "aug_f32": one(g100, w100, fr100, "f32", True)}
    for snr, r in res.items():
        if "plain_f32" in r and "aug_f32" in r:
            r["aug_minus_plain_us"] = r["aug_f32"]["us_per_frame"] - r["plain_f32"]["us_per_frame"]
    # tighter residual targets (at most 1000 iterations a frame), plain against
    # augmented, FP32 and FP64, on the first frames of both sequences
    ns = min(K, 20)
    sweep = {}
    for rt in (1e-3, 1e-4):
        for tag, g, wts, fr in ((snr0, geom, w, frames), ("snr100", g100, w100, fr100)):
            r = {}
            for prec in ("f32", "f64"):
                for aug in (False, True):
                    r["%s_%s" % ("aug" if aug else "plain", prec)] = one(g, wts, fr, prec, aug, rtol=rt, nframes=ns)
            sweep["rtol %g, %s" % (rt, tag)] = r
    res["rtol_sweep"] = sweep
    return res


def _oracle_worker(job):
    """One host core: the FP64 oracle over the frames of one sequence
    (independent of the other workers); returns (frames timed, seconds)."""
    import time as _t
    geom_name, snr, k, w, invJ, s, warm, iters, rtol, max_iter, aug = job
    sys.path.insert(0, ROOT)
    from oracle import Oracle
    from synth import configs
    geom = configs.get(geom_name)
    geom.snr = snr
    o = Oracle(geom, w, with_precond=False)
    o.set_invJ(invJ)
    st = o.new_state(k)
    for t in range(warm):
        o.solve(s[t], st, max_iter=max_iter, rtol=rtol, augmented=aug)
    t0 = _t.perf_counter()
    for t, it in enumerate(iters):
        o.solve(s[warm + t], st, max_iter=it, rtol=0.0, augmented=aug)
    return len(iters), _t.perf_counter() - t0


def run_cpu_baseline(geom, w, frames, gpu_iters, args, aug):
    """The FP64 oracle as it stands on the same frames with the same per-frame
    iteration counts as the GPU frames: single-threaded, and on all host
    cores (one independent copy of the sequence per core, spawned processes:
    whole-machine frames/s = frames of all workers / the slowest worker's
    time)."""
    import multiprocessing as mp
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
    cores = os.cpu_count() or 1
    job = (args.config, geom.snr, args.k, np.asarray(w), o.invJ(), s, args.warmup, list(gpu_iters[:nf]),
           args.rtol, args.max_iter, aug)
    all_cores = None
    if cores > 1 and not args.no_cpu_all:
        with mp.get_context("spawn").Pool(cores) as pool:
            t1 = time.perf_counter()
            parts = pool.map(_oracle_worker, [job] * cores)
            wall = time.perf_counter() - t1
        all_cores = {"value": sum(p[0] for p in parts) / max(p[1] for p in parts), "unit": UNIT,
                     "cores": cores, "workers": cores, "pool_wall_s": wall}
    model = cpu_model()
    return {"value": nf / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": model, "nproc": cores,
            "sample": "%d ELT frames after %d warm-up frames, FP64, single-threaded, same iteration counts as "
                      "the GPU frames (mean %.2f)" % (nf, args.warmup, float(np.mean(gpu_iters[:nf]))),
            "all_cores": all_cores}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, single-threaded on a
    host core (rank 0 only), one full frame of the same workload per step."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from oracle import Oracle, build_oracle
    from synth import FrozenFlowSensors, configs
    build_oracle()
    geom = configs.get(args.config)
    if args.snr:
        geom.snr = args.snr
    geom.k_recycle = args.k
    # a bounded sample: at most 60 timed frames after at most 10 warm-up frames
    # (~10 s of one core on the ELT workload), whatever --steps asks for
    nwarm, nsteps = min(args.warmup, 10), min(args.steps, 60)
    sim = FrozenFlowSensors(geom, seed=100)
    s, w = sim.sequence_chunked(nwarm + nsteps, seed=101, dtype=torch_float64())
    s = s.numpy()
    o = Oracle(geom, w)
    st = o.new_state(args.k)
    aug = not args.plain
    for t in range(nwarm):
        o.solve(s[t], st, max_iter=args.max_iter, rtol=args.rtol, augmented=aug)
    t0 = time.perf_counter()
    its = []
    for t in range(nsteps):
        r = o.solve(s[nwarm + t], st, max_iter=args.max_iter, rtol=args.rtol, augmented=aug)
        its.append(r["iterations"])
    dt = time.perf_counter() - t0
    v = nsteps / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / nsteps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded von Karman frozen-flow screens (r0=%.3f m, L0=%.0f m, wind 5-20 m/s) "
                    "seen by SH sensors, SNR %g" % (geom.r0, geom.L0, geom.snr),
            "config": bench_config(geom, args, not args.no_flush),
            "iterations": {"mean": float(np.mean(its))},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": "%d full frames after %d warm-up frames (FP64 oracle, its own stopping "
                                       "test), single-threaded; the first %d of the %d steps asked for"
                                       % (nsteps, nwarm, nsteps, args.steps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_trace(args):
    """Per-phase trace of the persistent time step (fewha_set_trace) on the
    configuration, plain and augmented PCG: 20 warm-up frames, 10 untimed-trace
    frames timed with CUDA events (L2 flushed before each), then 5 traced frames;
    per phase tag the mean span (last CTA done minus CTA 0 leaving the previous
    barrier), barrier wait and longest single-CTA phase, in microseconds."""
    import collections
    import numpy as np
    import torch
    from paper_2011_06842_gb300 import Fewha, build
    from synth import configs
    build.build()
    torch.cuda.set_device(0)
    geom = configs.get(args.config)
    if args.snr:
        geom.snr = args.snr
    geom.k_recycle = args.k
    frames, w = make_frames(geom, 35, seed=101, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {"metric": "per-phase trace of one time step", "unit": "us",
           "config": bench_config(geom, args, True), "forms": {}}
    for aug in (False, True):
        f = Fewha(geom, w, args.precision)
        sdt = torch.bfloat16 if args.precision == "bf16s" else f.dtype
        sl = frames.to(sdt)
        st, c = f.new_state(args.k), torch.zeros(f.n, dtype=f.dtype, device="cuda")
        for t in range(20):
            f.solve(sl[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug)
        torch.cuda.synchronize()
        us, its = [], []
        for t in range(20, 30):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            stt = f.solve(sl[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug)
            b.record()
            torch.cuda.synchronize()
            us.append(a.elapsed_time(b) * 1e3)
            its.append(f.read_stats(stt)["iterations"])
        buf = torch.zeros((512, 4), dtype=torch.int64, device="cuda")
        f.set_trace(buf)
        agg = collections.defaultdict(list)
        for t in range(30, 35):
            flush.zero_()
            f.solve(sl[t], c, st, args.max_iter, rtol=args.rtol, augmented=aug)
            for tag, span, bar, mx in f.read_trace():
                agg[tag].append((span, bar, mx))
        f.set_trace(None)
        f.close()
        phases = {tag: {"n_per_frame": len(v) / 5.0, "span_us": float(np.mean([x[0] for x in v])) / 1e3,
                        "barrier_us": float(np.mean([x[1] for x in v])) / 1e3,
                        "max_cta_us": float(np.mean([x[2] for x in v])) / 1e3} for tag, v in agg.items()}
        out["forms"]["augmented" if aug else "plain"] = {"us_per_frame": float(np.mean(us)),
                                                          "iterations": float(np.mean(its)), "phases": phases}
    return out


def run_conv_layers(args):
    """Device time of every convolution launch of the learned predictor's
    forward pass on the configuration's layer groups (random activations and
    weights): the tcgen05 kernel against the FP32 kernel, 3 warm-up and
    args.steps (at most 50) timed launches each, in forward order."""
    import torch
    from paper_2011_06842_gb300 import build, learned
    from synth import configs
    build.build()
    geom = configs.get(args.config)
    net = learned.ConvNet(geom, seed=7)
    x = torch.randn(learned.CHANNELS[0], net.n, device="cuda")
    y = torch.empty(learned.N_DIR, net.n, device="cuda")
    reps = max(1, min(args.steps, 50))
    out = {"metric": "3x3 convolution launches of the learned predictor", "unit": "us", "config": {
        "workload": "%s layer groups %s, channels %s" % (geom.name, [(c, n) for _, c, n in net.groups],
                                                         list(learned.CHANNELS))}, "layers": []}
    for tc in (True, False):
        for name, flops, launch in net.convolutions(x.data_ptr(), net.n, y, tensor_cores=tc):
            for _ in range(3):
                assert launch() == 0, name
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(reps):
                launch()
            b.record()
            torch.cuda.synchronize()
            us = a.elapsed_time(b) * 1e3 / reps
            out["layers"].append({"conv": name, "kernel": "tcgen05" if tc else "fp32", "us": us,
                                  "tflops": flops / us * 1e-6})
        if tc:
            out["tc_status"] = int(net.tc_status.item())
    return out


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
            "network_forward_us": ev_us(lambda: lw.net.forward(lw.ring[4].data_ptr(), -f.n, y, tensor_cores=True)),
            "network_forward_fp32_us": ev_us(lambda: lw.net.forward(lw.ring[4].data_ptr(), -f.n, y)),
            "apply_multi5_us": ev_us(lambda: f.apply_op_multi(x, out=y)),
            "apply_single_us": ev_us(lambda: f.apply_op(x[0], out=y[1]))}
    out = {"metric": METRIC, "mode": "learned warm start", "unit": "frames/s",
           "value": 1e6 / res["learned"]["us"], "plain_value": 1e6 / res["plain"]["us"],
           "higher_is_better": True, "n_gpus": 1, "dtype": "f32",
           "data": "synthetic: seeded von Karman frozen-flow screens seen by SH sensors, SNR %g" % geom.snr,
           "config": {"workload": workload_name(geom, args) + ", learned warm start",
                      "rtol": args.rtol, "max_iter": args.max_iter, "k_recycle": args.k,
                      "network": "3x3 conv 4-32-32-5, ReLU; inference on tcgen05 (bfloat16 operands, FP32 "
                                 "accumulation), training on FP32 kernels", "train_frames": args.learned_train,
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
    if args.conv_layers:
        print(json.dumps(run_conv_layers(args)))
        return
    if args.trace:
        print(json.dumps(run_trace(args)))
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
