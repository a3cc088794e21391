"""Multi-GPU measurement path on CPU: N independent replicas, the timed
region's maximum over ranks and the whole-job rate, with two gloo ranks (no
GPU; the same functions run under torchrun with NCCL on GPUs)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")  # rank r took 10 + 5 r ms
    out[rank] = (t, bench.whole_job_rate(20, ws, t))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert abs(res[0][1] - 2 * 20 / 0.015) < 1e-9


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.whole_job_rate(10, 1, 5.0) == 2000.0


def _replica(rank, ws, port, out):
    """One replica of the multi-GPU measurement, with the FP64 oracle standing
    in for the device solve: its own seeded frames (seed 100 + rank, as
    bench.run_ours draws them), a timed sequence of time steps, then the
    job-level maximum and rate."""
    import time
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from oracle import Oracle
    from synth import configs
    geom = configs.get("tiny")
    frames, w = bench.make_frames(geom, 3, seed=100 + rank, device="cpu")
    o = Oracle(geom, w.numpy() if hasattr(w, "numpy") else w)
    st = o.new_state(4)
    dist.barrier()
    t0 = time.perf_counter()
    its = [o.solve(frames[t].numpy(), st, max_iter=50, rtol=1e-2, augmented=True)["iterations"] for t in range(3)]
    ms = (time.perf_counter() - t0) * 1e3
    t = bench.max_over_ranks(ms, ws, "cpu")
    out[rank] = (ms, t, bench.whole_job_rate(3, ws, t), np.asarray(st["c"]).copy(), its)
    dist.destroy_process_group()


def test_two_replicas_solve_their_own_sequences():
    """Replicas only: each rank solves its own seeded sequence with no data
    exchange; the job time is the slowest rank's and the rate counts the
    frames of both ranks."""
    import numpy as np
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_replica, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    (ms0, t0, rate0, c0, it0), (ms1, t1, rate1, c1, it1) = res[0], res[1]
    assert t0 == t1 == max(ms0, ms1)
    assert rate0 == rate1 == 2 * 3 / (t0 / 1e3)
    assert all(i > 0 for i in it0 + it1)
    assert np.linalg.norm(c0 - c1) > 1e-3 * np.linalg.norm(c0)  # different problems, no shared state
