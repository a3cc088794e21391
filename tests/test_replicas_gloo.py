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
