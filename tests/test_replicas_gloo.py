"""The benchmark's multi-GPU path (independent replicas, no data-path collective) on CPU:
two gloo ranks with different local step times; the reported step time is the slowest
rank's and the whole-job value counts both ranks' cells."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t_ms, value = bench.whole_job(10.0 + 5.0 * rank, 1000000, ws, device="cpu")
        out[rank] = (t_ms, value)
    finally:
        torch.distributed.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(2):
        t_ms, value = res[r]
        assert t_ms == 15.0                           # max over ranks
        assert abs(value - 2 * 1000000 / 0.015 / 1e9) < 1e-12
