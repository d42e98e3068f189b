"""The N > 1 bench path on CPU: two gloo ranks as processes on 127.0.0.1.

The bench runs one replica of the solve per GPU (the method has no exchange
step between independent problems); its host side reduces the per-rank step
time to the slowest rank and reports weak scaling.  These tests run that
host logic with world_size 2, no GPU.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        fields = bench.replica_line_fields(times[rank], world)
        out[rank] = (fields["value"], fields["n_gpus"], fields["scaling"], fields["solves_per_s"])
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def _run(world, times):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    assert codes == [0] * world, codes
    return dict(out)


def test_two_replicas_report_the_slowest_rank():
    out = _run(2, [1.25, 2.5])
    for rank in range(2):
        value, n, scaling, sps = out[rank]
        assert value == 2.5
        assert n == 2
        assert scaling == "weak"
        assert sps == pytest.approx(2 / 2.5)


def test_single_rank_needs_no_process_group():
    import bench
    f = bench.replica_line_fields(3.0, 1)
    assert f == {"value": 3.0, "n_gpus": 1, "scaling": "weak", "solves_per_s": 1 / 3.0}
