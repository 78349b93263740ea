"""The benchmark's multi-rank path on CPU (gloo, world size 2): replicas share no data-path
collective; rank 0 reports all ranks' units over the slowest rank's time; a rank that
never joins makes the others fail with an error instead of hanging."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out, mode):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), PRS_BENCH_GLOO="1", PRS_BENCH_TIMEOUT_S="8")
    import bench

    if mode == "absent" and rank == 1:
        return  # never joins the group
    try:
        w, r, _ = bench.dist_setup(world)
        secs = [1.5, 2.0][r]
        smax = bench.allreduce_max(secs, w, "cpu")
        bench.barrier(w)
        out[r] = bench.aggregate(10 ** 6, w, smax)
        import torch.distributed as dist

        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        out[rank] = f"error: {type(e).__name__}"


def _run(mode):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out, mode)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
        return dict(out)


def test_two_replicas_report_the_slowest_rank():
    out = _run("both")
    assert out[0] == pytest.approx(2 * 10 ** 6 / 2.0)
    assert out[1] == out[0]


def test_absent_rank_is_detected():
    out = _run("absent")
    assert isinstance(out.get(0), str) and out[0].startswith("error")
