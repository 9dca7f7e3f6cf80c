"""The benchmark's multi-rank host logic (one replica per rank, slowest rank
timed, whole-job throughput) on two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    t = bench.reduce_max(10.0 * (rank + 1), dist, "cpu")
    v = bench.job_mbps(1_000_000, 5, ws, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, ws, local, t, v))


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    for _, _, _, t, v in res:
        assert t == 20.0                                  # max over ranks
        assert v == pytest.approx(2 * 1_000_000 * 5 / 0.020 / 1e6)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    import bench
    import types
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(types.SimpleNamespace(steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def test_dominant_kernel_skips_side_stream_spans():
    """Event spans of the side-stream transforms (mh_b.*) include waiting for
    SMs; the dominant kernel is chosen among the other traced kernels."""
    import bench
    tr = {"mh_b.p3_row_store": (2, 900.0), "mmh.p3_fwd_col": (2, 600.0), "mmh.p3_row_mac": (2, 550.0)}
    assert bench.dominant_kernel(tr) == "mmh.p3_fwd_col"
