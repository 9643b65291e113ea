"""bench.py's multi-GPU host logic on CPU with two gloo ranks: cases are sharded by rank (rank k steps the
recipe's cases k * cases .. (k + 1) * cases - 1, so no two ranks step the same case and one rank's shard equals
the single-process run's first cases), the job's time is the slowest rank's (a max all-reduce), the value is
all ranks' case-steps over that time, and the reference arm runs on rank 0 only.  No data-path collective
exists: the ranks' cases are independent."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import io
    import contextlib
    import torch
    import bench
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_env()
    ms = (12.0, 15.0)[r]                      # this rank's timed region
    t_max = bench.max_over_ranks(ms, w, "cpu")
    args = bench.parse(["--config", "medium", "--dims", "8,8,4", "--cases", "4"])
    mesh, tp = bench.make_mesh(args.config, args.dims)
    srcs = bench.make_sources(args.config, mesh, args.cases, first_case=bench.rank_first_case(r, args.cases))
    printed = io.StringIO()
    if r != 0:                                 # the reference arm: nothing to do and nothing printed off rank 0
        with contextlib.redirect_stdout(printed):
            bench.run_reference(args)
    torch.distributed.barrier()
    q.put((r, t_max, bench.job_value(w, args.cases, 10, t_max), [(s.node, s.f0) for s in srcs], printed.getvalue()))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_shard_cases_and_time_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, t_max, value, srcs, printed = q.get(timeout=300)
        res[r] = (t_max, value, srcs, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 15.0                    # both ranks hold the slowest rank's time
    assert res[0][1] == res[1][1] == pytest.approx(2 * 4 * 10 / 0.015)
    assert res[1][3] == ""                                     # rank 1 printed nothing for the reference arm
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse(["--config", "medium", "--dims", "8,8,4", "--cases", "8"])
    mesh, _ = bench.make_mesh(args.config, args.dims)
    single = [(s.node, s.f0) for s in bench.make_sources(args.config, mesh, 8)]
    assert res[0][2] == single[:4] and res[1][2] == single[4:]   # the two shards are the one-process cases
    assert not set(res[0][2]) & set(res[1][2])
