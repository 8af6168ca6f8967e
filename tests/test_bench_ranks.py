"""Host logic of bench.py under torchrun with N > 1, as two gloo ranks on the CPU:
max-over-ranks timing, the whole-job throughput, independent per-rank volumes
(weak scaling, no collective on the data path), and the reference arm printing
from rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 10 + 5 r ms; every rank must see the slowest
        ms_max = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
        value = bench.whole_job_rate(1e9, world, ms_max / 1e3)
        vol, phi0, _, _ = bench.make_workload("lightsheet512", rank, size=24, iters_override=2)
        digest = float(np.asarray(vol, dtype=np.float64).sum())
        # the reference arm: rank 0 prints one line, the others nothing
        args = type("A", (), dict(workload="tree64", bricks=None, size=None, iters=None, warmup=0, steps=1,
                                  force=None))()
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args, rank, world)
        dist.barrier()
        q.put((rank, ms_max, value, digest, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], f"rank exit codes {codes}"
    res = {}
    while not q.empty():
        r, ms_max, value, digest, out = q.get()
        res[r] = (ms_max, value, digest, out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        assert res[r][0] == pytest.approx(15.0)             # the slower rank's time on both
        assert res[r][1] == pytest.approx(2e9 / 15e-3 / 1e9)  # all ranks' units / max time
    assert res[0][2] != res[1][2], "ranks must evolve independent volumes"
    assert res[0][3].count("\n") == 1 and '"impl": "reference"' in res[0][3]
    assert res[1][3] == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(2e9, 1, 0.5) == pytest.approx(4.0)
