"""The multi-GPU path of bench.py runs independent replicas (the method's
patches need no exchange between replicas): two gloo ranks on the CPU
check the slowest-rank timing, the whole-job rate, and that replicas given
the same seeded input compute the same result with no data exchanged."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import oracle as O
    import synth as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        # each replica advances its own copy of a small acoustics grid
        grid = S.UniformGrid(S.Layout(8, 3), 2, 2)
        st = np.nan_to_num(grid.state(S.pulse_plus_vortex(), nq=2))
        res = O.run_uniform(O.cfg(O.ACOUSTICS, 8, grid.dx, grid.dy, 0.4 * grid.dx), 2, 2, 2, st, nthreads=1)
        mine = torch.tensor([float(np.abs(res).sum())], dtype=torch.float64)
        allv = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allv, mine)
        out.put((rank, ms, bench.job_rate(1000.0, world, ms), [float(v.item()) for v in allv]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, sums in got:
        assert ms == 2.5                       # the slower rank's time
        assert rate == pytest.approx(2 * 1000.0 / 2.5e-3)
        assert sums[0] == sums[1]              # identical replicas
