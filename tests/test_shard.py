"""View-sharded A^T (paper_2103_10329_gb300.shard): each rank back-projects
its own contiguous range of views and the partial volumes are summed over
the ranks in rank order.

CPU: two gloo ranks, with the FP64 oracle's A^T as the per-rank operator
(the host logic of the partition and the ordered sum), against the oracle
over all views.  GPU: two gloo ranks sharing cuda:0, each running the
library's A^T on its views (no kernel waits on another rank's), against one
process's A^T over all views, and bit for bit against the same two partial
volumes summed in rank order in one process."""
import os
import socket
import sys
from types import SimpleNamespace

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_view_range_partitions_every_view_once():
    from paper_2103_10329_gb300.shard import view_range
    for K in (1, 7, 90, 720, 2881):
        for world in (1, 2, 3, 8):
            got = [view_range(K, r, world) for r in range(world)]
            assert got[0][0] == 0
            for (a, n), (b, _) in zip(got, got[1:]):
                assert a + n == b
            assert got[-1][0] + got[-1][1] == K
            counts = [n for _, n in got]
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        view_range(10, 2, 2)


def _cpu_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2103_10329_gb300 import shard, synth
    from tests.helpers import oracle_scan, scan_desc
    d = scan_desc(16, 24, 24, 11, 2104)
    og = O.level_geometry(oracle_scan(d), 0)
    y = np.random.default_rng(3).standard_normal((11, 24, 24))
    v0, cnt = shard.view_range(11, rank, world)

    def bp(g, sino, level, views):
        a, c, _ = views
        return torch.from_numpy(O.backproject(og.subset(np.arange(a, a + c)), sino.numpy()))

    out = shard.backproject_sharded(SimpleNamespace(n_views=11), torch.from_numpy(y[v0:v0 + cnt]), rank, world,
                                    backproject=bp)
    q.put((rank, out.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_backprojection_two_gloo_ranks_cpu():
    sys.path.insert(0, ROOT)
    import oracle as O
    from tests.helpers import oracle_scan, scan_desc
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_cpu_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = scan_desc(16, 24, 24, 11, 2104)
    og = O.level_geometry(oracle_scan(d), 0)
    y = np.random.default_rng(3).standard_normal((11, 24, 24))
    full = O.backproject(og, y)
    parts = [O.backproject(og.subset(np.arange(a, a + c)), y[a:a + c])
             for a, c in ((0, 6), (6, 5))]
    np.testing.assert_array_equal(res[0], res[1])            # the same volume on every rank
    np.testing.assert_array_equal(res[0], parts[0] + parts[1])  # the rank-order sum, bit for bit
    assert np.abs(res[0] - full).max() <= 1e-12 * np.abs(full).max()


def _gpu_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2103_10329_gb300 import shard
    from tests.helpers import gpu_geom, scan_desc
    d = scan_desc(64, 96, 96, 90, 2104)
    g = gpu_geom(d)
    y = torch.rand((90, 96, 96), device="cuda", generator=torch.Generator("cuda").manual_seed(7)) - 0.3
    v0, cnt = shard.view_range(90, rank, world)
    out = shard.backproject_sharded(g, y[v0:v0 + cnt].contiguous(), rank, world)
    torch.cuda.synchronize()
    q.put((rank, out.cpu().numpy()))
    dist.barrier()
    dist.destroy_process_group()
    g.close()


@pytest.mark.gpu
def test_sharded_backprojection_two_gloo_ranks_gpu():
    from paper_2103_10329_gb300 import build, mgct
    from tests.helpers import TOL_F32, gpu_geom, scan_desc
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    d = scan_desc(64, 96, 96, 90, 2104)
    g = gpu_geom(d)
    y = torch.rand((90, 96, 96), device="cuda", generator=torch.Generator("cuda").manual_seed(7)) - 0.3
    full = mgct.backproject(g, y).cpu().numpy().astype(np.float64)
    absf = mgct.backproject(g, y.abs()).cpu().numpy().astype(np.float64)
    p0 = mgct.backproject(g, y[:45].contiguous(), views=(0, 45, 1))
    p1 = mgct.backproject(g, y[45:].contiguous(), views=(45, 45, 1))
    mgct.axpy(1.0, p1, p0)
    ordered = p0.cpu().numpy()
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], ordered)
    e = np.abs(res[0] - full) / np.maximum(absf, 1e-2 * absf.max())
    assert e.max() <= TOL_F32, e.max()
