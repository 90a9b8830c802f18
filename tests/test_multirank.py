"""N > 1 host path on CPU: world_size-2 gloo ranks (no GPU needed)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2412_09775_gb300.shard import job_throughput, tile_range


def test_tile_range_partitions_the_grid():
    for n in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            spans = [tile_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        tile_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2412_09775_gb300.shard import max_over_ranks
    ms = [3.0, 5.0][rank]
    mx = max_over_ranks(ms)
    dist.barrier()
    out[rank] = (mx, tile_range(256, rank, world))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == 5.0 and out[1][0] == 5.0
    assert out[0][1] == (0, 128) and out[1][1] == (128, 256)
    # whole-job value: both ranks' units over the slowest rank's time
    assert job_throughput(1e6, 2, 5.0) == pytest.approx(4e8)
