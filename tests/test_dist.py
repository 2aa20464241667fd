"""Range sharding across ranks (world size 2, gloo, CPU processes).

Each rank sums its share of the Gray-index range with the oracle (there is
no GPU here) and the partials are gathered and combined by the library's
host logic; the result must equal the unsharded value exactly."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import zxp_inputs as zi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, blob, k, q):
    import torch.distributed as dist
    import oracle
    from paper_2403_06777_gb300 import dist as zd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def eval_range(first, count):
            v = oracle.ps_sum(blob, first, count)
            return tuple(c & ((1 << 64) - 1) for c in v[:4]) + (v[4],)
        raw = zd.sharded_sum(eval_range, k, canonical=False)
        q.put((rank, raw))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_matches_whole(world):
    import oracle
    from paper_2403_06777_gb300 import dist as zd
    ps = zi.synthetic_ps(4, 11, n_lin=6, n_quad=4, n_node=10, n_pair=2, e0=5, G=(1, 2, 0, -1))
    blob = ps.pack()
    whole = oracle.ps_sum(blob)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, blob, 11, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, raw in got:
        assert raw[4] == whole[4]
        assert all((raw[i] - whole[i]) % (1 << 64) == 0 for i in range(4))


def test_shard_range_covers_everything_once():
    from paper_2403_06777_gb300 import dist as zd
    for k in range(0, 9):
        for world in range(1, 7):
            spans = [zd.shard_range(k, world, r) for r in range(world)]
            pos = 0
            for first, count in spans:
                assert first == pos
                pos += count
            assert pos == 1 << k
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        zd.shard_range(3, 2, 2)
