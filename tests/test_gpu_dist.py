"""The sharded sum on the GPU (dist.sharded_sum with zxp_eval per rank, the
partials all-gathered over NCCL), as one rank: this box has one GPU, so the
exchange runs with world size 1 here and the world-size 2 and 3 host logic is
covered on CPU (tests/test_dist.py).  The sharded value equals the oracle's
and the one-call amplitude exactly."""
import os
import socket

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi
from paper_2403_06777_gb300 import dist as zd

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def group():
    import torch
    import torch.distributed as dist
    assert torch.cuda.is_available(), "these tests need a GPU"
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    yield dist.group.WORLD
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def ctx():
    c = Z.zxp_ctx_create(0)
    yield c
    c.close()


def test_sharded_sum_of_circuit_amplitudes(group, ctx):
    w = zi.workload_medium(2)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    k = s.info["k"]
    got = zd.sharded_sum(lambda f, c: Z.zxp_eval(ctx, s, f, c), k, group)
    assert got == oracle.amp(w.gates, w.n, w.out_bits) == Z.zxp_amplitude(ctx, s)
    wl = zi.workload_large(0)
    sl = Z.zxp_compile(wl.gates, wl.n, wl.out_bits)
    assert zd.sharded_sum(lambda f, c: Z.zxp_eval(ctx, sl, f, c), sl.info["k"], group) == \
        Z.zxp_amplitude(ctx, sl)


def test_sharded_raw_partial_matches_the_oracle(group, ctx):
    ps = zi.synthetic_ps(77, 18, n_lin=12, n_quad=6, n_node=10, n_pair=2, density=0.25)
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    raw = zd.sharded_sum(lambda f, c: Z.zxp_eval(ctx, s, f, c), 18, group, canonical=False)
    o = oracle.ps_sum(blob, 0, 1 << 18, nthreads=NCPU)
    assert raw[4] == o[4] and all((raw[i] - o[i]) & ((1 << 64) - 1) == 0 for i in range(4))
