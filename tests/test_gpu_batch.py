"""Batched evaluation (one persistent launch per kernel variant, work-stealing
chunk queue, tuned launch shape, CUDA graph replay) against per-scalar
evaluation and the oracle: exact."""
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "these tests need a GPU"
    c = Z.zxp_ctx_create(0)
    yield c
    c.close()


def mixed_scalars():
    rng = random.Random(7)
    out = []
    for seed in range(40):                           # compiled: k from 0 up
        w = zi.workload_batch_item(seed)
        out.append(Z.zxp_compile(w.gates, w.n, w.out_bits))
    for i in range(24):                              # every kernel variant
        kind = i % 6
        k = rng.choice([0, 3, 9, 14, 18, 21])
        kw = [dict(n_node=3, odd_nodes_only=True), dict(n_node=9, odd_nodes_only=True),
              dict(n_node=40, odd_nodes_only=True), dict(n_node=12, n_pair=2),
              dict(n_node=10), dict(n_node=70, n_lin=70, odd_nodes_only=True)][kind]
        ps = zi.synthetic_ps(100 + i, k, n_quad=5, density=0.25, **({"n_lin": 20} | kw))
        out.append(Z.zxp_scalar_from_tables(ps.pack()))
    return out


def test_batch_equals_individual_sums(ctx):
    scalars = mixed_scalars()
    b = Z.zxp_batch_create(ctx, scalars)
    info = Z.zxp_batch_info(b)
    assert info["n_scalars"] == len(scalars) and info["candidates"] >= 2
    assert info["threads"] in (128, 256) and 12 <= info["chunk_log2"] <= 20
    want = [Z.zxp_eval(ctx, s) for s in scalars]
    for _ in range(2):                               # graph replay, twice
        assert Z.zxp_batch_run(b) == want
    b.close()


def test_batch_amplitudes_match_statevector(ctx):
    items = [zi.workload_batch_item(s) for s in range(200)]
    small = [w for w in items if w.n <= 14][:4]
    assert small
    scalars = [Z.zxp_compile(w.gates, w.n, w.out_bits) for w in small]
    b = Z.zxp_batch_create(ctx, scalars)
    for w, raw in zip(small, Z.zxp_batch_run(b)):
        assert Z.zxp_zomega_canon(raw) == oracle.amp(w.gates, w.n, w.out_bits)


def test_batch_of_one_large_scalar_matches_oracle_subrange(ctx):
    ps = zi.synthetic_ps(3, 20, n_lin=20, n_quad=8, n_node=6, odd_nodes_only=True)
    s = Z.zxp_scalar_from_tables(ps.pack())
    b = Z.zxp_batch_create(ctx, [s])
    raw = Z.zxp_batch_run(b)[0]
    o = oracle.ps_sum(ps.pack(), nthreads=8)
    assert raw[4] == o[4] and all((raw[i] - o[i]) % (1 << 64) == 0 for i in range(4))
