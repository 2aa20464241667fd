"""Weak simulation (chained marginals, every probability an exact parametric
evaluation on the device) and marginals by summing, against the oracle:
the drawn bitstrings and their exact probabilities are identical."""
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


@pytest.mark.parametrize("seed,n,g", [(0, 4, 40), (1, 5, 50), (2, 6, 60), (3, 8, 60)])
def test_samples_equal_the_oracle(ctx, seed, n, g):
    gates = zi.circuit_iid(900 + seed, n, g)
    rng = random.Random(seed)
    rows = [[rng.random() for _ in range(n)] for _ in range(64)]
    with Z.zxp_sampler_create(ctx, gates, n) as smp:
        ks = Z.zxp_sampler_info(smp)
        bits, probs = Z.zxp_sampler_draw(smp, rows)
    assert len(ks) == n and all(0 <= k <= 62 for k in ks)
    want_bits, want_probs = oracle.sample(gates, n, rows)
    assert bits == want_bits
    assert probs == want_probs


def test_samples_with_an_input_state(ctx):
    n = 5
    gates = zi.circuit_iid(77, n, 50)
    ib = [1, 0, 1, 1, 0]
    rng = random.Random(9)
    rows = [[rng.random() for _ in range(n)] for _ in range(32)]
    with Z.zxp_sampler_create(ctx, gates, n, in_bits=ib) as smp:
        bits, probs = Z.zxp_sampler_draw(smp, rows)
    assert (bits, probs) == oracle.sample(gates, n, rows, ib)


def test_marginal_by_sum_equals_doubled_diagram(ctx):
    rng = random.Random(2)
    for seed in range(6):
        n = 6
        gates = zi.circuit_iid(400 + seed, n, 60)
        mask = rng.randrange(1, 1 << n)
        bits = [rng.randrange(2) for _ in range(n)]
        got = Z.zxp_marginal_by_sum(ctx, gates, n, mask, bits)
        assert got == oracle.marginal(gates, n, mask, bits)
        s = Z.zxp_compile(gates, n, bits, marg_mask=mask, kind=Z.ZXP_MARGINAL_DOUBLED)
        assert got == Z.zxp_amplitude(ctx, s)
