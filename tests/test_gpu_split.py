"""Scalars with inner parameters on the GPU, through the C ABI.

The inner table (the Walsh-Hadamard transform of the inner rows' product,
built on the device) and the outer walk that multiplies each run of terms by
it are compared with the oracle, which sums every inner value of every term
on its own; raw partials agree modulo 2^64, amplitudes exactly."""
import os
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1
NCPU = os.cpu_count() or 4
INV = {zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "these tests need a GPU"
    c = Z.zxp_ctx_create(0)
    yield c
    c.close()


def same_raw(gpu, orc):
    assert gpu[4] == orc[4]
    return all((gpu[i] - orc[i]) & M64 == 0 for i in range(4))


def ranges(n, rng):
    r = [(0, n), (0, 0), (n, 0), (n - 1, 1), (0, 1)]
    if n > 8:
        r += [(1, n - 3), (n // 3, n // 2)]
        a = rng.randrange(n)
        r.append((a, rng.randrange(n - a + 1)))
    return r


@pytest.mark.parametrize("seed,k,n_node,n_pair,odd", [
    (1, 14, 3, 0, True),     # lane-private 32-bit counters
    (2, 16, 10, 0, True),    # lane-private 16-bit counters
    (3, 18, 20, 0, True),    # table path (more outer nodes than the counters hold)
    (4, 16, 6, 1, False),    # folded phase-pair and zero bits
    (5, 17, 8, 4, False),    # general: Z[w] phase-pair products
    (6, 20, 12, 2, False),
    (7, 12, 0, 0, False),    # no nodes at all
    (8, 14, 4, 8, False),    # many phase-pairs: general layout outside
])
def test_split_synthetic_ranges(ctx, seed, k, n_node, n_pair, odd):
    rng = random.Random(seed)
    ps = zi.synthetic_ps(700 + seed, k, n_lin=rng.randint(8, 20), n_quad=rng.randint(2, 10),
                         n_node=n_node, n_pair=n_pair, odd_nodes_only=odd, density=0.2,
                         e0=rng.randint(0, 6), G=(rng.randint(-5, 5), 1, rng.randint(-5, 5), 0))
    base = Z.zxp_scalar_from_tables(ps.pack())
    s = Z.zxp_scalar_split(base, min_k=6, max_inner=min(10, k - 6), low_free=4, max_cut=4, seed=seed)
    info = s.info
    assert info["k_inner"] > 0, info
    blob = Z.zxp_scalar_to_tables(s)
    for first, count in ranges(1 << info["k"], rng):
        g = Z.zxp_eval(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert same_raw(g, o), (info, first, count, g, o)
    # the same value as the scalar before the split, on the GPU
    assert Z.zxp_amplitude(ctx, s)[:5] == Z.zxp_zomega_canon(Z.zxp_eval(ctx, base))


@pytest.mark.parametrize("seed", range(4))
def test_split_medium_amplitudes_equal_the_state_vector(ctx, seed):
    # n = 20, 600 gates, t = 40, split by force: the whole sum on the GPU
    # equals the exact 2^20-entry state vector
    w = zi.workload_medium(seed)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=dict(min_k=8, max_inner=12, low_free=5, seed=seed + 1))
    assert s.info["k_inner"] > 0
    assert Z.zxp_amplitude(ctx, s) == oracle.amp(w.gates, w.n, w.out_bits)


def test_inner_table_recomputed(ctx):
    w = zi.workload_medium(1)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=dict(min_k=8, max_inner=10, low_free=4))
    a = Z.zxp_amplitude(ctx, s)
    Z.zxp_inner_sum(ctx, s)
    Z.zxp_inner_sum(ctx, s)
    assert Z.zxp_amplitude(ctx, s) == a == oracle.amp(w.gates, w.n, w.out_bits)


def test_large_workload_split_sampled_terms(ctx):
    # n = 50, 2000 gates, t = 80: the compiled scalar is split by default;
    # sampled outer terms (each the sum of 2^k_inner inner terms, from inner
    # table entries all over the table: every 32 MB chunk it is built in) and
    # ragged ranges equal the oracle
    w = zi.workload_large(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    info = s.info
    assert info["k_inner"] >= 16 and info["k"] <= 36, info
    blob = Z.zxp_scalar_to_tables(s)
    n = 1 << info["k"]
    rng = zi.SplitMix64(80)
    samples = [(0, 1), (n - 1, 1)] + [(rng.below(n - 4), 1 + rng.below(3)) for _ in range(12)]
    for first, count in samples:
        g = Z.zxp_eval(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert same_raw(g, o), (first, count)


def test_large_workload_full_sum_chunks_and_conjugate_transpose(ctx):
    """The full n = 50, 2000-gate, t = 80 amplitude: one launch equals the
    sum of eight launches over parts of the outer range, and <out|C|0>
    equals the conjugate of <0|C^dag|out> from the separately reduced and
    split inverse circuit (no state vector exists at n = 50)."""
    w = zi.workload_large(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    k = s.info["k"]
    a = Z.zxp_amplitude(ctx, s)
    n8 = (1 << k) // 8
    tot = Z.zxp_eval(ctx, s, 0, n8)
    for i in range(1, 8):
        tot = Z.zxp_zomega_add(tot, Z.zxp_eval(ctx, s, i * n8, n8))
    assert Z.zxp_zomega_canon(tot) == a
    dag = [(INV.get(op, op), q0, q1) for op, q0, q1 in reversed(w.gates)]
    sd = Z.zxp_compile(dag, w.n, [0] * w.n, in_bits=w.out_bits)
    assert sd.info["k_inner"] > 0
    b = Z.zxp_zomega_canon(Z.zxp_eval(ctx, sd))
    assert a == (b[0], -b[3], -b[2], -b[1], b[4])
    assert a != (0, 0, 0, 0, 0)


def test_split_scalar_limits(ctx):
    w = zi.workload_medium(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=dict(min_k=8, max_inner=10, low_free=4))
    assert s.info["k_inner"] > 0
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_batch_create(ctx, [s])
    assert e.value.code == Z.ZXP_EINVAL
    import torch
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_eval_noalloc(s, 0, 1, out.data_ptr())
    assert e.value.code == Z.ZXP_ETOOBIG
    with pytest.raises(Z.ZxpError):
        Z.zxp_scalar_split(s)             # already split
    with pytest.raises(Z.ZxpError):
        Z.zxp_eval(ctx, s, 0, (1 << s.info["k"]) + 1)
