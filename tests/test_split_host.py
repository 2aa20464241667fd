"""zxp_scalar_split on the host (no GPU).

The split rewrites a scalar in new variables with part of them summed inside
every term; its value must not change (the oracle sums both forms, the split
one every inner value of every outer term), and the partition it keeps is
the one of least estimated device time among those it builds and plans."""
import os
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

NCPU = os.cpu_count() or 4


@pytest.mark.parametrize("seed", range(6))
def test_split_keeps_the_value(seed):
    rng = random.Random(seed)
    k = rng.randint(12, 16)
    ps = zi.synthetic_ps(8100 + seed, k, n_lin=rng.randint(6, 14), n_quad=rng.randint(2, 8),
                         n_node=rng.choice([3, 5, 8]), n_pair=rng.choice([0, 1]),
                         odd_nodes_only=rng.random() < 0.5, density=rng.choice([0.15, 0.25]))
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    sp = Z.zxp_scalar_split(s, min_k=8, max_inner=min(8, k - 6), low_free=4, max_cut=3, seed=seed + 1)
    info = sp.info
    assert info["k_inner"] > 0 and info["k"] + info["k_inner"] == k
    whole = oracle.ps_sum(blob, 0, 1 << k, nthreads=NCPU)
    split = oracle.ps_sum(Z.zxp_scalar_to_tables(sp), 0, 1 << info["k"], nthreads=NCPU)
    assert Z.zxp_zomega_canon(split) == Z.zxp_zomega_canon(whole)


@pytest.mark.parametrize("seed", [0, 2, 3])
def test_large_workloads_split_for_the_block_lookup(seed):
    """n = 50, 2000 gates, T = 80 (k 51-55 before the split): every kept
    split walks its outer parameters with the lane-private block lookup
    (variants 14/15) and stays within the index limit; for seed 0 the
    estimated costs pick 21 inner parameters over a 2^22-entry table (one
    cut bit) and 30 outer ones, the balance measured best on GB300."""
    w = zi.workload_large(seed)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    info = s.info
    assert info["kernel_variant"] in (14, 15), info
    assert info["inner_bits"] <= 24 and info["k"] <= 34, info
    if seed == 0:
        assert (info["k"], info["k_inner"], info["inner_bits"]) == (30, 21, 22), info


@pytest.mark.parametrize("max_inner,max_bits", [(10, 12), (16, 18), (22, 24)])
def test_split_honours_its_limits(max_inner, max_bits):
    """Whatever the cost estimates prefer, the kept split stays within the
    limits asked for: inner parameters and index bits (inner parameters and
    crossing forms)."""
    w = zi.workload_large(0)
    base = Z.zxp_compile(w.gates, w.n, w.out_bits, split=False)
    sp = Z.zxp_scalar_split(base, max_inner=max_inner, max_index_bits=max_bits)
    info = sp.info
    assert 0 < info["k_inner"] <= max_inner and info["inner_bits"] <= max_bits, info
    assert info["k"] + info["k_inner"] == base.info["k"]
