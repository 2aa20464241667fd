"""zxp_scalar_reorder (host, no GPU): relabelling a scalar's parameters.

The relabelled scalar has the same rows with their masks' bits permuted by
one permutation of the parameters (checked here: the columns of the masks
are the same multiset), so every full sum is unchanged: the oracle sums both
exactly.  A new order is kept only when its plan has the better block lookup
(else the scalar comes back as it is); for scalars with the statistics of
compiled k ~ 36-40 scalars that is what lets the block lookup apply."""
import os

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

NCPU = os.cpu_count() or 4


@pytest.mark.parametrize("seed,k,n_pair", [(1, 10, 0), (2, 12, 2), (3, 9, 1), (4, 3, 0), (5, 14, 3)])
def test_reorder_is_a_relabelling_with_the_same_sum(seed, k, n_pair):
    ps = zi.synthetic_ps(4100 + seed, k, n_lin=12, n_quad=6, n_node=8, n_pair=n_pair, density=0.3,
                         e0=3, G=(2, -1, 0, 1))
    s = Z.zxp_scalar_from_tables(ps.pack())
    r = Z.zxp_scalar_reorder(s)
    q = zi.PSTables.unpack(Z.zxp_scalar_to_tables(r))
    assert (q.k, q.e0, q.G, len(q.lin), len(q.quad), len(q.node), len(q.pair)) == \
        (ps.k, ps.e0, ps.G, len(ps.lin), len(ps.quad), len(ps.node), len(ps.pair))
    # one permutation maps every row's mask bits: new bit j <- old bit perm[j]
    cols_old = {i: tuple((m >> i) & 1 for m, _ in ps.lin) + tuple((m >> i) & 1 for m, _ in ps.node)
                for i in range(k)}
    cols_new = {j: tuple((m >> j) & 1 for m, _ in q.lin) + tuple((m >> j) & 1 for m, _ in q.node)
                for j in range(k)}
    assert sorted(cols_old.values()) == sorted(cols_new.values())
    assert [c for _, c in q.lin] == [c for _, c in ps.lin] and [g for _, g in q.node] == [g for _, g in ps.node]
    # unchanged, or a better block lookup (variants 9-15 over none; one
    # table, 9-11, over two, 13)
    def rank(v):
        return 1 if v < 9 else (2 if v == 13 else 3)
    if q.pack() != ps.pack():
        assert rank(r.info["kernel_variant"]) > rank(s.info["kernel_variant"])
    # the same value (brute force over all 2^k assignments, both orders)
    a = oracle.ps_sum(ps.pack(), 0, 1 << k, nthreads=NCPU)
    b = oracle.ps_sum(q.pack(), 0, 1 << k, nthreads=NCPU)
    assert a[:5] == b[:5]


def test_reorder_enables_the_block_lookup_on_compiled_like_scalars():
    """Synthetic k = 36 scalars with the statistics of compiled k ~ 36-40
    scalars (48 linear, 36 quadratic, 10 odd node rows, mask density 0.13):
    in their drawn order most miss the block lookup (too many forms on
    parameters 0-2); relabelled, all of them take it (variant 9)."""
    before, after = [], []
    for seed in range(3600, 3610):
        ps = zi.synthetic_ps(seed, 36, n_lin=48, n_quad=36, n_node=10, odd_nodes_only=True, density=0.13)
        s = Z.zxp_scalar_from_tables(ps.pack())
        before.append(s.info["kernel_variant"])
        after.append(Z.zxp_scalar_reorder(s).info["kernel_variant"])
    assert sum(v >= 9 for v in before) <= 3
    assert all(v >= 9 for v in after), after


def test_reorder_rejects_split_scalars():
    w = zi.workload_medium(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=dict(min_k=8, max_inner=10, low_free=4))
    assert s.info["k_inner"] > 0
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_scalar_reorder(s)
    assert e.value.code == Z.ZXP_EINVAL
