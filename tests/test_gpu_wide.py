"""Sums modulo 2^128 on the GPU (zxp_eval_wide, zxp_amplitude_wide and
zxp_amplitude for 124 < e0 <= 252), through the C ABI.

The oracle sums in checked 128-bit integers (oracle.ps_sum raises when a
value leaves that range), so every raw partial here is compared exactly.
The synthetic scalars carry constants near 2^60, so that their sums leave
the 64-bit range the 64-bit kernels cover: each test asserts that it does.
"""
import os

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4
M64 = (1 << 64) - 1
INV = {zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "these tests need a GPU"
    c = Z.zxp_ctx_create(0)
    yield c
    c.close()


BIG_G = ((1 << 60) + 12345, -(1 << 59) + 7, 3 << 57, -((1 << 61) - 99))


def big(v):
    return max(abs(x) for x in v[:4]) >= 1 << 63


def ranges(n):
    r = [(0, n), (0, 0), (n - 1, 1), (1, n - 3), (n // 3, n // 2 + 5)]
    return [(a, c) for a, c in r if a + c <= n]


@pytest.mark.parametrize("seed,k,n_node,n_pair,odd,e0", [
    (1, 12, 10, 0, True, 130),     # table layout (odd nodes only)
    (2, 14, 12, 1, False, 200),    # folded phase-pair and zero bits
    (3, 13, 8, 4, False, 252),     # general: Z[w] phase-pair products
    (4, 15, 20, 0, False, 140),    # zero forms, many nodes
    (5, 10, 0, 0, False, 125),     # no nodes
])
def test_wide_sum_matches_oracle(ctx, seed, k, n_node, n_pair, odd, e0):
    ps = zi.synthetic_ps(900 + seed, k, n_lin=9, n_quad=5, n_node=n_node, n_pair=n_pair,
                         odd_nodes_only=odd, density=0.25, e0=e0, G=BIG_G)
    s = Z.zxp_scalar_from_tables(ps.pack())
    blob = ps.pack()
    n = 1 << k
    whole = oracle.ps_sum(blob, 0, n, nthreads=NCPU)
    assert big(whole), whole
    for first, count in ranges(n):
        g = Z.zxp_eval_wide(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert g == tuple(o[:5]), (first, count, g, o)
        # the 64-bit sum is the same value modulo 2^64
        n64 = Z.zxp_eval(ctx, s, first, count)
        assert all((n64[i] - o[i]) & M64 == 0 for i in range(4))
    can = oracle.canon(whole[:4], whole[4])
    assert Z.zxp_amplitude_wide(ctx, s) == tuple(can)
    fits = all(-(1 << 63) <= x < (1 << 63) for x in can[:4])
    if fits:
        assert Z.zxp_amplitude(ctx, s) == tuple(can)
    else:
        with pytest.raises(Z.ZxpError) as e:
            Z.zxp_amplitude(ctx, s)
        assert e.value.code == Z.ZXP_EOVERFLOW


@pytest.mark.parametrize("seed,k,ki,n_node,n_pair,odd", [
    (1, 16, 6, 6, 0, True),
    (2, 18, 8, 10, 2, False),
    (3, 17, 7, 8, 4, False),
])
def test_wide_split_sum_matches_oracle(ctx, seed, k, ki, n_node, n_pair, odd):
    ps = zi.synthetic_ps(950 + seed, k, n_lin=10, n_quad=6, n_node=n_node, n_pair=n_pair,
                         odd_nodes_only=odd, density=0.2, e0=180, G=BIG_G)
    base = Z.zxp_scalar_from_tables(ps.pack())
    s = Z.zxp_scalar_split(base, min_k=6, max_inner=ki, low_free=4, max_cut=4, seed=seed)
    info = s.info
    assert info["k_inner"] > 0, info
    blob = Z.zxp_scalar_to_tables(s)
    n = 1 << info["k"]
    whole = oracle.ps_sum(blob, 0, n, nthreads=NCPU)
    assert big(whole), whole
    for first, count in ranges(n):
        g = Z.zxp_eval_wide(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert g == tuple(o[:5]), (info, first, count, g, o)
    # the split scalar and the scalar before the split: one value
    assert Z.zxp_amplitude_wide(ctx, s) == Z.zxp_amplitude_wide(ctx, base) == \
        tuple(oracle.canon(whole[:4], whole[4]))


def test_wide_small_values_fit_and_overflow_boundary(ctx):
    """e0 = 252 is summed exactly; e0 = 253 is beyond the 128-bit bound
    (ZXP_EOVERFLOW from both entry points), whatever the value."""
    for e0, ok in ((200, True), (252, True), (253, False)):
        ps = zi.synthetic_ps(990, 12, n_lin=8, n_quad=4, n_node=6, e0=e0, G=(3, -1, 0, 2))
        s = Z.zxp_scalar_from_tables(ps.pack())
        blob = ps.pack()
        whole = oracle.ps_sum(blob, 0, 1 << 12, nthreads=NCPU)
        can = tuple(oracle.canon(whole[:4], whole[4]))
        assert Z.zxp_scalar_info(s)["acc_bits"] == (128 if ok else 0)
        if ok:
            assert Z.zxp_amplitude(ctx, s) == can
            assert Z.zxp_amplitude_wide(ctx, s) == can
        else:
            for f in (Z.zxp_amplitude, Z.zxp_amplitude_wide):
                with pytest.raises(Z.ZxpError) as e:
                    f(ctx, s)
                assert e.value.code == Z.ZXP_EOVERFLOW


def test_inverse_circuit_amplitude_wide_is_the_conjugate(ctx):
    """<0|C^dag|out> of the n = 50, 2000-gate, T = 80 circuit has e0 = 127:
    zxp_amplitude sums it modulo 2^128 (31 outer + 21 inner parameters) and
    must give the conjugate of <out|C|0>, which the 64-bit path sums."""
    w = zi.workload_large(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    assert s.info["e0"] <= 124
    a = Z.zxp_amplitude(ctx, s)
    dag = [(INV.get(op, op), q0, q1) for op, q0, q1 in reversed(w.gates)]
    sd = Z.zxp_compile(dag, w.n, [0] * w.n, in_bits=w.out_bits)
    info = sd.info
    assert 124 < info["e0"] <= 252 and info["acc_bits"] == 128 and info["k_inner"] > 0, info
    b = Z.zxp_amplitude(ctx, sd)
    assert a == (b[0], -b[3], -b[2], -b[1], b[4])
    assert Z.zxp_amplitude_wide(ctx, sd) == b


def test_server_sums_beyond_the_64_bit_bound_exactly(ctx):
    """Requests with 124 < e0 <= 252 leave the server with the value of the
    sum modulo 2^128 (ZXP_OK when the canonical value fits 64 bits,
    ZXP_EOVERFLOW otherwise); e0 <= 124 ones with the 64-bit sum."""
    cases = []
    for i, (e0, G) in enumerate(((100, (3, -1, 0, 2)), (150, (5, 0, -2, 1)), (240, (1, 1, 0, 0)),
                                 (130, BIG_G))):
        ps = zi.synthetic_ps(1200 + i, 11, n_lin=8, n_quad=4, n_node=7, e0=e0, G=G)
        whole = oracle.ps_sum(ps.pack(), 0, 1 << 11, nthreads=NCPU)
        cases.append((Z.zxp_scalar_from_tables(ps.pack()), tuple(oracle.canon(whole[:4], whole[4]))))
    with Z.zxp_server_create(ctx) as srv:
        tickets = [Z.zxp_server_submit_scalar(srv, s) for s, _ in cases]
        for t, (s, can) in zip(tickets, cases):
            status, value, _ = Z.zxp_server_poll(srv, t, -1)
            if all(-(1 << 63) <= x < (1 << 63) for x in can[:4]):
                assert status == Z.ZXP_OK and value == can, (Z.zxp_scalar_info(s)["e0"], value, can)
            else:
                assert status == Z.ZXP_EOVERFLOW
