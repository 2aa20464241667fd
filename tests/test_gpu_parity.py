"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Every comparison is exact: raw partial sums agree modulo 2^64 (the ring the
kernel computes in), canonical amplitudes agree as integers."""
import os
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1
NCPU = os.cpu_count() or 4


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


def check_ranges(ctx, ps, ranges):
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    for first, count in ranges:
        g = Z.zxp_eval(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert same_raw(g, o), (ps.k, first, count, g, o)


def std_ranges(k, rng):
    N = 1 << k
    r = [(0, N), (0, 0), (N, 0), (N - 1, 1), (0, 1)]
    if N > 8:
        r += [(1, N - 3), (N // 3, N // 2)]
        a = rng.randrange(N)
        r.append((a, rng.randrange(N - a + 1)))
    return r


@pytest.mark.parametrize("seed", range(16))
def test_synthetic_tables_all_row_kinds(ctx, seed):
    rng = random.Random(seed)
    k = rng.choice([0, 1, 3, 6, 9, 12, 14, 16])
    ps = zi.synthetic_ps(seed, k, n_lin=rng.randint(0, 12), n_quad=rng.randint(0, 6),
                         n_node=rng.randint(0, 24), n_pair=rng.randint(0, 4),
                         density=rng.choice([0.1, 0.3, 0.6]), e0=rng.randint(0, 9),
                         G=(rng.randint(-9, 9), rng.randint(-9, 9), rng.randint(-9, 9), 1))
    check_ranges(ctx, ps, std_ranges(k, rng))


@pytest.mark.parametrize("n_node,n_lin", [(31, 1), (32, 31), (33, 33), (64, 64), (65, 10),
                                          (100, 100), (128, 120), (5, 127)])
def test_synthetic_form_word_layouts(ctx, n_node, n_lin):
    # node words 1..4 and other words 1..4; odd nodes only (the common case)
    ps = zi.synthetic_ps(n_node * 1000 + n_lin, 11, n_lin=n_lin, n_quad=3, n_node=n_node,
                         odd_nodes_only=True, density=0.35)
    check_ranges(ctx, ps, std_ranges(11, random.Random(n_node)))


def test_synthetic_pairs_and_zero_nodes(ctx):
    ps = zi.synthetic_ps(99, 13, n_lin=6, n_quad=5, n_node=20, n_pair=12, density=0.3)
    ps.node += [(0b101, 0), (0b1100000, 4), (0b11, 2), (0b110, 6), (0, 3), (0, 1)]
    ps.pair += [(0, 3, 0, 5), (0b1, 2, 0, 6)]
    check_ranges(ctx, ps, std_ranges(13, random.Random(5)))


def test_largest_slices_and_ragged_tails(ctx):
    ps = zi.synthetic_ps(3, 22, n_lin=10, n_quad=6, n_node=30, odd_nodes_only=True, density=0.3)
    N = 1 << 22
    check_ranges(ctx, ps, [(0, N), (12345, N - 2 * 12345), (N - 777, 777), ((1 << 20) + 1, 3)])


@pytest.mark.parametrize("seed", range(40))
def test_compiled_small_amplitudes_exact(ctx, seed):
    n = 2 + seed % 6
    gates = zi.circuit_iid(seed + 4000, n, 30 + seed)
    out = zi.random_bits(seed, n)
    s = Z.zxp_compile(gates, n, out)
    assert Z.zxp_amplitude(ctx, s) == oracle.amp(gates, n, out)


@pytest.mark.parametrize("seed", range(12))
def test_compiled_small_marginals_exact(ctx, seed):
    n = 3 + seed % 4
    gates = zi.circuit_iid(seed + 8000, n, 40)
    bits = zi.random_bits(seed, n)
    mask = 1 << (seed % n)
    s = Z.zxp_compile(gates, n, bits, marg_mask=mask, kind=Z.ZXP_MARGINAL_DOUBLED)
    assert Z.zxp_amplitude(ctx, s) == oracle.marginal(gates, n, mask, bits)


def test_small_workload_every_output(ctx):
    w = zi.workload_small(0)
    want = oracle.amps_all(w.gates, w.n)
    for x in range(1 << w.n):
        bits = [(x >> q) & 1 for q in range(w.n)]
        assert Z.zxp_amplitude(ctx, Z.zxp_compile(w.gates, w.n, bits)) == want[x]


@pytest.mark.parametrize("seed", [0, 1])
def test_medium_workload_amplitude_exact(ctx, seed):
    # n = 20, 600 gates, t = 40: the full 2^k sum on the GPU (the benchmark's
    # workload and launch shape) against the exact 2^20-entry state vector
    w = zi.workload_medium(seed)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    assert Z.zxp_amplitude(ctx, s) == oracle.amp(w.gates, w.n, w.out_bits)


def test_large_workload_subranges_exact(ctx):
    # n = 50, 2000 gates, t = 80: seeded 2^20-term sub-ranges of the compiled
    # scalar against the oracle
    w = zi.workload_large(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=False)
    blob = Z.zxp_scalar_to_tables(s)
    k = Z.zxp_scalar_info(s)["k"]
    rng = zi.SplitMix64(2024)
    for _ in range(3):
        first = rng.below((1 << k) - (1 << 20))
        g = Z.zxp_eval(ctx, s, first, 1 << 20)
        o = oracle.ps_sum(blob, first, 1 << 20, nthreads=NCPU)
        assert same_raw(g, o)


def test_split_invariance_large_synthetic(ctx):
    # k = 30 synthetic scalar with compiled-like statistics: any chunking of
    # the range gives the same bits
    ps = zi.synthetic_ps(36, 30, n_lin=40, n_quad=20, n_node=50, odd_nodes_only=True, density=0.15)
    s = Z.zxp_scalar_from_tables(ps.pack())
    N = 1 << 30
    whole = Z.zxp_eval(ctx, s)
    cuts = sorted(random.Random(1).sample(range(1, N), 5))
    acc = None
    for a, b in zip([0] + cuts, cuts + [N]):
        part = Z.zxp_eval(ctx, s, a, b - a)
        acc = part if acc is None else Z.zxp_zomega_add(acc, part)
    assert acc == whole
    o = oracle.ps_sum(ps.pack(), 777777, 1 << 18, nthreads=NCPU)
    assert same_raw(Z.zxp_eval(ctx, s, 777777, 1 << 18), o)


def test_k36_counting_path_split_invariance(ctx):
    # k = 36 with few odd nodes: the counting (histogram) kernel, with several
    # slices per thread on the full range and one slice per thread on each
    # quarter; both must give the same bits, and a sub-range matches the oracle
    ps = zi.synthetic_ps(7, 36, n_lin=40, n_quad=25, n_node=4, odd_nodes_only=True, density=0.12)
    s = Z.zxp_scalar_from_tables(ps.pack())
    whole = Z.zxp_eval(ctx, s)
    q = 1 << 34
    acc = Z.zxp_eval(ctx, s, 0, q)
    for i in range(1, 4):
        acc = Z.zxp_zomega_add(acc, Z.zxp_eval(ctx, s, i * q, q))
    assert acc == whole
    o = oracle.ps_sum(ps.pack(), 123456789, 1 << 18, nthreads=NCPU)
    assert same_raw(Z.zxp_eval(ctx, s, 123456789, 1 << 18), o)


@pytest.mark.parametrize("n_node", [5, 6, 8, 11, 12])
def test_counting_paths_by_node_count(ctx, n_node):
    # 32-bit counters up to 5 odd nodes, packed 16-bit counters up to 11,
    # the table path beyond: identical results on ragged ranges
    ps = zi.synthetic_ps(n_node, 17, n_lin=30, n_quad=12, n_node=n_node, odd_nodes_only=True,
                         density=0.2)
    check_ranges(ctx, ps, std_ranges(17, random.Random(n_node)))


def test_k34_packed_counters_many_slices(ctx):
    # 8 odd nodes at k = 34: every thread takes several slices shorter than
    # 2^16 terms; chunking and the oracle agree
    ps = zi.synthetic_ps(8, 34, n_lin=40, n_quad=25, n_node=8, odd_nodes_only=True, density=0.12)
    s = Z.zxp_scalar_from_tables(ps.pack())
    whole = Z.zxp_eval(ctx, s)
    q = 1 << 32
    acc = Z.zxp_eval(ctx, s, 0, q)
    for i in range(1, 4):
        acc = Z.zxp_zomega_add(acc, Z.zxp_eval(ctx, s, i * q, q))
    assert acc == whole
    o = oracle.ps_sum(ps.pack(), 987654321, 1 << 18, nthreads=NCPU)
    assert same_raw(Z.zxp_eval(ctx, s, 987654321, 1 << 18), o)


def test_submit_poll_matches_eval(ctx):
    scalars = []
    for seed in range(6):
        ps = zi.synthetic_ps(seed, 14 + seed % 3, n_lin=8, n_node=12, n_pair=seed % 3)
        scalars.append(Z.zxp_scalar_from_tables(ps.pack()))
    tickets = [Z.zxp_submit(ctx, s) for s in scalars]
    tickets.append(Z.zxp_submit(ctx, scalars[0], 5, 0))
    got = [Z.zxp_poll(ctx, t, -1) for t in tickets]
    for s, g in zip(scalars, got):
        assert g == Z.zxp_eval(ctx, s)
    assert got[-1][:4] == (0, 0, 0, 0)
    with pytest.raises(Z.ZxpError):
        Z.zxp_poll(ctx, tickets[0], 0)        # already released


def test_streamed_requests_reuse_staging(ctx):
    """A client streaming fresh scalars (tables built per request), two to
    four requests in flight, with blocking and device-result evaluations
    interleaved: the context's staging buffers are reused many times, by
    tables of different sizes, and every result equals the oracle's."""
    import torch
    from collections import deque
    blobs = [zi.synthetic_ps(40 + i, 10 + i % 5, n_lin=6 + i, n_quad=3, n_node=5 + 3 * (i % 4),
                             n_pair=i % 3, odd_nodes_only=i % 2 == 0).pack() for i in range(7)]
    want = [oracle.ps_sum(b) for b in blobs]
    dev = torch.zeros(5, dtype=torch.int64, device="cuda")
    q = deque()
    n_done = 0
    for r in range(70):
        i = r % 7
        if r % 2:
            s = Z.zxp_scalar_from_tables(blobs[i])
            q.append((i, s, Z.zxp_submit(ctx, s)))
        else:                                         # the library owns the scalar
            q.append((i, None, Z.zxp_submit_tables(ctx, blobs[i])))
        if r % 5 == 0:
            j = (r + 3) % 7
            s2 = Z.zxp_scalar_from_tables(blobs[j])
            assert same_raw(Z.zxp_eval(ctx, s2), want[j]), (r, j)
            s2.free()
        if r % 9 == 0:
            j = (r + 5) % 7
            s3 = Z.zxp_scalar_from_tables(blobs[j])
            Z.zxp_eval_device(ctx, s3, 0, 1 << s3.info["k"], dev.data_ptr())
            torch.cuda.synchronize()
            v = dev.tolist()
            assert same_raw((v[0], v[1], v[2], v[3], v[4] & 0xFFFFFFFF), want[j]), (r, j)
            s3.free()
        while len(q) > 2 + r % 3 or (r == 69 and q):
            j, sj, tk = q.popleft()
            assert same_raw(Z.zxp_poll(ctx, tk, -1), want[j]), (r, j)
            if sj is not None:
                sj.free()
            n_done += 1
    assert n_done == 70


def test_submit_tables_errors_and_unpolled_tickets():
    """zxp_submit_tables rejects bad table bytes; a context destroyed with
    unpolled tickets frees the scalars it owns."""
    import torch
    c = Z.zxp_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(Z.ZxpError):
        Z.zxp_submit_tables(c, b"not a scalar")
    blob = zi.synthetic_ps(3, 16, n_node=6, odd_nodes_only=True).pack()
    t = Z.zxp_submit_tables(c, blob)
    assert same_raw(Z.zxp_poll(c, t, -1), oracle.ps_sum(blob))
    for _ in range(3):
        Z.zxp_submit_tables(c, blob)
    c.close()


def test_context_on_a_torch_stream():
    import torch
    st = torch.cuda.Stream()
    c = Z.zxp_ctx_create(0, st.cuda_stream)
    ps = zi.synthetic_ps(1, 12, n_node=10)
    s = Z.zxp_scalar_from_tables(ps.pack())
    assert same_raw(Z.zxp_eval(c, s), oracle.ps_sum(ps.pack()))
    c.close()


def test_range_errors(ctx):
    s = Z.zxp_scalar_from_tables(zi.synthetic_ps(1, 5).pack())
    with pytest.raises(Z.ZxpError):
        Z.zxp_eval(ctx, s, 30, 3)
    with pytest.raises(Z.ZxpError):
        Z.zxp_eval(ctx, s, 33, 0)


def test_block_lookup_variant_matches_oracle(ctx):
    """Scalars whose low variables touch few forms take the block-lookup
    kernel (variant 9; 10 with folded phase-pair / zero bits; 11 with
    lane-private counters and the phase row taken mod 8 by a mask); full sums
    and ragged ranges equal the oracle."""
    rng = random.Random(21)
    seen = 0
    seen10 = 0
    seen11 = 0
    blobs = []
    for seed in range(60, 140):
        w = zi.workload_batch_item(seed)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        if s.info["kernel_variant"] == 10 and s.info["k"] <= 24:
            blobs.append(Z.zxp_scalar_to_tables(s))
    for seed in range(4):
        w = zi.workload_medium(seed)
        blobs.append(Z.zxp_scalar_to_tables(Z.zxp_compile(w.gates, w.n, w.out_bits)))
    for i in range(12):
        k = rng.choice([3, 5, 8, 11, 14, 17])
        blobs.append(zi.synthetic_ps(800 + i, k, n_lin=rng.randint(2, 8), n_quad=rng.randint(0, 6),
                                     n_node=rng.randint(0, 7), odd_nodes_only=True,
                                     density=rng.choice([0.2, 0.4])).pack())
    for blob in blobs:
        s = Z.zxp_scalar_from_tables(blob)
        if s.info["kernel_variant"] not in (9, 10, 11):
            continue
        seen += 1
        seen10 += s.info["kernel_variant"] == 10
        seen11 += s.info["kernel_variant"] == 11
        k = s.info["k"]
        N = 1 << k
        ranges = [(0, N), (5, N - 11), (N // 3, N // 2), (N - 9, 9)] if N >= 32 else [(0, N), (1, N - 2)]
        if k > 20:
            ranges = [(0, N), (1 << 20, (1 << 19) + 13)]
        for first, count in ranges:
            g = Z.zxp_eval(ctx, s, first, count)
            o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
            assert same_raw(g, o), (k, first, count)
    assert seen >= 5 and seen10 >= 2 and seen11 >= 2


def test_two_table_block_lookup_matches_oracle(ctx):
    """Scalars with more forms on variables 0-2 than one lookup table takes
    (few odd nodes, no phase-pair or zero forms) take the two-table block
    lookup (variant 13): full sums and ragged ranges equal the oracle, a
    k = 28 sum is split-invariant, and the batch kernel gives the same
    values."""
    rng = random.Random(13)
    seen = []
    for i in range(40):
        k = rng.choice([8, 11, 14, 17, 20])
        ps = zi.synthetic_ps(900 + i, k, n_lin=rng.randint(14, 24), n_quad=rng.randint(0, 6),
                             n_node=rng.randint(0, 7), odd_nodes_only=True, density=rng.choice([0.2, 0.3]),
                             e0=rng.randint(0, 5), G=(1, rng.randint(-3, 3), 0, 1))
        blob = ps.pack()
        s = Z.zxp_scalar_from_tables(blob)
        if s.info["kernel_variant"] != 13:
            continue
        seen.append(s)
        N = 1 << k
        for first, count in [(0, N), (5, N - 11), (N // 3, N // 2), (N - 9, 9), (7, 16)]:
            g = Z.zxp_eval(ctx, s, first, count)
            o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
            assert same_raw(g, o), (i, k, first, count)
    assert len(seen) >= 10
    bt = Z.zxp_batch_create(ctx, seen)
    got = Z.zxp_batch_run(bt)
    bt.close()
    for s, g in zip(seen, got):
        assert tuple(g) == tuple(Z.zxp_eval(ctx, s))
    ps = zi.synthetic_ps(977, 28, n_lin=22, n_quad=8, n_node=5, odd_nodes_only=True, density=0.25)
    s = Z.zxp_scalar_from_tables(ps.pack())
    assert s.info["kernel_variant"] == 13
    full = Z.zxp_eval(ctx, s)
    n = 1 << 28
    parts = Z.zxp_eval(ctx, s, 0, 12345)
    for a, b in ((12345, n // 3 - 12345), (n // 3, n - n // 3 - 99), (n - 99, 99)):
        parts = Z.zxp_zomega_add(parts, Z.zxp_eval(ctx, s, a, b))
    assert Z.zxp_zomega_canon(parts) == Z.zxp_zomega_canon(full)
    blob = ps.pack()
    for first in (0, (1 << 27) + 3):
        assert same_raw(Z.zxp_eval(ctx, s, first, 1 << 16), oracle.ps_sum(blob, first, 1 << 16, nthreads=NCPU))


def test_large_compiled_t50_subranges(ctx):
    """n = 50, 2000 gates, T-count 50 (k = 37): seeded 2^20-term sub-ranges
    of the full sum equal the oracle, one of them across 2^32 (the flip of
    variable 32 in the middle of the walk)."""
    w = zi.workload_large_t50(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=False)
    blob = Z.zxp_scalar_to_tables(s)
    k = s.info["k"]
    rng = random.Random(37)
    for first in [rng.randrange((1 << k) - (1 << 20)) for _ in range(3)] + [(1 << 32) - (1 << 19) + 5]:
        g = Z.zxp_eval(ctx, s, first, 1 << 20)
        o = oracle.ps_sum(blob, first, 1 << 20, nthreads=NCPU)
        assert same_raw(g, o), first


def test_large_compiled_full_sum_conjugate_transpose(ctx):
    """The compiled n = 50, 2000-gate, T-count 50 circuit (k = 37) summed in
    full, 1.4e11 terms at the benchmark's launch shape (several slices per
    thread): the one-launch sum equals the sum of eight 2^34-term launches
    (one slice per thread), and <out|C|0> equals the conjugate of <0|C^dag|out>
    from the separately reduced inverse circuit (another scalar, another
    kernel variant; no state vector exists at n = 50)."""
    inv = {zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}
    w = zi.workload_large_t50(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=False)
    k = s.info["k"]
    assert k <= 40
    a = Z.zxp_amplitude(ctx, s)
    n8 = (1 << k) // 8
    tot = Z.zxp_eval(ctx, s, 0, n8)
    for i in range(1, 8):
        tot = Z.zxp_zomega_add(tot, Z.zxp_eval(ctx, s, i * n8, n8))
    assert Z.zxp_zomega_canon(tot) == a
    dag = [(inv.get(op, op), q0, q1) for op, q0, q1 in reversed(w.gates)]
    sd = Z.zxp_compile(dag, w.n, [0] * w.n, in_bits=w.out_bits, split=False)
    assert sd.info["k"] <= 40
    b = Z.zxp_amplitude(ctx, sd)
    assert a == (b[0], -b[3], -b[2], -b[1], b[4])


@pytest.mark.parametrize("seed,n_node,n_pair,odd,density", [
    (62, 5, 0, True, 0.05),     # block lookup, lane-private counters
    (66, 10, 0, True, 0.03),    # block lookup, warp-shared counters (more than 7 odd nodes)
    (63, 14, 1, False, 0.05),   # block lookup with folded bits
    (64, 14, 0, True, 0.4),     # warp-shared counters (too many forms on the low variables)
    (65, 40, 3, False, 0.3),    # general: Z[w] phase-pair products
])
def test_maximum_k_ranges(ctx, seed, n_node, n_pair, odd, density):
    """k = 62 (the largest supported): ranges at the start, in the middle and
    at the very end of the index space equal the oracle, on every kind of
    kernel."""
    ps = zi.synthetic_ps(seed, 62, n_lin=6, n_quad=8, n_node=n_node, n_pair=n_pair,
                         odd_nodes_only=odd, density=density)
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    N = 1 << 62
    # (ranges across 2^32 and 2^45: flips of variables 32 and 45 inside a
    # slice, whose quadratic bit the walk takes from the state itself; with
    # 64-term slices the crossing falls in a slice's first unaligned steps
    # or inside its aligned blocks of 16)
    for first, count in [(0, 1 << 16), (N // 2 - 4096, 12289), (N - (1 << 15) - 3, (1 << 15) + 3),
                         ((1 << 32) - 5003, 10007), ((1 << 32) - 5051, 10007), ((1 << 45) - 827, 4099),
                         (N - 1, 1), (N, 0)]:
        g = Z.zxp_eval(ctx, s, first, count)
        o = oracle.ps_sum(blob, first, count, nthreads=NCPU)
        assert same_raw(g, o), (first, count, s.info["kernel_variant"])


def test_block_lookup_smallest_k(ctx):
    """k = 3: one aligned 8-term block per full sum."""
    rng = random.Random(3)
    n = 0
    for i in range(40):
        ps = zi.synthetic_ps(1000 + i, 3, n_lin=rng.randint(1, 5), n_quad=rng.randint(0, 3),
                             n_node=rng.randint(0, 4), odd_nodes_only=True, density=0.5)
        blob = ps.pack()
        s = Z.zxp_scalar_from_tables(blob)
        for first, count in [(0, 8), (1, 6), (3, 5)]:
            g = Z.zxp_eval(ctx, s, first, count)
            o = oracle.ps_sum(blob, first, count)
            assert same_raw(g, o), (i, first, count)
        n += s.info["kernel_variant"] == 11
    assert n >= 10
    # more than 7 odd nodes: warp-shared counters
    n9 = 0
    for i in range(20):
        ps = zi.synthetic_ps(1100 + i, 3, n_lin=1, n_quad=rng.randint(0, 3), n_node=8,
                             odd_nodes_only=True, density=0.5)
        blob = ps.pack()
        s = Z.zxp_scalar_from_tables(blob)
        for first, count in [(0, 8), (1, 6), (3, 5)]:
            g = Z.zxp_eval(ctx, s, first, count)
            o = oracle.ps_sum(blob, first, count)
            assert same_raw(g, o), (i, first, count)
        n9 += s.info["kernel_variant"] == 9
    assert n9 >= 5


@pytest.mark.parametrize("seed,args,variant", [
    (7000, dict(n_lin=6, n_quad=8, n_node=5, odd_nodes_only=True, density=0.05), 11),
    (7003, dict(n_lin=28, n_quad=4, n_node=5, odd_nodes_only=True, density=0.3), 13),
])
def test_block_lookup_four_states_a_thread(ctx, seed, args, variant):
    """Lane-private block lookup over whole aligned blocks of 256 Gray
    indices with slices of 256 terms or more: each thread walks a slice as
    four states that differ in variables 6 and 7, along one Gray code of the
    other variables (another order of the same terms).  A 2^25-term range equals
    the oracle, and the whole 2^27-term sum taken that way equals the same
    sum split at an unaligned index (one state a thread there)."""
    ps = zi.synthetic_ps(seed, 27, **args)
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    assert s.info["kernel_variant"] == variant
    first, count = 1 << 26, 1 << 25
    assert same_raw(Z.zxp_eval(ctx, s, first, count), oracle.ps_sum(blob, first, count, nthreads=NCPU))
    n = 1 << 27
    whole = Z.zxp_eval(ctx, s)
    cut = n - 1000
    parts = Z.zxp_zomega_add(Z.zxp_eval(ctx, s, 0, cut), Z.zxp_eval(ctx, s, cut, n - cut))
    assert Z.zxp_zomega_canon(parts) == Z.zxp_zomega_canon(whole)
