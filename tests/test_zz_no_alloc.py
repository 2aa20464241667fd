"""zxp_eval_noalloc: the evaluation entry point for callers that cannot
allocate device memory (code under a memory manager that owns the device,
latency-critical loops where cudaMalloc would synchronise).  Its raw partials
must equal the oracle's (modulo 2^64) and zxp_eval's exactly, with the flags
word of a valid raw partial (bit 0 set, bit 1 clear), on two calls in a row
(the shared static scratch keeps the previous call's contents, which must
not leak into the next), on a stream of the caller's and on the legacy
default stream.

This file is collected last on purpose: it runs after every other test in a
full run, and it also passes alone in a fresh process."""
import os

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu


M64 = (1 << 64) - 1
NCPU = os.cpu_count() or 4


def decode(t):
    """(c0, c1, c2, c3, e) and the flags word of a 40-byte result."""
    v = t.tolist()
    return (v[0], v[1], v[2], v[3], v[4] & 0xFFFFFFFF), (v[4] >> 32) & 0xFFFFFFFF


def same_raw(g, o):
    return g[4] == o[4] and all((g[i] - o[i]) & M64 == 0 for i in range(4))


def scalars():
    w = zi.workload_medium(0)
    yield "medium", Z.zxp_compile(w.gates, w.n, w.out_bits), None
    ps = zi.synthetic_ps(8, 20, n_lin=30, n_quad=10, n_node=8, odd_nodes_only=True)
    yield "packed counters", Z.zxp_scalar_from_tables(ps.pack()), (12345, (1 << 20) - 2 * 12345)
    ps = zi.synthetic_ps(5, 16, n_lin=10, n_quad=5, n_node=12, n_pair=3)
    yield "phase-pairs", Z.zxp_scalar_from_tables(ps.pack()), None
    ps = zi.synthetic_ps(9, 18, n_lin=20, n_quad=8, n_node=40, odd_nodes_only=True)
    yield "table", Z.zxp_scalar_from_tables(ps.pack()), (777, 1000)


def test_no_alloc_matches_eval_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available(), "this test needs a GPU"
    ctx = Z.zxp_ctx_create(0)
    stream = torch.cuda.Stream()
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    for name, s, rng in scalars():
        k = Z.zxp_scalar_info(s)["k"]
        blob = Z.zxp_scalar_to_tables(s)
        first, count = rng if rng else (0, 1 << k)
        want = Z.zxp_eval(ctx, s, first, count)
        for call in range(2):
            out.fill_(-1)
            torch.cuda.synchronize()
            Z.zxp_eval_noalloc(s, first, count, out.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            got, flags = decode(out)
            assert got == want and flags == 1, (name, call, flags)
        # ragged ranges against the oracle, the last one on the legacy
        # default stream
        n = 1 << k
        for i, (a, c) in enumerate(((1, 999), (n - 77, 77), (n // 3, 4097))):
            out.fill_(-1)
            torch.cuda.synchronize()
            Z.zxp_eval_noalloc(s, a, c, out.data_ptr(), 0 if i == 2 else stream.cuda_stream)
            torch.cuda.synchronize()
            got, flags = decode(out)
            assert flags == 1 and same_raw(got, oracle.ps_sum(blob, a, c, nthreads=NCPU)), (name, a, c)
    ctx.close()


def test_no_alloc_rejects_tables_beyond_the_scratch():
    """Tables of 654 KB (150 nodes, folded phase-pair and zero bits) do not
    fit the 256 KB array: ZXP_ETOOBIG, nothing queued."""
    import torch
    ps = zi.synthetic_ps(2100, 24, n_lin=10, n_quad=6, n_node=150, n_pair=2, density=0.3)
    s = Z.zxp_scalar_from_tables(ps.pack())
    assert Z.zxp_scalar_info(s)["upload_bytes"] > 256 * 1024
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_eval_noalloc(s, 0, 1 << 10, out.data_ptr())
    assert e.value.code == Z.ZXP_ETOOBIG


def test_no_alloc_rejects_bad_arguments():
    import torch
    s = Z.zxp_scalar_from_tables(zi.synthetic_ps(1, 6).pack())
    out = torch.zeros(6, dtype=torch.int64, device="cuda")
    with pytest.raises(Z.ZxpError):
        Z.zxp_eval_noalloc(s, 60, 10, out.data_ptr())            # range beyond 2^k
    with pytest.raises(Z.ZxpError):
        Z.zxp_eval_noalloc(s, 0, 64, out.data_ptr() + 4)         # unaligned output
