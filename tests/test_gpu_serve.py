"""The request server (continuous batching on the device) against single
evaluation and the oracle: every value a request gets in the mix equals the
value of the same scalar evaluated alone, exactly (tolerance 0)."""
import random
import time

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


def synthetic_mix(n, seed, ks=(0, 2, 5, 9, 13, 17, 20, 22)):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        kind = i % 6
        kw = [dict(n_node=3, odd_nodes_only=True), dict(n_node=9, odd_nodes_only=True),
              dict(n_node=40, odd_nodes_only=True), dict(n_node=12, n_pair=2),
              dict(n_node=10), dict(n_node=20, n_pair=4)][kind]
        ps = zi.synthetic_ps(seed * 1000 + i, rng.choice(ks), n_lin=16, n_quad=5,
                             density=0.25, **kw)
        out.append(Z.zxp_scalar_from_tables(ps.pack()))
    return out


def drain(srv, tickets):
    res = {}
    for t in tickets:
        r = Z.zxp_server_poll(srv, t, -1)
        assert r is not None
        res[t] = r
    return res


@pytest.mark.parametrize("policy", [Z.ZXP_SERVE_BATCHED, Z.ZXP_SERVE_PLAIN])
def test_values_in_the_mix_equal_values_alone(ctx, policy):
    scalars = synthetic_mix(60, 1)
    alone = [Z.zxp_amplitude(ctx, s) for s in scalars]
    with Z.zxp_server_create(ctx, policy=policy, step_terms=1 << 20, small_terms=1 << 14,
                             chunk_log2=12) as srv:
        tickets = [Z.zxp_server_submit_scalar(srv, s) for s in scalars]
        res = drain(srv, tickets)
        st = Z.zxp_server_stats(srv)
    for t, want in zip(tickets, alone):
        status, value, timing = res[t]
        assert status == Z.ZXP_OK and value == want
        assert timing["done_us"] >= timing["admitted_us"] >= timing["submit_us"]
    assert st["completed"] == len(scalars) and st["rejected"] == 0
    if policy == Z.ZXP_SERVE_BATCHED:
        assert st["peak_active"] > 1


def test_small_scalars_match_the_oracle(ctx):
    blobs = []
    for i in range(12):
        ps = zi.synthetic_ps(500 + i, i % 9, n_lin=10, n_quad=4, n_node=8 + i, n_pair=i % 3,
                             e0=i, G=(1, i - 4, 0, 2))
        blobs.append(ps.pack())
    scalars = [Z.zxp_scalar_from_tables(b) for b in blobs]
    with Z.zxp_server_create(ctx) as srv:
        tickets = [Z.zxp_server_submit_scalar(srv, s) for s in scalars]
        res = drain(srv, tickets)
    for t, blob in zip(tickets, blobs):
        o = oracle.ps_sum(blob)
        assert res[t][0] == Z.ZXP_OK
        assert res[t][1] == oracle.canon(o[:4], o[4])


def test_circuit_requests_compiled_by_the_server(ctx):
    reqs = zi.serve_requests(3, 40)
    with Z.zxp_server_create(ctx, compile_threads=4) as srv:
        tickets = [Z.zxp_server_submit(srv, r["gates"], r["n"], r["bits"], marg_mask=r["mask"],
                                       kind=r["kind"]) for r in reqs]
        res = drain(srv, tickets)
    checked = 0
    for r, t in zip(reqs, tickets):
        status, value, timing = res[t]
        s = Z.zxp_compile(r["gates"], r["n"], r["bits"], marg_mask=r["mask"], kind=r["kind"])
        if s.info["k"] > 44:
            assert status == Z.ZXP_ETOOBIG
            continue
        assert status == Z.ZXP_OK and value == Z.zxp_amplitude(ctx, s)
        assert timing["compiled_us"] >= timing["submit_us"] and timing["k"] == s.info["k"]
        if r["n"] <= 14:   # independent check on the exact state vector
            if r["kind"] == Z.ZXP_AMPLITUDE:
                assert value == oracle.amp(r["gates"], r["n"], r["bits"])
            else:
                assert value == oracle.marginal(r["gates"], r["n"], r["mask"], r["bits"])
            checked += 1
    assert checked >= 1


def test_large_request_runs_in_resumable_chunks(ctx):
    ps = zi.synthetic_ps(77, 24, n_lin=20, n_quad=8, n_node=9, odd_nodes_only=True)
    s = Z.zxp_scalar_from_tables(ps.pack())
    want = Z.zxp_amplitude(ctx, s)
    with Z.zxp_server_create(ctx, step_terms=1 << 18, small_terms=1 << 10, chunk_log2=14) as srv:
        t = Z.zxp_server_submit_scalar(srv, s)
        status, value, timing = Z.zxp_server_poll(srv, t, -1)
    assert status == Z.ZXP_OK and value == want
    assert timing["steps"] >= (1 << 24) // (1 << 18)   # one share per step


def test_small_requests_pass_a_large_one(ctx):
    """Continuous batching: requests that arrive while a large one is on the
    device finish first; the one-scalar-per-launch policy serves in order."""
    # (2^34 terms: several milliseconds on the device under either policy,
    # so that the small requests arrive while it runs)
    big = Z.zxp_scalar_from_tables(
        zi.synthetic_ps(78, 34, n_lin=20, n_quad=8, n_node=9, odd_nodes_only=True).pack())
    small = synthetic_mix(8, 2, ks=(0, 4, 8))
    order = {}
    for policy in (Z.ZXP_SERVE_BATCHED, Z.ZXP_SERVE_PLAIN):
        with Z.zxp_server_create(ctx, policy=policy, step_terms=1 << 26) as srv:
            tb = Z.zxp_server_submit_scalar(srv, big)
            time.sleep(0.001)
            ts = [Z.zxp_server_submit_scalar(srv, s) for s in small]
            res = drain(srv, [tb] + ts)
        done_big = res[tb][2]["done_us"]
        assert all(res[t][2]["submit_us"] < done_big for t in ts)   # they overlapped it
        order[policy] = all(res[t][2]["done_us"] < done_big for t in ts)
        assert all(res[t][0] == Z.ZXP_OK for t in [tb] + ts)
    assert order[Z.ZXP_SERVE_BATCHED]
    assert not order[Z.ZXP_SERVE_PLAIN]


def test_admission_by_k(ctx):
    scalars = synthetic_mix(12, 3, ks=(2, 6, 12, 16))
    with Z.zxp_server_create(ctx, max_k=10) as srv:
        tickets = [Z.zxp_server_submit_scalar(srv, s) for s in scalars]
        res = drain(srv, tickets)
        st = Z.zxp_server_stats(srv)
    n_big = 0
    for s, t in zip(scalars, tickets):
        if s.info["k"] > 10:
            assert res[t][0] == Z.ZXP_ETOOBIG and res[t][1] is None
            n_big += 1
        else:
            assert res[t][0] == Z.ZXP_OK and res[t][1] == Z.zxp_amplitude(ctx, s)
    assert n_big and st["rejected"] == n_big


def test_admission_by_memory(ctx):
    """A small arena holds a few requests' tables at a time: the others wait
    for memory, and every value is still exact."""
    scalars = [s for s in synthetic_mix(60, 4, ks=(8, 12, 16))
               if s.info["device_bytes"] + 512 <= 16 * 1024][:30]
    assert len(scalars) == 30
    with Z.zxp_server_create(ctx, arena_bytes=48 * 1024, step_terms=1 << 14,
                             small_terms=1 << 10, chunk_log2=10) as srv:
        tickets = [Z.zxp_server_submit_scalar(srv, s) for s in scalars]
        res = drain(srv, tickets)
        st = Z.zxp_server_stats(srv)
    for s, t in zip(scalars, tickets):
        assert res[t][0] == Z.ZXP_OK and res[t][1] == Z.zxp_amplitude(ctx, s)
    assert st["arena_peak"] <= 48 * 1024
    assert 1 <= st["peak_active"] < len(scalars)


def test_tables_larger_than_the_arena_are_rejected(ctx):
    s = Z.zxp_scalar_from_tables(zi.synthetic_ps(9, 10, n_lin=8, n_node=60,
                                                 odd_nodes_only=True).pack())
    with Z.zxp_server_create(ctx, arena_bytes=4096) as srv:
        t = Z.zxp_server_submit_scalar(srv, s)
        status, value, _ = Z.zxp_server_poll(srv, t, -1)
    assert status == Z.ZXP_ETOOBIG and value is None


def test_poll_unknown_ticket_and_timeout(ctx):
    with Z.zxp_server_create(ctx) as srv:
        with pytest.raises(Z.ZxpError) as e:
            Z.zxp_server_poll(srv, 12345, 0)
        assert e.value.code == Z.ZXP_ENOTFOUND
        s = Z.zxp_scalar_from_tables(zi.synthetic_ps(5, 26, n_lin=20, n_quad=8, n_node=9,
                                                     odd_nodes_only=True).pack())
        t = Z.zxp_server_submit_scalar(srv, s)
        first = Z.zxp_server_poll(srv, t, 0)          # 2^26 terms: not done at once
        last = Z.zxp_server_poll(srv, t, -1) if first is None else first
        assert last[0] == Z.ZXP_OK and last[1] == Z.zxp_amplitude(ctx, s)


def test_destroy_finishes_queued_requests(ctx):
    scalars = synthetic_mix(20, 5)
    srv = Z.zxp_server_create(ctx)
    for s in scalars:
        Z.zxp_server_submit_scalar(srv, s)
    srv.close()   # must return with everything finished, not hang


def test_bind_requests_cover_every_output_bitstring(ctx):
    """One parametric reduction, every output bitstring through the server:
    each value equals the exact state vector amplitude."""
    w = zi.workload_small(2)
    n = w.n
    ps = Z.zxp_compile_param(w.gates, n, [0] * n, list(range(n)))
    amps = oracle.amps_all(w.gates, n)
    with Z.zxp_server_create(ctx) as srv:
        tickets = [Z.zxp_server_submit_bind(srv, ps, x) for x in range(1 << n)]
        res = drain(srv, tickets)
    for x, t in enumerate(tickets):
        assert res[t][0] == Z.ZXP_OK and res[t][1] == amps[x]


def test_bind_requests_equal_fixed_bit_compiles(ctx):
    w = zi.workload_medium(2)
    ps = Z.zxp_compile_param(w.gates, w.n, [0] * w.n, list(range(w.n)))
    rng = random.Random(5)
    bitstrings = [rng.getrandbits(w.n) for _ in range(6)]
    with Z.zxp_server_create(ctx) as srv:
        tickets = [Z.zxp_server_submit_bind(srv, ps, b) for b in bitstrings]
        res = drain(srv, tickets)
    for b, t in zip(bitstrings, tickets):
        bits = [(b >> q) & 1 for q in range(w.n)]
        s = Z.zxp_compile(w.gates, w.n, bits)
        assert res[t][0] == Z.ZXP_OK and res[t][1] == Z.zxp_amplitude(ctx, s)
