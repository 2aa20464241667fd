"""The seeded input generators (zxp_inputs) against their stated recipes:
splitmix64 against published outputs of its reference definition, the gate
mixes, the fixed T-counts, the size ranges of the batch and serving
workloads, the Poisson arrival rate and the synthetic tables' shapes."""
import math
import os

import zxp_inputs as zi


def test_splitmix64_published_outputs():
    # first outputs of splitmix64 (Steele, Lea, Flood) for seeds 0 and 1234567
    r = zi.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = zi.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423]


def test_iid_gate_mix_and_qubits():
    counts = {zi.CNOT: 0, zi.H: 0, zi.S: 0, zi.T: 0}
    total = 0
    for seed in range(40):
        g = zi.circuit_iid(seed, 7, 500)
        assert len(g) == 500
        for op, q0, q1 in g:
            counts[op] += 1
            assert 0 <= q0 < 7
            if op == zi.CNOT:
                assert 0 <= q1 < 7 and q1 != q0
        total += len(g)
    for op, p in ((zi.CNOT, 0.3), (zi.H, 0.3), (zi.S, 0.2), (zi.T, 0.2)):
        sd = math.sqrt(p * (1 - p) / total)
        assert abs(counts[op] / total - p) < 5 * sd, (op, counts[op] / total)


def test_fixed_t_circuits():
    other = {zi.CNOT: 0, zi.H: 0, zi.S: 0}
    for seed in range(20):
        g = zi.circuit_fixed_t(seed, 20, 600, 40)
        assert len(g) == 600 and zi.t_count(g) == 40
        for op, _, _ in g:
            if op != zi.T:
                other[op] += 1
    n = sum(other.values())
    for op, p in ((zi.CNOT, 0.375), (zi.H, 0.375), (zi.S, 0.25)):   # 0.3 : 0.3 : 0.2
        assert abs(other[op] / n - p) < 5 * math.sqrt(p * (1 - p) / n), op


def test_measured_workload_shapes():
    w = zi.workload_small(0)
    assert w.n == 6 and len(w.gates) == 80
    w = zi.workload_medium(0)
    assert w.n == 20 and len(w.gates) == 600 and zi.t_count(w.gates) == 40 and len(w.out_bits) == 20
    w = zi.workload_large(0)
    assert w.n == 50 and len(w.gates) == 2000 and zi.t_count(w.gates) == 80
    w = zi.workload_large_t50(0)
    assert w.n == 50 and len(w.gates) == 2000 and zi.t_count(w.gates) == 50
    ns, ts = set(), set()
    for seed in range(512):
        b = zi.workload_batch_item(seed)
        assert 10 <= b.n <= 40
        t = zi.t_count(b.gates)
        assert 20 <= t <= 60 and b.gates[-1][0] == zi.T   # drawn until the T-count is reached
        ns.add(b.n)
        ts.add(t)
    assert len(ns) > 25 and len(ts) > 35


def test_serving_arrivals():
    reqs = zi.serve_requests(0, 2000, rate_hz=2000.0)
    gaps = [b["t"] - a["t"] for a, b in zip(reqs, reqs[1:])]
    mean = sum(gaps) / len(gaps)
    assert abs(mean - 1 / 2000.0) < 5 * (1 / 2000.0) / math.sqrt(len(gaps))
    assert all(g > 0 for g in gaps)
    kinds = [r["kind"] for r in reqs]
    assert 0.4 < sum(kinds) / len(kinds) < 0.6
    for r in reqs:
        assert 10 <= r["n"] <= 50 and 10 <= zi.t_count(r["gates"]) <= 70
        if r["kind"] == 1:
            assert bin(r["mask"]).count("1") == 1 and r["mask"] < (1 << r["n"])


def test_synthetic_tables_shape():
    ps = zi.synthetic_ps(36, 36, n_lin=59, n_quad=36, n_node=13, n_pair=1, odd_nodes_only=True,
                         density=0.12)
    assert ps.k == 36 and len(ps.lin) == 59 and len(ps.quad) == 36 and len(ps.node) == 13
    assert len(ps.pair) == 1
    assert all(g % 2 == 1 for _, g in ps.node)
    masks = [m for m, _ in ps.lin] + [m for q in ps.quad for m in q] + [m for m, _ in ps.node]
    assert all(0 <= m < (1 << 36) for m in masks)
    back = zi.PSTables.unpack(ps.pack())
    assert back == ps


def test_committed_large_tables_match_a_fresh_compile():
    # the reference arm of the benchmark reads these bytes instead of
    # compiling; they must be what the compiler gives today
    import importlib.util
    import oracle
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "zxp_inputs", "tables", "make_tables.py")
    spec = importlib.util.spec_from_file_location("make_tables", path)
    mt = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mt)
    committed = open(mt.LARGE, "rb").read()
    assert committed == mt.large_blob()
    assert oracle.outer_k(committed) <= 36
