"""Host logic of the kernel plan (no GPU): the tables the sum kernel reads.

A small C++ program (tests/host/plan_test.cpp), built from the library's own
plan and table sources, prints for every parameter assignment of each scalar
the term its plan encodes (the constant K times the table entry its form
bits select); every such term must equal the oracle's term times G exactly.
Where the plan built a block lookup, the program also checks that the lookup
gives each term of every aligned block of 8 Gray steps the counter of its
own phase class and node count, and that the incremental lookup-slot
changes and the parameter copies of the low variables' rows agree with the
plan's forms."""
import os
import random
import shutil
import subprocess

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_06777_gb300", "csrc")
M64 = (1 << 64) - 1


def zmul(a, b):
    """Product in Z[w] (w^4 = -1), coefficients modulo 2^64."""
    r = [0, 0, 0, 0]
    for i in range(4):
        for j in range(4):
            if i + j < 4:
                r[i + j] += a[i] * b[j]
            else:
                r[i + j - 4] -= a[i] * b[j]
    return tuple(v & M64 for v in r)


def scalars():
    out = []
    for seed in range(8):
        w = zi.workload_small(seed)
        out.append(Z.zxp_scalar_to_tables(Z.zxp_compile(w.gates, w.n, w.out_bits)))
    for seed in range(60):
        w = zi.workload_batch_item(seed)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        if s.info["k"] <= 22:
            out.append(Z.zxp_scalar_to_tables(s))
    w = zi.workload_medium(0)
    out.append(Z.zxp_scalar_to_tables(Z.zxp_compile(w.gates, w.n, w.out_bits)))
    rng = random.Random(11)
    for i in range(60):
        k = rng.choice([0, 1, 3, 5, 8, 10, 12, 16])
        out.append(zi.synthetic_ps(3000 + i, k, n_lin=rng.randint(0, 12), n_quad=rng.randint(0, 6),
                                   n_node=rng.choice([0, 2, 5, 7, 8, 10, 14]),
                                   n_pair=rng.choice([0, 0, 1, 2, 3]),
                                   odd_nodes_only=rng.random() < 0.6,
                                   density=rng.choice([0.1, 0.25, 0.5])).pack())
    # many forms on the lowest variables, few odd nodes, no phase-pair or
    # zero forms: block lookups over two tables
    for i in range(24):
        out.append(zi.synthetic_ps(4000 + i, rng.randint(8, 16), n_lin=rng.randint(22, 34),
                                   n_quad=rng.randint(0, 6), n_node=rng.randint(0, 7),
                                   odd_nodes_only=True, density=rng.choice([0.25, 0.35])).pack())
    return out


def build_plan_test(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "plan_test")
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, os.path.join(ROOT, "tests", "host", "plan_test.cpp"),
                    os.path.join(CSRC, "ps.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


def split_scalars():
    """Scalars with inner parameters: compiled and synthetic scalars split
    with small limits, so that outer and inner parts are both nontrivial."""
    out = []
    for seed in range(40):
        w = zi.workload_batch_item(seed)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        if 10 <= s.info["k"] <= 22 and not s.info["k_inner"]:
            sp = Z.zxp_scalar_split(s, min_k=6, max_inner=min(10, s.info["k"] - 6), low_free=4, seed=seed + 1)
            if sp.info["k_inner"]:
                out.append(Z.zxp_scalar_to_tables(sp))
    rng = random.Random(23)
    for i in range(40):
        k = rng.randint(8, 18)
        ps = zi.synthetic_ps(5000 + i, k, n_lin=rng.randint(4, 16), n_quad=rng.randint(0, 8),
                             n_node=rng.choice([2, 5, 8, 12]), n_pair=rng.choice([0, 0, 1, 2, 3]),
                             odd_nodes_only=rng.random() < 0.6, density=rng.choice([0.1, 0.2, 0.35]))
        s = Z.zxp_scalar_from_tables(ps.pack())
        sp = Z.zxp_scalar_split(s, min_k=6, max_inner=min(8, k - 6), low_free=4, max_cut=4, seed=i + 1)
        if sp.info["k_inner"]:
            out.append(Z.zxp_scalar_to_tables(sp))
    return out


def test_split_plan_outer_terms_times_inner_table(tmp_path):
    # scalars with inner parameters: each outer term times the inner table
    # at its cut parities (built on the host from the inner plan) equals the
    # oracle's term of that Gray index, the sum over all inner values
    exe = build_plan_test(tmp_path)
    blobs = split_scalars()
    assert len(blobs) >= 40
    paths = []
    for i, b in enumerate(blobs):
        p = str(tmp_path / f"v{i}.bin")
        with open(p, "wb") as f:
            f.write(b)
        paths.append(p)
    r = subprocess.run([exe] + paths, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert lines[-2] == "ok"
    pos = n_terms = 0
    for i, blob in enumerate(blobs):
        head = lines[pos].split()
        pos += 1
        ko = int(head[3])
        assert ko == oracle.outer_k(blob)
        bits = Z.zxp_scalar_info(Z.zxp_scalar_from_tables(blob))["inner_bits"]
        if ko > 12 or bits > 16:
            continue
        for t in range(1 << ko):
            got = tuple(int(v, 16) for v in lines[pos].split())
            pos += 1
            want = tuple(c & M64 for c in oracle.ps_sum(blob, t, 1)[:4])
            assert got == want, (i, t, got, want)
            n_terms += 1
    assert n_terms > 5000


def test_plan_terms_and_block_lookup(tmp_path):
    exe = build_plan_test(tmp_path)
    blobs = scalars()
    paths = []
    for i, b in enumerate(blobs):
        p = str(tmp_path / f"s{i}.bin")
        with open(p, "wb") as f:
            f.write(b)
        paths.append(p)
    r = subprocess.run([exe] + paths, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert lines[-2] == "ok"
    pos = 0
    n_terms = n_lookup = n_lane = n_two = 0
    for i, blob in enumerate(blobs):
        head = lines[pos].split()
        pos += 1
        assert head[0] == "scalar" and head[1] == paths[i]
        k, lookup, lane, two = int(head[3]), int(head[5]), int(head[7]), int(head[9])
        n_lookup += lookup
        n_lane += lane
        n_two += two
        if k > 12:
            continue
        G = tuple(c & M64 for c in zi.PSTables.unpack(blob).G)
        for x in range(1 << k):
            got = tuple(int(v, 16) for v in lines[pos].split())
            pos += 1
            want = zmul(G, tuple(c & M64 for c in oracle.ps_term(blob, x)))
            assert got == want, (i, x, got, want)
            n_terms += 1
    assert n_terms > 20000 and n_lookup >= 20 and n_lane >= 10 and n_lookup - n_lane >= 3 and n_two >= 8, \
        (n_terms, n_lookup, n_lane, n_two)
