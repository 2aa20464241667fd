"""zxp_sum_resumable on the GPU, through the C ABI: a whole amplitude summed
in chunks whose progress is kept in a host file.  Child processes run a few
chunks each and exit between chunks (their kernels have ended: every chunk
is a synchronous evaluation), then this process resumes the file to the end;
the result equals the amplitude summed in one call, and the state vector
where one exists.  The n = 50, 2000-gate, T = 80 amplitude and its inverse
circuit's (e0 = 127: 128-bit partial sums) are summed this way too."""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INV = {zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi
    INV = {{zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}}
    kind, seed, cl, path, budget = {kind!r}, {seed}, {cl}, {path!r}, {budget}
    if kind == "medium":
        w = zi.workload_medium(seed)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    else:
        w = zi.workload_large(seed)
        gates, bits, ib = w.gates, w.out_bits, None
        if kind == "large_dag":
            gates = [(INV.get(op, op), q0, q1) for op, q0, q1 in reversed(w.gates)]
            bits, ib = [0] * w.n, w.out_bits
        s = Z.zxp_compile(gates, w.n, bits, in_bits=ib) if ib else Z.zxp_compile(gates, w.n, bits)
    ctx = Z.zxp_ctx_create(0)
    st, _, done, total = Z.zxp_sum_resumable(ctx, s, cl, path, budget)
    print(st, done, total)
""")


def child(kind, seed, cl, path, budget):
    code = CHILD.format(root=ROOT, kind=kind, seed=seed, cl=cl, path=str(path), budget=budget)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return [int(x) for x in r.stdout.split()]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "these tests need a GPU"
    c = Z.zxp_ctx_create(0)
    yield c
    c.close()


def test_medium_amplitude_resumed_across_processes(ctx, tmp_path):
    w = zi.workload_medium(1)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    k = s.info["k"]
    cl = k - 4   # 16 chunks
    p = tmp_path / "medium.ckpt"
    assert child("medium", 1, cl, p, 3) == [Z.ZXP_EAGAIN, 3, 16]
    assert child("medium", 1, cl, p, 5) == [Z.ZXP_EAGAIN, 8, 16]
    st, value, done, total = Z.zxp_sum_resumable(ctx, s, cl, str(p))
    assert (st, done, total) == (Z.ZXP_OK, 16, 16)
    assert value == Z.zxp_amplitude(ctx, s) == oracle.amp(w.gates, w.n, w.out_bits)
    # the finished file answers without running anything; another chunk
    # size does not match it
    assert Z.zxp_sum_resumable(ctx, s, cl, str(p))[:2] == (Z.ZXP_OK, value)
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_sum_resumable(ctx, s, cl - 1, str(p))
    assert e.value.code == Z.ZXP_EINVAL


def test_large_amplitude_and_inverse_resumed(ctx, tmp_path):
    """n = 50, 2000 gates, T = 80: 2^31 outer terms (times 2^20 inner) in
    eight chunks; the inverse circuit (e0 = 127) in 128-bit partial sums;
    the first equals the conjugate of the second."""
    w = zi.workload_large(0)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    k = s.info["k"]
    p = tmp_path / "large.ckpt"
    assert child("large", 0, k - 3, p, 3) == [Z.ZXP_EAGAIN, 3, 8]
    st, a, done, total = Z.zxp_sum_resumable(ctx, s, k - 3, str(p))
    assert (st, done, total) == (Z.ZXP_OK, 8, 8)
    assert a == Z.zxp_amplitude(ctx, s)
    dag = [(INV.get(op, op), q0, q1) for op, q0, q1 in reversed(w.gates)]
    sd = Z.zxp_compile(dag, w.n, [0] * w.n, in_bits=w.out_bits)
    kd = sd.info["k"]
    q = tmp_path / "dag.ckpt"
    assert child("large_dag", 0, kd - 2, q, 1) == [Z.ZXP_EAGAIN, 1, 4]
    st, b, done, total = Z.zxp_sum_resumable(ctx, sd, kd - 2, str(q))
    assert (st, done, total) == (Z.ZXP_OK, 4, 4)
    assert a == (b[0], -b[3], -b[2], -b[1], b[4])
