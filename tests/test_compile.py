"""Host compiler (circuit -> parametric scalar) checked on the CPU.

The compiled tables are summed by the oracle and compared with the oracle's
exact state vector: tolerance zero, canonical Z[w]/sqrt2^e values."""
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi


def compiled_value(gates, n, bits, kind=0, mask=0, in_bits=None):
    s = Z.zxp_compile(gates, n, bits, in_bits=in_bits, marg_mask=mask, kind=kind)
    blob = Z.zxp_scalar_to_tables(s)
    v = oracle.ps_sum(blob, nthreads=4)
    return oracle.canon(v[:4], v[4]), Z.zxp_scalar_info(s)


def small_circuit(seed, n, g):
    if n == 1:
        return [(op, 0, 0) for op, _, _ in zi.circuit_iid(seed, 2, g) if op != zi.CNOT]
    return zi.circuit_iid(seed, n, g)


@pytest.mark.parametrize("seed", range(120))
def test_amplitude_matches_statevector(seed):
    rng = random.Random(seed)
    n = 1 + seed % 7
    gates = small_circuit(seed, n, rng.randint(10, 70))
    extra = [(zi.SDG, 0, 0), (zi.TDG, n - 1, 0), (zi.X, 0, 0), (zi.Z, n - 1, 0)]
    if n > 1:
        extra.append((zi.CZ, n - 1, 0))
    gates = gates[: len(gates) // 2] + extra + gates[len(gates) // 2:]
    out = zi.random_bits(seed, n)
    inb = zi.random_bits(seed + 77, n) if seed % 3 == 0 else None
    got, _ = compiled_value(gates, n, out, in_bits=inb)
    assert got == oracle.amp(gates, n, out, inb)


@pytest.mark.parametrize("seed", range(60))
def test_doubled_marginal_matches_statevector(seed):
    n = 2 + seed % 5
    gates = zi.circuit_iid(seed + 500, n, 15 + seed % 35)
    mask = (seed * 2654435761) & ((1 << n) - 1) or 1
    bits = zi.random_bits(seed + 9, n)
    got, _ = compiled_value(gates, n, bits, kind=Z.ZXP_MARGINAL_DOUBLED, mask=mask)
    assert got == oracle.marginal(gates, n, mask, bits)
    assert got[1] == -got[3] and got[2] == 0          # a probability is real


def test_small_workload_all_outputs_sum_to_one():
    w = zi.workload_small(0)
    n = w.n
    vals = []
    for x in range(1 << n):
        bits = [(x >> q) & 1 for q in range(n)]
        v, _ = compiled_value(w.gates, n, bits)
        vals.append(v)
    assert vals == oracle.amps_all(w.gates, n)
    emax = max(v[4] for v in vals)
    tot = [0, 0, 0, 0]
    for c0, c1, c2, c3, e in vals:
        c, cj = (c0, c1, c2, c3), (c0, -c3, -c2, -c1)
        for i in range(4):
            for j in range(4):
                t = c[i] * cj[j] * 2 ** (emax - e)
                if i + j < 4:
                    tot[i + j] += t
                else:
                    tot[i + j - 4] -= t
    assert tot == [2 ** emax, 0, 0, 0]


def dagger(gates):
    inv = {zi.S: zi.SDG, zi.SDG: zi.S, zi.T: zi.TDG, zi.TDG: zi.T}
    return [(inv.get(op, op), a, b) for op, a, b in reversed(gates)]


@pytest.mark.parametrize("seed", range(10))
def test_conjugate_transpose_consistency(seed):
    # <x|C|0> = conj(<0|C^dag|x>), with no state vector involved
    n = 8
    gates = zi.circuit_iid(seed + 900, n, 60)
    x = zi.random_bits(seed, n)
    a, _ = compiled_value(gates, n, x)
    b, _ = compiled_value(dagger(gates), n, [0] * n, in_bits=x)
    c0, c1, c2, c3, e = b
    assert a == (c0, -c3, -c2, -c1, e)


def test_clifford_only_circuits_reduce_to_no_parameters():
    for seed in range(10):
        gates = [g for g in zi.circuit_iid(seed, 6, 80) if g[0] != zi.T]
        s = Z.zxp_compile(gates, 6, zi.random_bits(seed, 6))
        info = Z.zxp_scalar_info(s)
        assert info["k"] == 0 and info["n_node"] == 0 and info["n_pair"] == 0


def test_zero_amplitude_compiles_to_zero():
    s = Z.zxp_compile([(zi.X, 0, 0)], 2, [0, 0])      # <00|X_0|00> = 0
    blob = Z.zxp_scalar_to_tables(s)
    assert oracle.ps_sum(blob)[:4] == (0, 0, 0, 0)


def test_medium_workload_parameter_counts():
    # n = 20, 600 gates, 40 T: the reduction leaves far fewer parameters
    # than T gates, and the exponent stays inside the exact int64 range
    for seed in range(4):
        w = zi.workload_medium(seed)
        info = Z.zxp_scalar_info(Z.zxp_compile(w.gates, w.n, w.out_bits))
        assert info["t_count"] == 40
        assert info["k"] <= 30
        assert info["acc_bits"] == 64
