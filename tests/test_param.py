"""Parametric scalars (output or marginal bits left as parameters through the
reduction; no GPU): every binding, evaluated by the oracle, equals the exact
amplitude or probability of the state vector, and equals the reduction with
those bits fixed."""
import random

import pytest

import oracle
import paper_2403_06777_gb300 as Z
import zxp_inputs as zi


def value(s):
    """Canonical value of a scalar through the oracle (plain per-term sum)."""
    o = oracle.ps_sum(Z.zxp_scalar_to_tables(s), nthreads=4)
    return oracle.canon(o[:4], o[4])


@pytest.mark.parametrize("seed", range(8))
def test_every_output_bitstring_of_small_circuits(seed):
    w = zi.workload_small(seed)
    n = w.n
    ps = Z.zxp_compile_param(w.gates, n, [0] * n, list(range(n)))
    assert ps.info["n_params"] == n and Z.zxp_pscalar_params(ps) == list(range(n))
    amps = oracle.amps_all(w.gates, n)
    for x in range(1 << n):
        assert value(Z.zxp_bind(ps, x)) == amps[x], (seed, x)


@pytest.mark.parametrize("seed", range(6))
def test_some_qubits_parametric_others_fixed(seed):
    rng = random.Random(seed)
    n = 8
    gates = zi.circuit_iid(100 + seed, n, 70)
    params = sorted(rng.sample(range(n), 3))
    fixed = [rng.randrange(2) for _ in range(n)]
    ps = Z.zxp_compile_param(gates, n, fixed, params)
    amps = oracle.amps_all(gates, n)
    for b in range(8):
        bits = list(fixed)
        for j, q in enumerate(params):
            bits[q] = (b >> j) & 1
        x = sum(bit << q for q, bit in enumerate(bits))
        assert value(Z.zxp_bind(ps, b)) == amps[x]


@pytest.mark.parametrize("seed", range(5))
def test_marginal_bits_as_parameters(seed):
    rng = random.Random(50 + seed)
    n = 7
    gates = zi.circuit_iid(200 + seed, n, 60)
    mask_q = sorted(rng.sample(range(n), 3))
    mask = sum(1 << q for q in mask_q)
    params = mask_q[:2]
    ps = Z.zxp_compile_param(gates, n, [0] * n, params, marg_mask=mask, kind=Z.ZXP_MARGINAL_DOUBLED)
    assert ps.info["n_params"] == 2
    for b in range(4):   # the third masked qubit keeps its compile-time bit 0
        bits = [0] * n
        for j, q in enumerate(params):
            bits[q] = (b >> j) & 1
        assert value(Z.zxp_bind(ps, b)) == oracle.marginal(gates, n, mask, bits)


def test_bindings_equal_the_fixed_bit_reduction():
    checked = 0
    for seed in range(40):
        w = zi.workload_batch_item(seed)
        ps = Z.zxp_compile_param(w.gates, w.n, [0] * w.n, list(range(w.n)))
        if ps.info["k"] > 16:
            continue
        rng = random.Random(seed)
        for _ in range(3):
            bits = [rng.randrange(2) for _ in range(w.n)]
            b = sum(bit << q for q, bit in enumerate(bits))
            s_fixed = Z.zxp_compile(w.gates, w.n, bits)
            if s_fixed.info["k"] > 16:
                continue
            assert value(Z.zxp_bind(ps, b)) == value(s_fixed)
            checked += 1
    assert checked >= 10


def test_parameter_limits_and_errors():
    w = zi.workload_small(0)
    ps = Z.zxp_compile_param(w.gates, w.n, [0] * w.n, [0, 2])
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_bind(ps, 1 << 2)            # only two parameters
    assert e.value.code == Z.ZXP_EINVAL
    n = 70
    gates = [(zi.H, q, 0) for q in range(n)]
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_compile_param(gates, n, [0] * n, list(range(65)))
    assert e.value.code == Z.ZXP_EINVAL
    # no parameters: the ordinary reduction
    ps0 = Z.zxp_compile_param(w.gates, w.n, w.out_bits, [])
    assert ps0.info["n_params"] == 0
    assert value(Z.zxp_bind(ps0, 0)) == oracle.amp(w.gates, w.n, w.out_bits)
