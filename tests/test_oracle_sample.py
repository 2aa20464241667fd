"""Pins of the oracle's weak-simulation sampler and summing marginal (no
GPU): closed forms, forced outcomes, and the empirical distribution of many
draws against the exact Born probabilities (which only the conditional
ratio of Sec. 2.2 reproduces)."""
import random

import oracle
import zxp_inputs as zi

H, S, T, CNOT = zi.H, zi.S, zi.T, zi.CNOT


def test_single_qubit_closed_form():
    # H T H |0>: P(0) = |(1 + w)/2|^2 = (2 + sqrt2)/4
    g = [(H, 0, 0), (T, 0, 0), (H, 0, 0)]
    p0 = oracle.marginal(g, 1, 1, [0])
    assert p0 == (1, 1, 0, -1, 3)                       # (1 + sqrt2) / (2 sqrt2)
    assert abs(oracle.real_value(p0) - (2 + 2 ** 0.5) / 4) < 1e-15
    bits, probs = oracle.sample(g, 1, [[0.8535], [0.8536], [0.0], [0.999]])
    assert bits == [[0], [1], [0], [1]]
    assert probs[1] == (-1, 1, 0, -1, 3)                # (2 - sqrt2) / 4
    assert oracle.marginal_by_sum(g, 1, 1, [0]) == p0


def test_forced_second_bit_of_a_bell_state():
    g = [(H, 0, 0), (CNOT, 0, 1)]
    rng = random.Random(3)
    rows = [[rng.random(), rng.random()] for _ in range(50)]
    bits, probs = oracle.sample(g, 2, rows)
    for u, b, p in zip(rows, bits, probs):
        assert b[0] == (0 if u[0] < 0.5 else 1) and b[1] == b[0]
        assert p == (1, 0, 0, 0, 2)


def test_uniform_outputs():
    g = [(H, q, 0) for q in range(3)]
    rng = random.Random(4)
    rows = [[rng.random() for _ in range(3)] for _ in range(40)]
    bits, probs = oracle.sample(g, 3, rows)
    for u, b, p in zip(rows, bits, probs):
        assert b == [0 if x < 0.5 else 1 for x in u]
        assert p == (1, 0, 0, 0, 6)


def test_draws_follow_the_born_distribution():
    n = 4
    g = zi.circuit_iid(17, n, 40)
    amps = oracle.amps_all(g, n)
    exact = [abs(oracle.to_complex(a)) ** 2 for a in amps]
    rng = random.Random(11)
    rows = [[rng.random() for _ in range(n)] for _ in range(4000)]
    bits, probs = oracle.sample(g, n, rows)
    counts = [0] * (1 << n)
    for b, p in zip(bits, probs):
        x = sum(v << q for q, v in enumerate(b))
        counts[x] += 1
        assert abs(oracle.real_value(p) - exact[x]) < 1e-12   # the drawn string's probability
    tv = 0.5 * sum(abs(c / len(rows) - e) for c, e in zip(counts, exact))
    assert tv < 0.04, tv


def test_summing_marginal_equals_the_born_rule():
    rng = random.Random(5)
    for seed in range(6):
        n = 5
        g = zi.circuit_iid(300 + seed, n, 50)
        mask = rng.randrange(1, 1 << n)
        bits = [rng.randrange(2) for _ in range(n)]
        assert oracle.marginal_by_sum(g, n, mask, bits) == oracle.marginal(g, n, mask, bits)
