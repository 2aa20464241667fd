"""Pins of the CPU oracle against things other than itself.

Each check would fail on a plausible mistake in the oracle: a wrong table
entry (step-4 look-up), a transposed operand or sign in Lemma 6, a dropped
subterm, a wrong parity, a wrong gate matrix or a wrong sqrt2 reduction.
The independent references are complex128 evaluations written here from the
definitions (cmath.exp of the phases, numpy gate matrices), the paper's
printed worked values (tests/golden), closed forms and exact invariants.
"""
import cmath
import itertools
import math
import os
import random

import numpy as np
import pytest

import oracle
import zxp_inputs as zi

W = cmath.exp(1j * math.pi / 4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def abcd_to_complex(h):
    a2, b2, c2, d2 = h
    return a2 / 2 + b2 / 2 * math.sqrt(2) + 1j * (c2 / 2 + d2 / 2 * math.sqrt(2))


def wc(c):
    return sum(c[i] * W ** i for i in range(4))


def close(a, b, scale=1.0):
    return abs(a - b) <= 1e-9 * max(1.0, scale, abs(a), abs(b))


# --------------------------------------------------------------------------
# step-4 table, Lemma 5, Lemma 6
# --------------------------------------------------------------------------

def test_lut_is_exp_i_pi_a_over_4():
    for a in range(8):
        assert close(abcd_to_complex(oracle.lut(a)), cmath.exp(1j * math.pi * a / 4))


def _rand_zw_abcd(rng, lim):
    # doubled (2A, 2B, 2C, 2D) of an element of Z[w]: A, C integers, B = D mod 1
    A, C = rng.randint(-lim, lim), rng.randint(-lim, lim)
    b2 = rng.randint(-lim, lim)
    d2 = b2 + 2 * rng.randint(-lim, lim)
    return (2 * A, b2, 2 * C, d2)


def test_lemma5_lemma6_against_complex():
    rng = random.Random(5)
    for _ in range(2000):
        p, q = _rand_zw_abcd(rng, 1000), _rand_zw_abcd(rng, 1000)
        cp, cq = abcd_to_complex(p), abcd_to_complex(q)
        assert close(abcd_to_complex(oracle.abcd_mul(p, q)), cp * cq, abs(cp) * abs(cq))
        assert close(abcd_to_complex(oracle.abcd_add(p, q)), cp + cq, abs(cp) + abs(cq))


# --------------------------------------------------------------------------
# subterm kinds (App. C) and the closed identities of the paper
# --------------------------------------------------------------------------

def test_phase_pair_matches_eq3_and_zx_pair_scalar():
    # Eq. 3 / the Z(alpha)-X(beta) scalar of Fig. 1:
    # sqrt2 * diagram = 1 + e^{i alpha} + e^{i beta} - e^{i(alpha + beta)}
    for a, b, x, y in itertools.product(range(8), range(8), range(2), range(2)):
        psi = math.pi / 4 * (a + 4 * x)
        phi = math.pi / 4 * (b + 4 * y)
        want = 1 + cmath.exp(1j * psi) + cmath.exp(1j * phi) - cmath.exp(1j * (psi + phi))
        assert close(wc(oracle.subterm("pair", a, b, x, y)), want)


def test_node_matches_isolated_spider():
    # isolated Z(alpha) spider = 1 + e^{i alpha} (Fig. 1)
    for a, x in itertools.product(range(8), range(2)):
        want = 1 + cmath.exp(1j * math.pi / 4 * (a + 4 * x))
        assert close(wc(oracle.subterm("node", a, 0, x, 0)), want)


def test_pi_pair_lemma_cases():
    # App. C lemma: e^{i Psi Phi/pi} = 1/2 (1 + e^{iPsi} + e^{iPhi} - e^{i(Psi+Phi)})
    # when Phi is 0 or pi; both printed cases (Phi = 0 and Phi = pi).
    for a, y in itertools.product(range(8), range(2)):
        lin = oracle.subterm("pi_lin", a, 0, y, 0)         # e^{i (a pi/4)(pi y)/pi}
        pair = oracle.subterm("pair", a, 0, 0, y)          # Psi = a pi/4, Phi = pi y
        assert tuple(2 * v for v in lin) == pair
        assert close(wc(lin), cmath.exp(1j * math.pi / 4 * a * y))
    for x, y in itertools.product(range(2), range(2)):
        q = oracle.subterm("pi_quad", 0, 0, x, y)
        assert close(wc(q), (-1) ** (x * y))
        assert tuple(2 * v for v in q) == oracle.subterm("pair", 0, 0, x, y)


def test_node_to_phase_pair_constant():
    # App. C node lemma, read with C = (1 - i)/2 (the printed sqrt2/4 (1-i)
    # misses a factor sqrt2): 1 + e^{iPsi} = C (1 + e^{iPsi'} + i - e^{i(Psi'+pi/2)}),
    # Psi' = Psi + pi/2.  Exact check: 2 node = (1 - i) pair.
    one_minus_i = (1, 0, -1, 0)
    for a in range(8):
        node = oracle.subterm("node", a, 0, 0, 0)
        pair = oracle.subterm("pair", (a + 2) % 8, 2, 0, 0)
        lhs = [2 * v for v in node]
        rhs = _wmul(one_minus_i, pair)
        assert lhs == rhs
        assert close(wc(node), 0.5 * (1 - 1j) * wc(pair))


def test_half_pi_reading():
    # App. C half-pi lemma, read as e^{i Psi/2} = (w/2)(1 + e^{i(Psi - pi/2)} + i - e^{i Psi})
    # for Psi in {pi/2, 3pi/2}.
    for psi4 in (2, 6):
        pair = oracle.subterm("pair", (psi4 - 2) % 8, 2, 0, 0)
        val = 0.5 * W * wc(pair)
        assert close(val, cmath.exp(1j * math.pi / 4 * psi4 / 2))


def _wmul(p, q):
    t = [0, 0, 0, 0]
    for i in range(4):
        for j in range(4):
            if i + j < 4:
                t[i + j] += p[i] * q[j]
            else:
                t[i + j - 4] -= p[i] * q[j]
    return t


def test_conclusion_pair_cancellation_identities():
    # Sec. 5: (1 + e^{i pi (2/4 + a xor b)})(1 + e^{i pi (6/4 + a xor b)}) = 2 for
    # both values of a xor b, and constants 0 and pi give 0.
    ps = zi.PSTables(k=2, node=[(0b11, 2), (0b11, 6)])
    for x in range(4):
        assert oracle.ps_term(ps.pack(), x) == (2, 0, 0, 0)
    ps0 = zi.PSTables(k=2, node=[(0b11, 0), (0b11, 4)])
    for x in range(4):
        assert oracle.ps_term(ps0.pack(), x) == (0, 0, 0, 0)


# --------------------------------------------------------------------------
# App. E Algorithm 1 and the App. D worked table
# --------------------------------------------------------------------------

def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_algorithm1_trace():
    rows = _read_golden("alg1_trace.txt")
    inp = [int(v) for v in rows[0][1:]]
    passes = [[int(v) for v in r[1:]] for r in rows if r[0] == "pass"]
    total = int(rows[-1][1])
    trace = []
    assert oracle.psum_tree(inp, trace=trace) == total
    assert trace == passes
    # the same tree multiplies as well as it sums (App. E)
    assert oracle.psum_tree([1, 2, 3, 4, 5], add=lambda a, b: a * b) == 120
    rng = random.Random(1)
    for n in range(1, 40):
        arr = [rng.randint(-99, 99) for _ in range(n)]
        assert oracle.psum_tree(arr) == sum(arr)


def test_app_d_table_against_complex():
    rows = [[int(v) for v in r] for r in _read_golden("app_d_rows.txt")]
    table = []
    for r in rows:
        psi = sum(r[2 + j] << j for j in range(4))
        phi = sum(r[7 + j] << j for j in range(4))
        table.append((r[0], r[1], psi, r[6], phi))
    for p in range(16):
        got = wc(oracle.rows_eval(table, 3, [(1, 0, 0, 0), (1, 0, 0, 0)], p))
        want = 0
        for t in range(2):
            prod = 1
            for star, a, pm, b, fm in table[3 * t:3 * t + 3]:
                if not star:
                    continue
                x = bin(pm & p).count("1") & 1
                y = bin(fm & p).count("1") & 1
                psi = math.pi / 4 * a + math.pi * x
                phi = math.pi / 4 * b + math.pi * y
                prod *= 1 + cmath.exp(1j * psi) + cmath.exp(1j * phi) - cmath.exp(1j * (psi + phi))
            want += prod
        assert close(got, want, 10.0)


# --------------------------------------------------------------------------
# the exponential sum
# --------------------------------------------------------------------------

def complex_term(ps, x):
    par = lambda m: bin(m & x).count("1") & 1
    ph = sum(c * par(m) for m, c in ps.lin) + 4 * sum(par(a) * par(b) for a, b in ps.quad)
    v = cmath.exp(1j * math.pi / 4 * ph)
    for m, g in ps.node:
        v *= 1 + cmath.exp(1j * math.pi / 4 * (g + 4 * par(m)))
    for ma, a, mb, b in ps.pair:
        A = math.pi / 4 * (a + 4 * par(ma))
        B = math.pi / 4 * (b + 4 * par(mb))
        v *= 1 + cmath.exp(1j * A) + cmath.exp(1j * B) - cmath.exp(1j * (A + B))
    return v


@pytest.mark.parametrize("seed", range(12))
def test_ps_sum_brute_force_complex(seed):
    rng = random.Random(seed)
    k = rng.randint(0, 8)
    ps = zi.synthetic_ps(seed, k, n_lin=rng.randint(0, 6), n_quad=rng.randint(0, 4),
                         n_node=rng.randint(0, 8), n_pair=rng.randint(0, 3),
                         density=0.4, e0=rng.randint(0, 6),
                         G=(rng.randint(-3, 3), rng.randint(-3, 3), 1, 0))
    blob = ps.pack()
    v = oracle.ps_sum(blob)
    want = wc(ps.G) * sum(complex_term(ps, x) for x in range(1 << k)) / math.sqrt(2) ** ps.e0
    assert v[4] == ps.e0
    assert close(oracle.to_complex(v), want, 1e3)
    for x in range(1 << k):
        assert close(wc(oracle.ps_term(blob, x)), complex_term(ps, x), 1e3)


def test_ps_sum_ranges_add_up_and_threads_agree():
    ps = zi.synthetic_ps(3, 10, n_lin=5, n_quad=3, n_node=10, n_pair=2)
    blob = ps.pack()
    full = oracle.ps_sum(blob)
    for cut in (0, 1, 333, 512, 1023, 1024):
        a = oracle.ps_sum(blob, 0, cut)
        b = oracle.ps_sum(blob, cut, 1024 - cut)
        assert tuple(a[i] + b[i] for i in range(4)) == full[:4]
    assert oracle.ps_sum(blob, nthreads=4) == full
    # the full Gray-ordered sum equals the natural-order sum of single terms
    s = [0, 0, 0, 0]
    for x in range(1024):
        t = oracle.ps_term(blob, x)
        s = [s[i] + t[i] for i in range(4)]
    assert tuple(s) == full[:4]  # G = 1
    assert oracle.ps_sum(blob, 5, 0)[:4] == (0, 0, 0, 0)


@pytest.mark.parametrize("seed", range(10))
def test_ps_sum_inner_parameters_brute_force_complex(seed):
    # version-2 tables: the full value is Eq. 2 over all 2^k assignments, and
    # the term of outer Gray index t sums the inner parameters at gray(t)
    rng = random.Random(100 + seed)
    k = rng.randint(1, 9)
    ki = rng.randint(1, k)
    ko = k - ki
    ps = zi.synthetic_ps(200 + seed, k, n_lin=rng.randint(0, 6), n_quad=rng.randint(0, 4),
                         n_node=rng.randint(0, 8), n_pair=rng.randint(0, 2),
                         density=0.4, e0=rng.randint(0, 6),
                         G=(rng.randint(-3, 3), 1, rng.randint(-2, 2), 0), k_inner=ki)
    blob = ps.pack()
    assert oracle.outer_k(blob) == ko
    v = oracle.ps_sum(blob)
    want = wc(ps.G) * sum(complex_term(ps, x) for x in range(1 << k)) / math.sqrt(2) ** ps.e0
    assert v[4] == ps.e0
    assert close(oracle.to_complex(v), want, 1e3)
    for t in range(1 << ko):
        g = t ^ (t >> 1)
        term = wc(ps.G) * sum(complex_term(ps, g | (y << ko)) for y in range(1 << ki))
        assert close(oracle.to_complex(oracle.ps_sum(blob, t, 1)), term / math.sqrt(2) ** ps.e0, 1e3)


def test_ps_sum_inner_parameters_ranges_add_up():
    ps = zi.synthetic_ps(7, 10, n_lin=6, n_quad=3, n_node=9, n_pair=2, k_inner=4)
    blob = ps.pack()
    full = oracle.ps_sum(blob)
    assert oracle.ps_sum(zi.synthetic_ps(7, 10, n_lin=6, n_quad=3, n_node=9, n_pair=2).pack()) == full
    for cut in (0, 1, 17, 32, 63, 64):
        a = oracle.ps_sum(blob, 0, cut)
        b = oracle.ps_sum(blob, cut, 64 - cut)
        assert tuple(a[i] + b[i] for i in range(4)) == full[:4]
    assert oracle.ps_sum(blob, nthreads=3) == full
    with pytest.raises(ValueError):
        oracle.ps_sum(blob, 0, 65)


def test_ps_forms_of_a_known_amplitude():
    # <0|H T H|0> = (1 + w)/2, written three ways
    want = (1, 1, 0, 0, 2)
    lin = zi.PSTables(k=1, e0=2, lin=[(1, 1)])           # (1/2) sum_y w^y
    node = zi.PSTables(k=0, e0=2, node=[(0, 1)])         # (1/2)(1 + w)
    pair = zi.PSTables(k=0, e0=4, G=(1, 0, -1, 0), pair=[(0, 3, 0, 2)])  # node as phase-pair
    for ps in (lin, node, pair):
        v = oracle.ps_sum(ps.pack())
        assert oracle.canon(v[:4], v[4]) == want
    assert oracle.amp([(zi.H, 0, 0), (zi.T, 0, 0), (zi.H, 0, 0)], 1, [0]) == want


def test_ps_sum_reports_overflow_and_bad_input():
    with pytest.raises(ValueError):
        oracle.ps_sum(b"junk" * 20)
    big = zi.PSTables(k=2, node=[(0, 0)] * 140)   # 2^140 per term
    with pytest.raises(oracle.OracleOverflow):
        oracle.ps_sum(big.pack())


# --------------------------------------------------------------------------
# the state vector
# --------------------------------------------------------------------------

def numpy_statevector(gates, n, in_bits=None):
    psi = np.zeros(1 << n, dtype=np.complex128)
    idx = sum((in_bits[q] if in_bits else 0) << q for q in range(n))
    psi[idx] = 1
    Hm = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    diag = {zi.S: 1j, zi.T: W, zi.SDG: -1j, zi.TDG: np.conj(W), zi.Z: -1}
    ar = np.arange(1 << n)
    for op, q0, q1 in gates:
        if op == zi.H or op == zi.X:
            M = Hm if op == zi.H else np.array([[0, 1], [1, 0]])
            v = psi.reshape(1 << (n - q0 - 1), 2, 1 << q0)
            psi = np.einsum("ab,ibj->iaj", M, v).reshape(-1)
        elif op in diag:
            psi = np.where((ar >> q0) & 1, psi * diag[op], psi)
        elif op == zi.CNOT:
            src = np.where((ar >> q0) & 1, ar ^ (1 << q1), ar)
            psi = psi[src]
        elif op == zi.CZ:
            psi = np.where(((ar >> q0) & 1) & ((ar >> q1) & 1), -psi, psi)
    return psi


@pytest.mark.parametrize("seed", range(8))
def test_amp_against_numpy_statevector(seed):
    n = 1 + seed % 6
    gates = zi.circuit_iid(seed, n, 40) if n > 1 else [(op, 0, 0) for op, _, _ in
                                                         zi.circuit_iid(seed, 2, 40) if op != zi.CNOT]
    gates += [(zi.SDG, 0, 0), (zi.TDG, n - 1, 0), (zi.X, 0, 0), (zi.Z, n - 1, 0)]
    if n > 1:
        gates.append((zi.CZ, 0, n - 1))
    in_bits = zi.random_bits(seed + 100, n)
    psi = numpy_statevector(gates, n, in_bits)
    amps = oracle.amps_all(gates, n, in_bits)
    for x in range(1 << n):
        assert close(oracle.to_complex(amps[x]), psi[x])
    out = zi.random_bits(seed, n)
    xo = sum(b << q for q, b in enumerate(out))
    assert oracle.amp(gates, n, out, in_bits) == amps[xo]


def _norm2(v):
    c = v[:4]
    cj = (c[0], -c[3], -c[2], -c[1])
    return _wmul(c, cj), v[4]


@pytest.mark.parametrize("seed", range(4))
def test_born_rule_sums_to_one_exactly(seed):
    n = 6
    gates = zi.workload_small(seed).gates
    amps = oracle.amps_all(gates, n)
    emax = max(a[4] for a in amps)
    tot = [0, 0, 0, 0]
    for a in amps:
        m, e = _norm2(a)
        tot = [tot[i] + m[i] * 2 ** (emax - e) for i in range(4)]
    assert tot == [2 ** emax, 0, 0, 0]
    # marginals: P(q=0) + P(q=1) = 1, and each equals the sum of |amp|^2
    for q in range(n):
        p0 = oracle.marginal(gates, n, 1 << q, [0] * n)
        bits1 = [0] * n
        bits1[q] = 1
        p1 = oracle.marginal(gates, n, 1 << q, bits1)
        assert close(oracle.to_complex(p0) + oracle.to_complex(p1), 1.0)
        assert close(oracle.to_complex(p0),
                     sum(abs(oracle.to_complex(amps[x])) ** 2 for x in range(1 << n)
                         if not (x >> q) & 1))


def test_clifford_amplitudes_are_units_over_sqrt2_powers():
    for seed in range(6):
        gates = [g for g in zi.circuit_iid(seed, 5, 60) if g[0] != zi.T]
        for a in oracle.amps_all(gates, 5):
            nz = [c for c in a[:4] if c != 0]
            assert nz == [] or (len(nz) == 1 and abs(nz[0]) == 1)


def test_closed_form_amplitudes():
    n = 4
    hs = [(zi.H, q, 0) for q in range(n)]
    assert oracle.amp(hs, n, [0] * n) == (1, 0, 0, 0, 4)          # 1/sqrt2^4
    assert oracle.amp([(zi.H, 0, 0), (zi.T, 0, 0)], 1, [1]) == (0, 1, 0, 0, 1)   # w/sqrt2
    assert oracle.amp([(zi.X, 0, 0), (zi.CNOT, 0, 1)], 2, [1, 1]) == (1, 0, 0, 0, 0)
    assert oracle.amp([], 3, [0, 0, 1]) == (0, 0, 0, 0, 0)


def test_canon_divides_sqrt2_only_when_exact():
    assert oracle.canon((2, 0, 0, 0), 2) == (1, 0, 0, 0, 0)      # 2/2 = 1
    assert oracle.canon((1, 0, 1, 0), 1) == (0, 1, 0, 0, 0)      # (1+i)/sqrt2 = w
    assert oracle.canon((1, 0, 0, 0), 3) == (1, 0, 0, 0, 3)
    assert oracle.canon((0, 0, 0, 0), 7) == (0, 0, 0, 0, 0)
    assert oracle.canon((4, 0, 0, 0), 0) == (4, 0, 0, 0, 0)
