"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it draws random circuits,
random output bitstrings and random parametric-scalar tables, and packs them
into the byte layouts that both the oracle and the CUDA library read.  Every
draw comes from one counter-free splitmix64 stream per seed, so the same seed
gives the same circuit on every machine.

Workload recipes follow the paper's experiments (Sec. 4: random Clifford+T
circuits over the gate set {CNOT, H, S, T}); the concrete sizes are the five
workloads this library is measured on:

* ``small``    n=6, 80 gates drawn i.i.d. (CNOT 0.3, H 0.3, S 0.2, T 0.2)
* ``medium``   n=20, 600 gates with exactly 40 T gates (fixed-T)
* ``batch``    512 circuits, n ~ U[10,40], T-count ~ U[20,60]
* ``serve``    Poisson arrivals of amplitude / marginal requests
* ``large``    n=50, 2000 gates with exactly 80 T gates (fixed-T)
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

MASK64 = (1 << 64) - 1

# Gate opcodes (same numbering as the C header's zxp_op).
H, S, T, CNOT, SDG, TDG, X, Z, CZ = range(9)
OP_NAMES = {H: "H", S: "S", T: "T", CNOT: "CNOT", SDG: "Sdg", TDG: "Tdg",
            X: "X", Z: "Z", CZ: "CZ"}
TWO_QUBIT = (CNOT, CZ)


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) (n >= 1)."""
        return self.next_u64() % n

    def between(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def bits(self, n: int) -> List[int]:
        return [self.next_u64() >> 63 for _ in range(n)]


# ----------------------------------------------------------------------------
# circuits
# ----------------------------------------------------------------------------

Gate = Tuple[int, int, int]  # (op, q0, q1); q1 unused (0) for 1-qubit gates


def _draw_pair(rng: SplitMix64, n: int) -> Tuple[int, int]:
    c = rng.below(n)
    t = rng.below(n - 1)
    if t >= c:
        t += 1
    return c, t


def _draw_gate(rng: SplitMix64, n: int, op: int) -> Gate:
    if op in TWO_QUBIT:
        c, t = _draw_pair(rng, n)
        return (op, c, t)
    return (op, rng.below(n), 0)


def circuit_iid(seed: int, n: int, n_gates: int,
                mix=(0.3, 0.3, 0.2, 0.2)) -> List[Gate]:
    """n_gates gates drawn i.i.d. from CNOT/H/S/T with probabilities `mix`."""
    rng = SplitMix64(seed)
    p_cx, p_h, p_s, _ = mix
    out = []
    for _ in range(n_gates):
        u = rng.uniform()
        if u < p_cx:
            op = CNOT
        elif u < p_cx + p_h:
            op = H
        elif u < p_cx + p_h + p_s:
            op = S
        else:
            op = T
        out.append(_draw_gate(rng, n, op))
    return out


def circuit_fixed_t(seed: int, n: int, n_gates: int, t_count: int) -> List[Gate]:
    """Exactly `t_count` T gates at uniformly random positions among
    `n_gates`; the other gates are CNOT/H/S in ratio 0.3 : 0.3 : 0.2."""
    rng = SplitMix64(seed)
    positions = list(range(n_gates))
    # partial Fisher-Yates: the first t_count entries are the T positions
    for i in range(t_count):
        j = i + rng.below(n_gates - i)
        positions[i], positions[j] = positions[j], positions[i]
    t_pos = set(positions[:t_count])
    out = []
    for g in range(n_gates):
        if g in t_pos:
            out.append(_draw_gate(rng, n, T))
            continue
        u = rng.uniform() * 0.8
        op = CNOT if u < 0.3 else (H if u < 0.6 else S)
        out.append(_draw_gate(rng, n, op))
    return out


def circuit_until_t(seed: int, n: int, t_count: int,
                    mix=(0.3, 0.3, 0.2, 0.2)) -> List[Gate]:
    """Gates drawn i.i.d. from the full mix until the T-count reaches t_count."""
    rng = SplitMix64(seed)
    p_cx, p_h, p_s, _ = mix
    out, t_seen = [], 0
    while t_seen < t_count:
        u = rng.uniform()
        if u < p_cx:
            op = CNOT
        elif u < p_cx + p_h:
            op = H
        elif u < p_cx + p_h + p_s:
            op = S
        else:
            op = T
            t_seen += 1
        out.append(_draw_gate(rng, n, op))
    return out


def random_bits(seed: int, n: int) -> List[int]:
    return SplitMix64(seed ^ 0xB175B175B175B175).bits(n)


def t_count(gates: Sequence[Gate]) -> int:
    return sum(1 for g in gates if g[0] in (T, TDG))


# The five measured workloads (see module docstring).
@dataclass
class Workload:
    name: str
    n: int
    gates: List[Gate]
    out_bits: List[int]
    in_bits: List[int] = field(default_factory=list)


def workload_small(seed: int = 0) -> Workload:
    g = circuit_iid(seed, 6, 80)
    return Workload("small n=6 G=80 iid", 6, g, [0] * 6, [0] * 6)


def workload_medium(seed: int = 0) -> Workload:
    g = circuit_fixed_t(seed, 20, 600, 40)
    return Workload("medium n=20 G=600 t=40", 20, g, random_bits(seed, 20), [0] * 20)


def workload_large(seed: int = 0) -> Workload:
    g = circuit_fixed_t(seed, 50, 2000, 80)
    return Workload("large n=50 G=2000 t=80", 50, g, random_bits(seed, 50), [0] * 50)


def workload_large_t50(seed: int = 0) -> Workload:
    """The large circuit shape (n=50, 2000 gates) at T-count 50: seed 0
    reduces to k = 37, a full sum of 1.4e11 terms."""
    g = circuit_fixed_t(seed, 50, 2000, 50)
    return Workload("large n=50 G=2000 t=50", 50, g, random_bits(seed, 50), [0] * 50)


def workload_batch_item(seed: int) -> Workload:
    rng = SplitMix64(seed ^ 0x5EED0BA7C4)
    n = rng.between(10, 40)
    t = rng.between(20, 60)
    g = circuit_until_t(seed, n, t)
    return Workload(f"batch seed={seed} n={n} t={t}", n, g, random_bits(seed, n), [0] * n)


def serve_requests(seed: int, n_req: int, rate_hz: float = 2000.0):
    """Poisson arrivals of amplitude (kind 0) and single-qubit doubled-marginal
    (kind 1) requests on circuits with n ~ U[10,50], T-count ~ U[10,70].
    Returns a list of dicts with arrival time (s), circuit, bits, kind, mask."""
    import math
    rng = SplitMix64(seed ^ 0x5E4E)
    t = 0.0
    reqs = []
    for i in range(n_req):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        n = rng.between(10, 50)
        tc = rng.between(10, 70)
        cseed = rng.next_u64() & 0xFFFFFFFF
        gates = circuit_until_t(cseed, n, tc)
        kind = rng.below(2)
        if kind == 0:
            bits, mask = random_bits(cseed, n), 0
        else:
            q = rng.below(n)
            bits = [0] * n
            bits[q] = rng.below(2)
            mask = 1 << q
        reqs.append(dict(t=t, n=n, gates=gates, bits=bits, kind=kind, mask=mask))
    return reqs


# ----------------------------------------------------------------------------
# gate and scalar byte layouts
# ----------------------------------------------------------------------------

GATE_STRUCT = struct.Struct("<BBHHH")  # op, reserved, q0, q1, reserved


def pack_gates(gates: Sequence[Gate]) -> bytes:
    return b"".join(GATE_STRUCT.pack(op, 0, q0, q1, 0) for op, q0, q1 in gates)


def pack_bits(bits: Sequence[int]) -> bytes:
    return bytes(int(b) & 1 for b in bits)


PS_MAGIC = 0x5350585A  # "ZXPS"
PS_VERSION = 1
PS_VERSION_INNER = 2    # header followed by {u32 k_inner, u32 0}
PS_HEADER = struct.Struct("<IIIIIIIi4q")
PS_INNER = struct.Struct("<II")
PS_LIN = struct.Struct("<QII")
PS_QUAD = struct.Struct("<QQ")
PS_NODE = struct.Struct("<QII")
PS_PAIR = struct.Struct("<QQII")


@dataclass
class PSTables:
    """A parametric scalar in table form.

    value = G / sqrt(2)^e0 * sum over x in {0,1}^k of
        w^(sum_lin c*l(x) + 4*sum_quad lA(x)*lB(x))
        * prod_node (1 + w^(g + 4 l(x)))
        * prod_pair (1 + w^(a + 4 lA) + w^(b + 4 lB) - w^(a + b + 4 (lA xor lB)))
    with w = exp(i pi/4) and l(x) = parity(mask & x).  With k_inner > 0
    (packed as version 2) the last k_inner parameters are inner ones: the
    value is unchanged, but a term index runs over the first k - k_inner
    parameters and each term sums over every value of the inner ones.
    """
    k: int
    e0: int = 0
    G: Tuple[int, int, int, int] = (1, 0, 0, 0)
    lin: List[Tuple[int, int]] = field(default_factory=list)
    quad: List[Tuple[int, int]] = field(default_factory=list)
    node: List[Tuple[int, int]] = field(default_factory=list)
    pair: List[Tuple[int, int, int, int]] = field(default_factory=list)
    k_inner: int = 0

    def pack(self) -> bytes:
        ver = PS_VERSION_INNER if self.k_inner else PS_VERSION
        parts = [PS_HEADER.pack(PS_MAGIC, ver, self.k, len(self.lin),
                                len(self.quad), len(self.node), len(self.pair),
                                self.e0, *[_i64(c) for c in self.G])]
        if self.k_inner:
            parts.append(PS_INNER.pack(self.k_inner, 0))
        parts += [PS_LIN.pack(m, c, 0) for m, c in self.lin]
        parts += [PS_QUAD.pack(a, b) for a, b in self.quad]
        parts += [PS_NODE.pack(m, g, 0) for m, g in self.node]
        parts += [PS_PAIR.pack(ma, mb, a, b) for ma, a, mb, b in self.pair]
        return b"".join(parts)

    @staticmethod
    def unpack(blob: bytes) -> "PSTables":
        h = PS_HEADER.unpack_from(blob, 0)
        if h[0] != PS_MAGIC or h[1] not in (PS_VERSION, PS_VERSION_INNER):
            raise ValueError("not a parametric-scalar table blob")
        k, nl, nq, nn, npair, e0 = h[2], h[3], h[4], h[5], h[6], h[7]
        G = tuple(h[8:12])
        off = PS_HEADER.size
        k_inner = 0
        if h[1] == PS_VERSION_INNER:
            k_inner = PS_INNER.unpack_from(blob, off)[0]
            off += PS_INNER.size
        lin, quad, node, pair = [], [], [], []
        for _ in range(nl):
            m, c, _r = PS_LIN.unpack_from(blob, off); off += PS_LIN.size
            lin.append((m, c))
        for _ in range(nq):
            a, b = PS_QUAD.unpack_from(blob, off); off += PS_QUAD.size
            quad.append((a, b))
        for _ in range(nn):
            m, g, _r = PS_NODE.unpack_from(blob, off); off += PS_NODE.size
            node.append((m, g))
        for _ in range(npair):
            ma, mb, a, b = PS_PAIR.unpack_from(blob, off); off += PS_PAIR.size
            pair.append((ma, a, mb, b))
        return PSTables(k, e0, G, lin, quad, node, pair, k_inner)


def _i64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >> 63 else v


def _rand_mask(rng: SplitMix64, k: int, density: float) -> int:
    if k == 0:
        return 0
    m = 0
    for i in range(k):
        if rng.uniform() < density:
            m |= 1 << i
    if m == 0:
        m = 1 << rng.below(k)
    return m


def synthetic_ps(seed: int, k: int, n_lin: int = 8, n_quad: int = 4,
                 n_node: int = 16, n_pair: int = 0, density: float = 0.25,
                 odd_nodes_only: bool = False, e0: int = 0,
                 G=(1, 0, 0, 0), k_inner: int = 0) -> PSTables:
    """Random tables with the shape of a compiled scalar: k parameters,
    forms of the given mask density, node constants in Z8 (odd only when
    asked), linear coefficients in Z8, and optional phase-pair rows; the
    last k_inner parameters are declared inner (a version-2 table)."""
    rng = SplitMix64(seed * 0x9E3779B1 + k)
    ps = PSTables(k=k, e0=e0, G=tuple(G), k_inner=k_inner)
    for _ in range(n_lin):
        ps.lin.append((_rand_mask(rng, k, density), rng.below(8)))
    for _ in range(n_quad):
        ps.quad.append((_rand_mask(rng, k, density), _rand_mask(rng, k, density)))
    for _ in range(n_node):
        g = 2 * rng.below(4) + 1 if odd_nodes_only else rng.below(8)
        ps.node.append((_rand_mask(rng, k, density), g))
    for _ in range(n_pair):
        ps.pair.append((_rand_mask(rng, k, density), rng.below(8),
                        _rand_mask(rng, k, density), rng.below(8)))
    return ps
