"""CPU oracle for the parametric-scalar exponential sum (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library ``paper_2403_06777_gb300``: the C file ``zxp_oracle.c`` is compiled
on its own with gcc, and the only thing both sides read is the table layout
that ``zxp_inputs`` packs.

Functions and the paper passages they follow (Sutcliffe & Kissinger,
"Fast Classical Simulation of Quantum Circuits via Parametric Rewriting in
the ZX-Calculus"):

* ``ps_sum``       Eq. 2 summed over parameter assignments, subterms by the
                   steps of Sec. 3.3, arithmetic by App. E Lemmas 5 and 6.
* ``ps_term``      one term of Eq. 2.
* ``rows_eval``    the row table of Sec. 3.3 / App. D for one bitstring.
* ``subterm``      the App. C subterm kinds for given parities.
* ``amp``          <out|C|in> from an exact state vector (Sec. 2.2).
* ``amps_all``     every amplitude of C|in>.
* ``marginal``     a marginal probability by the Born rule (Sec. 2.2).
* ``psum_tree``    App. E Algorithm 1 (pairwise tree sum), pure Python.
* ``sample``       weak simulation by chained marginals: Sec. 2.2's product
                   rule, the loop of App. F Algorithm 2 with the conditional
                   ratio P(B||0) / P(B) (Sec. 2.2) in place of P(B||0).
* ``marginal_by_sum``  Sec. 2.2's summing approach, sum_b |amp|^2.
* ``lut``, ``abcd_mul``, ``abcd_add``  single operations, for pinning.

Values come back exact as Python integers: ``(c0, c1, c2, c3, e)`` meaning
(c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^e with w = exp(i pi/4).

Every function has pins in tests/test_oracle.py (closed forms, the paper's
worked values, complex128 evaluations, brute force, invariants).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zxp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libzxp_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP for the multi-threaded sum)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            u64p, i32p, i64p = C.POINTER(C.c_uint64), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
            lib.oracle_ps_sum.argtypes = [C.c_char_p, C.c_size_t, C.c_uint64, C.c_uint64,
                                          C.c_int, u64p, i32p]
            lib.oracle_ps_term.argtypes = [C.c_char_p, C.c_size_t, C.c_uint64, u64p]
            lib.oracle_canon.argtypes = [u64p, C.c_int32, u64p, i32p]
            lib.oracle_rows_eval.argtypes = [u64p, C.c_uint32, C.c_uint32, i64p, C.c_uint64, u64p]
            lib.oracle_abcd_lut.argtypes = [C.c_uint, i64p]
            lib.oracle_abcd_lut.restype = None
            lib.oracle_abcd_mul.argtypes = [i64p, i64p, i64p]
            lib.oracle_abcd_add.argtypes = [i64p, i64p, i64p]
            lib.oracle_subterm.argtypes = [C.c_int, C.c_uint, C.c_uint, C.c_uint, C.c_uint, i64p]
            lib.oracle_amp.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_char_p, C.c_char_p,
                                       u64p, i32p]
            lib.oracle_amps_all.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_char_p, u64p, i32p]
            lib.oracle_marginal.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_char_p, C.c_uint64,
                                            C.c_char_p, u64p, i32p]
            _lib = lib
    return _lib


class OracleOverflow(ArithmeticError):
    """A 128-bit intermediate overflowed: the oracle has no exact answer."""


def _i128(lo: int, hi: int) -> int:
    v = (hi << 64) | lo
    return v - (1 << 128) if v >> 127 else v


def _unpack(buf, e: int) -> Tuple[int, int, int, int, int]:
    return tuple(_i128(buf[2 * i], buf[2 * i + 1]) for i in range(4)) + (int(e),)


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what}: bad input")
    if rc > 0:
        raise OracleOverflow(f"oracle {what}: 128-bit overflow")


def outer_k(blob: bytes) -> int:
    """Parameters the term index runs over: k, less the inner parameters of
    a version-2 table (whose sum is taken inside every term)."""
    k = int.from_bytes(blob[8:12], "little")
    if int.from_bytes(blob[4:8], "little") == 2:
        k -= int.from_bytes(blob[64:68], "little")
    return k


def ps_sum(blob: bytes, first: int = 0, count: int | None = None, nthreads: int = 1):
    """G * sum of the terms with Gray-code index in [first, first+count),
    over sqrt2^e0 (not reduced).  Returns (c0, c1, c2, c3, e0).  For a
    version-2 table the index runs over the outer parameters and each term
    is summed over every value of the inner ones."""
    lib = _load()
    if count is None:
        count = (1 << outer_k(blob)) - first
    out = (C.c_uint64 * 8)()
    e = C.c_int32()
    rc = lib.oracle_ps_sum(blob, len(blob), first, count, nthreads, out, C.byref(e))
    _check(rc, "ps_sum")
    return _unpack(out, e.value)


def ps_term(blob: bytes, x: int):
    """One term of Eq. 2 at parameter bits x (without G): (c0..c3)."""
    lib = _load()
    out = (C.c_uint64 * 8)()
    _check(lib.oracle_ps_term(blob, len(blob), x, out), "ps_term")
    return _unpack(out, 0)[:4]


def canon(c: Sequence[int], e: int):
    """Canonical form: divide by sqrt2 while e > 0 and the numerator allows."""
    lib = _load()
    inp = (C.c_uint64 * 8)()
    for i in range(4):
        v = int(c[i]) & ((1 << 128) - 1)
        inp[2 * i], inp[2 * i + 1] = v & ((1 << 64) - 1), v >> 64
    out = (C.c_uint64 * 8)()
    oe = C.c_int32()
    _check(lib.oracle_canon(inp, e, out, C.byref(oe)), "canon")
    return _unpack(out, oe.value)


def rows_eval(rows: Sequence[Sequence[int]], rows_per_term: int,
              consts: Sequence[Sequence[int]], p: int):
    """Row table (star, a, psi_mask, b, phi_mask) with terms of rows_per_term
    consecutive rows and per-term constants (c0..c3) in the w basis;
    S(p) = sum_i C_i prod_j S_ij(p).  Returns (c0, c1, c2, c3)."""
    lib = _load()
    n_terms = len(rows) // rows_per_term
    flat = (C.c_uint64 * (5 * len(rows)))(*[int(v) & ((1 << 64) - 1) for r in rows for v in r])
    cs = (C.c_int64 * (4 * n_terms))(*[int(v) for c in consts for v in c])
    out = (C.c_uint64 * 8)()
    _check(lib.oracle_rows_eval(flat, n_terms, rows_per_term, cs, p, out), "rows_eval")
    return _unpack(out, 0)[:4]


def subterm(kind: str, a: int, b: int, x: int, y: int):
    """App. C subterm value for parities x (psi) and y (phi), in the w basis.
    kind: 'node' (1+e^{i(a+4x)pi/4}), 'pair' (Eq. 3 with a, b),
    'pi_quad' (e^{i pi x y}), 'pi_lin' (e^{i a x pi/4})."""
    lib = _load()
    kid = {"node": 0, "pair": 1, "pi_quad": 2, "pi_lin": 3}[kind]
    out = (C.c_int64 * 4)()
    _check(lib.oracle_subterm(kid, a, b, x, y, out), "subterm")
    return tuple(out)


def lut(a: int):
    """Doubled (2A, 2B, 2C, 2D) of e^{i pi a/4} from the step-4 table."""
    lib = _load()
    out = (C.c_int64 * 4)()
    lib.oracle_abcd_lut(a, out)
    return tuple(out)


def abcd_mul(p, q):
    lib = _load()
    a, b, out = (C.c_int64 * 4)(*p), (C.c_int64 * 4)(*q), (C.c_int64 * 4)()
    _check(lib.oracle_abcd_mul(a, b, out), "abcd_mul")
    return tuple(out)


def abcd_add(p, q):
    lib = _load()
    a, b, out = (C.c_int64 * 4)(*p), (C.c_int64 * 4)(*q), (C.c_int64 * 4)()
    _check(lib.oracle_abcd_add(a, b, out), "abcd_add")
    return tuple(out)


def _gates_bytes(gates) -> bytes:
    from zxp_inputs import pack_gates
    return gates if isinstance(gates, (bytes, bytearray)) else pack_gates(gates)


def amp(gates, n: int, out_bits: Sequence[int], in_bits: Sequence[int] | None = None):
    """<out|C|in> exactly, canonical (c0, c1, c2, c3, e)."""
    lib = _load()
    gb = _gates_bytes(gates)
    ib = bytes(in_bits) if in_bits is not None else bytes(n)
    out = (C.c_uint64 * 8)()
    e = C.c_int32()
    _check(lib.oracle_amp(gb, len(gb) // 8, n, ib, bytes(out_bits), out, C.byref(e)), "amp")
    return _unpack(out, e.value)


def amps_all(gates, n: int, in_bits: Sequence[int] | None = None):
    """Every <x|C|in>, x in [0, 2^n), canonical."""
    lib = _load()
    gb = _gates_bytes(gates)
    ib = bytes(in_bits) if in_bits is not None else bytes(n)
    out = (C.c_uint64 * (8 << n))()
    es = (C.c_int32 * (1 << n))()
    _check(lib.oracle_amps_all(gb, len(gb) // 8, n, ib, out, es), "amps_all")
    return [_unpack(out[8 * x:8 * x + 8], es[x]) for x in range(1 << n)]


def marginal(gates, n: int, mask: int, bits: Sequence[int],
             in_bits: Sequence[int] | None = None):
    """P(qubit q reads bits[q] for q in mask) of C|in>, canonical."""
    lib = _load()
    gb = _gates_bytes(gates)
    ib = bytes(in_bits) if in_bits is not None else bytes(n)
    out = (C.c_uint64 * 8)()
    e = C.c_int32()
    _check(lib.oracle_marginal(gb, len(gb) // 8, n, ib, mask, bytes(bits), out, C.byref(e)),
           "marginal")
    return _unpack(out, e.value)


def psum_tree(arr: List, add=lambda a, b: a + b, trace: list | None = None):
    """App. E Algorithm 1: repeated pairwise passes with split = 2, 4, 8, ...
    and gap = split/2; in each pass element i*split gains element
    i*split + gap when that index is inside the array.  (The printed bound
    elem + gap < N_ELEMS - 1 would skip the last element of the worked
    example, whose printed total 45 needs elem + gap < N_ELEMS.)"""
    a = list(arr)
    n = len(a)
    split, gap = 2, 1
    while gap < n:
        n_chunks = -(-n // split)
        for i in range(n_chunks):          # the n_chunks "threads" of one launch
            elem = i * split
            if elem + gap < n:
                a[elem] = add(a[elem], a[elem + gap])
        if trace is not None:
            trace.append(list(a))
        split *= 2
        gap *= 2
    return a[0] if a else None


def to_complex(v) -> complex:
    """(c0, c1, c2, c3, e) -> complex, for checks against floating point."""
    import cmath
    w = cmath.exp(1j * cmath.pi / 4)
    c0, c1, c2, c3, e = v
    return (c0 + c1 * w + c2 * w ** 2 + c3 * w ** 3) / (2 ** 0.5) ** e


_INV_SQRT2 = 0.70710678118654752440


def real_value(v) -> float:
    """The real part of an exact value as a double, by one fixed sequence of
    IEEE operations: (c0 + (c1 - c3) / sqrt2), an extra 1/sqrt2 for odd e,
    then the power of two 2^(-e/2) (exact)."""
    import math
    c0, c1, c2, c3, e = v
    r = float(c0) + float(c1 - c3) * _INV_SQRT2
    if e & 1:
        r *= _INV_SQRT2
        e -= 1
    return math.ldexp(r, -(e // 2))


def _sub(a, b):
    """a - b exactly (common sqrt2 exponent), canonical."""
    def up(v):   # x sqrt2 = (c1 - c3) + (c0 + c2) w + (c1 + c3) w^2 + (c2 - c0) w^3
        c0, c1, c2, c3, e = v
        return (c1 - c3, c0 + c2, c1 + c3, c2 - c0, e + 1)
    while a[4] < b[4]:
        a = up(a)
    while b[4] < a[4]:
        b = up(b)
    return canon([a[i] - b[i] for i in range(4)], a[4])


def sample(gates, n: int, u_rows, in_bits: Sequence[int] | None = None):
    """Draw one bitstring per row of uniforms: for qubit j = 0 .. n-1, bit j is
    0 when u[j] < P(B || 0) / P(B) (exact marginals of the state vector, the
    ratio as doubles by real_value), else 1.  Returns (bitstrings, exact
    probabilities of the drawn bitstrings)."""
    out, probs = [], []
    for u in u_rows:
        pB = (1, 0, 0, 0, 0)
        bits = [0] * n
        for j in range(n):
            mask = (2 << j) - 1
            bits[j] = 0
            p0 = marginal(gates, n, mask, bits, in_bits)
            if u[j] < real_value(p0) / real_value(pB):
                pB = p0
            else:
                bits[j] = 1
                pB = _sub(pB, p0)
        out.append(list(bits))
        probs.append(pB)
    return out, probs


def marginal_by_sum(gates, n: int, mask: int, bits: Sequence[int],
                    in_bits: Sequence[int] | None = None):
    """P(qubits in mask read bits) as sum over the other bits of |amp|^2,
    exact (Sec. 2.2, summing approach)."""
    amps = amps_all(gates, n, in_bits)
    acc = None
    want = sum((int(bits[q]) & 1) << q for q in range(n) if (mask >> q) & 1)
    for x, a in enumerate(amps):
        if (x & mask) != want:
            continue
        c0, c1, c2, c3, e = a
        r = (c0 * c0 + c1 * c1 + c2 * c2 + c3 * c3,
             c1 * c0 + c2 * c1 + c3 * c2 - c0 * c3,
             c2 * c0 + c3 * c1 - c0 * c2 - c1 * c3,
             c3 * c0 - c0 * c1 - c1 * c2 - c2 * c3, 2 * e)
        if acc is None:
            acc = r
        else:
            acc = _sub(acc, (-r[0], -r[1], -r[2], -r[3], r[4]))
    return canon(acc[:4], acc[4]) if acc else (0, 0, 0, 0, 0)
