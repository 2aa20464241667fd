"""Python binding of libzxp (argument marshalling only).

Every function keeps the C name of include/zxp.h.  The library must have
been built (``paper_2403_06777_gb300._build.build()`` or
``__graft_entry__.build()``); importing the package does not build it, and
every call fails with an error when the shared object is missing.  There is
no CPU fallback: GPU entry points raise ``ZxpError`` (ZXP_ECUDA) without a
device.

Scalars are returned as tuples ``(c0, c1, c2, c3, e)`` meaning
(c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^e with w = exp(i pi/4).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libzxp.so")

ZXP_OK, ZXP_EINVAL, ZXP_ENOMEM, ZXP_ETOOBIG, ZXP_EOVERFLOW = 0, -1, -2, -3, -4
ZXP_ECUDA, ZXP_ETIMEDOUT, ZXP_EAGAIN, ZXP_ENOTFOUND = -5, -6, -7, -8
ZXP_AMPLITUDE, ZXP_MARGINAL_DOUBLED = 0, 1


class ZxpError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {zxp_strerror(code)} ({code})" if what else zxp_strerror(code))


class zxp_zomega(C.Structure):
    _fields_ = [("c", C.c_int64 * 4), ("e", C.c_int32), ("flags", C.c_int32)]

    def tup(self) -> Tuple[int, int, int, int, int]:
        return (self.c[0], self.c[1], self.c[2], self.c[3], self.e)


class zxp_zomega_wide(C.Structure):
    _fields_ = [("c", C.c_int64 * 4), ("hi", C.c_int64 * 4), ("e", C.c_int32), ("flags", C.c_int32)]

    def tup(self) -> Tuple[int, int, int, int, int]:
        """(c0, c1, c2, c3, e), each coefficient the signed 128-bit integer."""
        v = []
        for i in range(4):
            x = ((self.hi[i] & ((1 << 64) - 1)) << 64) | (self.c[i] & ((1 << 64) - 1))
            v.append(x - (1 << 128) if x >> 127 else x)
        return (v[0], v[1], v[2], v[3], self.e)


class zxp_scalar_info_t(C.Structure):
    _fields_ = [("k", C.c_uint32), ("n_lin", C.c_uint32), ("n_quad", C.c_uint32),
                ("n_node", C.c_uint32), ("n_pair", C.c_uint32), ("e0", C.c_int32),
                ("acc_bits", C.c_uint32), ("form_bits", C.c_uint32), ("t_count", C.c_uint32),
                ("node_words", C.c_uint32), ("other_words", C.c_uint32),
                ("device_bytes", C.c_uint32), ("kernel_variant", C.c_uint32),
                ("k_inner", C.c_uint32), ("inner_bits", C.c_uint32),
                ("upload_bytes", C.c_uint32)]


class zxp_split_opts(C.Structure):
    _fields_ = [("min_k", C.c_uint32), ("max_inner", C.c_uint32), ("max_index_bits", C.c_uint32),
                ("max_cut", C.c_uint32), ("low_free", C.c_uint32), ("tries", C.c_uint32),
                ("seed", C.c_uint64), ("reserved", C.c_uint32 * 4)]


class zxp_batch_info_t(C.Structure):
    _fields_ = [("n_scalars", C.c_uint32), ("n_groups", C.c_uint32), ("n_chunks", C.c_uint32),
                ("threads", C.c_uint32), ("chunk_log2", C.c_uint32), ("candidates", C.c_uint32),
                ("tuned_us", C.c_double), ("total_terms", C.c_double),
                ("reserved", C.c_uint32 * 6)]


class zxp_server_opts(C.Structure):
    _fields_ = [("policy", C.c_uint32), ("max_k", C.c_uint32), ("compile_threads", C.c_uint32),
                ("max_active", C.c_uint32), ("arena_bytes", C.c_uint64), ("step_terms", C.c_uint64),
                ("small_terms", C.c_uint64), ("chunk_log2", C.c_uint32), ("threads", C.c_uint32),
                ("reserved", C.c_uint32 * 8)]


class zxp_request(C.Structure):
    _fields_ = [("gates", C.c_char_p), ("n_gates", C.c_size_t), ("n_qubits", C.c_int32),
                ("kind", C.c_int32), ("in_bits", C.c_char_p), ("out_bits", C.c_char_p),
                ("marg_mask", C.c_uint64)]


class zxp_request_timing(C.Structure):
    _fields_ = [("submit_us", C.c_double), ("compiled_us", C.c_double),
                ("admitted_us", C.c_double), ("done_us", C.c_double), ("k", C.c_uint32),
                ("steps", C.c_uint32), ("status", C.c_int32), ("reserved", C.c_uint32)]


class zxp_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("steps", C.c_uint64), ("launches", C.c_uint64), ("terms", C.c_double),
                ("device_busy_us", C.c_double), ("active", C.c_uint32),
                ("peak_active", C.c_uint32), ("arena_bytes", C.c_uint64),
                ("arena_peak", C.c_uint64), ("reserved", C.c_uint32 * 8)]


ZXP_SERVE_BATCHED, ZXP_SERVE_PLAIN = 0, 1


class zxp_pscalar_info_t(C.Structure):
    _fields_ = [("k", C.c_uint32), ("n_params", C.c_uint32), ("n_lin", C.c_uint32),
                ("n_quad", C.c_uint32), ("n_node", C.c_uint32), ("n_pair", C.c_uint32),
                ("e0", C.c_int32), ("t_count", C.c_uint32), ("reserved", C.c_uint32 * 8)]

_lib = None


def lib():
    """The loaded libzxp (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libzxp.so is not built ({LIB_PATH}); run "
                              "paper_2403_06777_gb300._build.build()")
        L = C.CDLL(LIB_PATH)
        vp, u64, i64, sz = C.c_void_p, C.c_uint64, C.c_int64, C.c_size_t
        zp = C.POINTER(zxp_zomega)
        L.zxp_strerror.argtypes, L.zxp_strerror.restype = [C.c_int], C.c_char_p
        L.zxp_version.argtypes, L.zxp_version.restype = [], C.c_char_p
        L.zxp_ctx_create.argtypes = [C.c_int, vp, C.POINTER(vp)]
        L.zxp_ctx_destroy.argtypes, L.zxp_ctx_destroy.restype = [vp], None
        L.zxp_compile.argtypes = [C.c_char_p, sz, C.c_int, C.c_char_p, C.c_char_p, u64, C.c_int,
                                  C.POINTER(vp)]
        L.zxp_compile_ex.argtypes = [C.c_char_p, sz, C.c_int, C.c_char_p, C.c_char_p, u64, C.c_int,
                                     C.POINTER(zxp_split_opts), C.POINTER(vp)]
        L.zxp_scalar_from_tables.argtypes = [C.c_char_p, sz, C.POINTER(vp)]
        L.zxp_scalar_to_tables.argtypes = [vp, vp, C.POINTER(sz)]
        L.zxp_scalar_info.argtypes = [vp, C.POINTER(zxp_scalar_info_t)]
        L.zxp_scalar_free.argtypes, L.zxp_scalar_free.restype = [vp], None
        L.zxp_scalar_split.argtypes = [vp, C.POINTER(zxp_split_opts), C.POINTER(vp)]
        L.zxp_scalar_reorder.argtypes = [vp, C.POINTER(vp)]
        L.zxp_inner_sum.argtypes = [vp, vp]
        L.zxp_eval.argtypes = [vp, vp, u64, u64, zp]
        L.zxp_amplitude.argtypes = [vp, vp, zp]
        L.zxp_eval_wide.argtypes = [vp, vp, u64, u64, C.POINTER(zxp_zomega_wide)]
        L.zxp_amplitude_wide.argtypes = [vp, vp, C.POINTER(zxp_zomega_wide)]
        L.zxp_sum_resumable.argtypes = [vp, vp, C.c_uint32, C.c_char_p, u64, zp, C.POINTER(u64),
                                        C.POINTER(u64)]
        L.zxp_eval_device.argtypes = [vp, vp, u64, u64, vp]
        L.zxp_eval_noalloc.argtypes = [vp, u64, u64, vp, vp]
        L.zxp_submit.argtypes = [vp, vp, u64, u64, C.POINTER(u64)]
        L.zxp_poll.argtypes = [vp, u64, i64, zp]
        L.zxp_submit_tables.argtypes = [vp, C.c_char_p, sz, C.POINTER(u64)]
        L.zxp_batch_create.argtypes = [vp, C.POINTER(vp), sz, C.POINTER(vp)]
        L.zxp_batch_run.argtypes = [vp, zp]
        L.zxp_batch_info.argtypes = [vp, C.POINTER(zxp_batch_info_t)]
        L.zxp_batch_destroy.argtypes, L.zxp_batch_destroy.restype = [vp], None
        L.zxp_compile_param.argtypes = [C.c_char_p, sz, C.c_int, C.c_char_p, C.c_char_p,
                                        C.c_char_p, u64, C.c_int, C.POINTER(vp)]
        L.zxp_pscalar_info.argtypes = [vp, C.POINTER(zxp_pscalar_info_t)]
        L.zxp_pscalar_params.argtypes = [vp, C.POINTER(C.c_uint32)]
        L.zxp_bind.argtypes = [vp, u64, C.POINTER(vp)]
        L.zxp_pscalar_free.argtypes, L.zxp_pscalar_free.restype = [vp], None
        L.zxp_server_submit_bind.argtypes = [vp, vp, u64, C.POINTER(u64)]
        L.zxp_sampler_create.argtypes = [vp, C.c_char_p, sz, C.c_int, C.c_char_p, C.POINTER(vp)]
        L.zxp_sampler_info.argtypes = [vp, C.POINTER(C.c_uint32)]
        L.zxp_sampler_draw.argtypes = [vp, sz, C.POINTER(C.c_double), C.POINTER(C.c_uint8), zp]
        L.zxp_sampler_destroy.argtypes, L.zxp_sampler_destroy.restype = [vp], None
        L.zxp_marginal_by_sum.argtypes = [vp, C.c_char_p, sz, C.c_int, C.c_char_p, u64, C.c_char_p, zp]
        L.zxp_server_create.argtypes = [vp, C.POINTER(zxp_server_opts), C.POINTER(vp)]
        L.zxp_server_submit.argtypes = [vp, C.POINTER(zxp_request), C.POINTER(u64)]
        L.zxp_server_submit_scalar.argtypes = [vp, vp, C.POINTER(u64)]
        L.zxp_server_poll.argtypes = [vp, u64, i64, zp, C.POINTER(zxp_request_timing)]
        L.zxp_server_stats.argtypes = [vp, C.POINTER(zxp_server_stats_t)]
        L.zxp_server_destroy.argtypes, L.zxp_server_destroy.restype = [vp], None
        L.zxp_int_peak.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.zxp_test_table_timeout.argtypes = [C.c_int]
        L.zxp_zomega_add.argtypes = [zp, zp, zp]
        L.zxp_zomega_canon.argtypes = [zp, zp]
        L.zxp_zomega_to_complex.argtypes = [zp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.zxp_zomega_to_complex.restype = None
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != ZXP_OK:
        raise ZxpError(rc, what)


def _z(v) -> zxp_zomega:
    z = zxp_zomega()
    for i in range(4):
        x = int(v[i]) & ((1 << 64) - 1)
        z.c[i] = x - (1 << 64) if x >> 63 else x
    z.e = int(v[4]) if len(v) > 4 else 0
    return z


def zxp_strerror(code: int) -> str:
    try:
        return lib().zxp_strerror(code).decode()
    except ImportError:
        return f"status {code}"


def zxp_version() -> str:
    return lib().zxp_version().decode()


class Ctx:
    """A zxp_ctx: device, stream and workspaces (zxp_ctx_destroy on close)."""

    def __init__(self, handle: int, device: int):
        self.handle = C.c_void_p(handle)
        self.device = device

    def close(self):
        if self.handle:
            lib().zxp_ctx_destroy(self.handle)
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scalar:
    """A compiled parametric scalar (zxp_scalar_free on deletion)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def free(self):
        if self.handle:
            lib().zxp_scalar_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return zxp_scalar_info(self)


def zxp_ctx_create(device: int = 0, cuda_stream: int | None = None) -> Ctx:
    """cuda_stream: a cudaStream_t as an integer (torch: stream.cuda_stream)."""
    h = C.c_void_p()
    _check(lib().zxp_ctx_create(device, C.c_void_p(cuda_stream) if cuda_stream else None,
                                C.byref(h)), "zxp_ctx_create")
    return Ctx(h.value, device)


def zxp_ctx_destroy(ctx: Ctx):
    ctx.close()


def _gate_bytes(gates) -> bytes:
    if isinstance(gates, (bytes, bytearray)):
        return bytes(gates)
    import struct
    st = struct.Struct("<BBHHH")
    return b"".join(st.pack(op, 0, q0, q1, 0) for op, q0, q1 in gates)


def _split_opts(opts: dict):
    o = zxp_split_opts()
    for k, v in opts.items():
        if k not in dict(zxp_split_opts._fields_) or k == "reserved":
            raise TypeError(f"unknown split option {k}")
        setattr(o, k, v)
    return o


def zxp_compile(gates, n_qubits: int, out_bits: Sequence[int],
                in_bits: Sequence[int] | None = None, marg_mask: int = 0,
                kind: int = ZXP_AMPLITUDE, split=True) -> Scalar:
    """split: True (zxp_compile: split with the default options when the
    reduction leaves 32 or more parameters), False (zxp_compile_ex without
    a split), or a dict of zxp_split_opts fields (zxp_compile_ex)."""
    gb = _gate_bytes(gates)
    h = C.c_void_p()
    ib = bytes(int(b) & 1 for b in in_bits) if in_bits is not None else None
    ob = bytes(int(b) & 1 for b in out_bits)
    if len(ob) != n_qubits or (ib is not None and len(ib) != n_qubits):
        raise ZxpError(ZXP_EINVAL, "zxp_compile: bit arrays must have n_qubits entries")
    if split is True:
        _check(lib().zxp_compile(gb, len(gb) // 8, n_qubits, ib, ob, marg_mask, kind, C.byref(h)),
               "zxp_compile")
    else:
        o = _split_opts(split) if split else None
        _check(lib().zxp_compile_ex(gb, len(gb) // 8, n_qubits, ib, ob, marg_mask, kind,
                                    C.byref(o) if o is not None else None, C.byref(h)),
               "zxp_compile_ex")
    return Scalar(h.value)


class PScalar:
    """A parametric scalar (zxp_pscalar_free on deletion)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def free(self):
        if self.handle:
            lib().zxp_pscalar_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return zxp_pscalar_info(self)


def zxp_compile_param(gates, n_qubits: int, out_bits: Sequence[int], param_qubits: Sequence[int],
                      in_bits: Sequence[int] | None = None, marg_mask: int = 0,
                      kind: int = ZXP_AMPLITUDE) -> PScalar:
    """param_qubits: the qubits whose bit is a parameter (parameter j = the
    j-th of them in ascending order)."""
    gb = _gate_bytes(gates)
    ob = bytes(int(b) & 1 for b in out_bits)
    ib = bytes(int(b) & 1 for b in in_bits) if in_bits is not None else None
    flags = bytearray(n_qubits)
    for q in param_qubits:
        flags[int(q)] = 1
    if len(ob) != n_qubits or (ib is not None and len(ib) != n_qubits):
        raise ZxpError(ZXP_EINVAL, "zxp_compile_param: bit arrays must have n_qubits entries")
    h = C.c_void_p()
    _check(lib().zxp_compile_param(gb, len(gb) // 8, n_qubits, ib, ob, bytes(flags), marg_mask,
                                   kind, C.byref(h)), "zxp_compile_param")
    return PScalar(h.value)


def zxp_pscalar_info(ps: PScalar) -> dict:
    info = zxp_pscalar_info_t()
    _check(lib().zxp_pscalar_info(ps.handle, C.byref(info)), "zxp_pscalar_info")
    return {f: getattr(info, f) for f, _ in zxp_pscalar_info_t._fields_ if f != "reserved"}


def zxp_pscalar_params(ps: PScalar):
    n = zxp_pscalar_info(ps)["n_params"]
    arr = (C.c_uint32 * max(1, n))()
    _check(lib().zxp_pscalar_params(ps.handle, arr), "zxp_pscalar_params")
    return list(arr[:n])


def zxp_bind(ps: PScalar, bits: int) -> Scalar:
    h = C.c_void_p()
    _check(lib().zxp_bind(ps.handle, bits, C.byref(h)), "zxp_bind")
    return Scalar(h.value)


def zxp_pscalar_free(ps: PScalar):
    ps.free()


def zxp_scalar_from_tables(blob: bytes) -> Scalar:
    h = C.c_void_p()
    _check(lib().zxp_scalar_from_tables(blob, len(blob), C.byref(h)), "zxp_scalar_from_tables")
    return Scalar(h.value)


def zxp_scalar_to_tables(s: Scalar) -> bytes:
    n = C.c_size_t(0)
    _check(lib().zxp_scalar_to_tables(s.handle, None, C.byref(n)), "zxp_scalar_to_tables")
    buf = C.create_string_buffer(n.value)
    _check(lib().zxp_scalar_to_tables(s.handle, buf, C.byref(n)), "zxp_scalar_to_tables")
    return buf.raw[:n.value]


def zxp_scalar_info(s: Scalar) -> dict:
    info = zxp_scalar_info_t()
    _check(lib().zxp_scalar_info(s.handle, C.byref(info)), "zxp_scalar_info")
    return {f: getattr(info, f) for f, _ in zxp_scalar_info_t._fields_ if f != "reserved"}


def zxp_scalar_free(s: Scalar):
    s.free()


def zxp_scalar_split(s: Scalar, **opts) -> Scalar:
    """The same scalar with part of its parameters summed inside every term
    (zxp_split_opts fields as keywords; omitted ones take the defaults)."""
    o = _split_opts(opts)
    h = C.c_void_p()
    _check(lib().zxp_scalar_split(s.handle, C.byref(o) if opts else None, C.byref(h)), "zxp_scalar_split")
    return Scalar(h.value)


def zxp_scalar_reorder(s: Scalar) -> Scalar:
    """The same scalar with the parameters that touch the fewest parity
    forms moved to positions 0-3 (the block lookup's parameters)."""
    h = C.c_void_p()
    _check(lib().zxp_scalar_reorder(s.handle, C.byref(h)), "zxp_scalar_reorder")
    return Scalar(h.value)


def zxp_int_peak(ctx: Ctx, kind: int):
    """(thread instructions per second, ms) of the integer microbenchmark:
    kind 0 lop3, 1 add, 2 popc, 3 mad.lo, 4 lop3 and mad.lo in turn."""
    r, ms = C.c_double(), C.c_double()
    _check(lib().zxp_int_peak(ctx.handle, kind, C.byref(r), C.byref(ms)), "zxp_int_peak")
    return r.value, ms.value


def zxp_inner_sum(ctx: Ctx, s: Scalar):
    """Queue the (re)computation of a split scalar's inner table."""
    _check(lib().zxp_inner_sum(ctx.handle, s.handle), "zxp_inner_sum")


def zxp_eval(ctx: Ctx, s: Scalar, first: int = 0, count: int | None = None):
    """Raw partial (c0, c1, c2, c3, e0) of the Gray-index range (default: all)."""
    if count is None:
        count = (1 << zxp_scalar_info(s)["k"]) - first
    out = zxp_zomega()
    _check(lib().zxp_eval(ctx.handle, s.handle, first, count, C.byref(out)), "zxp_eval")
    return out.tup()


def zxp_eval_device(ctx: Ctx, s: Scalar, first: int, count: int, dev_out_ptr: int):
    """Queue the range; the raw partial (40-byte zxp_zomega) lands at the
    device address dev_out_ptr (e.g. tensor.data_ptr() of 5 int64) when the
    context's stream reaches it.  Does not wait."""
    _check(lib().zxp_eval_device(ctx.handle, s.handle, first, count, C.c_void_p(dev_out_ptr)),
           "zxp_eval_device")


def zxp_eval_noalloc(s: Scalar, first: int, count: int, dev_out_ptr: int, cuda_stream: int = 0):
    """zxp_eval_device for callers that cannot allocate: no context, no
    allocation; the library's fixed static device scratch is used and the
    raw partial lands at the caller's device address dev_out_ptr when
    cuda_stream (0: legacy default stream) reaches it.  Calls that overlap
    on the GPU race (they share the scratch)."""
    _check(lib().zxp_eval_noalloc(s.handle, first, count, C.c_void_p(dev_out_ptr),
                                  C.c_void_p(cuda_stream) if cuda_stream else None),
           "zxp_eval_noalloc")


def zxp_amplitude(ctx: Ctx, s: Scalar):
    """The whole sum, canonical (c0, c1, c2, c3, e)."""
    out = zxp_zomega()
    _check(lib().zxp_amplitude(ctx.handle, s.handle, C.byref(out)), "zxp_amplitude")
    return out.tup()


def zxp_eval_wide(ctx: Ctx, s: Scalar, first: int = 0, count: int | None = None):
    """Raw partial modulo 2^128: (c0, c1, c2, c3, e0), signed 128-bit ints."""
    if count is None:
        count = (1 << zxp_scalar_info(s)["k"]) - first
    out = zxp_zomega_wide()
    _check(lib().zxp_eval_wide(ctx.handle, s.handle, first, count, C.byref(out)), "zxp_eval_wide")
    return out.tup()


def zxp_sum_resumable(ctx: Ctx, s: Scalar, chunk_log2: int, path: str, max_chunks: int = 0):
    """The whole sum in chunks of 2^chunk_log2 terms, checkpointed to the
    host file `path` after every chunk and resumed from it.  Returns
    (status, value, chunks_done, chunks_total): status ZXP_OK (value the
    canonical amplitude), ZXP_EOVERFLOW (value as zxp_amplitude's) or
    ZXP_EAGAIN (chunks remain; value None); other statuses raise."""
    out = zxp_zomega()
    done, total = C.c_uint64(), C.c_uint64()
    rc = lib().zxp_sum_resumable(ctx.handle, s.handle, chunk_log2, os.fsencode(path), max_chunks,
                                 C.byref(out), C.byref(done), C.byref(total))
    if rc not in (ZXP_OK, ZXP_EOVERFLOW, ZXP_EAGAIN):
        raise ZxpError(rc, "zxp_sum_resumable")
    return rc, (None if rc == ZXP_EAGAIN else out.tup()), done.value, total.value


def zxp_amplitude_wide(ctx: Ctx, s: Scalar):
    """The whole sum modulo 2^128, canonical (exact for e0 <= 252)."""
    out = zxp_zomega_wide()
    _check(lib().zxp_amplitude_wide(ctx.handle, s.handle, C.byref(out)), "zxp_amplitude_wide")
    return out.tup()


def zxp_submit(ctx: Ctx, s: Scalar, first: int = 0, count: int | None = None) -> int:
    if count is None:
        count = (1 << zxp_scalar_info(s)["k"]) - first
    t = C.c_uint64()
    _check(lib().zxp_submit(ctx.handle, s.handle, first, count, C.byref(t)), "zxp_submit")
    return t.value


def zxp_submit_tables(ctx: Ctx, blob: bytes) -> int:
    """Queue the whole sum of the scalar whose table bytes are `blob`; the
    library owns the scalar it builds until the ticket is polled."""
    t = C.c_uint64()
    _check(lib().zxp_submit_tables(ctx.handle, blob, len(blob), C.byref(t)), "zxp_submit_tables")
    return t.value


def zxp_poll(ctx: Ctx, ticket: int, timeout_us: int = -1):
    """Raw partial of a ticket, or None while it is not finished."""
    out = zxp_zomega()
    rc = lib().zxp_poll(ctx.handle, ticket, timeout_us, C.byref(out))
    if rc == ZXP_EAGAIN:
        return None
    _check(rc, "zxp_poll")
    return out.tup()


def zxp_test_table_timeout(enable: bool):
    """Tests: make every block's bounded wait for its table copies of the
    launches queued from now on run out (their host calls then report
    ZXP_ETIMEDOUT), or restore normal launches."""
    _check(lib().zxp_test_table_timeout(1 if enable else 0), "zxp_test_table_timeout")


class Batch:
    """A zxp_batch (zxp_batch_destroy on close); keeps its scalars alive."""

    def __init__(self, handle: int, scalars):
        self.handle = C.c_void_p(handle)
        self.scalars = list(scalars)

    def close(self):
        if self.handle:
            lib().zxp_batch_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zxp_batch_create(ctx: Ctx, scalars) -> Batch:
    """Tune and capture one batched evaluation of the full sums of `scalars`."""
    arr = (C.c_void_p * len(scalars))(*[s.handle.value for s in scalars])
    h = C.c_void_p()
    _check(lib().zxp_batch_create(ctx.handle, arr, len(scalars), C.byref(h)), "zxp_batch_create")
    return Batch(h.value, scalars)


def zxp_batch_run(b: Batch):
    """Raw full sums, one (c0, c1, c2, c3, e0) per scalar, in order."""
    out = (zxp_zomega * len(b.scalars))()
    _check(lib().zxp_batch_run(b.handle, out), "zxp_batch_run")
    return [z.tup() for z in out]


def zxp_batch_info(b: Batch) -> dict:
    info = zxp_batch_info_t()
    _check(lib().zxp_batch_info(b.handle, C.byref(info)), "zxp_batch_info")
    return {f: getattr(info, f) for f, _ in zxp_batch_info_t._fields_ if f != "reserved"}


def zxp_batch_destroy(b: Batch):
    b.close()


class Server:
    """A zxp_server (zxp_server_destroy on close: queued requests finish
    first); keeps borrowed scalars alive until their tickets are polled."""

    def __init__(self, handle: int, ctx: Ctx):
        self.handle = C.c_void_p(handle)
        self.ctx = ctx
        self.borrowed = {}

    def close(self):
        if self.handle:
            lib().zxp_server_destroy(self.handle)
            self.handle = C.c_void_p()
            self.borrowed.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zxp_server_create(ctx: Ctx, **opts) -> Server:
    """opts: the fields of zxp_server_opts (policy, max_k, compile_threads,
    max_active, arena_bytes, step_terms, small_terms, chunk_log2, threads);
    0 or absent means the default."""
    o = zxp_server_opts()
    for k, v in opts.items():
        if k not in dict(zxp_server_opts._fields_) or k == "reserved":
            raise ZxpError(ZXP_EINVAL, f"zxp_server_create: unknown option {k}")
        setattr(o, k, int(v))
    h = C.c_void_p()
    _check(lib().zxp_server_create(ctx.handle, C.byref(o), C.byref(h)), "zxp_server_create")
    return Server(h.value, ctx)


def zxp_server_submit(srv: Server, gates, n_qubits: int, out_bits: Sequence[int],
                      in_bits: Sequence[int] | None = None, marg_mask: int = 0,
                      kind: int = ZXP_AMPLITUDE) -> int:
    """Queue a circuit request (copied); returns its ticket."""
    gb = _gate_bytes(gates)
    ob = bytes(int(b) & 1 for b in out_bits)
    ib = bytes(int(b) & 1 for b in in_bits) if in_bits is not None else None
    if len(ob) != n_qubits or (ib is not None and len(ib) != n_qubits):
        raise ZxpError(ZXP_EINVAL, "zxp_server_submit: bit arrays must have n_qubits entries")
    r = zxp_request(gb, len(gb) // 8, n_qubits, kind, ib, ob, marg_mask)
    t = C.c_uint64()
    _check(lib().zxp_server_submit(srv.handle, C.byref(r), C.byref(t)), "zxp_server_submit")
    return t.value


def zxp_server_submit_scalar(srv: Server, s: Scalar) -> int:
    t = C.c_uint64()
    _check(lib().zxp_server_submit_scalar(srv.handle, s.handle, C.byref(t)),
           "zxp_server_submit_scalar")
    srv.borrowed[t.value] = s
    return t.value


def zxp_server_submit_bind(srv: Server, ps: PScalar, bits: int) -> int:
    """Queue the binding `bits` of a parametric scalar; returns its ticket."""
    t = C.c_uint64()
    _check(lib().zxp_server_submit_bind(srv.handle, ps.handle, bits, C.byref(t)),
           "zxp_server_submit_bind")
    srv.borrowed[t.value] = ps
    return t.value


def zxp_server_poll(srv: Server, ticket: int, timeout_us: int = -1):
    """None while the request runs; else (status, value, timing): value the
    canonical (c0, c1, c2, c3, e) when status is ZXP_OK or ZXP_EOVERFLOW,
    timing a dict of zxp_request_timing."""
    out = zxp_zomega()
    tm = zxp_request_timing()
    rc = lib().zxp_server_poll(srv.handle, ticket, timeout_us, C.byref(out), C.byref(tm))
    if rc == ZXP_EAGAIN:
        return None
    if rc == ZXP_ENOTFOUND or rc == ZXP_EINVAL:
        raise ZxpError(rc, "zxp_server_poll")
    srv.borrowed.pop(ticket, None)
    timing = {f: getattr(tm, f) for f, _ in zxp_request_timing._fields_ if f != "reserved"}
    return rc, (out.tup() if rc in (ZXP_OK, ZXP_EOVERFLOW) else None), timing


def zxp_server_stats(srv: Server) -> dict:
    st = zxp_server_stats_t()
    _check(lib().zxp_server_stats(srv.handle, C.byref(st)), "zxp_server_stats")
    return {f: getattr(st, f) for f, _ in zxp_server_stats_t._fields_ if f != "reserved"}


def zxp_server_destroy(srv: Server):
    srv.close()


class Sampler:
    """A zxp_sampler (zxp_sampler_destroy on close)."""

    def __init__(self, handle: int, n: int, ctx: Ctx):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.ctx = ctx

    def close(self):
        if self.handle:
            lib().zxp_sampler_destroy(self.handle)
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zxp_sampler_create(ctx: Ctx, gates, n_qubits: int, in_bits: Sequence[int] | None = None) -> Sampler:
    gb = _gate_bytes(gates)
    ib = bytes(int(b) & 1 for b in in_bits) if in_bits is not None else None
    h = C.c_void_p()
    _check(lib().zxp_sampler_create(ctx.handle, gb, len(gb) // 8, n_qubits, ib, C.byref(h)),
           "zxp_sampler_create")
    return Sampler(h.value, n_qubits, ctx)


def zxp_sampler_info(s: Sampler):
    arr = (C.c_uint32 * s.n)()
    _check(lib().zxp_sampler_info(s.handle, arr), "zxp_sampler_info")
    return list(arr)


def zxp_sampler_draw(s: Sampler, u):
    """u: n_samples rows of n uniforms in [0, 1).  Returns (bitstrings as
    lists of n bits, exact probabilities (c0, c1, c2, c3, e))."""
    rows = [list(r) for r in u]
    ns = len(rows)
    if any(len(r) != s.n for r in rows):
        raise ZxpError(ZXP_EINVAL, "zxp_sampler_draw: each row needs n uniforms")
    flat = (C.c_double * max(1, ns * s.n))(*[float(x) for r in rows for x in r])
    out = (C.c_uint8 * max(1, ns * s.n))()
    prob = (zxp_zomega * max(1, ns))()
    _check(lib().zxp_sampler_draw(s.handle, ns, flat, out, prob), "zxp_sampler_draw")
    bits = [list(out[i * s.n:(i + 1) * s.n]) for i in range(ns)]
    return bits, [prob[i].tup() for i in range(ns)]


def zxp_sampler_destroy(s: Sampler):
    s.close()


def zxp_marginal_by_sum(ctx: Ctx, gates, n_qubits: int, mask: int, bits: Sequence[int],
                        in_bits: Sequence[int] | None = None):
    gb = _gate_bytes(gates)
    ib = bytes(int(b) & 1 for b in in_bits) if in_bits is not None else None
    out = zxp_zomega()
    _check(lib().zxp_marginal_by_sum(ctx.handle, gb, len(gb) // 8, n_qubits, ib, mask,
                                     bytes(int(b) & 1 for b in bits), C.byref(out)),
           "zxp_marginal_by_sum")
    return out.tup()


def zxp_zomega_add(a, b):
    out = zxp_zomega()
    za, zb = _z(a), _z(b)
    _check(lib().zxp_zomega_add(C.byref(za), C.byref(zb), C.byref(out)), "zxp_zomega_add")
    return out.tup()


def zxp_zomega_canon(a):
    out = zxp_zomega()
    za = _z(a)
    _check(lib().zxp_zomega_canon(C.byref(za), C.byref(out)), "zxp_zomega_canon")
    return out.tup()


def zxp_zomega_to_complex(a) -> complex:
    re, im = C.c_double(), C.c_double()
    za = _z(a)
    lib().zxp_zomega_to_complex(C.byref(za), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


EXPORTED = ["zxp_ctx_create", "zxp_ctx_destroy", "zxp_compile", "zxp_scalar_from_tables",
            "zxp_scalar_to_tables", "zxp_scalar_info", "zxp_scalar_free", "zxp_eval",
            "zxp_eval_device", "zxp_eval_noalloc", "zxp_batch_create", "zxp_batch_run",
            "zxp_batch_info", "zxp_batch_destroy", "zxp_server_create", "zxp_server_submit",
            "zxp_server_submit_scalar", "zxp_server_poll", "zxp_server_stats", "zxp_server_destroy",
            "zxp_compile_param", "zxp_pscalar_info", "zxp_pscalar_params", "zxp_bind",
            "zxp_pscalar_free", "zxp_server_submit_bind", "zxp_sampler_create", "zxp_sampler_info",
            "zxp_sampler_draw", "zxp_sampler_destroy", "zxp_marginal_by_sum",
            "zxp_amplitude", "zxp_submit", "zxp_poll", "zxp_zomega_add", "zxp_zomega_canon",
            "zxp_zomega_to_complex", "zxp_strerror", "zxp_version"]
