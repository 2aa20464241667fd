"""The C ABI library: it loads, exports every entry point include/zxp.h
declares, and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2403_06777_gb300 as Z
import zxp_inputs as zi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "zxp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zxp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(Z.LIB_PATH)
    names = header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(Z.EXPORTED) <= set(names)
    assert "sm_103a" in Z.zxp_version()


def test_strerror_names_every_status():
    for code in range(0, -9, -1):
        assert Z.zxp_strerror(code) not in ("", "unknown status")


def test_tables_roundtrip_and_info():
    ps = zi.synthetic_ps(7, 12, n_lin=5, n_quad=3, n_node=9, n_pair=2, e0=3, G=(1, -2, 0, 5))
    blob = ps.pack()
    s = Z.zxp_scalar_from_tables(blob)
    assert Z.zxp_scalar_to_tables(s) == blob
    info = Z.zxp_scalar_info(s)
    assert (info["k"], info["n_lin"], info["n_quad"], info["n_node"], info["n_pair"], info["e0"]) == \
        (12, 5, 3, 9, 2, 3)


@pytest.mark.parametrize("bad", [
    b"", b"XXXX" * 20,
    zi.PSTables(k=63).pack(),                                    # k > 62
    zi.PSTables(k=3, lin=[(1 << 3, 1)]).pack(),                  # mask beyond k
    zi.PSTables(k=3, node=[(1, 9)]).pack(),                      # constant > 7
    zi.PSTables(k=2, lin=[(1, 1)]).pack()[:-4],                  # truncated
])
def test_tables_rejected(bad):
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_scalar_from_tables(bad)
    assert e.value.code in (Z.ZXP_EINVAL, Z.ZXP_ETOOBIG)


def test_compile_rejects_bad_circuits():
    with pytest.raises(Z.ZxpError):
        Z.zxp_compile([(zi.CNOT, 0, 0)], 2, [0, 0])       # control == target
    with pytest.raises(Z.ZxpError):
        Z.zxp_compile([(zi.H, 5, 0)], 2, [0, 0])          # qubit out of range
    with pytest.raises(Z.ZxpError):
        Z.zxp_compile([(42, 0, 0)], 2, [0, 0])            # opcode
    with pytest.raises(Z.ZxpError):
        Z.zxp_compile([], 70, [0] * 70, kind=Z.ZXP_MARGINAL_DOUBLED)   # > 64 qubits


def test_zomega_helpers():
    # (1 + i)/sqrt2 = w
    assert Z.zxp_zomega_canon((1, 0, 1, 0, 1)) == (0, 1, 0, 0, 0)
    assert Z.zxp_zomega_canon((0, 0, 0, 0, 9)) == (0, 0, 0, 0, 0)
    # a/sqrt2^1 + b/sqrt2^3 aligns a to e = 3 by two sqrt2 steps (x 2)
    assert Z.zxp_zomega_add((1, 0, 0, 0, 1), (1, 0, 0, 0, 3)) == (3, 0, 0, 0, 3)
    s = Z.zxp_zomega_add((1, 0, 0, 0, 1), (1, 0, 0, 0, 3))
    assert abs(Z.zxp_zomega_to_complex(s) - (2 ** -0.5 + 2 ** -1.5)) < 1e-12
    assert abs(Z.zxp_zomega_to_complex((0, 1, 0, 0, 0)) - (0.5 ** 0.5) * (1 + 1j)) < 1e-12


def test_ctx_create_fails_cleanly_without_a_device():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(Z.ZxpError) as e:
        Z.zxp_ctx_create(0)
    assert e.value.code == Z.ZXP_ECUDA
