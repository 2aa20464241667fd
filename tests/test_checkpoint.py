"""Resumable chunked sums on the host (no GPU): the checkpoint file and the
chunk loop of paper_2403_06777_gb300/csrc/checkpoint.cpp, driven by a small
C++ program (tests/host/checkpoint_test.cpp) whose chunk evaluator is a fixed
function of the chunk's range.

A process that is killed (SIGKILL, no clean-up) inside a chunk loses only
that chunk: a later run resumes from the file and ends with the sum an
uninterrupted run gives, bit for bit, which is also computed here in Python
from the same function.  A file for another scalar or other parameters, and
a damaged file, are refused and left as they are."""
import os
import shutil
import signal
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_06777_gb300", "csrc")
M64 = (1 << 64) - 1
OK, EINVAL, EAGAIN = 0, -1, -7


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("ckpt") / "checkpoint_test")
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, os.path.join(ROOT, "tests", "host", "checkpoint_test.cpp"),
                    os.path.join(CSRC, "checkpoint.cpp"), "-o", out], check=True)
    return out


def mix(z):
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def expected(width, k, cl):
    """The sum of every chunk's value modulo 2^width, per coefficient."""
    cl = min(cl, k)
    total, span = 1 << k, 1 << cl
    s = [0, 0, 0, 0]
    for first in range(0, total, span):
        count = min(span, total - first)
        for i in range(4):
            lo = (mix(4 * first + i) * count + i) & M64
            hi = (mix(4 * first + i + (1 << 40)) & 0xFFFFFFFF) if width == 128 else 0
            s[i] += (hi << 64) | lo
    mod = (1 << width) - 1
    return [v & mod for v in s]


def run(exe, path, width=64, k=10, cl=4, digest=77, e0=3, max_chunks=0, kill_at=-1):
    r = subprocess.run([exe, str(path), str(width), str(k), str(cl), str(digest), str(e0), str(max_chunks),
                        str(kill_at)], capture_output=True, text=True, timeout=120)
    if kill_at >= 0 and r.returncode == -signal.SIGKILL:
        return None
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split()
    status, done, n = int(lines[0]), int(lines[1]), int(lines[2])
    w = [int(x, 16) for x in lines[3:11]]
    sums = [w[i] | (w[4 + i] << 64) for i in range(4)]
    return status, done, n, sums


@pytest.mark.parametrize("width,k,cl", [(64, 10, 4), (128, 11, 3), (64, 7, 0), (128, 9, 9), (64, 0, 0),
                                        (64, 13, 5)])
def test_uninterrupted_sum(exe, tmp_path, width, k, cl):
    p = tmp_path / "c.ckpt"
    status, done, n, sums = run(exe, p, width, k, cl)
    assert status == OK and done == n == ((1 << k) + (1 << min(cl, k)) - 1) >> min(cl, k)
    assert sums == expected(width, k, cl)
    # a complete file: a further call runs nothing and returns the same
    assert run(exe, p, width, k, cl) == (OK, done, n, sums)
    assert not os.path.exists(str(p) + ".tmp")


@pytest.mark.parametrize("width", [64, 128])
def test_killed_inside_a_chunk_resumes_bit_identical(exe, tmp_path, width):
    p = tmp_path / "c.ckpt"
    k, cl = 12, 5
    full = expected(width, k, cl)
    # killed inside chunk 6, then inside chunk 20 of the resumed run, then
    # stopped by the chunk budget, then run to the end
    assert run(exe, p, width, k, cl, kill_at=6) is None
    st = run(exe, p, width, k, cl, max_chunks=1)
    assert st[0] == EAGAIN and st[1] == 7
    assert run(exe, p, width, k, cl, kill_at=13) is None
    st = run(exe, p, width, k, cl, max_chunks=40)
    assert st[0] == EAGAIN and st[1] == 20 + 40
    status, done, n, sums = run(exe, p, width, k, cl)
    assert status == OK and done == n == 128
    assert sums == full


def test_foreign_and_damaged_files_are_refused(exe, tmp_path):
    p = tmp_path / "c.ckpt"
    assert run(exe, p, 64, 10, 4, max_chunks=5)[0] == EAGAIN
    good = p.read_bytes()
    # another scalar, chunk size, k, width or exponent: refused, file kept
    for kw in (dict(digest=78), dict(cl=5), dict(k=11), dict(width=128), dict(e0=4)):
        args = dict(width=64, k=10, cl=4)
        args.update(kw)
        assert run(exe, p, **args)[0] == EINVAL, kw
        assert p.read_bytes() == good
    # a flipped bit anywhere, a truncated file, a foreign file
    for i in (0, 9, 30, 60, len(good) - 20, len(good) - 1):
        bad = bytearray(good)
        bad[i] ^= 0x10
        p.write_bytes(bytes(bad))
        assert run(exe, p, 64, 10, 4)[0] == EINVAL, i
    for cut in (0, 7, 40, len(good) - 1):
        p.write_bytes(good[:cut])
        assert run(exe, p, 64, 10, 4)[0] == EINVAL, cut
    p.write_bytes(b"not a checkpoint file")
    assert run(exe, p, 64, 10, 4)[0] == EINVAL
    # the intact file resumes
    p.write_bytes(good)
    status, done, n, sums = run(exe, p, 64, 10, 4)
    assert status == OK and sums == expected(64, 10, 4)


def test_unwritable_location_is_an_error(exe, tmp_path):
    st = run(exe, tmp_path / "missing_dir" / "c.ckpt", 64, 6, 2)
    assert st[0] == EINVAL and st[1] == 1   # the first chunk ran; its state could not be saved
