"""Index maps of the lookup walk with several states a thread (host, no GPU).

Over a range of Gray indices [t0, t1) made of whole aligned blocks of 256,
the kernel walks the Gray code of every variable but 7 (two states) or but 6
and 7 (four states), compressed index c = t / 2 or t / 4, the left-out
variables put in clear, and takes the states that set them.  These checks
restate the maps and test what the kernel relies on: the states visit
exactly the assignments gray(t) of the range, once each, and consecutive
compressed indices differ in one variable, v(ctz(c)), never a left-out one."""
import pytest


def gray(t):
    return t ^ (t >> 1)


def expand(c, xl):
    g = gray(c)
    return (g & ((1 << xl) - 1)) | ((g >> xl) << 8)


@pytest.mark.parametrize("ns", [2, 4])
@pytest.mark.parametrize("k,b0,b1", [(10, 0, 4), (11, 3, 7), (12, 5, 16), (9, 1, 2)])
def test_states_cover_the_range_once(ns, k, b0, b1):
    xl, sh = (7, 1) if ns == 2 else (6, 2)
    sbits = [0, 128] if ns == 2 else [0, 128, 64, 192]
    t0, t1 = 256 * b0, 256 * b1
    want = sorted(gray(t) for t in range(t0, t1))
    got = sorted(expand(c, xl) | s for c in range(t0 >> sh, t1 >> sh) for s in sbits)
    assert got == want
    assert all(x < (1 << k) for x in got)


@pytest.mark.parametrize("ns", [2, 4])
def test_compressed_steps_flip_one_variable(ns):
    xl = 7 if ns == 2 else 6
    skip = 1 if ns == 2 else 2
    for c in range(1, 1 << 12):
        d = expand(c, xl) ^ expand(c - 1, xl)
        ic = (c & -c).bit_length() - 1
        v = ic if ic < xl else ic + skip
        assert d == 1 << v
        assert v not in ((7,) if ns == 2 else (6, 7))
