"""Shared-memory layout of the inner table's transform rounds (host, no GPU).

The inner kernels (csrc/inner.cu) hold 2^RB entries a thread and exchange a
tile of 2^T entries through shared memory between rounds, entry e at 16-byte
slot slot(e).  These checks restate the two index maps and test what the
kernels rely on: in every round layout the threads' entries are a
permutation of the tile, slot() keeps every entry inside the tile, and the
eight threads of a quarter-warp (one 128-byte shared-memory wavefront of
16-byte accesses) always hit eight distinct 16-byte bank groups."""
import pytest


def spread(t, p, j, rb):
    low = (1 << p) - 1
    return (t & low) | (j << p) | ((t & ~low) << rb)


def slot(e, rb):
    if rb == 3:
        return e ^ ((e >> 3) & 7)
    return e ^ ((0x5630 >> (((e >> 3) & 3) << 2)) & 7)


@pytest.mark.parametrize("T,rb", [(11, 3), (10, 3), (11, 2), (10, 2)])
def test_round_layouts_permute_the_tile_without_bank_conflicts(T, rb):
    n, threads = 1 << T, (1 << T) >> rb
    assert sorted(slot(e, rb) for e in range(n)) == list(range(n))
    for p in range(0, T - rb + 1):
        es = [spread(t, p, j, rb) for t in range(threads) for j in range(1 << rb)]
        assert sorted(es) == list(range(n)), p
        for q in range(threads // 8):
            for j in range(1 << rb):
                banks = {slot(spread(8 * q + i, p, j, rb), rb) & 7 for i in range(8)}
                assert len(banks) == 8, (p, q, j)


@pytest.mark.parametrize("T,rb", [(11, 3), (11, 2)])
def test_rounds_cover_every_bit_once(T, rb):
    # the rounds' stage masks (as the kernels take them): bits [q, q + rb)
    # for q = 0, rb, 2 rb, ...; a round that would run past the tile's top
    # takes the top rb bits and only the bits not done yet
    for bits in range(1, T + 1):
        done = []
        for q in range(0, T, rb):
            if q >= bits:
                break
            p = T - rb if q + rb > T else q
            done += [p + b for b in range(rb) if q <= p + b < bits]
        assert sorted(done) == list(range(bits)), bits
