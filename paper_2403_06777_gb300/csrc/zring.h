// zring.h -- the ring Z[w] (w = e^{i pi/4}, w^4 = -1) with coefficients
// taken modulo 2^64 (zw64) or 2^128 (zw128), in the integer basis
// {1, w, w^2, w^3}.
//
// Every sum the library computes is an integer combination of powers of w,
// so computing modulo 2^b is a ring homomorphism: the true numerator is
// recovered exactly whenever its coefficients lie in [-2^(b-1), 2^(b-1)).
// For an amplitude a = N / sqrt2^e every Galois conjugate of a is the
// amplitude of a unitary circuit (T -> T^s, H -> +-H), so |N_j| <= 2^(e/2):
// e <= 124 guarantees exactness with 64-bit words, e <= 252 with 128-bit.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define ZXP_HD __host__ __device__ __forceinline__
#else
#define ZXP_HD inline
#endif

namespace zxp {

typedef unsigned __int128 u128;

template <class W>
struct zwt {
    W c[4];
};
typedef zwt<uint64_t> zw64;
typedef zwt<u128> zw128;
// the coefficient word of a ring type
template <class Z>
struct zw_word;
template <class W>
struct zw_word<zwt<W>> {
    typedef W type;
};

ZXP_HD zw64 zw_make(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    zw64 r;
    r.c[0] = a; r.c[1] = b; r.c[2] = c; r.c[3] = d;
    return r;
}
template <class W>
ZXP_HD zwt<W> zw_make_t(W a, W b, W c, W d) {
    zwt<W> r;
    r.c[0] = a; r.c[1] = b; r.c[2] = c; r.c[3] = d;
    return r;
}
template <class W = uint64_t>
ZXP_HD zwt<W> zw_zero() { return zw_make_t<W>(0, 0, 0, 0); }
template <class W = uint64_t>
ZXP_HD zwt<W> zw_one() { return zw_make_t<W>(1, 0, 0, 0); }

// a 64-bit value read as the two's-complement integer it encodes, modulo
// 2^128 (exact for ring elements whose coefficients fit 64 bits)
ZXP_HD zw128 zw_widen(zw64 a) {
    return zw_make_t<u128>((u128)(__int128)(int64_t)a.c[0], (u128)(__int128)(int64_t)a.c[1],
                           (u128)(__int128)(int64_t)a.c[2], (u128)(__int128)(int64_t)a.c[3]);
}

template <class W>
ZXP_HD zwt<W> zw_add(zwt<W> a, zwt<W> b) {
    return zw_make_t<W>(a.c[0] + b.c[0], a.c[1] + b.c[1], a.c[2] + b.c[2], a.c[3] + b.c[3]);
}
template <class W>
ZXP_HD zwt<W> zw_sub(zwt<W> a, zwt<W> b) {
    return zw_make_t<W>(a.c[0] - b.c[0], a.c[1] - b.c[1], a.c[2] - b.c[2], a.c[3] - b.c[3]);
}
template <class W>
ZXP_HD zwt<W> zw_neg(zwt<W> a) {
    return zw_make_t<W>(W(0) - a.c[0], W(0) - a.c[1], W(0) - a.c[2], W(0) - a.c[3]);
}

// a * w
template <class W>
ZXP_HD zwt<W> zw_mulw(zwt<W> a) { return zw_make_t<W>(W(0) - a.c[3], a.c[0], a.c[1], a.c[2]); }

// a * w^j, j taken mod 8
template <class W>
ZXP_HD zwt<W> zw_rot(zwt<W> a, unsigned j) {
    j &= 7;
    if (j & 4) a = zw_neg(a);
    if (j & 2) a = zw_make_t<W>(W(0) - a.c[2], W(0) - a.c[3], a.c[0], a.c[1]);
    if (j & 1) a = zw_mulw(a);
    return a;
}

// negacyclic product (w^4 = -1)
template <class W>
ZXP_HD zwt<W> zw_mul(zwt<W> a, zwt<W> b) {
    zwt<W> r;
    r.c[0] = a.c[0] * b.c[0] - a.c[1] * b.c[3] - a.c[2] * b.c[2] - a.c[3] * b.c[1];
    r.c[1] = a.c[0] * b.c[1] + a.c[1] * b.c[0] - a.c[2] * b.c[3] - a.c[3] * b.c[2];
    r.c[2] = a.c[0] * b.c[2] + a.c[1] * b.c[1] + a.c[2] * b.c[0] - a.c[3] * b.c[3];
    r.c[3] = a.c[0] * b.c[3] + a.c[1] * b.c[2] + a.c[2] * b.c[1] + a.c[3] * b.c[0];
    return r;
}

// a * n for an integer count n
template <class W>
ZXP_HD zwt<W> zw_scale(zwt<W> a, uint64_t n) {
    return zw_make_t<W>(a.c[0] * W(n), a.c[1] * W(n), a.c[2] * W(n), a.c[3] * W(n));
}

// acc + a * n for a 32-bit count n (64-bit words: one wide multiply-add per
// coefficient)
ZXP_HD zw64 zw_madd32(zw64 acc, zw64 a, uint32_t n) {
    zw64 r;
    for (int i = 0; i < 4; i++) {
        const uint64_t lo = (uint64_t)(uint32_t)a.c[i] * n + acc.c[i];
        r.c[i] = lo + ((uint64_t)((uint32_t)(a.c[i] >> 32) * n) << 32);
    }
    return r;
}
ZXP_HD zw128 zw_madd32(zw128 acc, zw128 a, uint32_t n) { return zw_add(acc, zw_scale(a, n)); }

// a * sqrt2, sqrt2 = w - w^3
template <class W>
ZXP_HD zwt<W> zw_mul_sqrt2(zwt<W> a) {
    return zw_make_t<W>(a.c[1] - a.c[3], a.c[0] + a.c[2], a.c[1] + a.c[3], a.c[2] - a.c[0]);
}

// w^j as a ring element
template <class W = uint64_t>
ZXP_HD zwt<W> zw_wpow(unsigned j) { return zw_rot(zw_one<W>(), j); }

template <class W>
ZXP_HD zwt<W> zw_pow(zwt<W> a, unsigned n) {
    zwt<W> r = zw_one<W>();
    while (n) {
        if (n & 1) r = zw_mul(r, a);
        a = zw_mul(a, a);
        n >>= 1;
    }
    return r;
}

// 1 + sqrt2 = 1 + w - w^3 (a unit; inverse sqrt2 - 1)
ZXP_HD zw64 zw_silver() { return zw_make(1, 1, 0, (uint64_t)-1); }
ZXP_HD zw64 zw_silver_inv() { return zw_make((uint64_t)-1, 1, 0, (uint64_t)-1); }

}  // namespace zxp
