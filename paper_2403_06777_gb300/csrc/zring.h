// zring.h -- the ring Z[w] (w = e^{i pi/4}, w^4 = -1) with coefficients
// taken modulo 2^64, in the integer basis {1, w, w^2, w^3}.
//
// Every sum the library computes is an integer combination of powers of w,
// so computing modulo 2^64 is a ring homomorphism: the true numerator is
// recovered exactly whenever its coefficients lie in [-2^63, 2^63).  For an
// amplitude a = N / sqrt2^e every Galois conjugate of a is the amplitude of
// a unitary circuit (T -> T^s, H -> +-H), so |N_j| <= 2^(e/2) and e <= 124
// guarantees exactness.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define ZXP_HD __host__ __device__ __forceinline__
#else
#define ZXP_HD inline
#endif

namespace zxp {

struct zw64 {
    uint64_t c[4];
};

ZXP_HD zw64 zw_make(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    zw64 r;
    r.c[0] = a; r.c[1] = b; r.c[2] = c; r.c[3] = d;
    return r;
}
ZXP_HD zw64 zw_zero() { return zw_make(0, 0, 0, 0); }
ZXP_HD zw64 zw_one() { return zw_make(1, 0, 0, 0); }

ZXP_HD zw64 zw_add(zw64 a, zw64 b) {
    return zw_make(a.c[0] + b.c[0], a.c[1] + b.c[1], a.c[2] + b.c[2], a.c[3] + b.c[3]);
}
ZXP_HD zw64 zw_sub(zw64 a, zw64 b) {
    return zw_make(a.c[0] - b.c[0], a.c[1] - b.c[1], a.c[2] - b.c[2], a.c[3] - b.c[3]);
}
ZXP_HD zw64 zw_neg(zw64 a) { return zw_make(0 - a.c[0], 0 - a.c[1], 0 - a.c[2], 0 - a.c[3]); }

// a * w
ZXP_HD zw64 zw_mulw(zw64 a) { return zw_make(0 - a.c[3], a.c[0], a.c[1], a.c[2]); }

// a * w^j, j taken mod 8
ZXP_HD zw64 zw_rot(zw64 a, unsigned j) {
    j &= 7;
    if (j & 4) a = zw_neg(a);
    if (j & 2) a = zw_make(0 - a.c[2], 0 - a.c[3], a.c[0], a.c[1]);
    if (j & 1) a = zw_mulw(a);
    return a;
}

// negacyclic product (w^4 = -1)
ZXP_HD zw64 zw_mul(zw64 a, zw64 b) {
    zw64 r;
    r.c[0] = a.c[0] * b.c[0] - a.c[1] * b.c[3] - a.c[2] * b.c[2] - a.c[3] * b.c[1];
    r.c[1] = a.c[0] * b.c[1] + a.c[1] * b.c[0] - a.c[2] * b.c[3] - a.c[3] * b.c[2];
    r.c[2] = a.c[0] * b.c[2] + a.c[1] * b.c[1] + a.c[2] * b.c[0] - a.c[3] * b.c[3];
    r.c[3] = a.c[0] * b.c[3] + a.c[1] * b.c[2] + a.c[2] * b.c[1] + a.c[3] * b.c[0];
    return r;
}

// a * n for an integer count n
ZXP_HD zw64 zw_scale(zw64 a, uint64_t n) {
    return zw_make(a.c[0] * n, a.c[1] * n, a.c[2] * n, a.c[3] * n);
}

// acc + a * n for a 32-bit count n (one wide multiply-add per coefficient)
ZXP_HD zw64 zw_madd32(zw64 acc, zw64 a, uint32_t n) {
    zw64 r;
    for (int i = 0; i < 4; i++) {
        const uint64_t lo = (uint64_t)(uint32_t)a.c[i] * n + acc.c[i];
        r.c[i] = lo + ((uint64_t)((uint32_t)(a.c[i] >> 32) * n) << 32);
    }
    return r;
}

// a * sqrt2, sqrt2 = w - w^3
ZXP_HD zw64 zw_mul_sqrt2(zw64 a) {
    return zw_make(a.c[1] - a.c[3], a.c[0] + a.c[2], a.c[1] + a.c[3], a.c[2] - a.c[0]);
}

// w^j as a ring element
ZXP_HD zw64 zw_wpow(unsigned j) { return zw_rot(zw_one(), j); }

ZXP_HD zw64 zw_pow(zw64 a, unsigned n) {
    zw64 r = zw_one();
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
