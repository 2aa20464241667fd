// inner.cu -- the inner table of a scalar with inner parameters (plan.h):
//   F[z | q << k_inner] = sum over x_I of g(x_I, q) (-1)^(x_I . z),
// g the product of the scalar's inner and crossing rows.  Exact in Z[w]
// modulo 2^64 (or 2^128: the same kernels on 64-byte entries), in two
// kernels:
//   1. inner_terms_low: a block evaluates 2^11 consecutive entries
//      u = (x_I, q) of g from the inner plan, as the sum kernel evaluates one
//      term (form bits by XOR of flip rows, the phase exponent from the
//      coefficient planes and the quadratic bit, the node count, the table
//      entry -- the inner constant included -- times phase-pair values beyond
//      the folded ones, zero when a zero form is set): the state of the
//      block's high bits once, that of an entry's low bits from the plan's
//      table of them, and the quadratic bit's cross part as the parity of
//      (A x_high) & x_low.  It transforms the low 11 bits and writes the tile
//      once;
//   2. wht_pass: each further pass transforms up to T more bits of tiles of
//      2^T entries (2^nb rows of those bits times 2^(T - nb) consecutive
//      low indices; T = 11, or 10 for 64-byte entries), read and written
//      once, two tiles per SM so that one block's loads overlap the other's
//      exchanges.
// Both transform in radix-4 rounds: a thread holds the four entries that
// differ in two bits of the tile index in registers and does both butterfly
// stages there; between rounds the tile is exchanged through shared memory
// as planes of 16-byte words (two or four per entry), at a swizzled slot that gives
// every quarter-warp the eight distinct 16-byte bank groups of a 128-byte
// row in every layout the rounds use.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "plan.h"
#include "zring.h"

namespace zxp {
namespace {

constexpr uint32_t kTileLog2 = kInnerLowBits;   // the plan tabulates these low bits
constexpr uint32_t kTile = 1u << kTileLog2;

// An entry as 16-byte planes: zw64 in two (c0 c1 | c2 c3), zw128 in four
// (one coefficient each, low word first).
template <class Z>
struct Planes;
template <>
struct Planes<zw64> {
    static constexpr int N = 2;
    __device__ static ulonglong2 get(const zw64& v, int k) { return make_ulonglong2(v.c[2 * k], v.c[2 * k + 1]); }
    __device__ static void set(zw64& v, int k, ulonglong2 x) {
        v.c[2 * k] = x.x;
        v.c[2 * k + 1] = x.y;
    }
};
template <>
struct Planes<zw128> {
    static constexpr int N = 4;
    __device__ static ulonglong2 get(const zw128& v, int k) {
        return make_ulonglong2((unsigned long long)v.c[k], (unsigned long long)(v.c[k] >> 64));
    }
    __device__ static void set(zw128& v, int k, ulonglong2 x) { v.c[k] = ((u128)x.y << 64) | (u128)x.x; }
};
// log2 of the entries of one wht_pass tile: 64 KB of shared memory, two
// blocks per SM
template <class Z>
__host__ __device__ constexpr uint32_t pass_log2() { return Planes<Z>::N == 2 ? 11u : 10u; }
template <class Z>
__host__ __device__ constexpr size_t pass_smem() { return (size_t)Planes<Z>::N << pass_log2<Z>() << 4; }
// tile-index bits one pass transforms at most: all of a tile's (one column
// of 2^11 rows for 32-byte entries)
template <class Z>
constexpr uint32_t pass_bits() { return pass_log2<Z>(); }

static_assert(kTileLog2 == 11, "the low kernel's rounds: five pairs of bits, then bit 10");

// Radix of the rounds: a thread holds 2^RB entries that differ in RB bits of
// the tile index, RB = 3 for 32-byte entries (eight a thread, three bits a
// round), 2 for 64-byte ones (four a thread: eight would take 128 registers
// for the values alone).
template <class Z>
__host__ __device__ constexpr uint32_t radix_bits() { return Planes<Z>::N == 2 ? 3u : 2u; }

// shared-memory slot of tile entry e, a linear map that keeps e's tile and
// gives the eight threads of every quarter-warp eight distinct 16-byte bank
// groups of a 128-byte row in every layout the rounds use (checked for all
// layouts on the host): RB = 3: bits 3-5 of e flip slot bits 0-2; RB = 2:
// bits 3 and 4 of e flip slot bits (0, 1) and (1, 2)
template <uint32_t RB>
__device__ __forceinline__ uint32_t slot(uint32_t e) {
    if constexpr (RB == 3) return e ^ ((e >> 3) & 7u);
    return e ^ ((0x5630u >> (((e >> 3) & 3u) << 2)) & 7u);
}

// tile index of the j-th entry that thread t holds in the round of bits
// [p, p + RB): j in those bits, t's bits around them
template <uint32_t RB>
__device__ __forceinline__ uint32_t spread(uint32_t t, uint32_t p, uint32_t j) {
    const uint32_t low = (1u << p) - 1u;
    return (t & low) | (j << p) | ((t & ~low) << RB);
}

template <class Z>
__device__ __forceinline__ void stage(Z& a, Z& b) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const auto x = a.c[k], y = b.c[k];
        a.c[k] = x + y;
        b.c[k] = x - y;
    }
}

// the butterfly stages of a round on the 2^RB entries held: bit b of the
// round (entry pairs that differ in bit b of j) when bit b of m is set
template <uint32_t RB, class Z>
__device__ __forceinline__ void radix(Z (&v)[1u << RB], uint32_t m) {
#pragma unroll
    for (uint32_t b = 0; b < RB; b++) {
        if ((m >> b) & 1u) {
#pragma unroll
            for (uint32_t j = 0; j < (1u << RB); j++)
                if (!((j >> b) & 1u)) stage(v[j], v[j | (1u << b)]);
        }
    }
}

// from the layout of round bits pf to that of round bits pt (plane k of
// the tile at sm + k * ps)
template <uint32_t RB, class Z>
__device__ __forceinline__ void exchange(ulonglong2* sm, uint32_t ps, Z (&v)[1u << RB], uint32_t t, uint32_t pf,
                                         uint32_t pt) {
#pragma unroll
    for (uint32_t j = 0; j < (1u << RB); j++) {
        const uint32_t a = slot<RB>(spread<RB>(t, pf, j));
#pragma unroll
        for (int k = 0; k < Planes<Z>::N; k++) sm[k * ps + a] = Planes<Z>::get(v[j], k);
    }
    __syncthreads();
#pragma unroll
    for (uint32_t j = 0; j < (1u << RB); j++) {
        const uint32_t a = slot<RB>(spread<RB>(t, pt, j));
#pragma unroll
        for (int k = 0; k < Planes<Z>::N; k++) Planes<Z>::set(v[j], k, sm[k * ps + a]);
    }
    __syncthreads();
}

// the round at tile bits [q, q + RB) of a T-bit tile index, of which the
// first `bits` are transformed: its layout p (T - RB when the bits run past
// the tile's top, the lower ones already done) and the stages to take
template <uint32_t RB>
__device__ __forceinline__ uint32_t round_at(uint32_t q, uint32_t T) {
    return q + RB > T ? T - RB : q;
}
template <uint32_t RB>
__device__ __forceinline__ uint32_t round_stages(uint32_t q, uint32_t T, uint32_t bits) {
    const uint32_t p = round_at<RB>(q, T);
    uint32_t m = 0;
#pragma unroll
    for (uint32_t b = 0; b < RB; b++)
        if (p + b >= q && p + b < bits) m |= 1u << b;
    return m;
}

// entries of the table (16-byte aligned: the table starts on 256)
template <class Z>
__device__ __forceinline__ Z ld_entry(const Z* q) {
    const ulonglong2* g = reinterpret_cast<const ulonglong2*>(q);
    Z v;
#pragma unroll
    for (int k = 0; k < Planes<Z>::N; k++) Planes<Z>::set(v, k, g[k]);
    return v;
}
template <class Z>
__device__ __forceinline__ void st_entry(Z* q, const Z& v) {
    ulonglong2* g = reinterpret_cast<ulonglong2*>(q);
#pragma unroll
    for (int k = 0; k < Planes<Z>::N; k++) g[k] = Planes<Z>::get(v, k);
}

// g at entry e of a block whose high bits give form bits LB, quadratic bit
// qb and the cross row ab
template <int NW, class Z>
__device__ __forceinline__ Z term_value(const KernelParams& p, const int nwn, const int general,
                                        const Z* __restrict__ table, const Z* __restrict__ pv,
                                           const uint32_t (&LB)[NW], const uint32_t qb, const uint32_t ab,
                                           const uint32_t* __restrict__ low, const uint32_t e) {
    const uint32_t* r = low + (size_t)e * (NW + 1);
    uint32_t L[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) L[w] = LB[w] ^ __ldg(r + w);
    const uint32_t q = qb ^ __ldg(r + NW) ^ ((uint32_t)__popc(ab & e) & 1u);
    uint32_t P0 = 0, P1 = 0, X2 = 0, M = 0, zb = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        if (w < nwn) {
            X2 ^= L[w] & p.CB[w];
            M += (uint32_t)__popc(L[w]);
        } else {
            const uint32_t v = L[w];
            P0 += (uint32_t)__popc(v & p.C0[w - nwn]);
            P1 += (uint32_t)__popc(v & p.C1[w - nwn]);
            X2 ^= v & p.C2[w - nwn];
            zb |= v & p.Z[w - nwn];
        }
    }
    const uint32_t J = (P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q)) & 7u;
    uint32_t idx = J * p.tab_stride + M;
    if (general) {
        if (p.has_zero && zb) return zw_zero<typename zw_word<Z>::type>();
        Z v = ld_entry(table + idx);
        for (uint32_t j = 0; j < p.npairs; j++) {
            const uint32_t a = (L[p.PA[j] >> 5] >> (p.PA[j] & 31)) & 1u;
            const uint32_t b = (L[p.PB[j] >> 5] >> (p.PB[j] & 31)) & 1u;
            v = zw_mul(v, pv[4 * j + (a | (b << 1))]);
        }
        return v;
    }
    if (p.xshift)
        idx = (idx << p.xshift) | (L[nwn] & p.pmask) | ((p.has_zero && zb ? 1u : 0u) << p.zshift);
    return ld_entry(table + idx);
}

// threads of a term-kernel block (2^RB entries a thread) and the blocks an
// SM should hold
template <class Z>
__host__ __device__ constexpr int low_threads() { return (int)(kTile >> radix_bits<Z>()); }
template <class Z>
__host__ __device__ constexpr int low_min_blocks() { return Planes<Z>::N == 2 ? 2 : 1; }

// The first 2^bits entries of g in tiles of 2^11, the low `low_bits` bits
// transformed.  Thread t evaluates entries 2^RB t .. 2^RB t + 2^RB - 1, the
// layout of the first round.
template <int NW, class Z>
__global__ void __launch_bounds__(low_threads<Z>(), low_min_blocks<Z>())
inner_terms_low(const __grid_constant__ KernelParams p, const int nwn, const int general,
                const Z* __restrict__ table, const Z* __restrict__ pv,
                const uint32_t* __restrict__ frows, const uint64_t* __restrict__ adj,
                const uint32_t* __restrict__ low, const uint32_t bits, const uint32_t low_bits,
                Z* __restrict__ out) {
    extern __shared__ ulonglong2 sm[];   // Planes<Z>::N planes of kTile slots
    const uint32_t tb = bits < kTileLog2 ? bits : kTileLog2, n = 1u << tb;
    const uint64_t base = (uint64_t)blockIdx.x << tb;
    // the high bits' state (form bits, A x_high, the quadratic bit): lane i
    // takes bit i of the block's first index (bits <= 26 < 32), a warp
    // reduction adds them up
    const uint32_t t = threadIdx.x, lane = t & 31u;
    const bool set = lane < bits && ((base >> lane) & 1u);
    uint32_t LB[NW];
    uint64_t AB = 0;
    uint32_t qb2 = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) LB[w] = set ? __ldg(frows + (size_t)lane * NW + w) : 0u;
    if (set) {
        AB = __ldg(adj + lane);
        qb2 = (uint32_t)__popcll(AB & base);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
#pragma unroll
        for (int w = 0; w < NW; w++) LB[w] ^= __shfl_xor_sync(0xffffffffu, LB[w], off);
        AB ^= __shfl_xor_sync(0xffffffffu, AB, off);
        qb2 += __shfl_xor_sync(0xffffffffu, qb2, off);
    }
#pragma unroll
    for (int w = 0; w < NW; w++) LB[w] ^= p.INV[w];
    // (every quadratic pair of the high bits was counted from both ends)
    const uint32_t qb = (qb2 >> 1) & 1u;
    const uint32_t ab = (uint32_t)AB;
    constexpr uint32_t RB = radix_bits<Z>(), E = 1u << RB;
    Z v[E];
#pragma unroll
    for (uint32_t j = 0; j < E; j++) {
        const uint32_t e = spread<RB>(t, 0, j);
        v[j] = e < n ? term_value<NW, Z>(p, nwn, general, table, pv, LB, qb, ab, low, e)
                     : zw_zero<typename zw_word<Z>::type>();
    }
    radix<RB>(v, round_stages<RB>(0, kTileLog2, low_bits));
    uint32_t pr = 0;
    // rounds at bits [q, q + RB) for q = RB, 2 RB, ...; the last one's top
    // bits alone in the layout of the tile's top RB bits
#pragma unroll
    for (uint32_t q = RB; q < kTileLog2; q += RB) {
        if (q < low_bits) {   // (the same for the whole block)
            const uint32_t qr = round_at<RB>(q, kTileLog2);
            exchange<RB>(sm, kTile, v, t, pr, qr);
            pr = qr;
            radix<RB>(v, round_stages<RB>(q, kTileLog2, low_bits));
        }
    }
#pragma unroll
    for (uint32_t j = 0; j < E; j++) {
        const uint32_t e = spread<RB>(t, pr, j);
        if (e < n) st_entry(out + (base | e), v[j]);
    }
}

// One later pass over bits [lo, lo + NB) of an array of 2^total entries: a
// block holds the 2^NB entries of those bits for 2^C consecutive low indices
// l (tile index e = row << C | col, C = T - NB <= 10 <= lo).  Rounds at bits
// C, C + RB, ... of the tile index; when NB is not a multiple of RB the last
// round takes the tile's top RB bits and transforms only those not done.
template <class Z, uint32_t NB>
__global__ void __launch_bounds__(1u << (pass_log2<Z>() - radix_bits<Z>()), 2)
wht_pass(Z* __restrict__ F, const uint32_t lo) {
    constexpr uint32_t RB = radix_bits<Z>(), E = 1u << RB;
    constexpr uint32_t T = pass_log2<Z>(), C = T - NB, NR = (NB + RB - 1) / RB, CM = (1u << C) - 1u;
    extern __shared__ ulonglong2 sm[];
    const uint32_t gl = lo - C;   // log2 of the tiles side by side in the low bits
    const uint64_t o = (uint64_t)blockIdx.x >> gl;
    const uint64_t l0 = (uint64_t)(blockIdx.x & ((1u << gl) - 1u)) << C;
    Z* const b = F + ((o << (lo + NB)) | l0);
    const uint32_t t = threadIdx.x;
    const uint32_t P0 = round_at<RB>(C, T);
    Z v[E];
#pragma unroll
    for (uint32_t j = 0; j < E; j++) {
        const uint32_t e = spread<RB>(t, P0, j);
        v[j] = ld_entry(b + ((uint64_t)(e >> C) << lo) + (e & CM));
    }
    uint32_t pr = P0;
#pragma unroll
    for (uint32_t r = 0; r < NR; r++) {
        const uint32_t q = C + RB * r, qr = round_at<RB>(q, T);
        if (r) exchange<RB>(sm, 1u << T, v, t, pr, qr);
        pr = qr;
        radix<RB>(v, round_stages<RB>(q, T, T));
    }
#pragma unroll
    for (uint32_t j = 0; j < E; j++) {
        const uint32_t e = spread<RB>(t, pr, j);
        st_entry(b + ((uint64_t)(e >> C) << lo) + (e & CM), v[j]);
    }
}

template <class Z, uint32_t NB>
cudaError_t launch_pass(Z* ftab, uint32_t lo, uint32_t bits, cudaStream_t stream) {
    constexpr uint32_t T = pass_log2<Z>();
    cudaError_t e = cudaFuncSetAttribute(wht_pass<Z, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem<Z>());
    if (e != cudaSuccess) return e;
    wht_pass<Z, NB><<<(unsigned)((1ull << bits) >> T), 1u << (T - radix_bits<Z>()), pass_smem<Z>(), stream>>>(
        ftab, lo);
    return cudaGetLastError();
}

template <int NW, class Z>
cudaError_t launch_low(const Plan& in, uint32_t low_bits, const Z* itab, const Z* ipv, const uint32_t* ifr,
                       const uint64_t* iadj, const uint32_t* ilow, Z* ftab, cudaStream_t stream) {
    const uint32_t bits = in.kp.k, tb = bits < kTileLog2 ? bits : kTileLog2;
    const size_t smem = (size_t)Planes<Z>::N * kTile * 16u;
    cudaError_t e = cudaFuncSetAttribute(inner_terms_low<NW, Z>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // (the 128-bit table holds (J, M) values only: every entry takes the
    // general path)
    const int general = (in.general || Planes<Z>::N == 4) ? 1 : 0;
    inner_terms_low<NW, Z><<<(unsigned)(1ull << (bits - tb)), low_threads<Z>(), smem, stream>>>(
        in.kp, in.nwn, general, itab, ipv, ifr, iadj, ilow, bits, low_bits, ftab);
    return cudaGetLastError();
}

template <class Z>
cudaError_t table_launch(const Plan& inner, uint32_t k_inner, const Z* itab, const Z* ipv, const uint32_t* ifr,
                         const uint64_t* iadj, const uint32_t* ilow, Z* ftab, cudaStream_t stream) {
    const uint32_t bits = inner.kp.k;
    if (bits > kMaxInnerBits || k_inner > bits) return cudaErrorInvalidValue;
    const int nw = inner.nwn + (inner.nwl < 1 ? 1 : inner.nwl);
    const uint32_t low = k_inner < kTileLog2 ? k_inner : kTileLog2;
    cudaError_t e;
    switch (nw) {
    case 1: e = launch_low<1, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 2: e = launch_low<2, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 3: e = launch_low<3, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 4: e = launch_low<4, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 5: e = launch_low<5, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 6: e = launch_low<6, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 7: e = launch_low<7, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 8: e = launch_low<8, Z>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    // the remaining inner bits in passes of at most pass_bits, split evenly
    // (every pass starts at lo = 11 or above, so its tile's 2^C <= 2^10
    // columns fit below it)
    const uint32_t rem = k_inner - low;
    const uint32_t passes = (rem + pass_bits<Z>() - 1) / pass_bits<Z>();
    for (uint32_t lo = low, left = rem, p = passes; left; p--) {
        const uint32_t nb = (left + p - 1) / p;
        switch (nb) {
        case 1: e = launch_pass<Z, 1>(ftab, lo, bits, stream); break;
        case 2: e = launch_pass<Z, 2>(ftab, lo, bits, stream); break;
        case 3: e = launch_pass<Z, 3>(ftab, lo, bits, stream); break;
        case 4: e = launch_pass<Z, 4>(ftab, lo, bits, stream); break;
        case 5: e = launch_pass<Z, 5>(ftab, lo, bits, stream); break;
        case 6: e = launch_pass<Z, 6>(ftab, lo, bits, stream); break;
        case 7: e = launch_pass<Z, 7>(ftab, lo, bits, stream); break;
        case 8: e = launch_pass<Z, 8>(ftab, lo, bits, stream); break;
        case 9: e = launch_pass<Z, 9>(ftab, lo, bits, stream); break;
        case 10: e = launch_pass<Z, 10>(ftab, lo, bits, stream); break;
        default:
            if constexpr (pass_bits<Z>() >= 11) e = launch_pass<Z, 11>(ftab, lo, bits, stream);
            else return cudaErrorInvalidValue;
            break;
        }
        if (e != cudaSuccess) return e;
        lo += nb;
        left -= nb;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t inner_table_launch(const Plan& inner, uint32_t k_inner, const zw64* itab, const zw64* ipv,
                               const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw64* ftab,
                               cudaStream_t stream) {
    return table_launch<zw64>(inner, k_inner, itab, ipv, ifr, iadj, ilow, ftab, stream);
}

cudaError_t inner_table_launch_wide(const Plan& inner, uint32_t k_inner, const zw128* itab_w, const zw128* ipv_w,
                                    const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw128* ftab_w,
                                    cudaStream_t stream) {
    return table_launch<zw128>(inner, k_inner, itab_w, ipv_w, ifr, iadj, ilow, ftab_w, stream);
}

}  // namespace zxp
