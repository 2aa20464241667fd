// inner.cu -- the inner table of a scalar with inner parameters (plan.h):
//   F[z | q << k_inner] = sum over x_I of g(x_I, q) (-1)^(x_I . z),
// g the product of the scalar's inner and crossing rows.  Exact in Z[w]
// modulo 2^64, in passes over the table:
//   1. a block evaluates 2^10 consecutive entries u = (x_I, q) of g from the
//      inner plan, as the sum kernel evaluates one term (form bits by XOR of
//      flip rows, the phase exponent from the coefficient planes and the
//      quadratic bit, the node count, the table entry -- the inner constant
//      included -- times phase-pair values beyond the folded ones, zero when
//      a zero form is set): the state of the block's high bits once, that of
//      an entry's low bits from the plan's table of them, and the quadratic
//      bit's cross part as the parity of (A x_high) & x_low; it keeps the
//      entries in shared memory, does the Walsh-Hadamard butterflies of the
//      low 10 bits there and writes the tile once;
//   2. every further pass does up to 8 more bits: a block stages the 2^nb
//      entries of those bits for 2^(10 - nb) consecutive low indices,
//      transforms them in shared memory and writes them back.
// Shared memory holds the four coefficients as separate planes, so that
// the 8-byte accesses of a warp's consecutive elements hit distinct banks.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "plan.h"
#include "zring.h"

namespace zxp {
namespace {

constexpr int kInnerThreads = 256;
constexpr uint32_t kTileLog2 = kInnerLowBits;   // the plan tabulates these low bits
constexpr uint32_t kTile = 1u << kTileLog2;   // 32 KB of shared memory per block
constexpr uint32_t kHighBits = 8;             // bits of one later pass

// one Walsh-Hadamard stage (bit s) over a tile of `rows` rows of `cols`
// columns held as four coefficient planes (entry (r, c) at r * cols + c)
__device__ __forceinline__ void butterfly(uint64_t (*t)[kTile], uint32_t n, uint32_t cols_log2, uint32_t s) {
    for (uint32_t e = threadIdx.x; e < n / 2; e += blockDim.x) {
        const uint32_t pr = e >> cols_log2, c = e & ((1u << cols_log2) - 1u);
        const uint32_t r0 = ((pr >> s) << (s + 1)) | (pr & ((1u << s) - 1u));
        const uint32_t i0 = (r0 << cols_log2) | c, i1 = ((r0 | (1u << s)) << cols_log2) | c;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint64_t a = t[k][i0], b = t[k][i1];
            t[k][i0] = a + b;
            t[k][i1] = a - b;
        }
    }
}

template <int NW>
__global__ void __launch_bounds__(kInnerThreads)
inner_terms_low(const __grid_constant__ KernelParams p, const int nwn, const int general,
                const zw64* __restrict__ table, const zw64* __restrict__ pv,
                const uint32_t* __restrict__ frows, const uint64_t* __restrict__ adj,
                const uint32_t* __restrict__ low, const uint32_t bits, const uint32_t low_bits,
                zw64* __restrict__ out) {
    __shared__ uint64_t tile[4][kTile];
    const uint32_t tb = bits < kTileLog2 ? bits : kTileLog2, n = 1u << tb;
    const uint64_t base = (uint64_t)blockIdx.x << tb;
    // the high bits' state: form bits, A x_high and the quadratic bit
    uint32_t LB[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) LB[w] = p.INV[w];
    uint64_t AB = 0;
    uint32_t qb2 = 0;
    for (uint64_t m = base; m; m &= m - 1) {
        const uint32_t i = (uint32_t)__ffsll((long long)m) - 1u;
#pragma unroll
        for (int w = 0; w < NW; w++) LB[w] ^= __ldg(frows + (size_t)i * NW + w);
        const uint64_t a = __ldg(adj + i);
        AB ^= a;
        qb2 += (uint32_t)__popcll(a & base);
    }
    // (every quadratic pair of the high bits was counted from both ends)
    const uint32_t qb = (qb2 >> 1) & 1u;
    const uint32_t ab = (uint32_t)AB;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
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
        zw64 v;
        if (general) {
            if (p.has_zero && zb) {
                v = zw_zero();
            } else {
                v = table[idx];
                for (uint32_t j = 0; j < p.npairs; j++) {
                    const uint32_t a = (L[p.PA[j] >> 5] >> (p.PA[j] & 31)) & 1u;
                    const uint32_t b = (L[p.PB[j] >> 5] >> (p.PB[j] & 31)) & 1u;
                    v = zw_mul(v, pv[4 * j + (a | (b << 1))]);
                }
            }
        } else {
            if (p.xshift)
                idx = (idx << p.xshift) | (L[nwn] & p.pmask) | ((p.has_zero && zb ? 1u : 0u) << p.zshift);
            v = table[idx];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) tile[k][e] = v.c[k];
    }
    __syncthreads();
    for (uint32_t s = 0; s < low_bits; s++) {
        butterfly(tile, n, 0, s);
        __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x)
        out[base | e] = zw_make(tile[0][e], tile[1][e], tile[2][e], tile[3][e]);
}

// One later pass over bits [lo, lo + nb) of an array of 2^total entries: a
// block holds the 2^nb entries of those bits for 2^cols_log2 consecutive low
// indices l (nb + cols_log2 = 10, 2^cols_log2 <= 2^lo).
__global__ void __launch_bounds__(kInnerThreads)
wht_pass(zw64* __restrict__ F, const uint32_t lo, const uint32_t nb, const uint32_t cols_log2) {
    __shared__ uint64_t tile[4][kTile];
    const uint32_t cols = 1u << cols_log2, n = (1u << nb) * cols;
    // block -> (high index o, first low index l0)
    const uint64_t groups_lo = (1ull << lo) >> cols_log2;
    const uint64_t o = (uint64_t)blockIdx.x / groups_lo;
    const uint64_t l0 = ((uint64_t)blockIdx.x % groups_lo) << cols_log2;
    const uint64_t base = (o << (lo + nb)) | l0;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const uint32_t r = e >> cols_log2, c = e & (cols - 1u);
        const ulonglong2* g = reinterpret_cast<const ulonglong2*>(F + base + ((uint64_t)r << lo) + c);
        const ulonglong2 a = g[0], b = g[1];
        tile[0][e] = a.x; tile[1][e] = a.y; tile[2][e] = b.x; tile[3][e] = b.y;
    }
    __syncthreads();
    for (uint32_t s = 0; s < nb; s++) {
        butterfly(tile, n, cols_log2, s);
        __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const uint32_t r = e >> cols_log2, c = e & (cols - 1u);
        ulonglong2* g = reinterpret_cast<ulonglong2*>(F + base + ((uint64_t)r << lo) + c);
        g[0] = make_ulonglong2(tile[0][e], tile[1][e]);
        g[1] = make_ulonglong2(tile[2][e], tile[3][e]);
    }
}

template <int NW>
cudaError_t launch_low(const Plan& in, uint32_t low_bits, const zw64* itab, const zw64* ipv,
                       const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw64* ftab,
                       cudaStream_t stream) {
    const uint32_t bits = in.kp.k, tb = bits < kTileLog2 ? bits : kTileLog2;
    inner_terms_low<NW><<<(unsigned)(1ull << (bits - tb)), kInnerThreads, 0, stream>>>(
        in.kp, in.nwn, in.general ? 1 : 0, itab, ipv, ifr, iadj, ilow, bits, low_bits, ftab);
    return cudaGetLastError();
}

}  // namespace

cudaError_t inner_table_launch(const Plan& inner, uint32_t k_inner, const zw64* itab, const zw64* ipv,
                               const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw64* ftab,
                               cudaStream_t stream) {
    const uint32_t bits = inner.kp.k;
    if (bits > kMaxInnerBits || k_inner > bits) return cudaErrorInvalidValue;
    const int nw = inner.nwn + (inner.nwl < 1 ? 1 : inner.nwl);
    const uint32_t low = k_inner < kTileLog2 ? k_inner : kTileLog2;
    cudaError_t e;
    switch (nw) {
    case 1: e = launch_low<1>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 2: e = launch_low<2>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 3: e = launch_low<3>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 4: e = launch_low<4>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 5: e = launch_low<5>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 6: e = launch_low<6>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 7: e = launch_low<7>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    case 8: e = launch_low<8>(inner, low, itab, ipv, ifr, iadj, ilow, ftab, stream); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    // the remaining inner bits in passes of at most kHighBits, split evenly
    const uint32_t rem = k_inner - low;
    if (!rem) return cudaSuccess;
    const uint32_t passes = (rem + kHighBits - 1) / kHighBits;
    for (uint32_t lo = low, left = rem, p = passes; left; p--) {
        const uint32_t nb = (left + p - 1) / p, cols_log2 = kTileLog2 - nb;
        const uint64_t blocks = (1ull << bits) >> kTileLog2;
        wht_pass<<<(unsigned)blocks, kInnerThreads, 0, stream>>>(ftab, lo, nb, cols_log2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        lo += nb;
        left -= nb;
    }
    return cudaSuccess;
}

}  // namespace zxp
