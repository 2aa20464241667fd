// kernel.cu -- exact exponential sum of a parametric scalar on sm_103a.
//
// Each thread walks contiguous Gray-code slices [t0, t0 + span) of the
// assignment space (x = t ^ (t >> 1)); consecutive assignments differ in the
// bit ctz(t), so a step XORs that variable's flip mask into the form bits
// (the AND / XOR-reduce steps of Sec. 3.3 done incrementally) and updates
// the quadratic phase with one bit of A x.  A term is then one table entry
// K * w^(J + 2M) (1 + sqrt2)^M (see plan.h), multiplied by any phase-pair
// values, and accumulated in four int64 coefficients modulo 2^64.
// Threads reduce by warp shuffles, then per block in shared memory, then the
// last block to finish adds the per-block partials (App. E's pairwise sum,
// done as a shuffle tree).  Integer adds make the result bit-exact and
// independent of the reduction order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "plan.h"

namespace zxp {

namespace {

constexpr int kThreads = 256;
// counting variants: 32-bit counters for at most 5 odd nodes (48 counters per
// lane, 48 KB per block), 16-bit counters packed two per word for at most 15
// (128 counters per lane, 64 KB per block; slices shorter than 2^16 terms)
constexpr uint32_t kHistMaxOdd32 = 5;
constexpr uint32_t kHistMaxOdd16 = 15;
constexpr uint64_t kSpan16 = 65528;   // largest multiple of 8 below 2^16

template <int NW>
__device__ __forceinline__ uint32_t bit_at(const uint32_t (&L)[NW], uint32_t pos) {
    uint32_t wsel = pos >> 5, v = 0;
#pragma unroll
    for (int q = 0; q < NW; q++) v = (wsel == (uint32_t)q) ? L[q] : v;
    return (v >> (pos & 31)) & 1u;
}

__device__ __forceinline__ zw64 lds_zw(const zw64* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    ulonglong2 a = q[0], b = q[1];
    return zw_make(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ zw64 shfl_xor_zw(zw64 v, int off) {
    zw64 r;
#pragma unroll
    for (int c = 0; c < 4; c++) r.c[c] = __shfl_xor_sync(0xffffffffu, v.c[c], off);
    return r;
}

__device__ __forceinline__ zw64 block_reduce(zw64 v, zw64* sred) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = zw_add(v, shfl_xor_zw(v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sred[lane] : zw_zero();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = zw_add(v, shfl_xor_zw(v, off));
    }
    return v;   // valid in thread 0
}

template <int NWN, int NWL, bool GENERAL, int HIST>
__global__ void __launch_bounds__(kThreads)
sum_kernel(const __grid_constant__ KernelParams p, const zw64* __restrict__ gtable,
           const zw64* __restrict__ gpv, const uint32_t* __restrict__ gF,
           const uint64_t* __restrict__ gADJ, uint64_t first, uint64_t count, uint64_t span,
           uint64_t nslices, zw64* __restrict__ partials, unsigned int* __restrict__ counter,
           const zw64 K, const int32_t e0, DevResult* __restrict__ result) {
    constexpr int NW = NWN + NWL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    zw64* sT = reinterpret_cast<zw64*>(smem_raw);
    const uint32_t ntab = 8u * p.tab_stride;
    zw64* sPV = sT + ntab;
    zw64* sred = sPV + 4u * p.npairs;
    uint64_t* sADJ = reinterpret_cast<uint64_t*>(sred + kThreads / 32);
    uint32_t* sF = reinterpret_cast<uint32_t*>(sADJ + kMaxK);
    // HIST (1: 32-bit, 2: 16-bit counters): per-lane counters of the table
    // index J * stride + M, laid out [warp][word][lane] so that every lane
    // owns one bank; HIST == 2 packs indices 2w and 2w + 1 into word w
    uint32_t* sH = sF + kMaxK * NW;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwords = HIST == 2 ? (ntab + 1) / 2 : ntab;
    if (HIST) {
        for (uint32_t i = threadIdx.x; i < nwords * kThreads; i += blockDim.x) sH[i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < ntab; i += blockDim.x) sT[i] = gtable[i];
    if (GENERAL)
        for (uint32_t i = threadIdx.x; i < 4u * p.npairs; i += blockDim.x) sPV[i] = gpv[i];
    for (uint32_t i = threadIdx.x; i < p.k; i += blockDim.x) sADJ[i] = gADJ[i];
    for (uint32_t i = threadIdx.x; i < p.k * NW; i += blockDim.x) sF[i] = gF[i];
    for (uint32_t i = p.k + threadIdx.x; i < 3; i += blockDim.x) sADJ[i] = 0;
    for (uint32_t i = p.k * NW + threadIdx.x; i < 3 * NW; i += blockDim.x) sF[i] = 0;
    __syncthreads();

    // flip rows and adjacency of the three lowest variables, in registers:
    // inside an aligned block of 8 Gray steps they are the only ones flipped
    uint32_t f0[NW], f1[NW], f2[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) { f0[w] = sF[w]; f1[w] = sF[NW + w]; f2[w] = sF[2 * NW + w]; }
    const uint64_t adj0 = sADJ[0], adj1 = sADJ[1], adj2 = sADJ[2];

    zw64 acc = zw_zero();
    const uint64_t end = first + count;
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    // HIST: acc += sum_idx count(idx) * T[idx] (mod 2^64), counters reset
    // The warp first adds each counter word over its 32 lanes (one redux);
    // lane (i mod 32) then owns word i's multiply-adds.
    auto fold = [&]() {
        __syncwarp();
        for (uint32_t i = 0; i < nwords; i++) {
            uint32_t* h = sH + ((warp * nwords + i) << 5) + lane;
            const uint32_t c = *h;
            *h = 0;
            if (HIST == 2) {
                const uint32_t lo = __reduce_add_sync(0xffffffffu, c & 0xFFFFu);
                const uint32_t hi = __reduce_add_sync(0xffffffffu, c >> 16);
                if ((i & 31u) == lane) {
                    if (lo) acc = zw_madd32(acc, lds_zw(sT + 2 * i), lo);
                    if (hi) acc = zw_madd32(acc, lds_zw(sT + 2 * i + 1), hi);
                }
            } else {
                // a lane counts at most one slice (<= 2^18 terms) between
                // folds, so the 32-lane sum fits in 32 bits
                const uint32_t n = __reduce_add_sync(0xffffffffu, c);
                if ((i & 31u) == lane && n) acc = zw_madd32(acc, lds_zw(sT + i), n);
            }
        }
    };
    // a thread with several slices folds after each one, so no counter can
    // overflow (16-bit counters: every slice is shorter than 2^16 terms)
    const bool fold_each = HIST == 2 || nslices > gstride;
    // warp-uniform slice loop: every lane of a warp runs the same number of
    // iterations (lanes past the end skip the work), so fold() can use
    // full-warp reductions
    for (uint64_t s0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); s0 < nslices;
         s0 += gstride) {
        const uint64_t s = s0 + lane;
        if (s < nslices) {
        uint64_t t = first + s * span;
        const uint64_t tend = (end - t < span) ? end : t + span;
        const uint64_t x = t ^ (t >> 1);
        // state at x: the form bits are the XOR of the flip rows of x's set
        // bits (plus the inversions); a = A x; q = x^T (upper A) x, as half
        // of sum_{j in x} |A_j & x|
        uint32_t L[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) L[w] = p.INV[w];
        uint64_t a = 0;
        uint32_t qs = 0;
        for (uint64_t y = x; y; y &= y - 1) {
            const int j = __ffsll((long long)y) - 1;
#pragma unroll
            for (int w = 0; w < NW; w++) L[w] ^= sF[j * NW + w];
            const uint64_t aj = sADJ[j];
            a ^= aj;
            qs += (uint32_t)__popcll(aj & x);
        }
        uint32_t q = (qs >> 1) & 1u;

        // one term at the current state
        auto term = [&]() {
            uint32_t M = 0, P0 = 0, P1 = 0, X2 = 0, Zb = 0;
#pragma unroll
            for (int w = 0; w < NWN; w++) {
                M += __popc(L[w]);
                X2 ^= L[w] & p.CB[w];
            }
#pragma unroll
            for (int w = 0; w < NWL; w++) {
                const uint32_t v = L[NWN + w];
                P0 += __popc(v & p.C0[w]);
                P1 += __popc(v & p.C1[w]);
                X2 ^= v & p.C2[w];
                if (GENERAL) Zb |= v & p.Z[w];
            }
            if (HIST) {
                const uint32_t J = (P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q)) & 7u;
                const uint32_t idx = J * p.tab_stride + M;
                if (HIST == 2)
                    atomicAdd(sH + ((warp * nwords + (idx >> 1)) << 5) + lane, 1u << ((idx & 1u) << 4));
                else
                    atomicAdd(sH + ((warp * nwords + idx) << 5) + lane, 1u);
            } else if (!GENERAL || Zb == 0) {
                const uint32_t J = (P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q)) & 7u;
                zw64 v = lds_zw(sT + J * p.tab_stride + M);
                if (GENERAL) {
                    for (uint32_t j = 0; j < p.npairs; j++) {
                        const uint32_t b = bit_at<NW>(L, p.PA[j]) | (bit_at<NW>(L, p.PB[j]) << 1);
                        v = zw_mul(v, lds_zw(sPV + 4 * j + b));
                    }
                }
                acc = zw_add(acc, v);
            }
        };
        // flip of a variable known at compile time (0, 1 or 2)
        auto flip = [&](const uint32_t (&f)[NW], uint64_t adj, int i) {
            q ^= (uint32_t)(a >> i) & 1u;
            a ^= adj;
#pragma unroll
            for (int w = 0; w < NW; w++) L[w] ^= f[w];
        };

        for (;;) {
            if ((t & 7u) == 0 && tend - t >= 8) {
                // Gray steps inside t .. t+7 flip variables 0,1,0,2,0,1,0
                term(); flip(f0, adj0, 0);
                term(); flip(f1, adj1, 1);
                term(); flip(f0, adj0, 0);
                term(); flip(f2, adj2, 2);
                term(); flip(f0, adj0, 0);
                term(); flip(f1, adj1, 1);
                term(); flip(f0, adj0, 0);
                term();
                t += 7;
            } else {
                term();
            }
            if (++t >= tend) break;
            // x(t) = x(t-1) ^ (1 << ctz(t))
            const uint32_t tl = (uint32_t)t;
            const int i = tl ? __ffs(tl) - 1 : 31 + __ffs((uint32_t)(t >> 32));
            q ^= (uint32_t)(a >> i) & 1u;
            a ^= sADJ[i];
#pragma unroll
            for (int w = 0; w < NW; w++) L[w] ^= sF[i * NW + w];
        }
        }   // s < nslices
        if (HIST && fold_each) fold();
    }
    if (HIST) fold();

    // reduction: warp shuffles, block, then the last block over the partials
    __shared__ unsigned int s_last;
    acc = block_reduce(acc, sred);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        __threadfence();
        const unsigned int done = atomicAdd(counter, 1u);
        s_last = (done == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        zw64 v = zw_zero();
        for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(partials + b);
            ulonglong2 lo = __ldcg(q2), hi = __ldcg(q2 + 1);
            v = zw_add(v, zw_make(lo.x, lo.y, hi.x, hi.y));
        }
        v = block_reduce(v, sred);
        if (threadIdx.x == 0) {
            const zw64 r = zw_mul(K, v);
            for (int c = 0; c < 4; c++) result->c[c] = (int64_t)r.c[c];
            result->e = e0;
            result->flags = 1;
            *counter = 0u;       // ready for the next launch on this workspace
        }
    }
}

using KernelFn = void (*)(const KernelParams, const zw64*, const zw64*, const uint32_t*,
                          const uint64_t*, uint64_t, uint64_t,
                          uint64_t, uint64_t, zw64*, unsigned int*, const zw64, const int32_t,
                          DevResult*);

template <int NWN, int NWL, bool G, int H>
constexpr KernelFn kfn() { return &sum_kernel<NWN, NWL, G, H>; }

#define ZXP_ROW(N, G) {kfn<N, 1, G, 0>(), kfn<N, 2, G, 0>(), kfn<N, 3, G, 0>(), kfn<N, 4, G, 0>()}
// [general][nwn][nwl - 1]
const KernelFn kTable[2][kMaxWordsNode + 1][kMaxWordsOther] = {
    {ZXP_ROW(0, false), ZXP_ROW(1, false), ZXP_ROW(2, false), ZXP_ROW(3, false), ZXP_ROW(4, false)},
    {ZXP_ROW(0, true), ZXP_ROW(1, true), ZXP_ROW(2, true), ZXP_ROW(3, true), ZXP_ROW(4, true)},
};
#undef ZXP_ROW
#define ZXP_ROW(N, H) {kfn<N, 1, false, H>(), kfn<N, 2, false, H>(), kfn<N, 3, false, H>(), kfn<N, 4, false, H>()}
// counting variants (no pairs or zero forms; at most 11 odd nodes, so nwn <= 1):
// [16-bit counters][nwn][nwl - 1]
const KernelFn kHist[2][2][kMaxWordsOther] = {
    {ZXP_ROW(0, 1), ZXP_ROW(1, 1)},
    {ZXP_ROW(0, 2), ZXP_ROW(1, 2)},
};
#undef ZXP_ROW

// 0: table path, 1: 32-bit counters, 2: 16-bit counters
int hist_mode(const Plan& pl) {
    if (pl.kp.npairs > 0 || pl.has_zero) return 0;
    if (pl.m_odd <= kHistMaxOdd32) return 1;
    if (pl.m_odd <= kHistMaxOdd16) return 2;
    return 0;
}

KernelFn pick(const Plan& pl) {
    const int nwl = pl.nwl < 1 ? 1 : pl.nwl;
    const int h = hist_mode(pl);
    if (h) return kHist[h - 1][pl.nwn][nwl - 1];
    const bool general = pl.kp.npairs > 0 || pl.has_zero;
    return kTable[general ? 1 : 0][pl.nwn][nwl - 1];
}

}  // namespace

size_t sum_smem_bytes(const Plan& pl) {
    const size_t nw = (size_t)pl.nwn + (size_t)(pl.nwl < 1 ? 1 : pl.nwl);
    const size_t ntab = 8u * (size_t)pl.kp.tab_stride;
    const int h = hist_mode(pl);
    const size_t hwords = h == 2 ? (ntab + 1) / 2 : (h == 1 ? ntab : 0);
    return sizeof(zw64) * (ntab + 4u * pl.kp.npairs + kThreads / 32) + sizeof(uint64_t) * kMaxK +
           sizeof(uint32_t) * kMaxK * nw + sizeof(uint32_t) * hwords * (size_t)kThreads;
}

uint64_t sum_max_span(const Plan& pl) { return hist_mode(pl) == 2 ? kSpan16 : (1ull << 18); }

int sum_threads() { return kThreads; }

cudaError_t sum_launch(const Plan& pl, const zw64* dtable, const zw64* dpv, const uint32_t* dF,
                       const uint64_t* dADJ, uint64_t first, uint64_t count, uint64_t span,
                       int grid, zw64* partials,
                       unsigned int* counter, DevResult* result, cudaStream_t stream) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint64_t nslices = (count + span - 1) / span;
    fn<<<grid, kThreads, smem, stream>>>(pl.kp, dtable, dpv, dF, dADJ, first, count, span, nslices,
                                         partials, counter, pl.K, pl.e0, result);
    return cudaGetLastError();
}

cudaError_t sum_occupancy(const Plan& pl, int* blocks_per_sm) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kThreads, smem);
}

}  // namespace zxp
