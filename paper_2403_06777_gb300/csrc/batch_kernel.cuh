// batch_kernel.cuh -- many parametric scalars of uneven k in one persistent launch.
//
// The host cuts every scalar's range [0, 2^k) into chunks; a grid of
// resident blocks pulls chunk indices from one global counter (work
// stealing: a block that finishes early takes the next chunk), loads the
// chunk's scalar tables into shared memory only when the scalar changes, sums
// the chunk with the same per-thread Gray-code walk as the single-scalar
// kernel, and adds K * (block sum) into that scalar's result with 64-bit
// atomics (integer adds: exact and order independent).  Scalars of one
// launch share a kernel variant (form words, counting mode); the host groups
// a batch by variant.
//
// The kernel's variants are instantiated in batch.cu (table and general) and
// batch_count.cu (counting) so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "kernel_core.cuh"
#include "plan.h"

namespace zxp {
namespace batchk {

using namespace core;

using BatchFn = void (*)(const unsigned char*, const BatchChunk*, uint32_t, unsigned int*, DevResult*,
                         uint32_t, uint32_t, uint32_t);


// variant tables: [variant][nwn][nwl - 1]
extern const BatchFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther];   // batch.cu
extern const BatchFn kHist[4][2][kMaxWordsOther];                    // batch_count.cu
extern const BatchFn kShared[2][kMaxWordsNode + 1][kMaxWordsOther];  // batch_count.cu
extern const BatchFn kLut[4][2][kMaxWordsOther];   // block lookup: variants 9, 10, 11, 13

namespace {

template <int NWN, int NWL, int VAR>
__global__ void __launch_bounds__(kMaxThreads)
batch_kernel(const unsigned char* __restrict__ scalars, const BatchChunk* __restrict__ chunks,
             uint32_t nchunks, unsigned int* __restrict__ queue, DevResult* __restrict__ results,
             uint32_t ntab_cap, uint32_t npairs_cap, uint32_t slices_per_thread) {
    constexpr int NW = NWN + NWL;
    constexpr bool GENERAL = var_general(VAR);
    constexpr int HIST = var_hist(VAR);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KernelParams sp;
    __shared__ uint32_t s_chunk, s_loaded;
    __shared__ __align__(8) uint64_t s_bar;
    const Smem sm = carve<NW, HIST>(smem_raw, ntab_cap, npairs_cap, kMaxK, lut_entries_cap(HIST));
    if (HIST)
        for (uint32_t i = threadIdx.x; i < counter_words(HIST, ntab_cap, blockDim.x); i += blockDim.x)
            sm.sH[i] = 0;
    if (threadIdx.x == 0) {
        s_loaded = 0xFFFFFFFFu;
        mbar_init(&s_bar);
    }
    uint32_t phase = 0;   // bulk loads so far (the barrier's phase parity)
    bool ok = true;       // the current scalar's tables are loaded
    const uint64_t per = (uint64_t)blockDim.x * slices_per_thread;
    const uint64_t cap = HIST == 2 ? kSpan16 : kSpan32;

    for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t c = s_chunk;
        if (c >= nchunks) break;
        const BatchChunk ch = chunks[c];
        const BatchScalar& bs =
            *reinterpret_cast<const BatchScalar*>(scalars + (size_t)ch.scalar * kBatchScalarBytes);
        if (ch.scalar != s_loaded) {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&bs.kp);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
            for (uint32_t i = threadIdx.x; i < sizeof(KernelParams) / 4; i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            const bool loaded =
                load_tables<NWN, NWL, GENERAL, HIST>(sp, sm, bs.table, bs.pv, bs.rows, bs.adj, bs.seek,
                                                     &s_bar, phase);
            if (threadIdx.x == 0) s_loaded = ch.scalar;
            ok = __syncthreads_and(loaded) != 0;
        }
        // slices: a multiple of 8 terms, 16 for the block lookup (chunk starts
        // are multiples of 8)
        uint64_t span = (ch.count + per - 1) / per;
        span = HIST >= 4 ? (span + 15) & ~15ull : (span + 7) & ~7ull;   // (see sum_shape)
        if (span < 16) span = 16;
        if (span > cap) span = cap;
        const uint64_t nslices = (ch.count + span - 1) / span;
        zw64 acc = zw_zero();
        if (ok)
            walk<NWN, NWL, GENERAL, HIST, var_xtra(VAR)>(sp, sm, ch.first, ch.count, span, nslices,
                                                         threadIdx.x & ~31u, blockDim.x,
                                                         HIST == 2 || nslices > blockDim.x, true, true, acc);
        acc = block_reduce(acc, sm.sred);
        if (threadIdx.x == 0) {
            const zw64 r = zw_mul(bs.K, acc);
            DevResult* out = results + ch.slot;
            for (int i = 0; i < 4; i++)
                atomicAdd(reinterpret_cast<unsigned long long*>(&out->c[i]), (unsigned long long)r.c[i]);
            out->e = bs.e0;
            // flag 2: this scalar's tables could not be loaded (not the sum)
            atomicOr(reinterpret_cast<int*>(&out->flags), ok ? 1 : 3);
        }
        __syncthreads();   // s_chunk and the reduction scratch are reused
    }
}

template <int NWN, int NWL, int V>
constexpr BatchFn bfn() { return &batch_kernel<NWN, NWL, V>; }

}  // namespace

}  // namespace batchk
}  // namespace zxp

#define ZXP_BATCH_ROW(N, V) {bfn<N, 1, V>(), bfn<N, 2, V>(), bfn<N, 3, V>(), bfn<N, 4, V>()}
#define ZXP_BATCH_ALL(V) {ZXP_BATCH_ROW(0, V), ZXP_BATCH_ROW(1, V), ZXP_BATCH_ROW(2, V), ZXP_BATCH_ROW(3, V), ZXP_BATCH_ROW(4, V)}
