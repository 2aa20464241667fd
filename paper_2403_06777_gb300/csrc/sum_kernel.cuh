// sum_kernel.cuh -- the single-scalar sum kernel template.  Its variants
// are instantiated in two translation units (kernel.cu: table and general
// variants; kernel_count.cu: counting variants) so that they compile in
// parallel; kernel.cu picks one per scalar.
//
// One thread per Gray-code slice of a resident grid (the walk itself is in
// kernel_core.cuh).  Threads reduce by warp shuffles, then per block in
// shared memory, then the last block to finish adds the per-block partials
// (App. E's pairwise sum, done as a shuffle tree) and multiplies by the
// scalar's constant K once.
#pragma once
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "kernel_core.cuh"
#include "plan.h"

namespace zxp {
namespace sumk {

using namespace core;
constexpr int kThreads = kMaxThreads;

using KernelFn = void (*)(const KernelParams, const zw64*, const zw64*, const uint32_t*,
                          const uint64_t*, const uint32_t*, uint64_t, uint64_t,
                          uint64_t, uint64_t, zw64*, unsigned int*, const zw64, const int32_t,
                          DevResult*, const int32_t);


// variant tables: [variant][nwn][nwl - 1]
extern const KernelFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther];   // kernel.cu
extern const KernelFn kHist[4][2][kMaxWordsOther];                    // kernel_count.cu (nwn <= 1)
extern const KernelFn kShared[2][kMaxWordsNode + 1][kMaxWordsOther];  // kernel_count.cu
extern const KernelFn kLut[6][2][kMaxWordsOther];   // block lookup: variants 9, 10, 11, 13, 14, 15

namespace {

// Write a result: its value, then its flags (never 0) with a release store:
// system scope when a host polls the flags word in pinned memory (it then
// reads the value only after it is complete), device scope for a result in
// device memory.
__device__ __forceinline__ void publish_result(DevResult* r, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               int32_t e, int32_t flags, bool host) {
    r->c[0] = (int64_t)c0;
    r->c[1] = (int64_t)c1;
    r->c[2] = (int64_t)c2;
    r->c[3] = (int64_t)c3;
    r->e = e;
    if (host)
        cuda::atomic_ref<int32_t, cuda::thread_scope_system>(r->flags).store(flags, cuda::memory_order_release);
    else
        cuda::atomic_ref<int32_t, cuda::thread_scope_device>(r->flags).store(flags, cuda::memory_order_release);
}

template <int NWN, int NWL, int VAR>
__global__ void __launch_bounds__(kThreads, VAR >= 11 ? 2 : (VAR >= 9 ? 5 : (VAR >= 7 ? 3 : 1)))
sum_kernel(const __grid_constant__ KernelParams p, const zw64* __restrict__ gtable,
           const zw64* __restrict__ gpv, const uint32_t* __restrict__ gR,
           const uint64_t* __restrict__ gADJ, const uint32_t* __restrict__ gS, uint64_t first,
           uint64_t count, uint64_t span,
           uint64_t nslices, zw64* __restrict__ acc_g, unsigned int* __restrict__ counter,
           const zw64 K, const int32_t e0, DevResult* __restrict__ result, const int32_t host_result) {
    constexpr int NW = NWN + NWL;
    constexpr bool GENERAL = var_general(VAR);
    constexpr int HIST = var_hist(VAR);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const uint32_t ntab = p.tab_size;
    const Smem sm = carve<NW, HIST>(smem_raw, ntab, p.npairs, k_cap(p.k),
                                    HIST >= 4 ? ((p.lut_entries + 1u) & ~1u) : 0u);
    // the table copies are in flight while the counters are cleared
    if (threadIdx.x == 0) {
        mbar_init(&s_bar);
        issue_tables<NWN, NWL, GENERAL, HIST>(p, sm, gtable, gpv, gR, gADJ, gS, &s_bar);
    }
    if (HIST >= 5) {
        // lane-private counters: only rows (J, M) with M < tab_stride are used
        constexpr uint32_t tm = (1u << kLaneRowShift) - 1u, nq = (uint32_t)kLaneCounters * 8u;
        uint4* h4 = reinterpret_cast<uint4*>(sm.sH);
        for (uint32_t i = threadIdx.x; i < (blockDim.x >> 5) * nq; i += blockDim.x)
            if ((((i % nq) >> 3) & tm) < p.tab_stride) h4[i] = make_uint4(0, 0, 0, 0);
    } else if (HIST) {
        uint4* h4 = reinterpret_cast<uint4*>(sm.sH);
        for (uint32_t i = threadIdx.x; i < counter_words(HIST, ntab, blockDim.x) / 4; i += blockDim.x)
            h4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    uint32_t phase = 0;
    const bool loaded = wait_tables(p, sm, &s_bar, phase);
    const bool ok = __syncthreads_and(loaded) != 0;

    zw64 acc = zw_zero();
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    const bool fold_each = HIST == 2 || nslices > gstride;
    // warp-shared counters with one slice per thread: one fold per block
    const bool block_fold = (HIST == 3 || HIST == 4) && !fold_each;
    if (ok)
        walk<NWN, NWL, GENERAL, HIST, var_xtra(VAR), var_outer(VAR)>(p, sm, first, count, span, nslices,
                                      (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u), gstride,
                                      fold_each, false, !block_fold, acc);

    // reduction: warp shuffles, then the block; each block adds K x (its sum)
    // into the accumulator acc_g with 64-bit atomic adds (exact mod 2^64, any
    // order), and the last block to finish moves it to the result and clears
    // it (acc_g and *counter are zero between launches)
    // (bit 31 of the counter: some block could not load its tables; the
    // result is then flagged 2 and is not the sum)
    if constexpr (HIST == 3 || HIST == 4) {
        if (block_fold) acc = fold_block_counters<HIST>(p, sm);   // (uniform branch)
        else acc = block_reduce(acc, sm.sred);
    } else {
        acc = block_reduce(acc, sm.sred);
    }
    if (threadIdx.x == 0) {
        const zw64 r = zw_mul(K, acc);
        if (gridDim.x == 1) {     // one block: its sum is the result
            publish_result(result, r.c[0], r.c[1], r.c[2], r.c[3], e0, ok ? 1 : 3, host_result != 0);
            return;
        }
        if (!ok) atomicOr(counter, 0x80000000u);
        unsigned long long* g = reinterpret_cast<unsigned long long*>(acc_g);
        for (int c = 0; c < 4; c++) atomicAdd(g + c, (unsigned long long)r.c[c]);
        // the acquire-release increment orders this block's adds before it and,
        // in the last block, every block's adds before the reads below
        const unsigned int done =
            cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(*counter).fetch_add(
                1u, cuda::memory_order_acq_rel);
        if ((done & 0x7FFFFFFFu) == gridDim.x - 1) {
            uint64_t v[4];
            for (int c = 0; c < 4; c++) {
                v[c] = __ldcg(g + c);
                g[c] = 0ull;
            }
            *counter = 0u;       // ready for the next launch on this workspace
            publish_result(result, v[0], v[1], v[2], v[3], e0, 1 | ((done >> 31) ? 2 : 0), host_result != 0);
        }
    }
}

template <int NWN, int NWL, int V>
constexpr KernelFn kfn() { return &sum_kernel<NWN, NWL, V>; }

}  // namespace

}  // namespace sumk
}  // namespace zxp

#define ZXP_SUM_ROW(N, V) {kfn<N, 1, V>(), kfn<N, 2, V>(), kfn<N, 3, V>(), kfn<N, 4, V>()}
#define ZXP_SUM_ALL(V) {ZXP_SUM_ROW(0, V), ZXP_SUM_ROW(1, V), ZXP_SUM_ROW(2, V), ZXP_SUM_ROW(3, V), ZXP_SUM_ROW(4, V)}
