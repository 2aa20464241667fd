// kernel.cu -- exact exponential sum of one parametric scalar on sm_103a.
//
// One thread per Gray-code slice of a resident grid (the walk itself is in
// kernel_core.cuh).  Threads reduce by warp shuffles, then per block in
// shared memory, then the last block to finish adds the per-block partials
// (App. E's pairwise sum, done as a shuffle tree) and multiplies by the
// scalar's constant K once.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "kernel.h"
#include "kernel_core.cuh"
#include "plan.h"

namespace zxp {

namespace {

using namespace core;
constexpr int kThreads = kMaxThreads;

template <int NWN, int NWL, int VAR>
__global__ void __launch_bounds__(kThreads)
sum_kernel(const __grid_constant__ KernelParams p, const zw64* __restrict__ gtable,
           const zw64* __restrict__ gpv, const uint32_t* __restrict__ gF,
           const uint64_t* __restrict__ gADJ, const uint32_t* __restrict__ gS, uint64_t first,
           uint64_t count, uint64_t span,
           uint64_t nslices, zw64* __restrict__ partials, unsigned int* __restrict__ counter,
           const zw64 K, const int32_t e0, DevResult* __restrict__ result) {
    constexpr int NW = NWN + NWL;
    constexpr bool GENERAL = var_general(VAR);
    constexpr int HIST = var_hist(VAR);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t ntab = p.tab_size;
    const Smem sm = carve<NW, HIST>(smem_raw, ntab, p.npairs);
    if (HIST) {
        const uint32_t nwords = HIST == 2 ? (ntab + 1) / 2 : ntab;
        uint4* h4 = reinterpret_cast<uint4*>(sm.sH);
        for (uint32_t i = threadIdx.x; i < nwords * blockDim.x / 4; i += blockDim.x)
            h4[i] = make_uint4(0, 0, 0, 0);
    }
    load_tables<NW, GENERAL>(p, sm, gtable, gpv, gF, gADJ, gS);
    __syncthreads();

    zw64 acc = zw_zero();
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    walk<NWN, NWL, GENERAL, HIST, var_xtra(VAR)>(p, sm, first, count, span, nslices,
                                  (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u), gstride,
                                  HIST == 2 || nslices > gstride, false, acc);

    // reduction: warp shuffles, block, then the last block over the partials
    __shared__ unsigned int s_last;
    acc = block_reduce(acc, sm.sred);
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
        v = block_reduce(v, sm.sred);
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
                          const uint64_t*, const uint32_t*, uint64_t, uint64_t,
                          uint64_t, uint64_t, zw64*, unsigned int*, const zw64, const int32_t,
                          DevResult*);

template <int NWN, int NWL, int V>
constexpr KernelFn kfn() { return &sum_kernel<NWN, NWL, V>; }

#define ZXP_ROW(N, V) {kfn<N, 1, V>(), kfn<N, 2, V>(), kfn<N, 3, V>(), kfn<N, 4, V>()}
#define ZXP_ALL(V) {ZXP_ROW(0, V), ZXP_ROW(1, V), ZXP_ROW(2, V), ZXP_ROW(3, V), ZXP_ROW(4, V)}
// table / general variants: [variant 0..2][nwn][nwl - 1]
const KernelFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther] = {ZXP_ALL(0), ZXP_ALL(1), ZXP_ALL(2)};
// counting variants (tables of at most 128 entries: nwn <= 1): [variant - 3][nwn][nwl - 1]
const KernelFn kHist[4][2][kMaxWordsOther] = {
    {ZXP_ROW(0, 3), ZXP_ROW(1, 3)}, {ZXP_ROW(0, 4), ZXP_ROW(1, 4)},
    {ZXP_ROW(0, 5), ZXP_ROW(1, 5)}, {ZXP_ROW(0, 6), ZXP_ROW(1, 6)},
};
#undef ZXP_ALL
#undef ZXP_ROW

KernelFn pick(const Plan& pl) {
    const int nwl = pl.nwl < 1 ? 1 : pl.nwl;
    const int v = variant(pl);
    if (v >= 3) return kHist[v - 3][pl.nwn][nwl - 1];
    return kTable[v][pl.nwn][nwl - 1];
}

}  // namespace

cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> set;   // (device, kernel) -> limit
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = set[std::make_pair(dev, fn)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

size_t sum_smem_bytes(const Plan& pl) {
    return smem_bytes(pl.kp.tab_size, pl.kp.npairs, kernel_words(pl), hist_mode(pl), kThreads);
}

uint64_t sum_max_span(const Plan& pl) { return max_span(hist_mode(pl)); }

int sum_threads() { return kThreads; }

cudaError_t sum_launch(const Plan& pl, const zw64* dtable, const zw64* dpv, const uint32_t* dF,
                       const uint64_t* dADJ, const uint32_t* dS, uint64_t first, uint64_t count,
                       uint64_t span,
                       int grid, zw64* partials,
                       unsigned int* counter, DevResult* result, cudaStream_t stream) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    const uint64_t nslices = (count + span - 1) / span;
    fn<<<grid, kThreads, smem, stream>>>(pl.kp, dtable, dpv, dF, dADJ, dS, first, count, span, nslices,
                                         partials, counter, pl.K, pl.e0, result);
    return cudaGetLastError();
}

cudaError_t sum_occupancy(const Plan& pl, int* blocks_per_sm) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kThreads, smem);
}

}  // namespace zxp
