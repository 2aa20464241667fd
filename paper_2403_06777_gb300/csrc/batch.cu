// batch.cu -- many parametric scalars of uneven k in one persistent launch.
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
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "kernel_core.cuh"
#include "plan.h"

namespace zxp {

namespace {

using namespace core;

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
    const Smem sm = carve<NW, HIST>(smem_raw, ntab_cap, npairs_cap);
    if (HIST) {
        const uint32_t nwords = HIST == 2 ? (ntab_cap + 1) / 2 : ntab_cap;
        for (uint32_t i = threadIdx.x; i < nwords * blockDim.x; i += blockDim.x) sm.sH[i] = 0;
    }
    if (threadIdx.x == 0) s_loaded = 0xFFFFFFFFu;
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
            load_tables<NW, GENERAL>(sp, sm, bs.table, bs.pv, bs.frows, bs.adj, bs.seek);
            if (threadIdx.x == 0) s_loaded = ch.scalar;
            __syncthreads();
        }
        // slices: a multiple of 8 terms (chunk starts are multiples of 8)
        uint64_t span = (ch.count + per - 1) / per;
        span = (span + 7) & ~7ull;
        if (span < 8) span = 8;
        if (span > cap) span = cap;
        const uint64_t nslices = (ch.count + span - 1) / span;
        zw64 acc = zw_zero();
        walk<NWN, NWL, GENERAL, HIST, var_xtra(VAR)>(sp, sm, ch.first, ch.count, span, nslices,
                                                     threadIdx.x & ~31u, blockDim.x,
                                                     HIST == 2 || nslices > blockDim.x, true, acc);
        acc = block_reduce(acc, sm.sred);
        if (threadIdx.x == 0) {
            const zw64 r = zw_mul(bs.K, acc);
            DevResult* out = results + ch.slot;
            for (int i = 0; i < 4; i++)
                atomicAdd(reinterpret_cast<unsigned long long*>(&out->c[i]), (unsigned long long)r.c[i]);
            out->e = bs.e0;
            out->flags = 1;
        }
        __syncthreads();   // s_chunk and the reduction scratch are reused
    }
}

using BatchFn = void (*)(const unsigned char*, const BatchChunk*, uint32_t, unsigned int*, DevResult*,
                         uint32_t, uint32_t, uint32_t);

template <int NWN, int NWL, int V>
constexpr BatchFn bfn() { return &batch_kernel<NWN, NWL, V>; }

#define ZXP_ROW(N, V) {bfn<N, 1, V>(), bfn<N, 2, V>(), bfn<N, 3, V>(), bfn<N, 4, V>()}
#define ZXP_ALL(V) {ZXP_ROW(0, V), ZXP_ROW(1, V), ZXP_ROW(2, V), ZXP_ROW(3, V), ZXP_ROW(4, V)}
const BatchFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther] = {ZXP_ALL(0), ZXP_ALL(1), ZXP_ALL(2)};
const BatchFn kHist[4][2][kMaxWordsOther] = {
    {ZXP_ROW(0, 3), ZXP_ROW(1, 3)}, {ZXP_ROW(0, 4), ZXP_ROW(1, 4)},
    {ZXP_ROW(0, 5), ZXP_ROW(1, 5)}, {ZXP_ROW(0, 6), ZXP_ROW(1, 6)},
};
#undef ZXP_ALL
#undef ZXP_ROW

// key: variant << 8 | nwn << 4 | nwl
BatchFn pick(int key) {
    const int nwn = (key >> 4) & 7, nwl = key & 7, v = (key >> 8) & 7;
    if (v >= 3) return kHist[v - 3][nwn][nwl - 1];
    return kTable[v][nwn][nwl - 1];
}

__global__ void __launch_bounds__(256)
gather_kernel(DevResult* __restrict__ results, const uint32_t* __restrict__ slots, uint32_t n,
              DevResult* __restrict__ out) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        DevResult* r = results + slots[i];
        out[i] = *r;
        *r = DevResult{{0, 0, 0, 0}, 0, 0};
    }
}

}  // namespace

cudaError_t gather_results(DevResult* results, const uint32_t* slots, uint32_t n, DevResult* out,
                           cudaStream_t stream) {
    if (!n) return cudaSuccess;
    gather_kernel<<<1, 256, 0, stream>>>(results, slots, n, out);
    return cudaGetLastError();
}

int batch_key(const Plan& pl) {
    const int nwl = pl.nwl < 1 ? 1 : pl.nwl;
    return (core::variant(pl) << 8) | (pl.nwn << 4) | nwl;
}

size_t batch_smem_bytes(int key, uint32_t ntab_cap, uint32_t npairs_cap, int threads) {
    const int nw = ((key >> 4) & 7) + (key & 7);
    return core::smem_bytes(ntab_cap, npairs_cap, nw, core::var_hist((key >> 8) & 7), threads);
}

cudaError_t batch_occupancy(int key, uint32_t ntab_cap, uint32_t npairs_cap, int threads,
                            int* blocks_per_sm) {
    BatchFn fn = pick(key);
    const size_t smem = batch_smem_bytes(key, ntab_cap, npairs_cap, threads);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t batch_launch(int key, const unsigned char* scalars, const BatchChunk* chunks,
                         uint32_t nchunks, unsigned int* queue, DevResult* results,
                         uint32_t ntab_cap, uint32_t npairs_cap, int threads, int grid,
                         uint32_t slices_per_thread, cudaStream_t stream) {
    BatchFn fn = pick(key);
    const size_t smem = batch_smem_bytes(key, ntab_cap, npairs_cap, threads);
    const cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, stream>>>(scalars, chunks, nchunks, queue, results, ntab_cap,
                                        npairs_cap, slices_per_thread);
    return cudaGetLastError();
}

}  // namespace zxp
