// kernel.cu -- exact exponential sum of one parametric scalar on sm_103a:
// the table and general variants of the sum kernel (sum_kernel.cuh), the
// choice of variant, and the launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "sum_kernel.cuh"

namespace zxp {

namespace sumk {
// table / general variants: [variant 0..2][nwn][nwl - 1]
extern const KernelFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther] = {
    ZXP_SUM_ALL(0), ZXP_SUM_ALL(1), ZXP_SUM_ALL(2)};
}  // namespace sumk

namespace {

using namespace sumk;

KernelFn pick(const Plan& pl) {
    const int nwl = pl.nwl < 1 ? 1 : pl.nwl;
    const int v = variant(pl);
    if (v >= 9) return kLut[v >= 13 ? v - 10 : v - 9][pl.nwn][nwl - 1];
    if (v >= 7) return kShared[v - 7][pl.nwn][nwl - 1];
    if (v >= 3) return kHist[v - 3][pl.nwn][nwl - 1];
    return kTable[v][pl.nwn][nwl - 1];
}

}  // namespace

cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
    // (set even below 48 KB: the default limit covers static and dynamic
    // shared memory together, and the kernels have static shared memory)
    if (bytes == 0) return cudaSuccess;
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

static size_t smem_for(const Plan& pl, int threads) {
    const int h = hist_mode(pl);
    return smem_bytes(pl.kp.tab_size, pl.kp.npairs, pl.nwn, kernel_words(pl) - pl.nwn, h, threads,
                      k_cap(pl.kp.k), h >= 4 ? ((pl.kp.lut_entries + 1u) & ~1u) : 0u);
}

// Threads per block: 128 for the lane-private block lookup (32 KB of
// counters per 128 threads), else 256.
static int block_threads(const Plan& pl) { return hist_mode(pl) >= 5 ? 128 : kThreads; }

size_t sum_smem_bytes(const Plan& pl) { return smem_for(pl, block_threads(pl)); }

uint64_t sum_max_span(const Plan& pl) { return max_span(hist_mode(pl)); }

int sum_threads() { return kThreads; }

int sum_variant(const Plan& pl) { return variant(pl); }

cudaError_t sum_launch(const Plan& pl, const zw64* dtable, const zw64* dpv, const uint32_t* dF,
                       const uint64_t* dADJ, const uint32_t* dS, const uint32_t* dzq, const zw64* dftab,
                       uint64_t first, uint64_t count, uint64_t span, int grid, zw64* acc,
                       unsigned int* counter, DevResult* result, bool host_result, cudaStream_t stream) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    if (pl.k_inner && (!dzq || !dftab)) return cudaErrorInvalidValue;
    KernelParams kp = pl.kp;
    kp.zqcol = dzq;
    kp.ftab = dftab;
    kp.extra_tx = test_extra_tx();
    // four states a thread (kernel_core.cuh, walk_lut_pair): the lane-private
    // block lookup over whole aligned blocks of 256 Gray indices, variables 6
    // and 7 below every cut parity
    kp.pair_walk = (hist_mode(pl) >= 5 && pl.kp.k >= 8 && (!pl.k_inner || pl.kp.zq_lo >= 8) &&
                    count && !(first & 255u) && !(count & 255u) && !(span & 255u))
                       ? 1u
                       : 0u;
    const uint64_t nslices = (count + span - 1) / span;
    fn<<<grid, block_threads(pl), smem, stream>>>(kp, dtable, dpv, dF, dADJ, dS, first, count, span, nslices,
                                         acc, counter, pl.K, pl.e0, result, host_result ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t sum_occupancy(const Plan& pl, int* blocks_per_sm) {
    KernelFn fn = pick(pl);
    const size_t smem = sum_smem_bytes(pl);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    // the answer depends on (device, kernel, shared memory) only: cache it
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, int> cache;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    const auto key = std::make_tuple(dev, reinterpret_cast<const void*>(fn), smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) { *blocks_per_sm = it->second; return cudaSuccess; }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block_threads(pl), smem);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = *blocks_per_sm;
    }
    return e;
}

void sum_shape(const Plan& pl, int sm_count, int max_grid_cap, uint64_t count, uint64_t* span, int* grid) {
    int bps = 1;
    if (sum_occupancy(pl, &bps) != cudaSuccess || bps < 1) bps = 1;
    const int bt = block_threads(pl);
    // Ranges too short to give every thread of a full-occupancy grid 256
    // terms run with at most 768 threads per SM: fewer, longer slices
    // amortise each thread's fixed work (seek, counter fold, reduction).
    const int short_bps = 3 * kThreads / bt;
    if (bps > short_bps && count < (uint64_t)sm_count * (uint64_t)bps * bt * 256u) bps = short_bps;
    int max_grid = sm_count * bps;
    if (max_grid > max_grid_cap) max_grid = max_grid_cap;
    const uint64_t threads = (uint64_t)max_grid * (uint64_t)bt;
    uint64_t sp = (count + threads - 1) / threads;
    // (block lookup: a multiple of 16, so that a warp's lanes reach the
    // flips of variable 3 together; inner parameters: a multiple of the run
    // over which the cut parities stay constant (at most 2^16 terms), so
    // that a warp's lanes fold their counters at the same step instead of
    // one after another)
    uint64_t al = hist_mode(pl) >= 4 ? 16 : 8;
    if (pl.k_inner && pl.kp.zq_lo < 64) al = std::max<uint64_t>(al, 1ull << std::min<uint32_t>(pl.kp.zq_lo, 16));
    // (lane-private block lookup: slices of whole blocks of 256, which the
    // walk takes four states at a time)
    if (hist_mode(pl) >= 5 && sp >= 256) al = std::max<uint64_t>(al, 256);
    sp = (sp + al - 1) & ~(al - 1);
    if (sp < 64) sp = 64;
    const uint64_t cap = sum_max_span(pl) & ~(al - 1);
    if (sp > cap) sp = cap;   // longer ranges: several slices per thread
    const uint64_t nslices = (count + sp - 1) / sp;
    uint64_t g = (nslices + (uint64_t)bt - 1) / (uint64_t)bt;
    if (g > (uint64_t)max_grid) g = (uint64_t)max_grid;
    if (g < 1) g = 1;
    *span = sp;
    *grid = (int)g;
}

}  // namespace zxp
