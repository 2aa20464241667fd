// batch.cu -- the batch kernel's table and general variants
// (batch_kernel.cuh), the choice of variant and the launch, and the gather
// of finished result slots.
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch_kernel.cuh"

namespace zxp {

namespace batchk {
extern const BatchFn kTable[3][kMaxWordsNode + 1][kMaxWordsOther] = {
    ZXP_BATCH_ALL(0), ZXP_BATCH_ALL(1), ZXP_BATCH_ALL(2)};
}  // namespace batchk

namespace {

using namespace batchk;

__global__ void __launch_bounds__(256)
gather_kernel(DevResult* __restrict__ results, const uint32_t* __restrict__ slots, uint32_t n,
              DevResult* __restrict__ out) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        DevResult* r = results + slots[i];
        out[i] = *r;
        *r = DevResult{{0, 0, 0, 0}, 0, 0};
    }
}

// key: variant << 8 | nwn << 4 | nwl
BatchFn pick(int key) {
    const int nwn = (key >> 4) & 7, nwl = key & 7, v = (key >> 8) & 15;
    if (v >= 9) return kLut[v == 13 ? 3 : v - 9][nwn][nwl - 1];
    if (v >= 7) return kShared[v - 7][nwn][nwl - 1];
    if (v >= 3) return kHist[v - 3][nwn][nwl - 1];
    return kTable[v][nwn][nwl - 1];
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
    const int h = core::var_hist((key >> 8) & 15);
    return core::smem_bytes(ntab_cap, npairs_cap, (key >> 4) & 7, key & 7, h, threads, kMaxK,
                            core::lut_entries_cap(h));
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
