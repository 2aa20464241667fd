// kernel_wide.cu -- the sum kernel with coefficients modulo 2^128, for
// scalars whose sqrt2 exponent e0 lies in (124, 252]: there the numerator of
// a circuit amplitude is bounded by 2^(e0/2) < 2^127 (zring.h), so the sum
// modulo 2^128 is the exact value (the paper's Eq. 2 is an exact sum).
//
// One thread per Gray-code slice, as the 64-bit kernels; every term is
// evaluated on its own (the general variant: the value of its phase exponent
// J and node count M from the (J, M) table, times the values of its
// phase-pair forms, zero when a zero form is set), so that one kernel family
// (node words x other words) serves every scalar.  The block's sum goes to
// the accumulator with 64-bit atomics that carry: the low word's add
// returns the old value, and a wrap of the low word adds one to the high
// word's addend.
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernel.h"
#include "kernel_core.cuh"
#include "plan.h"

namespace zxp {
namespace {

using namespace core;
constexpr int kWideThreads = kMaxThreads;

using WideFn = void (*)(const KernelParams, const zw128*, const zw128*, const uint32_t*, const uint64_t*,
                        const uint32_t*, uint64_t, uint64_t, uint64_t, uint64_t, uint64_t*, unsigned int*,
                        const zw128, const int32_t, DevResultW*);

template <int NWN, int NWL>
__global__ void __launch_bounds__(kWideThreads)
sum_kernel_w(const __grid_constant__ KernelParams p, const zw128* __restrict__ gtable,
             const zw128* __restrict__ gpv, const uint32_t* __restrict__ gR, const uint64_t* __restrict__ gADJ,
             const uint32_t* __restrict__ gS, uint64_t first, uint64_t count, uint64_t span, uint64_t nslices,
             uint64_t* __restrict__ acc_g, unsigned int* __restrict__ counter, const zw128 K, const int32_t e0,
             DevResultW* __restrict__ result) {
    constexpr int NW = NWN + NWL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    // (p.tab_size: the (J, M) table's entries, 8 * tab_stride)
    const Smem sm = carve<NW, 0, 2>(smem_raw, p.tab_size, p.npairs, k_cap(p.k));
    if (threadIdx.x == 0) {
        mbar_init(&s_bar);
        issue_tables<NWN, NWL, true, 0, 2>(p, sm, reinterpret_cast<const zw64*>(gtable),
                                           reinterpret_cast<const zw64*>(gpv), gR, gADJ, gS, &s_bar);
    }
    __syncthreads();
    uint32_t phase = 0;
    const bool loaded = wait_tables(p, sm, &s_bar, phase);
    const bool ok = __syncthreads_and(loaded) != 0;
    zw128 acc = zw_zero<u128>();
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    if (ok)
        walk<NWN, NWL, true, 0, false, false, zw128>(p, sm, first, count, span, nslices,
                                                     (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u),
                                                     gstride, false, false, true, acc);
    acc = block_reduce(acc, reinterpret_cast<zw128*>(sm.sred));
    if (threadIdx.x == 0) {
        const zw128 r = zw_mul(K, acc);
        if (!ok) atomicOr(counter, 0x80000000u);
        unsigned long long* g = reinterpret_cast<unsigned long long*>(acc_g);
        for (int c = 0; c < 4; c++) {
            const unsigned long long lo = (unsigned long long)r.c[c], hi = (unsigned long long)(r.c[c] >> 64);
            const unsigned long long old = atomicAdd(g + 2 * c, lo);
            atomicAdd(g + 2 * c + 1, hi + (old + lo < old ? 1ull : 0ull));
        }
        // the acquire-release increment orders this block's adds before it and,
        // in the last block, every block's adds before the reads below
        const unsigned int done =
            cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(*counter).fetch_add(
                1u, cuda::memory_order_acq_rel);
        if ((done & 0x7FFFFFFFu) == gridDim.x - 1) {
            for (int c = 0; c < 4; c++) {
                result->c[c] = (int64_t)__ldcg(g + 2 * c);
                result->hi[c] = (int64_t)__ldcg(g + 2 * c + 1);
                g[2 * c] = 0ull;
                g[2 * c + 1] = 0ull;
            }
            *counter = 0u;
            result->e = e0;
            result->flags = 1 | ((done >> 31) ? 2 : 0);
        }
    }
}

template <int NWN, int NWL>
constexpr WideFn wfn() { return &sum_kernel_w<NWN, NWL>; }
#define ZXP_WIDE_ROW(N) {wfn<N, 1>(), wfn<N, 2>(), wfn<N, 3>(), wfn<N, 4>()}
const WideFn kWide[kMaxWordsNode + 1][kMaxWordsOther] = {ZXP_WIDE_ROW(0), ZXP_WIDE_ROW(1), ZXP_WIDE_ROW(2),
                                                          ZXP_WIDE_ROW(3), ZXP_WIDE_ROW(4)};
static_assert(kMaxWordsNode == 4 && kMaxWordsOther == 4, "instantiation table");

}  // namespace

cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);   // kernel.cu

cudaError_t sum_launch_wide(const Plan& pl, const zw128* dtab_w, const zw128* dpv_w, const uint32_t* drows,
                            const uint64_t* dADJ, const uint32_t* dS, const uint32_t* dzq, const zw128* dftab_w,
                            uint64_t first, uint64_t count, int sm_count, uint64_t* acc, unsigned int* counter,
                            DevResultW* result, cudaStream_t stream) {
    if (pl.k_inner && (!dzq || !dftab_w)) return cudaErrorInvalidValue;
    const int nwl = pl.nwl < 1 ? 1 : pl.nwl;
    if (pl.nwn > kMaxWordsNode || nwl > kMaxWordsOther) return cudaErrorInvalidValue;
    const WideFn fn = kWide[pl.nwn][nwl - 1];
    KernelParams kp = pl.kp;
    kp.tab_size = 8u * kp.tab_stride;   // the (J, M) table
    kp.zqcol = dzq;
    kp.ftab = reinterpret_cast<const zw64*>(dftab_w);
    kp.extra_tx = test_extra_tx();
    const size_t smem = smem_bytes(kp.tab_size, kp.npairs, pl.nwn, nwl, 0, kWideThreads, k_cap(kp.k), 0, 2);
    cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kWideThreads, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    // one slice per thread of a resident grid: at least 64 terms, a
    // multiple of 8 (and of the run over which the cut parities stay
    // constant, so that a warp's lanes flush together), at most 2^18
    const uint64_t threads = (uint64_t)sm_count * bps * kWideThreads;
    uint64_t al = 8;
    if (pl.k_inner && pl.kp.zq_lo < 64) al = std::max<uint64_t>(al, 1ull << std::min<uint32_t>(pl.kp.zq_lo, 16));
    uint64_t sp = (count + threads - 1) / threads;
    sp = (sp + al - 1) & ~(al - 1);
    if (sp < 64) sp = 64;
    const uint64_t cap = kSpan32 & ~(al - 1);
    if (sp > cap) sp = cap;
    const uint64_t nslices = (count + sp - 1) / sp;
    uint64_t grid = (nslices + kWideThreads - 1) / kWideThreads;
    grid = std::min<uint64_t>(grid, (uint64_t)sm_count * bps);
    if (grid < 1) grid = 1;
    fn<<<(unsigned)grid, kWideThreads, smem, stream>>>(kp, dtab_w, dpv_w, drows, dADJ, dS, first, count, sp,
                                                      nslices, acc, counter, pl.K_w, pl.e0, result);
    return cudaGetLastError();
}

}  // namespace zxp
