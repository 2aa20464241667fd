// kernel_core.cuh -- device code shared by the single-scalar and the batched
// sum kernels: shared-memory layout of one scalar's tables, the per-thread
// Gray-code walk over slices, and the block reduction.
//
// Each thread walks contiguous Gray-code slices [t0, t0 + span) of the
// assignment space (x = t ^ (t >> 1)); consecutive assignments differ in the
// bit ctz(t), so a step XORs that variable's flip row into the form bits
// (the AND / XOR-reduce steps of Sec. 3.3 done incrementally) and updates the
// quadratic phase with one bit of A x.  A term is then one table entry
// K * w^(J + 2M) (1 + sqrt2)^M (see plan.h), multiplied by any phase-pair
// values, accumulated in four int64 coefficients modulo 2^64 -- or, in the
// counting variants, the pair (J, M) is counted and the counts are folded
// into Z[w] at the end of each slice batch.  Integer adds make the result
// bit-exact and independent of the reduction order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "kernel.h"
#include "plan.h"

namespace zxp {
namespace core {

constexpr int kMaxThreads = 256;
constexpr int kMaxWarps = kMaxThreads / 32;
// counting variants: 32-bit counters for tables of at most 48 entries (48 KB
// per 256-thread block), 16-bit counters packed two per word for at most 128
// (64 KB per block; slices shorter than 2^16 terms)
constexpr uint64_t kSpan16 = 65528;        // largest multiple of 8 below 2^16
constexpr uint64_t kSpan32 = 1ull << 18;   // longest slice of the other variants

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

// read-only global load of a Z[w] value (the inner table)
__device__ __forceinline__ zw64 ldg_zw(const zw64* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 a = __ldg(q), b = __ldg(q + 1);
    return zw_make(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ zw64 shfl_xor_zw(zw64 v, int off) {
    zw64 r;
#pragma unroll
    for (int c = 0; c < 4; c++) r.c[c] = __shfl_xor_sync(0xffffffffu, v.c[c], off);
    return r;
}

// the same for 128-bit coefficients (64-byte values, 16-byte aligned)
__device__ __forceinline__ u128 u128_of(unsigned long long lo, unsigned long long hi) {
    return ((u128)hi << 64) | (u128)lo;
}
__device__ __forceinline__ zw128 lds_zw(const zw128* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    zw128 r;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const ulonglong2 a = q[c];
        r.c[c] = u128_of(a.x, a.y);
    }
    return r;
}
__device__ __forceinline__ zw128 ldg_zw(const zw128* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    zw128 r;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const ulonglong2 a = __ldg(q + c);
        r.c[c] = u128_of(a.x, a.y);
    }
    return r;
}
__device__ __forceinline__ zw128 shfl_xor_zw(zw128 v, int off) {
    zw128 r;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v.c[c], off);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v.c[c] >> 64), off);
        r.c[c] = u128_of(lo, hi);
    }
    return r;
}

// warp shuffles, then one value per warp through shared memory; the block
// total is valid in thread 0
template <class W>
__device__ __forceinline__ zwt<W> block_reduce(zwt<W> v, zwt<W>* sred) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = zw_add(v, shfl_xor_zw(v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? sred[lane] : zw_zero<W>();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = zw_add(v, shfl_xor_zw(v, off));
    }
    return v;
}

// 0: table path, 1: lane-private 32-bit counters, 2: lane-private 16-bit
// counters, 3: warp-shared 32-bit counters (by the number of distinct term
// values the table holds), 4: block lookup with warp-shared counters over
// kLutRows rows of the table (when the plan built the lookup), 5: block
// lookup with lane-private 32-bit counters (rows of 2^lut_tsh counters, the
// phase exponent taken mod 8 by a mask), 6: the same over two lookup tables
constexpr uint32_t kHistMaxEntries32 = 48;
constexpr uint32_t kHistMaxEntries16 = 128;
constexpr uint32_t kHistMaxEntriesShared = 2048;
constexpr uint32_t kLutEntries = (1u << kLutMaxBits) + 8u;
constexpr uint32_t kLut2Entries = (2u << kLutMaxBits) + 8u;
// lookup words a block sized for any scalar of lookup kind h holds
__host__ __device__ constexpr uint32_t lut_entries_cap(int h) { return h == 6 ? kLut2Entries : kLutEntries; }
inline int hist_mode(const Plan& pl) {
    if (pl.general) return 0;
    // inner parameters: lane-private counters (folded per lane) or the table
    if (pl.k_inner && !pl.lut_ok)
        return pl.kp.tab_size <= kHistMaxEntries32 ? 1 : (pl.kp.tab_size <= kHistMaxEntries16 ? 2 : 0);
    if (pl.lut_ok) return pl.lut_lane ? (pl.lut_two ? 6 : 5) : 4;
    if (pl.kp.tab_size <= kHistMaxEntries32) return 1;
    if (pl.kp.tab_size <= kHistMaxEntries16) return 2;
    if (pl.kp.tab_size <= kHistMaxEntriesShared) return 3;
    return 0;
}
inline int kernel_words(const Plan& pl) { return pl.nwn + (pl.nwl < 1 ? 1 : pl.nwl); }
// kernel variant: 0 table, 1 table + extra index bits, 2 general (phase-pair
// products), 3/4 lane-private 32-bit counters (+ extra bits), 5/6
// lane-private 16-bit counters (+ extra), 7/8 warp-shared counters (+ extra),
// 9/10 block lookup (+ extra), 11 block lookup with lane-private counters,
// 13 the same with two lookup tables; 14 and 15: 11 and 13 for scalars with
// inner parameters (their lanes fold at cut flips)
inline int variant(const Plan& pl) {
    if (pl.general) return 2;
    const int x = pl.kp.xshift ? 1 : 0;
    const int h = hist_mode(pl);
    if (pl.k_inner && h >= 5) return h == 5 ? 14 : 15;
    return h == 0 ? x : 1 + 2 * h + x;   // block lookup: 9, or 10 with folded bits; 11
}
__host__ __device__ constexpr bool var_general(int v) { return v == 2; }
__host__ __device__ constexpr int var_hist(int v) { return v >= 14 ? v - 9 : (v >= 3 ? (v - 1) / 2 : 0); }
__host__ __device__ constexpr bool var_xtra(int v) { return v == 1 || (v >= 3 && v <= 10 && (v & 1) == 0); }
__host__ __device__ constexpr bool var_outer(int v) { return v >= 14; }
// 32-bit counter words of one block
__host__ __device__ constexpr uint32_t counter_words(int h, uint32_t ntab, uint32_t threads) {
    return h == 1 ? ntab * threads
                  : (h == 2 ? (ntab + 1) / 2 * threads
                            : (h == 3 ? ntab * (threads / 32)
                                      : (h == 4 ? (uint32_t)(kLutRows / 8) * ntab * (threads / 32)
                                                : (h >= 5 ? (uint32_t)kLaneCounters * threads : 0u))));
}
inline uint64_t max_span(int h) { return h == 2 ? kSpan16 : kSpan32; }

// Shared memory of one block: [table][pair values][reduction][adjacency]
// [flip rows][counters], sized for the largest scalar the block may hold.
struct Smem {
    zw64* sT;
    zw64* sPV;
    zw64* sred;
    uint64_t* sADJ;
    uint32_t* sS;   // seek tables
    uint64_t* sL;   // block lookup (HIST 4, 5)
    uint32_t* sF;
    uint32_t* sH;
};

// words of one seek-table entry (flip words, adjacency, quadratic bit)
__host__ __device__ constexpr uint32_t seek_stride(int nw) { return ((uint32_t)nw + 3u + 3u) & ~3u; }
__host__ __device__ constexpr uint32_t seek_words(int nw, uint32_t kcap = kMaxK) {
    return ((kcap + 3) / 4) * 16u * seek_stride(nw);
}
// Shared-memory capacities for a scalar with k variables and a block lookup
// over nU forms (a block sized for one scalar): variables rounded up to an
// even count (at least 4), lookup entries to an even count, so that every
// region stays 16-byte aligned.  Blocks that hold any scalar use kMaxK and
// kLutEntries.
__host__ __device__ constexpr uint32_t k_cap(uint32_t k) { return k < 4 ? 4u : (k + 1u) & ~1u; }
__host__ __device__ constexpr uint32_t lut_cap(uint32_t nU) { return ((1u << nU) + 9u) & ~1u; }

// ew: 32-byte words of one table value (1: 64-bit coefficients, 2: 128-bit)
__host__ __device__ inline size_t smem_bytes(uint32_t ntab_cap, uint32_t npairs_cap, int nwn, int nwl,
                                             int h, int threads, uint32_t kcap = kMaxK,
                                             uint32_t lutcap = kLutEntries, uint32_t ew = 1) {
    return sizeof(zw64) * ew * (ntab_cap + 4u * npairs_cap + kMaxWarps) + sizeof(uint64_t) * kcap +
           sizeof(uint32_t) * seek_words(nwn + nwl, kcap) + sizeof(uint32_t) * (size_t)kcap * row_words(nwn, nwl) +
           (h >= 4 ? sizeof(uint64_t) * lutcap : 0) +
           sizeof(uint32_t) * (size_t)counter_words(h, ntab_cap, (uint32_t)threads);
}

template <int NW, int HIST, uint32_t EW = 1>
__device__ __forceinline__ Smem carve(unsigned char* raw, uint32_t ntab_cap, uint32_t npairs_cap,
                                      uint32_t kcap = kMaxK, uint32_t lutcap = kLutEntries) {
    // (step rows last: 16-byte aligned after the 8-byte adjacency words, as
    // kcap is even)
    const uint32_t hist_words = counter_words(HIST, ntab_cap, blockDim.x);
    Smem s;
    s.sT = reinterpret_cast<zw64*>(raw);
    s.sPV = s.sT + EW * ntab_cap;
    s.sred = s.sPV + EW * 4u * npairs_cap;
    // 16-byte aligned first (vector loads and stores): seek tables, counters
    s.sS = reinterpret_cast<uint32_t*>(s.sred + EW * kMaxWarps);
    s.sL = reinterpret_cast<uint64_t*>(s.sS + seek_words(NW, kcap));
    s.sH = reinterpret_cast<uint32_t*>(s.sL + (HIST >= 4 ? lutcap : 0u));
    s.sADJ = reinterpret_cast<uint64_t*>(s.sH + hist_words);
    s.sF = reinterpret_cast<uint32_t*>(s.sADJ + kcap);
    return s;
}

// ---- bulk copies into shared memory (TMA, cp.async.bulk) -------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Each try_wait suspends the thread for a bounded time; kDefaultWaitTries
// of them (about a second in all) end a wait that would otherwise never end.
constexpr uint32_t kWaitTries = kDefaultWaitTries;

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

// Copy one scalar's tables into shared memory with bulk copies on the
// mbarrier `bar` (initialised, count 1).  Called by one thread; the copies
// complete the barrier's current phase.
template <int NWN, int NWL, bool GENERAL, int HIST, uint32_t EW = 1>
__device__ __forceinline__ void issue_tables(const KernelParams& p, const Smem& sm,
                                             const zw64* __restrict__ gtable,
                                             const zw64* __restrict__ gpv,
                                             const uint32_t* __restrict__ gR,
                                             const uint64_t* __restrict__ gADJ,
                                             const uint32_t* __restrict__ gS, uint64_t* bar) {
    constexpr int NW = NWN + NWL;
    constexpr uint32_t RW = row_words(NWN, NWL);
    const uint32_t ns = ((p.k + 3) / 4) * 16u * seek_stride(NW);
    const uint32_t bt = p.tab_size * 32u * EW, bs = ns * 4u, br = p.k * RW * 4u, ba = round16(p.k * 8u);
    const uint32_t bpv = GENERAL ? 4u * p.npairs * 32u * EW : 0u;
    const uint32_t bl = HIST >= 4 ? round16(p.lut_entries * 8u) : 0u;
    // order the shared-memory reads of a previous scalar before the
    // asynchronous writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // (p.extra_tx: bytes that no copy delivers, 0 unless a test asks for a
    // wait that runs out)
    mbar_expect_tx(bar, bt + bs + br + ba + bpv + bl + p.extra_tx);
    if (bt) bulk_copy(sm.sT, gtable, bt, bar);
    if (bs) bulk_copy(sm.sS, gS, bs, bar);
    if (br) bulk_copy(sm.sF, gR, br, bar);
    if (ba) bulk_copy(sm.sADJ, gADJ, ba, bar);
    if (bpv) bulk_copy(sm.sPV, gpv, bpv, bar);
    if (bl) bulk_copy(sm.sL, gS + ns, bl, bar);   // the block lookup follows the seek tables
}

// Wait (bounded) for the copies of issue_tables: the barrier's phase
// `phase` (the loads so far; advanced here).  Every thread calls it, after
// a block barrier that follows the barrier's initialisation.  Returns false
// if the wait gave up (the tables are then not valid).  Variables 0..2
// beyond k get zero adjacency rows.
__device__ __forceinline__ bool wait_tables(const KernelParams& p, const Smem& sm, uint64_t* bar,
                                            uint32_t& phase) {
    bool ok = false;
    for (uint32_t i = 0; i < kWaitTries; i++)
        if (mbar_try_wait(bar, phase & 1u)) { ok = true; break; }
    phase++;
    if (threadIdx.x < 3 && threadIdx.x >= p.k) sm.sADJ[threadIdx.x] = 0;
    return ok;
}

// issue_tables by thread 0, then wait_tables; the caller synchronises the
// block before and after.
template <int NWN, int NWL, bool GENERAL, int HIST>
__device__ __forceinline__ bool load_tables(const KernelParams& p, const Smem& sm,
                                            const zw64* __restrict__ gtable,
                                            const zw64* __restrict__ gpv,
                                            const uint32_t* __restrict__ gR,
                                            const uint64_t* __restrict__ gADJ,
                                            const uint32_t* __restrict__ gS, uint64_t* bar,
                                            uint32_t& phase) {
    if (threadIdx.x == 0) issue_tables<NWN, NWL, GENERAL, HIST>(p, sm, gtable, gpv, gR, gADJ, gS, bar);
    return wait_tables(p, sm, bar, phase);
}

// Walk the slices s = s_begin + lane, s_begin + stride + lane, ... (< nslices)
// of [first, first + count) and add the terms into acc.  s_begin must be
// the same for the 32 lanes of a warp (the loop is warp-uniform, lanes past
// the end skip the work) so that the counter fold can use full-warp
// reductions.  The counters (HIST) are zero on entry, and on exit when
// fold_each or clear_on_exit is set.
// Block-lookup walk (HIST 4, no phase-pair or zero forms).  A term's counter
// is J * stride + M with J = the phase exponent (rows up to kLutRows: J is not
// reduced mod 8 inside a block; the fold maps row r to table row r mod 8).
// An aligned block of 8 Gray steps costs one lookup: the forms holding
// variables 0, 1, 2 are the lowest node and linear bits, their values at the
// block's first state index sL, and (A x) restricted to variables 0-2
// indexes the quadratic part; byte s - 1 of the sum is term s's counter
// offset from the block's base.  Other steps update L, J and A x directly;
// the flip of variable 3 between the two blocks of an aligned 16 takes its
// step row and adjacency row from the parameters (the constant bank), so
// only one step in 16 reads a step row from shared memory.  (Slices that are
// a multiple of 16 keep a warp's lanes on one branch.)
// LANE (HIST 5): every lane owns kLaneCounters counters in its own bank
// (counter i of lane l at word i * 32 + l), so the counting atomics of a
// warp never conflict; a counter index is (J mod 8) * 2^tsh + M, the block's
// base plus the looked-up offset modulo 8 * 2^tsh.
template <int NWN, int NWL, bool XTRA, bool LANE, bool TWO, bool OUTER>
__device__ __forceinline__ void walk_lut(const KernelParams& p, const Smem& sm, uint64_t first,
                                         uint64_t count, uint64_t span, uint64_t nslices,
                                         uint64_t s_begin, uint64_t stride, bool fold_each,
                                         bool clear_on_exit, bool final_fold, zw64& acc) {
    constexpr int NW = NWN + NWL;
    constexpr uint32_t RW = row_words(NWN, NWL);
    constexpr uint32_t SW = seek_stride(NW);
    const zw64* __restrict__ sT = sm.sT;
    const uint64_t* __restrict__ sADJ = sm.sADJ;
    const uint32_t* __restrict__ sF = sm.sF;
    const uint32_t* __restrict__ sS = sm.sS;
    const uint64_t* __restrict__ sL = sm.sL;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ts = p.tab_stride;
    // one plane of kLutRows * ts counters per value of the folded phase-pair
    // and zero bits (constant inside a block)
    const uint32_t plane = (uint32_t)kLutRows * ts;
    const uint32_t nbins = plane << p.xshift;
    uint32_t* const wc = sm.sH + warp * nbins;
    const uint32_t no = p.lut_no, nn = p.lut_nn, lsh = p.lut_shift;
    const uint32_t mo = (1u << no) - 1u, mn = (1u << nn) - 1u;
    // two tables (TWO): the first na lookup bits index sL, the rest sLB
    const uint32_t na = TWO ? p.lut_na : no + nn, ma = (1u << na) - 1u;
    const uint64_t* __restrict__ sLB = sL + (1u << na);
    const uint64_t* __restrict__ qlut = TWO ? sLB + (1u << (no + nn - na)) : sL + (1u << (no + nn));
    // inner parameters (lane-private counters only)
    constexpr bool outer = LANE && OUTER;
    constexpr uint32_t tsh = kLaneRowShift, cm = (8u << tsh) - 1u;
    uint32_t* const lbase = sm.sH + warp * ((uint32_t)kLaneCounters * 32u);
    uint32_t* const wl = lbase + lane;
    unsigned char* const wlb = reinterpret_cast<unsigned char*>(wl);
    const uint32_t rb = p.lane_row_bytes;
    // lane-private counter idx: one multiply-add for its address
    auto lctr = [&](uint32_t idx) { return reinterpret_cast<uint32_t*>(wlb + idx * rb); };

    // counter i = x * plane + row * ts + m holds table entry
    // (((row mod 8) * ts + m) << xshift) | x, and (row mod 8) * ts + m = i mod 8 ts
    const uint32_t t8 = 8u * ts;
    auto fold = [&](bool clear) {
        __syncwarp();
        if constexpr (LANE) {
            // lane l adds up counter i = l (+32) over the 32 lanes with
            // 16-byte reads in lane-rotated order (the 8 lanes of a
            // quarter-warp read 8 different columns: 32 banks) and clears it;
            // counter i holds table entry (i >> tsh) * ts + (i & (2^tsh - 1))
            const uint32_t tm = (1u << tsh) - 1u;
            for (uint32_t i = lane; i <= cm; i += 32) {
                if ((i & tm) >= ts) continue;   // M < ts: never counted, never cleared
                uint4* row = reinterpret_cast<uint4*>(lbase + i * 32u);
                uint32_t c = 0;
#pragma unroll
                for (uint32_t j = 0; j < 8; j++) {
                    const uint4 v = row[(j + lane) & 7u];
                    c += v.x + v.y + v.z + v.w;
                }
                if (c) acc = zw_madd32(acc, lds_zw(sT + (i >> tsh) * ts + (i & tm)), c);
                if (clear) {
#pragma unroll
                    for (uint32_t j = 0; j < 8; j++) row[(j + lane) & 7u] = make_uint4(0, 0, 0, 0);
                }
            }
            __syncwarp();
            return;
        }
        uint32_t ti = lane, x = 0, r = lane;
        while (ti >= t8) ti -= t8;
        while (r >= plane) { r -= plane; x++; }
        for (uint32_t i = lane; i < nbins; i += 32) {
            const uint32_t c = wc[i];
            if (c) {
                acc = zw_madd32(acc, lds_zw(sT + ((ti << p.xshift) | x)), c);
                if (clear) wc[i] = 0;
            }
            ti += 32;
            while (ti >= t8) ti -= t8;
            r += 32;
            while (r >= plane) { r -= plane; x++; }
        }
        __syncwarp();
    };


    const uint64_t end = first + count;
    for (uint64_t s0 = s_begin; s0 < nslices; s0 += stride) {
        const uint64_t s = s0 + lane;
        if (s < nslices) {
            uint64_t t = first + s * span;
            const uint64_t tend = (end - t < span) ? end : t + span;
            const uint64_t x = t ^ (t >> 1);
            uint32_t L[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) L[w] = p.INV[w];
            uint64_t a64 = 0;
            uint32_t q = 0;
            const uint32_t nnib = (p.k + 3) >> 2;
            for (uint32_t b = 0; b < nnib; b++) {
                const uint32_t v = (uint32_t)(x >> (4 * b)) & 15u;
                const uint32_t* e = sS + (b * 16u + v) * SW;
                uint32_t ev[SW];
#pragma unroll
                for (uint32_t w4 = 0; w4 < SW; w4 += 4) {
                    const uint4 t4 = *reinterpret_cast<const uint4*>(e + w4);
                    ev[w4] = t4.x; ev[w4 + 1] = t4.y; ev[w4 + 2] = t4.z; ev[w4 + 3] = t4.w;
                }
                q ^= ev[NW + 2] ^ ((uint32_t)__popc(v & (uint32_t)(a64 >> (4 * b))) & 1u);
                a64 ^= ((uint64_t)ev[NW + 1] << 32) | ev[NW];
#pragma unroll
                for (int w = 0; w < NW; w++) L[w] ^= ev[w];
            }
            // the walk keeps bits 0-31 of A x: a flip of variable i >= 32
            // (once per 2^32 terms) takes its bit from the state itself
            uint32_t a = (uint32_t)a64;
            const uint32_t* __restrict__ sADJw = reinterpret_cast<const uint32_t*>(sADJ);
            // 4 (A x)_i (mod 8) for the state of Gray index tp, before flipping i
            auto quad4 = [&](int i, uint64_t tp) -> uint32_t {
                if (i < 32) return a >> i << 2;
                return ((uint32_t)__popcll(sADJ[i] & (tp ^ (tp >> 1))) & 1u) << 2;
            };
            uint32_t Jl;
            {
                uint32_t P0 = 0, P1 = 0, X2 = 0;
#pragma unroll
                for (int w = 0; w < NWN; w++) X2 ^= L[w] & p.CB[w];
#pragma unroll
                for (int w = 0; w < NWL; w++) {
                    const uint32_t v = L[NWN + w];
                    P0 += __popc(v & p.C0[w]);
                    P1 += __popc(v & p.C1[w]);
                    X2 ^= v & p.C2[w];
                }
                Jl = P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q);
            }
            // a = A x: flipping variable i adds 4 (A x)_i to J and XORs
            // adjacency row i into a.  us = the lookup slot of the current
            // state's bits (lut_slot is linear: each flip XORs its row's slot
            // change, bits 8 and up of the row's last word)
            uint32_t us;
            {
                uint32_t u = (L[NWN] >> lsh) & mo;
                if (NWN) u |= (L[0] & mn) << no;
                us = TWO ? (lut_slot(u & ma) | (lut_slot(u >> na) << na)) : lut_slot(u);
            }
            // inner parameters: the cut parities zq of the current state; a
            // lane folds its own counters, times the inner table at zq, when
            // a flip changes zq and at the end of the slice
            uint32_t zq = 0;
            if (outer)
                for (uint64_t m = x >> p.zq_lo; m; m &= m - 1)
                    zq ^= __ldg(p.zqcol + p.zq_lo + (uint32_t)__ffsll((long long)m) - 1u);
            // the inner table at the current cut parities, loaded when they
            // change, a whole run before the flush that uses it
            zw64 fz = zw_zero();
            if (outer) fz = ldg_zw(p.ftab + zq);
            // (lane-private counters have no folded bits, so the entry of
            // phase J and node count M is w^J u^M, u = w^2 (1 + sqrt2) =
            // w + w^2 + w^3: for each M the eight counts combine into the
            // integer element d_M = (c0 - c4) + (c1 - c5) w + (c2 - c6) w^2 +
            // (c3 - c7) w^3 (w^4 = -1), and sum_M d_M u^M is evaluated by
            // Horner's rule, a multiplication by u being seven additions of
            // coefficients.  In 32-bit integers: a run holds at most 2^18
            // terms (one slice) and each of at most eight steps at most
            // triples the coefficients, below 2^31.  One product with the
            // inner-table entry at the run's cut parities follows.)
            auto flush = [&]() {
                if constexpr (LANE) {
                    uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                    for (uint32_t Mi = ts; Mi-- > 0;) {
                        uint32_t c[8];
                        unsigned char* ptr = reinterpret_cast<unsigned char*>(lctr(Mi));
#pragma unroll
                        for (uint32_t J = 0; J < 8; J++) {
                            c[J] = *reinterpret_cast<uint32_t*>(ptr);
                            *reinterpret_cast<uint32_t*>(ptr) = 0u;
                            ptr += rb << tsh;
                        }
                        // (s0 + s1 w + s2 w^2 + s3 w^3) u + d_M
                        const uint32_t x = s1 + s2;
                        const uint32_t n0 = 0u - (x + s3), n1 = s0 - s2 - s3, n2 = s0 + s1 - s3, n3 = s0 + x;
                        s0 = n0 + (c[0] - c[4]);
                        s1 = n1 + (c[1] - c[5]);
                        s2 = n2 + (c[2] - c[6]);
                        s3 = n3 + (c[3] - c[7]);
                    }
                    const zw64 sum = zw_make((uint64_t)(int64_t)(int32_t)s0, (uint64_t)(int64_t)(int32_t)s1,
                                             (uint64_t)(int64_t)(int32_t)s2, (uint64_t)(int64_t)(int32_t)s3);
                    acc = zw_add(acc, zw_mul(sum, fz));
                }
            };
            auto cut_flip = [&](int i) {
                if (outer && (uint32_t)i >= p.zq_lo) {
                    const uint32_t dz = __ldg(p.zqcol + i);
                    if (dz) {
                        flush();
                        zq ^= dz;
                        fz = ldg_zw(p.ftab + zq);
                    }
                }
            };

            auto node_count = [&]() {
                uint32_t M = 0;
#pragma unroll
                for (int w = 0; w < NWN; w++) M += __popc(L[w]);
                return M;
            };
            // counter plane of the folded bits: the pair forms' bits and "some
            // zero form is set"
            auto plane_base = [&]() -> uint32_t {
                if (!XTRA) return 0u;
                uint32_t z = 0;
                if (p.has_zero) {
#pragma unroll
                    for (int w = 0; w < NWL; w++) z |= L[NWN + w] & p.Z[w];
                }
                return ((L[NWN] & p.pmask) | ((z != 0 ? 1u : 0u) << p.zshift)) * plane;
            };
            // the linear part of a flip with step row f (L before the XOR) and
            // the lookup slot change du
            auto step = [&](const uint32_t* f, uint32_t du) {
                // (4 d1 mod 8 needs only the parity of d1: one popcount)
                uint32_t d0 = 0, x1 = 0;
#pragma unroll
                for (int w = 0; w < NWL; w++) {
                    d0 += __popc(L[NWN + w] & f[NW + w]);
                    x1 ^= L[NWN + w] & f[NW + NWL + w];
                }
                Jl += f[NW + 2 * NWL] - 2u * d0 - 4u * (uint32_t)__popc(x1);
                us ^= du;
#pragma unroll
                for (int w = 0; w < NW; w++) L[w] ^= f[w];
            };
            // the 8 terms of an aligned block from one lookup, then the block's
            // net change: variable 2 flipped (Gray 000 -> 100), its forms, its
            // adjacency row and the block's phase change
            auto block8 = [&]() {
                uint32_t lo, hi;
                if constexpr (TWO) {
                    // (the entries' byte sums never carry into the next byte,
                    // so each 32-bit half adds on its own; with one table the
                    // 64-bit form measured faster)
                    const uint2 e1 = *reinterpret_cast<const uint2*>(sL + (us & ma));
                    const uint2 e2 = *reinterpret_cast<const uint2*>(sLB + (us >> na));
                    const uint2 eq = *reinterpret_cast<const uint2*>(qlut + (a & 7u));
                    lo = e1.x + e2.x + eq.x;
                    hi = e1.y + e2.y + eq.y;
                } else {
                    const uint64_t e = sL[us] + qlut[a & 7u];
                    lo = (uint32_t)e;
                    hi = (uint32_t)(e >> 32);
                }
                if constexpr (LANE) {
                    // the block's base (< 64) added to all offset bytes at once
                    // (each sum < 256: no carry between bytes) and every byte
                    // taken mod 8 * 2^tsh by one mask
                    const uint32_t b0 = TWO ? (((Jl << tsh) & (7u << tsh)) | node_count())
                                            : ((Jl & 7u) << tsh) + node_count();
                    const uint32_t bx = b0 * 0x01010101u, mk = cm * 0x01010101u;
                    const uint32_t w0 = (lo + bx) & mk, w1 = (hi + bx) & mk;
                    // (bytes by byte permutes: one instruction each, 5 % fewer
                    // cycles than shifts and masks, measured)
                    atomicAdd(lctr(b0), 1u);
                    atomicAdd(lctr(__byte_perm(w0, 0u, 0x4440u)), 1u);
                    atomicAdd(lctr(__byte_perm(w0, 0u, 0x4441u)), 1u);
                    atomicAdd(lctr(__byte_perm(w0, 0u, 0x4442u)), 1u);
                    atomicAdd(lctr(w0 >> 24), 1u);
                    atomicAdd(lctr(__byte_perm(w1, 0u, 0x4440u)), 1u);
                    atomicAdd(lctr(__byte_perm(w1, 0u, 0x4441u)), 1u);
                    atomicAdd(lctr(__byte_perm(w1, 0u, 0x4442u)), 1u);
                } else {
                    const int base = (int)(plane_base() + (Jl & 7u) * ts + node_count()) - (int)nn;
                    uint32_t* const wb = wc + base;
                    atomicAdd(wb + nn, 1u);
                    atomicAdd(wb + __byte_perm(lo, 0u, 0x4440u), 1u);
                    atomicAdd(wb + __byte_perm(lo, 0u, 0x4441u), 1u);
                    atomicAdd(wb + __byte_perm(lo, 0u, 0x4442u), 1u);
                    atomicAdd(wb + (lo >> 24), 1u);
                    atomicAdd(wb + __byte_perm(hi, 0u, 0x4440u), 1u);
                    atomicAdd(wb + __byte_perm(hi, 0u, 0x4441u), 1u);
                    atomicAdd(wb + __byte_perm(hi, 0u, 0x4442u), 1u);
                }
#pragma unroll
                for (int w = 0; w < NW; w++) L[w] ^= p.R[2][w];
                Jl += hi >> 24;
                a ^= (uint32_t)p.A4[2];
                us ^= p.U4[2];
            };
            // variable 3 (between the two blocks of 8 of an aligned 16): step
            // row and adjacency row in the parameters
            auto flip3 = [&]() {
                Jl += (a >> 1) & 4u;
                a ^= (uint32_t)p.A4[3];
                step(p.R[3], p.U4[3]);
            };
            auto load_row = [&](int i, uint32_t (&fr)[RW]) {
#pragma unroll
                for (uint32_t w4 = 0; w4 < RW; w4 += 4) {
                    const uint4 t4 = *reinterpret_cast<const uint4*>(sF + i * RW + w4);
                    fr[w4] = t4.x; fr[w4 + 1] = t4.y; fr[w4 + 2] = t4.z; fr[w4 + 3] = t4.w;
                }
            };
            auto ctz64 = [](uint64_t v) -> int {
                const uint32_t vl = (uint32_t)v;
                return vl ? __ffs(vl) - 1 : 31 + __ffs((uint32_t)(v >> 32));
            };
            for (;;) {
                if ((t & 15u) == 0 && tend - t >= 16) {
                    // aligned blocks of 16: two lookups, the flip of variable 3
                    // between them, and the flip of variable ctz(t + 16) >= 4
                    // after them, whose step row and adjacency row are read
                    // from shared memory before the block's lookups so that
                    // their latency overlaps the block's work.  (nb: whole
                    // blocks left, at most 2^14 in a slice; t in 32-bit
                    // halves, the high one changing once per 2^32 terms)
                    uint32_t nb = (uint32_t)((tend - t) >> 4);
                    const bool tail = ((tend - t) & 15u) != 0;
                    uint32_t tl = (uint32_t)t, th = (uint32_t)(t >> 32);
                    for (;;) {
                        tl += 16u;
                        if (tl == 0u) th++;
                        const bool more = --nb != 0u || tail;   // t + 16 < tend <= 2^k: ctz < k
                        const int i = !more ? 0 : (tl ? __ffs(tl) - 1 : 31 + __ffs(th));
                        uint32_t fr[RW];
                        load_row(i, fr);
                        const uint32_t adj = sADJw[2 * i];
                        block8();
                        flip3();
                        block8();
                        if (!more) break;
                        cut_flip(i);
                        // (bits above 2: only J mod 8 is used)
                        Jl += i < 32 ? a >> i << 2 : quad4(i, (((uint64_t)th << 32) | tl) - 1u);
                        a ^= adj;
                        step(fr, fr[NW + 2 * NWL] >> 8);
                        if (nb == 0u) break;
                    }
                    t = ((uint64_t)th << 32) | tl;
                    if (t >= tend) break;
                }
                if ((t & 7u) == 0 && tend - t >= 8) {
                    block8();
                    t += 7;
                } else if constexpr (LANE) {
                    atomicAdd(lctr(((Jl & 7u) << tsh) + node_count()), 1u);
                } else {
                    atomicAdd(wc + plane_base() + (Jl & 7u) * ts + node_count(), 1u);
                }
                if (++t >= tend) break;
                // flip variable i = ctz(t): 4 (A x)_i for the quadratic part,
                // the step row for the linear part
                if (((uint32_t)t & 15u) == 8u) {
                    flip3();
                } else {
                    const int i = ctz64(t);
                    cut_flip(i);
                    Jl += quad4(i, t - 1u);   // (bits above 2: only J mod 8 is used)
                    a ^= sADJw[2 * i];
                    uint32_t fr[RW];
                    load_row(i, fr);
                    step(fr, fr[NW + 2 * NWL] >> 8);
                }
            }
            if (outer) flush();
        }
        if (fold_each && !outer) fold(true);
    }
    if (!fold_each && final_fold && !outer) fold(clear_on_exit);
}

// The lane-private block lookup (LANE) over a range [first, first + count)
// whose start, length and slice span are multiples of 256, NS states a
// thread.  The Gray indices of such a range are whole aligned blocks of
// 256: the set of assignments whose bits 8 and up are the Gray code of one
// of the blocks' numbers, with any bits 0-7.  The same set is walked as the
// Gray code over every variable but 7 (NS = 2: compressed index c = t / 2,
// variable v(i) = i for i < 7, i + 1 above) or but 6 and 7 (NS = 4: c =
// t / 4, v(i) = i for i < 6, i + 2 above), in NS states that take every
// value of the variables left out: they take every flip together, so the
// flip rows, the loop and, those variables being below every cut parity
// (zq_lo >= 8), the counters, the cut parities and the folds are shared,
// while each state keeps its own form bits, A x, lookup slot and phase (and
// the warp has NS independent chains of dependent instructions to issue
// from).  The sum of the range is the same; the order of the terms within
// it is not.  Four states measured 3 % faster than two, two 9 % faster than
// one, on the n = 50, T = 80 outer walk.
template <int NWN, int NWL, bool TWO, bool OUTER, int NS = 2>
__device__ __forceinline__ void walk_lut_pair(const KernelParams& p, const Smem& sm, uint64_t first,
                                              uint64_t count, uint64_t span, uint64_t nslices,
                                              uint64_t s_begin, uint64_t stride, bool fold_each,
                                              bool clear_on_exit, bool final_fold, zw64& acc) {
    constexpr int NW = NWN + NWL;
    constexpr uint32_t RW = row_words(NWN, NWL);
    constexpr uint32_t SW = seek_stride(NW);
    const zw64* __restrict__ sT = sm.sT;
    const uint64_t* __restrict__ sADJ = sm.sADJ;
    const uint32_t* __restrict__ sADJw = reinterpret_cast<const uint32_t*>(sm.sADJ);
    const uint32_t* __restrict__ sF = sm.sF;
    const uint32_t* __restrict__ sS = sm.sS;
    const uint64_t* __restrict__ sL = sm.sL;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ts = p.tab_stride;
    const uint32_t no = p.lut_no, nn = p.lut_nn, lsh = p.lut_shift;
    const uint32_t mo = (1u << no) - 1u, mn = (1u << nn) - 1u;
    const uint32_t na = TWO ? p.lut_na : no + nn, ma = (1u << na) - 1u;
    const uint64_t* __restrict__ sLB = sL + (1u << na);
    const uint64_t* __restrict__ qlut = TWO ? sLB + (1u << (no + nn - na)) : sL + (1u << (no + nn));
    constexpr uint32_t tsh = kLaneRowShift, cm = (8u << tsh) - 1u;
    uint32_t* const lbase = sm.sH + warp * ((uint32_t)kLaneCounters * 32u);
    unsigned char* const wlb = reinterpret_cast<unsigned char*>(lbase + lane);
    const uint32_t rb = p.lane_row_bytes;
    auto lctr = [&](uint32_t idx) { return reinterpret_cast<uint32_t*>(wlb + idx * rb); };

    // a lane's counters summed over the 32 lanes (as walk_lut's fold)
    auto fold = [&](bool clear) {
        __syncwarp();
        const uint32_t tm = (1u << tsh) - 1u;
        for (uint32_t i = lane; i <= cm; i += 32) {
            if ((i & tm) >= ts) continue;
            uint4* row = reinterpret_cast<uint4*>(lbase + i * 32u);
            uint32_t c = 0;
#pragma unroll
            for (uint32_t j = 0; j < 8; j++) {
                const uint4 v = row[(j + lane) & 7u];
                c += v.x + v.y + v.z + v.w;
            }
            if (c) acc = zw_madd32(acc, lds_zw(sT + (i >> tsh) * ts + (i & tm)), c);
            if (clear) {
#pragma unroll
                for (uint32_t j = 0; j < 8; j++) row[(j + lane) & 7u] = make_uint4(0, 0, 0, 0);
            }
        }
        __syncwarp();
    };

    struct State {
        uint32_t L[NW];
        uint32_t a, us, Jl;
    };
    auto node_count = [](const State& w) {
        uint32_t M = 0;
#pragma unroll
        for (int v = 0; v < NWN; v++) M += __popc(w.L[v]);
        return M;
    };
    auto step = [&](State& w, const uint32_t* f, uint32_t du) {
        uint32_t d0 = 0, x1 = 0;
#pragma unroll
        for (int v = 0; v < NWL; v++) {
            d0 += __popc(w.L[NWN + v] & f[NW + v]);
            x1 ^= w.L[NWN + v] & f[NW + NWL + v];
        }
        w.Jl += f[NW + 2 * NWL] - 2u * d0 - 4u * (uint32_t)__popc(x1);
        w.us ^= du;
#pragma unroll
        for (int v = 0; v < NW; v++) w.L[v] ^= f[v];
    };
    auto lookup = [&](const State& w, uint32_t& lo, uint32_t& hi) {
        if constexpr (TWO) {
            const uint2 e1 = *reinterpret_cast<const uint2*>(sL + (w.us & ma));
            const uint2 e2 = *reinterpret_cast<const uint2*>(sLB + (w.us >> na));
            const uint2 eq = *reinterpret_cast<const uint2*>(qlut + (w.a & 7u));
            lo = e1.x + e2.x + eq.x;
            hi = e1.y + e2.y + eq.y;
        } else {
            const uint64_t e = sL[w.us] + qlut[w.a & 7u];
            lo = (uint32_t)e;
            hi = (uint32_t)(e >> 32);
        }
    };
    auto block8 = [&](State& w) {
        uint32_t lo, hi;
        lookup(w, lo, hi);
        const uint32_t b0 = TWO ? (((w.Jl << tsh) & (7u << tsh)) | node_count(w))
                                : ((w.Jl & 7u) << tsh) + node_count(w);
        const uint32_t bx = b0 * 0x01010101u, mk = cm * 0x01010101u;
        const uint32_t w0 = (lo + bx) & mk, w1 = (hi + bx) & mk;
        atomicAdd(lctr(b0), 1u);
        atomicAdd(lctr(__byte_perm(w0, 0u, 0x4440u)), 1u);
        atomicAdd(lctr(__byte_perm(w0, 0u, 0x4441u)), 1u);
        atomicAdd(lctr(__byte_perm(w0, 0u, 0x4442u)), 1u);
        atomicAdd(lctr(w0 >> 24), 1u);
        atomicAdd(lctr(__byte_perm(w1, 0u, 0x4440u)), 1u);
        atomicAdd(lctr(__byte_perm(w1, 0u, 0x4441u)), 1u);
        atomicAdd(lctr(__byte_perm(w1, 0u, 0x4442u)), 1u);
#pragma unroll
        for (int v = 0; v < NW; v++) w.L[v] ^= p.R[2][v];
        w.Jl += hi >> 24;
        w.a ^= (uint32_t)p.A4[2];
        w.us ^= p.U4[2];
    };
    auto flip3 = [&](State& w) {
        w.Jl += (w.a >> 1) & 4u;
        w.a ^= (uint32_t)p.A4[3];
        step(w, p.R[3], p.U4[3]);
    };
    auto load_row = [&](int i, uint32_t (&fr)[RW]) {
#pragma unroll
        for (uint32_t w4 = 0; w4 < RW; w4 += 4) {
            const uint4 t4 = *reinterpret_cast<const uint4*>(sF + i * RW + w4);
            fr[w4] = t4.x; fr[w4 + 1] = t4.y; fr[w4 + 2] = t4.z; fr[w4 + 3] = t4.w;
        }
    };
    // NS = 2: variable 7 left out of the Gray code, NS = 4: variables 6
    // and 7; the state of compressed index c: the Gray code of c with clear
    // bits put in there
    constexpr uint32_t XL = NS == 2 ? 7u : 6u;
    auto expand = [](uint64_t c) {
        const uint64_t g = c ^ (c >> 1);
        return (g & ((1u << XL) - 1u)) | ((g >> XL) << 8);
    };
    // the variables' bits of state s: s's bits at variables 7 and 6
    auto sbits = [](int st) -> uint32_t { return (st & 1 ? 128u : 0u) | (st & 2 ? 64u : 0u); };

    const uint64_t end = first + count;
    for (uint64_t s0 = s_begin; s0 < nslices; s0 += stride) {
        const uint64_t s = s0 + lane;
        if (s < nslices) {
            const uint64_t t = first + s * span;
            const uint64_t tend = (end - t < span) ? end : t + span;
            const uint64_t c0 = t >> (NS == 2 ? 1 : 2), x = expand(c0);
            // state A at x (as walk_lut's seek)
            State A;
#pragma unroll
            for (int v = 0; v < NW; v++) A.L[v] = p.INV[v];
            uint64_t a64 = 0;
            uint32_t q = 0;
            const uint32_t nnib = (p.k + 3) >> 2;
            for (uint32_t b = 0; b < nnib; b++) {
                const uint32_t v = (uint32_t)(x >> (4 * b)) & 15u;
                const uint32_t* e = sS + (b * 16u + v) * SW;
                uint32_t ev[SW];
#pragma unroll
                for (uint32_t w4 = 0; w4 < SW; w4 += 4) {
                    const uint4 t4 = *reinterpret_cast<const uint4*>(e + w4);
                    ev[w4] = t4.x; ev[w4 + 1] = t4.y; ev[w4 + 2] = t4.z; ev[w4 + 3] = t4.w;
                }
                q ^= ev[NW + 2] ^ ((uint32_t)__popc(v & (uint32_t)(a64 >> (4 * b))) & 1u);
                a64 ^= ((uint64_t)ev[NW + 1] << 32) | ev[NW];
#pragma unroll
                for (int v2 = 0; v2 < NW; v2++) A.L[v2] ^= ev[v2];
            }
            A.a = (uint32_t)a64;
            {
                uint32_t P0 = 0, P1 = 0, X2 = 0;
#pragma unroll
                for (int v = 0; v < NWN; v++) X2 ^= A.L[v] & p.CB[v];
#pragma unroll
                for (int v = 0; v < NWL; v++) {
                    const uint32_t u = A.L[NWN + v];
                    P0 += __popc(u & p.C0[v]);
                    P1 += __popc(u & p.C1[v]);
                    X2 ^= u & p.C2[v];
                }
                A.Jl = P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q);
            }
            {
                uint32_t u = (A.L[NWN] >> lsh) & mo;
                if (NWN) u |= (A.L[0] & mn) << no;
                A.us = TWO ? (lut_slot(u & ma) | (lut_slot(u >> na) << na)) : lut_slot(u);
            }
            // the other states: A with variable 7 (state 1), 6 (state 2) or
            // both (state 3) flipped
            State W[NS];
            W[0] = A;
#pragma unroll
            for (int st = 1; st < NS; st++) {
                const int i = st == 2 ? 6 : 7;
                W[st] = W[st == 3 ? 2 : 0];
                uint32_t fr[RW];
                load_row(i, fr);
                W[st].Jl += W[st].a >> i << 2;
                W[st].a ^= sADJw[2 * i];
                step(W[st], fr, fr[NW + 2 * NWL] >> 8);
            }
            // the cut parities (variable 7 is below zq_lo: the same for B)
            uint32_t zq = 0;
            if (OUTER)
                for (uint64_t m = x >> p.zq_lo; m; m &= m - 1)
                    zq ^= __ldg(p.zqcol + p.zq_lo + (uint32_t)__ffsll((long long)m) - 1u);
            zw64 fz = zw_zero();
            if (OUTER) fz = ldg_zw(p.ftab + zq);
            // the fold of the counts since the last change of the cut
            // parities, both states' (walk_lut's flush)
            auto flush = [&]() {
                uint32_t s0_ = 0, s1 = 0, s2 = 0, s3 = 0;
                for (uint32_t Mi = ts; Mi-- > 0;) {
                    uint32_t c[8];
                    unsigned char* ptr = reinterpret_cast<unsigned char*>(lctr(Mi));
#pragma unroll
                    for (uint32_t J = 0; J < 8; J++) {
                        c[J] = *reinterpret_cast<uint32_t*>(ptr);
                        *reinterpret_cast<uint32_t*>(ptr) = 0u;
                        ptr += rb << tsh;
                    }
                    const uint32_t xs = s1 + s2;
                    const uint32_t n0 = 0u - (xs + s3), n1 = s0_ - s2 - s3, n2 = s0_ + s1 - s3, n3 = s0_ + xs;
                    s0_ = n0 + (c[0] - c[4]);
                    s1 = n1 + (c[1] - c[5]);
                    s2 = n2 + (c[2] - c[6]);
                    s3 = n3 + (c[3] - c[7]);
                }
                const zw64 sum = zw_make((uint64_t)(int64_t)(int32_t)s0_, (uint64_t)(int64_t)(int32_t)s1,
                                         (uint64_t)(int64_t)(int32_t)s2, (uint64_t)(int64_t)(int32_t)s3);
                acc = zw_add(acc, zw_mul(sum, fz));
            };
            // blocks of 16 compressed steps (the slice's [c0, tend / NS) holds
            // a multiple of 64 of them): variables 0-2 by two lookups each,
            // variable 3 between them, then variable v(ctz(c + 16))
            uint32_t nb = (uint32_t)(((tend >> (NS == 2 ? 1 : 2)) - c0) >> 4);
            uint32_t cl = (uint32_t)c0, ch = (uint32_t)(c0 >> 32);
            for (;;) {
                cl += 16u;
                if (cl == 0u) ch++;
                const bool more = --nb != 0u;   // c + 16 < end / 2 <= 2^(k-1): ctz < k - 1
                const int ic = !more ? 0 : (cl ? __ffs(cl) - 1 : 31 + __ffs(ch));
                const int i = ic < (int)XL ? ic : ic + (NS == 2 ? 1 : 2);
                uint32_t fr[RW];
                load_row(i, fr);
                const uint32_t adj = sADJw[2 * i];
#pragma unroll
                for (int st = 0; st < NS; st++) block8(W[st]);
#pragma unroll
                for (int st = 0; st < NS; st++) flip3(W[st]);
#pragma unroll
                for (int st = 0; st < NS; st++) block8(W[st]);
                if (!more) break;
                if (OUTER && (uint32_t)i >= p.zq_lo) {
                    const uint32_t dz = __ldg(p.zqcol + i);
                    if (dz) {
                        flush();
                        zq ^= dz;
                        fz = ldg_zw(p.ftab + zq);
                    }
                }
                // (bits above 2: only J mod 8 is used; a flip of a variable
                // >= 32 takes its bit of A x from the state before it)
                if (i < 32) {
#pragma unroll
                    for (int st = 0; st < NS; st++) W[st].Jl += W[st].a >> i << 2;
                } else {
                    const uint64_t xa = expand((((uint64_t)ch << 32) | cl) - 1u);
#pragma unroll
                    for (int st = 0; st < NS; st++)
                        W[st].Jl += ((uint32_t)__popcll(sADJ[i] & (xa | sbits(st))) & 1u) << 2;
                }
#pragma unroll
                for (int st = 0; st < NS; st++) {
                    W[st].a ^= adj;
                    step(W[st], fr, fr[NW + 2 * NWL] >> 8);
                }
            }
            if (OUTER) flush();
        }
        if (fold_each && !OUTER) fold(true);
    }
    if (!fold_each && final_fold && !OUTER) fold(clear_on_exit);
}

// final_fold false (counting variants with warp-shared counters, one slice
// per thread): the counters are left for the caller to fold (see
// fold_block_counters).
// Z: the table values' ring (zw64; zw128 with the table and general
// variants, HIST 0).
template <int NWN, int NWL, bool GENERAL, int HIST, bool XTRA, bool OUTER = false, class Z = zw64>
__device__ __forceinline__ void walk(const KernelParams& p, const Smem& sm, uint64_t first,
                                     uint64_t count, uint64_t span, uint64_t nslices,
                                     uint64_t s_begin, uint64_t stride, bool fold_each,
                                     bool clear_on_exit, bool final_fold, Z& acc) {
    if constexpr (HIST >= 4) {
        if constexpr (HIST >= 5 && std::is_same<Z, zw64>::value) {
            if (p.pair_walk) {   // (the same for the whole launch)
                walk_lut_pair<NWN, NWL, HIST == 6, OUTER, 4>(p, sm, first, count, span, nslices, s_begin, stride,
                                                          fold_each, clear_on_exit, final_fold, acc);
                return;
            }
        }
        walk_lut<NWN, NWL, XTRA, HIST >= 5, HIST == 6, OUTER>(p, sm, first, count, span, nslices, s_begin,
                                                              stride, fold_each, clear_on_exit, final_fold, acc);
        return;
    }
    constexpr int NW = NWN + NWL;
    constexpr uint32_t RW = row_words(NWN, NWL);
    typedef typename zw_word<Z>::type W;
    const Z* __restrict__ sT = reinterpret_cast<const Z*>(sm.sT);
    const Z* __restrict__ sPV = reinterpret_cast<const Z*>(sm.sPV);
    const Z* __restrict__ ftab = reinterpret_cast<const Z*>(p.ftab);
    const uint64_t* __restrict__ sADJ = sm.sADJ;
    const uint32_t* __restrict__ sF = sm.sF;
    uint32_t* __restrict__ sH = sm.sH;
    const uint32_t* __restrict__ sS = sm.sS;
    constexpr uint32_t SW = seek_stride(NW);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t ntab = p.tab_size;
    const uint32_t nwords = HIST == 2 ? (ntab + 1) / 2 : ntab;
    uint32_t* const wshared = sH + warp * ntab;   // HIST 3: this warp's counters
    // inner parameters (table, general and lane-private counting variants)
    const bool outer = (HIST == 0 || HIST == 1 || HIST == 2) && p.zq_lo < 64u;

    // flip rows and adjacency of the three lowest variables, in registers:
    // inside an aligned block of 8 Gray steps they are the only ones flipped
    // (the step rows of variables 0, 1, 2 are read from the parameters: the
    // constant bank in the single-scalar kernel)
    const uint64_t adj0 = sADJ[0], adj1 = sADJ[1], adj2 = sADJ[2];

    // HIST: acc += sum_idx count(idx) * T[idx] (mod 2^64).  Lane l adds up
    // counter word i = l (+32, ...) over the warp's 32 lanes, reading them in
    // lane-rotated order so that the 32 reads of a step hit 32 banks; the
    // owning lane then does that word's multiply-add.  clear: reset the
    // counters for further counting.
    auto fold = [&](bool clear) {
        __syncwarp();
        if (HIST == 3) {
            // one counter per index for the whole warp: at most 32 lanes x one
            // slice (<= 2^18 terms) between folds, so it fits in 32 bits
            for (uint32_t i = lane; i < ntab; i += 32) {
                const uint32_t c = wshared[i];
                if (c) {
                    acc = zw_madd32(acc, lds_zw(sT + i), c);
                    if (clear) wshared[i] = 0;
                }
            }
            __syncwarp();
            return;
        }
        uint32_t* wbase = sH + warp * nwords * 32u;
        for (uint32_t i0 = 0; i0 < nwords; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t lo = 0, hi = 0;
            if (i < nwords) {
                const uint32_t* row = wbase + i * 32u;
#pragma unroll 8
                for (uint32_t j = 0; j < 32; j++) {
                    const uint32_t c = row[(j + lane) & 31u];
                    if (HIST == 2) { lo += c & 0xFFFFu; hi += c >> 16; } else lo += c;
                }
                // HIST == 1: a lane counts at most one slice (<= 2^18 terms)
                // between folds, so the 32-lane sum fits in 32 bits
                if (HIST == 2) {
                    if (lo) acc = zw_madd32(acc, lds_zw(sT + 2 * i), lo);
                    if (hi) acc = zw_madd32(acc, lds_zw(sT + 2 * i + 1), hi);
                } else if (lo) {
                    acc = zw_madd32(acc, lds_zw(sT + i), lo);
                }
            }
        }
        if (clear) {
            __syncwarp();
            for (uint32_t i = 0; i < nwords; i++) wbase[i * 32u + lane] = 0;
            __syncwarp();
        }
    };

    const uint64_t end = first + count;
    for (uint64_t s0 = s_begin; s0 < nslices; s0 += stride) {
        const uint64_t s = s0 + lane;
        if (s < nslices) {
            uint64_t t = first + s * span;
            const uint64_t tend = (end - t < span) ? end : t + span;
            const uint64_t x = t ^ (t >> 1);
            // state at x: the form bits are the XOR of the flip rows of x's set
            // bits (plus the inversions); a = A x; q = x^T (upper A) x, as half
            // of sum_{j in x} |A_j & x|
            // (4-bit groups: the quadratic cross terms of group b with the
            // lower groups are the bits of v_b against the running A x)
            uint32_t L[NW];
#pragma unroll
            for (int w = 0; w < NW; w++) L[w] = p.INV[w];
            uint64_t a = 0;
            uint32_t q = 0;
            // phase exponent mod 8: linear forms, class-B node bits and 4 x the
            // quadratic part (updated by 4 x bit i of A x when x_i flips)
            uint32_t Jl;
            const uint32_t nnib = (p.k + 3) >> 2;
            for (uint32_t b = 0; b < nnib; b++) {
                const uint32_t v = (uint32_t)(x >> (4 * b)) & 15u;
                const uint32_t* e = sS + (b * 16u + v) * SW;
                uint32_t ev[SW];
#pragma unroll
                for (uint32_t w4 = 0; w4 < SW; w4 += 4) {
                    const uint4 t4 = *reinterpret_cast<const uint4*>(e + w4);
                    ev[w4] = t4.x; ev[w4 + 1] = t4.y; ev[w4 + 2] = t4.z; ev[w4 + 3] = t4.w;
                }
                q ^= ev[NW + 2] ^ ((uint32_t)__popc(v & (uint32_t)(a >> (4 * b))) & 1u);
                a ^= ((uint64_t)ev[NW + 1] << 32) | ev[NW];
#pragma unroll
                for (int w = 0; w < NW; w++) L[w] ^= ev[w];
            }
            {
                uint32_t P0 = 0, P1 = 0, X2 = 0;
#pragma unroll
                for (int w = 0; w < NWN; w++) X2 ^= L[w] & p.CB[w];
#pragma unroll
                for (int w = 0; w < NWL; w++) {
                    const uint32_t v = L[NWN + w];
                    P0 += __popc(v & p.C0[w]);
                    P1 += __popc(v & p.C1[w]);
                    X2 ^= v & p.C2[w];
                }
                Jl = P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q);
            }
            // the run's sum (table and general variants), and with inner
            // parameters the cut parities zq of the current assignment
            Z ai = zw_zero<W>();
            uint32_t zq = 0;
            if (outer)
                for (uint64_t m = x >> p.zq_lo; m; m &= m - 1)
                    zq ^= __ldg(p.zqcol + p.zq_lo + (uint32_t)__ffsll((long long)m) - 1u);
            // inner parameters: the terms since the last flush times the
            // inner table at zq (a lane-private count fold for HIST 1, 2)
            auto flush = [&]() {
                Z sum = ai;
                if (HIST == 1 || HIST == 2) {
                    uint32_t* const wb = sH + warp * nwords * 32u + lane;
                    for (uint32_t i = 0; i < nwords; i++) {
                        const uint32_t c = wb[i * 32u];
                        if (!c) continue;
                        wb[i * 32u] = 0u;
                        if (HIST == 2) {
                            if (c & 0xFFFFu) sum = zw_madd32(sum, lds_zw(sT + 2 * i), c & 0xFFFFu);
                            if (c >> 16) sum = zw_madd32(sum, lds_zw(sT + 2 * i + 1), c >> 16);
                        } else {
                            sum = zw_madd32(sum, lds_zw(sT + i), c);
                        }
                    }
                }
                acc = zw_add(acc, zw_mul(sum, ldg_zw(ftab + zq)));
                ai = zw_zero<W>();
            };

            // one term at the current state
            auto term = [&]() {
                uint32_t M = 0, Zb = 0;
#pragma unroll
                for (int w = 0; w < NWN; w++) M += __popc(L[w]);
                if (GENERAL && p.has_zero) {
#pragma unroll
                    for (int w = 0; w < NWL; w++) Zb |= L[NWN + w] & p.Z[w];
                }
                if (!GENERAL) {
                    // term value = table[(J, M, pair bits, zero bit)]
                    const uint32_t J = Jl & 7u;
                    uint32_t idx = J * p.tab_stride + M;
                    if (XTRA) {   // phase-pair or zero forms present
                        uint32_t z = 0;
                        if (p.has_zero) {
#pragma unroll
                            for (int w = 0; w < NWL; w++) z |= L[NWN + w] & p.Z[w];
                        }
                        idx = (idx << p.xshift) | (L[NWN] & p.pmask) | ((z != 0 ? 1u : 0u) << p.zshift);
                    }
                    if (HIST == 3)
                        atomicAdd(wshared + idx, 1u);
                    else if (HIST == 2)
                        atomicAdd(sH + ((warp * nwords + (idx >> 1)) << 5) + lane, 1u << ((idx & 1u) << 4));
                    else if (HIST == 1)
                        atomicAdd(sH + ((warp * nwords + idx) << 5) + lane, 1u);
                    else
                        ai = zw_add(ai, lds_zw(sT + idx));
                } else if (Zb == 0) {
                    const uint32_t J = Jl & 7u;
                    Z v = lds_zw(sT + J * p.tab_stride + M);
                    if (GENERAL) {
                        for (uint32_t j = 0; j < p.npairs; j++) {
                            const uint32_t b = bit_at<NW>(L, p.PA[j]) | (bit_at<NW>(L, p.PB[j]) << 1);
                            v = zw_mul(v, lds_zw(sPV + 4 * j + b));
                        }
                    }
                    ai = zw_add(ai, v);
                }
            };
            // flip of variable i with step row f (before the XOR: the phase
            // change depends on the forms' current bits)
            auto step = [&](const uint32_t* f) {
                // (4 d1 mod 8 needs only the parity of d1: one popcount)
                uint32_t d0 = 0, x1 = 0;
#pragma unroll
                for (int w = 0; w < NWL; w++) {
                    d0 += __popc(L[NWN + w] & f[NW + w]);
                    x1 ^= L[NWN + w] & f[NW + NWL + w];
                }
                Jl += f[NW + 2 * NWL] - 2u * d0 - 4u * (uint32_t)__popc(x1);
#pragma unroll
                for (int w = 0; w < NW; w++) L[w] ^= f[w];
            };
            // flip of a variable known at compile time (0, 1 or 2)
            auto flip = [&](const uint32_t* f, uint64_t adj, int i) {
                Jl += ((uint32_t)a >> i & 1u) << 2;
                a ^= adj;
                step(f);
            };

            for (;;) {
                if ((t & 7u) == 0 && tend - t >= 8) {
                    // Gray steps inside t .. t+7 flip variables 0,1,0,2,0,1,0
                    term(); flip(p.R[0], adj0, 0);
                    term(); flip(p.R[1], adj1, 1);
                    term(); flip(p.R[0], adj0, 0);
                    term(); flip(p.R[2], adj2, 2);
                    term(); flip(p.R[0], adj0, 0);
                    term(); flip(p.R[1], adj1, 1);
                    term(); flip(p.R[0], adj0, 0);
                    term();
                    t += 7;
                } else {
                    term();
                }
                if (++t >= tend) break;
                // x(t) = x(t-1) ^ (1 << ctz(t))
                const uint32_t tl = (uint32_t)t;
                const int i = tl ? __ffs(tl) - 1 : 31 + __ffs((uint32_t)(t >> 32));
                if (outer && (uint32_t)i >= p.zq_lo) {
                    // a flip that changes the cut parities ends the run
                    const uint32_t dz = __ldg(p.zqcol + i);
                    if (dz) { flush(); zq ^= dz; }
                }
                Jl += ((uint32_t)(a >> i) & 1u) << 2;
                a ^= sADJ[i];
                uint32_t fr[RW];
#pragma unroll
                for (uint32_t w4 = 0; w4 < RW; w4 += 4) {
                    const uint4 t4 = *reinterpret_cast<const uint4*>(sF + i * RW + w4);
                    fr[w4] = t4.x; fr[w4 + 1] = t4.y; fr[w4 + 2] = t4.z; fr[w4 + 3] = t4.w;
                }
                step(fr);
            }
            if (outer) flush();
            else if (HIST == 0) acc = zw_add(acc, ai);
        }
        // a thread with several slices folds after each one, so no counter
        // can overflow (16-bit counters: every slice is shorter than 2^16);
        // with inner parameters every lane has folded its own counters
        if (HIST && fold_each && !outer) fold(true);
    }
    if (HIST && !outer && !fold_each && (final_fold || HIST < 3)) fold(clear_on_exit);
}

// Warp-shared counters (HIST 3, 4) left unfolded by walk: merge the warps'
// counters bin by bin into warp 0's, then warp 0 folds them and reduces; the
// block's sum is valid in thread 0.  Every thread calls it after the walk.
template <int HIST>
__device__ __forceinline__ zw64 fold_block_counters(const KernelParams& p, const Smem& sm) {
    static_assert(HIST == 3 || HIST == 4, "warp-shared counters only");
    const uint32_t nb = HIST == 4 ? ((uint32_t)kLutRows * p.tab_stride) << p.xshift : p.tab_size;
    const uint32_t nwarps = blockDim.x >> 5;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        uint32_t c = 0;
        for (uint32_t w = 0; w < nwarps; w++) c += sm.sH[w * nb + i];
        sm.sH[i] = c;
    }
    __syncthreads();
    zw64 acc = zw_zero();
    if (threadIdx.x < 32) {
        // block lookup: bin i = x * plane + row * ts + m holds table entry
        // (((row mod 8) * ts + m) << xshift) | x, (row mod 8) * ts + m = i mod 8 ts
        const uint32_t t8 = HIST == 4 ? 8u * p.tab_stride : nb;
        const uint32_t plane = HIST == 4 ? (uint32_t)kLutRows * p.tab_stride : nb;
        const uint32_t xs = HIST == 4 ? p.xshift : 0u;
        uint32_t ti = threadIdx.x, x = 0, r = threadIdx.x;
        while (ti >= t8) ti -= t8;
        while (r >= plane) { r -= plane; x++; }
        for (uint32_t i = threadIdx.x; i < nb; i += 32) {
            const uint32_t c = sm.sH[i];
            if (c) acc = zw_madd32(acc, lds_zw(sm.sT + ((ti << xs) | x)), c);
            ti += 32;
            while (ti >= t8) ti -= t8;
            r += 32;
            while (r >= plane) { r -= plane; x++; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc = zw_add(acc, shfl_xor_zw(acc, off));
    }
    return acc;
}

}  // namespace core
}  // namespace zxp
