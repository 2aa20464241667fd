// objects.h -- the library's opaque objects (zxp_scalar, zxp_ctx) and the
// small helpers that the C ABI's translation units share.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "zxp.h"
#include "kernel.h"
#include "param.h"
#include "plan.h"
#include "ps.h"
#include "zring.h"

static_assert(sizeof(zxp::DevResult) == sizeof(zxp_zomega), "result record layout");

namespace zxp {

// Device addresses of one scalar's tables.  With inner parameters also the
// inner plan's term table, phase-pair values, flip rows and adjacency, the
// outer variables' cut columns and the inner table (plan.h).
struct DevTables {
    zw64* table = nullptr;
    zw64* pv = nullptr;
    uint32_t* rows = nullptr;
    uint64_t* adj = nullptr;
    uint32_t* seek = nullptr;
    zw64* itab = nullptr;
    zw64* ipv = nullptr;
    uint32_t* ifr = nullptr;
    uint64_t* iadj = nullptr;
    uint32_t* ilow = nullptr;
    uint32_t* zq = nullptr;
    zw64* ftab = nullptr;
};

// Byte offsets of the tables in one contiguous block:
// term table | phase-pair values | step rows | adjacency | seek tables,
// then with inner parameters: inner term table | inner pair values | inner
// flip rows | inner adjacency | inner low-bit states | cut columns | inner
// table.  The first
// `copied` bytes come from the host; the inner table is written on the
// device.
struct TableLayout {
    size_t o_pv = 0, o_f = 0, o_adj = 0, o_seek = 0;
    size_t o_itab = 0, o_ipv = 0, o_ifr = 0, o_iadj = 0, o_ilow = 0, o_zq = 0, o_ftab = 0;
    size_t copied = 0, total = 0;
};

inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

inline TableLayout table_layout(const Plan& pl) {
    TableLayout L;
    const size_t tb = pl.table.size() * sizeof(zw64), pb = pl.pv.size() * sizeof(zw64);
    const size_t fb = pl.rows.size() * sizeof(uint32_t), ab = pl.adj.size() * sizeof(uint64_t);
    // seek tables, then the block lookup (if any) right after them
    const size_t sb = pl.seek.size() * sizeof(uint32_t) + pl.lut.size() * sizeof(uint64_t);
    L.o_pv = tb;
    L.o_f = align16(L.o_pv + pb);
    L.o_adj = align16(L.o_f + fb);   // every region 16-byte aligned (bulk copies)
    L.o_seek = align16(L.o_adj + ab);
    L.total = L.o_seek + sb + 16;
    L.copied = L.total;
    if (pl.k_inner && pl.inner) {
        const Plan& in = *pl.inner;
        L.o_itab = align16(L.total);
        L.o_ipv = align16(L.o_itab + in.table.size() * sizeof(zw64));
        L.o_ifr = align16(L.o_ipv + in.pv.size() * sizeof(zw64));
        L.o_iadj = align16(L.o_ifr + in.frows.size() * sizeof(uint32_t));
        L.o_ilow = align16(L.o_iadj + in.adj.size() * sizeof(uint64_t));
        L.o_zq = align16(L.o_ilow + pl.inner_low.size() * sizeof(uint32_t));
        L.o_ftab = (L.o_zq + pl.zqcol.size() * sizeof(uint32_t) + 255) & ~(size_t)255;
        L.copied = L.o_ftab;
        L.total = L.o_ftab + (sizeof(zw64) << pl.inner_bits);
    }
    return L;
}

// Fill dst (L.copied bytes, zeroed by the caller) with the tables.
inline void pack_tables(const Plan& pl, const TableLayout& L, unsigned char* dst) {
    if (!pl.table.empty()) memcpy(dst, pl.table.data(), pl.table.size() * sizeof(zw64));
    if (!pl.pv.empty()) memcpy(dst + L.o_pv, pl.pv.data(), pl.pv.size() * sizeof(zw64));
    if (!pl.rows.empty()) memcpy(dst + L.o_f, pl.rows.data(), pl.rows.size() * sizeof(uint32_t));
    if (!pl.adj.empty()) memcpy(dst + L.o_adj, pl.adj.data(), pl.adj.size() * sizeof(uint64_t));
    if (!pl.seek.empty()) memcpy(dst + L.o_seek, pl.seek.data(), pl.seek.size() * sizeof(uint32_t));
    if (!pl.lut.empty())
        memcpy(dst + L.o_seek + pl.seek.size() * sizeof(uint32_t), pl.lut.data(), pl.lut.size() * sizeof(uint64_t));
    if (pl.k_inner && pl.inner) {
        const Plan& in = *pl.inner;
        if (!in.table.empty()) memcpy(dst + L.o_itab, in.table.data(), in.table.size() * sizeof(zw64));
        if (!in.pv.empty()) memcpy(dst + L.o_ipv, in.pv.data(), in.pv.size() * sizeof(zw64));
        if (!in.frows.empty()) memcpy(dst + L.o_ifr, in.frows.data(), in.frows.size() * sizeof(uint32_t));
        if (!in.adj.empty()) memcpy(dst + L.o_iadj, in.adj.data(), in.adj.size() * sizeof(uint64_t));
        memcpy(dst + L.o_ilow, pl.inner_low.data(), pl.inner_low.size() * sizeof(uint32_t));
        memcpy(dst + L.o_zq, pl.zqcol.data(), pl.zqcol.size() * sizeof(uint32_t));
    }
}

inline DevTables device_tables(const TableLayout& L, unsigned char* base) {
    DevTables d;
    d.table = reinterpret_cast<zw64*>(base);
    d.pv = reinterpret_cast<zw64*>(base + L.o_pv);
    d.rows = reinterpret_cast<uint32_t*>(base + L.o_f);
    d.adj = reinterpret_cast<uint64_t*>(base + L.o_adj);
    d.seek = reinterpret_cast<uint32_t*>(base + L.o_seek);
    if (L.o_ftab) {
        d.itab = reinterpret_cast<zw64*>(base + L.o_itab);
        d.ipv = reinterpret_cast<zw64*>(base + L.o_ipv);
        d.ifr = reinterpret_cast<uint32_t*>(base + L.o_ifr);
        d.iadj = reinterpret_cast<uint64_t*>(base + L.o_iadj);
        d.ilow = reinterpret_cast<uint32_t*>(base + L.o_ilow);
        d.zq = reinterpret_cast<uint32_t*>(base + L.o_zq);
        d.ftab = reinterpret_cast<zw64*>(base + L.o_ftab);
    }
    return d;
}

// Queue the computation of a scalar's inner table (device tables d).
inline cudaError_t queue_inner_table(const Plan& pl, const DevTables& d, cudaStream_t stream) {
    if (!pl.k_inner || !pl.inner) return cudaSuccess;
    return inner_table_launch(*pl.inner, pl.k_inner, d.itab, d.ipv, d.ifr, d.iadj, d.ilow, d.ftab, stream);
}

// The 128-bit values of one scalar on one device (plan.h table_w, pv_w and
// the inner plan's), allocated when the 128-bit sum first needs them:
// term table | pair values | inner term table | inner pair values | inner
// table (written on the device).  Rows, adjacency, seek tables, cut columns
// and low-bit states are the 64-bit upload's.
struct DevWide {
    void* base = nullptr;
    zw128* table = nullptr;
    zw128* pv = nullptr;
    zw128* itab = nullptr;
    zw128* ipv = nullptr;
    zw128* ftab = nullptr;
};

struct WideLayout {
    size_t o_pv = 0, o_itab = 0, o_ipv = 0, o_ftab = 0, copied = 0, total = 0;
};

inline WideLayout wide_layout(const Plan& pl) {
    WideLayout L;
    L.o_pv = align16(pl.table_w.size() * sizeof(zw128));
    L.o_itab = align16(L.o_pv + pl.pv_w.size() * sizeof(zw128));
    L.total = L.copied = L.o_itab;
    if (pl.k_inner && pl.inner) {
        const Plan& in = *pl.inner;
        L.o_ipv = align16(L.o_itab + in.table_w.size() * sizeof(zw128));
        L.o_ftab = (L.o_ipv + in.pv_w.size() * sizeof(zw128) + 255) & ~(size_t)255;
        L.copied = L.o_ftab;
        L.total = L.o_ftab + (sizeof(zw128) << pl.inner_bits);
    }
    if (L.total == 0) L.total = 16;
    return L;
}

inline void pack_wide(const Plan& pl, const WideLayout& L, unsigned char* dst) {
    if (!pl.table_w.empty()) memcpy(dst, pl.table_w.data(), pl.table_w.size() * sizeof(zw128));
    if (!pl.pv_w.empty()) memcpy(dst + L.o_pv, pl.pv_w.data(), pl.pv_w.size() * sizeof(zw128));
    if (pl.k_inner && pl.inner) {
        const Plan& in = *pl.inner;
        if (!in.table_w.empty()) memcpy(dst + L.o_itab, in.table_w.data(), in.table_w.size() * sizeof(zw128));
        if (!in.pv_w.empty()) memcpy(dst + L.o_ipv, in.pv_w.data(), in.pv_w.size() * sizeof(zw128));
    }
}

inline DevWide device_wide(const WideLayout& L, unsigned char* base) {
    DevWide d;
    d.base = base;
    d.table = reinterpret_cast<zw128*>(base);
    d.pv = reinterpret_cast<zw128*>(base + L.o_pv);
    if (L.o_ftab) {
        d.itab = reinterpret_cast<zw128*>(base + L.o_itab);
        d.ipv = reinterpret_cast<zw128*>(base + L.o_ipv);
        d.ftab = reinterpret_cast<zw128*>(base + L.o_ftab);
    }
    return d;
}

// Descriptor the batch kernel reads for a scalar whose tables are at d.
inline BatchScalar batch_descriptor(const Plan& pl, const DevTables& d) {
    BatchScalar bs;
    memset(&bs, 0, sizeof bs);
    bs.kp = pl.kp;
    bs.table = d.table;
    bs.pv = d.pv;
    bs.rows = d.rows;
    bs.adj = d.adj;
    bs.seek = d.seek;
    bs.K = pl.K;
    bs.e0 = pl.e0;
    bs.key = batch_key(pl);
    return bs;
}

// A pending zxp_submit: device and pinned result slots and its event.
// A ticket's result lives in pinned host memory that the kernel writes
// directly (dres is its device address).
struct Ticket {
    DevResult* dres = nullptr;
    DevResult* hres = nullptr;
    int32_t e0 = 0;
    bool trivial = false;        // no launch: the value is zero
    uint64_t seq = 0;            // the launch's number on the context's stream
    zxp_scalar* owned = nullptr; // zxp_submit_tables: freed when the ticket is released
};

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = -1;
};

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? ZXP_OK : ZXP_ECUDA; }

inline zw64 to_zw(const zxp_zomega& z) {
    return zw_make((uint64_t)z.c[0], (uint64_t)z.c[1], (uint64_t)z.c[2], (uint64_t)z.c[3]);
}
inline void from_zw(const zw64& v, int32_t e, int32_t flags, zxp_zomega* out) {
    for (int i = 0; i < 4; i++) out->c[i] = (int64_t)v.c[i];
    out->e = e;
    out->flags = flags;
}

// Canonical form of an exact numerator (int64 coefficients) over sqrt2^e:
// divide by sqrt2 (x / sqrt2 = x (w - w^3) / 2) while e > 0 and the
// coefficients allow it; zero becomes e = 0.
inline void canon_i128(__int128 c[4], int32_t* e) {
    if (!c[0] && !c[1] && !c[2] && !c[3]) { *e = 0; return; }
    while (*e > 0 && ((c[0] - c[2]) & 1) == 0 && ((c[1] - c[3]) & 1) == 0) {
        __int128 n0 = c[1] - c[3], n1 = c[0] + c[2], n2 = c[1] + c[3], n3 = c[2] - c[0];
        c[0] = n0 / 2; c[1] = n1 / 2; c[2] = n2 / 2; c[3] = n3 / 2;
        *e -= 1;
    }
}

inline void canon_result(const DevResult& r, zxp_zomega* out) {
    __int128 c[4] = {r.c[0], r.c[1], r.c[2], r.c[3]};
    int32_t e = r.e;
    canon_i128(c, &e);
    for (int i = 0; i < 4; i++) out->c[i] = (int64_t)c[i];
    out->e = e;
    out->flags = 0;
}

}  // namespace zxp

struct zxp_scalar {
    zxp::PS ps;
    zxp::Plan plan;
    int plan_status = ZXP_OK;
    mutable std::mutex mu;
    // Per-device copies of the tables, allocated from the library's table
    // pool in the order of the stream of the context that first needed them
    // (`stream`, context `ctx_id`).  A copy that another stream has used is
    // `shared`: that stream waited for the device once before its first use,
    // and freeing the copy waits for the device too.
    struct DevCopy {
        zxp::DevTables t;
        cudaStream_t stream = nullptr;
        uint64_t ctx_id = 0;
        bool shared = false;
    };
    mutable std::map<int, DevCopy> dev;
    // per-device 128-bit values (zxp_eval_wide), freed with the scalar
    mutable std::map<int, zxp::DevWide> devw;

    ~zxp_scalar();
};

struct zxp_ctx {
    uint64_t id = 0;                    // never reused within the process
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t upload = nullptr;      // table copies (the stream waits for them)
    int sm_count = 0;
    int max_grid = 0;
    zxp::zw64* acc = nullptr;           // the sum kernels' accumulator, 64 bytes (zero between launches)
    zxp::DevResultW* wres = nullptr;    // device result of the 128-bit sum
    unsigned int* counter = nullptr;
    zxp::DevResult* hres = nullptr;     // pinned; the kernel writes it directly
    zxp::DevResult* hres_dev = nullptr; // its device address
    // Device table buffers of released zxp_submit_tables scalars (pointer,
    // bytes; allocated from the table pool), reused by later uploads: their
    // last kernel has ended (its result was seen), so no wait is needed.
    static constexpr size_t kTableCache = 8;
    std::vector<std::pair<void*, size_t>> table_cache;
    // Pinned staging for table uploads: a ring of buffers, each reused once
    // the copy out of it (event) has completed.
    static constexpr int kStages = 4;
    unsigned char* stage[kStages] = {};
    size_t stage_cap[kStages] = {};
    cudaEvent_t stage_ev[kStages] = {};
    // Launches on `stream` are numbered (enq_seq); done_seq is the highest
    // whose published result the host has seen, so every launch up to it
    // has ended (one stream: they end in order).  A staging slot whose copy
    // fed launch stage_seq <= done_seq is free without asking its event
    // (the launch waited for the copy); 0: not known.
    uint64_t enq_seq = 0, done_seq = 0;
    uint64_t stage_seq[kStages] = {};
    int stage_next = 0;
    uint64_t next_ticket = 1;
    std::map<uint64_t, zxp::Ticket> tickets;
    std::vector<zxp::Ticket> free_slots;
};

struct zxp_pscalar {
    zxp::PPS pps;
};

namespace zxp {
// Compile a circuit or decode tables into a new scalar (api.cu).
int make_scalar(PS&& ps, zxp_scalar** out);
}  // namespace zxp
