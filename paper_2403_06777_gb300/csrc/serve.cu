// serve.cu -- the request server of the C ABI (include/zxp.h, "request
// server"): host compile workers, one scheduler thread that owns the
// context's stream, a device arena of resident tables, and per-step
// continuous batching through the batch kernel.
//
// Threads and data:
//   * submit (any thread) copies the request under the server mutex and
//     queues it for the compile workers (or, for a compiled scalar, straight
//     for admission);
//   * compile workers turn circuits into scalars (the host reduction of
//     Sec. 3 / App. B) and queue them for admission;
//   * the scheduler admits queued scalars while the arena has room and a
//     result slot is free (FIFO: a request that does not fit waits, and the
//     ones behind it wait too), plans a step over every resident request
//     (serve_sched.h), and launches it: one host-to-device copy of the
//     step's chunk list and queue counters, one batch-kernel launch per
//     kernel variant, a gather of the finished requests' results and one
//     device-to-host copy.  Two steps are in flight; a step's finished
//     requests are completed when its event has fired.  Resident requests
//     keep their tables and their partial sums (a result slot that every
//     step adds into) on the device until they finish.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "zxp.h"
#include "compile.h"
#include "kernel.h"
#include "objects.h"
#include "serve_sched.h"

using namespace zxp;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kPipeline = 2;              // steps in flight
constexpr uint32_t kMaxGroups = 128;      // kernel variants in one step (queue counters)
constexpr size_t kStageTables = 8u << 20; // pinned bytes per step for newly admitted tables

struct Request {
    uint64_t ticket = 0;
    // a circuit request (copied at submit)
    bool circuit = false;
    std::vector<zxp_gate> gates;
    std::vector<uint8_t> in_bits, out_bits;
    int32_t n_qubits = 0, kind = 0;
    uint64_t mask = 0;
    // a binding request: a parametric scalar (borrowed) and parameter values
    const PPS* pps = nullptr;
    uint64_t bits = 0;
    // the scalar: compiled or bound here (owned) or the caller's (borrowed)
    std::unique_ptr<zxp_scalar> owned;
    const zxp_scalar* scalar = nullptr;
    // completion (under the server mutex)
    bool done = false;
    int status = ZXP_EAGAIN;
    zxp_zomega value{};
    zxp_request_timing timing{};
    // residency (scheduler thread only)
    uint64_t arena_off = 0, arena_bytes = 0;
    uint32_t slot = 0;
    int key = 0;
};
using ReqPtr = std::shared_ptr<Request>;

struct StepSlot {
    unsigned char* h_stage = nullptr;   // pinned: counters | chunks | finishing slots, then tables
    unsigned char* d_step = nullptr;    // device: counters | chunks | finishing slots | results out
    DevResult* h_out = nullptr;         // pinned copy of the finished results
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool busy = false;
    std::vector<ReqPtr> finishing;
    uint64_t terms = 0;
};

}  // namespace

struct zxp_server {
    zxp_ctx* ctx = nullptr;
    // options, defaults resolved
    // (chunks of 2^20 terms on 128-thread blocks: 2^13 terms per thread per
    // chunk, enough to amortise a chunk's seek, fold and reduction; 1024
    // chunks per 2^30-term step, more than the resident blocks, and few
    // enough steps that their fixed costs stay small: measured on the serving
    // mix, device time within 10 % of one launch per scalar)
    uint32_t policy = ZXP_SERVE_BATCHED, max_k = 44, max_active = 4096, chunk_log2 = 20;
    uint32_t threads = 128;
    uint64_t arena_bytes = 64ull << 20, step_terms = 1ull << 30, small_terms = 1ull << 22;
    size_t chunk_cap = 0;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_compile, cv_sched, cv_done;
    std::deque<ReqPtr> compile_q, ready_q;
    std::unordered_map<uint64_t, ReqPtr> tickets;
    uint64_t next_ticket = 1;
    uint32_t compiling = 0;
    bool stopping = false;
    zxp_server_stats_t stats{};
    int fatal = ZXP_OK;                 // a CUDA error stops the scheduler

    std::vector<std::thread> workers;
    std::thread sched;

    // device state (scheduler thread)
    unsigned char* d_arena = nullptr;
    DevResult* d_results = nullptr;
    StepSlot steps[kPipeline];
    Arena arena;
    std::vector<uint32_t> free_slots;
    std::map<uint64_t, int> occupancy;  // (key, caps, threads) -> blocks per SM

    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte layout of one step buffer (host stage and device copy alike).
struct StepLayout {
    size_t o_chunks, o_slots, o_out, o_tables, total_dev, total_host;
};
StepLayout step_layout(const zxp_server* s) {
    StepLayout L;
    L.o_chunks = align_up(kMaxGroups * sizeof(unsigned int), 256);
    L.o_slots = align_up(L.o_chunks + s->chunk_cap * sizeof(BatchChunk), 256);
    L.o_out = align_up(L.o_slots + (size_t)s->max_active * sizeof(uint32_t), 256);
    L.total_dev = L.o_out + (size_t)s->max_active * sizeof(DevResult);
    L.o_tables = L.o_out;              // host stage: admitted tables follow the slot list
    L.total_host = L.o_tables + kStageTables;
    return L;
}

// Mark a request finished and wake pollers (takes the server mutex).
void complete(zxp_server* s, const ReqPtr& r, int status, const zxp_zomega* v) {
    std::lock_guard<std::mutex> lk(s->mu);
    r->status = status;
    if (v) r->value = *v;
    r->timing.status = status;
    r->timing.done_us = s->now_us();
    r->done = true;
    s->stats.completed++;
    if (status == ZXP_ETOOBIG) s->stats.rejected++;
    s->cv_done.notify_all();
}

void compile_worker(zxp_server* s) {
    for (;;) {
        ReqPtr r;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_compile.wait(lk, [&] { return s->stopping || !s->compile_q.empty(); });
            if (s->compile_q.empty()) return;   // stopping and drained
            r = s->compile_q.front();
            s->compile_q.pop_front();
            s->compiling++;
        }
        PS ps;
        int st = ZXP_OK;
        if (r->pps) {
            bind(*r->pps, r->bits, &ps);
        } else {
            CompileOptions opt;
            st = compile_circuit(r->gates.data(), r->gates.size(), r->n_qubits,
                                 r->in_bits.empty() ? nullptr : r->in_bits.data(), r->out_bits.data(),
                                 r->mask, r->kind, opt, &ps);
        }
        zxp_scalar* sc = nullptr;
        if (st == ZXP_OK) st = make_scalar(std::move(ps), &sc);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->compiling--;
            r->timing.compiled_us = s->now_us();
            if (st == ZXP_OK) {
                r->owned.reset(sc);
                r->scalar = sc;
                r->timing.k = sc->ps.k;
                s->ready_q.push_back(r);
            }
            s->cv_sched.notify_one();
        }
        if (st != ZXP_OK) complete(s, r, st, nullptr);
    }
}

int blocks_per_sm(zxp_server* s, int key, uint32_t ntab, uint32_t npairs) {
    const uint64_t id = ((uint64_t)(uint32_t)key << 40) | ((uint64_t)ntab << 20) | npairs;
    auto it = s->occupancy.find(id);
    if (it != s->occupancy.end()) return it->second;
    int bps = 0;
    if (batch_occupancy(key, ntab, npairs, (int)s->threads, &bps) != cudaSuccess || bps < 1) bps = 0;
    s->occupancy[id] = bps;
    return bps;
}

// Everything the scheduler owns.
struct Scheduler {
    zxp_server* s;
    StepLayout L;
    std::deque<ReqPtr> pending;         // compiled, not admitted (FIFO)
    std::vector<ReqPtr> active;         // resident, range not fully planned
    std::vector<WorkItem> items;        // parallel to active
    uint64_t order = 0;
    int next_step = 0;
    std::vector<PlannedChunk> planned;

    explicit Scheduler(zxp_server* srv) : s(srv), L(step_layout(srv)) {}

    bool any_busy() const {
        for (auto& st : s->steps)
            if (st.busy) return true;
        return false;
    }

    // Complete the requests of a finished step.  wait: block until it ends.
    int retire(StepSlot& st, bool wait) {
        if (!st.busy) return ZXP_OK;
        if (wait) {
            if (cudaEventSynchronize(st.ev1) != cudaSuccess) return ZXP_ECUDA;
        } else {
            const cudaError_t e = cudaEventQuery(st.ev1);
            if (e == cudaErrorNotReady) return ZXP_EAGAIN;
            if (e != cudaSuccess) return ZXP_ECUDA;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, st.ev0, st.ev1);
        for (size_t i = 0; i < st.finishing.size(); i++) {
            const ReqPtr& r = st.finishing[i];
            zxp_zomega v;
            canon_result(st.h_out[i], &v);
            s->arena.release(r->arena_off);
            s->free_slots.push_back(r->slot);
            const int32_t e0 = r->scalar->ps.e0;
            if (st.h_out[i].flags & 2) {
                complete(s, r, ZXP_ETIMEDOUT, nullptr);
            } else if (e0 > 124 && e0 <= 252) {
                // beyond the 64-bit bound: the sum again modulo 2^128, on this
                // thread's stream (synchronous: it waits for the steps in flight)
                zxp_zomega w;
                const int st2 = zxp_amplitude(s->ctx, r->scalar, &w);
                complete(s, r, st2, (st2 == ZXP_OK || st2 == ZXP_EOVERFLOW) ? &w : nullptr);
            } else {
                complete(s, r, e0 > 252 ? ZXP_EOVERFLOW : ZXP_OK, &v);
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.device_busy_us += ms * 1e3;
            s->stats.terms += (double)st.terms;
            s->stats.active = (uint32_t)(active.size());
        }
        st.finishing.clear();
        st.busy = false;
        return ZXP_OK;
    }

    int retire_ready() {
        for (auto& st : s->steps) {
            const int e = retire(st, false);
            if (e != ZXP_OK && e != ZXP_EAGAIN) return e;
        }
        return ZXP_OK;
    }

    // Admit pending requests into the step that uses stage `st`; returns the
    // number of table bytes staged.  Copies are queued on the stream.
    int admit(StepSlot& st, size_t* staged_bytes) {
        size_t used = 0;
        const uint32_t cap_active = s->policy == ZXP_SERVE_PLAIN ? 1u : s->max_active;
        while (!pending.empty() && active.size() < cap_active && !s->free_slots.empty()) {
            ReqPtr r = pending.front();
            const zxp_scalar* sc = r->scalar;
            const Plan& pl = sc->plan;
            if (sc->ps.k > s->max_k) {
                pending.pop_front();
                complete(s, r, ZXP_ETOOBIG, nullptr);
                continue;
            }
            if (pl.zero) {   // identically zero: nothing to sum
                pending.pop_front();
                zxp_zomega z{};
                r->timing.admitted_us = s->now_us();
                complete(s, r, ZXP_OK, &z);
                continue;
            }
            const TableLayout TL = table_layout(pl);
            const uint64_t bytes = kBatchScalarBytes + TL.total;
            if (!s->arena.fits_at_all(bytes) || bytes > kStageTables) {
                pending.pop_front();
                complete(s, r, ZXP_ETOOBIG, nullptr);
                continue;
            }
            if (used + align_up(bytes, 256) > kStageTables) break;   // next step
            uint64_t off = 0;
            if (!s->arena.alloc(bytes, &off)) break;                   // wait for memory
            pending.pop_front();
            unsigned char* h = st.h_stage + L.o_tables + used;
            memset(h, 0, bytes);
            unsigned char* dbase = s->d_arena + off;
            const DevTables d = device_tables(TL, dbase + kBatchScalarBytes);
            pack_tables(pl, TL, h + kBatchScalarBytes);
            *reinterpret_cast<BatchScalar*>(h) = batch_descriptor(pl, d);
            if (cudaMemcpyAsync(dbase, h, bytes, cudaMemcpyHostToDevice, s->ctx->stream) != cudaSuccess)
                return ZXP_ECUDA;
            used += align_up(bytes, 256);
            r->arena_off = off;
            r->arena_bytes = bytes;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            r->key = batch_key(pl);
            r->timing.admitted_us = s->now_us();
            active.push_back(r);
            WorkItem w;
            w.total = 1ull << sc->ps.k;
            w.next = 0;
            w.order = order++;
            items.push_back(w);
        }
        *staged_bytes = used;
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.active = (uint32_t)active.size();
        s->stats.peak_active = std::max(s->stats.peak_active, s->stats.active);
        s->stats.arena_bytes = s->arena.used();
        s->stats.arena_peak = s->arena.peak();
        return ZXP_OK;
    }

    // Plan and launch one step on stage `st`.  Returns ZXP_EAGAIN when there
    // was nothing to run.
    int launch(StepSlot& st) {
        cudaStream_t stream = s->ctx->stream;
        if (s->policy == ZXP_SERVE_PLAIN) {
            // one request, its whole range, one launch of the single-scalar kernel
            planned.clear();
            size_t pick = 0;
            bool found = false;
            for (size_t i = 0; i < items.size(); i++)
                if (items[i].next < items[i].total && (!found || items[i].order < items[pick].order)) {
                    pick = i;
                    found = true;
                }
            if (!found) return ZXP_EAGAIN;
            planned.push_back(PlannedChunk{pick, items[pick].next, items[pick].total - items[pick].next});
            items[pick].next = items[pick].total;
        } else {
            plan_step(items, s->step_terms, s->chunk_log2, s->small_terms, &planned);
            if (planned.empty()) return ZXP_EAGAIN;
            if (planned.size() > s->chunk_cap) return ZXP_ECUDA;   // cannot happen: cap covers the budget
        }

        // finished requests leave the resident set; their chunks stay in this step
        std::vector<char> fin(active.size(), 0);
        for (size_t i = 0; i < active.size(); i++) fin[i] = items[i].next == items[i].total;
        std::vector<size_t> step_items;
        for (auto& c : planned)
            if (step_items.empty() || step_items.back() != c.item) step_items.push_back(c.item);

        // chunk list grouped by kernel variant
        unsigned int* h_counters = reinterpret_cast<unsigned int*>(st.h_stage);
        BatchChunk* h_chunks = reinterpret_cast<BatchChunk*>(st.h_stage + L.o_chunks);
        uint32_t* h_slots = reinterpret_cast<uint32_t*>(st.h_stage + L.o_slots);
        struct Group { int key; uint32_t ntab, npairs, off, count; };
        std::vector<Group> groups;
        std::map<int, size_t> gi;
        for (auto& c : planned) {
            const ReqPtr& r = active[c.item];
            if (!gi.count(r->key)) { gi[r->key] = groups.size(); groups.push_back(Group{r->key, 0, 0, 0, 0}); }
            Group& g = groups[gi[r->key]];
            g.count++;
            g.ntab = std::max(g.ntab, r->scalar->plan.kp.tab_size);
            g.npairs = std::max(g.npairs, r->scalar->plan.kp.npairs);
        }
        if (groups.size() > kMaxGroups) return ZXP_ECUDA;
        uint32_t off = 0;
        for (auto& g : groups) { g.off = off; off += g.count; g.count = 0; }
        uint64_t terms = 0;
        for (auto& c : planned) {
            const ReqPtr& r = active[c.item];
            Group& g = groups[gi[r->key]];
            h_chunks[g.off + g.count++] =
                BatchChunk{(uint32_t)(r->arena_off / kBatchScalarBytes), r->slot, c.first, c.count};
            terms += c.count;
        }
        memset(h_counters, 0, kMaxGroups * sizeof(unsigned int));
        st.finishing.clear();
        for (size_t i = 0; i < active.size(); i++)
            if (fin[i]) {
                h_slots[st.finishing.size()] = active[i]->slot;
                st.finishing.push_back(active[i]);
            }
        const uint32_t nfin = (uint32_t)st.finishing.size();
        for (size_t i : step_items) active[i]->timing.steps++;

        // one copy of the step's descriptors, then the launches
        const size_t bytes = L.o_slots + nfin * sizeof(uint32_t);
        if (cudaMemcpyAsync(st.d_step, st.h_stage, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return ZXP_ECUDA;
        if (cudaEventRecord(st.ev0, stream) != cudaSuccess) return ZXP_ECUDA;
        unsigned int* d_counters = reinterpret_cast<unsigned int*>(st.d_step);
        const BatchChunk* d_chunks = reinterpret_cast<const BatchChunk*>(st.d_step + L.o_chunks);
        uint32_t launches = 0;
        if (s->policy == ZXP_SERVE_PLAIN) {
            const ReqPtr& r = active[planned[0].item];
            const Plan& pl = r->scalar->plan;
            const DevTables d = device_tables(table_layout(pl), s->d_arena + r->arena_off + kBatchScalarBytes);
            const uint64_t count = planned[0].count;
            uint64_t sp = 64;
            int grid = 1;
            sum_shape(pl, s->ctx->sm_count, s->ctx->max_grid, count, &sp, &grid);
            if (sum_launch(pl, d.table, d.pv, d.rows, d.adj, d.seek, d.zq, d.ftab, planned[0].first, count, sp,
                           grid,
                           s->ctx->acc, s->ctx->counter, s->d_results + r->slot, false, stream) != cudaSuccess)
                return ZXP_ECUDA;
            launches = 1;
        } else {
            for (size_t g = 0; g < groups.size(); g++) {
                const Group& G = groups[g];
                const int bps = blocks_per_sm(s, G.key, G.ntab, G.npairs);
                if (bps < 1) return ZXP_ECUDA;
                const int grid = (int)std::min<uint64_t>((uint64_t)s->ctx->sm_count * bps, G.count);
                if (batch_launch(G.key, s->d_arena, d_chunks + G.off, G.count, d_counters + g, s->d_results,
                                 G.ntab, G.npairs, (int)s->threads, grid, 1, stream) != cudaSuccess)
                    return ZXP_ECUDA;
                launches++;
            }
        }
        DevResult* d_out = reinterpret_cast<DevResult*>(st.d_step + L.o_out);
        if (gather_results(s->d_results, reinterpret_cast<const uint32_t*>(st.d_step + L.o_slots), nfin,
                           d_out, stream) != cudaSuccess)
            return ZXP_ECUDA;
        if (nfin && cudaMemcpyAsync(st.h_out, d_out, nfin * sizeof(DevResult), cudaMemcpyDeviceToHost,
                                    stream) != cudaSuccess)
            return ZXP_ECUDA;
        if (cudaEventRecord(st.ev1, stream) != cudaSuccess) return ZXP_ECUDA;
        st.busy = true;
        st.terms = terms;

        // drop the finished requests from the resident set
        size_t w = 0;
        for (size_t i = 0; i < active.size(); i++)
            if (!fin[i]) { active[w] = active[i]; items[w] = items[i]; w++; }
        active.resize(w);
        items.resize(w);
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.steps++;
        s->stats.launches += launches + (nfin ? 1 : 0);
        return ZXP_OK;
    }

    void run() {
        DeviceGuard dg(s->ctx->device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(s->mu);
                for (auto& r : s->ready_q) pending.push_back(r);
                s->ready_q.clear();
                const bool idle = pending.empty() && active.empty() && !any_busy();
                if (idle && s->stopping && s->compile_q.empty() && s->compiling == 0) return;
                if (idle) {
                    s->cv_sched.wait(lk, [&] {
                        return !s->ready_q.empty() ||
                               (s->stopping && s->compile_q.empty() && s->compiling == 0);
                    });
                    continue;
                }
            }
            int e = retire_ready();
            if (e != ZXP_OK) { fail(e); return; }
            StepSlot& st = s->steps[next_step];
            if (st.busy) {   // both steps in flight: wait for the older one
                if ((e = retire(st, true)) != ZXP_OK) { fail(e); return; }
            }
            size_t staged = 0;
            if ((e = admit(st, &staged)) != ZXP_OK) { fail(e); return; }
            e = launch(st);
            if (e == ZXP_OK) {
                next_step = (next_step + 1) % kPipeline;
                continue;
            }
            if (e != ZXP_EAGAIN) { fail(e); return; }
            // nothing to launch now: wait for arrivals or for a step to end
            if (any_busy()) {
                std::unique_lock<std::mutex> lk(s->mu);
                s->cv_sched.wait_for(lk, std::chrono::microseconds(50), [&] { return !s->ready_q.empty(); });
            } else if (!pending.empty()) {
                // pending requests that cannot be admitted with nothing in flight
                // (cannot happen: an empty arena admits any request that fits at all)
                fail(ZXP_ENOMEM);
                return;
            }
        }
    }

    // A CUDA error: fail every request the scheduler holds and stop.
    void fail(int e) {
        for (auto& st : s->steps) {
            for (auto& r : st.finishing) complete(s, r, e, nullptr);
            st.finishing.clear();
            st.busy = false;
        }
        for (auto& r : active) complete(s, r, e, nullptr);
        for (auto& r : pending) complete(s, r, e, nullptr);
        active.clear();
        pending.clear();
        std::unique_lock<std::mutex> lk(s->mu);
        s->fatal = e;
        for (auto& r : s->ready_q) {
            r->status = e; r->timing.status = e; r->done = true;
        }
        s->ready_q.clear();
        s->cv_done.notify_all();
    }
};

void scheduler_main(zxp_server* s) {
    Scheduler sc(s);
    sc.run();
    // after a fatal error keep failing late arrivals until the server stops
    std::unique_lock<std::mutex> lk(s->mu);
    while (s->fatal != ZXP_OK) {
        for (auto& r : s->ready_q) { r->status = s->fatal; r->timing.status = s->fatal; r->done = true; }
        s->ready_q.clear();
        s->cv_done.notify_all();
        if (s->stopping && s->compile_q.empty() && s->compiling == 0) break;
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(10));
    }
}

void free_device(zxp_server* s) {
    for (auto& st : s->steps) {
        if (st.ev0) cudaEventDestroy(st.ev0);
        if (st.ev1) cudaEventDestroy(st.ev1);
        cudaFreeHost(st.h_stage);
        cudaFreeHost(st.h_out);
        cudaFree(st.d_step);
    }
    cudaFree(s->d_arena);
    cudaFree(s->d_results);
}

int submit_common(zxp_server* s, ReqPtr r, bool compiled, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return ZXP_EINVAL;
    r->ticket = s->next_ticket++;
    r->timing.submit_us = s->now_us();
    r->timing.status = ZXP_EAGAIN;
    s->tickets[r->ticket] = r;
    s->stats.submitted++;
    if (s->fatal != ZXP_OK) {
        r->status = r->timing.status = s->fatal;
        r->done = true;
    } else if (compiled) {
        r->timing.compiled_us = r->timing.submit_us;
        s->ready_q.push_back(r);
        s->cv_sched.notify_one();
    } else {
        s->compile_q.push_back(r);
        s->cv_compile.notify_one();
    }
    *ticket = r->ticket;
    return ZXP_OK;
}

}  // namespace

extern "C" {

int zxp_server_create(zxp_ctx* ctx, const zxp_server_opts* opts, zxp_server** out) {
    if (!ctx || !out) return ZXP_EINVAL;
    *out = nullptr;
    std::unique_ptr<zxp_server> s(new (std::nothrow) zxp_server());
    if (!s) return ZXP_ENOMEM;
    s->ctx = ctx;
    uint32_t nthreads = 0;
    if (opts) {
        if (opts->policy > ZXP_SERVE_PLAIN) return ZXP_EINVAL;
        if (opts->max_k > 62) return ZXP_EINVAL;
        if (opts->threads && opts->threads != 128 && opts->threads != 256) return ZXP_EINVAL;
        if (opts->chunk_log2 && (opts->chunk_log2 < 3 || opts->chunk_log2 > 30)) return ZXP_EINVAL;
        s->policy = opts->policy;
        if (opts->max_k) s->max_k = opts->max_k;
        if (opts->max_active) s->max_active = opts->max_active;
        if (opts->arena_bytes) s->arena_bytes = opts->arena_bytes;
        if (opts->step_terms) s->step_terms = opts->step_terms;
        if (opts->small_terms) s->small_terms = opts->small_terms;
        if (opts->chunk_log2) s->chunk_log2 = opts->chunk_log2;
        if (opts->threads) s->threads = opts->threads;
        nthreads = opts->compile_threads;
    }
    if (s->max_active > (1u << 20)) return ZXP_EINVAL;
    if (!nthreads) nthreads = std::min(16u, std::max(1u, std::thread::hardware_concurrency()));
    // chunks in one step: the budget (which the first small request may
    // overrun by up to small_terms) in whole chunks, plus one partial chunk
    // per request
    s->chunk_cap = (size_t)((s->step_terms + s->small_terms) >> s->chunk_log2) + 2 * (size_t)s->max_active + 16;
    s->t0 = Clock::now();

    DeviceGuard dg(ctx->device);
    s->arena.reset(s->arena_bytes, kBatchScalarBytes);
    int st = ZXP_OK;
    if (cudaMalloc(&s->d_arena, s->arena.capacity()) != cudaSuccess ||
        cudaMalloc(&s->d_results, (size_t)s->max_active * sizeof(DevResult)) != cudaSuccess)
        st = ZXP_ENOMEM;
    if (st == ZXP_OK && cudaMemset(s->d_results, 0, (size_t)s->max_active * sizeof(DevResult)) != cudaSuccess)
        st = ZXP_ECUDA;
    const StepLayout L = step_layout(s.get());
    for (auto& sl : s->steps) {
        if (st != ZXP_OK) break;
        if (cudaMallocHost(&sl.h_stage, L.total_host) != cudaSuccess ||
            cudaMallocHost(&sl.h_out, (size_t)s->max_active * sizeof(DevResult)) != cudaSuccess ||
            cudaMalloc(&sl.d_step, L.total_dev) != cudaSuccess)
            st = ZXP_ENOMEM;
        else if (cudaEventCreate(&sl.ev0) != cudaSuccess || cudaEventCreate(&sl.ev1) != cudaSuccess)
            st = ZXP_ECUDA;
    }
    if (st != ZXP_OK) {
        free_device(s.get());
        return st;
    }
    for (uint32_t i = s->max_active; i > 0; i--) s->free_slots.push_back(i - 1);
    zxp_server* raw = s.get();
    for (uint32_t i = 0; i < nthreads; i++) raw->workers.emplace_back(compile_worker, raw);
    raw->sched = std::thread(scheduler_main, raw);
    *out = s.release();
    return ZXP_OK;
}

int zxp_server_submit(zxp_server* s, const zxp_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || !req->out_bits || req->n_qubits <= 0 || (req->n_gates && !req->gates))
        return ZXP_EINVAL;
    if (req->kind != ZXP_AMPLITUDE && req->kind != ZXP_MARGINAL_DOUBLED) return ZXP_EINVAL;
    ReqPtr r = std::make_shared<Request>();
    r->circuit = true;
    r->gates.assign(req->gates, req->gates + req->n_gates);
    r->n_qubits = req->n_qubits;
    r->kind = req->kind;
    r->mask = req->marg_mask;
    r->out_bits.assign(req->out_bits, req->out_bits + req->n_qubits);
    if (req->in_bits) r->in_bits.assign(req->in_bits, req->in_bits + req->n_qubits);
    return submit_common(s, r, false, ticket);
}

int zxp_server_submit_bind(zxp_server* s, const zxp_pscalar* ps, uint64_t bits, uint64_t* ticket) {
    if (!s || !ps || !ticket) return ZXP_EINVAL;
    if (ps->pps.p < 64 && (bits >> ps->pps.p)) return ZXP_EINVAL;
    ReqPtr r = std::make_shared<Request>();
    r->pps = &ps->pps;
    r->bits = bits;
    return submit_common(s, r, false, ticket);
}

int zxp_server_submit_scalar(zxp_server* s, const zxp_scalar* sc, uint64_t* ticket) {
    if (!s || !sc || !ticket) return ZXP_EINVAL;
    if (sc->ps.k_inner) return ZXP_EINVAL;   // inner parameters: single-scalar path only
    ReqPtr r = std::make_shared<Request>();
    r->scalar = sc;
    r->timing.k = sc->ps.k;
    return submit_common(s, r, true, ticket);
}

int zxp_server_poll(zxp_server* s, uint64_t ticket, int64_t timeout_us, zxp_zomega* out,
                    zxp_request_timing* timing) {
    if (!s) return ZXP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return ZXP_ENOTFOUND;
    ReqPtr r = it->second;
    if (!r->done) {
        if (timeout_us < 0) {
            s->cv_done.wait(lk, [&] { return r->done; });
        } else if (timeout_us > 0) {
            s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
        }
    }
    if (!r->done) return ZXP_EAGAIN;
    if (out) *out = r->value;
    if (timing) *timing = r->timing;
    s->tickets.erase(it);
    return r->status;
}

int zxp_server_stats(zxp_server* s, zxp_server_stats_t* out) {
    if (!s || !out) return ZXP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return ZXP_OK;
}

void zxp_server_destroy(zxp_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv_compile.notify_all();
        s->cv_sched.notify_all();
    }
    for (auto& t : s->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv_sched.notify_all();
    }
    s->sched.join();
    {
        DeviceGuard dg(s->ctx->device);
        cudaStreamSynchronize(s->ctx->stream);
        free_device(s);
    }
    delete s;
}

}  // extern "C"
