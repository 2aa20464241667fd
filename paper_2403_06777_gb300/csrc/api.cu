// api.cu -- the C ABI of libzxp (include/zxp.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "zxp.h"
#include "compile.h"
#include "kernel.h"
#include "checkpoint.h"
#include "objects.h"
#include "plan.h"
#include "ps.h"
#include "split.h"
#include "zring.h"

using namespace zxp;

namespace {

// Live contexts by id: a scalar's tables go back to the pool in the order
// of the stream they were allocated on while that context lives.
std::mutex g_ctx_mu;
std::map<uint64_t, cudaStream_t> g_live_ctx;
uint64_t g_next_ctx_id = 1;

// One memory pool per device for scalar tables (stream-ordered allocation:
// no device synchronisation on allocation or free).  It keeps up to 64 MB of
// freed memory for reuse.
cudaMemPool_t table_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = 64ull << 20;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // A block freed on a context's stream (behind kernels still queued
    // there) is not handed to the upload stream with a wait for that stream:
    // the copy would queue behind those kernels.
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    pools[device] = pool;
    return pool;
}

// seq: the number of the launch on ctx->stream that reads the tables (0:
// none known).
int ensure_device_tables(const zxp_scalar* s, zxp_ctx* ctx, DevTables* out, uint64_t seq = 0) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->dev.find(ctx->device);
    if (it != s->dev.end()) {
        // a copy queued on another stream: wait for it once
        if (!it->second.shared && it->second.stream != ctx->stream) {
            if (cudaDeviceSynchronize() != cudaSuccess) return ZXP_ECUDA;
            it->second.shared = true;
        }
        *out = it->second.t;
        return ZXP_OK;
    }
    const TableLayout L = table_layout(s->plan);
    // pack into the next pinned staging buffer once its last copy is done
    const int slot = ctx->stage_next;
    ctx->stage_next = (slot + 1) % zxp_ctx::kStages;
    if (!ctx->stage_ev[slot] && cudaEventCreateWithFlags(&ctx->stage_ev[slot], cudaEventDisableTiming) != cudaSuccess)
        return ZXP_ECUDA;
    if (!ctx->stage_seq[slot] || ctx->stage_seq[slot] > ctx->done_seq) {
        cudaError_t q = cudaEventQuery(ctx->stage_ev[slot]);
        if (q == cudaErrorNotReady) q = cudaEventSynchronize(ctx->stage_ev[slot]);
        if (q != cudaSuccess) return ZXP_ECUDA;
    }
    ctx->stage_seq[slot] = 0;
    if (ctx->stage_cap[slot] < L.copied) {
        if (ctx->stage[slot]) cudaFreeHost(ctx->stage[slot]);
        ctx->stage[slot] = nullptr;
        ctx->stage_cap[slot] = 0;
        const size_t cap = std::max(L.copied, (size_t)64 << 10);
        if (cudaMallocHost(&ctx->stage[slot], cap) != cudaSuccess) return ZXP_ENOMEM;
        ctx->stage_cap[slot] = cap;
    }
    unsigned char* host = ctx->stage[slot];
    memset(host, 0, L.copied);
    pack_tables(s->plan, L, host);
    cudaMemPool_t pool = table_pool(ctx->device);
    if (!pool) return ZXP_ECUDA;
    unsigned char* base = nullptr;
    // copy on the upload stream, so that it overlaps the kernels still queued
    // on the context's stream; that stream waits for the copy
    for (size_t i = 0; i < ctx->table_cache.size(); i++) {
        const size_t b = ctx->table_cache[i].second;
        if (b >= L.total && b <= 2 * L.total) {
            base = static_cast<unsigned char*>(ctx->table_cache[i].first);
            ctx->table_cache.erase(ctx->table_cache.begin() + (ptrdiff_t)i);
            break;
        }
    }
    if (!base && cudaMallocFromPoolAsync((void**)&base, L.total, pool, ctx->upload) != cudaSuccess)
        return ZXP_ENOMEM;
    if (cudaMemcpyAsync(base, host, L.copied, cudaMemcpyHostToDevice, ctx->upload) != cudaSuccess ||
        cudaEventRecord(ctx->stage_ev[slot], ctx->upload) != cudaSuccess) {
        cudaFreeAsync(base, ctx->upload);
        return ZXP_ECUDA;
    }
    if (cudaStreamWaitEvent(ctx->stream, ctx->stage_ev[slot], 0) != cudaSuccess) {
        cudaStreamSynchronize(ctx->upload);
        cudaFreeAsync(base, ctx->upload);
        return ZXP_ECUDA;
    }
    ctx->stage_seq[slot] = seq;
    zxp_scalar::DevCopy c;
    c.t = device_tables(L, base);
    c.stream = ctx->stream;
    c.ctx_id = ctx->id;
    // the inner table (inner parameters) is computed on the device, after
    // the copy, in the order of the context's stream
    if (queue_inner_table(s->plan, c.t, ctx->stream) != cudaSuccess) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeAsync(base, ctx->stream);
        return ZXP_ECUDA;
    }
    s->dev[ctx->device] = c;
    *out = c.t;
    return ZXP_OK;
}

// The 128-bit values of `s` on ctx's device (DevWide), uploaded on first use
// in the order of ctx's stream, after the 64-bit tables `d` (whose rows and
// low-bit states the 128-bit inner table reads); the inner table is then
// computed on the device.
int ensure_wide_tables(const zxp_scalar* s, zxp_ctx* ctx, const DevTables& d, DevWide* out) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->devw.find(ctx->device);
    if (it != s->devw.end()) {
        *out = it->second;
        return ZXP_OK;
    }
    const WideLayout L = wide_layout(s->plan);
    std::vector<unsigned char> host(L.copied ? L.copied : 16, 0);
    pack_wide(s->plan, L, host.data());
    void* base = nullptr;
    if (cudaMalloc(&base, L.total) != cudaSuccess) return ZXP_ENOMEM;
    // (pageable source: the stream is synchronised before `host` goes away)
    if ((L.copied && cudaMemcpyAsync(base, host.data(), L.copied, cudaMemcpyHostToDevice, ctx->stream) !=
                         cudaSuccess) ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaFree(base);
        return ZXP_ECUDA;
    }
    DevWide w = device_wide(L, static_cast<unsigned char*>(base));
    if (s->plan.k_inner && s->plan.inner &&
        inner_table_launch_wide(*s->plan.inner, s->plan.k_inner, w.itab, w.ipv, d.ifr, d.iadj, d.ilow, w.ftab,
                                ctx->stream) != cudaSuccess) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(base);
        return ZXP_ECUDA;
    }
    s->devw[ctx->device] = w;
    *out = w;
    return ZXP_OK;
}

// Wait until a kernel has published its result into pinned memory `h`
// (flags != 0, stored after the value with release semantics; the caller
// zeroes flags before the launch).  Spins on the flags word; every 20 us it
// asks the stream whether work failed or ended without a result, and after
// the first 200 us it sleeps between checks.  timeout_us < 0: no limit.
int wait_published(cudaStream_t stream, const DevResult* h, int64_t timeout_us) {
    auto published = [h] { return __atomic_load_n(&h->flags, __ATOMIC_ACQUIRE) != 0; };
    if (published()) return ZXP_OK;
    const auto t0 = std::chrono::steady_clock::now();
    int64_t next_check = 0;
    for (uint32_t it = 0;; it++) {
        if (published()) return ZXP_OK;
        if (timeout_us != 0 && (it & 63) != 63) continue;
        const int64_t el = std::chrono::duration_cast<std::chrono::microseconds>(
                               std::chrono::steady_clock::now() - t0).count();
        if (el < next_check) continue;
        next_check = el + 20;
        const cudaError_t e = cudaStreamQuery(stream);
        if (e != cudaSuccess && e != cudaErrorNotReady) return ZXP_ECUDA;
        if (published()) return ZXP_OK;
        if (e == cudaSuccess) return ZXP_ECUDA;   // the stream is idle and nothing was written
        if (timeout_us >= 0 && el >= timeout_us) return ZXP_EAGAIN;
        if (el >= 200) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Slice length and grid for `count` terms (slices a multiple of 8 terms so
// that the lanes of a warp run the unrolled 8-step blocks in step).
void launch_shape(const zxp_ctx* ctx, const Plan& pl, uint64_t count, uint64_t* span, int* grid) {
    sum_shape(pl, ctx->sm_count, ctx->max_grid, count, span, grid);
}

// Terms of a scalar: assignments of its outer parameters.
uint64_t term_count(const zxp_scalar* s) { return 1ull << (s->ps.k - s->ps.k_inner); }

int check_range(const zxp_scalar* s, uint64_t first, uint64_t count) {
    const uint64_t total = term_count(s);
    if (first > total || count > total - first) return ZXP_EINVAL;
    return ZXP_OK;
}

// Free a zxp_submit_tables scalar whose launch has ended (its result was
// seen): its device tables go to the context's cache for the next upload
// instead of back to the pool.
void release_owned(zxp_ctx* ctx, zxp_scalar* s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->dev.find(ctx->device);
        if (it != s->dev.end() && !it->second.shared && it->second.ctx_id == ctx->id &&
            ctx->table_cache.size() < zxp_ctx::kTableCache) {
            ctx->table_cache.push_back({static_cast<void*>(it->second.t.table), table_layout(s->plan).total});
            s->dev.erase(it);
        }
    }
    zxp_scalar_free(s);
}

// Queue one range on ctx->stream: the raw partial into dres, the device
// address of pinned host memory hres that the host polls (or, with hres
// null, device memory).
// seq: the launch's number on ctx->stream (0: not tracked).
int enqueue(zxp_ctx* ctx, const zxp_scalar* s, uint64_t first, uint64_t count, DevResult* dres,
            const DevResult* hres, uint64_t seq) {
    const bool host_result = hres != nullptr;
    DevTables d;
    int st = ensure_device_tables(s, ctx, &d, seq);
    if (st != ZXP_OK) return st;
    uint64_t span;
    int grid;
    launch_shape(ctx, s->plan, count, &span, &grid);
    return cuda_status(sum_launch(s->plan, d.table, d.pv, d.rows, d.adj, d.seek, d.zq, d.ftab, first, count,
                                  span, grid, ctx->acc, ctx->counter, dres, host_result, ctx->stream));
}

}  // namespace

zxp_scalar::~zxp_scalar() {
    int prev = -1;
    cudaGetDevice(&prev);
    for (auto& e : dev) {
        cudaSetDevice(e.first);
        void* p = e.second.t.table;   // one allocation holds every table
        bool queued = false;
        if (!e.second.shared) {
            // in the order of the allocating stream, while its context lives
            std::lock_guard<std::mutex> lk(g_ctx_mu);
            auto it = g_live_ctx.find(e.second.ctx_id);
            if (it != g_live_ctx.end() && it->second == e.second.stream)
                queued = cudaFreeAsync(p, e.second.stream) == cudaSuccess;
        }
        if (!queued) {
            // shared copy, or its context is gone: nothing may still use it
            cudaDeviceSynchronize();
            cudaFreeAsync(p, 0);
        }
    }
    for (auto& e : devw) {
        cudaSetDevice(e.first);
        cudaDeviceSynchronize();
        cudaFree(e.second.base);
    }
    if (prev >= 0) cudaSetDevice(prev);
}

int zxp::make_scalar(PS&& ps, zxp_scalar** out) {
    std::unique_ptr<zxp_scalar> s(new (std::nothrow) zxp_scalar());
    if (!s) return ZXP_ENOMEM;
    s->ps = std::move(ps);
    s->plan_status = build_plan(s->ps, &s->plan);
    if (s->plan_status != ZXP_OK) return s->plan_status;
    *out = s.release();
    return ZXP_OK;
}

namespace zxp {
namespace {
std::atomic<uint32_t> g_extra_tx{0};
}  // namespace
uint32_t test_extra_tx() { return g_extra_tx.load(std::memory_order_relaxed); }
}  // namespace zxp

extern "C" {

int zxp_test_table_timeout(int enable) {
    g_extra_tx.store(enable ? 16u : 0u, std::memory_order_relaxed);
    return ZXP_OK;
}

const char* zxp_strerror(int status) {
    switch (status) {
    case ZXP_OK: return "ok";
    case ZXP_EINVAL: return "invalid argument";
    case ZXP_ENOMEM: return "out of memory";
    case ZXP_ETOOBIG: return "problem exceeds the kernel's limits (k > 62 or too many forms)";
    case ZXP_EOVERFLOW: return "sqrt2 exponent too large for exact 64-bit numerators";
    case ZXP_ECUDA: return "CUDA error";
    case ZXP_ETIMEDOUT: return "timed out";
    case ZXP_EAGAIN: return "not finished";
    case ZXP_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

const char* zxp_version(void) { return "zxp 0.1 sm_103a"; }

int zxp_ctx_create(int device, void* cuda_stream, zxp_ctx** out) {
    if (!out) return ZXP_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return ZXP_ECUDA;
    if (device < 0 || device >= ndev) return ZXP_EINVAL;
    DeviceGuard g(device);
    std::unique_ptr<zxp_ctx> c(new (std::nothrow) zxp_ctx());
    if (!c) return ZXP_ENOMEM;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return ZXP_ECUDA;
    c->max_grid = c->sm_count * 16;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return ZXP_ECUDA;
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking) != cudaSuccess) return ZXP_ECUDA;
    // the sum kernels' accumulator starts at zero (64 bytes: the 128-bit
    // sum uses all of it, the 64-bit one the first half)
    if (cudaMalloc(&c->acc, 2 * sizeof(zw64)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMemset(c->acc, 0, 2 * sizeof(zw64)) != cudaSuccess) return ZXP_ECUDA;
    if (cudaMalloc(&c->wres, sizeof(DevResultW)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMalloc(&c->counter, sizeof(unsigned int)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMemset(c->counter, 0, sizeof(unsigned int)) != cudaSuccess) return ZXP_ECUDA;
    if (cudaMallocHost(&c->hres, sizeof(DevResult)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaHostGetDevicePointer((void**)&c->hres_dev, c->hres, 0) != cudaSuccess) return ZXP_ECUDA;
    {
        std::lock_guard<std::mutex> lk(g_ctx_mu);
        c->id = g_next_ctx_id++;
        g_live_ctx[c->id] = c->stream;
    }
    *out = c.release();
    return ZXP_OK;
}

void zxp_ctx_destroy(zxp_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    {
        // scalars freed from now on no longer queue on this stream
        std::lock_guard<std::mutex> lk(g_ctx_mu);
        g_live_ctx.erase(c->id);
    }
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->upload);
    for (auto& e : c->tickets) {
        if (e.second.owned) zxp_scalar_free(e.second.owned);
        c->free_slots.push_back(e.second);
    }
    for (auto& b : c->table_cache) cudaFreeAsync(b.first, c->upload);
    cudaStreamSynchronize(c->upload);
    for (auto& t : c->free_slots) cudaFreeHost(t.hres);
    for (int i = 0; i < zxp_ctx::kStages; i++) {
        if (c->stage[i]) cudaFreeHost(c->stage[i]);
        if (c->stage_ev[i]) cudaEventDestroy(c->stage_ev[i]);
    }
    cudaFree(c->acc);
    cudaFree(c->wres);
    cudaFree(c->counter);
    cudaFreeHost(c->hres);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->upload) cudaStreamDestroy(c->upload);
    delete c;
}


namespace {
int split_options(const zxp_split_opts* opts, SplitOptions* so) {
    if (!opts) return ZXP_OK;
    if (opts->min_k) so->min_k = opts->min_k;
    if (opts->max_inner) so->max_inner = opts->max_inner;
    if (opts->max_index_bits) so->max_index_bits = opts->max_index_bits;
    if (opts->max_cut) so->max_cut = opts->max_cut;
    if (opts->low_free) so->low_free = opts->low_free;
    if (opts->tries) so->tries = (int)opts->tries;
    if (opts->seed) so->seed = opts->seed;
    if (so->low_free < 4 || so->max_index_bits > kMaxInnerBits) return ZXP_EINVAL;
    return ZXP_OK;
}
}  // namespace

int zxp_compile(const zxp_gate* gates, size_t n_gates, int n_qubits, const uint8_t* in_bits,
                const uint8_t* out_bits, uint64_t marg_mask, int kind, zxp_scalar** out) {
    const zxp_split_opts defaults = {};
    return zxp_compile_ex(gates, n_gates, n_qubits, in_bits, out_bits, marg_mask, kind, &defaults, out);
}

int zxp_compile_ex(const zxp_gate* gates, size_t n_gates, int n_qubits, const uint8_t* in_bits,
                   const uint8_t* out_bits, uint64_t marg_mask, int kind, const zxp_split_opts* split,
                   zxp_scalar** out) {
    if (!out) return ZXP_EINVAL;
    *out = nullptr;
    PS ps;
    CompileOptions opt;
    opt.split = split != nullptr;
    int st = split_options(split, &opt.split_opt);
    if (st != ZXP_OK) return st;
    st = compile_circuit(gates, n_gates, n_qubits, in_bits, out_bits, marg_mask, kind, opt, &ps);
    if (st != ZXP_OK) return st;
    return make_scalar(std::move(ps), out);
}

int zxp_scalar_split(const zxp_scalar* s, const zxp_split_opts* opts, zxp_scalar** out) {
    if (!s || !out) return ZXP_EINVAL;
    *out = nullptr;
    if (s->ps.k_inner) return ZXP_EINVAL;
    SplitOptions so;
    int st = split_options(opts, &so);
    if (st != ZXP_OK) return st;
    PS ps;
    st = split_scalar(s->ps, so, &ps);
    if (st != ZXP_OK) return st;
    return make_scalar(std::move(ps), out);
}

int zxp_scalar_reorder(const zxp_scalar* s, zxp_scalar** out) {
    if (!s || !out) return ZXP_EINVAL;
    *out = nullptr;
    PS ps;
    const int st = reorder_scalar(s->ps, &ps);
    if (st != ZXP_OK) return st;
    return make_scalar(std::move(ps), out);
}

int zxp_inner_sum(zxp_ctx* ctx, const zxp_scalar* s) {
    if (!ctx || !s) return ZXP_EINVAL;
    if (!s->ps.k_inner) return ZXP_OK;
    DeviceGuard g(ctx->device);
    DevTables d;
    int st = ensure_device_tables(s, ctx, &d);
    if (st != ZXP_OK) return st;
    std::lock_guard<std::mutex> lk(s->mu);
    return cuda_status(queue_inner_table(s->plan, d, ctx->stream));
}

int zxp_compile_param(const zxp_gate* gates, size_t n_gates, int n_qubits, const uint8_t* in_bits,
                      const uint8_t* out_bits, const uint8_t* param_qubits, uint64_t marg_mask,
                      int kind, zxp_pscalar** out) {
    if (!out || !param_qubits) return ZXP_EINVAL;
    *out = nullptr;
    std::unique_ptr<zxp_pscalar> p(new (std::nothrow) zxp_pscalar());
    if (!p) return ZXP_ENOMEM;
    CompileOptions opt;
    int st = compile_circuit_param(gates, n_gates, n_qubits, in_bits, out_bits, param_qubits, marg_mask,
                                   kind, opt, &p->pps);
    if (st != ZXP_OK) return st;
    *out = p.release();
    return ZXP_OK;
}

int zxp_pscalar_info(const zxp_pscalar* ps, zxp_pscalar_info_t* info) {
    if (!ps || !info) return ZXP_EINVAL;
    memset(info, 0, sizeof *info);
    const PPS& p = ps->pps;
    info->k = p.k;
    info->n_params = p.p;
    info->n_lin = (uint32_t)p.lin.size();
    info->n_quad = (uint32_t)p.quad.size();
    info->n_node = (uint32_t)p.node.size();
    info->n_pair = (uint32_t)p.pair.size();
    info->e0 = p.e0;
    info->t_count = p.t_count;
    return ZXP_OK;
}

int zxp_pscalar_params(const zxp_pscalar* ps, uint32_t* qubits) {
    if (!ps || (!qubits && ps->pps.p)) return ZXP_EINVAL;
    for (uint32_t j = 0; j < ps->pps.p; j++) qubits[j] = ps->pps.param_qubit[j];
    return ZXP_OK;
}

int zxp_bind(const zxp_pscalar* ps, uint64_t bits, zxp_scalar** out) {
    if (!ps || !out) return ZXP_EINVAL;
    *out = nullptr;
    if (ps->pps.p < 64 && (bits >> ps->pps.p)) return ZXP_EINVAL;
    PS b;
    bind(ps->pps, bits, &b);
    return make_scalar(std::move(b), out);
}

void zxp_pscalar_free(zxp_pscalar* ps) { delete ps; }

int zxp_scalar_from_tables(const void* blob, size_t nbytes, zxp_scalar** out) {
    if (!out) return ZXP_EINVAL;
    *out = nullptr;
    PS ps;
    int st = ps_from_blob(blob, nbytes, &ps);
    if (st != ZXP_OK) return st;
    return make_scalar(std::move(ps), out);
}

int zxp_scalar_to_tables(const zxp_scalar* s, void* buf, size_t* nbytes) {
    if (!s || !nbytes) return ZXP_EINVAL;
    size_t need = ps_blob_size(s->ps);
    if (!buf) { *nbytes = need; return ZXP_OK; }
    if (*nbytes < need) { *nbytes = need; return ZXP_EINVAL; }
    ps_to_blob(s->ps, buf);
    *nbytes = need;
    return ZXP_OK;
}

int zxp_scalar_info(const zxp_scalar* s, zxp_scalar_info_t* info) {
    if (!s || !info) return ZXP_EINVAL;
    memset(info, 0, sizeof *info);
    info->k = s->ps.k - s->ps.k_inner;
    info->k_inner = s->ps.k_inner;
    info->inner_bits = s->plan.inner_bits;
    info->n_lin = (uint32_t)s->ps.lin.size();
    info->n_quad = (uint32_t)s->ps.quad.size();
    info->n_node = (uint32_t)s->ps.node.size();
    info->n_pair = (uint32_t)s->ps.pair.size();
    info->e0 = s->ps.e0;
    info->acc_bits = s->ps.e0 <= 124 ? 64 : (s->ps.e0 <= 252 ? 128 : 0);
    info->form_bits = s->plan.kp.nbits;
    info->t_count = s->ps.t_count;
    info->node_words = (uint32_t)s->plan.nwn;
    info->other_words = (uint32_t)(s->plan.nwl < 1 ? 1 : s->plan.nwl);
    const TableLayout L = table_layout(s->plan);
    info->device_bytes = (uint32_t)std::min<size_t>(L.total, 0xFFFFFFFFu);
    info->upload_bytes = (uint32_t)L.copied;
    info->kernel_variant = (uint32_t)sum_variant(s->plan);
    return ZXP_OK;
}

void zxp_scalar_free(zxp_scalar* s) { delete s; }

int zxp_eval(zxp_ctx* ctx, const zxp_scalar* s, uint64_t first, uint64_t count, zxp_zomega* out) {
    if (!ctx || !s || !out) return ZXP_EINVAL;
    int st = check_range(s, first, count);
    if (st != ZXP_OK) return st;
    if (count == 0 || s->plan.zero) { from_zw(zw_zero(), s->ps.e0, 1, out); return ZXP_OK; }
    DeviceGuard g(ctx->device);
    ctx->hres->flags = 0;
    const uint64_t seq = ++ctx->enq_seq;
    st = enqueue(ctx, s, first, count, ctx->hres_dev, ctx->hres, seq);   // the kernel writes the pinned result
    if (st != ZXP_OK) return st;
    if ((st = wait_published(ctx->stream, ctx->hres, -1)) != ZXP_OK) return st;
    if (seq > ctx->done_seq) ctx->done_seq = seq;
    memcpy(out, ctx->hres, sizeof *out);
    return (out->flags & 2) ? ZXP_ETIMEDOUT : ZXP_OK;
}

int zxp_eval_device(zxp_ctx* ctx, const zxp_scalar* s, uint64_t first, uint64_t count,
                    zxp_zomega* dev_out) {
    if (!ctx || !s || !dev_out || ((uintptr_t)dev_out & 7)) return ZXP_EINVAL;
    int st = check_range(s, first, count);
    if (st != ZXP_OK) return st;
    DeviceGuard g(ctx->device);
    return enqueue(ctx, s, first, count, reinterpret_cast<DevResult*>(dev_out), nullptr, ++ctx->enq_seq);
}

int zxp_zomega_canon(const zxp_zomega* in, zxp_zomega* out) {
    if (!in || !out) return ZXP_EINVAL;
    __int128 c[4] = {in->c[0], in->c[1], in->c[2], in->c[3]};
    int32_t e = in->e;
    canon_i128(c, &e);
    for (int i = 0; i < 4; i++) out->c[i] = (int64_t)c[i];
    out->e = e;
    out->flags = 0;
    return ZXP_OK;
}

int zxp_amplitude(zxp_ctx* ctx, const zxp_scalar* s, zxp_zomega* out) {
    if (!s || !out) return ZXP_EINVAL;
    if (s->ps.e0 > 124 && s->ps.e0 <= 252) {
        // modulo 2^128, then back to 64-bit words if the canonical value fits
        zxp_zomega_wide w;
        const int st = zxp_amplitude_wide(ctx, s, &w);
        if (st != ZXP_OK) return st;
        bool fits = true;
        for (int i = 0; i < 4; i++) {
            out->c[i] = w.c[i];
            fits = fits && w.hi[i] == (w.c[i] < 0 ? -1 : 0);
        }
        out->e = w.e;
        out->flags = 0;
        return fits ? ZXP_OK : ZXP_EOVERFLOW;
    }
    zxp_zomega raw;
    int st = zxp_eval(ctx, s, 0, term_count(s), &raw);
    if (st != ZXP_OK) return st;
    zxp_zomega_canon(&raw, out);
    return s->ps.e0 > 252 ? ZXP_EOVERFLOW : ZXP_OK;
}

int zxp_eval_wide(zxp_ctx* ctx, const zxp_scalar* s, uint64_t first, uint64_t count, zxp_zomega_wide* out) {
    if (!ctx || !s || !out) return ZXP_EINVAL;
    int st = check_range(s, first, count);
    if (st != ZXP_OK) return st;
    memset(out, 0, sizeof *out);
    out->e = s->ps.e0;
    out->flags = 1;
    if (count == 0 || s->plan.zero) return ZXP_OK;
    DeviceGuard g(ctx->device);
    DevTables d;
    const uint64_t seq = ++ctx->enq_seq;
    if ((st = ensure_device_tables(s, ctx, &d, seq)) != ZXP_OK) return st;
    DevWide w;
    if ((st = ensure_wide_tables(s, ctx, d, &w)) != ZXP_OK) return st;
    const cudaError_t e = sum_launch_wide(s->plan, w.table, w.pv, d.rows, d.adj, d.seek, d.zq, w.ftab, first, count,
                                          ctx->sm_count, reinterpret_cast<uint64_t*>(ctx->acc), ctx->counter,
                                          ctx->wres, ctx->stream);
    if (e != cudaSuccess) return ZXP_ECUDA;
    DevResultW r;
    if (cudaMemcpyAsync(&r, ctx->wres, sizeof r, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (seq > ctx->done_seq) ctx->done_seq = seq;
    static_assert(sizeof(DevResultW) == sizeof(zxp_zomega_wide), "result record layout");
    memcpy(out, &r, sizeof r);
    return (out->flags & 2) ? ZXP_ETIMEDOUT : ZXP_OK;
}

int zxp_sum_resumable(zxp_ctx* ctx, const zxp_scalar* s, uint32_t chunk_log2, const char* path,
                      uint64_t max_chunks, zxp_zomega* out, uint64_t* chunks_done, uint64_t* chunks_total) {
    if (!ctx || !s || !path || !*path || !out) return ZXP_EINVAL;
    const uint32_t k = s->ps.k - s->ps.k_inner;
    const uint32_t width = s->ps.e0 > 124 ? 128 : 64;
    std::vector<uint8_t> blob(ps_blob_size(s->ps));
    ps_to_blob(s->ps, blob.data());
    const uint64_t digest = ckpt::fnv1a(blob.data(), blob.size());
    auto eval = [&](uint64_t first, uint64_t count, uint64_t lo[4], uint64_t hi[4]) -> int {
        if (width == 128) {
            zxp_zomega_wide w;
            const int st = zxp_eval_wide(ctx, s, first, count, &w);
            for (int i = 0; i < 4; i++) {
                lo[i] = (uint64_t)w.c[i];
                hi[i] = (uint64_t)w.hi[i];
            }
            return st;
        }
        zxp_zomega z;
        const int st = zxp_eval(ctx, s, first, count, &z);
        for (int i = 0; i < 4; i++) lo[i] = (uint64_t)z.c[i];
        return st;
    };
    ckpt::State st;
    const int r = ckpt::run(path, width, digest, k, chunk_log2, s->ps.e0, max_chunks, eval, &st);
    if (chunks_done) *chunks_done = st.done_count;
    if (chunks_total) *chunks_total = st.n_chunks;
    if (r != ZXP_OK) return r;
    __int128 c[4];
    for (int i = 0; i < 4; i++)
        c[i] = width == 128 ? (__int128)(((u128)st.sum[4 + i] << 64) | (u128)st.sum[i]) : (__int128)(int64_t)st.sum[i];
    int32_t e = s->ps.e0;
    canon_i128(c, &e);
    bool fits = true;
    for (int i = 0; i < 4; i++) {
        out->c[i] = (int64_t)c[i];
        fits = fits && c[i] == (__int128)(int64_t)c[i];
    }
    out->e = e;
    out->flags = 0;
    return (s->ps.e0 > 252 || !fits) ? ZXP_EOVERFLOW : ZXP_OK;
}

int zxp_amplitude_wide(zxp_ctx* ctx, const zxp_scalar* s, zxp_zomega_wide* out) {
    if (!s || !out) return ZXP_EINVAL;
    const int st = zxp_eval_wide(ctx, s, 0, term_count(s), out);
    if (st != ZXP_OK) return st;
    __int128 c[4];
    for (int i = 0; i < 4; i++) c[i] = (__int128)(((u128)(uint64_t)out->hi[i] << 64) | (u128)(uint64_t)out->c[i]);
    int32_t e = out->e;
    canon_i128(c, &e);
    for (int i = 0; i < 4; i++) {
        out->c[i] = (int64_t)(uint64_t)(u128)c[i];
        out->hi[i] = (int64_t)(uint64_t)((u128)c[i] >> 64);
    }
    out->e = e;
    out->flags = 0;
    return s->ps.e0 > 252 ? ZXP_EOVERFLOW : ZXP_OK;
}

int zxp_submit(zxp_ctx* ctx, const zxp_scalar* s, uint64_t first, uint64_t count, uint64_t* ticket) {
    if (!ctx || !s || !ticket) return ZXP_EINVAL;
    int st = check_range(s, first, count);
    if (st != ZXP_OK) return st;
    Ticket t;
    t.e0 = s->ps.e0;
    if (count == 0 || s->plan.zero) {
        t.trivial = true;
    } else {
        DeviceGuard g(ctx->device);
        if (!ctx->free_slots.empty()) {
            t.dres = ctx->free_slots.back().dres;
            t.hres = ctx->free_slots.back().hres;
            ctx->free_slots.pop_back();
        } else {
            if (cudaMallocHost(&t.hres, sizeof(DevResult)) != cudaSuccess) return ZXP_ENOMEM;
            if (cudaHostGetDevicePointer((void**)&t.dres, t.hres, 0) != cudaSuccess) {
                cudaFreeHost(t.hres);
                return ZXP_ECUDA;
            }
        }
        t.hres->flags = 0;
        t.seq = ++ctx->enq_seq;
        st = enqueue(ctx, s, first, count, t.dres, t.hres, t.seq);   // the kernel writes the pinned result
        if (st != ZXP_OK) { ctx->free_slots.push_back(t); return st; }
    }
    *ticket = ctx->next_ticket++;
    ctx->tickets[*ticket] = t;
    return ZXP_OK;
}

int zxp_poll(zxp_ctx* ctx, uint64_t ticket, int64_t timeout_us, zxp_zomega* out) {
    if (!ctx || !out) return ZXP_EINVAL;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return ZXP_ENOTFOUND;
    Ticket& t = it->second;
    if (!t.trivial) {
        DeviceGuard g(ctx->device);
        const int st = wait_published(ctx->stream, t.hres, timeout_us);
        if (st != ZXP_OK) return st;
        if (t.seq > ctx->done_seq) ctx->done_seq = t.seq;
        memcpy(out, t.hres, sizeof *out);
        if (out->flags & 2) {
            if (t.owned) release_owned(ctx, t.owned);
            ctx->free_slots.push_back(t);
            ctx->tickets.erase(it);
            return ZXP_ETIMEDOUT;
        }
    } else {
        from_zw(zw_zero(), t.e0, 1, out);
    }
    if (t.owned) release_owned(ctx, t.owned);
    if (!t.trivial) ctx->free_slots.push_back(t);
    ctx->tickets.erase(it);
    return ZXP_OK;
}

int zxp_submit_tables(zxp_ctx* ctx, const void* blob, size_t nbytes, uint64_t* ticket) {
    if (!ctx || !blob || !ticket) return ZXP_EINVAL;
    zxp_scalar* s = nullptr;
    int st = zxp_scalar_from_tables(blob, nbytes, &s);
    if (st != ZXP_OK) return st;
    st = zxp_submit(ctx, s, 0, term_count(s), ticket);
    if (st != ZXP_OK) {
        zxp_scalar_free(s);
        return st;
    }
    ctx->tickets[*ticket].owned = s;
    return ZXP_OK;
}

int zxp_zomega_add(const zxp_zomega* a, const zxp_zomega* b, zxp_zomega* out) {
    if (!a || !b || !out) return ZXP_EINVAL;
    zw64 x = to_zw(*a), y = to_zw(*b);
    int32_t ea = a->e, eb = b->e;
    while (ea < eb) { x = zw_mul_sqrt2(x); ea++; }
    while (eb < ea) { y = zw_mul_sqrt2(y); eb++; }
    from_zw(zw_add(x, y), ea, (a->flags | b->flags) & 1, out);
    return ZXP_OK;
}

void zxp_zomega_to_complex(const zxp_zomega* z, double* re, double* im) {
    if (!z) return;
    const double h = 0.70710678118654752440;
    double c0 = (double)z->c[0], c1 = (double)z->c[1], c2 = (double)z->c[2], c3 = (double)z->c[3];
    double r = c0 + h * c1 - h * c3, i = h * c1 + c2 + h * c3;
    double s = 1.0;
    for (int k = 0; k < z->e; k++) s *= h;
    for (int k = 0; k < -z->e; k++) s *= 1.41421356237309504880;
    if (re) *re = r * s;
    if (im) *im = i * s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

struct zxp_batch {
    zxp_ctx* ctx = nullptr;
    size_t n = 0;
    struct Group {
        int key;
        uint32_t ntab_cap, npairs_cap;
        std::vector<uint32_t> members;
        uint32_t off = 0, count = 0;   // chunk range of this group
        int grid = 1;
    };
    std::vector<Group> groups;
    unsigned char* d_scalars = nullptr;   // n descriptors, kBatchScalarBytes apart
    BatchChunk* d_chunks = nullptr;
    size_t chunk_cap = 0;
    unsigned int* d_queue = nullptr;
    DevResult* d_results = nullptr;
    DevResult* h_results = nullptr;
    int threads = 256;
    uint32_t chunk_log2 = 16;
    uint32_t candidates = 0;
    double tuned_us = 0, total_terms = 0;
    std::vector<uint32_t> k;   // per scalar
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    ~zxp_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_scalars);
        cudaFree(d_chunks);
        cudaFree(d_queue);
        cudaFree(d_results);
        cudaFreeHost(h_results);
    }
};

namespace {

// Chunk list for chunk length 2^clog: groups contiguous, a scalar's chunks
// in index order.
std::vector<BatchChunk> batch_chunks(zxp_batch* b, uint32_t clog) {
    std::vector<BatchChunk> out;
    for (auto& g : b->groups) {
        g.off = (uint32_t)out.size();
        for (uint32_t m : g.members) {
            const uint64_t total = 1ull << b->k[m];
            const uint64_t len = 1ull << clog;
            for (uint64_t f = 0; f < total; f += len)
                out.push_back(BatchChunk{m, m, f, (total - f < len) ? total - f : len});
        }
        g.count = (uint32_t)out.size() - g.off;
    }
    return out;
}

int batch_upload_chunks(zxp_batch* b, const std::vector<BatchChunk>& ch) {
    if (ch.size() > b->chunk_cap) {
        cudaFree(b->d_chunks);
        b->d_chunks = nullptr;
        b->chunk_cap = 0;
        if (cudaMalloc(&b->d_chunks, ch.size() * sizeof(BatchChunk)) != cudaSuccess) return ZXP_ENOMEM;
        b->chunk_cap = ch.size();
    }
    if (cudaMemcpy(b->d_chunks, ch.data(), ch.size() * sizeof(BatchChunk), cudaMemcpyHostToDevice) != cudaSuccess)
        return ZXP_ECUDA;
    return ZXP_OK;
}

int batch_shape(zxp_batch* b, int threads) {
    for (auto& g : b->groups) {
        int bps = 0;
        if (batch_occupancy(g.key, g.ntab_cap, g.npairs_cap, threads, &bps) != cudaSuccess || bps < 1)
            return ZXP_ECUDA;
        int grid = b->ctx->sm_count * bps;
        if ((uint32_t)grid > g.count) grid = (int)g.count;
        g.grid = grid < 1 ? 1 : grid;
    }
    return ZXP_OK;
}

// clears, one launch per group, and the result copy, all on the stream
int batch_enqueue(zxp_batch* b, bool copy_out) {
    cudaStream_t st = b->ctx->stream;
    if (cudaMemsetAsync(b->d_results, 0, b->n * sizeof(DevResult), st) != cudaSuccess) return ZXP_ECUDA;
    if (cudaMemsetAsync(b->d_queue, 0, b->groups.size() * sizeof(unsigned int), st) != cudaSuccess) return ZXP_ECUDA;
    for (size_t i = 0; i < b->groups.size(); i++) {
        const auto& g = b->groups[i];
        if (!g.count) continue;
        if (batch_launch(g.key, b->d_scalars, b->d_chunks + g.off, g.count, b->d_queue + i,
                         b->d_results, g.ntab_cap, g.npairs_cap, b->threads, g.grid, 1, st) != cudaSuccess)
            return ZXP_ECUDA;
    }
    if (copy_out && cudaMemcpyAsync(b->h_results, b->d_results, b->n * sizeof(DevResult),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ZXP_ECUDA;
    return ZXP_OK;
}

}  // namespace

extern "C" int zxp_batch_create(zxp_ctx* ctx, const zxp_scalar* const* scalars, size_t n,
                                zxp_batch** out) {
    if (!ctx || !scalars || !out || n == 0 || n > 0xFFFFFFFFu) return ZXP_EINVAL;
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    std::unique_ptr<zxp_batch> b(new (std::nothrow) zxp_batch());
    if (!b) return ZXP_ENOMEM;
    b->ctx = ctx;
    b->n = n;
    std::vector<unsigned char> hs(n * kBatchScalarBytes, 0);
    std::map<int, size_t> gidx;
    for (size_t i = 0; i < n; i++) {
        const zxp_scalar* s = scalars[i];
        if (!s || s->ps.k_inner) return ZXP_EINVAL;   // (inner parameters: single-scalar path only)
        DevTables d;
        int st = ensure_device_tables(s, ctx, &d);
        if (st != ZXP_OK) return st;
        const Plan& pl = s->plan;
        BatchScalar& bs = *reinterpret_cast<BatchScalar*>(hs.data() + i * kBatchScalarBytes);
        bs = batch_descriptor(pl, d);
        b->k.push_back(s->ps.k);
        b->total_terms += std::ldexp(1.0, (int)s->ps.k);
        auto it = gidx.find(bs.key);
        if (it == gidx.end()) {
            it = gidx.emplace(bs.key, b->groups.size()).first;
            b->groups.push_back(zxp_batch::Group{bs.key, 0, 0, {}, 0, 0, 1});
        }
        auto& g = b->groups[it->second];
        g.members.push_back((uint32_t)i);
        g.ntab_cap = std::max(g.ntab_cap, pl.kp.tab_size);
        g.npairs_cap = std::max(g.npairs_cap, pl.kp.npairs);
    }
    if (cudaMalloc(&b->d_scalars, hs.size()) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMemcpy(b->d_scalars, hs.data(), hs.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return ZXP_ECUDA;
    if (cudaMalloc(&b->d_queue, b->groups.size() * sizeof(unsigned int)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMalloc(&b->d_results, n * sizeof(DevResult)) != cudaSuccess) return ZXP_ENOMEM;
    if (cudaMallocHost(&b->h_results, n * sizeof(DevResult)) != cudaSuccess) return ZXP_ENOMEM;

    // tuner: time every (chunk length, block size) candidate on this batch
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ZXP_ECUDA;
    double best = -1;
    uint32_t best_clog = 16;
    int best_threads = 256;
    int st = ZXP_OK;
    for (uint32_t clog = 12; clog <= 20 && st == ZXP_OK; clog += 2) {
        std::vector<BatchChunk> ch = batch_chunks(b.get(), clog);
        if (ch.size() > (1u << 22)) continue;
        if ((st = batch_upload_chunks(b.get(), ch)) != ZXP_OK) break;
        for (int threads : {128, 256}) {
            b->threads = threads;
            if ((st = batch_shape(b.get(), threads)) != ZXP_OK) break;
            if ((st = batch_enqueue(b.get(), false)) != ZXP_OK) break;   // warm-up
            double t_min = -1;
            for (int rep = 0; rep < 2; rep++) {
                cudaEventRecord(e0, ctx->stream);
                if ((st = batch_enqueue(b.get(), false)) != ZXP_OK) break;
                cudaEventRecord(e1, ctx->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = ZXP_ECUDA; break; }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (t_min < 0 || ms < t_min) t_min = ms;
            }
            b->candidates++;
            if (st == ZXP_OK && (best < 0 || t_min < best)) {
                best = t_min;
                best_clog = clog;
                best_threads = threads;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ZXP_OK) return st;
    b->chunk_log2 = best_clog;
    b->threads = best_threads;
    b->tuned_us = best * 1e3;
    if ((st = batch_upload_chunks(b.get(), batch_chunks(b.get(), best_clog))) != ZXP_OK) return st;
    if ((st = batch_shape(b.get(), best_threads)) != ZXP_OK) return st;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ZXP_ECUDA;

    // capture the evaluation as a graph on the context's stream
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ZXP_ECUDA;
    st = batch_enqueue(b.get(), true);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != ZXP_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != ZXP_OK ? st : ZXP_ECUDA;
    }
    b->graph = graph;
    if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) return ZXP_ECUDA;
    *out = b.release();
    return ZXP_OK;
}

extern "C" int zxp_batch_run(zxp_batch* b, zxp_zomega* out) {
    if (!b || !out) return ZXP_EINVAL;
    DeviceGuard dg(b->ctx->device);
    if (cudaGraphLaunch(b->exec, b->ctx->stream) != cudaSuccess) return ZXP_ECUDA;
    if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) return ZXP_ECUDA;
    memcpy(out, b->h_results, b->n * sizeof(zxp_zomega));
    for (size_t i = 0; i < b->n; i++)
        if (out[i].flags & 2) return ZXP_ETIMEDOUT;
    return ZXP_OK;
}

extern "C" int zxp_batch_info(const zxp_batch* b, zxp_batch_info_t* info) {
    if (!b || !info) return ZXP_EINVAL;
    memset(info, 0, sizeof *info);
    info->n_scalars = (uint32_t)b->n;
    info->n_groups = (uint32_t)b->groups.size();
    uint32_t nch = 0;
    for (auto& g : b->groups) nch += g.count;
    info->n_chunks = nch;
    info->threads = (uint32_t)b->threads;
    info->chunk_log2 = b->chunk_log2;
    info->candidates = b->candidates;
    info->tuned_us = b->tuned_us;
    info->total_terms = b->total_terms;
    return ZXP_OK;
}

extern "C" void zxp_batch_destroy(zxp_batch* b) {
    if (!b) return;
    DeviceGuard dg(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    delete b;
}

// ---------------------------------------------------------------------------
// Evaluation without any allocation.
//
// Some callers cannot allocate device memory through the CUDA runtime: code
// that runs under a memory manager owning the whole device (a framework's
// caching allocator or a serving runtime's fixed arena, where a foreign
// cudaMalloc breaks the accounting or fails), and latency-critical loops,
// where cudaMalloc / cudaFree synchronise the device.  zxp_eval_noalloc
// serves them: it stages the scalar's tables and keeps the kernel's scratch
// (the 64-bit accumulator and the completion counter) in one file-scope
// device array of fixed size, and writes the result to a buffer the caller
// owns.  It makes no device allocation and calls neither cudaMalloc nor
// cudaFree.  (On the host, the first call for a kernel variant on a device
// fills the launch-shape caches, and the runtime stages the pageable table
// copies in its own host buffers.)
// ---------------------------------------------------------------------------

namespace {

// Layout of the static scratch: [counter at 0, accumulator at 64; 256 B]
// [tables].  Launches use at most kNoAllocMaxBlocks blocks.
constexpr size_t kNoAllocBytes = 256 * 1024;
constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocAccOff = 64;
constexpr size_t kNoAllocTablesOff = 256;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

extern "C" int zxp_eval_noalloc(const zxp_scalar* s, uint64_t first, uint64_t count,
                                zxp_zomega* dev_out, void* cuda_stream) {
    if (!s || !dev_out || ((uintptr_t)dev_out & 7)) return ZXP_EINVAL;
    int st = check_range(s, first, count);
    if (st != ZXP_OK) return st;
    const Plan& pl = s->plan;
    if (pl.k_inner) return ZXP_ETOOBIG;   // the inner table does not fit the static scratch
    const size_t tb = pl.table.size() * sizeof(zw64), pb = pl.pv.size() * sizeof(zw64);
    const size_t fb = pl.rows.size() * sizeof(uint32_t), ab = pl.adj.size() * sizeof(uint64_t);
    const size_t o_pv = kNoAllocTablesOff + tb, o_f = (o_pv + pb + 15) & ~(size_t)15;
    const size_t o_adj = (o_f + fb + 15) & ~(size_t)15;
    const size_t sb = pl.seek.size() * sizeof(uint32_t), lb = pl.lut.size() * sizeof(uint64_t);
    const size_t o_seek = (o_adj + ab + 15) & ~(size_t)15;
    if (o_seek + sb + lb + 16 > kNoAllocBytes) return ZXP_ETOOBIG;   // tables exceed the static scratch

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return ZXP_ECUDA;
    // the array's device address on the current device, looked up at every
    // call (a host-side lookup: an address kept from an earlier call would
    // be stale after the device's primary context was reset)
    struct {
        unsigned char* base;
        int sm_count;
    } d = {nullptr, 0};
    {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ZXP_ECUDA;
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ZXP_ECUDA;
        d.base = static_cast<unsigned char*>(p);
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // launch shape: at most kNoAllocMaxBlocks blocks
    uint64_t sp = 64;
    int grid = 1;
    sum_shape(pl, d.sm_count, kNoAllocMaxBlocks, count, &sp, &grid);
    const uint64_t g = (uint64_t)grid;

    // stage the tables (each call: the array keeps the last call's contents)
    // and clear the completion counter and the accumulator, which must start
    // at zero
    unsigned char* base = d.base;
    if (tb && cudaMemcpyAsync(base + kNoAllocTablesOff, pl.table.data(), tb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (pb && cudaMemcpyAsync(base + o_pv, pl.pv.data(), pb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (fb && cudaMemcpyAsync(base + o_f, pl.rows.data(), fb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (ab && cudaMemcpyAsync(base + o_adj, pl.adj.data(), ab, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (sb && cudaMemcpyAsync(base + o_seek, pl.seek.data(), sb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (lb && cudaMemcpyAsync(base + o_seek + sb, pl.lut.data(), lb, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return ZXP_ECUDA;
    if (cudaMemsetAsync(base, 0, kNoAllocAccOff + sizeof(zw64), stream) != cudaSuccess) return ZXP_ECUDA;
    return cuda_status(sum_launch(pl, reinterpret_cast<const zw64*>(base + kNoAllocTablesOff),
                                  reinterpret_cast<const zw64*>(base + o_pv),
                                  reinterpret_cast<const uint32_t*>(base + o_f),
                                  reinterpret_cast<const uint64_t*>(base + o_adj),
                                  reinterpret_cast<const uint32_t*>(base + o_seek), nullptr, nullptr, first,
                                  count, sp,
                                  (int)g, reinterpret_cast<zw64*>(base + kNoAllocAccOff),
                                  reinterpret_cast<unsigned int*>(base),
                                  reinterpret_cast<DevResult*>(dev_out), false, stream));
}
