// sample.cpp -- weak simulation by chained marginals (Sec. 2.2, App. F's
// Algorithm 2) and marginals by summing amplitudes (Sec. 2.2), on top of
// the request server: every probability is an exact parametric evaluation
// on the device.
//
// Algorithm 2 reduces the n doubled diagrams P(a_1 .. a_j) (j = 1..n) once,
// with the bits a_1 .. a_j as parameters, and then, for j = 1..n, evaluates
// P(B_i || 0) for every sample i together and sets bit j of sample i to 0
// when u < P(B_i || 0) / P(B_i), else 1.  The algorithm as printed compares u
// with P(B_i || 0) alone; the conditional probability of Sec. 2.2 (the ratio)
// is what samples the output distribution and is what this file does.
//
// The decision compares doubles computed from the exact values with one
// fixed sequence of IEEE operations (real_value below), so it is
// reproducible bit for bit by any program holding the same exact values.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <memory>
#include <new>
#include <vector>

#include "zxp.h"

namespace {

constexpr double kInvSqrt2 = 0.70710678118654752440;

// Real part of (c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^e as a double:
// (double(c0) + double(c1 - c3) * (1/sqrt2)) scaled by 2^(-e/2), with one
// more factor 1/sqrt2 for odd e.
double real_value(const zxp_zomega& z) {
    double r = (double)z.c[0] + (double)(z.c[1] - z.c[3]) * kInvSqrt2;
    int e = z.e;
    if (e & 1) {
        r *= kInvSqrt2;
        e -= 1;
    }
    return ldexp(r, -e / 2);
}

zxp_zomega neg(const zxp_zomega& a) {
    zxp_zomega r = a;
    for (int i = 0; i < 4; i++) r.c[i] = (int64_t)(0 - (uint64_t)a.c[i]);
    return r;
}

}  // namespace

struct zxp_sampler {
    zxp_ctx* ctx = nullptr;
    int n = 0;
    std::vector<zxp_pscalar*> marg;   // marg[j]: P(a_0 .. a_j), bits a_0 .. a_j parameters
    zxp_server* srv = nullptr;

    ~zxp_sampler() {
        if (srv) zxp_server_destroy(srv);
        for (auto* p : marg) zxp_pscalar_free(p);
    }
};

extern "C" {

int zxp_sampler_create(zxp_ctx* ctx, const zxp_gate* gates, size_t n_gates, int n_qubits,
                       const uint8_t* in_bits, zxp_sampler** out) {
    if (!ctx || !out || n_qubits < 1 || n_qubits > 64 || (n_gates && !gates)) return ZXP_EINVAL;
    *out = nullptr;
    std::unique_ptr<zxp_sampler> s(new (std::nothrow) zxp_sampler());
    if (!s) return ZXP_ENOMEM;
    s->ctx = ctx;
    s->n = n_qubits;
    std::vector<uint8_t> zeros((size_t)n_qubits, 0), flags((size_t)n_qubits, 0);
    for (int j = 0; j < n_qubits; j++) {
        flags[(size_t)j] = 1;
        const uint64_t mask = (j == 63) ? ~0ull : ((2ull << j) - 1);
        zxp_pscalar* p = nullptr;
        int st = zxp_compile_param(gates, n_gates, n_qubits, in_bits, zeros.data(), flags.data(), mask,
                                   ZXP_MARGINAL_DOUBLED, &p);
        if (st != ZXP_OK) return st;
        s->marg.push_back(p);
    }
    zxp_server_opts opts;
    memset(&opts, 0, sizeof opts);
    opts.max_k = 62;
    int st = zxp_server_create(ctx, &opts, &s->srv);
    if (st != ZXP_OK) return st;
    *out = s.release();
    return ZXP_OK;
}

int zxp_sampler_info(const zxp_sampler* s, uint32_t* k_per_prefix) {
    if (!s || !k_per_prefix) return ZXP_EINVAL;
    for (int j = 0; j < s->n; j++) {
        zxp_pscalar_info_t info;
        int st = zxp_pscalar_info(s->marg[(size_t)j], &info);
        if (st != ZXP_OK) return st;
        k_per_prefix[j] = info.k;
    }
    return ZXP_OK;
}

int zxp_sampler_draw(zxp_sampler* s, size_t n_samples, const double* u, uint8_t* out_bits,
                     zxp_zomega* prob) {
    if (!s || (n_samples && (!u || !out_bits))) return ZXP_EINVAL;
    const int n = s->n;
    std::vector<uint64_t> prefix(n_samples, 0);
    std::vector<zxp_zomega> pB(n_samples);                // P(B_i), exact
    for (auto& z : pB) { memset(&z, 0, sizeof z); z.c[0] = 1; }
    std::vector<uint64_t> tickets(n_samples);
    for (int j = 0; j < n; j++) {
        // P(B_i || 0): bit j of the binding is 0
        for (size_t i = 0; i < n_samples; i++) {
            int st = zxp_server_submit_bind(s->srv, s->marg[(size_t)j], prefix[i], &tickets[i]);
            if (st != ZXP_OK) return st;
        }
        for (size_t i = 0; i < n_samples; i++) {
            zxp_zomega p0;
            int st = zxp_server_poll(s->srv, tickets[i], -1, &p0, nullptr);
            if (st != ZXP_OK) return st;
            const double r = real_value(p0) / real_value(pB[i]);
            if (u[i * (size_t)n + (size_t)j] < r) {
                pB[i] = p0;
            } else {
                zxp_zomega p1, c;
                const zxp_zomega m = neg(p0);
                zxp_zomega_add(&pB[i], &m, &p1);
                zxp_zomega_canon(&p1, &c);
                pB[i] = c;
                prefix[i] |= 1ull << j;
            }
        }
    }
    for (size_t i = 0; i < n_samples; i++) {
        for (int j = 0; j < n; j++) out_bits[i * (size_t)n + (size_t)j] = (uint8_t)((prefix[i] >> j) & 1);
        if (prob) prob[i] = pB[i];
    }
    return ZXP_OK;
}

void zxp_sampler_destroy(zxp_sampler* s) { delete s; }

int zxp_marginal_by_sum(zxp_ctx* ctx, const zxp_gate* gates, size_t n_gates, int n_qubits,
                        const uint8_t* in_bits, uint64_t mask, const uint8_t* bits, zxp_zomega* out) {
    if (!ctx || !out || !bits || n_qubits < 1 || n_qubits > 64 || (n_gates && !gates)) return ZXP_EINVAL;
    const uint64_t all = n_qubits == 64 ? ~0ull : ((1ull << n_qubits) - 1);
    if (mask & ~all) return ZXP_EINVAL;
    // amplitude with the unmasked output bits as parameters
    std::vector<uint8_t> flags((size_t)n_qubits, 0), ob((size_t)n_qubits, 0);
    int nfree = 0;
    for (int q = 0; q < n_qubits; q++) {
        ob[(size_t)q] = bits[q] & 1;
        if (!((mask >> q) & 1)) { flags[(size_t)q] = 1; nfree++; }
    }
    if (nfree > 30) return ZXP_ETOOBIG;   // 2^nfree amplitudes
    zxp_pscalar* p = nullptr;
    int st = zxp_compile_param(gates, n_gates, n_qubits, in_bits, ob.data(), flags.data(), 0,
                               ZXP_AMPLITUDE, &p);
    if (st != ZXP_OK) return st;
    zxp_server* srv = nullptr;
    zxp_server_opts opts;
    memset(&opts, 0, sizeof opts);
    opts.max_k = 62;
    st = zxp_server_create(ctx, &opts, &srv);
    if (st != ZXP_OK) { zxp_pscalar_free(p); return st; }
    const uint64_t count = 1ull << nfree;
    std::vector<uint64_t> tickets(count);
    for (uint64_t b = 0; b < count && st == ZXP_OK; b++) st = zxp_server_submit_bind(srv, p, b, &tickets[b]);
    // sum |a|^2 = a conj(a) exactly: conj maps w^j to w^-j
    __int128 acc[4] = {0, 0, 0, 0};
    int32_t e_acc = -1;
    for (uint64_t b = 0; b < count && st == ZXP_OK; b++) {
        zxp_zomega a;
        st = zxp_server_poll(srv, tickets[b], -1, &a, nullptr);
        if (st != ZXP_OK) break;
        // a conj(a) in the basis {1, w, w^2, w^3} (w^4 = -1), over sqrt2^(2 e)
        const __int128 c0 = a.c[0], c1 = a.c[1], c2 = a.c[2], c3 = a.c[3];
        __int128 r[4];
        r[0] = c0 * c0 + c1 * c1 + c2 * c2 + c3 * c3;
        r[1] = c1 * c0 + c2 * c1 + c3 * c2 - c0 * c3;
        r[2] = c2 * c0 + c3 * c1 - c0 * c2 - c1 * c3;
        r[3] = c3 * c0 - c0 * c1 - c1 * c2 - c2 * c3;
        int32_t e = 2 * a.e;
        if (!(c0 | c1 | c2 | c3)) continue;
        // bring to a common exponent (x sqrt2 per step)
        auto mul_sqrt2 = [](__int128 v[4]) {
            __int128 n0 = v[1] - v[3], n1 = v[0] + v[2], n2 = v[1] + v[3], n3 = v[2] - v[0];
            v[0] = n0; v[1] = n1; v[2] = n2; v[3] = n3;
        };
        if (e_acc < 0) { e_acc = e; for (int i = 0; i < 4; i++) acc[i] = r[i]; continue; }
        while (e_acc < e) { mul_sqrt2(acc); e_acc++; }
        while (e < e_acc) { mul_sqrt2(r); e++; }
        for (int i = 0; i < 4; i++) acc[i] += r[i];
    }
    zxp_server_destroy(srv);
    zxp_pscalar_free(p);
    if (st != ZXP_OK) return st;
    zxp_zomega raw;
    for (int i = 0; i < 4; i++) {
        if (acc[i] > (__int128)INT64_MAX || acc[i] < (__int128)INT64_MIN) return ZXP_EOVERFLOW;
        raw.c[i] = (int64_t)acc[i];
    }
    raw.e = e_acc < 0 ? 0 : e_acc;
    raw.flags = 0;
    return zxp_zomega_canon(&raw, out);
}

}  // extern "C"
