// plan.cpp -- rewrite a parametric scalar into the kernel's per-term tables.
#include "plan.h"

#include <string.h>

#include <algorithm>
#include <vector>

#include "zxp.h"

namespace zxp {

namespace {

zw64 from_i64(const int64_t G[4]) {
    return zw_make((uint64_t)G[0], (uint64_t)G[1], (uint64_t)G[2], (uint64_t)G[3]);
}

// 1 + w^a + w^b - w^(a+b): the phase-pair value of Eq. 3 for fixed phases
zw64 pair_value(unsigned a, unsigned b) {
    return zw_sub(zw_add(zw_add(zw_one(), zw_wpow(a)), zw_wpow(b)), zw_wpow(a + b));
}

struct Form {
    uint64_t mask;
    uint32_t inv;
};

int build_split_plan(const PS& ps, Plan* out);

// allow_lut: the block lookup may be built; lane_only: only with
// lane-private counters (the outer rows of a scalar with inner parameters,
// whose walk folds each lane's counters by itself).
int build_plain_plan(const PS& ps, bool allow_lut, bool lane_only, Plan* out) {
    Plan pl;
    memset(&pl.kp, 0, sizeof pl.kp);
    KernelParams& kp = pl.kp;
    kp.zq_lo = 64;
    const uint32_t k = ps.k;
    if (k > (uint32_t)kMaxK) return ZXP_ETOOBIG;
    kp.k = k;
    zw64 K = from_i64(ps.G);
    zw128 Kw = zw_widen(K);   // the same constant modulo 2^128
    bool exact_zero = !(ps.G[0] | ps.G[1] | ps.G[2] | ps.G[3]);

    // quadratic rows -> symmetric adjacency (+ 4 x_i on the diagonal); the
    // linear coefficients are collected as (mask, c) terms and merged by
    // mask (mod 8) once every row has contributed
    std::vector<std::pair<uint64_t, uint32_t>> lin_terms;
    lin_terms.reserve(ps.lin.size() + ps.node.size() + k);
    uint64_t adj[kMaxK] = {0};
    const uint64_t kmask = k >= 64 ? ~0ull : (1ull << k) - 1;
    for (const QuadRow& q : ps.quad) {
        if (!q.a || !q.b) continue;     // 4 * 0 * l = 0
        // row i gains b for every i in a and a for every i in b (bit i itself
        // is cleared below); i in a & b also gives 4 x_i
        for (uint64_t m = q.a & kmask; m; m &= m - 1) adj[__builtin_ctzll(m)] ^= q.b;
        for (uint64_t m = q.b & kmask; m; m &= m - 1) adj[__builtin_ctzll(m)] ^= q.a;
        for (uint64_t m = q.a & q.b & kmask; m; m &= m - 1) lin_terms.push_back({m & (0 - m), 4u});
    }
    for (uint32_t i = 0; i < k; i++) adj[i] &= ~(1ull << i);
    for (const LinRow& l : ps.lin)
        if (l.mask) lin_terms.push_back({l.mask, l.c & 7u});

    // nodes
    std::vector<Form> odd, zero;
    std::vector<uint8_t> odd_b;
    uint32_t nB = 0;
    for (const NodeRow& n : ps.node) {
        unsigned g = n.g & 7;
        if (!n.mask) {
            if (g == 4) exact_zero = true;
            K = zw_mul(K, zw_add(zw_one(), zw_wpow(g)));
            Kw = zw_mul(Kw, zw_widen(zw_add(zw_one(), zw_wpow(g))));
            continue;
        }
        if (g == 2 || g == 6) {        // 1 + w^(2+4l) = sqrt2 w w^(6l); 1 + w^(6+4l) = sqrt2 w^7 w^(2l)
            K = zw_rot(zw_mul_sqrt2(K), g == 2 ? 1 : 7);
            Kw = zw_rot(zw_mul_sqrt2(Kw), g == 2 ? 1 : 7);
            lin_terms.push_back({n.mask, g == 2 ? 6u : 2u});
        } else if (g == 0 || g == 4) { // 2 when the effective exponent is 0, else 0
            K = zw_add(K, K);
            Kw = zw_add(Kw, Kw);
            zero.push_back(Form{n.mask, g == 4 ? 1u : 0u});
        } else {                       // odd: bit set <=> effective exponent in {1, 7}
            odd.push_back(Form{n.mask, (g == 1 || g == 7) ? 1u : 0u});
            odd_b.push_back((g == 3 || g == 7) ? 1 : 0);
            nB += (g == 3 || g == 7);
        }
    }
    // pairs
    std::vector<uint64_t> pair_masks;
    for (const PairRow& p : ps.pair) {
        if (!p.ma && !p.mb) {
            zw64 v = pair_value(p.a, p.b);
            if (!(v.c[0] | v.c[1] | v.c[2] | v.c[3])) exact_zero = true;
            K = zw_mul(K, v);
            Kw = zw_mul(Kw, zw_widen(v));
            continue;
        }
        if (pl.pv.size() / 4 >= (size_t)kMaxPairs) return ZXP_ETOOBIG;
        for (unsigned b = 0; b < 4; b++)
            pl.pv.push_back(pair_value(p.a + 4 * (b & 1), p.b + 4 * (b >> 1)));
        pair_masks.push_back(p.ma);
        pair_masks.push_back(p.mb);
    }
    kp.npairs = (uint32_t)(pair_masks.size() / 2);

    // every odd node: (1 - w) w^j (1 + sqrt2)^beta; class B contributes w^3
    pl.m_odd = (uint32_t)odd.size();
    K = zw_mul(K, zw_pow(zw_make(1, (uint64_t)-1, 0, 0), pl.m_odd));
    K = zw_rot(K, 3 * nB);
    Kw = zw_mul(Kw, zw_pow(zw_widen(zw_make(1, (uint64_t)-1, 0, 0)), pl.m_odd));
    Kw = zw_rot(Kw, 3 * nB);

    // layout
    // linear forms in ascending mask order, coefficients summed mod 8, zero
    // coefficients dropped
    auto merge = [](std::vector<std::pair<uint64_t, uint32_t>>& terms) {
        std::vector<std::pair<uint64_t, uint32_t>> out;
        std::sort(terms.begin(), terms.end(),
                  [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) {
                      return x.first < y.first;
                  });
        for (size_t i = 0; i < terms.size();) {
            uint32_t c = 0;
            size_t j = i;
            for (; j < terms.size() && terms[j].first == terms[i].first; j++) c += terms[j].second;
            if (c & 7) out.push_back({terms[i].first, c & 7});
            i = j;
        }
        return out;
    };
    std::vector<std::pair<uint64_t, uint32_t>> lins = merge(lin_terms);
    // An even coefficient on a parity of several variables is a Clifford
    // phase that needs no form bit: c (x_1 ^ .. ^ x_m) = c sum_i x_i
    // + 4 sum_{i<j} x_i x_j (mod 8) for c = 2 mod 4, and 4 sum_i x_i for
    // c = 4 -- singletons, which merge into one form per variable, and
    // quadratic terms, which the adjacency rows carry.
    {
        std::vector<std::pair<uint64_t, uint32_t>> t2;
        bool expanded = false;
        for (auto& e : lins) {
            if ((e.second & 1) || __builtin_popcountll(e.first) < 2) { t2.push_back(e); continue; }
            expanded = true;
            for (uint64_t m = e.first; m; m &= m - 1) t2.push_back({m & (0 - m), e.second});
            if ((e.second & 3) == 2)
                for (uint64_t m = e.first; m; m &= m - 1) adj[__builtin_ctzll(m)] ^= e.first & ~(m & (0 - m));
        }
        if (expanded) lins = merge(t2);
    }
    // block lookup candidates: no phase-pair or zero forms (their bits would
    // vary inside a block); forms holding variable 0, 1 or 2 go first
    const uint64_t low3 = 7;
    // (phase-pair and zero forms may not hold variables 0-2: their bits are
    // then constant inside a block and select the block's counter plane)
    bool lut_try = allow_lut && k >= 3 && pair_masks.size() <= 2 * (size_t)kFoldPairs;
    for (uint64_t m : pair_masks) lut_try = lut_try && !(m & 7);
    for (auto& z : zero) lut_try = lut_try && !(z.mask & 7);
    uint32_t lut_nn = 0, lut_no = 0, lut_na = 0;
    bool lut_two = false;
    if (lut_try) {
        std::vector<Form> o2;
        std::vector<uint8_t> b2;
        for (int pass = 0; pass < 2; pass++)
            for (size_t j = 0; j < odd.size(); j++)
                if (((odd[j].mask & low3) != 0) == (pass == 0)) { o2.push_back(odd[j]); b2.push_back(odd_b[j]); }
        odd.swap(o2);
        odd_b.swap(b2);
        std::stable_partition(lins.begin(), lins.end(),
                              [&](const std::pair<uint64_t, uint32_t>& e) { return (e.first & low3) != 0; });
        for (auto& f : odd) lut_nn += (f.mask & low3) ? 1 : 0;
        for (auto& e : lins) lut_no += (e.first & low3) ? 1 : 0;
        const uint32_t stride = (uint32_t)odd.size() + 1;
        const uint32_t planes = (1u << (uint32_t)pair_masks.size()) << (zero.empty() ? 0 : 1);
        const uint32_t nU = lut_nn + lut_no;
        const bool lane = pair_masks.empty() && zero.empty() && odd.size() + 1 <= (1u << kLaneRowShift);
        const bool one = nU <= (uint32_t)kLutMaxBits && 11 * stride + 2 * lut_nn <= 255 &&
                         (uint32_t)kLutRows * stride * planes <= 2048;
        // more forms than one table takes: two tables, lane-private counters
        lut_two = lane && nU > (uint32_t)kLutMaxBits && nU <= (uint32_t)kLut2MaxBits && lut_no <= 32;
        lut_na = lut_two ? (nU + 1) / 2 : nU;
        lut_try = (one && (lane || !lane_only)) || lut_two;
    }
    // lookup slot of the lookup-index bits u (linear forms, then node forms)
    auto slot_of = [&](uint32_t u) {
        return lut_two ? (lut_slot(u & ((1u << lut_na) - 1u)) | (lut_slot(u >> lut_na) << lut_na)) : lut_slot(u);
    };
    size_t n_other = lins.size() + zero.size() + pair_masks.size();
    pl.nwn = (int)((odd.size() + 31) / 32);
    pl.nwl = (int)((n_other + 31) / 32);
    if (pl.nwn > kMaxWordsNode || pl.nwl > kMaxWordsOther) return ZXP_ETOOBIG;
    kp.nbits = 32u * (uint32_t)(pl.nwn + pl.nwl);
    const uint32_t nw = (uint32_t)(pl.nwn + (pl.nwl < 1 ? 1 : pl.nwl));   // kernel words
    pl.frows.assign((size_t)k * nw, 0u);
    auto put = [&](uint32_t bit, uint64_t mask, uint32_t inv) {
        if (inv) kp.INV[bit >> 5] |= 1u << (bit & 31);
        for (uint64_t m = mask & kmask; m; m &= m - 1)
            pl.frows[(size_t)__builtin_ctzll(m) * nw + (bit >> 5)] |= 1u << (bit & 31);
    };
    for (size_t j = 0; j < odd.size(); j++) {
        uint32_t bit = (uint32_t)j;
        put(bit, odd[j].mask, odd[j].inv);
        if (odd_b[j]) kp.CB[bit >> 5] |= 1u << (bit & 31);
    }
    uint32_t base = 32u * (uint32_t)pl.nwn, pos = 0;
    // phase-pair forms first (bits 0.. of the first other word), so that up
    // to kFoldPairs of them index the term table directly
    for (size_t j = 0; j < pair_masks.size(); j++) {
        uint32_t bit = base + pos++;
        put(bit, pair_masks[j], 0);
        if (j & 1) kp.PB[j / 2] = (uint16_t)bit; else kp.PA[j / 2] = (uint16_t)bit;
    }
    for (auto& e : lins) {
        uint32_t bit = base + pos++;
        put(bit, e.first, 0);
        uint32_t w = (bit - base) >> 5, b = 1u << (bit & 31);
        if (e.second & 1) kp.C0[w] |= b;
        if (e.second & 2) kp.C1[w] |= b;
        if (e.second & 4) kp.C2[w] |= b;
    }
    for (auto& z : zero) {
        uint32_t bit = base + pos++;
        put(bit, z.mask, z.inv);
        kp.Z[(bit - base) >> 5] |= 1u << (bit & 31);
    }
    pl.adj.assign(adj, adj + k);
    for (uint32_t i = 0; i < 4 && i < k; i++) kp.A4[i] = adj[i];
    // seek tables (stride padded to a multiple of 4 words for vector loads)
    pl.seek_stride = (nw + 3 + 3) & ~3u;
    const uint32_t nnib = (k + 3) / 4;
    pl.seek.assign((size_t)nnib * 16 * pl.seek_stride, 0u);
    // entry v is entry v' = v without its lowest bit i, plus variable 4b+i:
    // its flip row, its adjacency row, and the quadratic bits of the pairs
    // (i, j) with j in v' (every bit of v' is above i)
    for (uint32_t b = 0; b < nnib; b++)
        for (uint32_t v = 1; v < 16; v++) {
            const uint32_t i = (uint32_t)__builtin_ctz(v), vp = v & (v - 1), var = 4 * b + i;
            uint32_t* e = &pl.seek[((size_t)b * 16 + v) * pl.seek_stride];
            const uint32_t* ep = &pl.seek[((size_t)b * 16 + vp) * pl.seek_stride];
            for (uint32_t w = 0; w < nw + 3; w++) e[w] = ep[w];
            if (var >= k) continue;
            for (uint32_t w = 0; w < nw; w++) e[w] ^= pl.frows[(size_t)var * nw + w];
            const uint64_t a = adj[var];
            e[nw] ^= (uint32_t)a;
            e[nw + 1] ^= (uint32_t)(a >> 32);
            e[nw + 2] ^= (uint32_t)__builtin_popcount((uint32_t)(a >> (4 * b)) & vp & 15u) & 1u;
        }

    // step rows (the lowest four also in the kernel parameters, zero rows
    // for variables beyond k)
    {
        const int nwl_k = pl.nwl < 1 ? 1 : pl.nwl;
        const uint32_t rw = row_words(pl.nwn, nwl_k);
        pl.row_stride = rw;
        pl.rows.assign((size_t)k * rw, 0u);
        for (uint32_t i = 0; i < k; i++) {
            uint32_t* r = &pl.rows[(size_t)i * rw];
            uint32_t S = 0;
            for (uint32_t w = 0; w < nw; w++) {
                const uint32_t f = pl.frows[(size_t)i * nw + w];
                r[w] = f;
                if ((int)w < pl.nwn) {
                    S += 4u * (uint32_t)__builtin_popcount(f & kp.CB[w]);
                } else {
                    const uint32_t o = w - (uint32_t)pl.nwn;
                    r[nw + o] = f & kp.C0[o];
                    r[nw + nwl_k + o] = f & kp.C1[o];
                    S += (uint32_t)__builtin_popcount(f & kp.C0[o]) + 2u * (uint32_t)__builtin_popcount(f & kp.C1[o]) +
                         4u * (uint32_t)__builtin_popcount(f & kp.C2[o]);
                }
            }
            uint32_t du = 0;
            if (lut_try) {
                const uint32_t fo_i = (r[pl.nwn] >> pair_masks.size()) & ((1u << lut_no) - 1u);
                const uint32_t fn_i = pl.nwn ? (r[0] & ((1u << lut_nn) - 1u)) : 0u;
                du = slot_of((fn_i << lut_no) | fo_i);
            }
            r[nw + 2 * nwl_k] = (S & 7u) | (du << 8);
            if (i < 4) kp.U4[i] = du;
        }
        for (uint32_t i = 0; i < 4 && i < k; i++)
            for (uint32_t w = 0; w < rw; w++) kp.R[i][w] = pl.rows[(size_t)i * rw + w];
    }

    // block lookup (see plan.h)
    if (lut_try) {
        // lane-private counters: one row of 2^kLaneRowShift >= m_odd + 1
        // counters per phase exponent mod 8
        const uint32_t tsh = kLaneRowShift;
        pl.lut_lane = pair_masks.empty() && zero.empty() && pl.m_odd + 1 <= (1u << tsh);
        kp.lut_tsh = pl.lut_lane ? tsh : 0u;
        kp.lane_row_bytes = 32u * 4u;
        const uint32_t nU = lut_nn + lut_no, stride = pl.lut_lane ? (1u << tsh) : pl.m_odd + 1;
        const uint32_t mo = (1u << lut_no) - 1, mn = (1u << lut_nn) - 1;
        const int nwn_k = pl.nwn;
        uint32_t fo[3], fn[3];
        for (int i = 0; i < 3; i++) {
            fo[i] = (pl.frows[(size_t)i * nw + (uint32_t)nwn_k] >> pair_masks.size()) & mo;
            fn[i] = nwn_k ? (pl.frows[(size_t)i * nw] & mn) : 0u;
        }
        static const int seq[7] = {0, 1, 0, 2, 0, 1, 0};
        // Flipping variable i changes J by sum_{r in F_i} c_r (1 - 2 l_r) + 4
        // per class-B node bit it flips, and M by the sum over its node bits of
        // (1 - 2 l_r).  Each form's share of the change after steps 1..s
        // depends only on its own bit at the block's first state, so an entry
        // is a sum of per-form byte vectors (byte s-1: the share after step
        // s; the phase shares taken mod 8, every byte sum below 256), built
        // for all first states in Gray-code order, one vector update each.
        auto share = [&](uint32_t r, const uint32_t* f, int weight, uint32_t b, int bias, bool mod8) {
            uint32_t bit = b;
            int acc = 0;
            uint64_t v = 0;
            for (int s = 1; s <= 7; s++) {
                if ((f[seq[s - 1]] >> r) & 1) {
                    acc += weight * (1 - 2 * (int)bit);
                    bit ^= 1u;
                }
                v |= (uint64_t)(uint32_t)(mod8 ? (acc & 7) : acc + bias) << (8 * (s - 1));
            }
            return v;
        };
        auto gray_fill = [](uint32_t n, uint64_t s0, const uint64_t* d, std::vector<uint64_t>& out,
                            auto finish) {
            out.assign((size_t)1 << n, 0);
            uint64_t sum = s0;
            uint32_t x = 0;
            out[0] = finish(sum);
            for (uint32_t g = 1; g < (1u << n); g++) {
                const uint32_t r = (uint32_t)__builtin_ctz(g);
                x ^= 1u << r;
                sum += ((x >> r) & 1) ? d[r] : (uint64_t)0 - d[r];
                out[x] = finish(sum);
            }
        };
        uint32_t nb_mask = 0;
        for (uint32_t r = 0; r < lut_nn; r++) nb_mask |= (uint32_t)odd_b[r] << r;
        kp.lut_no = lut_no;
        kp.lut_nn = lut_nn;
        kp.lut_shift = (uint32_t)pair_masks.size();   // linear forms follow the pair bits
        pl.lut_two = lut_two;
        kp.lut_na = lut_two ? lut_na : 0u;
        // the 8 quadratic entries, indexed by the bits of A x on variables 0-2
        uint64_t qent[8];
        for (uint32_t h = 0; h < 8; h++) {
            uint32_t a = h, Q = 0;
            uint64_t e = 0;
            for (int s = 1; s <= 7; s++) {
                const int i = seq[s - 1];
                Q ^= (a >> i) & 1u;
                a ^= (uint32_t)(adj[i] & low3);
                if (s < 7) e |= (uint64_t)(4 * Q * stride) << (8 * (s - 1));
                else e |= ((uint64_t)(4 * Q * stride) << 48) | ((uint64_t)(4 * Q) << 56);
            }
            qent[h] = e;
        }
        if (lut_two) {
            // Two tables over the first lut_na lookup bits and the rest.  An
            // entry is the sum of its forms' shares as integers per byte:
            // bytes 0-6 the counter offset after step s, (dJ_s mod 8) * 2^tsh
            // + dM_s, taken mod 8 * 2^tsh; byte 7 the block's phase change
            // mod 8.  The class-B nodes' phase change (the same for every
            // entry) goes into the first table.  The kernel adds the two
            // entries, the quadratic entry and the block's base: every byte
            // stays below 256.
            auto steps = [&](uint32_t r, const uint32_t* f, uint32_t b, int acc[7]) {
                uint32_t bit = b;
                int a = 0;
                for (int st = 1; st <= 7; st++) {
                    if ((f[seq[st - 1]] >> r) & 1) {
                        a += 1 - 2 * (int)bit;
                        bit ^= 1u;
                    }
                    acc[st - 1] = a;
                }
            };
            const int m8 = 8 << tsh;
            auto add_phase = [&](int v[8], const int acc[7], int c) {
                for (int st = 0; st < 7; st++) v[st] += (((c * acc[st]) % 8 + 8) % 8) * (1 << tsh);
                v[7] += ((c * acc[6]) % 8 + 8) % 8;
            };
            int cst[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            {
                int acc[7], a = 0;
                for (int st = 1; st <= 7; st++) {
                    a += 4 * __builtin_popcount(fn[seq[st - 1]] & nb_mask);
                    acc[st - 1] = a;
                }
                add_phase(cst, acc, 1);
            }
            // shares of lookup bit r for bit value b
            auto form_bytes = [&](uint32_t r, uint32_t b, int v[8]) {
                int acc[7];
                if (r < lut_no) {
                    steps(r, fo, b, acc);
                    add_phase(v, acc, (int)lins[r].second);
                } else {
                    steps(r - lut_no, fn, b, acc);
                    for (int st = 0; st < 7; st++) v[st] += acc[st];
                }
            };
            const uint32_t nb = nU - lut_na;
            pl.lut.assign(((size_t)1 << lut_na) + ((size_t)1 << nb) + 8, 0ull);
            for (int t = 0; t < 2; t++) {
                const uint32_t lo = t ? lut_na : 0u, n = t ? nb : lut_na;
                uint64_t* tab = pl.lut.data() + (t ? ((size_t)1 << lut_na) : 0);
                for (uint32_t u = 0; u < (1u << n); u++) {
                    int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (!t) for (int j = 0; j < 8; j++) v[j] = cst[j];
                    for (uint32_t j = 0; j < n; j++) form_bytes(lo + j, (u >> j) & 1u, v);
                    uint64_t e = 0;
                    for (int j = 0; j < 7; j++) e |= (uint64_t)(((v[j] % m8) + m8) % m8) << (8 * j);
                    e |= (uint64_t)(((v[7] % 8) + 8) % 8) << 56;
                    tab[lut_slot(u)] = e;
                }
            }
            for (uint32_t h = 0; h < 8; h++) pl.lut[((size_t)1 << lut_na) + ((size_t)1 << nb) + h] = qent[h];
            kp.lut_entries = (uint32_t)pl.lut.size();
            pl.lut_ok = true;
        } else {
            // linear part: bytes 0..6 hold (dJ_s mod 8) * stride, byte 7 dJ_7 mod 8
            uint64_t so = 0, dout[kLutMaxBits], dnod[kLutMaxBits];
            {
                int acc = 0;   // class-B node bits: 4 per flip, whatever their state
                for (int s = 1; s <= 7; s++) {
                    acc += 4 * __builtin_popcount(fn[seq[s - 1]] & nb_mask);
                    so |= (uint64_t)(uint32_t)(acc & 7) << (8 * (s - 1));
                }
            }
            for (uint32_t r = 0; r < lut_no; r++) {
                const int c = (int)lins[r].second;
                const uint64_t p0 = share(r, fo, c, 0, 0, true), p1 = share(r, fo, c, 1, 0, true);
                so += p0;
                dout[r] = p1 - p0;
            }
            const uint64_t st = stride;
            std::vector<uint64_t> eo, en;
            gray_fill(lut_no, so, dout, eo, [st](uint64_t x) {
                x &= 0x0007070707070707ull;
                return x * st | ((x >> 48) << 56);
            });
            // node part: bytes 0..6 hold dM_s + lut_nn (each form's share + 1)
            uint64_t sn = 0;
            for (uint32_t r = 0; r < lut_nn; r++) {
                const uint64_t q0 = share(r, fn, 1, 0, 1, false), q1 = share(r, fn, 1, 1, 1, false);
                sn += q0;
                dnod[r] = q1 - q0;
            }
            gray_fill(lut_nn, sn, dnod, en, [](uint64_t x) { return x; });
            pl.lut.assign(((size_t)1 << nU) + 8, 0ull);
            // lane-private counters: offsets taken mod 8 * 2^tsh with the bias
            // lut_nn removed (the kernel adds the block's base and masks)
            const uint64_t b7 = 0x0001010101010101ull, cm = (8ull << tsh) - 1;
            for (uint32_t Ln = 0; Ln < (1u << lut_nn); Ln++)
                for (uint32_t Lo = 0; Lo < (1u << lut_no); Lo++) {
                    uint64_t e = eo[Lo] + en[Ln];
                    if (pl.lut_lane) e = ((e + (cm + 1 - lut_nn) * b7) & (cm * b7)) | (e & ~(0xFFull * b7));
                    pl.lut[lut_slot((Ln << lut_no) | Lo)] = e;
                }
            for (uint32_t h = 0; h < 8; h++) pl.lut[((size_t)1 << nU) + h] = qent[h];
            kp.lut_entries = (uint32_t)pl.lut.size();
            pl.lut_ok = true;
        }
    }

    // T[J][M][pair bits][zero] = w^(J + 2M) (1 + sqrt2)^M * prod_j PV_j(bits_j) * [not zero]
    const uint32_t np = kp.npairs;
    pl.general = np > (uint32_t)kFoldPairs;
    const uint32_t pbits = pl.general ? 0 : 2 * np;
    const uint32_t zbit = (!pl.general && !zero.empty()) ? 1 : 0;
    kp.has_zero = zero.empty() ? 0 : 1;
    kp.xshift = pbits + zbit;
    kp.pmask = (1u << pbits) - 1;
    kp.zshift = pbits;
    kp.tab_stride = pl.m_odd + 1;
    kp.tab_size = (8u * kp.tab_stride) << kp.xshift;
    pl.table.assign(kp.tab_size, zw_zero());
    zw64 s = zw_one();
    for (uint32_t M = 0; M <= pl.m_odd; M++) {
        for (unsigned J = 0; J < 8; J++) {
            const zw64 base_v = zw_rot(s, J + 2 * M);
            for (uint32_t x = 0; x < (1u << kp.xshift); x++) {
                zw64 v = base_v;
                if (zbit && ((x >> pbits) & 1)) v = zw_zero();
                for (uint32_t j = 0; j < pbits / 2; j++) v = zw_mul(v, pl.pv[4 * j + ((x >> (2 * j)) & 3)]);
                pl.table[((J * kp.tab_stride + M) << kp.xshift) | x] = v;
            }
        }
        s = zw_mul(s, zw_silver());
    }
    // modulo 2^128: (J, M) values only (the pair values are small, so their
    // 64-bit words widen exactly)
    pl.table_w.assign((size_t)8 * kp.tab_stride, zw_zero<u128>());
    zw128 sw = zw_one<u128>();
    for (uint32_t M = 0; M <= pl.m_odd; M++) {
        for (unsigned J = 0; J < 8; J++) pl.table_w[(size_t)J * kp.tab_stride + M] = zw_rot(sw, J + 2 * M);
        sw = zw_mul(sw, zw_widen(zw_silver()));
    }
    pl.pv_w.clear();
    for (const zw64& v : pl.pv) pl.pv_w.push_back(zw_widen(v));
    pl.K_w = Kw;
    pl.K = K;
    pl.e0 = ps.e0;
    pl.zero = exact_zero;
    pl.has_zero = !zero.empty();
    *out = std::move(pl);
    return ZXP_OK;
}

// A scalar with inner parameters (the last k_inner bits of every mask):
// every row is split by its masks' inner and outer parts.
//   * rows on outer bits only stay outer rows;
//   * rows on inner bits only become rows of the inner product g(u);
//   * the Clifford coupling of the two groups is bilinear: a quadratic row
//     4 (aI ^ aO)(bI ^ bO) = 4 aI bI + 4 aI bO + 4 aO bI + 4 aO bO (mod 8), an
//     even linear row c (lI ^ lO) = c lI + c lO (+ 4 lI lO when c = 2 mod 4);
//     its cut terms 4 x_i . z_i(x_O) are the Walsh-Hadamard kernel, z_i the
//     XOR of the outer forms paired with inner variable i;
//   * a non-Clifford row (odd linear phase, node, phase-pair) on both groups
//     keeps its inner form and gains one cut bit q_j = its outer form
//     (identical outer forms share a bit): it becomes a row of g over
//     u = (x_I, q).
// The inner table is then F[z | q << k_inner] = sum over x_I of
// g(x_I, q) (-1)^(x_I . z), and the scalar's value is
//   K_outer sum_{x_O} T_outer(x_O) F[z(x_O) | q(x_O) << k_inner].
int build_split_plan(const PS& ps, Plan* out) {
    const uint32_t k = ps.k, ki = ps.k_inner;
    if (ki == 0 || ki > k) return ZXP_EINVAL;
    const uint32_t ko = k - ki;
    const uint64_t om = ko ? ((1ull << ko) - 1) : 0ull;
    PS outer, inner;
    outer.k = ko;
    outer.e0 = ps.e0;
    for (int i = 0; i < 4; i++) outer.G[i] = ps.G[i];
    outer.t_count = ps.t_count;
    std::vector<uint64_t> z(ki, 0ull), q;
    auto in_part = [&](uint64_t m) { return m >> ko; };
    auto qbit = [&](uint64_t mo) -> uint64_t {
        size_t j = 0;
        while (j < q.size() && q[j] != mo) j++;
        if (j == q.size()) q.push_back(mo);
        return 1ull << (ki + j);
    };
    auto cut = [&](uint64_t inner_mask, uint64_t outer_mask) {
        for (uint64_t m = inner_mask; m; m &= m - 1) z[(size_t)__builtin_ctzll(m)] ^= outer_mask;
    };
    for (const LinRow& r : ps.lin) {
        const uint64_t mi = in_part(r.mask), mo = r.mask & om;
        if (!mi) { outer.lin.push_back(r); continue; }
        if (!mo) { inner.lin.push_back({mi, r.c}); continue; }
        if (r.c & 1) { inner.lin.push_back({mi | qbit(mo), r.c}); continue; }
        inner.lin.push_back({mi, r.c});
        outer.lin.push_back({mo, r.c});
        if ((r.c & 3) == 2) cut(mi, mo);
    }
    for (const QuadRow& r : ps.quad) {
        const uint64_t ai = in_part(r.a), ao = r.a & om, bi = in_part(r.b), bo = r.b & om;
        if (ai && bi) inner.quad.push_back({ai, bi});
        if (ao && bo) outer.quad.push_back({ao, bo});
        cut(ai, bo);
        cut(bi, ao);
    }
    for (const NodeRow& r : ps.node) {
        const uint64_t mi = in_part(r.mask), mo = r.mask & om;
        if (!mi) outer.node.push_back(r);
        else inner.node.push_back({mi | (mo ? qbit(mo) : 0ull), r.g});
    }
    for (const PairRow& r : ps.pair) {
        if (!in_part(r.ma | r.mb)) { outer.pair.push_back(r); continue; }
        const uint64_t ma = in_part(r.ma) | ((r.ma & om) ? qbit(r.ma & om) : 0ull);
        const uint64_t mb = in_part(r.mb) | ((r.mb & om) ? qbit(r.mb & om) : 0ull);
        inner.pair.push_back({ma, mb, r.a, r.b});
    }
    const uint32_t bits = ki + (uint32_t)q.size();
    if (bits > kMaxInnerBits) return ZXP_ETOOBIG;
    inner.k = bits;
    std::vector<uint32_t> zqcol(ko, 0u);
    for (uint32_t j = 0; j < ki; j++)
        for (uint64_t m = z[j]; m; m &= m - 1) zqcol[(size_t)__builtin_ctzll(m)] ^= 1u << j;
    for (size_t j = 0; j < q.size(); j++)
        for (uint64_t m = q[j]; m; m &= m - 1) zqcol[(size_t)__builtin_ctzll(m)] ^= 1u << (ki + j);
    uint32_t lo = 64;
    for (uint32_t i = 0; i < ko; i++)
        if (zqcol[i]) { lo = i; break; }
    // the walk's unrolled steps flip variables 0-3 without looking at zq
    if (lo < 4) return ZXP_EINVAL;
    auto ip = std::make_shared<Plan>();
    int st = build_plain_plan(inner, false, false, ip.get());
    if (st != ZXP_OK) return st;
    // the inner constant into the inner table, so that an entry is one
    // table value (times phase-pair values beyond the folded ones)
    for (zw64& t : ip->table) t = zw_mul(ip->K, t);
    ip->K = zw_one();
    for (zw128& t : ip->table_w) t = zw_mul(ip->K_w, t);
    ip->K_w = zw_one<u128>();
    // the low bits' flip-row XOR and quadratic bit, per value
    const uint32_t tb = bits < kInnerLowBits ? bits : kInnerLowBits;
    const uint32_t inw = (uint32_t)(ip->nwn + (ip->nwl < 1 ? 1 : ip->nwl));
    std::vector<uint32_t> low((size_t)(inw + 1) << tb, 0u);
    for (uint32_t e = 1; e < (1u << tb); e++) {
        const uint32_t i = (uint32_t)__builtin_ctz(e), ep = e & (e - 1);
        uint32_t* r = &low[(size_t)e * (inw + 1)];
        const uint32_t* rp = &low[(size_t)ep * (inw + 1)];
        for (uint32_t w = 0; w < inw; w++) r[w] = rp[w] ^ ip->frows[(size_t)i * inw + w];
        // adding variable i (below every bit of ep) flips the quadratic bit
        // by its pairs with the bits of ep
        r[inw] = rp[inw] ^ ((uint32_t)__builtin_popcountll(ip->adj[i] & ep) & 1u);
    }
    Plan pl;
    if ((st = build_plain_plan(outer, true, true, &pl)) != ZXP_OK) return st;
    pl.kp.zq_lo = lo;
    pl.k_inner = ki;
    pl.inner_bits = bits;
    pl.zqcol = std::move(zqcol);
    pl.zero = pl.zero || ip->zero;
    pl.inner_low = std::move(low);
    pl.inner = std::move(ip);
    *out = std::move(pl);
    return ZXP_OK;
}

}  // namespace

int build_plan(const PS& ps, Plan* out) {
    if (ps.k_inner) return build_split_plan(ps, out);
    return build_plain_plan(ps, true, false, out);
}

}  // namespace zxp
