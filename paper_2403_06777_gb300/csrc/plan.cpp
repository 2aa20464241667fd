// plan.cpp -- rewrite a parametric scalar into the kernel's per-term tables.
#include "plan.h"

#include <string.h>

#include <algorithm>
#include <map>
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

}  // namespace

int build_plan(const PS& ps, Plan* out) {
    Plan pl;
    memset(&pl.kp, 0, sizeof pl.kp);
    KernelParams& kp = pl.kp;
    const uint32_t k = ps.k;
    if (k > (uint32_t)kMaxK) return ZXP_ETOOBIG;
    kp.k = k;
    zw64 K = from_i64(ps.G);
    bool exact_zero = !(ps.G[0] | ps.G[1] | ps.G[2] | ps.G[3]);

    // quadratic rows -> symmetric adjacency (+ 4 x_i on the diagonal)
    std::map<uint64_t, uint32_t> lin;   // mask -> coefficient (mod 8)
    uint64_t adj[kMaxK] = {0};
    for (const QuadRow& q : ps.quad) {
        if (!q.a || !q.b) continue;     // 4 * 0 * l = 0
        for (uint32_t i = 0; i < k; i++) {
            uint64_t r = (((q.a >> i) & 1) ? q.b : 0) ^ (((q.b >> i) & 1) ? q.a : 0);
            r &= ~(1ull << i);
            adj[i] ^= r;
            if (((q.a & q.b) >> i) & 1) lin[1ull << i] = (lin[1ull << i] + 4) & 7;
        }
    }
    for (const LinRow& l : ps.lin)
        if (l.mask) lin[l.mask] = (lin[l.mask] + l.c) & 7;

    // nodes
    std::vector<Form> odd, zero;
    std::vector<uint8_t> odd_b;
    uint32_t nB = 0;
    for (const NodeRow& n : ps.node) {
        unsigned g = n.g & 7;
        if (!n.mask) {
            if (g == 4) exact_zero = true;
            K = zw_mul(K, zw_add(zw_one(), zw_wpow(g)));
            continue;
        }
        if (g == 2 || g == 6) {        // 1 + w^(2+4l) = sqrt2 w w^(6l); 1 + w^(6+4l) = sqrt2 w^7 w^(2l)
            K = zw_rot(zw_mul_sqrt2(K), g == 2 ? 1 : 7);
            lin[n.mask] = (lin[n.mask] + (g == 2 ? 6 : 2)) & 7;
        } else if (g == 0 || g == 4) { // 2 when the effective exponent is 0, else 0
            K = zw_add(K, K);
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

    // layout
    std::vector<std::pair<uint64_t, uint32_t>> lins;
    for (auto& e : lin) if (e.second) lins.push_back(e);
    // block lookup candidates: no phase-pair or zero forms (their bits would
    // vary inside a block); forms holding variable 0, 1 or 2 go first
    const uint64_t low3 = 7;
    // (phase-pair and zero forms may not hold variables 0-2: their bits are
    // then constant inside a block and select the block's counter plane)
    bool lut_try = k >= 3 && pair_masks.size() <= 2 * (size_t)kFoldPairs;
    for (uint64_t m : pair_masks) lut_try = lut_try && !(m & 7);
    for (auto& z : zero) lut_try = lut_try && !(z.mask & 7);
    uint32_t lut_nn = 0, lut_no = 0;
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
        lut_try = lut_nn + lut_no <= (uint32_t)kLutMaxBits && 11 * stride + 2 * lut_nn <= 255 &&
                  (uint32_t)kLutRows * stride * planes <= 2048;
    }
    size_t n_other = lins.size() + zero.size() + pair_masks.size();
    pl.nwn = (int)((odd.size() + 31) / 32);
    pl.nwl = (int)((n_other + 31) / 32);
    if (pl.nwn > kMaxWordsNode || pl.nwl > kMaxWordsOther) return ZXP_ETOOBIG;
    kp.nbits = 32u * (uint32_t)(pl.nwn + pl.nwl);
    const uint32_t nw = (uint32_t)(pl.nwn + (pl.nwl < 1 ? 1 : pl.nwl));   // kernel words
    pl.frows.assign((size_t)k * nw, 0u);
    auto put = [&](uint32_t bit, uint64_t mask, uint32_t inv) {
        if (inv) kp.INV[bit >> 5] |= 1u << (bit & 31);
        for (uint32_t i = 0; i < k; i++)
            if ((mask >> i) & 1) pl.frows[(size_t)i * nw + (bit >> 5)] |= 1u << (bit & 31);
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
    for (uint32_t b = 0; b < nnib; b++)
        for (uint32_t v = 0; v < 16; v++) {
            uint32_t* e = &pl.seek[((size_t)b * 16 + v) * pl.seek_stride];
            uint64_t a = 0;
            uint32_t q = 0;
            for (uint32_t i = 0; i < 4; i++) {
                const uint32_t var = 4 * b + i;
                if (!((v >> i) & 1) || var >= k) continue;
                for (uint32_t w = 0; w < nw; w++) e[w] ^= pl.frows[(size_t)var * nw + w];
                for (uint32_t j = 0; j < i; j++)     // pairs inside the group
                    if (((v >> j) & 1) && ((adj[var] >> (4 * b + j)) & 1)) q ^= 1u;
                a ^= adj[var];
            }
            e[nw] = (uint32_t)a;
            e[nw + 1] = (uint32_t)(a >> 32);
            e[nw + 2] = q;
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
            r[nw + 2 * nwl_k] = S & 7u;
        }
        for (uint32_t i = 0; i < 4 && i < k; i++)
            for (uint32_t w = 0; w < rw; w++) kp.R[i][w] = pl.rows[(size_t)i * rw + w];
    }

    // block lookup (see plan.h)
    if (lut_try) {
        // lane-private counters: one row of 2^tsh >= m_odd + 1 counters per
        // phase exponent mod 8, at most kLaneCounters per lane
        uint32_t tsh = 0;
        while ((1u << tsh) < pl.m_odd + 1) tsh++;
        pl.lut_lane = pair_masks.empty() && zero.empty() && (8u << tsh) <= (uint32_t)kLaneCounters;
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
        // csum[v]: the sum of the coefficients of the linear forms in v;
        // flipping variable i changes J by sum_{r in F_i} c_r (1 - 2 l_r) + 4 per
        // class-B node bit it flips, and M by |F_i nodes| - 2 |F_i nodes & L|
        std::vector<int> csum((size_t)1 << lut_no, 0);
        for (uint32_t v = 1; v < (1u << lut_no); v++) {
            const uint32_t r = (uint32_t)__builtin_ctz(v);
            csum[v] = csum[v & (v - 1)] + (int)lins[r].second;
        }
        // node-bit counts by table (no popcount instruction needed on the host)
        std::vector<int> pcount((size_t)1 << lut_nn, 0);
        for (uint32_t v = 1; v < (1u << lut_nn); v++) pcount[v] = pcount[v & (v - 1)] + 1;
        uint32_t nb_mask = 0;
        for (uint32_t r = 0; r < lut_nn; r++) nb_mask |= (uint32_t)odd_b[r] << r;
        int sJ[3], sM[3];
        for (int i = 0; i < 3; i++) {
            sJ[i] = csum[fo[i]] + 4 * pcount[fn[i] & nb_mask];
            sM[i] = pcount[fn[i]];
        }
        // ΔJ depends on the linear bits only and ΔM on the node bits only, and
        // no byte of an entry carries into the next (each is at most 255), so
        // an entry is the sum of a linear-bit part and a node-bit part.
        std::vector<uint64_t> eo((size_t)1 << lut_no), en((size_t)1 << lut_nn);
        for (uint32_t Lo0 = 0; Lo0 < (1u << lut_no); Lo0++) {
            uint32_t Lo = Lo0;
            int dJ = 0;
            uint64_t e = 0;
            for (int s = 1; s <= 7; s++) {
                const int i = seq[s - 1];
                dJ += sJ[i] - 2 * csum[fo[i] & Lo];
                Lo ^= fo[i];
                const uint64_t j8 = (uint32_t)dJ & 7u;
                e |= (j8 * stride) << (8 * (s - 1));
                if (s == 7) e |= j8 << 56;
            }
            eo[Lo0] = e;
        }
        for (uint32_t Ln0 = 0; Ln0 < (1u << lut_nn); Ln0++) {
            uint32_t Ln = Ln0;
            int dM = 0;
            uint64_t e = 0;
            for (int s = 1; s <= 7; s++) {
                const int i = seq[s - 1];
                dM += sM[i] - 2 * pcount[fn[i] & Ln];
                Ln ^= fn[i];
                e |= (uint64_t)(uint32_t)(dM + (int)lut_nn) << (8 * (s - 1));
            }
            en[Ln0] = e;
        }
        pl.lut.assign(((size_t)1 << nU) + 8, 0ull);
        for (uint32_t Ln = 0; Ln < (1u << lut_nn); Ln++)
            for (uint32_t Lo = 0; Lo < (1u << lut_no); Lo++)
                pl.lut[lut_slot((Ln << lut_no) | Lo)] = eo[Lo] + en[Ln];
        for (uint32_t h = 0; h < 8; h++) {
            uint32_t a = h, Q = 0;
            uint64_t e = 0;
            for (int s = 1; s <= 7; s++) {
                const int i = seq[s - 1];
                Q ^= (a >> i) & 1u;
                a ^= (uint32_t)(adj[i] & low3);
                if (s < 7) e |= (uint64_t)(4 * Q * stride) << (8 * (s - 1));
                else e |= ((uint64_t)(4 * Q * stride) << 48) | ((uint64_t)((4 * Q) | (a << 5)) << 56);
            }
            pl.lut[((size_t)1 << nU) + h] = e;
        }
        kp.lut_no = lut_no;
        kp.lut_nn = lut_nn;
        kp.lut_shift = (uint32_t)pair_masks.size();   // linear forms follow the pair bits
        pl.lut_ok = true;
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
    pl.K = K;
    pl.e0 = ps.e0;
    pl.zero = exact_zero;
    pl.has_zero = !zero.empty();
    *out = std::move(pl);
    return ZXP_OK;
}

}  // namespace zxp
