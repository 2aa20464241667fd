// plan.cpp -- rewrite a parametric scalar into the kernel's per-term tables.
#include "plan.h"

#include <string.h>

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
    for (size_t j = 0; j < pair_masks.size(); j++) {
        uint32_t bit = base + pos++;
        put(bit, pair_masks[j], 0);
        if (j & 1) kp.PB[j / 2] = (uint16_t)bit; else kp.PA[j / 2] = (uint16_t)bit;
    }
    pl.adj.assign(adj, adj + k);

    // T[J][M] = w^(J + 2M) (1 + sqrt2)^M
    kp.tab_stride = pl.m_odd + 1;
    pl.table.assign(8 * (size_t)kp.tab_stride, zw_zero());
    zw64 s = zw_one();
    for (uint32_t M = 0; M <= pl.m_odd; M++) {
        for (unsigned J = 0; J < 8; J++) pl.table[J * kp.tab_stride + M] = zw_rot(s, J + 2 * M);
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
