// reorder.cpp -- relabelling a scalar's parameters (zxp_scalar_reorder).
//
// The sum over x in {0,1}^k (Eq. 2) does not depend on the order of the
// parameters, but the Gray-code walk does: parameters 0, 1 and 2 flip in
// every aligned block of 8 steps, and the block lookup that costs one
// table read per 8 terms applies only when few parity forms hold them and
// none of them is a phase-pair or zero-test form.  This moves to positions
// 0-2 the three parameters whose forms, together, are fewest (among the
// parameters that no phase-pair or zero-test form holds, where possible),
// then the next lightest parameter to position 3, keeping the others in
// their order; the new order is kept only when its plan has the better
// block lookup (one table before two, two before none), else the scalar is
// returned as it is.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "plan.h"
#include "ps.h"
#include "zxp.h"

namespace zxp {

namespace {

uint64_t relabel(uint64_t m, const std::vector<uint32_t>& perm) {   // perm[new] = old
    uint64_t r = 0;
    for (uint32_t i = 0; i < perm.size(); i++)
        if ((m >> perm[i]) & 1) r |= 1ull << i;
    return r;
}

}  // namespace

int reorder_scalar(const PS& in, PS* out) {
    if (in.k_inner) return ZXP_EINVAL;
    const uint32_t k = in.k;
    // the forms (rows with a parity mask) that hold each parameter, as bit sets
    const size_t nf = in.lin.size() + in.node.size() + in.pair.size(), words = (nf + 63) / 64;
    std::vector<std::vector<uint64_t>> held(k, std::vector<uint64_t>(words, 0));
    std::vector<uint32_t> cost(k, 0);
    std::vector<uint8_t> blocked(k, 0);
    size_t f = 0;
    auto add = [&](uint64_t m, bool block) {
        for (uint32_t i = 0; i < k; i++)
            if ((m >> i) & 1) {
                cost[i]++;
                held[i][f >> 6] |= 1ull << (f & 63);
                if (block) blocked[i] = 1;
            }
        f++;
    };
    for (const LinRow& r : in.lin) add(r.mask, false);
    // zero tests: 1 + w^(0 or 4 + 4 l)
    for (const NodeRow& r : in.node) add(r.mask, (r.g & 3) == 0);
    for (const PairRow& r : in.pair) add(r.ma | r.mb, true);
    std::vector<uint32_t> order(k);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        if (blocked[a] != blocked[b]) return blocked[a] < blocked[b];
        return cost[a] < cost[b];
    });
    // the triple with the fewest forms in all, among the lightest candidates
    const uint32_t nc = k < 16 ? k : 16;
    std::vector<uint32_t> best;
    size_t best_u = ~(size_t)0;
    for (uint32_t a = 0; a < nc; a++)
        for (uint32_t b = a + 1; b < nc; b++)
            for (uint32_t c = b + 1; c < nc; c++) {
                const uint32_t x = order[a], y = order[b], z = order[c];
                const size_t u0 = (size_t)blocked[x] + blocked[y] + blocked[z];
                size_t u = 0;
                for (size_t w = 0; w < words; w++)
                    u += (size_t)__builtin_popcountll(held[x][w] | held[y][w] | held[z][w]);
                u += u0 << 32;   // unblocked triples first
                if (u < best_u) {
                    best_u = u;
                    best = {x, y, z};
                }
            }
    if (best.empty()) best.assign(order.begin(), order.begin() + (k < 3 ? k : 3));
    std::vector<uint32_t> perm = best;
    for (uint32_t i : order)
        if (perm.size() < (k < 4 ? k : 4) && std::find(perm.begin(), perm.end(), i) == perm.end()) perm.push_back(i);
    std::vector<uint8_t> low(k, 0);
    for (uint32_t i : perm) low[i] = 1;
    for (uint32_t i = 0; i < k; i++)
        if (!low[i]) perm.push_back(i);
    PS ps = in;
    for (LinRow& r : ps.lin) r.mask = relabel(r.mask, perm);
    for (QuadRow& r : ps.quad) {
        r.a = relabel(r.a, perm);
        r.b = relabel(r.b, perm);
    }
    for (NodeRow& r : ps.node) r.mask = relabel(r.mask, perm);
    for (PairRow& r : ps.pair) {
        r.ma = relabel(r.ma, perm);
        r.mb = relabel(r.mb, perm);
    }
    // keep the new order only when its block lookup is better
    auto rank = [](const PS& p) {
        Plan pl;
        if (build_plan(p, &pl) != ZXP_OK) return 0;
        return pl.lut_ok ? (pl.lut_two ? 2 : 3) : 1;
    };
    if (rank(ps) > rank(in)) *out = std::move(ps);
    else *out = in;
    return ZXP_OK;
}

}  // namespace zxp
