// reorder.cpp -- relabelling a scalar's parameters (zxp_scalar_reorder).
//
// The sum over x in {0,1}^k (Eq. 2) does not depend on the order of the
// parameters, but the Gray-code walk does: parameters 0, 1 and 2 flip in
// every aligned block of 8 steps, and the block lookup that costs one
// table read per 8 terms applies only when few parity forms hold them and
// none of them is a phase-pair or zero-test form.  This moves the four
// parameters that touch the fewest forms (and none of those two kinds where
// possible) to positions 0-3, keeping the others in their order.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

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
    std::vector<uint32_t> cost(k, 0);
    std::vector<uint8_t> blocked(k, 0);
    auto add = [&](uint64_t m, bool block) {
        for (uint32_t i = 0; i < k; i++)
            if ((m >> i) & 1) {
                cost[i]++;
                if (block) blocked[i] = 1;
            }
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
    const uint32_t nlow = k < 4 ? k : 4;
    std::vector<uint32_t> perm(order.begin(), order.begin() + nlow);
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
    *out = std::move(ps);
    return ZXP_OK;
}

}  // namespace zxp
