// param.cpp -- binding the parameters of a parametric scalar (param.h).
#include "param.h"

#include "zring.h"

namespace zxp {

namespace {

uint32_t parity(uint64_t m) { return (uint32_t)__builtin_popcountll(m) & 1u; }

}  // namespace

void bind(const PPS& pps, uint64_t bits, PS* out) {
    PS ps;
    ps.k = pps.k;
    ps.e0 = pps.e0;
    ps.t_count = pps.t_count;
    if (pps.zero) {
        ps.k = 0;
        ps.e0 = 0;
        ps.G[0] = ps.G[1] = ps.G[2] = ps.G[3] = 0;
        *out = ps;
        return;
    }
    uint32_t phase = 0;   // w^phase collected from rows that become constant
    std::vector<LinRow> extra;
    for (const PLin& r : pps.lin) {
        const uint32_t beta = parity(r.mb & bits);
        const uint32_t c = r.c & 7u;
        if (!r.mx) { phase += c * beta; continue; }
        if (beta) { phase += c; ps.lin.push_back({r.mx, (8u - c) & 7u}); }
        else ps.lin.push_back({r.mx, c});
    }
    for (const PQuad& q : pps.quad) {
        const uint32_t al = parity(q.ab & bits), be = parity(q.bb & bits);
        if (q.ax && q.bx) ps.quad.push_back({q.ax, q.bx});
        if (al && q.bx) extra.push_back({q.bx, 4});
        if (be && q.ax) extra.push_back({q.ax, 4});
        if (al && be) phase += 4;
    }
    ps.lin.insert(ps.lin.end(), extra.begin(), extra.end());
    for (const PNode& n : pps.node)
        ps.node.push_back({n.mx, (n.g + 4u * parity(n.mb & bits)) & 7u});
    for (const PPair& r : pps.pair)
        ps.pair.push_back({r.mxa, r.mxb, (r.a + 4u * parity(r.mba & bits)) & 7u,
                           (r.b + 4u * parity(r.mbb & bits)) & 7u});
    zw64 G = zw_make((uint64_t)pps.G[0], (uint64_t)pps.G[1], (uint64_t)pps.G[2], (uint64_t)pps.G[3]);
    G = zw_mul(G, zw_wpow(phase & 7u));
    for (int i = 0; i < 4; i++) ps.G[i] = (int64_t)G.c[i];
    *out = std::move(ps);
}

}  // namespace zxp
