// ps.cpp -- table layout of a parametric scalar (little endian):
//   header  u32 magic, u32 version, u32 k, u32 n_lin, u32 n_quad, u32 n_node,
//           u32 n_pair, i32 e0, i64 G[4]
//   version 2 only: u32 k_inner, u32 0
//   rows    lin {u64 mask, u32 c, u32 0}, quad {u64, u64},
//           node {u64 mask, u32 g, u32 0}, pair {u64 ma, u64 mb, u32 a, u32 b}
#include "ps.h"

#include <string.h>

#include "zxp.h"

namespace zxp {

namespace {
struct Header {
    uint32_t magic, version, k, n_lin, n_quad, n_node, n_pair;
    int32_t e0;
    int64_t G[4];
};
static_assert(sizeof(Header) == 64, "header layout");

template <class T> T rd(const uint8_t* p) { T v; memcpy(&v, p, sizeof v); return v; }
template <class T> void wr(uint8_t* p, T v) { memcpy(p, &v, sizeof v); }
}  // namespace

int ps_from_blob(const void* blob, size_t nbytes, PS* out) {
    if (!blob || !out || nbytes < sizeof(Header)) return ZXP_EINVAL;
    Header h;
    memcpy(&h, blob, sizeof h);
    if (h.magic != kPsMagic || (h.version != kPsVersion && h.version != kPsVersionInner)) return ZXP_EINVAL;
    if (h.k > 62) return ZXP_ETOOBIG;
    const size_t hsize = sizeof(Header) + (h.version == kPsVersionInner ? 8u : 0u);
    uint64_t need = hsize + 16ull * h.n_lin + 16ull * h.n_quad + 16ull * h.n_node + 24ull * h.n_pair;
    if (nbytes < need) return ZXP_EINVAL;
    const uint64_t allowed = h.k ? ((h.k == 64) ? ~0ull : ((1ull << h.k) - 1)) : 0ull;
    PS ps;
    ps.k = h.k;
    if (h.version == kPsVersionInner) {
        ps.k_inner = rd<uint32_t>((const uint8_t*)blob + sizeof(Header));
        if (ps.k_inner == 0 || ps.k_inner > ps.k) return ZXP_EINVAL;
    }
    ps.e0 = h.e0;
    for (int i = 0; i < 4; i++) ps.G[i] = h.G[i];
    const uint8_t* p = (const uint8_t*)blob + hsize;
    for (uint32_t i = 0; i < h.n_lin; i++, p += 16) {
        LinRow r{rd<uint64_t>(p), rd<uint32_t>(p + 8)};
        if ((r.mask & ~allowed) || r.c > 7) return ZXP_EINVAL;
        ps.lin.push_back(r);
    }
    for (uint32_t i = 0; i < h.n_quad; i++, p += 16) {
        QuadRow r{rd<uint64_t>(p), rd<uint64_t>(p + 8)};
        if ((r.a | r.b) & ~allowed) return ZXP_EINVAL;
        ps.quad.push_back(r);
    }
    for (uint32_t i = 0; i < h.n_node; i++, p += 16) {
        NodeRow r{rd<uint64_t>(p), rd<uint32_t>(p + 8)};
        if ((r.mask & ~allowed) || r.g > 7) return ZXP_EINVAL;
        ps.node.push_back(r);
    }
    for (uint32_t i = 0; i < h.n_pair; i++, p += 24) {
        PairRow r{rd<uint64_t>(p), rd<uint64_t>(p + 8), rd<uint32_t>(p + 16), rd<uint32_t>(p + 20)};
        if (((r.ma | r.mb) & ~allowed) || r.a > 7 || r.b > 7) return ZXP_EINVAL;
        ps.pair.push_back(r);
    }
    *out = std::move(ps);
    return ZXP_OK;
}

size_t ps_blob_size(const PS& ps) {
    return sizeof(Header) + (ps.k_inner ? 8 : 0) + 16 * ps.lin.size() + 16 * ps.quad.size() + 16 * ps.node.size() +
           24 * ps.pair.size();
}

void ps_to_blob(const PS& ps, void* buf) {
    Header h;
    h.magic = kPsMagic;
    h.version = ps.k_inner ? kPsVersionInner : kPsVersion;
    h.k = ps.k;
    h.n_lin = (uint32_t)ps.lin.size();
    h.n_quad = (uint32_t)ps.quad.size();
    h.n_node = (uint32_t)ps.node.size();
    h.n_pair = (uint32_t)ps.pair.size();
    h.e0 = ps.e0;
    for (int i = 0; i < 4; i++) h.G[i] = ps.G[i];
    uint8_t* p = (uint8_t*)buf;
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    if (ps.k_inner) { wr(p, ps.k_inner); wr(p + 4, (uint32_t)0); p += 8; }
    for (auto& r : ps.lin) { wr(p, r.mask); wr(p + 8, r.c); wr(p + 12, (uint32_t)0); p += 16; }
    for (auto& r : ps.quad) { wr(p, r.a); wr(p + 8, r.b); p += 16; }
    for (auto& r : ps.node) { wr(p, r.mask); wr(p + 8, r.g); wr(p + 12, (uint32_t)0); p += 16; }
    for (auto& r : ps.pair) { wr(p, r.ma); wr(p + 8, r.mb); wr(p + 16, r.a); wr(p + 20, r.b); p += 24; }
}

}  // namespace zxp
