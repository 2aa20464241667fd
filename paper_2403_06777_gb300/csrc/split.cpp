// split.cpp -- host transform of a scalar into inner and outer parameters
// (see split.h).
//
// Every row of a scalar is a function of parity forms of x, so a linear
// change of variables x = M^-1 y rewrites the scalar exactly: a form m
// becomes the XOR of the rows of M^-1 selected by m.  Three steps:
//
//  1. coordinates: y_i = f_i(x) for k independent forms f_i of the
//     non-Clifford rows (odd linear phases, nodes, phase-pair forms),
//     lightest first -- the graph form of the diagram, in which nearly
//     every such row sits on one coordinate;
//  2. partition: inner coordinates I are added greedily (coordinates
//     holding a node first, coordinates under few multi-coordinate forms
//     next) while the outer forms the inner sum depends on -- the cut rows
//     B x_O of the Clifford coupling and the outer parts of the crossing
//     rows -- span at most |O| - low_free dimensions;
//  3. outer coordinates: the lowest ones are a basis of the outer
//     assignments that leave every such form unchanged (their kernel),
//     lightest first, so that the inner sum is constant while the Gray-code
//     walk flips only them.
// Several random tie-breaks and every limit on the crossing forms are
// tried; the least estimated device time wins (split_cost), over the
// prefixes of each greedy order.
#include "split.h"

#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.h"
#include "zxp.h"

namespace zxp {
namespace {

inline int popc(uint64_t v) { return __builtin_popcountll(v); }
inline uint32_t par(uint64_t v) { return (uint32_t)__builtin_parityll(v); }

uint64_t mix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// GF(2) span kept in reduced form: every row's lowest set bit (its pivot)
// appears in no other row.
struct Span {
    std::vector<uint64_t> rows;
    uint64_t reduce(uint64_t v) const {
        for (uint64_t r : rows)
            if (v & r & (0 - r)) v ^= r;
        return v;
    }
    bool add(uint64_t v) {
        v = reduce(v);
        if (!v) return false;
        const uint64_t p = v & (0 - v);
        for (uint64_t& r : rows)
            if (r & p) r ^= v;
        rows.push_back(v);
        return true;
    }
    size_t rank() const { return rows.size(); }
};

// Rows of M^-1 for an invertible k x k matrix M given by rows (bit j of
// M[i] = M_ij): x_j = parity(inv[j] & y) when y_i = parity(M[i] & x).
bool invert(std::vector<uint64_t> a, uint32_t k, std::vector<uint64_t>* inv) {
    std::vector<uint64_t> b(k);
    for (uint32_t i = 0; i < k; i++) b[i] = 1ull << i;
    for (uint32_t col = 0; col < k; col++) {
        uint32_t r = col;
        while (r < k && !((a[r] >> col) & 1)) r++;
        if (r == k) return false;
        std::swap(a[r], a[col]);
        std::swap(b[r], b[col]);
        for (uint32_t i = 0; i < k; i++)
            if (i != col && ((a[i] >> col) & 1)) { a[i] ^= a[col]; b[i] ^= b[col]; }
    }
    *inv = std::move(b);
    return true;
}

uint64_t transform(uint64_t m, const std::vector<uint64_t>& inv) {
    uint64_t r = 0;
    for (; m; m &= m - 1) r ^= inv[(size_t)__builtin_ctzll(m)];
    return r;
}

// Scalar rows in graph coordinates, with what the partition needs.
struct Graph {
    PS ps;                       // rows rewritten
    std::vector<uint64_t> adj;   // Clifford coupling: coefficient 4 of x_i x_j
    std::vector<uint64_t> fac;   // forms of the non-Clifford rows
    // the non-Clifford rows as (form, second form or 0): a row that touches
    // the inner coordinates is summed inside, so every outer part of its
    // forms becomes a cut form
    std::vector<std::pair<uint64_t, uint64_t>> rows;
    std::vector<int> cover;      // multi-coordinate forms holding coordinate i
    uint64_t node_coords = 0;    // coordinates that are a node's form
};

Graph to_graph(const PS& in, uint64_t& rng) {
    const uint32_t k = in.k;
    std::vector<uint64_t> fac;
    for (auto& r : in.lin) if ((r.c & 1) && r.mask) fac.push_back(r.mask);
    for (auto& r : in.node) if (r.mask) fac.push_back(r.mask);
    for (auto& r : in.pair) { if (r.ma) fac.push_back(r.ma); if (r.mb) fac.push_back(r.mb); }
    // lightest forms first, random order among equal weights
    std::vector<std::pair<uint64_t, uint64_t>> keyed;
    for (uint64_t f : fac) keyed.push_back({((uint64_t)popc(f) << 40) | (mix(rng) >> 24), f});
    std::sort(keyed.begin(), keyed.end());
    Span sp;
    std::vector<uint64_t> basis;
    for (auto& kf : keyed)
        if (basis.size() < k && sp.add(kf.second)) basis.push_back(kf.second);
    for (uint32_t i = 0; i < k && basis.size() < k; i++)
        if (sp.add(1ull << i)) basis.push_back(1ull << i);
    std::vector<uint64_t> inv;
    invert(basis, k, &inv);   // the basis is independent by construction
    Graph g;
    g.ps = in;
    for (auto& r : g.ps.lin) r.mask = transform(r.mask, inv);
    for (auto& r : g.ps.quad) { r.a = transform(r.a, inv); r.b = transform(r.b, inv); }
    for (auto& r : g.ps.node) r.mask = transform(r.mask, inv);
    for (auto& r : g.ps.pair) { r.ma = transform(r.ma, inv); r.mb = transform(r.mb, inv); }
    g.adj.assign(k, 0);
    // 4 a(x) b(x) = 4 sum_{i in a, j in b} x_i x_j: x_i x_j (i != j) keeps
    // coefficient 4 iff exactly one of (i in a, j in b), (j in a, i in b)
    for (auto& q : g.ps.quad) {
        for (uint64_t m = q.a; m; m &= m - 1) g.adj[(size_t)__builtin_ctzll(m)] ^= q.b;
        for (uint64_t m = q.b; m; m &= m - 1) g.adj[(size_t)__builtin_ctzll(m)] ^= q.a;
    }
    // c (x1 ^ .. ^ xm), c = 2 mod 4: 4 x_i x_j for every pair of the form
    for (auto& r : g.ps.lin)
        if ((r.c & 3) == 2)
            for (uint64_t m = r.mask; m; m &= m - 1) g.adj[(size_t)__builtin_ctzll(m)] ^= r.mask;
    for (uint32_t i = 0; i < k; i++) g.adj[i] &= ~(1ull << i);
    for (auto& r : g.ps.lin) if ((r.c & 1) && r.mask) g.fac.push_back(r.mask);
    for (auto& r : g.ps.node) {
        if (!r.mask) continue;
        g.fac.push_back(r.mask);
        if (popc(r.mask) == 1) g.node_coords |= r.mask;
    }
    for (auto& r : g.ps.pair) { if (r.ma) g.fac.push_back(r.ma); if (r.mb) g.fac.push_back(r.mb); }
    for (auto& r : g.ps.lin) if ((r.c & 1) && r.mask) g.rows.push_back({r.mask, 0});
    for (auto& r : g.ps.node) if (r.mask) g.rows.push_back({r.mask, 0});
    for (auto& r : g.ps.pair) if (r.ma | r.mb) g.rows.push_back({r.ma, r.mb});
    g.cover.assign(k, 0);
    for (uint64_t f : g.fac)
        if (popc(f) > 1)
            for (uint64_t m = f; m; m &= m - 1) g.cover[(size_t)__builtin_ctzll(m)]++;
    return g;
}

// Forms of the outer parameters that the inner sum depends on, for inner
// coordinates I: the cut rows of the coupling and the distinct outer parts
// of the non-Clifford rows that touch I (those count in `ncut`).
std::vector<uint64_t> cut_forms(const Graph& g, uint64_t I, uint64_t O, uint32_t* ncut) {
    std::vector<uint64_t> w, q;
    for (uint64_t m = I; m; m &= m - 1) {
        const uint64_t r = g.adj[(size_t)__builtin_ctzll(m)] & O;
        if (r) w.push_back(r);
    }
    for (auto& r : g.rows) {
        if (!((r.first | r.second) & I)) continue;
        for (uint64_t f : {r.first, r.second})
            if ((f & O) && std::find(q.begin(), q.end(), f & O) == q.end()) q.push_back(f & O);
    }
    *ncut = (uint32_t)q.size();
    w.insert(w.end(), q.begin(), q.end());
    return w;
}

// Estimated device time (ps) of one full sum after a split into n_inner
// inner parameters (an inner table of 2^bits entries) and k_o outer ones,
// from rates measured on GB300: the inner table 20.5 ps per entry for the
// term kernel (the low 11 bits transformed) and 19.3 ps per entry for each
// further pass of up to 11 bits; the walk 0.374 ps per outer term with the
// block lookup (0.94 without it) plus an 11 ps fold per run of 2^low_free
// terms between cut-parity changes.
double split_cost(uint32_t n_inner, uint32_t bits, uint32_t k_o, uint32_t low_free, bool lookup = true) {
    const uint32_t passes = (n_inner > 11 ? n_inner - 11 + 10 : 0) / 11;
    const double inner = (20.5 + 19.3 * passes) * (double)(1ull << bits);
    const double walk = ((lookup ? 0.374 : 0.94) + 11.0 / (double)(1ull << low_free)) * (double)(1ull << k_o);
    return inner + walk;
}

struct Choice {
    uint32_t k_o = 0, bits = 0, outer_nodes = 0;
    double cost = 0;
    uint64_t I = 0;
    bool ok = false;
    bool better(const Choice& o) const {
        if (!o.ok) return ok;
        if (cost != o.cost) return cost < o.cost;
        if (bits != o.bits) return bits < o.bits;
        return outer_nodes < o.outer_nodes;
    }
};

Choice partition(const Graph& g, const SplitOptions& opt, uint64_t& rng) {
    const uint32_t k = g.ps.k;
    const uint64_t all = k >= 64 ? ~0ull : (1ull << k) - 1;
    std::vector<std::pair<double, uint32_t>> order;
    for (uint32_t i = 0; i < k; i++) {
        const double node_first = ((g.node_coords >> i) & 1) ? 0.0 : 1.0;
        order.push_back({node_first + g.cover[i] + 1.5 * (double)(mix(rng) >> 11) * 0x1.0p-53, i});
    }
    std::sort(order.begin(), order.end());
    // the greedy order's additions, and among the prefixes of it the one of
    // least estimated cost (more inner parameters halve the walk and double
    // the inner table)
    uint64_t I = 0, bestI = 0;
    uint32_t nI = 0, bits = 0, best_n = 0, best_bits = 0;
    double best_cost = 0;
    for (auto& oi : order) {
        const uint64_t I2 = I | (1ull << oi.second);
        const uint32_t n2 = nI + 1;
        if (n2 > opt.max_inner || k - n2 < opt.low_free) break;
        uint32_t ncut = 0;
        const std::vector<uint64_t> w = cut_forms(g, I2, all & ~I2, &ncut);
        if (ncut > opt.max_cut || n2 + ncut > opt.max_index_bits) continue;
        Span sp;
        for (uint64_t f : w) sp.add(f);
        if (sp.rank() + opt.low_free > k - n2) continue;
        I = I2;
        nI = n2;
        bits = n2 + ncut;
        const double cost = split_cost(nI, bits, k - nI, opt.low_free);
        if (!best_n || cost < best_cost) {
            bestI = I;
            best_n = nI;
            best_bits = bits;
            best_cost = cost;
        }
    }
    Choice c;
    c.ok = best_n > 0;
    c.I = bestI;
    c.k_o = k - best_n;
    c.bits = best_bits;
    c.cost = best_cost;
    for (auto& r : g.ps.node)
        if (r.mask && !(r.mask & bestI)) c.outer_nodes++;
    return c;
}

// Outer coordinates (compact positions of O): the lowest ones a basis of
// the kernel of the cut forms, lightest (fewest outer forms flipped) first;
// the rest complete a basis.  Returns the columns A_i: outer coordinate y_j
// of the graph = parity over i of A_i[j] z_i.
std::vector<uint64_t> outer_columns(const Graph& g, uint64_t I, uint64_t& rng) {
    const uint32_t k = g.ps.k;
    const uint64_t all = k >= 64 ? ~0ull : (1ull << k) - 1, O = all & ~I;
    std::vector<uint32_t> opos;
    for (uint32_t i = 0; i < k; i++) if ((O >> i) & 1) opos.push_back(i);
    const uint32_t ko = (uint32_t)opos.size();
    auto compact = [&](uint64_t m) {
        uint64_t r = 0;
        for (uint32_t j = 0; j < ko; j++) if ((m >> opos[j]) & 1) r |= 1ull << j;
        return r;
    };
    uint32_t ncut = 0;
    std::vector<uint64_t> w;
    for (uint64_t f : cut_forms(g, I, O, &ncut)) w.push_back(compact(f));
    // kernel of w: reduced row echelon form over ko columns
    std::vector<uint64_t> rref;
    std::vector<uint32_t> pivc;
    for (uint64_t f : w) {
        for (size_t i = 0; i < rref.size(); i++) if ((f >> pivc[i]) & 1) f ^= rref[i];
        if (!f) continue;
        const uint32_t p = (uint32_t)__builtin_ctzll(f);
        for (size_t i = 0; i < rref.size(); i++) if ((rref[i] >> p) & 1) rref[i] ^= f;
        rref.push_back(f);
        pivc.push_back(p);
    }
    uint64_t is_piv = 0;
    for (uint32_t p : pivc) is_piv |= 1ull << p;
    std::vector<uint64_t> kb;
    for (uint32_t j = 0; j < ko; j++) {
        if ((is_piv >> j) & 1) continue;
        uint64_t v = 1ull << j;
        for (size_t i = 0; i < rref.size(); i++) if ((rref[i] >> j) & 1) v |= 1ull << pivc[i];
        kb.push_back(v);
    }
    // Outer forms that hold form bits in the walk: odd linear phases,
    // nodes and phase-pair forms on outer coordinates only (even linear
    // phases become one singleton per variable and quadratic terms, so they
    // add at most one form per variable).
    std::vector<uint64_t> forms;
    for (auto& r : g.ps.lin) if ((r.c & 1) && r.mask && !(r.mask & I)) forms.push_back(compact(r.mask));
    for (auto& r : g.ps.node) if (r.mask && !(r.mask & I)) forms.push_back(compact(r.mask));
    for (auto& r : g.ps.pair)
        if ((r.ma | r.mb) && !((r.ma | r.mb) & I)) {
            if (r.ma) forms.push_back(compact(r.ma));
            if (r.mb) forms.push_back(compact(r.mb));
        }
    // candidate kernel vectors: the whole kernel when small, else samples
    const size_t dim = kb.size();
    std::vector<uint64_t> cand;
    if (dim <= 16) {
        for (uint64_t c = 1; c < (1ull << dim); c++) {
            uint64_t v = 0;
            for (size_t j = 0; j < dim; j++) if ((c >> j) & 1) v ^= kb[j];
            cand.push_back(v);
        }
    } else {
        cand = kb;
        for (int s = 0; s < 65536; s++) {
            uint64_t v = 0;
            const uint64_t c = mix(rng);
            for (size_t j = 0; j < dim; j++) if ((c >> (j & 63)) & 1) v ^= kb[j];
            if (v) cand.push_back(v);
        }
    }
    // the forms each candidate flips, as a bitset
    const size_t nfw = (forms.size() + 63) / 64 + 1;
    std::vector<uint64_t> H(cand.size() * nfw, 0ull);
    std::vector<int> nh(cand.size(), 0);
    for (size_t c = 0; c < cand.size(); c++) {
        for (size_t f = 0; f < forms.size(); f++)
            if (par(forms[f] & cand[c])) H[c * nfw + f / 64] |= 1ull << (f % 64);
        for (size_t w = 0; w < nfw; w++) nh[c] += popc(H[c * nfw + w]);
    }
    auto uni = [&](std::initializer_list<size_t> cs) {
        int n = 0;
        for (size_t w = 0; w < nfw; w++) {
            uint64_t u = 0;
            for (size_t c : cs) u |= H[c * nfw + w];
            n += popc(u);
        }
        return n;
    };
    // Variables 0-2 (their forms are the block lookup's index): three
    // independent kernel vectors whose flipped forms have the smallest
    // union, from the lightest vectors and the best pairs among them.
    std::vector<size_t> order(cand.size());
    for (size_t c = 0; c < cand.size(); c++) order[c] = c;
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        return nh[x] != nh[y] ? nh[x] < nh[y] : popc(cand[x]) < popc(cand[y]);
    });
    std::vector<uint64_t> cols;
    if (dim >= 3) {
        std::vector<std::pair<int, std::pair<size_t, size_t>>> pairs;
        const size_t n0 = std::min<size_t>(order.size(), 32);
        for (size_t x = 0; x < n0; x++)
            for (size_t y = 0; y < cand.size(); y++)
                if (cand[y] != cand[order[x]]) pairs.push_back({uni({order[x], y}), {order[x], y}});
        std::sort(pairs.begin(), pairs.end());
        int best = -1;
        size_t b0 = 0, b1 = 0, b2 = 0;
        for (size_t p = 0; p < pairs.size() && p < 64; p++) {
            const size_t c0 = pairs[p].second.first, c1 = pairs[p].second.second;
            for (size_t z = 0; z < cand.size(); z++) {
                const uint64_t v = cand[z];
                if (v == cand[c0] || v == cand[c1] || v == (cand[c0] ^ cand[c1])) continue;
                const int u = uni({c0, c1, z});
                if (best < 0 || u < best) { best = u; b0 = c0; b1 = c1; b2 = z; }
            }
        }
        if (best >= 0) {
            // the lightest of the three flips most often
            size_t t[3] = {b0, b1, b2};
            std::sort(t, t + 3, [&](size_t x, size_t y) { return nh[x] < nh[y]; });
            for (size_t c : t) cols.push_back(cand[c]);
        }
    }
    Span sp;
    for (uint64_t c : cols) sp.add(c);
    for (size_t c : order) {
        if (cols.size() == dim) break;
        if (sp.add(cand[c])) cols.push_back(cand[c]);
    }
    for (uint32_t j = 0; j < ko && cols.size() < ko; j++)
        if (sp.add(1ull << j)) cols.push_back(1ull << j);
    // back to graph coordinates
    for (uint64_t& c : cols) {
        uint64_t r = 0;
        for (uint32_t j = 0; j < ko; j++) if ((c >> j) & 1) r |= 1ull << opos[j];
        c = r;
    }
    return cols;
}

// The scalar in the variables of graph g with inner coordinates I: outer
// parameters first (outer_columns), then the inner ones.
PS make_split(const Graph& g, uint64_t I, uint64_t& rng) {
    const uint32_t k = g.ps.k;
    const uint32_t ko = k - (uint32_t)popc(I);
    const std::vector<uint64_t> cols = outer_columns(g, I, rng);
    std::vector<uint32_t> ipos;
    for (uint32_t i = 0; i < k; i++) if ((I >> i) & 1) ipos.push_back(i);
    auto remap = [&](uint64_t m) {
        uint64_t r = 0;
        for (uint32_t j = 0; j < ko; j++) r |= (uint64_t)par(m & cols[j]) << j;
        for (size_t j = 0; j < ipos.size(); j++) r |= ((m >> ipos[j]) & 1ull) << (ko + j);
        return r;
    };
    PS ps = g.ps;
    for (auto& r : ps.lin) r.mask = remap(r.mask);
    for (auto& r : ps.quad) { r.a = remap(r.a); r.b = remap(r.b); }
    for (auto& r : ps.node) r.mask = remap(r.mask);
    for (auto& r : ps.pair) { r.ma = remap(r.ma); r.mb = remap(r.mb); }
    ps.k_inner = k - ko;
    return ps;
}

}  // namespace

int split_scalar(const PS& in, const SplitOptions& opt, PS* out) {
    if (!out || in.k_inner != 0 || in.k > 62) return ZXP_EINVAL;
    *out = in;
    if (in.k < opt.min_k || in.k < opt.low_free + 1 || opt.low_free < 4) return ZXP_OK;
    uint64_t rng = opt.seed ^ ((uint64_t)in.k << 32) ^ (in.lin.size() * 0x9E37ull) ^ in.node.size();
    // the partitions of least estimated cost (with the block lookup's walk
    // rate), distinct ones, and the graph each was found in
    constexpr size_t kCands = 6;
    std::vector<std::pair<Choice, Graph>> cands;
    // (every limit on the crossing forms up to max_cut: a greedy order under
    // a looser limit can take a coordinate that brings crossing forms and
    // miss a partition with fewer index bits)
    for (int t = 0; t < std::max(1, opt.tries); t++) {
        Graph g = to_graph(in, rng);
        for (int r = 0; r < 4; r++) {
            SplitOptions o = opt;
            for (o.max_cut = 0; o.max_cut <= opt.max_cut; o.max_cut++) {
                Choice c = partition(g, o, rng);
                if (!c.ok || c.k_o >= in.k) continue;
                if (cands.size() == kCands && !c.better(cands.back().first)) continue;
                // (the same partition again, under another crossing limit)
                bool dup = false;
                for (auto& e : cands) dup = dup || (e.first.I == c.I && e.first.cost == c.cost);
                if (dup) continue;
                auto at = std::find_if(cands.begin(), cands.end(), [&](const std::pair<Choice, Graph>& e) {
                    return c.better(e.first);
                });
                cands.insert(at, std::make_pair(c, g));
                if (cands.size() > kCands) cands.pop_back();
            }
        }
    }
    // each candidate as the scalar it gives: whether its plan takes the
    // block lookup (the outer basis decides; another random basis is drawn
    // when it does not) sets the walk rate of the estimate
    double best_cost = 0;
    bool found = false;
    for (auto& e : cands) {
        for (int b = 0; b < 3; b++) {
            PS ps = make_split(e.second, e.first.I, rng);
            Plan pl;
            if (build_plan(ps, &pl) != ZXP_OK) break;
            const double cost = split_cost(ps.k_inner, pl.inner_bits, ps.k - ps.k_inner, pl.kp.zq_lo, pl.lut_ok);
            if (!found || cost < best_cost) {
                best_cost = cost;
                found = true;
                *out = std::move(ps);
            }
            if (pl.lut_ok) break;
        }
    }
    return ZXP_OK;
}

}  // namespace zxp
