// compile.cpp -- host-side parametric reduction (Sec. 3.1-3.2 of the paper).
//
// The closed diagram <out|C|in> is handled in its sum-over-paths form, which
// is the phase-polynomial reading of a graph-like ZX-diagram: one Boolean
// variable y per Hadamard (an X-spider pair / Hadamard edge), a phase
// polynomial P(y) mod 8 (P = sum of c * parity-forms, w^P), and a global
// scalar.  The rewrite rules of Fig. 1 act on it as follows:
//
//   * spider fusion / pi-commutation: phases add on equal parity forms;
//     a form picks up a constant pi when a pi spider is commuted through
//     (the polarised phases of Eq. 1: each parametric phase is alpha or
//     alpha + pi);
//   * state copy / the Z(alpha)-X(beta) and isolated-spider scalars: summing
//     a variable y that appears as y (c + 4 l(rest)) gives 1 + w^(c + 4l),
//     the node subterm of App. C; two adjacent such variables give the
//     phase-pair subterm of Eq. 3; a pi-pair e^{i Psi Phi/pi} is the
//     quadratic term 4 l l';
//   * local complementation (c in {2,6}) and pivoting (c in {0,4}) remove
//     Clifford variables for a factor sqrt2 w^(+-1) or 2 (Clifford
//     simplification);
//   * a T-like phase on a multi-variable form, which blocks the removal of
//     its variables (Lemma 1), is decomposed with one Boolean parameter a:
//        w^l = 1/2 sum_a (1 + w^(1 + 4a)) (-1)^(a l),
//     i.e. a node subterm in a and a pi-pair between a and the form.
//
// Every step holds for all values of the remaining variables at once (the
// parametric rules): no step branches on a parameter, so the result is one
// parametric scalar S = G/sqrt2^e0 sum_x prod_j S_j(x) (Eq. 2).
#include "compile.h"

#include <string.h>

#include <algorithm>
#include <unordered_set>
#include <vector>

#include "zxp.h"
#include "zring.h"

namespace zxp {
namespace {

// ---------------------------------------------------------------------------
// dynamic bitset over variables
// ---------------------------------------------------------------------------
struct Bits {
    std::vector<uint64_t> w;
    Bits() {}
    explicit Bits(int nw) : w((size_t)nw, 0) {}
    bool get(int i) const { return (w[(size_t)i >> 6] >> (i & 63)) & 1; }
    void set(int i) { w[(size_t)i >> 6] |= 1ull << (i & 63); }
    void clr(int i) { w[(size_t)i >> 6] &= ~(1ull << (i & 63)); }
    void flip(int i) { w[(size_t)i >> 6] ^= 1ull << (i & 63); }
    void xor_with(const Bits& o) { for (size_t j = 0; j < w.size(); j++) w[j] ^= o.w[j]; }
    void or_with(const Bits& o) { for (size_t j = 0; j < w.size(); j++) w[j] |= o.w[j]; }
    void and_not(const Bits& o) { for (size_t j = 0; j < w.size(); j++) w[j] &= ~o.w[j]; }
    bool any() const { for (uint64_t v : w) if (v) return true; return false; }
    int count() const { int c = 0; for (uint64_t v : w) c += __builtin_popcountll(v); return c; }
    int first() const {
        for (size_t j = 0; j < w.size(); j++) if (w[j]) return (int)(j * 64 + __builtin_ctzll(w[j]));
        return -1;
    }
    int count_and(const Bits& o) const {
        int c = 0;
        for (size_t j = 0; j < w.size(); j++) c += __builtin_popcountll(w[j] & o.w[j]);
        return c;
    }
    bool operator==(const Bits& o) const { return w == o.w; }
    void resize(int nw) { w.resize((size_t)nw, 0); }
    template <class F> void each(F f) const {
        for (size_t j = 0; j < w.size(); j++) {
            uint64_t v = w[j];
            while (v) { f((int)(j * 64 + __builtin_ctzll(v))); v &= v - 1; }
        }
    }
    std::vector<int> list() const { std::vector<int> r; each([&](int i) { r.push_back(i); }); return r; }
};
struct BitsHash {
    size_t operator()(const Bits& b) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (uint64_t v : b.w) { h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2); }
        return (size_t)h;
    }
};

struct NodeF { int g; Bits f; };
struct PairF { int a; Bits fa; int b; Bits fb; };

uint64_t mix64(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// the path sum: sum_y w^P(y) * prod nodes * prod pairs * global / sqrt2^e0
// ---------------------------------------------------------------------------
class PathSum {
  public:
    int cap = 0, nw = 0, nvars = 0;
    std::vector<uint8_t> live, sing;     // sing[v]: coefficient of y_v (mod 8)
    // Parameters: variables that are never summed (output bits left open);
    // they appear in forms like summed variables, are never pivots, and
    // remain in the result as the parameter part of each form.
    std::vector<uint8_t> ext;
    Bits extm;
    std::vector<Bits> adj;               // 4 y_u y_v terms (symmetric, no loops)
    std::unordered_set<Bits, BitsHash> tf;  // coefficient-1 parity forms, >= 2 vars
    std::vector<NodeF> nodes;
    std::vector<PairF> pairs;
    std::vector<Bits> qf;                // qubit wires: parity form + constant
    std::vector<uint8_t> qc;
    int phase = 0;   // global w^phase
    int e0 = 0;      // global 1/sqrt2^e0
    int v1w = 0;     // global (1 - w)^v1w
    int unitN = 0;   // global (1 + sqrt2)^unitN
    bool zero = false;
    std::vector<PairF> const_pairs;  // constant phase-pairs (kept as rows)
    uint64_t rng = 1;
    bool allow_pairs = true;

    explicit PathSum(int n_qubits, int capacity) {
        cap = std::max(64, capacity);
        nw = (cap + 63) / 64;
        live.assign((size_t)cap, 0);
        sing.assign((size_t)cap, 0);
        ext.assign((size_t)cap, 0);
        extm = Bits(nw);
        adj.assign((size_t)cap, Bits(nw));
        qf.assign((size_t)n_qubits, Bits(nw));
        qc.assign((size_t)n_qubits, 0);
    }

    void grow() {
        int ncap = cap * 2, nnw = (ncap + 63) / 64;
        live.resize((size_t)ncap, 0);
        sing.resize((size_t)ncap, 0);
        ext.resize((size_t)ncap, 0);
        extm.resize(nnw);
        for (auto& b : adj) b.resize(nnw);
        adj.resize((size_t)ncap, Bits(nnw));
        std::vector<Bits> t(tf.begin(), tf.end());
        tf.clear();
        for (auto& b : t) { b.resize(nnw); tf.insert(b); }
        for (auto& n : nodes) n.f.resize(nnw);
        for (auto& p : pairs) { p.fa.resize(nnw); p.fb.resize(nnw); }
        for (auto& q : qf) q.resize(nnw);
        cap = ncap; nw = nnw;
    }

    int new_var() {
        if (nvars == cap) grow();
        int v = nvars++;
        live[(size_t)v] = 1;
        sing[(size_t)v] = 0;
        ext[(size_t)v] = 0;
        return v;
    }
    int new_param() {
        int v = new_var();
        ext[(size_t)v] = 1;
        extm.set(v);
        return v;
    }
    // the summed variables of a form
    Bits internal(const Bits& f) const { Bits r = f; r.and_not(extm); return r; }
    Bits unit(int v) const { Bits b(nw); b.set(v); return b; }

    void toggle_edge(int i, int j) { adj[(size_t)i].flip(j); adj[(size_t)j].flip(i); }

    // coef * (form xor cst)
    void add_lin(int coef, const Bits& form, int cst) {
        coef &= 7;
        if (!coef) return;
        if (cst) { phase = (phase + coef) & 7; coef = (8 - coef) & 7; }   // c(1 - l) = c - c l
        int cnt = form.count();
        if (cnt == 0) return;
        if (cnt == 1) { int i = form.first(); sing[(size_t)i] = (uint8_t)((sing[(size_t)i] + coef) & 7); return; }
        if (coef & 1) {
            auto it = tf.find(form);
            if (it != tf.end()) { tf.erase(it); add_even(2, form); }   // l + l = 2l
            else tf.insert(form);
            coef -= 1;
        }
        if (coef) add_even(coef, form);
    }
    // even coef on a parity form of >= 2 variables:
    //   c (y1 ^ ... ^ ym) = c sum y_i + 4 [c = 2 mod 4] sum_{i<j} y_i y_j  (mod 8)
    void add_even(int coef, const Bits& form) {
        form.each([&](int i) { sing[(size_t)i] = (uint8_t)((sing[(size_t)i] + coef) & 7); });
        if (coef & 2) {
            form.each([&](int i) { adj[(size_t)i].xor_with(form); adj[(size_t)i].flip(i); });
        }
    }
    // 4 (A xor a0)(B xor b0)
    void add_quad(const Bits& A, int a0, const Bits& B, int b0) {
        if (a0 && b0) phase = (phase + 4) & 7;
        if (a0) add_lin(4, B, 0);
        if (b0) add_lin(4, A, 0);
        Bits u = A;
        u.or_with(B);
        u.each([&](int i) {
            Bits r(nw);
            if (A.get(i)) r.xor_with(B);
            if (B.get(i)) r.xor_with(A);
            r.clr(i);
            adj[(size_t)i].xor_with(r);
            if (A.get(i) && B.get(i)) sing[(size_t)i] = (uint8_t)((sing[(size_t)i] + 4) & 7);
        });
    }

    // y_p := A xor a   (p not in A)
    void substitute(int p, const Bits& A, int a) {
        Bits ua = A;              // the change applied to every form holding p
        ua.flip(p);
        // T-forms holding p
        std::vector<Bits> hit;
        for (auto& f : tf) if (f.get(p)) hit.push_back(f);
        for (auto& f : hit) tf.erase(f);
        // nodes, pairs, wires
        for (auto& n : nodes) if (n.f.get(p)) { n.f.xor_with(ua); n.g = (n.g + 4 * a) & 7; }
        for (auto& q : pairs) {
            if (q.fa.get(p)) { q.fa.xor_with(ua); q.a = (q.a + 4 * a) & 7; }
            if (q.fb.get(p)) { q.fb.xor_with(ua); q.b = (q.b + 4 * a) & 7; }
        }
        for (size_t q = 0; q < qf.size(); q++) if (qf[q].get(p)) { qf[q].xor_with(ua); qc[q] ^= (uint8_t)a; }
        // singleton and quadratic terms of p
        int c = sing[(size_t)p];
        Bits nb = adj[(size_t)p];
        nb.each([&](int j) { adj[(size_t)j].clr(p); });
        adj[(size_t)p] = Bits(nw);
        sing[(size_t)p] = 0;
        live[(size_t)p] = 0;
        for (auto& f : hit) { Bits g = f; g.xor_with(ua); add_lin(1, g, a); }
        add_lin(c, A, a);
        nb.each([&](int j) { add_quad(A, a, unit(j), 0); });
        simplify_nodes();
    }

    // lock counts: how many T-forms / node forms / pair forms hold each variable
    std::vector<int> lock_counts() const {
        std::vector<int> cnt((size_t)nvars, 0);
        auto add = [&](const Bits& b) { b.each([&](int i) { cnt[(size_t)i]++; }); };
        for (auto& f : tf) add(f);
        for (auto& n : nodes) add(n.f);
        for (auto& p : pairs) { add(p.fa); add(p.fb); }
        return cnt;
    }

    // node / pair forms: a variable held there can only leave by substitution
    std::vector<int> hard_lock_counts() const {
        std::vector<int> cnt((size_t)nvars, 0);
        auto add = [&](const Bits& b) { b.each([&](int i) { cnt[(size_t)i]++; }); };
        for (auto& n : nodes) add(n.f);
        for (auto& p : pairs) { add(p.fa); add(p.fb); }
        return cnt;
    }

    // Pick a pivot in F.  Substituting a variable rewrites every form that
    // holds it: a node or pair form grows and locks the new variables for
    // good, a T-form only grows (it can still be decomposed later).  So
    // prefer no node/pair membership, then few T-forms, then small degree.
    int pick_pivot(const Bits& F, const std::vector<int>& locks, const std::vector<int>& hard) {
        int best = -1;
        long bestkey = 0;
        F.each([&](int i) {
            if (ext[(size_t)i]) return;
            long key = (long)hard[(size_t)i] * 100000000L + (long)locks[(size_t)i] * 100000L +
                       adj[(size_t)i].count() * 16 + (long)(mix64(rng) & 15);
            if (best < 0 || key < bestkey) { best = i; bestkey = key; }
        });
        return best;
    }

    // require (F xor c) = 0
    void constrain(const Bits& F, int c) {
        if (!F.any()) { if (c) zero = true; return; }
        if (!internal(F).any()) {
            // a condition on the parameters alone stays a factor of the result:
            // [l xor c = 0] = (1 + w^(4c + 4l)) / 2
            e0 += 2;
            nodes.push_back(NodeF{c ? 4 : 0, F});
            return;
        }
        std::vector<int> locks = lock_counts(), hard = hard_lock_counts();
        int p = pick_pivot(F, locks, hard);
        Bits A = F;
        A.clr(p);
        substitute(p, A, c);
    }

    // constant node 1 + w^g
    void const_node(int g) {
        g &= 7;
        switch (g) {
        case 0: e0 -= 2; break;                          // 2
        case 4: zero = true; break;                      // 0
        case 2: e0 -= 1; phase = (phase + 1) & 7; break; // 1 + i = sqrt2 w
        case 6: e0 -= 1; phase = (phase + 7) & 7; break; // 1 - i = sqrt2 w^7
        // odd: 1 + w^g = (1 - w) w^j (1 + sqrt2)^beta
        case 1: v1w++; phase = (phase + 2) & 7; unitN++; break;
        case 3: v1w++; phase = (phase + 3) & 7; break;
        case 5: v1w++; break;
        case 7: v1w++; phase = (phase + 1) & 7; unitN++; break;
        }
    }

    void add_node(int g, const Bits& f) {
        if (!f.any()) { const_node(g); return; }
        nodes.push_back(NodeF{g & 7, f});
        simplify_nodes();
    }

    // Node pairs on one form whose constants differ by pi cancel to a
    // constant (Sec. 5): (1 + w^(g+4l))(1 + w^(g+4+4l)) = 1 - w^(2g).
    // Even-constant nodes are Clifford and go back into the phase:
    //   1 + w^(2+4l) = sqrt2 w w^(6l),  1 + w^(6+4l) = sqrt2 w^7 w^(2l),
    //   1 + w^(0+4l) = 2 [l = 0],       1 + w^(4+4l) = 2 [l = 1].
    void simplify_nodes() {
        bool again = true;
        while (again && !zero) {
            again = false;
            for (size_t i = 0; i < nodes.size() && !again; i++) {
                if (!nodes[i].f.any()) {
                    int g = nodes[i].g;
                    nodes.erase(nodes.begin() + (long)i);
                    const_node(g);
                    again = true;
                    break;
                }
                int g = nodes[i].g;
                if (g == 2 || g == 6) {
                    Bits f = nodes[i].f;
                    nodes.erase(nodes.begin() + (long)i);
                    e0 -= 1;
                    phase = (phase + (g == 2 ? 1 : 7)) & 7;
                    add_lin(g == 2 ? 6 : 2, f, 0);
                    again = true;
                    break;
                }
                if ((g == 0 || g == 4) && !internal(nodes[i].f).any()) {
                    // a condition on the parameters: kept (see constrain);
                    // the same condition with the opposite value is zero
                    for (size_t j = i + 1; j < nodes.size(); j++)
                        if (nodes[j].f == nodes[i].f && ((nodes[j].g - g) & 7) == 4) zero = true;
                    continue;
                }
                if (g == 0 || g == 4) {
                    Bits f = nodes[i].f;
                    nodes.erase(nodes.begin() + (long)i);
                    e0 -= 2;
                    constrain(f, g == 4 ? 1 : 0);
                    again = true;
                    break;
                }
                for (size_t j = i + 1; j < nodes.size(); j++) {
                    if ((nodes[i].g & 1) && nodes[j].f == nodes[i].f && ((nodes[j].g - nodes[i].g) & 7) == 4) {
                        int gi = nodes[i].g;
                        nodes.erase(nodes.begin() + (long)j);
                        nodes.erase(nodes.begin() + (long)i);
                        // 1 - w^(2g) for odd g: 1 - i or 1 + i
                        int two_g = (2 * gi) & 7;  // 2 or 6
                        e0 -= 1;
                        phase = (phase + (two_g == 2 ? 7 : 1)) & 7;
                        again = true;
                        break;
                    }
                }
            }
        }
    }

    void remove_var_from_graph(int v) {
        adj[(size_t)v].each([&](int j) { adj[(size_t)j].clr(v); });
        adj[(size_t)v] = Bits(nw);
        sing[(size_t)v] = 0;
        live[(size_t)v] = 0;
    }

    // sum over a free variable with even coefficient (local complementation
    // for c = 2, 6; pivot for c = 0, 4)
    void elim_clifford(int v) {
        int c = sing[(size_t)v];
        Bits N = adj[(size_t)v];
        remove_var_from_graph(v);
        if (c == 2 || c == 6) {
            // 1 + w^(c + 4 l) = sqrt2 w^(+-1) w^(-+2 l)
            e0 -= 1;
            phase = (phase + (c == 2 ? 1 : 7)) & 7;
            add_lin(c == 2 ? 6 : 2, N, 0);
        } else {
            // 1 + w^(c + 4 l) = 2 [l = c/4]
            e0 -= 2;
            constrain(N, c == 4 ? 1 : 0);
        }
    }

    // sum over a free variable with odd coefficient: node 1 + w^(c + 4 l(N))
    void elim_node(int v) {
        int c = sing[(size_t)v];
        Bits N = adj[(size_t)v];
        remove_var_from_graph(v);
        add_node(c, N);
    }

    // sum over two adjacent free variables with odd coefficients: Eq. 3
    void elim_pair(int u, int w) {
        int a = sing[(size_t)u], b = sing[(size_t)w];
        Bits la = adj[(size_t)u], lb = adj[(size_t)w];
        la.clr(w);
        lb.clr(u);
        remove_var_from_graph(u);
        remove_var_from_graph(w);
        if (!la.any() && !lb.any()) {
            const_pairs.push_back(PairF{a, la, b, lb});
            return;
        }
        pairs.push_back(PairF{a, la, b, lb});
    }

    // w^l = 1/2 sum_a (1 + w^(1 + 4a)) (-1)^(a l)
    void decompose(Bits form) {
        tf.erase(form);
        int a = new_var();          // may grow every bitset
        form.resize(nw);
        Bits fa = unit(a);
        nodes.push_back(NodeF{1, fa});
        add_quad(fa, 0, form, 0);
        e0 += 2;
    }

    // ------------------------------------------------------------------
    // the reduction loop
    // ------------------------------------------------------------------
    // w^(c y_v) = 1/2 sum_a (1 + w^(c + 4a)) (-1)^(a y_v): the odd phase of a
    // T-like spider moves onto a new parameter a; y_v becomes Clifford.
    void decompose_sing(int v) {
        int c = sing[(size_t)v];
        sing[(size_t)v] = 0;
        int a = new_var();
        nodes.push_back(NodeF{c, unit(a)});
        toggle_edge(a, v);
        e0 += 2;
    }

    // Change of variables y_p := y_p xor y_q (a bijection of the summation
    // domain): every form holding p gains q; the Clifford terms of p are
    // rewritten.  On the matrix of factor forms it adds column p to column q.
    void shear(int p, int q) {
        std::vector<Bits> hit;
        for (auto& f : tf) if (f.get(p)) hit.push_back(f);
        for (auto& f : hit) tf.erase(f);
        for (auto& n : nodes) if (n.f.get(p)) n.f.flip(q);
        for (auto& pr : pairs) {
            if (pr.fa.get(p)) pr.fa.flip(q);
            if (pr.fb.get(p)) pr.fb.flip(q);
        }
        for (size_t w = 0; w < qf.size(); w++) if (qf[w].get(p)) qf[w].flip(q);
        // 4 y_p y_j -> 4 y_p y_j + 4 y_q y_j
        Bits nb = adj[(size_t)p];
        nb.each([&](int j) {
            if (j == q) sing[(size_t)q] = (uint8_t)((sing[(size_t)q] + 4) & 7);
            else toggle_edge(q, j);
        });
        int c = sing[(size_t)p];
        sing[(size_t)p] = 0;
        Bits pq(nw);
        pq.set(p);
        pq.set(q);
        add_lin(c, pq, 0);
        for (auto& f : hit) { Bits g = f; g.flip(q); add_lin(1, g, 0); }
        simplify_nodes();
    }

    // All non-Clifford factor forms (T-forms, odd singletons, node and pair
    // forms) as rows.
    std::vector<Bits> factor_rows() const {
        std::vector<Bits> rows;
        for (auto& f : tf) rows.push_back(f);
        for (int v = 0; v < nvars; v++)
            if (live[(size_t)v] && !ext[(size_t)v] && (sing[(size_t)v] & 1)) rows.push_back(unit(v));
        for (auto& n : nodes) rows.push_back(n.f);
        for (auto& p : pairs) { rows.push_back(p.fa); rows.push_back(p.fb); }
        return rows;
    }

    // Only rank(factor rows) variables need to be summed: reduce the rows to
    // echelon form and shear every non-pivot variable out of all of them,
    // leaving it Clifford.  Returns true if some variable was freed.
    bool compact() {
        std::vector<Bits> rows = factor_rows();
        std::vector<int> piv;
        std::vector<Bits> basis;
        for (auto& r0 : rows) {
            Bits r = internal(r0);      // parameters are not summed: not pivots
            for (size_t i = 0; i < basis.size(); i++)
                if (r.get(piv[i])) r.xor_with(basis[i]);
            int p = r.first();
            if (p < 0) continue;
            // keep the basis reduced: clear p from earlier rows
            for (size_t i = 0; i < basis.size(); i++)
                if (basis[i].get(p)) basis[i].xor_with(r);
            basis.push_back(r);
            piv.push_back(p);
        }
        Bits is_piv(nw);
        for (int p : piv) is_piv.set(p);
        bool freed = false;
        for (int q = 0; q < nvars; q++) {
            if (!live[(size_t)q] || ext[(size_t)q] || is_piv.get(q)) continue;
            bool inrow = false;
            for (auto& b : basis) if (b.get(q)) { inrow = true; break; }
            if (!inrow) continue;     // already free of factor forms
            for (size_t i = 0; i < basis.size(); i++)
                if (basis[i].get(q)) shear(piv[i], q);
            freed = true;
        }
        return freed;
    }

    struct Strategy {
        int node_damage_max;   // node-eliminate only if it locks <= this many free vars
        int pair_damage_max;
        int tform_gain_min;    // decompose a T-form only if it frees >= this many vars
        bool decompose_sings;  // else fall back to the least damaging node
    };

    void reduce(const Strategy& st) {
        for (int iter = 0; iter < 1000000 && !zero; iter++) {
            std::vector<int> locks = lock_counts();
            // 1. Clifford variables
            int cv = -1;
            for (int v = 0; v < nvars; v++)
                if (live[(size_t)v] && !ext[(size_t)v] && !locks[(size_t)v] && !(sing[(size_t)v] & 1)) {
                    cv = v;
                    break;
                }
            if (cv >= 0) { elim_clifford(cv); continue; }
            // 2. free T-like variables: node, pair or decomposition
            Bits freev(nw);
            for (int v = 0; v < nvars; v++)
                if (live[(size_t)v] && !ext[(size_t)v] && !locks[(size_t)v]) freev.set(v);
            if (freev.any()) {
                long nkey = -1, pkey = -1, wkey = -1;
                int nu = -1, pu = -1, pw = -1, wu = -1, ndam = 0, pdam = 0;
                freev.each([&](int v) {
                    int d = adj[(size_t)v].count_and(freev);
                    long r = (long)(mix64(rng) & 63);
                    long key = (long)d * 64 + r;
                    if (nkey < 0 || key < nkey) { nkey = key; nu = v; ndam = d; }
                    long key_w = (long)d * 64 + r;      // most damaging: decompose it
                    if (wkey < 0 || key_w > wkey) { wkey = key_w; wu = v; }
                    // at most kFoldPairs phase-pairs: the kernel folds that many into
                    // its term table; more would need a Z[w] product per pair and term
                    if (!allow_pairs || pairs.size() >= 2) return;
                    adj[(size_t)v].each([&](int w) {
                        if (w <= v || !freev.get(w)) return;
                        Bits un = adj[(size_t)v];
                        un.or_with(adj[(size_t)w]);
                        un.clr(v);
                        un.clr(w);
                        int d2 = un.count_and(freev);
                        long k2 = (long)d2 * 64 + (long)(mix64(rng) & 63);
                        if (pkey < 0 || k2 < pkey) { pkey = k2; pu = v; pw = w; pdam = d2; }
                    });
                });
                if (pu >= 0 && pdam <= st.pair_damage_max && (nu < 0 || pdam - 2 <= ndam - 1)) {
                    elim_pair(pu, pw);
                } else if (nu >= 0 && ndam <= st.node_damage_max) {
                    elim_node(nu);
                } else if (st.decompose_sings) {
                    decompose_sing(wu);
                } else {
                    elim_node(nu);
                }
                continue;
            }
            // 3. every live variable is locked: decompose the T-form that frees most
            if (tf.empty()) {
                if (compact()) continue;
                break;
            }
            long bestkey = -1;
            const Bits* best = nullptr;
            int bestgain = 0;
            for (auto& f : tf) {
                if (!internal(f).any()) continue;   // a phase on the parameters alone
                int gain = 0;
                f.each([&](int v) { if (!ext[(size_t)v] && locks[(size_t)v] == 1) gain++; });
                long key = (long)gain * 64 + (long)(mix64(rng) & 31);
                if (key > bestkey) { bestkey = key; best = &f; bestgain = gain; }
            }
            if (!best || bestgain < st.tform_gain_min) {
                if (compact()) continue;
                break;
            }
            Bits f = *best;
            decompose(f);
        }
    }
};

int count_h(const zxp_gate* g, size_t n) {
    int c = 0;
    for (size_t i = 0; i < n; i++) c += g[i].op == ZXP_H;
    return c;
}

int apply_gate(PathSum& ps, const zxp_gate& g, bool dagger) {
    int q0 = g.q0, q1 = g.q1;
    switch (g.op) {
    case ZXP_H: {
        int y = ps.new_var();
        Bits fy = ps.unit(y);
        Bits f = ps.qf[(size_t)q0];    // copy: qf may be rewritten by new_var growth
        ps.add_quad(f, ps.qc[(size_t)q0], fy, 0);
        ps.qf[(size_t)q0] = fy;
        ps.qc[(size_t)q0] = 0;
        ps.e0 += 1;
        break;
    }
    case ZXP_S: ps.add_lin(dagger ? 6 : 2, ps.qf[(size_t)q0], ps.qc[(size_t)q0]); break;
    case ZXP_SDG: ps.add_lin(dagger ? 2 : 6, ps.qf[(size_t)q0], ps.qc[(size_t)q0]); break;
    case ZXP_T: ps.add_lin(dagger ? 7 : 1, ps.qf[(size_t)q0], ps.qc[(size_t)q0]); break;
    case ZXP_TDG: ps.add_lin(dagger ? 1 : 7, ps.qf[(size_t)q0], ps.qc[(size_t)q0]); break;
    case ZXP_Z: ps.add_lin(4, ps.qf[(size_t)q0], ps.qc[(size_t)q0]); break;
    case ZXP_X: ps.qc[(size_t)q0] ^= 1; break;
    case ZXP_CNOT:
        ps.qf[(size_t)q1].xor_with(ps.qf[(size_t)q0]);
        ps.qc[(size_t)q1] ^= ps.qc[(size_t)q0];
        break;
    case ZXP_CZ: {
        Bits a = ps.qf[(size_t)q0], b = ps.qf[(size_t)q1];
        ps.add_quad(a, ps.qc[(size_t)q0], b, ps.qc[(size_t)q1]);
        break;
    }
    default: return ZXP_EINVAL;
    }
    return ZXP_OK;
}

struct Result {
    PPS ps;
    int status = ZXP_OK;
    long score = 0;
};

// Materialise the global factor w^phase (1+sqrt2)^N (1-w)^v / sqrt2^e0
// with small integer coefficients.
void finish_global(PathSum& s, PPS& ps) {
    int h = s.v1w / 2;                     // (1 - w)^2 = sqrt2 (1+sqrt2)^-1 w^5
    int e0 = s.e0 - h;
    int N = s.unitN - h;
    int ph = (s.phase + 5 * h) & 7;
    // keep |N| small: (1+sqrt2) = (1+w)(1+w^7)/sqrt2, (sqrt2-1) = (1+w^3)(1+w^5)/sqrt2
    while (N > 24) { ps.node.push_back({0, 0, 1}); ps.node.push_back({0, 0, 7}); e0 += 1; N--; }
    while (N < -24) { ps.node.push_back({0, 0, 3}); ps.node.push_back({0, 0, 5}); e0 += 1; N++; }
    zw64 G = zw_wpow((unsigned)ph);
    if (N > 0) G = zw_mul(G, zw_pow(zw_silver(), (unsigned)N));
    if (N < 0) G = zw_mul(G, zw_pow(zw_silver_inv(), (unsigned)-N));
    if (s.v1w & 1) G = zw_mul(G, zw_make(1, (uint64_t)-1, 0, 0));
    while (e0 < 0) { G = zw_mul_sqrt2(G); e0++; }
    for (int i = 0; i < 4; i++) ps.G[i] = (int64_t)G.c[i];
    ps.e0 = e0;
}

// One reduction.  param_q (nullable): qubits whose output bit (kind 0) or
// projected bit (kind 1, inside marg_mask) is a parameter instead of
// out_bits[q]; parameter j is the j-th such qubit in ascending order.
Result run_once(const zxp_gate* gates, size_t n_gates, int n, const uint8_t* in_bits,
                const uint8_t* out_bits, const uint8_t* param_q, uint64_t marg_mask, int kind,
                uint64_t seed, const PathSum::Strategy& strat, bool allow_pairs) {
    Result res;
    int nh = count_h(gates, n_gates) * (kind == 1 ? 2 : 1);
    PathSum s(n, nh + 64);
    s.rng = seed;
    s.allow_pairs = allow_pairs;
    std::vector<int> pvar((size_t)n, -1);
    std::vector<int> params;
    for (int q = 0; q < n; q++)
        if (param_q && param_q[q] && (kind == 0 || ((marg_mask >> q) & 1))) {
            pvar[(size_t)q] = s.new_param();
            params.push_back(q);
        }
    for (int q = 0; q < n; q++) s.qc[(size_t)q] = in_bits ? (in_bits[q] & 1) : 0;
    for (size_t i = 0; i < n_gates; i++) apply_gate(s, gates[i], false);
    // the output constraint of qubit q: its wire equals the bit (or parameter)
    auto out_form = [&](int q) {
        Bits f = s.qf[(size_t)q];
        f.resize(s.nw);
        if (pvar[(size_t)q] >= 0) f.flip(pvar[(size_t)q]);
        return f;
    };
    auto out_value = [&](int q) { return pvar[(size_t)q] >= 0 ? 0 : (out_bits[q] & 1); };
    if (kind == 0) {
        for (int q = 0; q < n && !s.zero; q++) {
            Bits f = out_form(q);
            s.constrain(f, s.qc[(size_t)q] ^ out_value(q));
        }
    } else {
        for (int q = 0; q < n && !s.zero; q++) {
            if (!((marg_mask >> q) & 1)) continue;
            Bits f = out_form(q);
            int b = out_value(q);
            s.constrain(f, s.qc[(size_t)q] ^ b);
            s.qf[(size_t)q] = pvar[(size_t)q] >= 0 ? s.unit(pvar[(size_t)q]) : Bits(s.nw);
            s.qc[(size_t)q] = (uint8_t)b;
        }
        for (size_t i = n_gates; i-- > 0 && !s.zero;) apply_gate(s, gates[i], true);
        for (int q = 0; q < n && !s.zero; q++) {
            Bits f = s.qf[(size_t)q];
            s.constrain(f, s.qc[(size_t)q] ^ (in_bits ? (in_bits[q] & 1) : 0));
        }
    }
    if (!s.zero) {
        s.simplify_nodes();
        s.reduce(strat);
    }
    PPS& ps = res.ps;
    ps.p = (uint32_t)params.size();
    for (int q : params) ps.param_qubit.push_back((uint32_t)q);
    if (s.zero) {
        ps.k = 0;
        ps.e0 = 0;
        ps.G[0] = ps.G[1] = ps.G[2] = ps.G[3] = 0;
        ps.zero = true;
        res.score = 0;
        return res;
    }
    // order the remaining summed variables: fewest forms first (the low
    // Gray-code bits flip most often)
    std::vector<int> locks = s.lock_counts();
    std::vector<int> vars;
    for (int v = 0; v < s.nvars; v++) if (s.live[(size_t)v] && !s.ext[(size_t)v]) vars.push_back(v);
    if (vars.size() > 62) { res.status = ZXP_ETOOBIG; res.score = 1L << 40; return res; }
    std::stable_sort(vars.begin(), vars.end(), [&](int a, int b) {
        return locks[(size_t)a] < locks[(size_t)b];
    });
    std::vector<int> idx((size_t)s.nvars, -1), pidx((size_t)s.nvars, -1);
    for (size_t i = 0; i < vars.size(); i++) idx[(size_t)vars[i]] = (int)i;
    for (size_t j = 0; j < params.size(); j++) pidx[(size_t)pvar[(size_t)params[j]]] = (int)j;
    auto mask_x = [&](const Bits& b) {
        uint64_t m = 0;
        b.each([&](int v) { if (idx[(size_t)v] >= 0) m |= 1ull << idx[(size_t)v]; });
        return m;
    };
    auto mask_b = [&](const Bits& b) {
        uint64_t m = 0;
        b.each([&](int v) { if (pidx[(size_t)v] >= 0) m |= 1ull << pidx[(size_t)v]; });
        return m;
    };
    ps.k = (uint32_t)vars.size();
    for (size_t i = 0; i < vars.size(); i++) {
        int v = vars[i];
        if (s.sing[(size_t)v]) ps.lin.push_back({1ull << i, 0, s.sing[(size_t)v]});
    }
    for (size_t j = 0; j < params.size(); j++) {
        int v = pvar[(size_t)params[j]];
        if (s.sing[(size_t)v]) ps.lin.push_back({0, 1ull << j, s.sing[(size_t)v]});
    }
    for (auto& f : s.tf) ps.lin.push_back({mask_x(f), mask_b(f), 1});
    // 4 y_v (sum of its neighbours): summed rows take their later summed
    // neighbours and all parameter neighbours, parameter rows their later
    // parameter neighbours
    for (size_t i = 0; i < vars.size(); i++) {
        const Bits& row = s.adj[(size_t)vars[i]];
        uint64_t upper = mask_x(row) & ~((2ull << i) - 1), rb = mask_b(row);
        if (upper || rb) ps.quad.push_back({1ull << i, 0, upper, rb});
    }
    for (size_t j = 0; j < params.size(); j++) {
        uint64_t upper = mask_b(s.adj[(size_t)pvar[(size_t)params[j]]]) & ~((2ull << j) - 1);
        if (upper) ps.quad.push_back({0, 1ull << j, 0, upper});
    }
    for (auto& nd : s.nodes) ps.node.push_back({mask_x(nd.f), mask_b(nd.f), (uint32_t)nd.g});
    for (auto& p : s.pairs)
        ps.pair.push_back({mask_x(p.fa), mask_b(p.fa), mask_x(p.fb), mask_b(p.fb), (uint32_t)p.a, (uint32_t)p.b});
    for (auto& p : s.const_pairs) ps.pair.push_back({0, 0, 0, 0, (uint32_t)p.a, (uint32_t)p.b});
    finish_global(s, ps);
    // score: terms first, then per-term work
    res.score = ((long)ps.k << 20) + (long)ps.pair.size() * 64 + (long)(ps.node.size() + ps.lin.size());
    return res;
}

int compile_impl(const zxp_gate* gates, size_t n_gates, int n, const uint8_t* in_bits,
                 const uint8_t* out_bits, const uint8_t* param_q, uint64_t marg_mask, int kind,
                 const CompileOptions& opt, PPS* out) {
    if (n < 1 || n > 65535 || (!gates && n_gates) || !out_bits || !out) return ZXP_EINVAL;
    if (kind != 0 && kind != 1) return ZXP_EINVAL;
    if (kind == 1 && n > 64) return ZXP_EINVAL;
    uint32_t tcount = 0;
    for (size_t i = 0; i < n_gates; i++) {
        const zxp_gate& g = gates[i];
        if (g.op > ZXP_CZ || g.q0 >= n) return ZXP_EINVAL;
        if ((g.op == ZXP_CNOT || g.op == ZXP_CZ) && (g.q1 >= n || g.q1 == g.q0)) return ZXP_EINVAL;
        tcount += (g.op == ZXP_T || g.op == ZXP_TDG);
    }
    if (param_q) {
        int np = 0;
        for (int q = 0; q < n; q++) np += param_q[q] && (kind == 0 || ((marg_mask >> q) & 1));
        if (np > 64) return ZXP_EINVAL;
    }
    Result best;
    best.status = ZXP_ETOOBIG;
    best.score = -1;
    uint64_t seed = opt.seed;
    int tries = std::max(1, opt.tries);
    for (int t = 0; t < tries; t++) {
        static const PathSum::Strategy kStrategies[] = {
            {0, 1, 2, true}, {1, 2, 2, true}, {0, 0, 1, true}, {1000, 1000, 2, false},
            {2, 3, 2, true}, {0, 1, 1, true}, {1, 1, 0, true}, {1000, 1000, 1, false},
        };
        PathSum::Strategy strat = kStrategies[t % 8];
        Result r = run_once(gates, n_gates, n, in_bits, out_bits, param_q, marg_mask, kind,
                            mix64(seed), strat, opt.allow_pairs);
        if (r.status != ZXP_OK) continue;
        if (best.score < 0 || r.score < best.score) best = std::move(r);
    }
    if (best.score < 0) return ZXP_ETOOBIG;
    best.ps.t_count = tcount * (kind == 1 ? 2u : 1u);
    *out = std::move(best.ps);
    return ZXP_OK;
}

}  // namespace

int compile_circuit(const zxp_gate* gates, size_t n_gates, int n, const uint8_t* in_bits,
                    const uint8_t* out_bits, uint64_t marg_mask, int kind,
                    const CompileOptions& opt, PS* out) {
    if (!out) return ZXP_EINVAL;
    PPS pps;
    int st = compile_impl(gates, n_gates, n, in_bits, out_bits, nullptr, marg_mask, kind, opt, &pps);
    if (st != ZXP_OK) return st;
    bind(pps, 0, out);
    if (opt.split && out->k >= opt.split_opt.min_k) {
        PS sp;
        if ((st = split_scalar(*out, opt.split_opt, &sp)) != ZXP_OK) return st;
        *out = std::move(sp);
    }
    return ZXP_OK;
}

int compile_circuit_param(const zxp_gate* gates, size_t n_gates, int n, const uint8_t* in_bits,
                          const uint8_t* out_bits, const uint8_t* param_qubits, uint64_t marg_mask,
                          int kind, const CompileOptions& opt, PPS* out) {
    if (!param_qubits) return ZXP_EINVAL;
    return compile_impl(gates, n_gates, n, in_bits, out_bits, param_qubits, marg_mask, kind, opt, out);
}

}  // namespace zxp
