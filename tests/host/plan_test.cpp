// Host tests of the kernel plan (paper_2403_06777_gb300/csrc/plan.cpp) for
// the scalars whose table blobs are given on the command line.
//
// For every parameter assignment x of a scalar with k <= 12 it prints the
// term the plan encodes, K * T[index(x)] (with the phase-pair values
// multiplied in for the general layout), as four hex words, so that the
// caller can compare them with the oracle's terms.  Where the plan built a
// block lookup it also checks, at every aligned block of 8 Gray steps, that
// the lookup gives each of the 8 terms the counter of its own phase class
// and node count, and that the step rows' lookup-slot changes and the
// parameter copies of the low variables' rows agree with the plan's forms;
// for every scalar, that each variable's step row updates the form bits
// and the phase exponent of sampled states to those of the flipped state.
// For a scalar with inner parameters (outer k <= 12, inner table of at
// most 2^16 entries) it prints instead, for every Gray index t of the
// outer parameters, the outer term times the inner table at the term's cut
// parities, the table built here from the inner plan's terms by a
// Walsh-Hadamard transform over the inner bits.
// Exits 1 with a message on the first failed check.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <fstream>
#include <iterator>
#include <vector>

#include "plan.h"
#include "ps.h"
#include "zring.h"

using namespace zxp;

#define CHECK(c)                                                                  \
    do {                                                                          \
        if (!(c)) {                                                               \
            fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
            exit(1);                                                              \
        }                                                                         \
    } while (0)

namespace {

int popc(uint32_t v) { return __builtin_popcount(v); }

// The plan's state for parameter bits x: the form bits, the phase exponent
// J (mod 8), the node count M and A x.
struct Term {
    std::vector<uint32_t> L;
    uint32_t J, M;
    uint64_t ax;
};

struct Model {
    const Plan& pl;
    uint32_t k, nw, nwn, nwl;
    explicit Model(const Plan& p)
        : pl(p), k(p.kp.k), nw((uint32_t)(p.nwn + (p.nwl < 1 ? 1 : p.nwl))), nwn((uint32_t)p.nwn),
          nwl(nw - (uint32_t)p.nwn) {}

    Term at(uint64_t x) const {
        const KernelParams& kp = pl.kp;
        Term t;
        t.L.assign(nw, 0);
        for (uint32_t w = 0; w < nw; w++) t.L[w] = kp.INV[w];
        t.ax = 0;
        uint32_t q = 0;
        for (uint32_t i = 0; i < k; i++) {
            if (!((x >> i) & 1)) continue;
            for (uint32_t w = 0; w < nw; w++) t.L[w] ^= pl.frows[(size_t)i * nw + w];
            t.ax ^= pl.adj[i];
            q ^= (uint32_t)__builtin_popcountll(pl.adj[i] & x & ((2ull << i) - 1) & ~(1ull << i)) & 1u;
        }
        uint32_t J = 4 * q;
        for (uint32_t w = 0; w < nwn; w++) J += 4 * (uint32_t)popc(t.L[w] & kp.CB[w]);
        for (uint32_t w = 0; w < nwl; w++) {
            const uint32_t v = t.L[nwn + w];
            J += (uint32_t)popc(v & kp.C0[w]) + 2 * (uint32_t)popc(v & kp.C1[w]) + 4 * (uint32_t)popc(v & kp.C2[w]);
        }
        t.J = J & 7;
        t.M = 0;
        for (uint32_t w = 0; w < nwn; w++) t.M += (uint32_t)popc(t.L[w]);
        return t;
    }

    bool bit(const Term& t, uint32_t pos) const { return (t.L[pos >> 5] >> (pos & 31)) & 1; }

    // K * (the term's table value), the phase-pair values multiplied in
    // for the general layout
    zw64 value(const Term& t) const {
        const KernelParams& kp = pl.kp;
        uint32_t z = 0;
        for (uint32_t w = 0; w < nwl; w++) z |= t.L[nwn + w] & kp.Z[w];
        zw64 v;
        if (pl.general) {
            if (z) return zw_zero();
            v = pl.table[t.J * kp.tab_stride + t.M];
            for (uint32_t j = 0; j < kp.npairs; j++) {
                const uint32_t b = (bit(t, kp.PA[j]) ? 1u : 0u) | (bit(t, kp.PB[j]) ? 2u : 0u);
                v = zw_mul(v, pl.pv[4 * j + b]);
            }
        } else {
            uint32_t idx = t.J * kp.tab_stride + t.M;
            idx = (idx << kp.xshift) | (t.L[nwn] & kp.pmask) | ((z ? 1u : 0u) << kp.zshift);
            v = pl.table[idx];
        }
        return zw_mul(pl.K, v);
    }

    // the lookup slot of lookup bits u, and the lookup's entry for them
    // (two tables: the first lut_na bits and the rest, entries added)
    uint32_t slot(uint32_t u) const {
        const uint32_t na = pl.kp.lut_na;
        if (!pl.lut_two) return lut_slot(u);
        return lut_slot(u & ((1u << na) - 1u)) | (lut_slot(u >> na) << na);
    }
    uint64_t entry(uint32_t u) const {
        const uint32_t na = pl.kp.lut_na;
        if (!pl.lut_two) return pl.lut[lut_slot(u)];
        return pl.lut[lut_slot(u & ((1u << na) - 1u))] + pl.lut[((size_t)1 << na) + lut_slot(u >> na)];
    }
    // the index of the 8 quadratic entries
    size_t qbase() const {
        const uint32_t nU = pl.kp.lut_no + pl.kp.lut_nn, na = pl.kp.lut_na;
        return pl.lut_two ? ((size_t)1 << na) + ((size_t)1 << (nU - na)) : (size_t)1 << nU;
    }

    // the lookup's bits of a state (linear forms, then node forms)
    uint32_t lookup_bits(const Term& t) const {
        const KernelParams& kp = pl.kp;
        uint32_t u = (t.L[nwn] >> kp.lut_shift) & ((1u << kp.lut_no) - 1u);
        if (nwn) u |= (t.L[0] & ((1u << kp.lut_nn) - 1u)) << kp.lut_no;
        return u;
    }
};

uint64_t gray(uint64_t t) { return t ^ (t >> 1); }

// Inner table of a plan with inner parameters: every inner term, then the
// transform over the low k_inner bits.
std::vector<zw64> inner_table(const Plan& pl) {
    const Model mi(*pl.inner);
    const uint64_t n = 1ull << pl.inner_bits;
    std::vector<zw64> F(n);
    for (uint64_t u = 0; u < n; u++) F[u] = pl.inner->zero ? zw_zero() : mi.value(mi.at(u));
    for (uint32_t b = 0; b < pl.k_inner; b++)
        for (uint64_t u = 0; u < n; u++)
            if (!((u >> b) & 1)) {
                const zw64 a = F[u], c = F[u | (1ull << b)];
                F[u] = zw_add(a, c);
                F[u | (1ull << b)] = zw_sub(a, c);
            }
    return F;
}

// The step rows: flipping variable i at state x changes J by
// S_i - 2 |L & F_i & C0| - 4 |L & F_i & C1| + 4 (A x)_i (mod 8) and the form
// bits by F_i, for sampled states x and every variable.
void check_step_rows(const Model& m) {
    const Plan& pl = m.pl;
    const uint32_t k = m.k, rw = pl.row_stride, nw = m.nw, nwl = m.nwl, nwn = m.nwn;
    const uint64_t nx = k < 64 ? (1ull << k) : 0;
    const uint64_t step = nx > 256 ? nx / 256 + 1 : 1;
    for (uint64_t x = 0; x < nx; x += step) {
        const Term s0 = m.at(x);
        for (uint32_t i = 0; i < k; i++) {
            const uint32_t* f = &pl.rows[(size_t)i * rw];
            uint32_t d0 = 0, d1 = 0;
            for (uint32_t w = 0; w < nwl; w++) {
                d0 += (uint32_t)popc(s0.L[nwn + w] & f[nw + w]);
                d1 += (uint32_t)popc(s0.L[nwn + w] & f[nw + nwl + w]);
            }
            const uint32_t ai = (uint32_t)(s0.ax >> i) & 1u;
            const Term s1 = m.at(x ^ (1ull << i));
            CHECK(((s0.J + f[nw + 2 * nwl] - 2 * d0 - 4 * d1 + 4 * ai) & 7) == s1.J);
            for (uint32_t w = 0; w < nw; w++) CHECK((s0.L[w] ^ f[w]) == s1.L[w]);
        }
    }
}

void check_lookup(const Model& m) {
    const Plan& pl = m.pl;
    const KernelParams& kp = pl.kp;
    const uint32_t k = m.k, ts = kp.tab_stride;
    CHECK(pl.lut.size() == kp.lut_entries && m.qbase() + 8 == pl.lut.size());
    const uint32_t rw = pl.row_stride, sw = m.nw + 2 * m.nwl;
    // parameter copies of the low variables' step and adjacency rows
    for (uint32_t i = 0; i < 4 && i < k; i++) {
        for (uint32_t w = 0; w < rw; w++) CHECK(kp.R[i][w] == pl.rows[(size_t)i * rw + w]);
        CHECK(kp.A4[i] == pl.adj[i]);
        CHECK(kp.U4[i] == (pl.rows[(size_t)i * rw + sw] >> 8));
    }
    const uint64_t nblocks = k >= 3 ? (1ull << (k - 3)) : 0;
    const uint64_t step = nblocks > 512 ? nblocks / 512 : 1;
    for (uint64_t b = 0; b < nblocks; b += step) {
        const uint64_t t0 = b * 8;
        const Term s0 = m.at(gray(t0));
        const uint32_t u = m.lookup_bits(s0);
        // each variable's step row changes the lookup slot by its slot change
        for (uint32_t i = 0; i < k; i++) {
            const Term s1 = m.at(gray(t0) ^ (1ull << i));
            CHECK((m.slot(m.lookup_bits(s1)) ^ m.slot(u)) == (pl.rows[(size_t)i * rw + sw] >> 8));
        }
        const uint64_t e = m.entry(u) + pl.lut[m.qbase() + (uint32_t)(s0.ax & 7)];
        const Term s7 = m.at(gray(t0 + 7));
        CHECK(((s0.J + (uint32_t)(e >> 56)) & 7) == s7.J);
        for (uint32_t s = 1; s < 8; s++) {
            const Term st = m.at(gray(t0 + s));
            const uint32_t off = (uint32_t)(e >> (8 * (s - 1))) & 0xFFu;
            if (pl.lut_lane) {
                const uint32_t b0 = (s0.J << kLaneRowShift) + s0.M;
                const uint32_t idx = (b0 + off) & ((8u << kLaneRowShift) - 1u);
                CHECK(idx == (st.J << kLaneRowShift) + st.M);
            } else {
                // counter row * ts + m, rows not reduced mod 8 inside a block
                const int c = (int)(s0.J * ts + s0.M) - (int)kp.lut_nn + (int)off;
                CHECK(c >= 0);
                CHECK((uint32_t)c % ts == st.M);
                CHECK(((uint32_t)c / ts) % 8 == st.J);
                CHECK((uint32_t)c / ts < (uint32_t)kLutRows);
            }
        }
    }
}

// The 128-bit values: the constant and pair values reduce to the 64-bit
// ones modulo 2^64, and entry (J, M) of the (J, M) table is
// K w^(J + 2M) (1 + sqrt2)^M (K = 1 except in an inner plan, whose table
// holds its constant), with (1 + sqrt2)^M = a_M + b_M sqrt2 from the
// recurrence a' = a + 2b, b' = a + b modulo 2^128 (sqrt2 = w - w^3:
// coefficients (a, b, 0, -b)) and w^j applied as a cyclic shift with sign
// changes.
void check_wide(const Plan& pl, const zw128& k_folded) {
    const KernelParams& kp = pl.kp;
    CHECK(pl.pv_w.size() == pl.pv.size());
    for (size_t j = 0; j < pl.pv.size(); j++)
        for (int i = 0; i < 4; i++) CHECK((uint64_t)pl.pv_w[j].c[i] == pl.pv[j].c[i]);
    for (int i = 0; i < 4; i++) CHECK((uint64_t)pl.K_w.c[i] == pl.K.c[i]);
    CHECK(pl.table_w.size() == (size_t)8 * kp.tab_stride);
    u128 a = 1, b = 0;
    for (uint32_t M = 0; M <= pl.m_odd; M++) {
        for (uint32_t J = 0; J < 8; J++) {
            zw128 c = zw_make_t<u128>(a, b, 0, (u128)0 - b);
            for (uint32_t r = 0; r < ((J + 2 * M) & 7); r++) {   // times w
                const u128 t = c.c[3];
                c.c[3] = c.c[2]; c.c[2] = c.c[1]; c.c[1] = c.c[0]; c.c[0] = (u128)0 - t;
            }
            const zw128 want = zw_mul(k_folded, c);
            const zw128& v = pl.table_w[(size_t)J * kp.tab_stride + M];
            for (int i = 0; i < 4; i++) CHECK(v.c[i] == want.c[i]);
            // the 64-bit table at pair bits 0 and zero bit 0 (without phase-pair
            // index bits the entries coincide modulo 2^64)
            if (kp.xshift == 0)
                for (int i = 0; i < 4; i++)
                    CHECK((uint64_t)v.c[i] == pl.table[(size_t)J * kp.tab_stride + M].c[i]);
        }
        const u128 a2 = a + 2 * b, b2 = a + b;
        a = a2;
        b = b2;
    }
}

}  // namespace

int main(int argc, char** argv) {
    for (int a = 1; a < argc; a++) {
        std::ifstream in(argv[a], std::ios::binary);
        std::vector<char> blob((std::istreambuf_iterator<char>(in)), {});
        PS ps;
        CHECK(ps_from_blob(blob.data(), blob.size(), &ps) == 0);
        Plan pl;
        CHECK(build_plan(ps, &pl) == 0);
        const Model m(pl);
        printf("scalar %s k %u lookup %d lane %d two %d\n", argv[a], m.k, pl.lut_ok ? 1 : 0, pl.lut_lane ? 1 : 0,
               pl.lut_two ? 1 : 0);
        if (pl.lut_lane) {
            // the lane-private walk folds a run's counts by Horner's rule in
            // u = w + w^2 + w^3: the phase-0 entries must be u^M
            CHECK(pl.kp.xshift == 0);
            zw64 um = zw_one();
            for (uint32_t M = 0; M < pl.kp.tab_stride; M++) {
                for (int c = 0; c < 4; c++) CHECK(pl.table[M].c[c] == um.c[c]);
                um = zw_mul(um, zw_make(0, 1, 1, 1));
            }
        }
        if (pl.k_inner) {
            // the walk's rules: variables 0-3 never change the cut parities
            CHECK(pl.kp.zq_lo >= 4 && (!pl.lut_ok || pl.lut_lane));
            // the inner table's low-bit states: XOR of the flip rows and the
            // quadratic bit of every low value e
            {
                const Plan& in = *pl.inner;
                const uint32_t inw = (uint32_t)(in.nwn + (in.nwl < 1 ? 1 : in.nwl));
                const uint32_t tb = pl.inner_bits < kInnerLowBits ? pl.inner_bits : kInnerLowBits;
                CHECK(pl.inner_low.size() == ((size_t)(inw + 1) << tb));
                for (uint32_t e = 0; e < (1u << tb); e++) {
                    uint32_t q = 0;
                    for (uint32_t w = 0; w < inw; w++) {
                        uint32_t x = 0;
                        for (uint32_t i = 0; i < tb; i++)
                            if ((e >> i) & 1) x ^= in.frows[(size_t)i * inw + w];
                        CHECK(pl.inner_low[(size_t)e * (inw + 1) + w] == x);
                    }
                    for (uint32_t i = 0; i < tb; i++)
                        for (uint32_t j = i + 1; j < tb; j++)
                            if (((e >> i) & 1) && ((e >> j) & 1)) q ^= (uint32_t)((in.adj[i] >> j) & 1);
                    CHECK(pl.inner_low[(size_t)e * (inw + 1) + inw] == q);
                }
            }
            for (uint32_t i = 0; i < m.k && i < 4; i++) CHECK(pl.zqcol[i] == 0);
            if (m.k <= 12 && pl.inner_bits <= 16) {
                const std::vector<zw64> F = inner_table(pl);
                for (uint64_t t = 0; t < (1ull << m.k); t++) {
                    const uint64_t x = gray(t);
                    uint32_t zq = 0;
                    for (uint32_t i = 0; i < m.k; i++)
                        if ((x >> i) & 1) zq ^= pl.zqcol[i];
                    const zw64 v = pl.zero ? zw_zero() : zw_mul(m.value(m.at(x)), F[zq]);
                    printf("%llx %llx %llx %llx\n", (unsigned long long)v.c[0], (unsigned long long)v.c[1],
                           (unsigned long long)v.c[2], (unsigned long long)v.c[3]);
                }
            }
        } else if (m.k <= 12)
            for (uint64_t x = 0; x < (1ull << m.k); x++) {
                const zw64 v = pl.zero ? zw_zero() : m.value(m.at(x));
                printf("%llx %llx %llx %llx\n", (unsigned long long)v.c[0], (unsigned long long)v.c[1],
                       (unsigned long long)v.c[2], (unsigned long long)v.c[3]);
            }
        if (!pl.zero) check_step_rows(m);
        if (pl.lut_ok) check_lookup(m);
        check_wide(pl, zw_one<u128>());
        if (pl.k_inner) check_wide(*pl.inner, pl.inner->table_w[0]);
    }
    printf("ok\n");
    return 0;
}
