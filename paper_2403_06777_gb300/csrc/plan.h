// plan.h -- a parametric scalar rewritten for the sum kernel.
//
// The kernel tracks, per assignment x, one bit per "form" (a parity of x,
// optionally inverted) in NW = NWN + NWL 32-bit words:
//   node words  [0, NWN):        one bit per odd-constant node, set when the
//                                node takes the larger of its two magnitudes
//                                (effective exponent 1 or 7)
//   other words [NWN, NWN+NWL):  linear forms (coefficient bit-planes C0, C1,
//                                C2), zero forms (Z: a set bit zeroes the
//                                term) and phase-pair forms.
// With M = number of set node bits and
//   J = sum_lin c l + 4 (quadratic part) + 4 (set class-B node bits)  mod 8,
// every term equals  K * w^(J + 2M) (1 + sqrt2)^M * prod_pairs PV  where K is
// one constant for the whole sum, because every odd node satisfies
//   1 + w^e = (1 - w) w^j_e (1 + sqrt2)^beta_e,
//   (j, beta) = (2,1), (3,0), (0,0), (1,1) for e = 1, 3, 5, 7.
#pragma once
#include <stdint.h>

#include <memory>
#include <vector>

#include "ps.h"
#include "zring.h"

namespace zxp {

constexpr int kMaxK = 62;
constexpr int kMaxWordsNode = 4;
constexpr int kMaxWordsOther = 4;
constexpr int kMaxNW = kMaxWordsNode + kMaxWordsOther;
constexpr int kMaxPairs = 32;
constexpr int kFoldPairs = 2;        // phase-pairs folded into the term table

// Words of one variable's step row: its flip row F_i (NW = nwn + nwl words),
// F_i & C0 and F_i & C1 on the linear words (2 nwl), and the constant S_i
// (padded to a multiple of 4 words).
ZXP_HD constexpr uint32_t row_words(int nwn, int nwl) {
    return ((uint32_t)(nwn + 3 * nwl + 1) + 3u) & ~3u;
}
constexpr int kMaxRowWords = (int)row_words(kMaxWordsNode, kMaxWordsOther);
// Block lookup (variant 9): at most this many forms may hold one of the
// variables 0, 1, 2 (the lookup has 2^bits entries of 8 bytes), and the
// counters span kLutRows rows of the term table.  Entry u is stored at
// lut_slot(u): bits 4-11 of u are folded into bits 0-3 (an involution), so
// that lanes whose u differ only in high bits read different bank pairs.
constexpr int kLutMaxBits = 10;
constexpr int kLutRows = 24;
// With lane-private counters the forms may be split over two lookup tables
// whose entries add (each form's share of an entry depends on its own bit
// only): up to 2 * kLutMaxBits forms.
constexpr int kLut2MaxBits = 2 * kLutMaxBits;
// Block lookup with lane-private counters (variant 11): a lane's counters are
// indexed by (J mod 8) * 2^kLaneRowShift + M (M <= 7: at most 7 odd nodes).
constexpr int kLaneRowShift = 3;
constexpr int kLaneCounters = 8 << kLaneRowShift;
ZXP_HD constexpr uint32_t lut_slot(uint32_t u) { return u ^ (((u >> 4) ^ (u >> 8)) & 15u); }

// Passed by value as the kernel parameter block (kept in the constant bank).
struct KernelParams {
    uint32_t k;
    uint32_t nbits;          // 32 * (NWN + NWL) form bits (unused bits stay 0)
    uint32_t npairs;
    uint32_t tab_stride;     // m_odd + 1
    uint32_t tab_size;       // table entries: 8 * tab_stride << xshift
    // Extra table index bits below (J, M): the bits of up to kFoldPairs
    // phase-pair forms (first other word, bits 0 .. 2 np - 1) and one bit
    // for "some zero form is set" (bit zshift).  idx =
    //   ((J * tab_stride + M) << xshift) | (L[NWN] & pmask) | (zero << zshift)
    uint32_t xshift, pmask, zshift, has_zero;
    uint32_t CB[kMaxWordsNode];                       // class-B node bits
    uint32_t C0[kMaxWordsOther], C1[kMaxWordsOther], C2[kMaxWordsOther], Z[kMaxWordsOther];
    uint32_t INV[kMaxNW];    // initial inversion of each form bit
    uint16_t PA[kMaxPairs], PB[kMaxPairs];            // bit positions of pair forms
    uint32_t R[4][kMaxRowWords];                      // step rows of variables 0, 1, 2, 3
    // block lookup: forms holding variable 0, 1 or 2 are node bits [0, lut_nn)
    // and linear bits [lut_shift, lut_shift + lut_no) of the first other word
    // (after the phase-pair bits)
    uint32_t lut_no, lut_nn, lut_shift;
    uint32_t lut_tsh;        // variant 11: log2 of the counter row stride (kLaneRowShift)
    // two lookup tables (variant 13): the first lut_na bits of the lookup
    // index u (linear form bits, then node form bits) select an entry of
    // the first table, the rest one of the second; 0 with one table
    uint32_t lut_na;
    uint32_t lut_entries;    // 64-bit words of the lookup: its table(s) and the 8 quadratic entries
    uint64_t A4[4];          // adjacency rows of variables 0..3 (0 beyond k)
    // variant 11: bytes between a lane's consecutive counters (32 lanes x 4
    // bytes).  A parameter rather than a constant, so that the counter
    // address is one multiply-add (not a shift and an add on the integer
    // ALU, the kernel's busiest pipe).
    uint32_t lane_row_bytes;
    // block lookup: the lookup slot changes of variables 0..3 (see rows)
    uint32_t U4[4];
    // Inner parameters (PS::k_inner > 0): the sum over the inner parameters
    // is the table ftab, indexed by the cut parities zq of the outer
    // assignment.  A lane folds the terms it counted while zq was constant,
    // multiplies them by ftab[zq] and adds; flipping outer variable
    // i >= zq_lo XORs zqcol[i] into zq.  zq_lo = 64 without inner parameters.
    uint32_t zq_lo;
    const uint32_t* zqcol;   // device addresses, set at launch
    const zw64* ftab;
    // Bytes the table copies' barrier expects beyond those the copies
    // deliver: 0, or 16 when a test makes every block's bounded wait run out
    // (zxp_test_table_timeout).  The copies themselves are unchanged, so they
    // have landed long before the wait gives up.
    uint32_t extra_tx;
    // Lane-private block lookup over a range whose start, length and slices
    // are multiples of 256 (variables 6 and 7 below every cut parity): set
    // at launch, every thread walks each slice as four states that differ in
    // variables 6 and 7, along one Gray code of the other variables.
    uint32_t pair_walk;
};

// each wait suspends the thread for a bounded time (about 4 us measured on a
// GB300): this many of them are about a second in all, against microseconds
// for any table copy
constexpr uint32_t kDefaultWaitTries = 1u << 18;
// extra_tx for the launches queued now (api.cu)
uint32_t test_extra_tx();

struct Plan {
    int nwn = 0, nwl = 0;           // node / other words
    uint32_t m_odd = 0;
    KernelParams kp;
    std::vector<uint32_t> frows;    // k x NW: form bits holding variable i (flip rows)
    // k x row_words: step rows.  Flipping variable i changes the phase
    // exponent J = sum_lin c l + 4 (class-B node bits) by
    //   S_i - 2 |L & F_i & C0| - 4 |L & F_i & C1|  (mod 8, L before the flip)
    // with S_i = sum of c over the forms F_i holds + 4 per class-B node it holds.
    // The row's last word holds S_i in bits 0-2 and, with the block lookup,
    // the change of the block's lookup slot in bits 8 and up (the slot of
    // the forms F_i holds among those the lookup reads, lut_slot being
    // linear); only J mod 8 is ever used, so the high bits may ride along.
    std::vector<uint32_t> rows;
    uint32_t row_stride = 0;
    std::vector<uint64_t> adj;      // k: quadratic part 4 sum_{i<j} A_ij x_i x_j, row i
    // Seek tables, per 4-bit group b of x and value v (ceil(k/4) x 16 entries
    // of seek_stride words): XOR of the flip rows of v's bits, XOR of their
    // adjacency rows (two words), and the quadratic bit of v inside the group.
    std::vector<uint32_t> seek;
    uint32_t seek_stride = 0;
    std::vector<zw64> table;        // w^(J + 2M) (1 + sqrt2)^M x pair values x (1 - zero)
    std::vector<zw64> pv;           // 4 per pair: value at (lA, lB) = (b & 1, b >> 1)
    zw64 K;                         // constant factor, G included
    // The same values modulo 2^128 (exact sums for 124 < e0 <= 252): the
    // term table indexed by (J, M) alone, w^(J + 2M) (1 + sqrt2)^M at
    // J * tab_stride + M (phase-pair values and zero forms are applied per
    // term), the pair values and the constant.
    std::vector<zw128> table_w;
    std::vector<zw128> pv_w;
    zw128 K_w;
    int32_t e0 = 0;
    bool zero = false;              // the scalar is identically zero
    bool has_zero = false;          // some term can vanish (zero forms present)
    bool general = false;           // more phase-pairs than fold into the table
    // Block lookup for aligned blocks of 8 Gray steps (variables 0,1,0,2,0,1,0
    // flip): entry u (the block's first-state bits of the forms holding
    // variables 0-2) holds, in byte s-1 for s = 1..7, the offset of term s's
    // counter from the block's base, dJ_s * stride + dM_s + lut_nn, and in
    // byte 7 dJ_7; the 8 entries after them, indexed by the three bits h of
    // A x for variables 0-2, add the quadratic part 4 Q_s * stride (byte 7:
    // 4 Q_7).  With lut_lane (no phase-pair or zero forms, at most 7 odd
    // nodes) the row stride in the offsets is 2^lut_tsh instead of
    // m_odd + 1 and bytes 0-6 hold (dJ_s * stride + dM_s) mod 8 * 2^lut_tsh,
    // so that a counter index (J mod 8) * 2^lut_tsh + M is the sum of the
    // block's base and the offset taken modulo 8 * 2^lut_tsh.
    bool lut_ok = false;
    bool lut_lane = false;
    bool lut_two = false;           // two tables (lane-private counters only)
    std::vector<uint64_t> lut;
    // Inner parameters: the scalar's outer rows are this plan; `inner` is the
    // plan of the product of its inner and crossing rows as a function of
    // u = (inner parameters, cut bits), inner_bits = |u| bits.  The inner
    // table is the Walsh-Hadamard transform of that product over the inner
    // parameters' bits of u.  zqcol[i] (outer variable i < k): the cut bits
    // that flipping i changes.
    uint32_t k_inner = 0, inner_bits = 0;
    std::vector<uint32_t> zqcol;
    std::shared_ptr<const Plan> inner;
    // The inner plan's state for the low min(inner_bits, 11) bits of u: per
    // value e, the XOR of their flip rows (inner nw words) and the quadratic
    // bit of e (one more word); a block of the inner table combines it with
    // its high bits' state.  (The inner plan's table already includes its
    // constant K.)
    std::vector<uint32_t> inner_low;
};

// Low bits of u tabulated for the inner table (a block's 2^11 entries).
constexpr uint32_t kInnerLowBits = 11;

// Largest inner table index (inner parameters + crossing forms).
constexpr uint32_t kMaxInnerBits = 26;

// Returns 0 or ZXP_ETOOBIG (more forms / pairs than the kernel supports).
int build_plan(const PS& ps, Plan* out);

}  // namespace zxp
