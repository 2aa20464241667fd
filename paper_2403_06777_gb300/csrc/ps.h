// ps.h -- the parametric scalar (Eq. 2 of the paper, with Boolean
// decomposition parameters x in {0,1}^k) and its table layout.
//
//   value = G / sqrt2^e0 * sum_x  w^(sum_lin c l(x) + 4 sum_quad lA(x) lB(x))
//                               * prod_node (1 + w^(g + 4 l(x)))
//                               * prod_pair (1 + w^(a+4lA) + w^(b+4lB) - w^(a+b+4(lA^lB)))
//
// l(x) = parity(mask & x).  The row kinds are the subterm types of App. C:
// linear rows are pi-pairs with a fixed Psi = c pi/4, quadratic rows are
// pi-pairs of two parametric phases, nodes are 1 + e^{i Psi}, pairs are the
// phase-pair normal form of Eq. 3.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <vector>

namespace zxp {

struct LinRow { uint64_t mask; uint32_t c; };
struct QuadRow { uint64_t a, b; };
struct NodeRow { uint64_t mask; uint32_t g; };
struct PairRow { uint64_t ma, mb; uint32_t a, b; };

struct PS {
    uint32_t k = 0;
    // The last k_inner of the k parameters are inner ones: a term index
    // runs over the first k - k_inner, and each term is summed over every
    // value of the inner parameters (the full sum is unchanged).
    uint32_t k_inner = 0;
    int32_t e0 = 0;
    int64_t G[4] = {1, 0, 0, 0};
    std::vector<LinRow> lin;
    std::vector<QuadRow> quad;
    std::vector<NodeRow> node;
    std::vector<PairRow> pair;
    uint32_t t_count = 0;   // T-like gates of the source circuit (0 for tables)
};

constexpr uint32_t kPsMagic = 0x5350585Au;
constexpr uint32_t kPsVersion = 1;
constexpr uint32_t kPsVersionInner = 2;   // header followed by {u32 k_inner, u32 0}

// Parse and validate a table blob; returns 0 or a negative zxp_status.
int ps_from_blob(const void* blob, size_t nbytes, PS* out);
size_t ps_blob_size(const PS& ps);
void ps_to_blob(const PS& ps, void* buf);

// The same scalar with its parameters relabelled so that the four that
// touch the fewest parity forms (phase-pair and zero-test forms last) come
// first (reorder.cpp); k_inner must be 0 (else ZXP_EINVAL).
int reorder_scalar(const PS& in, PS* out);

}  // namespace zxp
