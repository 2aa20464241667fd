// param.h -- parametric scalars: the paper's own setting (Sec. 3, Sec. 4),
// where some output (or marginal) bits of the circuit stay Boolean
// parameters b through the whole reduction, so that one reduction serves
// every bitstring.  Rows carry two masks: over the summed variables x
// (k bits) and over the parameters b (p bits).  Binding b turns every
// parity l(x, b) = l_x(x) xor l_b(b) into l_x(x) xor beta with a constant
// beta, which yields an ordinary scalar (ps.h):
//   linear   c (l xor beta)            = c l + c beta - 2 c beta l
//            (beta = 1: w^c and coefficient -c)
//   quadratic 4 (lA xor alpha)(lB xor beta)
//            = 4 lA lB + 4 alpha lB + 4 beta lA + 4 alpha beta   (mod 8)
//   node     1 + w^(g + 4 (l xor beta)) = node (g + 4 beta) on l
//   pair     constants a + 4 beta_a, b + 4 beta_b on the x parts
#pragma once
#include <stdint.h>

#include <vector>

#include "ps.h"

namespace zxp {

struct PLin { uint64_t mx, mb; uint32_t c; };
struct PQuad { uint64_t ax, ab, bx, bb; };           // 4 lA lB
struct PNode { uint64_t mx, mb; uint32_t g; };
struct PPair { uint64_t mxa, mba, mxb, mbb; uint32_t a, b; };

struct PPS {
    uint32_t k = 0;            // summed variables
    uint32_t p = 0;            // parameters (bit j of a binding = parameter j)
    int32_t e0 = 0;
    int64_t G[4] = {1, 0, 0, 0};
    std::vector<PLin> lin;
    std::vector<PQuad> quad;
    std::vector<PNode> node;
    std::vector<PPair> pair;
    std::vector<uint32_t> param_qubit;   // qubit of parameter j
    uint32_t t_count = 0;
    bool zero = false;         // identically zero for every binding
};

// The ordinary scalar for parameter values `bits` (bit j = parameter j).
void bind(const PPS& pps, uint64_t bits, PS* out);

}  // namespace zxp
