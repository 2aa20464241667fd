// split.h -- summing part of a scalar's parameters inside every term.
//
// A parametric scalar (Eq. 2) is a sum over x in {0,1}^k of a product of
// subterms, each a function of one or two parity forms of x.  After a
// change of variables in which the non-Clifford subterms' forms are
// coordinates, the parameters fall into two groups, inner I and outer O,
// such that only Clifford terms couple them (pi-pairs 4 x_I . B x_O) apart
// from a few subterms whose forms cross the cut.  The sum over the inner
// parameters is then, for every outer assignment, a Walsh-Hadamard
// transform of the inner subterms' product, read at the parities B x_O and
// at the outer parts of the crossing forms.  The result is written as a
// version-2 table (PS::k_inner): the same rows in the new variables, outer
// parameters first, with the lowest outer parameters free of every form the
// inner sum depends on, so that the inner sum is constant along aligned
// runs of the Gray-code walk over the outer parameters.
#pragma once
#include <stdint.h>

#include "ps.h"

namespace zxp {

struct SplitOptions {
    uint32_t min_k = 32;           // scalars with fewer parameters are left as they are
    uint32_t max_inner = 22;       // inner parameters
    uint32_t max_index_bits = 24;  // inner parameters + crossing forms (table of 2^bits entries)
    uint32_t max_cut = 3;          // crossing non-Clifford forms
    uint32_t low_free = 8;         // lowest outer parameters no cut form may involve (>= 4)
    int tries = 24;                // randomized change-of-variables / partition attempts
    uint64_t seed = 0x5917d;
};

// *out is a version-2 scalar with the same value when some split lowers the
// number of outer parameters (the one of least estimated device time among
// those found), else a copy of `in`.  `in` must have
// k_inner == 0.  Returns ZXP_OK or ZXP_EINVAL.
int split_scalar(const PS& in, const SplitOptions& opt, PS* out);

}  // namespace zxp
