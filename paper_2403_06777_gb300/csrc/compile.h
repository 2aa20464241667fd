// compile.h -- reduce a Clifford+T circuit amplitude (or a doubled-diagram
// marginal) to a parametric scalar in Boolean decomposition parameters.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include "param.h"
#include "ps.h"
#include "split.h"

struct zxp_gate;

namespace zxp {

struct CompileOptions {
    int tries = 8;            // randomized reduction orders; the smallest k wins
    bool allow_pairs = true;  // emit phase-pair rows (Eq. 3) for adjacent T-like pairs
    uint64_t seed = 0x5eed;
    bool split = false;       // sum inner parameters inside each term (split.h)
    SplitOptions split_opt;
};

struct CompileStats {
    uint32_t k = 0, nodes = 0, lin = 0, quad = 0, pairs = 0;
    int32_t e0 = 0;
};

// kind 0: <out|C|in>; kind 1: <in|C^dag (|b><b|_mask (x) I) C|in>.
int compile_circuit(const zxp_gate* gates, size_t n_gates, int n_qubits,
                    const uint8_t* in_bits, const uint8_t* out_bits, uint64_t marg_mask,
                    int kind, const CompileOptions& opt, PS* out);

// The same reduction with the bits of the qubits flagged in param_qubits
// (n_qubits entries; for kind 1 only those inside marg_mask count) left as
// parameters (at most 64); out_bits gives the other qubits' bits.
int compile_circuit_param(const zxp_gate* gates, size_t n_gates, int n_qubits,
                          const uint8_t* in_bits, const uint8_t* out_bits,
                          const uint8_t* param_qubits, uint64_t marg_mask, int kind,
                          const CompileOptions& opt, PPS* out);

}  // namespace zxp
