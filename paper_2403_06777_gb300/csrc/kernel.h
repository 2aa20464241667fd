// kernel.h -- launch interface of the sum kernel (kernel.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "plan.h"

namespace zxp {

// Raise a kernel's dynamic shared memory limit on the current device to at
// least `bytes` (never lowers it: launches of the same kernel with larger
// tables may be in flight from other threads).
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);

// Dynamic shared memory of one block: the w^(J+2M)(1+sqrt2)^M table, the
// phase-pair values and the reduction scratch.
size_t sum_smem_bytes(const Plan& pl);
int sum_threads();
// Kernel variant chosen for a scalar (see zxp_scalar_info_t).
int sum_variant(const Plan& pl);
// Longest slice one thread may take (a multiple of 8).
uint64_t sum_max_span(const Plan& pl);
cudaError_t sum_occupancy(const Plan& pl, int* blocks_per_sm);
// Slice length (a multiple of 8, at least 64 terms) and grid (at most
// max_grid_cap blocks) for `count` terms: one slice per thread of a
// resident grid.
void sum_shape(const Plan& pl, int sm_count, int max_grid_cap, uint64_t count, uint64_t* span, int* grid);

// Device copy of the public result record (same layout as zxp_zomega).
struct DevResult {
    int64_t c[4];
    int32_t e;
    int32_t flags;
};

// Sum Gray-code indices [first, first + count) in slices of `span` terms
// over `grid` blocks.  acc (4 x 64-bit accumulator) and *counter must be 0
// on entry and are 0 again when the kernel ends; *result receives
// K * (sum of the table terms) over sqrt2^e0, flagged raw, its flags word
// written last with a release store (system scope when host_result: a host
// may poll it in pinned memory; else device scope).
// With inner parameters (pl.k_inner > 0), dzq holds the plan's zqcol and
// dftab its inner table (inner_table_launch); both null otherwise.
cudaError_t sum_launch(const Plan& pl, const zw64* dtable, const zw64* dpv, const uint32_t* drows,
                       const uint64_t* dADJ, const uint32_t* dS, const uint32_t* dzq, const zw64* dftab,
                       uint64_t first, uint64_t count, uint64_t span, int grid, zw64* acc,
                       unsigned int* counter, DevResult* result, bool host_result, cudaStream_t stream);

// The inner table of a scalar with inner parameters (inner.cu): 2^bits
// entries (bits = inner.kp.k) at ftab, the Walsh-Hadamard transform over the
// low k_inner bits of the inner product that the plan `inner` describes;
// its term table, phase-pair values, flip rows, adjacency rows and low-bit
// states (Plan::inner_low) are at itab, ipv, ifr, iadj, ilow (device memory).
cudaError_t inner_table_launch(const Plan& inner, uint32_t k_inner, const zw64* itab, const zw64* ipv,
                               const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw64* ftab,
                               cudaStream_t stream);

// ---- 128-bit coefficients (kernel_wide.cu, inner.cu) -------------------------

// Device copy of the public 128-bit result record (zxp_zomega_wide): the
// low and high 64-bit words of each coefficient.
struct DevResultW {
    int64_t c[4];
    int64_t hi[4];
    int32_t e;
    int32_t flags;
};

// The sum of sum_launch modulo 2^128: the per-term walk (table value by
// (J, M), phase-pair values and zero forms applied per term) over the
// plan's rows, adjacency and seek tables (drows, dADJ, dS, the 64-bit upload)
// and its 128-bit values: the (J, M) table Plan::table_w at dtab_w, the pair
// values Plan::pv_w at dpv_w and the inner table (inner_table_launch_wide)
// at dftab_w.  acc (8 x 64-bit words) and *counter must be 0 on entry and
// are 0 again when the kernel ends; *result (device memory) receives
// K_w * (sum) over sqrt2^e0.
cudaError_t sum_launch_wide(const Plan& pl, const zw128* dtab_w, const zw128* dpv_w, const uint32_t* drows,
                            const uint64_t* dADJ, const uint32_t* dS, const uint32_t* dzq, const zw128* dftab_w,
                            uint64_t first, uint64_t count, int sm_count, uint64_t* acc, unsigned int* counter,
                            DevResultW* result, cudaStream_t stream);

// inner_table_launch modulo 2^128: the inner plan's 128-bit (J, M) table
// (inner constant folded in) and pair values at itab_w, ipv_w, the rest as
// for inner_table_launch; 64-byte entries at ftab_w.
cudaError_t inner_table_launch_wide(const Plan& inner, uint32_t k_inner, const zw128* itab_w, const zw128* ipv_w,
                                    const uint32_t* ifr, const uint64_t* iadj, const uint32_t* ilow, zw128* ftab_w,
                                    cudaStream_t stream);

// ---- batches (batch.cu) -----------------------------------------------------

// One scalar of a batch, as the batch kernel reads it (device memory).
struct BatchScalar {
    KernelParams kp;
    const zw64* table;
    const zw64* pv;
    const uint32_t* rows;
    const uint64_t* adj;
    const uint32_t* seek;
    zw64 K;
    int32_t e0;
    int32_t key;
};

// Scalar descriptors sit at multiples of this many bytes from a base
// address (an array of them, or blocks of a device arena).
constexpr size_t kBatchScalarBytes = 1024;
static_assert(sizeof(BatchScalar) <= kBatchScalarBytes, "scalar descriptor too large");

// A range [first, first + count) of one scalar; first is a multiple of 8.
// The descriptor is at base + scalar * kBatchScalarBytes; the range's sum
// times K is added into results[slot].
struct BatchChunk {
    uint32_t scalar;
    uint32_t slot;
    uint64_t first;
    uint64_t count;
};

// Kernel variant of a scalar: scalars with equal keys share a launch.
int batch_key(const Plan& pl);
size_t batch_smem_bytes(int key, uint32_t ntab_cap, uint32_t npairs_cap, int threads);
cudaError_t batch_occupancy(int key, uint32_t ntab_cap, uint32_t npairs_cap, int threads,
                            int* blocks_per_sm);
// Persistent launch over chunks[0, nchunks) (one variant); *queue must be 0
// and results[] zero for the slots it touches.
cudaError_t batch_launch(int key, const unsigned char* scalars, const BatchChunk* chunks,
                         uint32_t nchunks, unsigned int* queue, DevResult* results,
                         uint32_t ntab_cap, uint32_t npairs_cap, int threads, int grid,
                         uint32_t slices_per_thread, cudaStream_t stream);

// Copy results[slots[i]] to out[i] and zero the slots (i < n), one block.
cudaError_t gather_results(DevResult* results, const uint32_t* slots, uint32_t n, DevResult* out,
                           cudaStream_t stream);

}  // namespace zxp
