// inner.cu -- the inner table of a scalar with inner parameters (plan.h):
//   F[z | q << k_inner] = sum over x_I of g(x_I, q) (-1)^(x_I . z),
// g the product of the scalar's inner and crossing rows.  Two steps on the
// device, both exact in Z[w] modulo 2^64:
//   1. one thread per u = (x_I, q) evaluates g(u) from the inner plan, as
//      the sum kernel evaluates one term: form bits by XOR of flip rows,
//      the phase exponent from the coefficient planes and the quadratic
//      bit, the node count, then K * table entry (times phase-pair values
//      beyond the folded ones; zero when a zero form is set);
//   2. the Walsh-Hadamard transform over the low k_inner bits of u, in
//      passes over groups of bits: a block stages a tile (the pass's 2^nb
//      entries of up to 32 consecutive low indices, 32 KB) in shared memory,
//      does the pass's butterfly stages there and writes it back, so that
//      the whole transform reads and writes the table ceil((k_inner - 10)/5)
//      + 1 times.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel.h"
#include "plan.h"
#include "zring.h"

namespace zxp {
namespace {

constexpr int kInnerThreads = 256;
constexpr uint32_t kTileEntries = 1024;   // 32 KB of shared memory per block

__global__ void __launch_bounds__(kInnerThreads)
inner_terms(const __grid_constant__ KernelParams p, const int nwn, const int nw, const int general,
            const zw64 K, const zw64* __restrict__ table, const zw64* __restrict__ pv,
            const uint32_t* __restrict__ frows, const uint64_t* __restrict__ adj,
            const uint32_t bits, zw64* __restrict__ out) {
    const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >> bits) return;
    uint32_t L[kMaxNW];
#pragma unroll
    for (int w = 0; w < kMaxNW; w++) L[w] = w < nw ? p.INV[w] : 0u;
    uint32_t q2 = 0;
    for (uint64_t m = u; m; m &= m - 1) {
        const uint32_t i = (uint32_t)__ffsll((long long)m) - 1u;
#pragma unroll
        for (int w = 0; w < kMaxNW; w++)
            if (w < nw) L[w] ^= __ldg(frows + (size_t)i * (uint32_t)nw + (uint32_t)w);
        q2 += (uint32_t)__popcll(__ldg(adj + i) & u);
    }
    // every quadratic pair (i, j) of u was counted from both ends
    const uint32_t q = (q2 >> 1) & 1u;
    uint32_t P0 = 0, P1 = 0, X2 = 0, M = 0, zb = 0;
#pragma unroll
    for (int w = 0; w < kMaxWordsNode; w++)
        if (w < nwn) {
            X2 ^= L[w] & p.CB[w];
            M += (uint32_t)__popc(L[w]);
        }
#pragma unroll
    for (int o = 0; o < kMaxWordsOther; o++)
        if (nwn + o < nw) {
            const uint32_t v = L[nwn + o];
            P0 += (uint32_t)__popc(v & p.C0[o]);
            P1 += (uint32_t)__popc(v & p.C1[o]);
            X2 ^= v & p.C2[o];
            zb |= v & p.Z[o];
        }
    const uint32_t J = (P0 + 2u * P1 + 4u * ((uint32_t)__popc(X2) + q)) & 7u;
    uint32_t idx = J * p.tab_stride + M;
    zw64 v;
    if (general) {
        if (p.has_zero && zb) {
            v = zw_zero();
        } else {
            v = table[idx];
            for (uint32_t j = 0; j < p.npairs; j++) {
                const uint32_t a = (L[p.PA[j] >> 5] >> (p.PA[j] & 31)) & 1u;
                const uint32_t b = (L[p.PB[j] >> 5] >> (p.PB[j] & 31)) & 1u;
                v = zw_mul(v, pv[4 * j + (a | (b << 1))]);
            }
        }
    } else {
        if (p.xshift)
            idx = (idx << p.xshift) | (L[nwn] & p.pmask) | ((p.has_zero && zb ? 1u : 0u) << p.zshift);
        v = table[idx];
    }
    out[u] = zw_mul(K, v);
}

// One pass of the transform over bits [lo, lo + nb) of an array of 2^total
// entries: a block holds the 2^nb entries of the pass for `cols`
// consecutive low indices l (cols = 2^lo up to 32; 2^nb * cols <= 1024).
__global__ void __launch_bounds__(kInnerThreads)
wht_pass(zw64* __restrict__ F, const uint32_t lo, const uint32_t nb, const uint32_t cols_log2) {
    __shared__ zw64 tile[kTileEntries];
    const uint32_t cols = 1u << cols_log2, rows = 1u << nb, n = rows * cols;
    // block -> (high index o, first low index l0)
    const uint64_t groups_lo = (1ull << lo) >> cols_log2;   // low-index groups
    const uint64_t o = (uint64_t)blockIdx.x / groups_lo;
    const uint64_t l0 = ((uint64_t)blockIdx.x % groups_lo) << cols_log2;
    const uint64_t base = (o << (lo + nb)) | l0;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const uint32_t r = e >> cols_log2, c = e & (cols - 1u);
        tile[e] = F[base + ((uint64_t)r << lo) + c];
    }
    __syncthreads();
    for (uint32_t s = 0; s < nb; s++) {
        for (uint32_t e = threadIdx.x; e < n / 2; e += blockDim.x) {
            const uint32_t pr = e >> cols_log2, c = e & (cols - 1u);
            // row with bit s clear: insert a zero at bit s of the pair index
            const uint32_t r0 = ((pr >> s) << (s + 1)) | (pr & ((1u << s) - 1u));
            const uint32_t i0 = (r0 << cols_log2) | c, i1 = ((r0 | (1u << s)) << cols_log2) | c;
            const zw64 a = tile[i0], b = tile[i1];
            tile[i0] = zw_add(a, b);
            tile[i1] = zw_sub(a, b);
        }
        __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
        const uint32_t r = e >> cols_log2, c = e & (cols - 1u);
        F[base + ((uint64_t)r << lo) + c] = tile[e];
    }
}

}  // namespace

cudaError_t inner_table_launch(const Plan& inner, uint32_t k_inner, const zw64* itab, const zw64* ipv,
                               const uint32_t* ifr, const uint64_t* iadj, zw64* ftab, cudaStream_t stream) {
    const uint32_t bits = inner.kp.k;
    if (bits > kMaxInnerBits || k_inner > bits) return cudaErrorInvalidValue;
    const int nw = inner.nwn + (inner.nwl < 1 ? 1 : inner.nwl);
    const uint64_t n = 1ull << bits;
    inner_terms<<<(unsigned)((n + kInnerThreads - 1) / kInnerThreads), kInnerThreads, 0, stream>>>(
        inner.kp, inner.nwn, nw, inner.general ? 1 : 0, inner.K, itab, ipv, ifr, iadj, bits, ftab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (uint32_t lo = 0; lo < k_inner;) {
        // bits [lo, lo + nb): the first pass takes up to 10 bits of one
        // contiguous tile, later ones up to 5 bits of 32 columns
        const uint32_t cols_log2 = lo < 5 ? lo : 5;
        uint32_t nb = 10 - cols_log2;
        if (nb > k_inner - lo) nb = k_inner - lo;
        const uint64_t blocks = n >> (nb + cols_log2);
        wht_pass<<<(unsigned)blocks, kInnerThreads, 0, stream>>>(ftab, lo, nb, cols_log2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        lo += nb;
    }
    return cudaSuccess;
}

}  // namespace zxp
