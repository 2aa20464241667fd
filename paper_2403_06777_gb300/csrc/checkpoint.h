// checkpoint.h -- resumable chunked sums: the whole range of a scalar's
// terms in chunks of 2^chunk_log2, the running partial sum and the set of
// finished chunks kept in a host file after every chunk, so that a process
// that ends between chunks (a job that is preempted, killed or runs out of
// time) loses at most the chunk in flight and a later call continues where
// it stopped.  Host code only: the chunk evaluator is passed in.
//
// File layout (host byte order; every field fixed-size):
//   char     magic[8]      "ZXPCKPT1"
//   uint32   version       1
//   uint32   width         64 or 128: the partial sum's coefficient width
//   uint64   digest        FNV-1a 64 of the scalar's table bytes
//   uint32   k             parameters summed (the scalar's outer ones)
//   uint32   chunk_log2
//   uint64   n_chunks      ceil(2^k / 2^chunk_log2)
//   int32    e0, uint32 0
//   uint64   sum[8]        low words of the 4 coefficients, then the high
//                          words (0 for width 64); sums modulo 2^width
//   uint64   done_count
//   uint8    done[ceil(n_chunks / 8)]   bit c of byte c / 8: chunk c is in sum
//   uint64   check         FNV-1a 64 of every byte before it
// A new state is written to `path`.tmp, flushed to the disk and renamed over
// `path`, so the file always holds one complete state.
#pragma once
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

namespace zxp {
namespace ckpt {

struct State {
    uint32_t width = 64;
    uint64_t digest = 0;
    uint32_t k = 0, chunk_log2 = 0;
    uint64_t n_chunks = 0;
    int32_t e0 = 0;
    uint64_t sum[8] = {};
    uint64_t done_count = 0;
    std::vector<uint8_t> done;
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull);

// A fresh state for a sum of 2^k terms (chunk_log2 clamped to k).
State fresh(uint32_t width, uint64_t digest, uint32_t k, uint32_t chunk_log2, int32_t e0);

// Read `path`: 1 if it holds a valid state, 0 if it does not exist, a
// negative ZXP status if it exists but is damaged (ZXP_EINVAL).
int load(const std::string& path, State* st);
// Replace `path` with the state (ZXP_OK or ZXP_EINVAL when writing failed).
int save(const std::string& path, const State& st);

// Evaluates chunk c (terms [c << chunk_log2, ...), the last one ragged):
// the raw partial's low words lo[4] and, for width 128, high words hi[4].
using ChunkFn = std::function<int(uint64_t first, uint64_t count, uint64_t lo[4], uint64_t hi[4])>;

// Continue (or start) the sum that `path` records for (width, digest, k,
// chunk_log2, e0): a file for another scalar or other parameters is an
// error (ZXP_EINVAL), not overwritten.  Runs at most max_chunks further
// chunks (0: no limit), saving after each; returns ZXP_OK with *st complete,
// ZXP_EAGAIN when chunks remain, or the evaluator's or the file's error.
int run(const std::string& path, uint32_t width, uint64_t digest, uint32_t k, uint32_t chunk_log2, int32_t e0,
        uint64_t max_chunks, const ChunkFn& eval, State* st);

}  // namespace ckpt
}  // namespace zxp
