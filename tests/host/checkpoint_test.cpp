// Host test program for resumable chunked sums
// (paper_2403_06777_gb300/csrc/checkpoint.cpp), without a GPU: the chunk
// evaluator is a fixed function of the chunk's first term and length.
//
//   checkpoint_test <path> <width> <k> <chunk_log2> <digest> <e0> <max_chunks> <kill_at>
//
// runs ckpt::run on <path>; the evaluator of chunk [first, first + count)
// returns, for coefficient i, lo = mix(4 first + i) * count + i and (width
// 128) hi = mix(4 first + i + 2^40) mod 2^32, mix the SplitMix64 finaliser.
// kill_at >= 0: the process sends itself SIGKILL inside the evaluation of
// its (kill_at + 1)-th chunk, after kill_at chunks were saved.  Prints
// "status done n_chunks" and the 8 sum words in hex.
#include <signal.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "checkpoint.h"

using namespace zxp;

namespace {

uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 9) {
        fprintf(stderr, "usage: %s path width k chunk_log2 digest e0 max_chunks kill_at\n", argv[0]);
        return 2;
    }
    const std::string path = argv[1];
    const uint32_t width = (uint32_t)strtoul(argv[2], nullptr, 10);
    const uint32_t k = (uint32_t)strtoul(argv[3], nullptr, 10);
    const uint32_t cl = (uint32_t)strtoul(argv[4], nullptr, 10);
    const uint64_t digest = strtoull(argv[5], nullptr, 10);
    const int32_t e0 = (int32_t)strtol(argv[6], nullptr, 10);
    const uint64_t max_chunks = strtoull(argv[7], nullptr, 10);
    const long kill_at = strtol(argv[8], nullptr, 10);
    long calls = 0;
    auto eval = [&](uint64_t first, uint64_t count, uint64_t lo[4], uint64_t hi[4]) -> int {
        if (kill_at >= 0 && calls++ == kill_at) raise(SIGKILL);
        for (int i = 0; i < 4; i++) {
            lo[i] = mix(4 * first + (uint64_t)i) * count + (uint64_t)i;
            hi[i] = width == 128 ? (mix(4 * first + (uint64_t)i + (1ull << 40)) & 0xFFFFFFFFull) : 0;
        }
        return 0;
    };
    ckpt::State st;
    const int r = ckpt::run(path, width, digest, k, cl, e0, max_chunks, eval, &st);
    printf("%d %llu %llu\n", r, (unsigned long long)st.done_count, (unsigned long long)st.n_chunks);
    for (int i = 0; i < 8; i++) printf("%llx\n", (unsigned long long)st.sum[i]);
    return 0;
}
