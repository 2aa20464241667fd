// kernel_count.cu -- the counting variants of the sum kernel
// (sum_kernel.cuh): lane-private 32- and 16-bit counters and warp-shared
// counters, each with and without folded phase-pair / zero index bits.
#include "sum_kernel.cuh"

namespace zxp {
namespace sumk {

// lane-private counters (tables of at most 128 entries: nwn <= 1): [variant - 3][nwn][nwl - 1]
extern const KernelFn kHist[4][2][kMaxWordsOther] = {
    {ZXP_SUM_ROW(0, 3), ZXP_SUM_ROW(1, 3)}, {ZXP_SUM_ROW(0, 4), ZXP_SUM_ROW(1, 4)},
    {ZXP_SUM_ROW(0, 5), ZXP_SUM_ROW(1, 5)}, {ZXP_SUM_ROW(0, 6), ZXP_SUM_ROW(1, 6)},
};
// warp-shared counters: [variant - 7][nwn][nwl - 1]
extern const KernelFn kShared[2][kMaxWordsNode + 1][kMaxWordsOther] = {ZXP_SUM_ALL(7), ZXP_SUM_ALL(8)};

// block lookup (at most 22 odd nodes: nwn <= 1): [variant 9, 10, 11, 13, 14, 15][nwn][nwl - 1]
extern const KernelFn kLut[6][2][kMaxWordsOther] = {{ZXP_SUM_ROW(0, 9), ZXP_SUM_ROW(1, 9)},
                                                    {ZXP_SUM_ROW(0, 10), ZXP_SUM_ROW(1, 10)},
                                                    {ZXP_SUM_ROW(0, 11), ZXP_SUM_ROW(1, 11)},
                                                    {ZXP_SUM_ROW(0, 13), ZXP_SUM_ROW(1, 13)},
                                                    {ZXP_SUM_ROW(0, 14), ZXP_SUM_ROW(1, 14)},
                                                    {ZXP_SUM_ROW(0, 15), ZXP_SUM_ROW(1, 15)}};

}  // namespace sumk
}  // namespace zxp
