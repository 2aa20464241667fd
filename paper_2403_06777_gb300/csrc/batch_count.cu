// batch_count.cu -- the counting variants of the batch kernel
// (batch_kernel.cuh).
#include "batch_kernel.cuh"

namespace zxp {
namespace batchk {

extern const BatchFn kHist[4][2][kMaxWordsOther] = {
    {ZXP_BATCH_ROW(0, 3), ZXP_BATCH_ROW(1, 3)}, {ZXP_BATCH_ROW(0, 4), ZXP_BATCH_ROW(1, 4)},
    {ZXP_BATCH_ROW(0, 5), ZXP_BATCH_ROW(1, 5)}, {ZXP_BATCH_ROW(0, 6), ZXP_BATCH_ROW(1, 6)},
};
extern const BatchFn kShared[2][kMaxWordsNode + 1][kMaxWordsOther] = {ZXP_BATCH_ALL(7), ZXP_BATCH_ALL(8)};

// block lookup (at most 22 odd nodes: nwn <= 1): [variant 9, 10, 11, 13][nwn][nwl - 1]
extern const BatchFn kLut[4][2][kMaxWordsOther] = {{ZXP_BATCH_ROW(0, 9), ZXP_BATCH_ROW(1, 9)},
                                                   {ZXP_BATCH_ROW(0, 10), ZXP_BATCH_ROW(1, 10)},
                                                   {ZXP_BATCH_ROW(0, 11), ZXP_BATCH_ROW(1, 11)},
                                                   {ZXP_BATCH_ROW(0, 13), ZXP_BATCH_ROW(1, 13)}};

}  // namespace batchk
}  // namespace zxp
