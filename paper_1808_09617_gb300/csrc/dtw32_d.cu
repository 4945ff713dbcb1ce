// FP32 DTW kernel instantiations (H = 27 28 29 30 31 32).
#include "dtw32_inst.cuh"
namespace nndtw {
NNDTW_INST_DTW32(27)
NNDTW_INST_DTW32(28)
NNDTW_INST_DTW32(29)
NNDTW_INST_DTW32(30)
NNDTW_INST_DTW32(31)
NNDTW_INST_DTW32(32)
}  // namespace nndtw
