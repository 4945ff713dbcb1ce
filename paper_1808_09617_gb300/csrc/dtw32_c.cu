// FP32 DTW kernel instantiations (H = 21 22 23 24 25 26).
#include "dtw32_inst.cuh"
namespace nndtw {
NNDTW_INST_DTW32(21)
NNDTW_INST_DTW32(22)
NNDTW_INST_DTW32(23)
NNDTW_INST_DTW32(24)
NNDTW_INST_DTW32(25)
NNDTW_INST_DTW32(26)
}  // namespace nndtw
