// FP32 DTW kernel instantiations, unequal-length form (H = 21 22 23 24 25 26).
#include "dtw32_inst.cuh"
namespace nndtw {
NNDTW_INST_DTW32_VAR(21)
NNDTW_INST_DTW32_VAR(22)
NNDTW_INST_DTW32_VAR(23)
NNDTW_INST_DTW32_VAR(24)
NNDTW_INST_DTW32_VAR(25)
NNDTW_INST_DTW32_VAR(26)
}  // namespace nndtw
