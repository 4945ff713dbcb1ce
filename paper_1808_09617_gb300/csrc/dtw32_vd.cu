// FP32 DTW kernel instantiations, unequal-length form (H = 27 28 29 30 31 32).
#include "dtw32_inst.cuh"
namespace nndtw {
NNDTW_INST_DTW32_VAR(27)
NNDTW_INST_DTW32_VAR(28)
NNDTW_INST_DTW32_VAR(29)
NNDTW_INST_DTW32_VAR(30)
NNDTW_INST_DTW32_VAR(31)
NNDTW_INST_DTW32_VAR(32)
}  // namespace nndtw
