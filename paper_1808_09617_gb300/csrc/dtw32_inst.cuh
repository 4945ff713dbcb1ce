// Explicit instantiation helpers for the FP32 DTW kernel (one per H).
#pragma once
#include "dtw32.cuh"

namespace nndtw {

// Super-steps per register-window block: the windows are realigned with
// 2H-1 moves once per block, so larger U costs fewer moves and more code.
template <int H> struct Dtw32U { static constexpr int value = H > 24 ? 4 : 8; };

template <int H> Dtw32Fn1 dtw32_fn();
template <int H> Dtw32FnN dtw32_fn_n();
template <int H> Dtw32Fn1 dtw32_var_fn();   // unequal lengths (one dataset)

#define NNDTW_INST_DTW32(H)                                                          \
    template <> Dtw32Fn1 dtw32_fn<H>() {                                             \
        return &dtw32_kernel<H, Dtw32U<H>::value, Src1<DtwJob32>>;                    \
    }                                                                                \
    template <> Dtw32FnN dtw32_fn_n<H>() {                                           \
        return &dtw32_kernel<H, Dtw32U<H>::value, SrcN<DtwJob32>>;                    \
    }

#define NNDTW_INST_DTW32_VAR(H)                                                      \
    template <> Dtw32Fn1 dtw32_var_fn<H>() {                                         \
        return &dtw32_kernel<H, Dtw32U<H>::value, Src1<DtwJob32>, true>;              \
    }

}  // namespace nndtw
