// nn_dtw_search_noalloc: the FP32 search with its scratch memory in a fixed
// device array compiled into the library, for callers that cannot allocate
// device memory themselves (the paper has no counterpart).
#include "internal.cuh"

namespace {

// The search's scratch.  It is part of the library's device image, so every
// GPU that loads the library holds these NNDTW_NOALLOC_SCRATCH_BYTES until
// the process exits.  In host code `g_noalloc_scratch` only names the symbol;
// its device address comes from cudaGetSymbolAddress in the current context.
__device__ __align__(256) unsigned char g_noalloc_scratch[NNDTW_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int nn_dtw_search_noalloc(const float *d_train, const int32_t *d_train_labels,
                                     int64_t N, const float *d_test, int64_t Q, int L, int W,
                                     int V, const float *d_env, unsigned flags,
                                     int32_t *d_nn_idx, int32_t *d_nn_label, double *d_nn_dist,
                                     nndtw_stats *stats, void *stream) {
    const size_t need = nn_dtw_workspace_size(N, Q, L, W, V, 0);
    if (need == 0) return NNDTW_EINVAL;
    if (need > NNDTW_NOALLOC_SCRATCH_BYTES) return NNDTW_ENOSPACE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        nndtw::set_last_cuda_error(e);
        return NNDTW_ECUDA;
    }
    if (dev < 0 || dev >= 64) return NNDTW_EUNSUPPORTED;
    // The array's address in the current device's context, looked up on every
    // call (a host-side table lookup once the library's device code is loaded
    // in this context), so that no address outlives a device reset or is used
    // in another context.  The first call in a context loads the module; that
    // is why the first call must come before any stream capture.
    void *ptr = nullptr;
    e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
        nndtw::set_last_cuda_error(e);
        return NNDTW_ECUDA;
    }
    // The search clears every part of its scratch that must start at zero
    // (counters, best-so-far keys, per-query tallies) at the start of each
    // call, so the previous call's contents do no harm.  Stage timing would
    // create CUDA events, so it is not offered here.
    return nn_dtw_search(d_train, d_train_labels, N, d_test, Q, L, W, V, d_env,
                         flags & ~NNDTW_TIME_STAGES, d_nn_idx, d_nn_label, d_nn_dist, ptr,
                         NNDTW_NOALLOC_SCRATCH_BYTES, stats, stream);
}
