// nn_dtw_search_batched: many independent datasets (each its own training
// set, test set, L, W and V) searched by one call.  The call forks from the
// caller's stream onto the library's internal streams, runs each dataset's
// search (the same kernels as nn_dtw_search) on one of them, and joins back,
// so the datasets' kernels overlap on the GPU; captured into a CUDA graph the
// whole batch is one graph launch with one branch per internal stream.
// Datasets are issued largest first (by N * Q * L) and dealt round-robin over
// the streams.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kBatchStreams = 16;

struct DeviceStreams {
    bool ready = false;
    // held for a whole call: the fork, the searches issued on the internal
    // streams and the join use this device's one set of streams and events,
    // so two calls must not interleave (one thread's fork event re-recorded
    // by another before the first one's streams wait on it)
    std::mutex call_mu;
    cudaStream_t s[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kBatchStreams] = {};
};
std::mutex g_bs_mu;
DeviceStreams g_bs[64];

cudaError_t device_streams(DeviceStreams **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_bs_mu);
    DeviceStreams &d = g_bs[dev];
    if (!d.ready) {
        for (int i = 0; i < kBatchStreams; i++) {
            e = cudaStreamCreateWithFlags(&d.s[i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            e = cudaEventCreateWithFlags(&d.join[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace nndtw

using namespace nndtw;

extern "C" {

size_t nn_dtw_batch_workspace_size(const nndtw_dataset *h_sets, int n) {
    if (!h_sets || n < 0) return 0;
    size_t tot = 256;
    for (int i = 0; i < n; i++) {
        const nndtw_dataset &d = h_sets[i];
        const size_t b = nn_dtw_workspace_size(d.N, d.Q, d.L, d.W, d.V, 0);
        if (b == 0) return 0;
        tot += align256(b);
    }
    return tot;
}

int nn_dtw_search_batched(const nndtw_dataset *h_sets, int n, void *d_workspace,
                          size_t workspace_bytes, unsigned flags, void *stream) {
    if (n < 0 || (n > 0 && !h_sets)) return NNDTW_EINVAL;
    if (n == 0) return NNDTW_OK;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return NNDTW_EINVAL;
    if (flags & NNDTW_TIME_STAGES) return NNDTW_EINVAL;
    std::vector<size_t> off(n), bytes(n);
    size_t tot = 0;
    for (int i = 0; i < n; i++) {
        const nndtw_dataset &d = h_sets[i];
        bytes[i] = nn_dtw_workspace_size(d.N, d.Q, d.L, d.W, d.V, 0);
        if (bytes[i] == 0) return NNDTW_EINVAL;
        if (d.Q > 0 && (!d.d_train || !d.d_train_labels || !d.d_test || !d.d_nn_idx ||
                        !d.d_nn_label || !d.d_nn_dist))
            return NNDTW_EINVAL;
        off[i] = tot;
        tot += align256(bytes[i]);
    }
    if (workspace_bytes < tot) return NNDTW_ENOSPACE;

    DeviceStreams *ds = nullptr;
    cudaError_t e = device_streams(&ds);
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> call_lock(ds->call_mu);

    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)h_sets[a].N * h_sets[a].Q * h_sets[a].L;
        const double wb = (double)h_sets[b].N * h_sets[b].Q * h_sets[b].L;
        return wa > wb;
    });
    const int ns = n < kBatchStreams ? n : kBatchStreams;
    e = cudaEventRecord(ds->fork, s);
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    for (int k = 0; k < ns; k++) {
        e = cudaStreamWaitEvent(ds->s[k], ds->fork, 0);
        if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    }
    int rc = NNDTW_OK;
    for (int r = 0; r < n && rc == NNDTW_OK; r++) {
        const int i = order[r];
        const nndtw_dataset &d = h_sets[i];
        const unsigned f = (flags | d.flags) & ~NNDTW_TIME_STAGES;
        rc = nn_dtw_search(d.d_train, d.d_train_labels, d.N, d.d_test, d.Q, d.L, d.W, d.V, d.d_env,
                           f, d.d_nn_idx, d.d_nn_label, d.d_nn_dist,
                           static_cast<char *>(d_workspace) + off[i], bytes[i], nullptr,
                           ds->s[r % ns]);
    }
    // join every forked stream back, even after an error, so no branch is left open
    for (int k = 0; k < ns; k++) {
        e = cudaEventRecord(ds->join[k], ds->s[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ds->join[k], 0);
        if (e != cudaSuccess && rc == NNDTW_OK) { set_last_cuda_error(e); rc = NNDTW_ECUDA; }
    }
    return rc;
}

}  // extern "C"
