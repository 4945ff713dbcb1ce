// Window learning (Sec. 1 and Sec. 4): the window W of a dataset is chosen by
// leave-one-out 1-NN accuracy on its training set.  For every candidate
// window this runs the FP32 search with every training series as a query
// against all the others (NNDTW_LEAVE_ONE_OUT), all windows at once through
// the batched search, and counts on the device the series whose neighbour
// has the same label.
#include <vector>

#include "internal.cuh"

namespace nndtw {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// correct[k] += number of q with labels[idx[k N + q]] == labels[q]
__global__ void count_correct_kernel(const int32_t *__restrict__ idx,
                                     const int32_t *__restrict__ labels, int64_t N, int nw,
                                     unsigned long long *__restrict__ correct) {
    __shared__ int block_sum;
    for (int k = blockIdx.y; k < nw; k += gridDim.y) {
        if (threadIdx.x == 0) block_sum = 0;
        __syncthreads();
        int mine = 0;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N;
             q += (int64_t)gridDim.x * blockDim.x) {
            const int32_t t = idx[(int64_t)k * N + q];
            mine += (t >= 0 && t < N && labels[t] == labels[q]) ? 1 : 0;
        }
        for (int off = 16; off > 0; off >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, off);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&block_sum, mine);
        __syncthreads();
        if (threadIdx.x == 0 && block_sum)
            atomicAdd(correct + k, (unsigned long long)block_sum);
        __syncthreads();
    }
}

// Output buffers (idx, labels, distances for every window) at the front of
// the workspace, then the batched search's workspace.
struct LearnLayout {
    size_t out_bytes, batch_bytes;
};

bool learn_descriptors(const float *d_train, const int32_t *d_labels, int64_t N, int L,
                       const int32_t *h_windows, int nw, int V, char *base,
                       std::vector<nndtw_dataset> &sets, LearnLayout *lay) {
    sets.resize(nw);
    size_t off = 0;
    const size_t idx_b = align256(sizeof(int32_t) * (size_t)N * nw);
    const size_t dist_b = align256(sizeof(double) * (size_t)N * nw);
    for (int k = 0; k < nw; k++) {
        if (h_windows[k] < 0) return false;
        nndtw_dataset &d = sets[k];
        d = nndtw_dataset{};
        d.d_train = d_train; d.d_train_labels = d_labels; d.N = N;
        d.d_test = d_train; d.Q = N;
        d.L = L; d.W = h_windows[k]; d.V = V;
        d.d_env = nullptr;
        d.d_nn_idx = base ? reinterpret_cast<int32_t *>(base) + (size_t)k * N : nullptr;
        d.d_nn_label =
            base ? reinterpret_cast<int32_t *>(base + idx_b) + (size_t)k * N : nullptr;
        d.d_nn_dist =
            base ? reinterpret_cast<double *>(base + 2 * idx_b) + (size_t)k * N : nullptr;
        d.flags = NNDTW_LEAVE_ONE_OUT;
    }
    off = 2 * idx_b + dist_b;
    lay->out_bytes = off;
    lay->batch_bytes = nn_dtw_batch_workspace_size(sets.data(), nw);
    return lay->batch_bytes != 0;
}

}  // namespace
}  // namespace nndtw

using namespace nndtw;

extern "C" {

size_t nn_dtw_learn_window_workspace_size(int64_t N, int L, const int32_t *h_windows,
                                          int n_windows, int V) {
    if (N < 2 || n_windows < 1 || !h_windows) return 0;
    std::vector<nndtw_dataset> sets;
    LearnLayout lay{};
    if (!learn_descriptors(nullptr, nullptr, N, L, h_windows, n_windows, V, nullptr, sets, &lay))
        return 0;
    return lay.out_bytes + lay.batch_bytes;
}

int nn_dtw_learn_window(const float *d_train, const int32_t *d_train_labels, int64_t N, int L,
                        const int32_t *h_windows, int n_windows, int V, unsigned flags,
                        int64_t *d_correct, void *d_workspace, size_t workspace_bytes,
                        void *stream) {
    if (N < 2 || n_windows < 1 || !h_windows || !d_train || !d_train_labels || !d_correct)
        return NNDTW_EINVAL;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return NNDTW_EINVAL;
    if (flags & NNDTW_TIME_STAGES) return NNDTW_EINVAL;
    std::vector<nndtw_dataset> sets;
    LearnLayout lay{};
    char *base = static_cast<char *>(d_workspace);
    if (!learn_descriptors(d_train, d_train_labels, N, L, h_windows, n_windows, V, base, sets,
                           &lay))
        return NNDTW_EINVAL;
    if (workspace_bytes < lay.out_bytes + lay.batch_bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_correct, 0, sizeof(int64_t) * n_windows, s);
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    const int rc = nn_dtw_search_batched(sets.data(), n_windows, base + lay.out_bytes,
                                         lay.batch_bytes, flags, stream);
    if (rc != NNDTW_OK) return rc;
    const unsigned gx = (unsigned)((N + 255) / 256 < 64 ? (N + 255) / 256 : 64);
    const unsigned gy = (unsigned)(n_windows < 1024 ? n_windows : 1024);
    count_correct_kernel<<<dim3(gx, gy), 256, 0, s>>>(
        reinterpret_cast<const int32_t *>(base), d_train_labels, N, n_windows,
        reinterpret_cast<unsigned long long *>(d_correct));
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    return NNDTW_OK;
}

}  // extern "C"
