// Measurement aid: the FP32 CUDA-core rate of the DTW cell update with
// independent cells and no memory traffic (the denominator of the DTW
// kernel's ALU roofline).  Each thread updates 16 register cells per
// iteration with the instruction mix of the FP32 DTW kernel:
//   d = x - y;  D = fma(d, d, min3(D, D_left, D_right)).
#include "internal.cuh"
#include "dtw32.cuh"

namespace nndtw {
namespace {

constexpr int kProbeThreads = 256, kProbeBlocksPerSM = 8, kCells = 16;

__global__ void __launch_bounds__(kProbeThreads)
probe_cell_kernel(float *sink, int iters, float seed) {
    float R[kCells], B[kCells];
    const float t = seed + 1e-3f * (float)threadIdx.x;
#pragma unroll
    for (int k = 0; k < kCells; k++) { R[k] = t * (k + 1); B[k] = t - k; }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kCells; k += 2) {   // even cells read odd neighbours
            const float d = R[(k + 3) & (kCells - 1)] - B[k];
            R[k] = fmaf(d, d, min3f(R[k], R[(k + 1) & (kCells - 1)], R[(k + kCells - 1) & (kCells - 1)]));
        }
#pragma unroll
        for (int k = 1; k < kCells; k += 2) {   // odd cells read even neighbours
            const float d = R[(k + 3) & (kCells - 1)] - B[k];
            R[k] = fmaf(d, d, min3f(R[k], R[(k + 1) & (kCells - 1)], R[(k + kCells - 1) & (kCells - 1)]));
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kCells; k++) acc += R[k];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace
}  // namespace nndtw

using namespace nndtw;

extern "C" {

size_t nn_dtw_probe_sink_bytes(void) {
    return sizeof(float) * (size_t)kProbeThreads * kProbeBlocksPerSM * 256;
}

int nn_dtw_probe_cell_rate(void *d_sink, size_t sink_bytes, int iters, double *h_cells_per_s,
                           void *stream) {
    if (!d_sink || !h_cells_per_s || iters < 1) return NNDTW_EINVAL;
    const int sms = device_sm_count();
    const long long blocks = (long long)sms * kProbeBlocksPerSM;
    if (sms > 256 || sink_bytes < sizeof(float) * (size_t)kProbeThreads * blocks)
        return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) { cudaEventDestroy(a); set_last_cuda_error(e); return NNDTW_ECUDA; }
    // warm-up launch, then the timed one
    probe_cell_kernel<<<(unsigned)blocks, kProbeThreads, 0, s>>>((float *)d_sink, iters / 10 + 1, 1.0f);
    cudaEventRecord(a, s);
    probe_cell_kernel<<<(unsigned)blocks, kProbeThreads, 0, s>>>((float *)d_sink, iters, 1.0f);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) { set_last_cuda_error(e); return NNDTW_ECUDA; }
    const double cells = (double)blocks * kProbeThreads * kCells * (double)iters;
    *h_cells_per_s = cells / (ms * 1e-3);
    return NNDTW_OK;
}

}  // extern "C"
