// LB_New (Sec. 2.2.5) for every (query, training series) pair: the two ends
// (boundary condition) plus, for every interior i, the smallest delta(A_i, B_j)
// over B's window max(1, i-W) <= j <= min(L, i+W) (continuity: the path pairs
// A_i with some B_j there).  One of the comparison bounds of the paper's
// tightness study; the search itself prunes with LB_Enhanced^V.
//
// A CTA of 128 threads takes one training series (staged whole in shared
// memory) and 128 queries, one per thread.  The queries stream through in
// chunks of 32 elements staged transposed (row stride 129: conflict-free
// for both the coalesced staging writes and the per-thread reads); every
// thread then scans the window of its element in the shared series, which
// all threads read at the same address (a broadcast).  Work per pair is
// O(L (2W + 1)): three instructions per (i, j) (difference, product, minimum).
#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kNewThreads = 128, kNewChunk = 32, kNewStride = kNewThreads + 1;

__device__ __forceinline__ float nsq(float a, float b) { float d = a - b; return d * d; }
__device__ __forceinline__ double nsq(double a, double b) {
    double d = __dsub_rn(a, b); return __dmul_rn(d, d);
}
__device__ __forceinline__ float nmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double nmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float nscale(float x, float lo, float abs_s) {
    const float v = __fsub_rd(__fmul_rd(x, lo), abs_s);
    return v > 0.f ? v : 0.f;
}
__device__ __forceinline__ double nscale(double x, double lo, double abs_s) {
    const double v = __dsub_rd(__dmul_rd(x, lo), abs_s);
    return v > 0.0 ? v : 0.0;
}

template <typename T>
__host__ __device__ size_t lb_new_series_bytes(int L) {
    return ((size_t)L * sizeof(T) + 15) / 16 * 16;
}
template <typename T>
size_t lb_new_smem(int L) {
    return lb_new_series_bytes<T>(L) + sizeof(T) * kNewChunk * kNewStride;
}

template <typename T>
__global__ void __launch_bounds__(kNewThreads)
lb_new_kernel(const T *__restrict__ test, int64_t Q, const T *__restrict__ train, int64_t N,
              int L, int W, bool safe, T lb_lo, T lb_abs, T *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    T *sB = reinterpret_cast<T *>(smem);
    T *sA = reinterpret_cast<T *>(smem + lb_new_series_bytes<T>(L));
    const int tid = threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.x * kNewThreads;
    const int64_t q = q0 + tid;
    for (int64_t t = blockIdx.y; t < N; t += gridDim.y) {
        __syncthreads();   // the previous series and chunk are no longer read
        const T *b = train + t * L;
        for (int j = tid; j < L; j += kNewThreads) sB[j] = b[j];
        T acc = T(0);
        for (int c0 = 0; c0 < L; c0 += kNewChunk) {
            __syncthreads();
            // queries q0 .. q0+127, elements c0 .. c0+31: a warp reads 32
            // consecutive elements of one query
            for (int k = tid; k < kNewThreads * kNewChunk; k += kNewThreads) {
                const int r = k / kNewChunk, e = k % kNewChunk;
                const int64_t qq = q0 + r;
                const int i = c0 + e;
                sA[e * kNewStride + r] = (qq < Q && i < L) ? test[qq * L + i] : T(0);
            }
            __syncthreads();
            const int cend = L - c0 < kNewChunk ? L - c0 : kNewChunk;
            for (int e = 0; e < cend; e++) {
                const int i = c0 + e;
                const T a = sA[e * kNewStride + tid];
                if (i == 0 || i == L - 1) {          // the two ends
                    acc = acc + nsq(a, sB[i]);
                    continue;
                }
                const int jlo = i - W > 0 ? i - W : 0;
                const int jhi = i + W < L - 1 ? i + W : L - 1;
                T m = nsq(a, sB[jlo]);
                for (int j = jlo + 1; j <= jhi; j++) m = nmin(m, nsq(a, sB[j]));
                acc = acc + m;
            }
        }
        if (q < Q) out[q * N + t] = safe ? nscale(acc, lb_lo, lb_abs) : acc;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_lb_new(const T *test, int64_t Q, const T *train, int64_t N, int L, int W,
                          bool safe, T lb_lo, T lb_abs, T *out, cudaStream_t s) {
    if (Q <= 0 || N <= 0) return cudaSuccess;
    const int Weff = W > L - 1 ? L - 1 : W;
    const size_t smem = lb_new_smem<T>(L);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(
            lb_new_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((unsigned)((Q + kNewThreads - 1) / kNewThreads),
                    (unsigned)(N < 65535 ? N : 65535));
    lb_new_kernel<T><<<grid, kNewThreads, smem, s>>>(test, Q, train, N, L, Weff, safe, lb_lo,
                                                    lb_abs, out);
    return cudaGetLastError();
}

template cudaError_t launch_lb_new<float>(const float *, int64_t, const float *, int64_t, int, int,
                                          bool, float, float, float *, cudaStream_t);
template cudaError_t launch_lb_new<double>(const double *, int64_t, const double *, int64_t, int,
                                           int, bool, double, double, double *, cudaStream_t);

}  // namespace nndtw
