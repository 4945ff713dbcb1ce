// LB_Enhanced^V (Sec. 3.1, Eq. 7) and LB_Keogh (Sec. 2.2.3) for series of
// unequal lengths (Sec. 2: the equal-length exposition generalises), and the
// first-candidate list of the unequal-length search.
//
// Reading, for a query A of length L_A and a training series B of length L_B:
// the pair has a warping path inside the window only if |L_A - L_B| <= W,
// otherwise its DTW and its bound are +inf.  Otherwise the bound is
//   delta(A_1, B_1) + delta(A_LA, B_LB)
//   + sum_{i=2..n} [min over the start corner's band i + min over the end
//                   corner's band i]
//   + sum_{i=n+1..L_A-n} LB_Keogh term of A_i against B's envelope row i,
// n = min(floor(min(L_A, L_B) / 2), V); band i of the start corner holds the
// cells (i, j) and (j, i), j <= i, of the window, band i of the end corner
// the cells (L_A-i+1, L_B-j+1) and (L_A-j+1, L_B-i+1), j <= i, of the window.
// B's envelope rows come from the ragged envelope kernel (rows up to
// L_B + W, stride E).  With L_A = L_B this is Eq. 7 / Algorithm 1.
//
// One CTA of 256 threads takes one query (staged in shared memory) and
// kVarChunk training series; each warp computes one pair at a time, its
// lanes striding over the bridge rows (coalesced envelope loads, the query
// read from shared memory) and, for the bands, one band per lane.  A pair's
// value is summed per lane and then across the warp, at most 2 L + 16
// roundings on any chain, the margin the caller's lb_lo covers.  The CTA's
// smallest (bound, index) key of the query's feasible pairs is merged into
// seed_keys[q] with one atomic per warp: the query's first candidate
// (the Euclidean distance being undefined for unequal lengths).
#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kVarThreads = 256, kVarChunk = 64;

__device__ __forceinline__ float sqd(float a, float b) {
    const float d = a - b;
    return d * d;
}

__device__ __forceinline__ bool in_window(int i, int j, int W) {
    return i - j <= W && j - i <= W;
}

__global__ void __launch_bounds__(kVarThreads) lb_var_kernel(const LbVarJob job) {
    extern __shared__ __align__(16) float As[];
    const int chunks = (int)((job.N + kVarChunk - 1) / kVarChunk);
    const int64_t q = (int64_t)(blockIdx.x / chunks);
    const int64_t t_begin = (int64_t)(blockIdx.x % chunks) * kVarChunk;
    const int64_t t_end = t_begin + kVarChunk < job.N ? t_begin + kVarChunk : job.N;
    const int W = job.W, V = job.V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float INF = inf_of<float>();

    const long long a0 = job.test_off[q];
    const int LA = (int)(job.test_off[q + 1] - a0);
    const bool qok = LA >= 2 && LA <= job.max_len;
    if (qok)
        for (int i = threadIdx.x; i < LA; i += kVarThreads) As[i] = job.test[a0 + i];
    else if (threadIdx.x == 0 && t_begin == 0 && job.bad)
        atomicAdd(job.bad, 1ull);
    __syncthreads();

    unsigned long long best = ~0ull;
    for (int64_t t = t_begin + warp; t < t_end; t += kVarThreads / 32) {
        const long long b0 = job.train_off[t];
        const int LB = (int)(job.train_off[t + 1] - b0);
        const bool tok = LB >= 2 && LB <= job.max_len;
        if (!tok && q == 0 && lane == 0 && job.bad) atomicAdd(job.bad, 1ull);
        float lb = INF;
        if (qok && tok && in_window(LA, LB, W)) {
            const float *B = job.train + b0;
            const float2 *env = reinterpret_cast<const float2 *>(job.env) + t * (int64_t)job.E;
            const int n = job.keogh ? 0 : min(min(LA, LB) / 2, V);
            float acc = 0.f;
            // bridge: LB_Keogh terms of rows n+1 .. L_A-n (0-based [n, L_A-n))
            for (int i = n + lane; i < LA - n; i += 32) {
                const float a = As[i];
                const float2 e = env[i];
                const float d = fmaxf(fmaxf(a - e.x, e.y - a), 0.f);
                acc = fmaf(d, d, acc);
            }
            // ends (lane 0) and bands i = 2..n (lane i-1), 1-based indices
            if (lane < n) {
                const int i = lane + 1;
                if (i == 1) {
                    acc += sqd(As[0], B[0]) + sqd(As[LA - 1], B[LB - 1]);
                } else {
                    float mL = sqd(As[i - 1], B[i - 1]);
                    float mR = sqd(As[LA - i], B[LB - i]);
                    for (int j = 1; j < i; j++) {
                        if (in_window(i, j, W)) {
                            mL = fminf(mL, sqd(As[i - 1], B[j - 1]));
                            mL = fminf(mL, sqd(As[j - 1], B[i - 1]));
                        }
                        if (in_window(LA - i + 1, LB - j + 1, W))
                            mR = fminf(mR, sqd(As[LA - i], B[LB - j]));
                        if (in_window(LA - j + 1, LB - i + 1, W))
                            mR = fminf(mR, sqd(As[LA - j], B[LB - i]));
                    }
                    acc += mL + mR;
                }
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            lb = acc;
        }
        if (lane == 0) {
            float v = lb;
            if (job.safe && lb < INF) {
                v = __fsub_rd(__fmul_rd(lb, job.lb_lo), job.abs_slack);
                v = v > 0.f ? v : 0.f;
            }
            job.lb_out[q * job.N + t] = v;
            if (lb < INF) {
                const unsigned long long key = pack_key(v, (uint32_t)t);
                best = key < best ? key : best;
            }
        }
    }
    if (job.seed_keys && lane == 0 && best != ~0ull) atomicMin(job.seed_keys + q, best);
}

// The first-candidate pairs (q, key index) of the queries that have one.
__global__ void seed_pairs_kernel(const unsigned long long *__restrict__ seed_keys, int64_t Q,
                                  uint2 *__restrict__ pairs, unsigned long long *count) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = seed_keys[q];
        if (k == ~0ull) continue;
        const unsigned long long slot = atomicAdd(count, 1ull);
        pairs[slot] = make_uint2((uint32_t)q, key_idx(k));
    }
}

}  // namespace

cudaError_t launch_lb_var(const LbVarJob &job, cudaStream_t s) {
    if (job.Q <= 0 || job.N <= 0) return cudaSuccess;
    const long long chunks = (job.N + kVarChunk - 1) / kVarChunk;
    const long long blocks = chunks * job.Q;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)job.max_len;
    cudaError_t e = cudaFuncSetAttribute(lb_var_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    lb_var_kernel<<<(unsigned)blocks, kVarThreads, smem, s>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_seed_pairs(const unsigned long long *seed_keys, int64_t Q, uint2 *pairs,
                              unsigned long long *count, int sm_count, cudaStream_t s) {
    if (Q <= 0) return cudaSuccess;
    long long blocks = (Q + 255) / 256;
    if (blocks > (long long)sm_count * 4) blocks = (long long)sm_count * 4;
    seed_pairs_kernel<<<(unsigned)blocks, 256, 0, s>>>(seed_keys, Q, pairs, count);
    return cudaGetLastError();
}

}  // namespace nndtw
