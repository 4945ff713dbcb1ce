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
// One CTA of 256 threads takes QB queries (staged in shared memory) and
// kVarChunk training series, a warp one training series at a time against
// all QB queries: its lanes stride over the bridge rows, each envelope row
// loaded once (coalesced) and applied to the QB queries, so a row is read
// from L2 once per QB pairs.  The rows every pair shares, V .. L_A - V, run
// without per-pair tests, up to the shortest query's end first and then
// with a per-query row limit; the ends, the bands and (for series shorter
// than 2V) the bridge rows between n and V are computed one (query, band)
// per lane and added through shared memory.  A pair's value is summed per
// lane and then across the warp, at most 2 L + 16 roundings on any chain,
// the margin the caller's lb_lo covers.  Each query's smallest (bound,
// index) key among its feasible pairs is merged into seed_keys[q]: the
// query's first candidate (the Euclidean distance being undefined for
// unequal lengths).
#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kVarThreads = 256, kVarWarps = kVarThreads / 32, kVarChunk = 64;
constexpr int kBandStage = 32;   // B values staged at each end for the band tasks

__device__ __forceinline__ float sqd(float a, float b) {
    const float d = a - b;
    return d * d;
}

__device__ __forceinline__ bool in_window(int i, int j, int W) {
    return i - j <= W && j - i <= W;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// acc + the LB_Keogh term of a against envelope row e (one fused rounding)
__device__ __forceinline__ float keogh_acc(float acc, float a, float2 e) {
    const float d = max3f(a - e.x, e.y - a, 0.f);
    return fmaf(d, d, acc);
}

// Position of query k's value of row i in the interleaved staging: row i
// holds the QB queries' values; with QB = 8 its two 16-byte halves swap
// places every four rows, so that the 16-byte loads of a warp (one row per
// lane, rows 32 bytes apart) spread over all banks.
template <int QB> __device__ __forceinline__ int slot(int i, int k) {
    if constexpr (QB == 8) return i * 8 + (k ^ (((i >> 2) & 1) << 2));
    return i * QB + k;
}

// The part of pair (A, B)'s bound outside the shared bridge rows
// [V, L_A - V): the ends, bands i = 2..n of both corners (1-based), and the
// bridge rows [n, V) and [L_A - V, L_A - n) when n < V.  Band b of the task
// (0-based, b < V) contributes band b+1; task b = 0 also the extra rows.
// A's value x is As[slot<S>(x, k)] (the queries are interleaved in shared
// memory);
// hd[x] = B[x] and tl[x] = B[L_B - 1 - x] for x < kBandStage (staged), else
// read from B.  Without CHECK every band cell lies inside the window (W >=
// V - 1 + |L_A - L_B|).
template <int S, bool CHECK>
__device__ float outer_part(const float *As, int k, int LA, const float *B, const float *hd,
                            const float *tl, int LB, const float2 *env, int W, int V, int n,
                            int b) {
    auto head = [&](int x) { return x < kBandStage ? hd[x] : B[x]; };
    auto tail = [&](int x) { return x < kBandStage ? tl[x] : B[LB - 1 - x]; };
    auto in_win = [&](int i, int j) { return !CHECK || in_window(i, j, W); };
    auto A = [&](int x) { return As[slot<S>(x, k)]; };
    float v = 0.f;
    if (b < n) {
        const int i = b + 1;
        if (i == 1) {
            v = sqd(A(0), head(0)) + sqd(A(LA - 1), tail(0));
        } else {
            const float bi = head(i - 1), bti = tail(i - 1);
            const float ai = A(i - 1), ati = A(LA - i);
            float mL = sqd(ai, bi);
            float mR = sqd(ati, bti);
            for (int j = 1; j < i; j++) {
                if (in_win(i, j)) {
                    mL = fminf(mL, sqd(ai, head(j - 1)));
                    mL = fminf(mL, sqd(A(j - 1), bi));
                }
                if (in_win(LA - i + 1, LB - j + 1)) mR = fminf(mR, sqd(ati, tail(j - 1)));
                if (in_win(LA - j + 1, LB - i + 1)) mR = fminf(mR, sqd(A(LA - j), bti));
            }
            v = mL + mR;
        }
    }
    if (b == 0 && n < V) {
        // bridge rows the shared loop leaves out (short series)
        const int lo_end = V < LA - n ? V : LA - n;
        for (int i = n; i < lo_end; i++) v = keogh_acc(v, A(i), env[i]);
        for (int i = (LA - V > lo_end ? LA - V : lo_end); i < LA - n; i++)
            v = keogh_acc(v, A(i), env[i]);
    }
    return v;
}

// The QB queries' values of row i (interleaved: As[slot<QB>(i, k)]).
template <int QB>
__device__ __forceinline__ void load_row(const float *As, int i, float (&a)[QB]) {
    const float *p = As + i * QB;
    if constexpr (QB == 8) {
        const int sw = ((i >> 2) & 1) << 2;   // the halves' swap (slot)
        const float4 u = reinterpret_cast<const float4 *>(p)[sw >> 2];
        const float4 w = reinterpret_cast<const float4 *>(p)[1 - (sw >> 2)];
        a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
        a[4] = w.x; a[5] = w.y; a[6] = w.z; a[7] = w.w;
    } else if constexpr (QB == 4) {
        const float4 u = reinterpret_cast<const float4 *>(p)[0];
        a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
    } else {
        const float2 u = reinterpret_cast<const float2 *>(p)[0];
        a[0] = u.x; a[1] = u.y;
    }
}

template <int QB>
__global__ void __launch_bounds__(kVarThreads, 3) lb_var_kernel(const LbVarJob job) {
    // the queries interleaved by row, As[slot<QB>(i, k)], so that one row of
    // all QB queries is one or two vector loads
    extern __shared__ __align__(16) float As[];
    __shared__ float bsum[kVarWarps][QB];
    __shared__ float bends[kVarWarps][2][kBandStage];   // B's first and last values
    __shared__ unsigned long long sbest[QB];
    __shared__ int sLA[QB];
    const int chunks = (int)((job.N + kVarChunk - 1) / kVarChunk);
    const int64_t q0 = (int64_t)(blockIdx.x / chunks) * QB;
    const int64_t t_begin = (int64_t)(blockIdx.x % chunks) * kVarChunk;
    const int64_t t_end = t_begin + kVarChunk < job.N ? t_begin + kVarChunk : job.N;
    const int W = job.W, V = job.keogh ? 0 : job.V, ML = job.max_len;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float INF = inf_of<float>();
    const unsigned FULL = 0xffffffffu;

    // the block's queries: lengths (0 = none or out of range) and values
    if (threadIdx.x < QB) {
        const int64_t q = q0 + threadIdx.x;
        int la = 0;
        if (q < job.Q) {
            la = (int)(job.test_off[q + 1] - job.test_off[q]);
            if (la < 2 || la > ML) {
                if (t_begin == 0 && job.bad) atomicAdd(job.bad, 1ull);
                la = 0;
            }
        }
        sLA[threadIdx.x] = la;
        sbest[threadIdx.x] = ~0ull;
    }
    __syncthreads();
    int minlim = ML, maxlim = 0;
    int lim[QB];   // each query's shared bridge rows end here (no query: -V)
#pragma unroll
    for (int k = 0; k < QB; k++) {
        const int la = sLA[k];
        lim[k] = la - V;
        if (la) {
            const long long a0 = job.test_off[q0 + k];
            for (int i = threadIdx.x; i < la; i += kVarThreads)
                As[slot<QB>(i, k)] = job.test[a0 + i];
            minlim = lim[k] < minlim ? lim[k] : minlim;
            maxlim = lim[k] > maxlim ? lim[k] : maxlim;
        }
    }
    if (minlim > maxlim) minlim = maxlim;   // (no query in the block)
    __syncthreads();

    unsigned long long best[QB];
#pragma unroll
    for (int k = 0; k < QB; k++) best[k] = ~0ull;
    for (int64_t t = t_begin + warp; t < t_end; t += kVarWarps) {
        const long long b0 = job.train_off[t];
        const int LB = (int)(job.train_off[t + 1] - b0);
        const bool tok = LB >= 2 && LB <= ML;
        if (!tok && q0 == 0 && lane == 0 && job.bad) atomicAdd(job.bad, 1ull);
        const float2 *env = reinterpret_cast<const float2 *>(job.env) + t * (int64_t)job.E;
        float acc[QB];
#pragma unroll
        for (int k = 0; k < QB; k++) acc[k] = 0.f;
        if (tok) {
            // shared bridge rows: every query up to the shortest one's end,
            // four envelope rows per lane in flight ...
            int i = V + lane;
            for (; i + 96 < minlim; i += 128) {
                float2 e[4];
#pragma unroll
                for (int r = 0; r < 4; r++) e[r] = env[i + 32 * r];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    float a[QB];
                    load_row<QB>(As, i + 32 * r, a);
#pragma unroll
                    for (int k = 0; k < QB; k++) acc[k] = keogh_acc(acc[k], a[k], e[r]);
                }
            }
            for (; i < minlim; i += 32) {
                const float2 e = env[i];
                float a[QB];
                load_row<QB>(As, i, a);
#pragma unroll
                for (int k = 0; k < QB; k++) acc[k] = keogh_acc(acc[k], a[k], e);
            }
            // ... then each query up to its own (rows past a query's end
            // hold stale values: their terms are computed and discarded)
            for (i = (V > minlim ? V : minlim) + lane; i < maxlim; i += 32) {
                const float2 e = env[i];
                float a[QB];
                load_row<QB>(As, i, a);
#pragma unroll
                for (int k = 0; k < QB; k++) {
                    const float t2 = keogh_acc(acc[k], a[k], e);
                    acc[k] = i < lim[k] ? t2 : acc[k];
                }
            }
            // ends, bands and short-series rows: one (query, band) per lane,
            // B's first and last kBandStage values staged in shared memory
            if (lane < QB) bsum[warp][lane] = 0.f;
            {
                const float *B = job.train + b0;
                bends[warp][0][lane] = lane < LB ? B[lane] : 0.f;
                bends[warp][1][lane] = LB - 1 - lane >= 0 ? B[LB - 1 - lane] : 0.f;
            }
            __syncwarp();
            const int nt = V > 0 ? V : 1;
            for (int task = lane; task < QB * nt; task += 32) {
                const int k = task / nt, b = task % nt;
                const int LA = sLA[k];
                if (LA && in_window(LA, LB, W)) {
                    const int n = job.keogh ? 0 : min(min(LA, LB) / 2, V);
                    const int dl = LA > LB ? LA - LB : LB - LA;
                    const float v =
                        W >= V - 1 + dl
                            ? outer_part<QB, false>(As, k, LA, job.train + b0, bends[warp][0],
                                                    bends[warp][1], LB, env, W, V, n, b)
                            : outer_part<QB, true>(As, k, LA, job.train + b0, bends[warp][0],
                                                   bends[warp][1], LB, env, W, V, n, b);
                    if (v != 0.f) atomicAdd(&bsum[warp][k], v);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < QB; k++) {
            float v = acc[k];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
            acc[k] = v;
        }
        if (lane < QB) {
            const int k = lane;
            const int LA = sLA[k];
            float lb = INF;
            if (tok && LA && in_window(LA, LB, W)) {
                float s = 0.f;
#pragma unroll
                for (int kk = 0; kk < QB; kk++) s = kk == k ? acc[kk] : s;
                lb = s + bsum[warp][k];
            }
            float v = lb;
            if (job.safe && lb < INF) {
                v = __fsub_rd(__fmul_rd(lb, job.lb_lo), job.abs_slack);
                v = v > 0.f ? v : 0.f;
            }
            if (q0 + k < job.Q) {
                job.lb_out[(q0 + k) * job.N + t] = v;
                if (lb < INF) {
                    const unsigned long long key = pack_key(v, (uint32_t)t);
#pragma unroll
                    for (int kk = 0; kk < QB; kk++)
                        if (kk == k) best[kk] = key < best[kk] ? key : best[kk];
                }
            }
        }
        __syncwarp();
    }
    if (job.seed_keys) {
        if (lane < QB) {
#pragma unroll
            for (int kk = 0; kk < QB; kk++)
                if (kk == lane && best[kk] != ~0ull) atomicMin(&sbest[kk], best[kk]);
        }
        __syncthreads();
        if (threadIdx.x < QB && sbest[threadIdx.x] != ~0ull)
            atomicMin(job.seed_keys + q0 + threadIdx.x, sbest[threadIdx.x]);
    }
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

template <int QB>
cudaError_t launch_lb_var_qb(const LbVarJob &job, cudaStream_t s) {
    const long long chunks = (job.N + kVarChunk - 1) / kVarChunk;
    const long long blocks = chunks * ((job.Q + QB - 1) / QB);
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)job.max_len * QB;
    cudaError_t e = cudaFuncSetAttribute(lb_var_kernel<QB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lb_var_kernel<QB><<<(unsigned)blocks, kVarThreads, smem, s>>>(job);
    return cudaGetLastError();
}

}  // namespace

// Queries per CTA: eight while their staging fits 64 KB of shared memory,
// fewer for long series.
cudaError_t launch_lb_var(const LbVarJob &job, cudaStream_t s) {
    if (job.Q <= 0 || job.N <= 0) return cudaSuccess;
    const size_t per_query = sizeof(float) * (size_t)job.max_len;
    if (8 * per_query <= 64u * 1024u) return launch_lb_var_qb<8>(job, s);
    if (4 * per_query <= 64u * 1024u) return launch_lb_var_qb<4>(job, s);
    return launch_lb_var_qb<2>(job, s);
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
