// The cascade's second stage, tested on the pairs that survived
// LB_Enhanced^V(A, B) before their DTW is due, and the dense form of the
// LB_Improved bridge behind the lb_enhanced_improved entry point.
//
// Reverse bound.  LB_Enhanced^V(B, A) is Eq. 7 with the two series
// exchanged.  Its two ends and its bands equal those of LB_Enhanced(A, B) (a
// band takes the minimum over the cells (i, j) and (j, i) alike), which the
// bound pass stores per pair; what differs is the bridge, here LB_Keogh of the
// training series B against the query's envelope (U^A, Lo^A) over
// [n_b, L - n_b).
//
// LB_Improved bridge.  LB_Improved (Sec. 2.2.4) follows LB_Keogh(A, B) with a
// second pass: LB_Keogh of B against the envelope of A', the projection of A
// onto B's envelope (Eq. 5); Sec. 5 proposes it as the bridge of
// LB_Enhanced.  The second pass needs no per-pair envelope: for |i - j| <= W,
// Lo_i <= B_j <= U_i, so A'_i >= B_j exactly when max(A_i, Lo_i) >= B_j, and
// when no i of j's window does so the window maximum of A' is
// max(U^A_j, max_i Lo_i).  With the mirrored argument below, the term of B_j
// is its LB_Keogh term against
//   [min(Lo^A_j, env2_j.y), max(U^A_j, env2_j.x)],
// env2 = (window max of Lo, window min of U), the training series' second
// envelopes.  The bound is the pair's LB_Enhanced(A, B) plus these terms.
//
// In the FP32 search each training element is read as one 8-byte record
// (BGap): B_j and the two gaps B_j - env2_j.x and env2_j.y - B_j, both >= 0,
// rounded down to half precision.  Above the query's envelope the term is
// min(B_j - U^A_j, gap_up)^2, below it min(Lo^A_j - B_j, gap_dn)^2; a gap
// rounded down only makes a term smaller, so the bound stays a lower bound.
// The reverse bound's term, max(B_j - U^A_j, Lo^A_j - B_j, 0)^2, reuses the
// same differences.
//
// A pair is dropped when a bound, scaled down by the bound's rounding margin,
// exceeds (strictly) the query's upper bound at this point: the inflated DTW
// of its best candidate so far.
//
// Eight lanes per pair (four pairs per warp at a time), each lane loading
// every eighth element, so that the loads of a pair are coalesced and four
// pairs' loads are in flight per warp; consecutive queue entries mostly share
// their query (the compaction appends them query by query), so its envelope
// is mostly served by L1.  A warp takes 32 consecutive queue entries and
// appends the survivors with one atomic, so the queue's order (most
// promising bucket first) is kept within each run of 32.
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kGroup = 8;   // lanes per pair

__device__ __forceinline__ float mul_rd(float a, float b) { return __fmul_rd(a, b); }
__device__ __forceinline__ double mul_rd(double a, double b) { return __dmul_rd(a, b); }
__device__ __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }
__device__ __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
// max(a, b, c) in one three-input instruction
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

// The LB_Keogh term of b against [lo, hi] (squared distance to the interval).
template <typename T>
__device__ __forceinline__ T keogh_term(T b, T lo, T hi) {
    const T d = b - tmin(tmax(b, lo), hi);
    return d * d;
}

// bg[k] = (B_k, gaps to the second envelopes rounded down), in place over
// env2 (each thread reads its element before writing it).
template <typename Src>
__global__ void pack_bgap_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const PackJob &job = src.get(bid, nblk);
    const float *__restrict__ train = job.train;
    float2 *env2 = reinterpret_cast<float2 *>(job.env2);
    const long long n = job.n;
    for (long long k = (long long)bid * blockDim.x + threadIdx.x; k < n;
         k += (long long)nblk * blockDim.x) {
        const float b = train[k];
        const float2 o = env2[k];
        BGap r;
        r.b = b;
        r.g = __halves2half2(__float2half_rd(__fsub_rd(b, o.x)), __float2half_rd(__fsub_rd(o.y, b)));
        reinterpret_cast<BGap *>(env2)[k] = r;
    }
}

template <bool REV, bool IMP, typename Src>
__global__ void __launch_bounds__(256) cascade_filter_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const CascadeJob &job = src.get(bid, nblk);
    constexpr int G = kGroup;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), grp = lane / G;
    const long long n = (long long)*job.in_count;
    const long long warp = ((long long)bid * blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)nblk * blockDim.x) >> 5;
    const int L = job.L, nb = job.nb;
    for (long long base = warp * 32; base < n; base += n_warps * 32) {
        const int m = (int)(n - base < 32 ? n - base : 32);
        const uint2 mine = lane < m ? job.in[base + lane] : make_uint2(0u, 0u);
        unsigned keep = 0, by_imp = 0;
        for (int r = 0; r < G; r++) {
            // round r: group grp takes entry k = r * (32 / G) + grp of the run
            const int k = r * (32 / G) + grp;
            const int q = (int)__shfl_sync(FULL, mine.x, k);
            const int t = (int)__shfl_sync(FULL, mine.y, k);
            const bool valid = k < m;
            float pr = 0.f, pi = 0.f;
            if (valid) {
                const float2 *e = job.envq + (long long)q * L;
                if (IMP) {
                    const BGap *bg = job.bgap + (long long)t * L;
#pragma unroll 8
                    for (int j = nb + gl; j < L - nb; j += G) {
                        const BGap r = bg[j];
                        const float2 ej = e[j];
                        const float2 g = __half22float2(r.g);
                        const float up = r.b - ej.x, dn = ej.y - r.b;
                        if (REV) {
                            const float d = max3f(up, dn, 0.f);
                            pr = fmaf(d, d, pr);
                        }
                        const float d = max3f(fminf(up, g.x), fminf(dn, g.y), 0.f);
                        pi = fmaf(d, d, pi);
                    }
                } else {
                    const float *b = job.train + (long long)t * L;
#pragma unroll 8
                    for (int j = nb + gl; j < L - nb; j += G) {
                        const float bj = b[j];
                        const float2 ej = e[j];
                        const float d = max3f(bj - ej.x, ej.y - bj, 0.f);
                        pr = fmaf(d, d, pr);
                    }
                }
            }
#pragma unroll
            for (int off = 1; off < G; off <<= 1) {
                if (REV) pr += __shfl_xor_sync(FULL, pr, off, G);
                if (IMP) pi += __shfl_xor_sync(FULL, pi, off, G);
            }
            bool k_keep = valid, k_imp = false;
            if (valid && gl == 0) {
                const unsigned long long kb = job.bsf[q];
                if (kb != ~0ull) {
                    const float ub = upper32(key_dist(kb), job.dtw_hi, job.abs32);
                    const long long pq = (long long)q * job.N + t;
                    if (IMP) {
                        const float si = fmaxf(lower32(pi, job.lb_lo, job.lb_abs), 0.f);
                        k_imp = __fadd_rd(job.lb[pq], si) > ub;
                    }
                    bool k_rev = false;
                    if (REV) {
                        const float lb = job.ends[pq] + pr;
                        k_rev = fmaxf(lower32(lb, job.lb_lo, job.lb_abs), 0.f) > ub;
                    }
                    k_keep = !(k_imp || k_rev);
                }
            }
            // bit k of the run's masks, from each group's first lane
            const unsigned keep_mask = __ballot_sync(FULL, gl == 0 && k_keep);
            const unsigned imp_mask = __ballot_sync(FULL, gl == 0 && k_imp);
            for (int g = 0; g < 32 / G; g++) {
                if ((keep_mask >> (g * G)) & 1u) keep |= 1u << (r * (32 / G) + g);
                if ((imp_mask >> (g * G)) & 1u) by_imp |= 1u << (r * (32 / G) + g);
            }
        }
        const int nk = __popc(keep);
        unsigned long long at = 0;
        if (lane == 0 && nk) at = atomicAdd(job.out_count, (unsigned long long)nk);
        at = __shfl_sync(FULL, at, 0);
        if (lane < m && ((keep >> lane) & 1u))
            job.out[at + __popc(keep & ((1u << lane) - 1u))] = mine;
        if (lane == 0 && job.counters && nk < m) {
            const int ni = __popc(by_imp);
            if (ni) atomicAdd(job.counters + C_IMPPRUNED, (unsigned long long)ni);
            if (m - nk - ni) atomicAdd(job.counters + C_REVPRUNED, (unsigned long long)(m - nk - ni));
        }
    }
}

// lb[p] += the second pass of the LB_Improved bridge of pair p = q N + t,
// for every pair; eight lanes per pair.
template <typename T, typename T2>
__global__ void __launch_bounds__(256)
improved_terms_kernel(const T *__restrict__ train, const T2 *__restrict__ envq,
                      const T2 *__restrict__ env2, int64_t Q, int64_t N, int L, int nb,
                      bool safe, T lb_lo, T lb_abs, T *__restrict__ lb) {
    constexpr int G = kGroup;
    const unsigned FULL = 0xffffffffu;
    const int gl = threadIdx.x & (G - 1);
    const long long n_groups = ((long long)gridDim.x * blockDim.x) / G;
    const long long total = Q * N;
    // every lane of a warp runs the same number of rounds (shuffles below)
    const long long rounds = (total + n_groups - 1) / n_groups;
    long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    for (long long r = 0; r < rounds; r++, p += n_groups) {
        const bool valid = p < total;
        T part = T(0);
        if (valid) {
            const long long q = p / N, t = p % N;
            const T *b = train + t * L;
            const T2 *e = envq + q * L;
            const T2 *o = env2 + t * L;
            for (int j = nb + gl; j < L - nb; j += G) {
                const T bj = b[j];
                const T2 ej = e[j], oj = o[j];
                const T v = keogh_term(bj, tmin(ej.y, oj.y), tmax(ej.x, oj.x));
                part = part + v;
            }
        }
#pragma unroll
        for (int off = 1; off < G; off <<= 1) part += __shfl_xor_sync(FULL, part, off, G);
        if (valid && gl == 0) {
            if (safe) {
                T s = sub_rd(mul_rd(part, lb_lo), lb_abs);
                s = s > T(0) ? s : T(0);
                lb[p] = add_rd(lb[p], s);
            } else {
                lb[p] = lb[p] + part;
            }
        }
    }
}

}  // namespace

long long cascade_filter_blocks(long long max_pairs, int sm_count) {
    if (max_pairs <= 0) return 0;
    // warps: enough for the largest possible queue, at most 64 per SM
    // (residency is what hides the load latency)
    long long warps = (max_pairs + 31) / 32;
    const long long cap = (long long)sm_count * 64;
    if (warps > cap) warps = cap;
    return (warps + 7) / 8;
}

CascadeFns cascade_filter_fns(bool rev, bool imp) {
    CascadeFns f{};
    if (rev && imp) {
        f.fn1 = cascade_filter_kernel<true, true, Src1<CascadeJob>>;
        f.fnN = cascade_filter_kernel<true, true, SrcN<CascadeJob>>;
    } else if (rev) {
        f.fn1 = cascade_filter_kernel<true, false, Src1<CascadeJob>>;
        f.fnN = cascade_filter_kernel<true, false, SrcN<CascadeJob>>;
    } else if (imp) {
        f.fn1 = cascade_filter_kernel<false, true, Src1<CascadeJob>>;
        f.fnN = cascade_filter_kernel<false, true, SrcN<CascadeJob>>;
    }
    return f;
}

cudaError_t launch_cascade_filter(const CascadeJob &job, long long max_pairs, int sm_count,
                                  cudaStream_t s) {
    const long long grid = cascade_filter_blocks(max_pairs, sm_count);
    if (grid <= 0) return cudaSuccess;
    const bool rev = job.ends != nullptr, imp = job.bgap != nullptr;
    if (!rev && !imp) return cudaErrorInvalidValue;
    cascade_filter_fns(rev, imp).fn1<<<(unsigned)grid, 256, 0, s>>>(Src1<CascadeJob>{job});
    return cudaGetLastError();
}

long long pack_bgap_blocks(long long n) {
    if (n <= 0) return 0;
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)device_sm_count() * 16;
    return blocks > cap ? cap : blocks;
}

PackFns pack_bgap_fns() {
    PackFns f;
    f.fn1 = pack_bgap_kernel<Src1<PackJob>>;
    f.fnN = pack_bgap_kernel<SrcN<PackJob>>;
    return f;
}

cudaError_t launch_pack_bgap(const float *train, float *env2, long long n, cudaStream_t s) {
    const long long blocks = pack_bgap_blocks(n);
    if (blocks <= 0) return cudaSuccess;
    PackJob j{train, env2, n};
    pack_bgap_kernel<<<(unsigned)blocks, 256, 0, s>>>(Src1<PackJob>{j});
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_improved_terms(const T *train, const T *envq, const T *env2, int64_t Q,
                                  int64_t N, int L, int nb, bool safe, T lb_lo, T lb_abs, T *lb,
                                  cudaStream_t s) {
    const long long total = Q * N;
    if (total <= 0) return cudaSuccess;
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    long long blocks = (total * kGroup + 255) / 256;
    const long long cap = (long long)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    improved_terms_kernel<T, T2><<<(unsigned)blocks, 256, 0, s>>>(
        train, reinterpret_cast<const T2 *>(envq), reinterpret_cast<const T2 *>(env2), Q, N, L,
        nb, safe, lb_lo, lb_abs, lb);
    return cudaGetLastError();
}

template cudaError_t launch_improved_terms<float>(const float *, const float *, const float *,
                                                  int64_t, int64_t, int, int, bool, float, float,
                                                  float *, cudaStream_t);
template cudaError_t launch_improved_terms<double>(const double *, const double *,
                                                   const double *, int64_t, int64_t, int, int,
                                                   bool, double, double, double *, cudaStream_t);

}  // namespace nndtw
