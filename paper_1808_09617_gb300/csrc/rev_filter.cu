// The cascade's second bound: LB_Enhanced^V(B, A), Eq. 7 with the two series
// exchanged, tested on the pairs that survived LB_Enhanced^V(A, B) before
// their DTW is due.
//
// Its two ends and its bands equal those of LB_Enhanced(A, B) (a band takes
// the minimum over the cells (i, j) and (j, i) alike), which the bound pass
// stores per pair; what differs is the bridge, here LB_Keogh of the training
// series B against the query's envelope over [n_b, L - n_b).  A pair is
// dropped when the bound, scaled down by the bound's rounding margin,
// exceeds (strictly) the query's upper bound at this point: the inflated
// DTW of its first candidate.
//
// Eight lanes per pair (four pairs per warp at a time), each lane loading
// every eighth element, so that the loads of a pair are coalesced and four
// pairs' loads are in flight per warp; consecutive queue entries mostly share
// their query (the compaction appends them query by query), so its envelope
// is mostly served by L1.  A warp takes 32 consecutive queue entries and
// appends the survivors with one atomic, so the queue's order (most
// promising bucket first) is kept within each run of 32.
#include "internal.cuh"

namespace nndtw {
namespace {

__global__ void __launch_bounds__(256)
rev_filter_kernel(const uint2 *__restrict__ in, const unsigned long long *__restrict__ in_count,
                  const float *__restrict__ train, const float2 *__restrict__ envq,
                  const float *__restrict__ ends, long long N, int L, int nb,
                  const unsigned long long *__restrict__ bsf, float lb_lo, float lb_abs,
                  float dtw_hi, float abs32, uint2 *__restrict__ out,
                  unsigned long long *__restrict__ out_count, unsigned long long *counters) {
    constexpr int G = 8;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), grp = lane / G;
    const long long n = (long long)*in_count;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * 32; base < n; base += n_warps * 32) {
        const int m = (int)(n - base < 32 ? n - base : 32);
        const uint2 mine = lane < m ? in[base + lane] : make_uint2(0u, 0u);
        unsigned keep = 0;
        for (int r = 0; r < G; r++) {
            // round r: group grp takes entry k = r * (32 / G) + grp of the run
            const int k = r * (32 / G) + grp;
            const int q = (int)__shfl_sync(FULL, mine.x, k);
            const int t = (int)__shfl_sync(FULL, mine.y, k);
            const bool valid = k < m;
            float part = 0.f;
            if (valid) {
                const float *b = train + (long long)t * L;
                const float2 *e = envq + (long long)q * L;
#pragma unroll 4
                for (int j = nb + gl; j < L - nb; j += G) {
                    const float bj = b[j];
                    const float2 ej = e[j];
                    const float d = bj - fminf(fmaxf(bj, ej.y), ej.x);
                    part = fmaf(d, d, part);
                }
            }
#pragma unroll
            for (int off = 1; off < G; off <<= 1) part += __shfl_xor_sync(FULL, part, off, G);
            bool k_keep = valid;
            if (valid && gl == 0) {
                const unsigned long long kb = bsf[q];
                if (kb != ~0ull) {
                    const float lb = ends[(long long)q * N + t] + part;
                    const float safe = fmaxf(__fmul_rd(lb, lb_lo) - lb_abs, 0.f);
                    k_keep = !(safe > upper32(key_dist(kb), dtw_hi, abs32));
                }
            }
            // bit k of the run's keep mask, from each group's first lane
            const unsigned kb_mask = __ballot_sync(FULL, gl == 0 && k_keep);
            for (int g = 0; g < 32 / G; g++)
                if ((kb_mask >> (g * G)) & 1u) keep |= 1u << (r * (32 / G) + g);
        }
        const int nk = __popc(keep);
        unsigned long long at = 0;
        if (lane == 0 && nk) at = atomicAdd(out_count, (unsigned long long)nk);
        at = __shfl_sync(FULL, at, 0);
        if (lane < m && ((keep >> lane) & 1u))
            out[at + __popc(keep & ((1u << lane) - 1u))] = mine;
        if (lane == 0 && counters && nk < m)
            atomicAdd(counters + C_REVPRUNED, (unsigned long long)(m - nk));
    }
}

}  // namespace

cudaError_t launch_rev_filter(const uint2 *in, const unsigned long long *in_count,
                              const float *train, const float2 *envq, const float *ends,
                              long long N, int L, int nb, const unsigned long long *bsf,
                              float lb_lo, float lb_abs, float dtw_hi, float abs32, uint2 *out,
                              unsigned long long *out_count, unsigned long long *counters,
                              long long max_pairs, int sm_count, cudaStream_t s) {
    if (max_pairs <= 0) return cudaSuccess;
    // warps: enough for the largest possible queue, at most 64 per SM
    // (residency is what hides the load latency)
    long long warps = (max_pairs + 31) / 32;
    const long long cap = (long long)sm_count * 64;
    if (warps > cap) warps = cap;
    const unsigned grid = (unsigned)((warps + 7) / 8);
    rev_filter_kernel<<<grid, 256, 0, s>>>(in, in_count, train, envq, ends, N, L, nb, bsf, lb_lo,
                                           lb_abs, dtw_hi, abs32, out, out_count, counters);
    return cudaGetLastError();
}

}  // namespace nndtw
