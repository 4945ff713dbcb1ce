// FP32 DTW (Sec. 2.1, Eq. 1) for full windows (W >= L-1, unconstrained
// DTW), L <= 32 * 64: one pair per warp, laid out by rows.
//
// Lane g owns C consecutive columns j = gC .. gC+C-1 of the cost matrix and
// keeps their training values B_j and their latest D values in registers.
// The query values stream through the warp: row i reaches lane g at step
// i + g (one shuffle per step), so at every step lane g updates row s - g
// of its columns, needing from lane g-1 only that row's value in column
// gC-1 (computed at the previous step, one shuffle) and the row above's
// (kept from the step before).  Unlike the diagonal layout used for banded
// windows, no cell outside the L x L matrix is ever swept, so a full window
// costs L (L + 31) lane-cells per pair instead of about 2 L^2.  Lanes update
// only rows 0..L-1, so after the sweep the lane owning column L-1 still
// holds D(L-1, L-1).  Early abandoning takes the minimum over the last
// computed row of every column block together with, for each block, the
// cell of the row above it in the previous block's last column: a warping
// path leaves the computed region either from a block's last computed row
// or by a diagonal step out of that cell, so one of them lies on every path.
#include <utility>

#include "dtw32.cuh"

namespace nndtw {

template <int C>
__global__ void __launch_bounds__(128)
dtw32_rows_kernel(DtwJob32 job) {
    const float INF = inf_of<float>();
    const int L = job.L;
    const int lane = threadIdx.x & 31;
    const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const int last_lane = (L - 1) / C, last_c = (L - 1) % C;
    long long next_static = warp_g;

    while (true) {
        long long p;
        if (job.head) {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(job.head, 1ull);
            p = (long long)__shfl_sync(0xffffffffu, v, 0);
        } else {
            p = next_static;
            next_static += n_warps;
        }
        if (p >= n_work) break;
        int q, t;
        if (job.pairs) {
            const uint2 pr = job.pairs[p];
            q = (int)pr.x; t = (int)pr.y;
        } else {
            q = (int)p; t = (int)key_idx(job.seed_keys[p]);
        }
        const float *ap = job.test + (long long)q * L;
        const float *bp = job.train + (long long)t * L;
        float ub = INF;
        if (job.abandon && job.bsf) {
            const unsigned long long kb = *((volatile unsigned long long *)job.bsf + q);
            if (kb != ~0ull) ub = upper32(key_dist(kb), job.dtw_hi, job.abs32);
        }
        if (lane == 0 && job.counters) atomicAdd(job.counters + C_STARTED, 1ull);

        float B[C], D[C];
#pragma unroll
        for (int c = 0; c < C; c++) {
            const int j = lane * C + c;
            B[c] = j < L ? bp[j] : Pad<float>::v;   // columns past L: delta = +inf
            D[c] = INF;
        }
        float a_cur = 0.f;                 // query value of this lane's current row
        float a_next = ap[0];              // lane 0's value for the next step
        float diag_in = INF;               // D(i-1, gC-1) from lane g-1
        bool abandoned = false;
        const int steps = L + 31;
        int s = 0;
        for (; s < steps; s++) {
            // stream the query: lane g receives lane g-1's value of the last step
            float a_in = __shfl_up_sync(0xffffffffu, a_cur, 1);
            if (lane == 0) {
                a_in = a_next;
                a_next = (s + 1 < L) ? ap[s + 1] : 0.f;
            }
            a_cur = a_in;
            // row s - lane of column gC-1 from lane g-1 (computed last step)
            float left = __shfl_up_sync(0xffffffffu, D[C - 1], 1);
            const int i = s - lane;
            float diag = diag_in;
            if (lane == 0) {
                left = INF;
                diag = (i == 0) ? 0.f : INF;
            }
            diag_in = left;
            if (i >= 0 && i < L) {
                float l = left, dg = diag;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    const float old = D[c];
                    const float d = a_cur - B[c];
                    D[c] = fmaf(d, d, min3f(old, l, dg));
                    dg = old;
                    l = D[c];
                }
            }
            if (job.abandon && (s & 15) == 15) {
                // the cut: every lane's last computed row, plus the row above
                // in the last column of the lane to its left (diag_in), through
                // which a path can leave diagonally
                float mn = diag_in;
#pragma unroll
                for (int c = 0; c < C; c++) mn = fminf(mn, D[c]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
                if (job.bsf) {
                    const unsigned long long kb = *((volatile unsigned long long *)job.bsf + q);
                    if (kb != ~0ull) ub = upper32(key_dist(kb), job.dtw_hi, job.abs32);
                }
                if (lower32(mn, job.dtw_lo, job.abs32) > ub) { abandoned = true; break; }
            }
        }
        float res = INF;
#pragma unroll
        for (int c = 0; c < C; c++) res = (lane == last_lane && c == last_c) ? D[c] : res;
        res = __shfl_sync(0xffffffffu, res, last_lane);
        if (lane == 0) {
            if (job.counters) {
                long long cells = (long long)L * L;
                if (abandoned) {   // lane g finished rows 0 .. min(s-g, L-1) of its columns
                    cells = 0;
                    for (int g = 0; g < 32; g++) {
                        const int cols = min(max(L - g * C, 0), C);
                        const int rows = min(s - g, L - 1) + 1;
                        if (rows > 0) cells += (long long)cols * rows;
                    }
                }
                atomicAdd(job.counters + C_CELLS, (unsigned long long)cells);
                if (abandoned) atomicAdd(job.counters + C_ABANDONED, 1ull);
            }
            if (!abandoned) {
                if (job.out) job.out[p] = res;
                if (job.bsf) {
                    const unsigned long long key = pack_key(res, (uint32_t)t);
                    const unsigned long long old = atomicMin(job.bsf + q, key);
                    const unsigned long long cur = old < key ? old : key;
                    const float ubn = upper32(key_dist(cur), job.dtw_hi, job.abs32);
                    if (job.cand && lower32(res, job.dtw_lo, job.abs32) <= ubn) {
                        const unsigned long long slot = atomicAdd(job.cand_count, 1ull);
                        Cand cd;
                        cd.q = q; cd.t = t; cd.d = res; cd.pad = 0;
                        job.cand[slot] = cd;
                    }
                }
            }
        }
    }
}

namespace {
using RowsFn = void (*)(DtwJob32);
template <int C> RowsFn rows_fn() { return &dtw32_rows_kernel<C>; }
template <int... Cs> RowsFn pick_rows(int c, std::integer_sequence<int, Cs...>) {
    RowsFn fns[] = {rows_fn<Cs + 1>()...};
    return (c >= 1 && c <= (int)sizeof...(Cs)) ? fns[c - 1] : nullptr;
}
}  // namespace

bool dtw32_rows_ok(int L, int W) { return W >= L - 1 && L >= 1 && L <= 32 * 64; }

cudaError_t launch_dtw32_rows(const DtwJob32 &job, int sm_count, cudaStream_t s) {
    const int C = (job.L + 31) / 32;
    RowsFn fn = pick_rows(C, std::make_integer_sequence<int, 64>{});
    if (!fn) return cudaErrorNotSupported;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 128, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        if (n <= 0) return cudaSuccess;
        const long long need = (n + 3) / 4;
        if (need < grid) grid = need;
    }
    fn<<<(unsigned)grid, 128, 0, s>>>(job);
    return cudaGetLastError();
}

}  // namespace nndtw
