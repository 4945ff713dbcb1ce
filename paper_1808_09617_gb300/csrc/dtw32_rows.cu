// FP32 DTW (Sec. 2.1, Eq. 1) for full windows (W >= L-1, unconstrained
// DTW), L <= 32 * 64: one pair per warp, laid out by rows.
//
// Lane g owns C consecutive columns j = gC .. gC+C-1 of the cost matrix and
// keeps their training values B_j and their latest D values in registers.
// The columns of a lane form two halves (K = 2; one when C < 4), each a
// dependency chain along its row, and the second half runs one row behind
// the first so that the two chains are independent.  The query values
// stream through the warp: the first half of lane g works on row s - K g at
// step s, needing from lane g-1 only that row's value in column gC-1
// (computed at the previous step, one shuffle) and the row above's (kept
// from the step before).  The row values alternate between two register
// arrays, two steps per loop iteration, so that no value is ever copied.  Unlike the diagonal layout used for banded
// windows, no cell outside the L x L matrix is ever swept, so a full window
// costs L (L + 32K - 1) lane-cells per pair instead of about 2 L^2.  Rows
// past L-1 are never updated, so after the sweep the lane owning column L-1
// still holds D(L-1, L-1).
#include <utility>

#include "dtw32.cuh"

namespace nndtw {

// Resident 128-thread blocks per SM asked of the register allocator for C
// columns per lane (the kernel needs about 2C + 80 registers); from a compile
// sweep, the largest count without spills.
__host__ __device__ constexpr int rows_min_blocks(int C) {
    return C <= 12 ? 6 : C <= 15 ? 5 : C <= 25 ? 4 : C <= 38 ? 3 : 2;
}

// One step of one lane, from the row values in Din to those in Dout (two
// register arrays used in turn, so that no value is copied between steps).
// The first half of the lane's columns (0..C0-1) advances to row
// i0 = s - K g, the second half (C0..C-1, when K = 2) to row i0 - 1; each
// half is a chain Dout[c] = fma(d, d, min3(Din[c], Dout[c-1], Din[c-1]))
// along its columns, and the two chains are independent.  Rows before the
// start see the query sentinel and come out +inf; in the drain (DRAIN: some
// rows past L-1) a half whose row is past the end passes its values on.
template <int C, int K, int C0, bool DRAIN>
__device__ __forceinline__ void rows_advance(const float (&Din)[C], float (&Dout)[C],
                                             const float (&B)[C], float &a0, float &a1,
                                             float &qa, float &qn, float &diag_in, float &h0prev,
                                             const float *ap, int s, int lane, int L) {
    const unsigned FULL = 0xffffffffu;
    const float INF = inf_of<float>();
    // the query: lane g's new first-half value is the one lane g-1's last
    // half used at the last step; lane 0 takes a[s] from the chunk
    float a_in = __shfl_up_sync(FULL, K == 2 ? a1 : a0, 1);
    const float feed = __shfl_sync(FULL, qa, s & 31);
    if (lane == 0) a_in = feed;
    if (K == 2) a1 = a0;
    a0 = a_in;
    if ((s & 31) == 31) {
        qa = qn;
        const int idx = s + 33 + lane;
        qn = idx < L ? ap[idx] : 0.f;
    }
    // first half: D(i0, gC-1) and D(i0-1, gC-1) from lane g-1's last column
    float left0 = __shfl_up_sync(FULL, Din[C - 1], 1);
    const int i0 = s - K * lane;
    float diag0 = diag_in;
    if (lane == 0) {
        left0 = INF;
        diag0 = (i0 == 0) ? 0.f : INF;
    }
    diag_in = left0;
    // second half: the first half's last column one and two rows up
    const float left1 = Din[C0 - 1];
    const float diag1 = h0prev;
    if (K == 2) h0prev = left1;
    const bool run0 = !DRAIN || i0 < L;
    const bool run1 = !DRAIN || i0 - 1 < L;
#pragma unroll
    for (int c = 0; c < C0; c++) {
        {
            const float d = a0 - B[c];
            const float v = fmaf(d, d, min3f(Din[c], c == 0 ? left0 : Dout[c - 1],
                                             c == 0 ? diag0 : Din[c - 1]));
            Dout[c] = run0 ? v : Din[c];
        }
        if (K == 2 && C0 + c < C) {
            const int e = C0 + c;
            const float d = a1 - B[e];
            const float v = fmaf(d, d, min3f(Din[e], c == 0 ? left1 : Dout[e - 1],
                                             c == 0 ? diag1 : Din[e - 1]));
            Dout[e] = run1 ? v : Din[e];
        }
    }
}

// Early abandoning.  The computed cells form a staircase whose row extent
// drops by at most one from each half-block of columns to the next, so every
// warping path leaves it from a half-block's last computed row, or
// diagonally out of the cell one row above that in the previous half-block's
// last column (h0prev inside a lane, diag_in across lanes).  The minimum over
// those cells is a lower bound of D(L-1, L-1); scaled down by the FP32
// margin, a value above the query's upper bound abandons the pair.  The
// bound uses the query best read at the previous check and requests the
// next one.
template <int C>
__device__ __forceinline__ bool rows_cut_exceeds(const float (&D)[C], float diag_in, float h0prev,
                                                 unsigned &kb, float &ub, const DtwJob32 &job,
                                                 int q) {
    float mn = fminf(diag_in, h0prev);
#pragma unroll
    for (int c = 0; c < C; c++) mn = fminf(mn, D[c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    if (job.bsf) {
        if (kb != ~0u) ub = upper32(__uint_as_float(kb), job.dtw_hi, job.abs32);
        kb = bsf_dist_bits(job.bsf, q);
    }
    return lower32(mn, job.dtw_lo, job.abs32) > ub;
}

template <int C, typename Src>
__global__ void __launch_bounds__(128, rows_min_blocks(C))
dtw32_rows_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    // K independent dependency chains per lane: with K = 2 the lane's columns
    // are split into halves, the second half one row behind the first.
    constexpr int K = C >= 4 ? 2 : 1;
    constexpr int C0 = K == 2 ? (C + 1) / 2 : C;   // columns of the first half
    const float INF = inf_of<float>();
    const float APAD = -Pad<float>::v;   // query before the start: delta = +inf
    const unsigned FULL = 0xffffffffu;
    const int L = job.L;
    const int lane = threadIdx.x & 31;
    const int warp_g = (bid * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (nblk * blockDim.x) >> 5;
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const int last_lane = (L - 1) / C, last_c = (L - 1) % C;
    const bool check_bsf = job.abandon && job.bsf;

    // Claims run two pairs ahead so that no memory latency sits between two
    // sweeps: p1 is the next pair (its item w1 already requested).
    long long nxt = warp_g;   // next static index, or lane 0's claim in flight
    long long p1;
    if (job.head) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(job.head, 1ull);
        p1 = (long long)__shfl_sync(FULL, v, 0);
        if (lane == 0) nxt = (long long)atomicAdd(job.head, 1ull);
    } else {
        p1 = nxt;
        nxt += n_warps;
    }
    uint2 w1 = work_item(job, p1, n_work);
    // live pruning (job.lb), as in the diagonal-layout kernel
    float lb1 = 0.f;
    unsigned kb1 = ~0u;
    if (job.lb && p1 < n_work) {
        lb1 = job.lb[(long long)w1.x * job.lb_n + w1.y];
        kb1 = bsf_dist_bits(job.bsf, (int)w1.x);
    }

    while (true) {
        const long long p = p1;
        if (p >= n_work) break;
        const int q = (int)w1.x, t = (int)w1.y;
        const float lb_cur = lb1;
        const unsigned kb_cur = kb1;
        if (job.head) {
            p1 = __shfl_sync(FULL, nxt, 0);
            if (lane == 0) nxt = (long long)atomicAdd(job.head, 1ull);
        } else {
            p1 = nxt;
            nxt += n_warps;
        }
        w1 = work_item(job, p1, n_work);
        if (job.lb && p1 < n_work) {
            lb1 = job.lb[(long long)w1.x * job.lb_n + w1.y];
            kb1 = bsf_dist_bits(job.bsf, (int)w1.x);
        }
        if (kb_cur != ~0u && lb_cur > upper32(__uint_as_float(kb_cur), job.dtw_hi, job.abs32)) {
            if (lane == 0 && job.counters) atomicAdd(job.counters + C_LIVEPRUNED, 1ull);
            continue;
        }

        const float *ap = job.test + (long long)q * L;
        const float *bp = job.train + (long long)t * L;
        unsigned kb = ~0u;
        if (check_bsf) kb = bsf_dist_bits(job.bsf, q);
        float ub = INF;
        if (lane == 0 && job.counters) atomicAdd(job.counters + C_STARTED, 1ull);

        float B[C], D[C], E[C];
#pragma unroll
        for (int c = 0; c < C; c++) {
            const int j = lane * C + c;
            B[c] = j < L ? bp[j] : Pad<float>::v;   // columns past L: delta = +inf
            D[c] = INF;
        }
        // The query enters at lane 0, one value per step, from 32-value chunks
        // held one per lane (qa: the current chunk, qn: the next, requested a
        // chunk ahead).
        float qa = lane < L ? ap[lane] : 0.f;
        float qn = 32 + lane < L ? ap[32 + lane] : 0.f;
        float a0 = APAD, a1 = APAD;        // query values of the halves' rows
        float diag_in = INF;               // D(i0-1, gC-1) from lane g-1
        float h0prev = INF;                // first half's last column, one row up
        bool abandoned = false;
        const int steps = L + 32 * K - 1;
        // Two steps per iteration (D -> E -> D); every row is below L while
        // s + 1 < L, and the drain runs the remaining steps (a step past the
        // last one changes nothing).  Checks every 8 iterations.
        int s = 0, it = 0;
        for (; s + 1 < L; s += 2) {
            rows_advance<C, K, C0, false>(D, E, B, a0, a1, qa, qn, diag_in, h0prev, ap, s, lane, L);
            rows_advance<C, K, C0, false>(E, D, B, a0, a1, qa, qn, diag_in, h0prev, ap, s + 1,
                                          lane, L);
            if (job.abandon && (++it & 7) == 0 &&
                rows_cut_exceeds<C>(D, diag_in, h0prev, kb, ub, job, q)) {
                abandoned = true;
                break;
            }
        }
        if (!abandoned) {
            for (; s < steps; s += 2) {
                rows_advance<C, K, C0, true>(D, E, B, a0, a1, qa, qn, diag_in, h0prev, ap, s,
                                             lane, L);
                rows_advance<C, K, C0, true>(E, D, B, a0, a1, qa, qn, diag_in, h0prev, ap, s + 1,
                                             lane, L);
                if (job.abandon && (++it & 7) == 0 &&
                    rows_cut_exceeds<C>(D, diag_in, h0prev, kb, ub, job, q)) {
                    abandoned = true;
                    break;
                }
            }
        }
        float res = INF;
#pragma unroll
        for (int c = 0; c < C; c++) res = (lane == last_lane && c == last_c) ? D[c] : res;
        res = __shfl_sync(FULL, res, last_lane);
        if (lane == 0) {
            if (job.counters) {
                long long cells = (long long)L * L;
                if (abandoned) {   // half-block b of lane g finished rows 0 .. s+1 - K g - b
                    cells = 0;
                    for (int g = 0; g < 32; g++) {
                        for (int h = 0; h < K; h++) {
                            const int lo = g * C + (h ? C0 : 0);
                            const int hi = g * C + (h ? C : C0);
                            const int cols = min(max(L - lo, 0), hi - lo);
                            const int rows = min(s + 1 - (K * g + h), L - 1) + 1;
                            if (rows > 0 && cols > 0) cells += (long long)cols * rows;
                        }
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
template <int C> Dtw32Fn1 rows_fn1() { return &dtw32_rows_kernel<C, Src1<DtwJob32>>; }
template <int C> Dtw32FnN rows_fnn() { return &dtw32_rows_kernel<C, SrcN<DtwJob32>>; }
template <int... Cs>
void pick_rows(int c, std::integer_sequence<int, Cs...>, Dtw32Fn1 *f1, Dtw32FnN *fn) {
    const Dtw32Fn1 a[] = {rows_fn1<Cs + 1>()...};
    const Dtw32FnN b[] = {rows_fnn<Cs + 1>()...};
    const bool ok = c >= 1 && c <= (int)sizeof...(Cs);
    *f1 = ok ? a[c - 1] : nullptr;
    *fn = ok ? b[c - 1] : nullptr;
}
}  // namespace

bool dtw32_rows_ok(int L, int W) { return W >= L - 1 && L >= 1 && L <= 32 * 64; }

cudaError_t plan_dtw32_rows(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    const int C = (job.L + 31) / 32;
    pick_rows(C, std::make_integer_sequence<int, 64>{}, &p->fn1, &p->fnN);
    if (!p->fn1) return cudaErrorNotSupported;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->fn1, 128, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        const long long need = n > 0 ? (n + 3) / 4 : 0;
        if (need < grid) grid = need;
    }
    p->threads = 128;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = 32;
    return cudaSuccess;
}

}  // namespace nndtw
