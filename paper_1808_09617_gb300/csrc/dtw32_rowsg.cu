// FP32 DTW (Sec. 2.1, Eq. 1) for full windows (W >= L-1), laid out by rows
// with a group of G = 8 or 16 lanes per pair (32 / G pairs per warp),
// L <= 64 G.
//
// The row layout of the one-pair-per-warp kernel: lane g of a group owns C
// consecutive columns, split into K independent parts (K = 2, one for C < 4),
// each one row behind the one before, and the rows stream through the group.
// With fewer lanes per pair the wavefront fills in K G steps instead of
// 2 x 32, which is what matters when most pairs are abandoned after a few
// dozen rows.  The pairs of a warp
// advance independently, so everything that differs between them is kept
// out of the step loop:
//  - the G C columns are placed so that column L-1 is the last column of
//    the last lane; the G C - L columns in front of column 0 hold a
//    training sentinel (their cells are +inf).  The one just before column
//    0 starts at 0, which is D(-1,-1) for cell (0,0), and holds the query's
//    own sentinel, so that the rows before the start (which see that
//    sentinel) give it delta = 0 and keep the 0 until row 0 reads it;
//  - the query enters at the group's lane 0 from a load one step ahead,
//    clamped to the series (rows past L-1 are never used);
//  - the result is picked from the last lane when its second half finishes
//    row L-1 (a select, no branch);
//  - pairs start, finish and are abandoned only every 16 steps (claims,
//    completion and the abandon test), at the same step for the whole warp.
// Abandoning uses the staircase cut of the one-pair-per-warp kernel; it is
// only tested while every computed row is below L (the drain after that
// sweeps rows past the end, whose values are never used).
#include <utility>

#include "dtw32.cuh"

namespace nndtw {
namespace {

__host__ __device__ constexpr int rowsg_min_blocks(int C) {
    return C <= 12 ? 6 : C <= 15 ? 5 : C <= 25 ? 4 : C <= 38 ? 3 : 2;
}

// The K parts of a lane's C columns: part k holds columns [part_lo(k),
// part_lo(k+1)), every part non-empty (K <= C).  Part k of lane gl works on
// row s - K gl - k at step s: each part is a dependency chain along its row,
// and the K chains of a lane are independent.  Two parts (K = 2) measured as
// fast as four on the full-window datasets of the batched workload (7.0
// Tcell/s with 16 lanes per pair at L = 1012 either way) and fill the
// wavefront in half the steps, so the kernel uses two.
template <int C> __host__ __device__ constexpr int rowsg_parts() {
    return C >= 4 ? 2 : 1;
}
template <int C, int K> __host__ __device__ constexpr int part_lo(int k) { return k * C / K; }

// One step of one lane from Din to Dout.  a[k] is part k's query value,
// hprev[k] (k >= 1) the previous step's value of the column in front of part
// k (part k-1's last column): the diagonal predecessor of part k's first cell.
template <int C, int K>
__device__ __forceinline__ void rowsg_step(const float (&Din)[C], float (&Dout)[C],
                                           const float (&B)[C], float (&a)[K], float &anext,
                                           float &diag_in, float (&hprev)[K],
                                           const float *ap, int s, int gl, int G, int L) {
    const unsigned FULL = 0xffffffffu;
    const float INF = inf_of<float>();
    // part 0 takes the query value lane gl-1's last part used at the last
    // step; lane 0 takes a[s]
    float a_in = __shfl_up_sync(FULL, a[K - 1], 1, G);
    if (gl == 0) a_in = anext;                 // query value a[s]
    anext = ap[min(s + 1, L - 1)];             // the next one (clamped)
#pragma unroll
    for (int k = K - 1; k >= 1; k--) a[k] = a[k - 1];
    a[0] = a_in;
    float left[K], diag[K];
    left[0] = __shfl_up_sync(FULL, Din[C - 1], 1, G);
    const int i0 = s - K * gl;
    diag[0] = diag_in;
    if (gl == 0) {
        left[0] = INF;
        diag[0] = (i0 == 0) ? 0.f : INF;
    }
    diag_in = left[0];
#pragma unroll
    for (int k = 1; k < K; k++) {
        left[k] = Din[part_lo<C, K>(k) - 1];
        diag[k] = hprev[k];
        hprev[k] = left[k];
    }
    constexpr int kMaxPart = (C + K - 1) / K;
#pragma unroll
    for (int c = 0; c < kMaxPart; c++) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            const int e = part_lo<C, K>(k) + c;
            if (e < part_lo<C, K>(k + 1)) {
                const float d = a[k] - B[e];
                Dout[e] = fmaf(d, d, min3f(Din[e], c == 0 ? left[k] : Dout[e - 1],
                                           c == 0 ? diag[k] : Din[e - 1]));
            }
        }
    }
}

template <int C, typename Src>
__global__ void __launch_bounds__(128, rowsg_min_blocks(C))
dtw32_rowsg_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    const int G = job.lanes;
    constexpr int K = rowsg_parts<C>();
    const float INF = inf_of<float>();
    const float APAD = -Pad<float>::v;   // query before the start: delta = +inf
    const float BPAD = Pad<float>::v;    // columns in front of column 0
    const unsigned FULL = 0xffffffffu;
    const int L = job.L;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int off = G * C - L;                 // padding columns before column 0
    const int steps_total = L + K * G - 1;     // the last part finishes row L-1 at step steps_total-1
    const int s_final = steps_total - 1;
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const long long n_groups = (long long)nblk * (blockDim.x / G);
    const bool check_bsf = job.abandon && job.bsf;

    // claims two pairs ahead per group (see the diagonal-layout kernel)
    long long nxt = ((long long)bid * blockDim.x + threadIdx.x) / G;
    long long p1;
    if (job.head) {
        unsigned long long v = 0;
        if (gl == 0) v = atomicAdd(job.head, 1ull);
        p1 = (long long)__shfl_sync(FULL, v, 0, G);
        if (gl == 0) nxt = (long long)atomicAdd(job.head, 1ull);
    } else {
        p1 = nxt;
        nxt += n_groups;
    }
    uint2 w1 = work_item(job, p1, n_work);
    // live pruning (job.lb), as in the diagonal-layout kernel
    float lb1 = 0.f;
    unsigned kb1 = ~0u;
    if (job.lb && p1 < n_work) {
        lb1 = job.lb[(long long)w1.x * job.lb_n + w1.y];
        kb1 = bsf_dist_bits(job.bsf, (int)w1.x);
    }

    float B[C], D[C], E[C];
#pragma unroll
    for (int c = 0; c < C; c++) { B[c] = BPAD; D[c] = INF; }
    long long pid = -1;
    int q = 0, t = 0, ws = 0, w = 0;
    bool done = true, finished = false;
    float ub = INF, res = INF;
    unsigned kb = ~0u;
    const float *ap = job.test;
    float a[K], hprev[K];
    float anext = 0.f, diag_in = INF;
#pragma unroll
    for (int k = 0; k < K; k++) { a[k] = APAD; hprev[k] = INF; }

    while (true) {
        // ---- start pairs (every 16 steps) ----------------------------------
        const bool need = done && !finished;
        if (__any_sync(FULL, need)) {
            if (need) {
                // claim until a pair survives the live test or the list ends
                bool take = false;
                while (!take && p1 < n_work) {
                    pid = p1;
                    q = (int)w1.x; t = (int)w1.y;
                    const float lb_cur = lb1;
                    const unsigned kb_cur = kb1;
                    if (job.head) {
                        p1 = __shfl_sync(gmask, nxt, 0, G);
                        if (gl == 0) nxt = (long long)atomicAdd(job.head, 1ull);
                    } else {
                        p1 = nxt;
                        nxt += n_groups;
                    }
                    w1 = work_item(job, p1, n_work);
                    if (job.lb && p1 < n_work) {
                        lb1 = job.lb[(long long)w1.x * job.lb_n + w1.y];
                        kb1 = bsf_dist_bits(job.bsf, (int)w1.x);
                    }
                    take = kb_cur == ~0u ||
                           !(lb_cur > upper32(__uint_as_float(kb_cur), job.dtw_hi, job.abs32));
                    if (!take && job.counters && gl == 0)
                        atomicAdd(job.counters + C_LIVEPRUNED, 1ull);
                }
                if (!take) {
                    finished = true;
                    pid = -1;
                } else {
                    ap = job.test + (long long)q * L;
                    const float *bp = job.train + (long long)t * L;
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        const int j = gl * C + c - off;
                        B[c] = j >= 0 ? bp[j] : (j == -1 ? APAD : BPAD);
                        D[c] = j == -1 ? 0.f : INF;
                    }
#pragma unroll
                    for (int k = 0; k < K; k++) { a[k] = APAD; hprev[k] = INF; }
                    anext = ap[0];
                    diag_in = INF;
                    res = INF; ub = INF;
                    kb = check_bsf ? bsf_dist_bits(job.bsf, q) : ~0u;
                    ws = w;
                    done = false;
                    if (job.counters && gl == 0) atomicAdd(job.counters + C_STARTED, 1ull);
                }
            }
        }
        if (__all_sync(FULL, finished)) break;

        // ---- 16 steps, two per iteration (D -> E -> D) ---------------------
#pragma unroll 1
        for (int it = 0; it < 8; it++) {
            const int s = w - ws;
            rowsg_step<C, K>(D, E, B, a, anext, diag_in, hprev, ap, s, gl, G, L);
            res = s == s_final ? E[C - 1] : res;
            rowsg_step<C, K>(E, D, B, a, anext, diag_in, hprev, ap, s + 1, gl, G, L);
            res = s + 1 == s_final ? D[C - 1] : res;
            w += 2;
        }
        const int sd = w - ws;     // steps done in the current pair

        // ---- completion -----------------------------------------------------
        if (!done && sd >= steps_total) {
            const float r = __shfl_sync(gmask, res, G - 1, G);
            if (gl == 0) {
                if (job.out) job.out[pid] = r;
                if (job.bsf) {
                    const unsigned long long key = pack_key(r, (uint32_t)t);
                    const unsigned long long old = atomicMin(job.bsf + q, key);
                    const unsigned long long cur = old < key ? old : key;
                    const float ubn = upper32(key_dist(cur), job.dtw_hi, job.abs32);
                    if (job.cand && lower32(r, job.dtw_lo, job.abs32) <= ubn) {
                        const unsigned long long slot = atomicAdd(job.cand_count, 1ull);
                        Cand cd;
                        cd.q = q; cd.t = t; cd.d = r; cd.pad = 0;
                        job.cand[slot] = cd;
                    }
                }
                if (job.counters) atomicAdd(job.counters + C_CELLS, (unsigned long long)L * L);
            }
            done = true;
        }

        // ---- early abandoning (selects per group) ---------------------------
        if (job.abandon) {
            // the cut: every part's last computed row (D), and the cell one
            // row above it in the column in front of every part (hprev inside
            // the lane, diag_in across lanes)
            float mn = diag_in;
#pragma unroll
            for (int k = 1; k < K; k++) mn = fminf(mn, hprev[k]);
#pragma unroll
            for (int c = 0; c < C; c++) mn = fminf(mn, D[c]);
            for (int o = 1; o < G; o <<= 1) mn = fminf(mn, __shfl_xor_sync(FULL, mn, o, G));
            const bool live = !done && sd <= L;    // every computed row is below L
            const unsigned kbn = check_bsf ? bsf_dist_bits(job.bsf, q) : ~0u;
            const float ubn = kb != ~0u ? upper32(__uint_as_float(kb), job.dtw_hi, job.abs32) : ub;
            ub = live ? ubn : ub;
            kb = live ? kbn : kb;
            const bool drop = live && lower32(mn, job.dtw_lo, job.abs32) > ub;
            if (drop && gl == 0 && job.counters) {
                // part h of lane g has finished rows 0 .. sd-1 - (K g + h)
                long long cells = 0;
                for (int g = 0; g < G; g++) {
                    for (int h = 0; h < K; h++) {
                        const int lo = max(g * C + part_lo<C, K>(h) - off, 0);
                        const int hi = min(g * C + part_lo<C, K>(h + 1) - off, L);
                        const int rows = min(sd - 1 - (K * g + h), L - 1) + 1;
                        if (rows > 0 && hi > lo) cells += (long long)(hi - lo) * rows;
                    }
                }
                atomicAdd(job.counters + C_ABANDONED, 1ull);
                atomicAdd(job.counters + C_CELLS, (unsigned long long)cells);
            }
            done = done || drop;
        }
    }
}

template <int C> Dtw32Fn1 rowsg_fn1() { return &dtw32_rowsg_kernel<C, Src1<DtwJob32>>; }
template <int C> Dtw32FnN rowsg_fnn() { return &dtw32_rowsg_kernel<C, SrcN<DtwJob32>>; }
template <int... Cs>
void pick_rowsg(int c, std::integer_sequence<int, Cs...>, Dtw32Fn1 *f1, Dtw32FnN *fn) {
    const Dtw32Fn1 a[] = {rowsg_fn1<Cs + 1>()...};
    const Dtw32FnN b[] = {rowsg_fnn<Cs + 1>()...};
    const bool ok = c >= 1 && c <= (int)sizeof...(Cs);
    *f1 = ok ? a[c - 1] : nullptr;
    *fn = ok ? b[c - 1] : nullptr;
}

}  // namespace

bool dtw32_rowsg_ok(int L, int W, int G) {
    return (G == 8 || G == 16) && W >= L - 1 && L >= 1 && L <= 64 * G;
}

cudaError_t plan_dtw32_rowsg(const DtwJob32 &job, int G, int sm_count, Dtw32Plan *p) {
    if (!dtw32_rowsg_ok(job.L, job.W, G)) return cudaErrorNotSupported;
    const int C = (job.L + G - 1) / G;
    pick_rowsg(C, std::make_integer_sequence<int, 64>{}, &p->fn1, &p->fnN);
    if (!p->fn1) return cudaErrorNotSupported;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->fn1, 128, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        const long long per_block = 128 / G;
        const long long need = n > 0 ? (n + per_block - 1) / per_block : 0;
        if (need < grid) grid = need;
    }
    p->threads = 128;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = G;
    return cudaSuccess;
}

}  // namespace nndtw
