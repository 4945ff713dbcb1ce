// FP32 DTW (Sec. 2.1, Eq. 1) for full windows of long series, 2048 < L <=
// 8192: the row layout of the one-pair-per-warp kernel spread over a CTA of
// NW warps (four up to L = 4096, eight beyond; 32 NW lanes, C = ceil(L / (32
// NW)) columns each).
//
// Inside a warp the lanes exchange values by shuffles exactly as in that
// kernel: the query streams from lane to lane, and each lane needs the last
// column of the lane to its left one step late.  Across warps, the last lane
// of warp w leaves after each step the two values the first lane of warp w+1
// needs at the next step (its query value and its last column) in shared
// memory, and one barrier per step orders the exchange.  The slots are used
// in turn by step modulo 3: a warp can run at most one step ahead of
// another (the barrier), so a slot is never rewritten before it is read.
// Early abandoning uses the same staircase cut, reduced over the CTA.
#include <utility>

#include "dtw32.cuh"

namespace nndtw {
namespace {

// resident CTAs per SM (of NW warps) for C columns per lane
__host__ __device__ constexpr int rowsc_min_blocks(int C, int NW) {
    return (C <= 20 ? 4 : 3) * 4 / NW > 0 ? (C <= 20 ? 4 : 3) * 4 / NW : 1;
}

// One step of one lane (global lane g of the CTA), from Din to Dout: as in
// the one-pair-per-warp kernel, with the first lane of warps 1..3 taking its
// left neighbour's values from the exchange slots (ax: query value, lx: last
// column) instead of a shuffle.
template <int C, int K, int C0, bool DRAIN>
__device__ __forceinline__ void rowsc_advance(const float (&Din)[C], float (&Dout)[C],
                                              const float (&B)[C], float &a0, float &a1,
                                              float &qa, float &qn, float &diag_in,
                                              float &h0prev, const float *ap, int s, int lane,
                                              int g, int L, float ax, float lx) {
    const unsigned FULL = 0xffffffffu;
    const float INF = inf_of<float>();
    float a_in = __shfl_up_sync(FULL, K == 2 ? a1 : a0, 1);
    const float feed = __shfl_sync(FULL, qa, s & 31);
    if (lane == 0) a_in = (g == 0) ? feed : ax;
    if (K == 2) a1 = a0;
    a0 = a_in;
    if ((s & 31) == 31) {
        qa = qn;
        const int idx = s + 33 + lane;
        qn = idx < L ? ap[idx] : 0.f;
    }
    float left0 = __shfl_up_sync(FULL, Din[C - 1], 1);
    if (lane == 0) left0 = (g == 0) ? INF : lx;
    const int i0 = s - K * g;
    float diag0 = diag_in;
    if (g == 0) diag0 = (i0 == 0) ? 0.f : INF;
    diag_in = left0;
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

template <int C, int NW, typename Src>
__global__ void __launch_bounds__(32 * NW, rowsc_min_blocks(C, NW))
dtw32_rowsc_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    constexpr int kWarps = NW, kLanes = 32 * NW;
    constexpr int K = C >= 4 ? 2 : 1;
    constexpr int C0 = K == 2 ? (C + 1) / 2 : C;
    const float INF = inf_of<float>();
    const float APAD = -Pad<float>::v;
    const unsigned FULL = 0xffffffffu;
    const int L = job.L;
    const int g = threadIdx.x, lane = g & 31, warp = g >> 5;
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const int last_g = (L - 1) / C, last_c = (L - 1) % C;
    const bool check_bsf = job.abandon && job.bsf;

    __shared__ float xa[3][kWarps], xl[3][kWarps];   // exchange slots (step mod 3, warp)
    __shared__ float red[kWarps];
    __shared__ long long claim;
    __shared__ int stop;
    __shared__ float result;

    long long next_static = bid;
    while (true) {
        long long p;
        if (job.head) {
            if (g == 0) claim = (long long)atomicAdd(job.head, 1ull);
            __syncthreads();
            p = claim;
            __syncthreads();
        } else {
            p = next_static;
            next_static += nblk;
        }
        if (p >= n_work) break;
        const uint2 w1 = work_item(job, p, n_work);
        const int q = (int)w1.x, t = (int)w1.y;
        const float *ap = job.test + (long long)q * L;
        const float *bp = job.train + (long long)t * L;
        unsigned kb = ~0u;
        if (check_bsf) kb = bsf_dist_bits(job.bsf, q);
        float ub = INF;
        if (g == 0 && job.counters) atomicAdd(job.counters + C_STARTED, 1ull);

        float B[C], D[C], E[C];
#pragma unroll
        for (int c = 0; c < C; c++) {
            const int j = g * C + c;
            B[c] = j < L ? bp[j] : Pad<float>::v;
            D[c] = INF;
        }
        float qa = lane < L ? ap[lane] : 0.f;
        float qn = 32 + lane < L ? ap[32 + lane] : 0.f;
        float a0 = APAD, a1 = APAD, diag_in = INF, h0prev = INF;
        if (g < kWarps) { xa[2][g] = APAD; xl[2][g] = INF; }   // "step -1"
        __syncthreads();
        bool abandoned = false;
        const int steps = L + K * kLanes - 1;
        int s = 0, it = 0;
        // one step and the exchange behind it; DRAIN as in rowsc_advance
#define NNDTW_ROWSC_STEP(DIN, DOUT, DRAIN)                                                    \
        {                                                                                     \
            const int r = (s + 2) % 3, wsl = s % 3;                                           \
            const float ax = warp ? xa[r][warp - 1] : 0.f;                                    \
            const float lx = warp ? xl[r][warp - 1] : 0.f;                                    \
            rowsc_advance<C, K, C0, DRAIN>(DIN, DOUT, B, a0, a1, qa, qn, diag_in, h0prev, ap, \
                                           s, lane, g, L, ax, lx);                            \
            if (lane == 31) { xa[wsl][warp] = K == 2 ? a1 : a0; xl[wsl][warp] = DOUT[C - 1]; } \
            __syncthreads();                                                                  \
            s++;                                                                              \
        }
        for (bool drain = false;; ) {
            if (!drain && s + 1 >= L) drain = true;
            if (s >= steps) break;
            if (!drain) {
                NNDTW_ROWSC_STEP(D, E, false)
                NNDTW_ROWSC_STEP(E, D, false)
            } else {
                NNDTW_ROWSC_STEP(D, E, true)
                NNDTW_ROWSC_STEP(E, D, true)
            }
            if (job.abandon && (++it & 7) == 0) {
                // the staircase cut of the one-pair-per-warp kernel, over the CTA
                float mn = fminf(diag_in, h0prev);
#pragma unroll
                for (int c = 0; c < C; c++) mn = fminf(mn, D[c]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    mn = fminf(mn, __shfl_xor_sync(FULL, mn, off));
                if (lane == 0) red[warp] = mn;
                __syncthreads();
                if (g == 0) {
                    float m = red[0];
                    for (int w = 1; w < kWarps; w++) m = fminf(m, red[w]);
                    if (check_bsf) {
                        if (kb != ~0u) ub = upper32(__uint_as_float(kb), job.dtw_hi, job.abs32);
                        kb = bsf_dist_bits(job.bsf, q);
                    }
                    stop = lower32(m, job.dtw_lo, job.abs32) > ub;
                }
                __syncthreads();
                const bool st = stop != 0;
                __syncthreads();
                if (st) { abandoned = true; break; }
            }
        }
#undef NNDTW_ROWSC_STEP
        // s is now the number of steps done
#pragma unroll
        for (int c = 0; c < C; c++)
            if (g == last_g && c == last_c) result = D[c];
        __syncthreads();
        const float res = result;
        if (g == 0) {
            if (job.counters) {
                long long cells = (long long)L * L;
                if (abandoned) {   // half-block h of lane x has finished rows 0 .. s-1 - (K x + h)
                    cells = 0;
                    for (int x = 0; x < kLanes; x++) {
                        for (int h = 0; h < K; h++) {
                            const int lo = x * C + (h ? C0 : 0);
                            const int hi = x * C + (h ? C : C0);
                            const int cols = min(max(L - lo, 0), hi - lo);
                            const int rows = min(s - 1 - (K * x + h), L - 1) + 1;
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
        __syncthreads();
    }
}

// C = 17 .. 32 columns per lane: L in (2048, 4096] over 4 warps, (4096, 8192]
// over 8 warps
constexpr int kCMin = 17, kCMax = 32;
// (one-dataset form only: series this long are rare in a batch, whose
// planner then launches them on their own)
template <int C, int NW> Dtw32Fn1 rowsc_fn() {
    return &dtw32_rowsc_kernel<C, NW, Src1<DtwJob32>>;
}
template <int NW, int... Cs> Dtw32Fn1 pick_rowsc(int c, std::integer_sequence<int, Cs...>) {
    Dtw32Fn1 fns[] = {rowsc_fn<Cs + kCMin, NW>()...};
    return (c >= kCMin && c <= kCMax) ? fns[c - kCMin] : nullptr;
}

int rowsc_warps(int L) { return L > 32 * 4 * kCMax ? 8 : 4; }

}  // namespace

bool dtw32_rowsc_ok(int L, int W) { return W >= L - 1 && L > 32 * 64 && L <= 32 * 8 * kCMax; }

cudaError_t plan_dtw32_rowsc(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    if (!dtw32_rowsc_ok(job.L, job.W)) return cudaErrorNotSupported;
    const int NW = rowsc_warps(job.L), kLanes = 32 * NW;
    const int C = (job.L + kLanes - 1) / kLanes;
    using Seq = std::make_integer_sequence<int, kCMax - kCMin + 1>;
    p->fn1 = NW == 8 ? pick_rowsc<8>(C, Seq{}) : pick_rowsc<4>(C, Seq{});
    p->fnN = nullptr;
    if (!p->fn1) return cudaErrorNotSupported;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->fn1, kLanes, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        if (n < grid) grid = n > 0 ? n : 0;
    }
    p->threads = kLanes;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = kLanes;
    return cudaSuccess;
}

}  // namespace nndtw
