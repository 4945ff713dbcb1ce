// S4: windowed DTW (Sec. 2.1, Eq. 1) in FP32 with early abandoning, one
// pair per group of G lanes (G = 1, 2, ..., 32), persistent over a work list.
//
// Layout.  The band |i - j| <= W is stored by diagonals: diagonal
// k = j - i + W (0 <= k <= 2W) holds the cells (i, i + k - W).  The cells with
// the same anti-diagonal t = i + j are mutually independent, and the cell of
// diagonal k at anti-diagonal t depends only on diagonal k at t-2 and on
// diagonals k-1, k+1 at t-1.  So each diagonal keeps ONE register (its latest
// value) and the sweep alternates between even and odd diagonals: a
// "super-step" advances every diagonal by one cell.  Lane g of a group owns
// C_g consecutive diagonals (C_g = 2H, or 2H-2 for the first s lanes, with
// sum C_g = 2W + 2): one slot beyond the band (diagonal 2W+1, kept at +inf)
// and no per-cell masking.  A lane exchanges one boundary value with each
// neighbour per super-step (warp shuffles), and the series values flow
// through the group: query values A_i enter at lane 0 and move right, training
// values B_j enter at the last lane and move left, one per super-step, each
// lane keeping a window of H of each in registers.  Per cell the work is
// d = A_i - B_j; D = fma(d, d, min3(D_diag, D_left, D_up)).
//
// Cells outside the L x L matrix read sentinels: +1e30 for the query outside
// [0, L), -1e30 for the training series before its start and +1e30 after its
// end.  A cell with one index inside and one outside, or both before the
// start, gets delta = +inf and never wins a minimum; cells with both indices
// past the end get delta = 0, so they inherit exactly D(L,L) (their only
// finite entry is the diagonal step out of (L,L)) and diagonal W keeps the
// result after the sweep ends.  D(-1,-1) = 0 is seeded in the register of
// diagonal W.
//
// Unequal lengths (VAR = true; Sec. 2 generalised): the pair's series come
// from offset tables, query A of length L_A and training series B of length
// L_B, and the sentinels above start at each series' own end.  The end cell
// (L_A, L_B) lies on diagonal W + L_B - L_A; the cells after it on that
// diagonal have both indices past the ends and inherit its value, and the
// sweep ends once anti-diagonal L_A + L_B - 2 is behind it.
//
// Early abandoning: every path from (1,1) to (L,L) visits one of any two
// consecutive anti-diagonals, and D never decreases along a path, so the
// minimum of all current diagonal registers (which hold anti-diagonals t and
// t-1) is a lower bound on D(L,L).  Scaled down by the FP32 rounding margin,
// a value above the query's current upper bound abandons the pair (strict
// test, so ties are never abandoned).
#pragma once

#include "internal.cuh"

namespace nndtw {

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The (query, training series) of work item p: an explicit pair list, or
// query p with its seed candidate.  Items past the end read nothing.
__device__ __forceinline__ uint2 work_item(const DtwJob32 &job, long long p, long long n_work) {
    if (p >= n_work) return make_uint2(0u, 0u);
    if (job.pairs) return job.pairs[p];
    return make_uint2((unsigned)p, (unsigned)key_idx(job.seed_keys[p]));
}

// The distance half (float bits) of query q's best key, read past the
// caches; ~0u while the query has no candidate yet.
__device__ __forceinline__ unsigned bsf_dist_bits(const unsigned long long *bsf, int q) {
    return *(reinterpret_cast<const volatile unsigned *>(bsf + q) + 1);
}

// Number of band cells (i, j) in [0,L)^2 with |i-j| <= W and i + j <= S, in
// closed form: anti-diagonals d <= W hold d+1 cells, the middle ones W or W+1
// alternately, the last W ones 2L-1-d.
__device__ inline long long band_cells_upto(int L, int W, long long S) {
    if (S < 0) return 0;
    if (W > L - 1) W = L - 1;
    if (S > 2ll * L - 2) S = 2ll * L - 2;
    const long long a = S < W ? S : W;
    long long tot = (a + 1) * (a + 2) / 2;
    if (W >= L - 1) {
        if (S >= L) tot += (3ll * L - 2 - S) * (S - L + 1) / 2;
        return tot;
    }
    if (S > W) {
        const long long m_end = S < 2ll * L - 3 - W ? S : 2ll * L - 3 - W;
        const long long n = m_end - W;
        if (n > 0) tot += n * W + n / 2;
    }
    if (S >= 2ll * L - 2 - W) tot += (W + 2ll * L - S) * (S - (2ll * L - 2 - W) + 1) / 2;
    return tot;
}

// Band cells (i, j) of an L_A x L_B grid with |i-j| <= W and i + j <= S
// (work counters of the unequal-length form only), row by row.
__device__ inline long long band_cells_var(int LA, int LB, int W, long long S) {
    long long tot = 0;
    for (int i = 0; i < LA; i++) {
        const long long lo = i - W > 0 ? i - W : 0;
        long long hi = i + W < LB - 1 ? i + W : LB - 1;
        if (S - i < hi) hi = S - i;
        if (hi >= lo) tot += hi - lo + 1;
    }
    return tot;
}

// Resident 128-thread blocks per SM requested from the register allocator for
// each H (the diagonal registers, the two windows and the per-pair state need
// about 4H + 2U + 50 registers); chosen from a compile sweep as the largest
// count that causes no more than a few bytes of spills.
__host__ __device__ constexpr int dtw32_min_blocks(int H) {
    return H <= 4 ? 8 : H <= 9 ? 6 : H <= 11 ? 5 : H <= 15 ? 4 : H <= 23 ? 3 : 2;
}

template <int H, int U, typename Src, bool VAR = false>
__global__ void __launch_bounds__(128, dtw32_min_blocks(H))
dtw32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    const int G = job.lanes;
    constexpr int C = 2 * H;
    const float INF = __int_as_float(0x7f800000);
    const float APAD = Pad<float>::v, BPAD = -Pad<float>::v, EPAD = Pad<float>::v;
    const unsigned FULL = 0xffffffffu;
    const int L = job.L, W = job.W;

    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int s = G * H - (W + 1);               // short lanes: 0 <= s <= G-1
    const bool shortl = gl < s;
    const int k0 = gl * C - 2 * (gl < s ? gl : s);
    const int Cg = shortl ? C - 2 : C;
    const bool lastl = gl == G - 1;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const bool hasW = W >= k0 && W < k0 + Cg;
    const int cW = W - k0;
    const int t_first = -(W & 1);
    const int I0 = (W >> 1) - (k0 >> 1);        // I at the first super-step's A step
    const int J0 = t_first - I0;
    // The group's series streams: at super-step u its lane 0 takes query
    // value IA0 + u and its last lane training value JB0 + u.
    const int k0_last = (G - 1) * C - 2 * (G - 1 < s ? G - 1 : s);
    const int IA0 = (W >> 1) + 1;
    const int JB0 = t_first - ((W >> 1) - (k0_last >> 1)) + H;

    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const long long n_groups = (long long)nblk * (blockDim.x / G);
    const bool check_bsf = job.abandon && job.bsf;
    // abandon checks every 16 super-steps, at the same block for the whole warp
    constexpr int kCheckBlocks = 16 / U > 1 ? 16 / U : 1;

    // Claiming, equal lengths: claims run two pairs ahead per group so that
    // no memory latency sits between two sweeps (the whole warp would wait
    // for it): p1 is the group's next pair with its item w1 already
    // requested.  `nxt` is the next static index, or (dynamic claims) the
    // claim after p1, still in flight in the group's lane 0.  Live pruning
    // (job.lb): with p1 come its pair's safe bound and its query's best
    // (float bits), tested when the pair is due; a bound above the best's
    // upper bound at that moment drops the pair unstarted (the compaction's
    // test against a tighter best).
    long long nxt = ((long long)bid * blockDim.x + threadIdx.x) / G;
    long long p1 = 0;
    uint2 w1 = make_uint2(0u, 0u);
    float lb1 = 0.f;
    unsigned kb1 = ~0u;
    if constexpr (!VAR) {
        if (job.head) {
            unsigned long long v = 0;
            if (gl == 0) v = atomicAdd(job.head, 1ull);
            p1 = (long long)__shfl_sync(FULL, v, 0, G);
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
    }
    // Claiming, unequal lengths (VAR): batches of consecutive items, one item
    // per lane of the group, two claims ahead: nw is this lane's item of the
    // next batch (first item nb, nbs items), already requested with its
    // pair's bound and its query's best, and bnxt the claim after it (nxs
    // items), in flight in the group's lane 0.  When a batch is due, each
    // lane applies the live test to its item and the group starts the
    // batch's surviving pairs one after another (bits of bmask), so that a
    // batch dropped whole waits once for the next batch's loads, not once
    // per pair: the bound-nearest first candidate of the unequal-length
    // search leaves most of its queue to be dropped live.  Dynamic claims
    // take min(G, job.claim) items at a time, static assignment one.  (With
    // equal lengths, where few queued pairs are dropped, batches of a
    // query's consecutive pairs swept by one group were measured slower.)
    const long long gidx = ((long long)bid * blockDim.x + threadIdx.x) / G;
    const unsigned gbits = G == 32 ? FULL : ((1u << G) - 1u);
    const int bs = job.head && job.claim > 1 ? (G < job.claim ? G : job.claim) : 1;
    int nbs = 1, nxs = 1;
    long long nb = 0, cbase = 0, bnxt = 0;
    uint2 nw = make_uint2(0u, 0u), bw = make_uint2(0u, 0u);
    float nlb = 0.f;
    unsigned nkb = ~0u, bmask = 0u;
    auto claim = [&](bool first) {
        if (job.head) {
            nb = (long long)__shfl_sync(gmask, bnxt, 0, G);
            nbs = nxs;
            if (gl == 0) bnxt = (long long)atomicAdd(job.head, (unsigned long long)bs);
            nxs = bs;
        } else {
            nb = first ? gidx : nb + n_groups;
            nbs = 1;
        }
        const bool mine = gl < nbs && nb + gl < n_work;
        nw = mine ? work_item(job, nb + gl, n_work) : make_uint2(0u, 0u);
        nlb = 0.f;
        nkb = ~0u;
        if (job.lb && mine) {
            nlb = job.lb[(long long)nw.x * job.lb_n + nw.y];
            nkb = bsf_dist_bits(job.bsf, (int)nw.x);
        }
    };
    if constexpr (VAR) {
        if (job.head && gl == 0) bnxt = (long long)atomicAdd(job.head, (unsigned long long)bs);
        nxs = bs;
        claim(true);
    }

    float R[C], Aw[H + U], Bw[H + U];
    // per-pair state
    long long pid = -1;
    int q = 0, tt = 0;
    int ws = 0;                     // warp step at which the pair started
    bool done = true, finished = false;
    float ub = INF;
    unsigned kb = ~0u;              // query best (float bits) read at one check, used at the next
    const float *ap = job.test, *bp = job.train;
    // lengths, the super-steps of a full sweep and the end cell's register
    // (the equal-length values unless VAR)
    int LA = L, LB = L, ue = L, cE = cW;
    bool hasE = hasW;
    // Stream values come in chunks of G, one per lane of the group: for warp
    // steps cG .. cG+G-1, lane k of the group holds the values of warp step
    // cG + k (the current chunk in ca/cb, the next one in na_/nb_).
    float ca = 0.f, cb = 0.f, na_ = 0.f, nb_ = 0.f;
    int wblk = 0;                   // warp step at the start of this block

    while (true) {
        // ---- start new pairs at a block boundary ---------------------------
        // (branches on group-uniform state; shuffles use the group's mask)
        const bool need = done && !finished;
        if (__any_sync(FULL, need)) {
            if (need) {
                bool take = false;
                if constexpr (!VAR) {
                    // claim until a pair survives the live test or the list ends
                    while (!take && p1 < n_work) {
                        pid = p1;
                        q = (int)w1.x; tt = (int)w1.y;
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
                } else {
                    // the current batch's next surviving pair; batches are taken
                    // in (and the next one claimed) until one has a survivor or
                    // the list ends
                    while (bmask == 0u && nb < n_work) {
                        cbase = nb;
                        bw = nw;
                        const bool valid = gl < nbs && nb + gl < n_work;
                        const bool keep = valid && (nkb == ~0u ||
                            !(nlb > upper32(__uint_as_float(nkb), job.dtw_hi, job.abs32)));
                        const int sh = lane & ~(G - 1);
                        bmask = (__ballot_sync(gmask, keep) >> sh) & gbits;
                        const unsigned vm = (__ballot_sync(gmask, valid) >> sh) & gbits;
                        if (job.counters && gl == 0 && vm != bmask)
                            atomicAdd(job.counters + C_LIVEPRUNED,
                                      (unsigned long long)__popc(vm & ~bmask));
                        claim(false);
                    }
                    take = bmask != 0u;
                    if (take) {
                        const int k = __ffs(bmask) - 1;
                        bmask &= bmask - 1u;
                        pid = cbase + k;
                        q = (int)__shfl_sync(gmask, bw.x, k, G);
                        tt = (int)__shfl_sync(gmask, bw.y, k, G);
                    }
                }
                if (!take) {
                    finished = true;
                    pid = -1;
                } else {
                    if constexpr (VAR) {
                        const long long a0 = job.test_off[q], b0 = job.train_off[tt];
                        ap = job.test + a0;
                        bp = job.train + b0;
                        LA = (int)(job.test_off[q + 1] - a0);
                        LB = (int)(job.train_off[tt + 1] - b0);
                        ue = (LA + LB + (W & 1)) >> 1;
                        const int kE = W + LB - LA;
                        hasE = kE >= k0 && kE < k0 + Cg;
                        cE = kE - k0;
                    } else {
                        ap = job.test + (long long)q * L;
                        bp = job.train + (long long)tt * L;
                    }
                    done = false;
                    ws = wblk;
                    ub = INF;
                    kb = ~0u;
                    if (check_bsf) kb = bsf_dist_bits(job.bsf, q);
                    // windows for the first super-step (v = 0 mappings)
#pragma unroll
                    for (int m = 0; m < H; m++) {
                        const int ia = I0 - m;
                        Aw[m + U - 1] = (ia >= 0 && ia < LA) ? ap[ia] : APAD;
                        const int jb = J0 + m;
                        Bw[m] = jb < 0 ? BPAD : (jb < LB ? bp[jb] : EPAD);
                    }
#pragma unroll
                    for (int c = 0; c < C; c++) R[c] = (hasW && c == cW) ? 0.f : INF;
                    {   // the stream chunks holding warp steps wblk and on
                        const int u0 = (wblk & ~(G - 1)) + gl - wblk;
                        const int ia = IA0 + u0, jb = JB0 + u0;
                        ca = (ia >= 0 && ia < LA) ? ap[ia] : APAD;
                        cb = jb < 0 ? BPAD : (jb < LB ? bp[jb] : EPAD);
                        const int ia2 = ia + G, jb2 = jb + G;
                        na_ = (ia2 >= 0 && ia2 < LA) ? ap[ia2] : APAD;
                        nb_ = jb2 < 0 ? BPAD : (jb2 < LB ? bp[jb2] : EPAD);
                    }
                    if (job.counters && gl == 0) atomicAdd(job.counters + C_STARTED, 1ull);
                }
            }
        }
        if (__all_sync(FULL, finished)) break;

        // ---- one block of U super-steps ------------------------------------
#pragma unroll
        for (int v = 0; v < U; v++) {
            const int w = wblk + v;
            const int src = w & (G - 1);
            const float acur = __shfl_sync(FULL, ca, src, G);
            const float bcur = __shfl_sync(FULL, cb, src, G);
            if (src == G - 1) {
                // next chunk in, and the one after it requested
                ca = na_;
                cb = nb_;
                const int u2 = w + 1 + G + gl - ws;
                const int ia = IA0 + u2, jb = JB0 + u2;
                na_ = (ia >= 0 && ia < LA) ? ap[ia] : APAD;
                nb_ = jb < 0 ? BPAD : (jb < LB ? bp[jb] : EPAD);
            }
            // step A: even slots
            {
                float send;
                if constexpr (H >= 2) send = shortl ? R[C - 3] : R[C - 1];
                else send = R[C - 1];
                float left = __shfl_up_sync(FULL, send, 1, G);
                if (gl == 0) left = INF;
#pragma unroll
                for (int m = 0; m < H; m++) {
                    const int c = 2 * m;
                    const float a = Aw[m + U - 1 - v];
                    const float b = Bw[m + v];
                    const float lft = (m == 0) ? left : R[c - 1];
                    const float d = a - b;
                    R[c] = fmaf(d, d, min3f(R[c], lft, R[c + 1]));
                }
            }
            // b-shift
            {
                const float sendb = Bw[v];
                float nb = __shfl_down_sync(FULL, sendb, 1, G);
                if (lastl) nb = bcur;
                Bw[H + v] = nb;
                if constexpr (H >= 2) {
                    if (shortl) Bw[H - 1 + v] = nb;
                }
            }
            // step B: odd slots
            {
                float right = __shfl_down_sync(FULL, R[0], 1, G);
                if (lastl) right = INF;
#pragma unroll
                for (int m = 0; m < H; m++) {
                    const int c = 2 * m + 1;
                    const float a = Aw[m + U - 1 - v];
                    const float b = Bw[m + v + 1];
                    float rgt;
                    if (c == C - 1) rgt = right;
                    else if (c == C - 3) rgt = shortl ? right : R[c + 1];
                    else rgt = R[c + 1];
                    const float d = a - b;
                    R[c] = fmaf(d, d, min3f(R[c], R[c - 1], rgt));
                }
                if (lastl) R[C - 1] = INF;
            }
            // a-shift
            {
                float senda;
                if constexpr (H >= 2) senda = shortl ? Aw[H - 2 + U - 1 - v] : Aw[H - 1 + U - 1 - v];
                else senda = Aw[H - 1 + U - 1 - v];
                float na = __shfl_up_sync(FULL, senda, 1, G);
                if (gl == 0) na = acur;
                if (v + 1 < U) {
                    Aw[U - 2 - v] = na;
                } else {
#pragma unroll
                    for (int m = H - 1; m >= 1; m--) Aw[m + U - 1] = Aw[m - 1];
                    Aw[U - 1] = na;
                }
            }
        }
        // realign the b window
#pragma unroll
        for (int m = 0; m < H; m++) Bw[m] = Bw[m + U];
        wblk += U;
        const int u = wblk - ws;     // super-steps of the current pair so far

        // ---- completion / abandon ------------------------------------------
        const bool completed = !done && u >= ue;
        if (completed) {
            // the result: diagonal W (W + L_B - L_A) holds D(L,L) (D(L_A,L_B)),
            // kept by the past-the-end cells
            float r = INF;
#pragma unroll
            for (int c = 0; c < C; c++) r = (hasE && c == cE) ? R[c] : r;
            for (int off = 1; off < G; off <<= 1) r = fminf(r, __shfl_xor_sync(gmask, r, off, G));
            if (gl == 0) {
                if (job.out) job.out[pid] = r;
                if (job.bsf) {
                    const unsigned long long key = pack_key(r, (uint32_t)tt);
                    const unsigned long long old = atomicMin(job.bsf + q, key);
                    const unsigned long long cur = old < key ? old : key;
                    const float ubn = upper32(key_dist(cur), job.dtw_hi, job.abs32);
                    if (job.cand && lower32(r, job.dtw_lo, job.abs32) <= ubn) {
                        const unsigned long long slot = atomicAdd(job.cand_count, 1ull);
                        Cand cd;
                        cd.q = q; cd.t = tt; cd.d = r; cd.pad = 0;
                        job.cand[slot] = cd;
                    }
                }
                if (job.counters)
                    atomicAdd(job.counters + C_CELLS,
                              (unsigned long long)(VAR ? band_cells_var(LA, LB, W, 2ll * L)
                                                       : band_cells_upto(L, W, 2ll * L)));
            }
            done = true;
        }
        if (job.abandon && ((wblk / U) % kCheckBlocks) == 0) {
            // The whole warp reduces; each running group decides with selects
            // rather than branches (branches here cost register copies in
            // the sweep).  The bound uses the query best read at the last
            // check and requests the next one.
            float mn = R[0];
#pragma unroll
            for (int c = 1; c < C; c++) mn = fminf(mn, R[c]);
            for (int off = 1; off < G; off <<= 1)
                mn = fminf(mn, __shfl_xor_sync(FULL, mn, off, G));
            const unsigned kbn = check_bsf ? bsf_dist_bits(job.bsf, q) : ~0u;
            const float ubn = kb != ~0u ? upper32(__uint_as_float(kb), job.dtw_hi, job.abs32) : ub;
            ub = done ? ub : ubn;
            kb = done ? kb : kbn;
            const bool drop = !done && lower32(mn, job.dtw_lo, job.abs32) > ub;
            if (drop && gl == 0 && job.counters) {
                atomicAdd(job.counters + C_ABANDONED, 1ull);
                atomicAdd(job.counters + C_CELLS,
                          (unsigned long long)(VAR ? band_cells_var(LA, LB, W, 2ll * u + t_first - 1)
                                                   : band_cells_upto(L, W, 2ll * u + t_first - 1)));
            }
            done = done || drop;
        }
    }
}

}  // namespace nndtw
