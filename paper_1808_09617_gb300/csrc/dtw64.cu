// FP64 windowed DTW (Sec. 2.1, Eq. 1), one pair per CTA.
//
// Used for the near-tie recheck of the FP32 search and for the all-FP64
// search.  Every cell is evaluated exactly as the plain definition writes it,
// d = A_i - B_j; t = d * d; D = t + min(D(i-1,j-1), D(i,j-1), D(i-1,j)), with
// one rounding per operation (__dsub_rn / __dmul_rn / __dadd_rn forbid
// contraction) and the minimum exact, so the value is bit-identical to a
// sequential FP64 evaluation of the recurrence.  The minimum is taken on the
// bit patterns as 64-bit integers (D is never negative, and +inf orders
// last), which keeps it off GB300's narrow FP64 pipe.
//
// Both series are staged in shared memory as FP64 while they fit next to the
// band (FP32 inputs of the recheck converted once, exactly); beyond that the
// recheck stages its FP32 inputs as FP32 and converts them in every cell,
// and FP64 series are read from global memory, where L2 holds them.  The
// band is kept by diagonals
// k = j - i + W in shared memory, one slot per diagonal plus two +inf
// sentinels.  Anti-diagonal t updates the diagonals of its parity that hold a
// cell inside the L x L matrix, spread over the CTA's threads, reading only
// diagonals of the other parity; one barrier per anti-diagonal orders the
// sweep.  Slots of diagonals not yet reached keep their initial +inf, and
// D(-1,-1) = 0 is seeded in the slot of diagonal W.
//
// Early abandoning (FP64 search): the minimum over all slots is at most the
// minimum over anti-diagonals t-1 and t, which every path crosses, so it is a
// lower bound of D(L,L); it is compared (strictly) with the query's exact
// current best.  Before a pair's sweep, the reverse bound LB_Enhanced(B, A)
// (the pair's stored ends and bands plus the LB_Keogh bridge of the training
// series against the query's envelope, scaled down by the bound's rounding
// margin) is compared with the same best, and the pair is dropped when it is
// larger.
//
// With offset tables (unequal lengths, Sec. 2 generalised) series k of the
// test / training set is [off[k], off[k+1]) of its array, the pair's grid is
// L_A x L_B, and its end cell lies on diagonal W + L_B - L_A; L is then the
// longest length (the staging size).
#include <type_traits>

#include "internal.cuh"

namespace nndtw {
namespace {

constexpr size_t kDtw64SmemCap = 227 * 1024;

__device__ __forceinline__ long long lmin(long long a, long long b) { return a < b ? a : b; }

template <bool F32IN, bool F32STAGE, bool STAGED, typename Src>
__global__ void __launch_bounds__(256)
dtw64_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob64 &job = src.get(bid, nblk);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = job.L, W = job.W;
    const int nslot = 2 * W + 3;
    using ST = typename std::conditional<F32STAGE, float, double>::type;   // staged type
    using IT = typename std::conditional<F32IN, float, double>::type;      // input type
    long long *Rs = reinterpret_cast<long long *>(smem_raw);  // Rs[k+1]: double bits
    ST *As = reinterpret_cast<ST *>(Rs + nslot);
    ST *Bs = As + L;
    __shared__ long long red[32];
    __shared__ long long claim;
    __shared__ int bcast;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long INFB = 0x7ff0000000000000ll;
    const long long n_work = job.count ? (long long)*job.count : job.n_pairs;
    long long next_static = bid;

    while (true) {
        long long p;
        if (job.head) {
            if (tid == 0) claim = (long long)atomicAdd(job.head, 1ull);
            __syncthreads();
            p = claim;
            __syncthreads();
        } else {
            p = next_static;
            next_static += nblk;
        }
        if (p >= n_work) break;
        int q, t;
        if (job.pairs) {
            const uint2 pr = job.pairs[p];
            q = (int)pr.x; t = (int)pr.y;
        } else {
            q = (int)p; t = (int)key_idx(job.seed_keys[p]);
        }
        if (!F32IN && job.envq) {
            // the cascade's second stage: the reverse bound (job.rev) and the
            // bound with the LB_Improved bridge (job.env2), over [nb, L - nb)
            const double2 *eq = job.envq + (long long)q * L;
            const double2 *e2 = job.env2 ? job.env2 + (long long)t * L : nullptr;
            const double *bp = job.train + (long long)t * L;
            double pr = 0.0, pi = 0.0;
            for (int j = job.nb + tid; j < L - job.nb; j += nthr) {
                const double b = bp[j];
                const double2 e = eq[j];
                const double d = b - fmin(fmax(b, e.y), e.x);
                pr = fma(d, d, pr);
                if (e2) {
                    const double2 o = e2[j];
                    const double di = b - fmin(fmax(b, fmin(e.y, o.y)), fmax(e.x, o.x));
                    pi = fma(di, di, pi);
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                pr += __shfl_xor_sync(0xffffffffu, pr, off);
                pi += __shfl_xor_sync(0xffffffffu, pi, off);
            }
            if ((tid & 31) == 0) {
                red[tid >> 5] = __double_as_longlong(pr);
                red[16 + (tid >> 5)] = __double_as_longlong(pi);
            }
            __syncthreads();
            if (tid == 0) {
                const long long pq = (long long)q * job.N + t;
                const long long ubits = (long long)*((volatile unsigned long long *)job.bsf64 + q);
                bool by_imp = false, by_rev = false;
                if (e2) {
                    double tot = 0.0;
                    for (int w = 0; w < (nthr >> 5); w++) tot += __longlong_as_double(red[16 + w]);
                    double si = __dsub_rd(__dmul_rd(tot, job.lb_lo), job.lb_abs);
                    si = si > 0.0 ? si : 0.0;
                    by_imp = __double_as_longlong(__dadd_rd(job.lb[pq], si)) > ubits;   // strict
                }
                if (job.rev && !by_imp) {
                    double tot = job.ends_bands[pq];
                    for (int w = 0; w < (nthr >> 5); w++) tot += __longlong_as_double(red[w]);
                    double safe = __dsub_rd(__dmul_rd(tot, job.lb_lo), job.lb_abs);
                    safe = safe > 0.0 ? safe : 0.0;
                    by_rev = __double_as_longlong(safe) > ubits;   // strict
                }
                bcast = by_imp || by_rev;
                if (job.counters && by_imp) atomicAdd(job.counters + C_IMPPRUNED, 1ull);
                if (job.counters && by_rev) atomicAdd(job.counters + C_REVPRUNED, 1ull);
            }
            __syncthreads();
            const bool drop = bcast != 0;
            __syncthreads();
            if (drop) continue;
        }
        const IT *Ag, *Bg;
        const IT *tst = F32IN ? reinterpret_cast<const IT *>(job.test32)
                              : reinterpret_cast<const IT *>(job.test);
        const IT *trn = F32IN ? reinterpret_cast<const IT *>(job.train32)
                              : reinterpret_cast<const IT *>(job.train);
        int LA = L, LB = L;
        if (job.test_off) {
            const long long a0 = job.test_off[q], b0 = job.train_off[t];
            Ag = tst + a0;
            Bg = trn + b0;
            LA = (int)(job.test_off[q + 1] - a0);
            LB = (int)(job.train_off[t + 1] - b0);
        } else {
            Ag = tst + (long long)q * L;
            Bg = trn + (long long)t * L;
        }
        // (a ragged length that does not fit the staging: no value)
        if (LA < 1 || LB < 1 || LA > L || LB > L) continue;
        // staged copies (shared-memory loads in the sweep), or (FP64 inputs
        // only) the series in global memory
        if (STAGED) {
            for (int i = tid; i < LA; i += nthr) As[i] = (ST)Ag[i];
            for (int i = tid; i < LB; i += nthr) Bs[i] = (ST)Bg[i];
        }
        const ST *Ap = STAGED ? As : reinterpret_cast<const ST *>(Ag);
        const ST *Bp = STAGED ? Bs : reinterpret_cast<const ST *>(Bg);
        for (int k = tid; k < nslot; k += nthr) Rs[k] = INFB;
        __syncthreads();
        if (tid == 0) {
            Rs[W + 1] = 0;   // bits of +0.0
            if (job.counters) atomicAdd(job.counters + C_STARTED, 1ull);
        }
        __syncthreads();

        bool abandoned = false;
        long long cells = 0;
        for (int s = 0; s <= LA + LB - 2; s++) {
            if (job.abandon && job.bsf64 && (s & 15) == 15) {
                long long mn = INFB;
                for (int k = tid; k < nslot; k += nthr) mn = lmin(mn, Rs[k]);
                for (int off = 16; off > 0; off >>= 1)
                    mn = lmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
                if ((tid & 31) == 0) red[tid >> 5] = mn;
                __syncthreads();
                if (tid < 32) {
                    long long v = tid < (nthr >> 5) ? red[tid] : INFB;
                    for (int off = 16; off > 0; off >>= 1)
                        v = lmin(v, __shfl_xor_sync(0xffffffffu, v, off));
                    if (tid == 0) {
                        const long long ub = (long long)*((volatile unsigned long long *)job.bsf64 + q);
                        bcast = v > ub;   // exact: larger bits = larger value
                    }
                }
                __syncthreads();
                const bool stop = bcast != 0;
                __syncthreads();
                if (stop) { abandoned = true; break; }
            }
            // cells (i, j) = ((s + W - k) / 2, s - i) inside [0, L_A) x [0, L_B)
            int klo = W - s;
            if (klo < s + W - 2 * LA + 2) klo = s + W - 2 * LA + 2;
            if (klo < 0) klo = 0;
            int khi = s + W;
            if (khi > 2 * LB - 2 - s + W) khi = 2 * LB - 2 - s + W;
            if (khi > 2 * W) khi = 2 * W;
            if (((s + W - klo) & 1) != 0) klo++;
            for (int k = klo + 2 * tid; k <= khi; k += 2 * nthr) {
                const int i = (s + W - k) >> 1, j = s - i;
                const long long m = lmin(lmin(Rs[k + 1], Rs[k]), Rs[k + 2]);
                const double d = __dsub_rn((double)Ap[i], (double)Bp[j]);
                const double tt = __dmul_rn(d, d);
                Rs[k + 1] = __double_as_longlong(__dadd_rn(tt, __longlong_as_double(m)));
            }
            if (job.counters && khi >= klo) cells += (khi - klo) / 2 + 1;
            __syncthreads();
        }
        if (tid == 0) {
            if (job.counters) {
                atomicAdd(job.counters + C_CELLS, (unsigned long long)cells);
                if (abandoned) atomicAdd(job.counters + C_ABANDONED, 1ull);
            }
            if (!abandoned) {
                const int kE = W + LB - LA;   // outside [0, 2W]: no warping path
                const double D = (kE >= 0 && kE <= 2 * W) ? __longlong_as_double(Rs[kE + 1])
                                                          : __longlong_as_double(INFB);
                if (job.out) job.out[p] = D;
                if (job.bsf64) {
                    const unsigned long long old = atomicMin(job.bsf64 + q, dbits(D));
                    if (job.cand && dbits(D) <= old) {
                        const unsigned long long slot = atomicAdd(job.cand_count, 1ull);
                        Cand64 c;
                        c.q = q; c.t = t; c.d = D;
                        job.cand[slot] = c;
                    }
                }
            }
        }
        __syncthreads();
    }
}


template <bool F32IN, bool F32STAGE, bool STAGED>
cudaError_t plan_dtw64_as(const DtwJob64 &job, size_t smem, int sm_count, Dtw64Plan *p) {
    p->fn1 = dtw64_kernel<F32IN, F32STAGE, STAGED, Src1<DtwJob64>>;
    p->fnN = dtw64_kernel<F32IN, F32STAGE, STAGED, SrcN<DtwJob64>>;
    // threads: enough for the widest anti-diagonal (W+1 cells), 32..256
    int threads = ((job.W / 2 + 1) + 31) / 32 * 32;
    if (threads > 256) threads = 256;
    if (threads < 32) threads = 32;
    cudaError_t e = cudaFuncSetAttribute(p->fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(p->fnN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->fn1, threads, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const long long cap = (long long)sm_count * bps;
    long long grid = job.count ? cap : (job.n_pairs < cap ? job.n_pairs : cap);
    p->threads = threads;
    p->smem = smem;
    p->blocks = grid > 0 ? grid : 0;
    return cudaSuccess;
}

}  // namespace

cudaError_t plan_dtw64(const DtwJob64 &job, int sm_count, Dtw64Plan *p) {
    const size_t band = sizeof(long long) * (size_t)(2 * job.W + 3);
    const size_t as_f64 = sizeof(double) * 2 * (size_t)job.L;
    const size_t as_f32 = sizeof(float) * 2 * (size_t)job.L;
    if (band + as_f64 <= kDtw64SmemCap)
        return job.test32 ? plan_dtw64_as<true, false, true>(job, band + as_f64, sm_count, p)
                          : plan_dtw64_as<false, false, true>(job, band + as_f64, sm_count, p);
    if (job.test32) {
        if (band + as_f32 > kDtw64SmemCap) return cudaErrorInvalidValue;
        return plan_dtw64_as<true, true, true>(job, band + as_f32, sm_count, p);
    }
    return plan_dtw64_as<false, false, false>(job, band, sm_count, p);
}

cudaError_t launch_dtw64(const DtwJob64 &job, int sm_count, cudaStream_t s) {
    if (!job.count && job.n_pairs <= 0) return cudaSuccess;
    Dtw64Plan p{};
    cudaError_t e = plan_dtw64(job, sm_count, &p);
    if (e != cudaSuccess) return e;
    if (p.blocks <= 0) return cudaSuccess;
    p.fn1<<<(unsigned)p.blocks, p.threads, p.smem, s>>>(Src1<DtwJob64>{job});
    return cudaGetLastError();
}

}  // namespace nndtw
