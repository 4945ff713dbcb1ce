// FP32 DTW at W = 0: DTW_0 is the squared Euclidean distance (Sec. 2.1; the
// only warping path is the diagonal), so a pair needs no recurrence.  One
// warp per pair: each lane accumulates the squared differences of the
// elements lane, lane + 32, ... with fused multiply-adds, and a butterfly adds
// the 32 partial sums.  A value takes at most 2 L / 32 + 7 roundings along
// any chain, fewer than the 2 L + 8 the DTW margins allow, so the search's
// rounding-safe bounds and the FP64 recheck of near ties apply unchanged.
// Same work list, best-so-far keys and candidate list as the other FP32 DTW
// kernels; pairs are never abandoned (a W = 0 pair costs L / 32 steps).
#include "dtw32.cuh"

namespace nndtw {
namespace {

template <typename Src>
__global__ void __launch_bounds__(128) dtw32_ed_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    const unsigned FULL = 0xffffffffu;
    const int L = job.L;
    const int lane = threadIdx.x & 31;
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const long long n_warps = ((long long)nblk * blockDim.x) >> 5;
    long long next_static = ((long long)bid * blockDim.x + threadIdx.x) >> 5;
    while (true) {
        long long p;
        if (job.head) {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(job.head, 1ull);
            p = (long long)__shfl_sync(FULL, v, 0);
        } else {
            p = next_static;
            next_static += n_warps;
        }
        if (p >= n_work) break;
        const uint2 w = work_item(job, p, n_work);
        const int q = (int)w.x, t = (int)w.y;
        const float *ap = job.test + (long long)q * L;
        const float *bp = job.train + (long long)t * L;
        float acc = 0.f;
        for (int i = lane; i < L; i += 32) {
            const float d = ap[i] - bp[i];
            acc = fmaf(d, d, acc);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
        if (lane == 0) {
            if (job.counters) {
                atomicAdd(job.counters + C_STARTED, 1ull);
                atomicAdd(job.counters + C_CELLS, (unsigned long long)L);
            }
            if (job.out) job.out[p] = acc;
            if (job.bsf) {
                const unsigned long long key = pack_key(acc, (uint32_t)t);
                const unsigned long long old = atomicMin(job.bsf + q, key);
                const unsigned long long cur = old < key ? old : key;
                const float ubn = upper32(key_dist(cur), job.dtw_hi, job.abs32);
                if (job.cand && lower32(acc, job.dtw_lo, job.abs32) <= ubn) {
                    const unsigned long long slot = atomicAdd(job.cand_count, 1ull);
                    Cand cd;
                    cd.q = q; cd.t = t; cd.d = acc; cd.pad = 0;
                    job.cand[slot] = cd;
                }
            }
        }
    }
}

}  // namespace

cudaError_t plan_dtw32_ed(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    p->fn1 = &dtw32_ed_kernel<Src1<DtwJob32>>;
    p->fnN = &dtw32_ed_kernel<SrcN<DtwJob32>>;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->fn1, 128, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        const long long need = n > 0 ? (n + 3) / 4 : 0;   // four warps per CTA
        if (need < grid) grid = need;
    }
    p->threads = 128;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = 32;
    return cudaSuccess;
}

}  // namespace nndtw
