// FP32 windowed DTW (Sec. 2.1, Eq. 1) for windows too wide for the register
// kernel (W >= 1024, up to L-1 <= 4095): one pair per warp, the band kept by
// diagonals k = j - i + W in shared memory (one slot per diagonal plus two
// +inf sentinels).  Anti-diagonal t updates the diagonals of its parity that
// hold a cell inside the L x L matrix, reading only diagonals of the other
// parity, so one __syncwarp per anti-diagonal orders the sweep; slots of
// diagonals not yet reached keep their initial +inf and D(-1,-1) = 0 is seeded
// in the slot of diagonal W.  Same work list, margins, packed best-so-far
// keys, candidate list and early abandoning as the register kernel (the
// minimum over all slots is at most the minimum over anti-diagonals t-1 and
// t, which every path crosses).  With offset tables (unequal lengths) the
// pair's grid is L_A x L_B and its end cell lies on diagonal W + L_B - L_A.
#include "dtw32.cuh"

namespace nndtw {
namespace {

constexpr int kWideWarps = 4;

template <typename Src>
__global__ void __launch_bounds__(32 * kWideWarps)
dtw32_wide_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const DtwJob32 &job = src.get(bid, nblk);
    const int warps_per_block = job.lanes;   // this kernel's launch shape: warps per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= warps_per_block) return;
    const int L = job.L, W = job.W;
    const int nslot = 2 * W + 3;
    float *Rs = reinterpret_cast<float *>(smem_raw) + (size_t)warp * nslot;  // Rs[k+1]
    const float INF = inf_of<float>();
    const long long n_work = job.pairs ? (job.count ? (long long)*job.count : job.n_pairs)
                                       : job.n_seed;
    const long long n_warps = (long long)nblk * warps_per_block;
    long long next_static = (long long)bid * warps_per_block + warp;

    while (true) {
        unsigned long long p = 0;
        if (job.head) {
            if (lane == 0) p = atomicAdd(job.head, 1ull);
            p = __shfl_sync(0xffffffffu, p, 0);
        } else {
            p = (unsigned long long)next_static;
            next_static += n_warps;
        }
        if ((long long)p >= n_work) break;
        int q, t;
        if (job.pairs) {
            const uint2 pr = job.pairs[p];
            q = (int)pr.x; t = (int)pr.y;
        } else {
            q = (int)p; t = (int)key_idx(job.seed_keys[p]);
        }
        const float *a, *b;
        int LA = L, LB = L;
        if (job.test_off) {
            const long long a0 = job.test_off[q], b0 = job.train_off[t];
            a = job.test + a0;
            b = job.train + b0;
            LA = (int)(job.test_off[q + 1] - a0);
            LB = (int)(job.train_off[t + 1] - b0);
        } else {
            a = job.test + (long long)q * L;
            b = job.train + (long long)t * L;
        }
        for (int k = lane; k < nslot; k += 32) Rs[k] = INF;
        __syncwarp();
        if (lane == 0) Rs[W + 1] = 0.f;
        __syncwarp();
        if (lane == 0 && job.counters) atomicAdd(job.counters + C_STARTED, 1ull);

        bool abandoned = false;
        long long cells = 0;
        for (int s = 0; s <= LA + LB - 2; s++) {
            if (job.abandon && job.bsf && (s & 15) == 15) {
                float mn = INF;
                for (int k = lane; k < nslot; k += 32) mn = fminf(mn, Rs[k]);
                for (int off = 16; off > 0; off >>= 1)
                    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
                const unsigned long long kb = *((volatile unsigned long long *)job.bsf + q);
                const float ub = kb == ~0ull ? INF : upper32(key_dist(kb), job.dtw_hi, job.abs32);
                if (lower32(mn, job.dtw_lo, job.abs32) > ub) { abandoned = true; break; }
            }
            // cells (i, j) = ((s + W - k) / 2, s - i) inside [0, L_A) x [0, L_B)
            int klo = W - s;
            if (klo < s + W - 2 * LA + 2) klo = s + W - 2 * LA + 2;
            if (klo < 0) klo = 0;
            int khi = s + W;
            if (khi > 2 * LB - 2 - s + W) khi = 2 * LB - 2 - s + W;
            if (khi > 2 * W) khi = 2 * W;
            if (((s + W - klo) & 1) != 0) klo++;
            for (int k = klo + 2 * lane; k <= khi; k += 64) {
                const int i = (s + W - k) >> 1, j = s - i;
                const float d = a[i] - b[j];
                Rs[k + 1] = fmaf(d, d, min3f(Rs[k + 1], Rs[k], Rs[k + 2]));
            }
            if (job.counters && khi >= klo) cells += (khi - klo) / 2 + 1;
            __syncwarp();
        }
        if (lane == 0) {
            if (job.counters) {
                atomicAdd(job.counters + C_CELLS, (unsigned long long)cells);
                if (abandoned) atomicAdd(job.counters + C_ABANDONED, 1ull);
            }
            if (!abandoned) {
                // (|L_A - L_B| > W: no warping path inside the window)
                const int kE = W + LB - LA;
                const float res = (kE >= 0 && kE <= 2 * W) ? Rs[kE + 1] : INF;
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
        __syncwarp();
    }
}

}  // namespace

cudaError_t plan_dtw32_wide(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    const long long n = job.pairs ? job.n_pairs : job.n_seed;
    const size_t per_warp = sizeof(float) * (size_t)(2 * job.W + 3);
    int wpb = (int)((200u * 1024u) / per_warp);
    if (wpb > kWideWarps) wpb = kWideWarps;
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp * wpb;
    p->fn1 = &dtw32_wide_kernel<Src1<DtwJob32>>;
    p->fnN = &dtw32_wide_kernel<SrcN<DtwJob32>>;
    cudaError_t e = cudaFuncSetAttribute(p->fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(p->fnN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long cap = (long long)sm_count * 16;
    long long grid = (job.pairs && job.count) ? cap : (n > 0 ? (n + wpb - 1) / wpb : 0);
    if (grid > cap) grid = cap;
    p->threads = 32 * kWideWarps;
    p->smem = smem;
    p->blocks = grid;
    p->lanes = wpb;
    return cudaSuccess;
}

}  // namespace nndtw
