// FP64 windowed DTW (Sec. 2.1, Eq. 1), one pair per warp.
//
// Used for the near-tie recheck of the FP32 search and for the all-FP64
// search.  Every cell is evaluated exactly as the plain definition writes it,
// d = A_i - B_j; t = d * d; D = t + min(D(i-1,j-1), D(i,j-1), D(i-1,j)), with
// one rounding per operation (__dsub_rn / __dmul_rn / __dadd_rn forbid
// contraction) and min exact, so the value is bit-identical to a sequential
// FP64 evaluation of the recurrence.
//
// The band is kept by diagonals k = j - i + W in shared memory, one slot per
// diagonal plus two +inf sentinels; each anti-diagonal t updates the diagonals
// of its parity that hold a cell inside the L x L matrix, reading only
// diagonals of the other parity, so one __syncwarp per anti-diagonal orders
// the sweep.  Slots of diagonals not yet reached keep their initial +inf;
// D(-1,-1) = 0 is seeded in the slot of diagonal W.
//
// Early abandoning (FP64 search): the minimum over all slots is at most the
// minimum over anti-diagonals t-1 and t, which every path crosses, so it is a
// lower bound of D(L,L); it is compared (strictly) with the query's exact
// current best.  GB300's FP64 pipe bounds this kernel; its layout is chosen
// for simplicity, not speed.
#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kWarps64 = 4;

__device__ __forceinline__ double dmin_exact(double a, double b) { return a < b ? a : b; }

template <bool F32IN>
__global__ void __launch_bounds__(32 * kWarps64)
dtw64_kernel(DtwJob64 job, int warps_per_block) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= warps_per_block) return;
    const int L = job.L, W = job.W;
    const int nslot = 2 * W + 3;
    double *Rs = reinterpret_cast<double *>(smem_raw) + (size_t)warp * nslot;  // Rs[k+1]
    const double INF = inf_of<double>();
    const long long n_work = job.count ? (long long)*job.count : job.n_pairs;

    const long long n_warps = (long long)gridDim.x * warps_per_block;
    long long next_static = (long long)blockIdx.x * warps_per_block + warp;

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
        const double *a64 = F32IN ? nullptr : job.test + (long long)q * L;
        const double *b64 = F32IN ? nullptr : job.train + (long long)t * L;
        const float *a32 = F32IN ? job.test32 + (long long)q * L : nullptr;
        const float *b32 = F32IN ? job.train32 + (long long)t * L : nullptr;
        for (int k = lane; k < nslot; k += 32) Rs[k] = INF;
        __syncwarp();
        if (lane == 0) Rs[W + 1] = 0.0;
        __syncwarp();
        if (lane == 0 && job.counters) atomicAdd(job.counters + C_STARTED, 1ull);

        double ub = INF;
        bool abandoned = false;
        long long cells = 0;
        for (int s = 0; s <= 2 * L - 2; s++) {
            if (job.abandon && job.bsf64 && (s & 15) == 15) {
                double mn = INF;
                for (int k = lane; k < nslot; k += 32) mn = dmin_exact(mn, Rs[k]);
                for (int off = 16; off > 0; off >>= 1)
                    mn = dmin_exact(mn, __shfl_xor_sync(0xffffffffu, mn, off));
                ub = __longlong_as_double(
                    (long long)*((volatile unsigned long long *)job.bsf64 + q));
                if (mn > ub) { abandoned = true; break; }
            }
            int klo = W - s;
            if (klo < s + W - 2 * L + 2) klo = s + W - 2 * L + 2;
            if (klo < 0) klo = 0;
            int khi = s + W;
            if (khi > 2 * L - 2 - s + W) khi = 2 * L - 2 - s + W;
            if (khi > 2 * W) khi = 2 * W;
            if (((s + W - klo) & 1) != 0) klo++;
            for (int k = klo + 2 * lane; k <= khi; k += 64) {
                const int i = (s + W - k) >> 1, j = s - i;
                const double a = F32IN ? (double)a32[i] : a64[i];
                const double b = F32IN ? (double)b32[j] : b64[j];
                const double m = dmin_exact(dmin_exact(Rs[k + 1], Rs[k]), Rs[k + 2]);
                const double d = __dsub_rn(a, b);
                const double tt = __dmul_rn(d, d);
                Rs[k + 1] = __dadd_rn(tt, m);
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
                const double D = Rs[W + 1];
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
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_dtw64(const DtwJob64 &job, int sm_count, cudaStream_t s) {
    if (!job.count && job.n_pairs <= 0) return cudaSuccess;
    const size_t per_warp = sizeof(double) * (size_t)(2 * job.W + 3);
    int wpb = (int)((200u * 1024u) / per_warp);
    if (wpb > kWarps64) wpb = kWarps64;
    if (wpb < 1) return cudaErrorInvalidValue;
    const size_t smem = per_warp * wpb;
    const bool f32 = job.test32 != nullptr;
    cudaError_t e;
    if (f32)
        e = cudaFuncSetAttribute(dtw64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    else
        e = cudaFuncSetAttribute(dtw64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e != cudaSuccess) return e;
    long long want = job.count ? (long long)sm_count * 16 : (job.n_pairs + wpb - 1) / wpb;
    long long cap = (long long)sm_count * 16;
    long long grid = want < cap ? want : cap;
    if (grid < 1) grid = 1;
    if (f32)
        dtw64_kernel<true><<<(unsigned)grid, 32 * kWarps64, smem, s>>>(job, wpb);
    else
        dtw64_kernel<false><<<(unsigned)grid, 32 * kWarps64, smem, s>>>(job, wpb);
    return cudaGetLastError();
}

}  // namespace nndtw
