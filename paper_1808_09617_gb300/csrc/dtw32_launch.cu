// Launcher of the FP32 DTW kernel: picks the group width G and per-lane
// diagonal-pair count H for a window W and sizes the persistent grid.
#include <mutex>

#include "dtw32_inst.cuh"

namespace nndtw {

namespace {

bool pick_fn(int H, Dtw32Fn1 *f1, Dtw32FnN *fn) {
    switch (H) {
#define C_(h) case h: *f1 = dtw32_fn<h>(); *fn = dtw32_fn_n<h>(); return true;
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13)
        C_(14) C_(15) C_(16) C_(17) C_(18) C_(19) C_(20) C_(21) C_(22) C_(23) C_(24) C_(25)
        C_(26) C_(27) C_(28) C_(29) C_(30) C_(31) C_(32)
#undef C_
        default: return false;
    }
}

bool pick_var_fn(int H, Dtw32Fn1 *f1) {
    switch (H) {
#define C_(h) case h: *f1 = dtw32_var_fn<h>(); return true;
        C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(9) C_(10) C_(11) C_(12) C_(13)
        C_(14) C_(15) C_(16) C_(17) C_(18) C_(19) C_(20) C_(21) C_(22) C_(23) C_(24) C_(25)
        C_(26) C_(27) C_(28) C_(29) C_(30) C_(31) C_(32)
#undef C_
        default: return false;
    }
}

struct OccCache {
    std::mutex mu;
    int blocks[2][33][64] = {};  // [form][H][device]
};
OccCache g_occ;

// The persistent grid of the diagonal kernel f (form 0: equal lengths, 1:
// unequal) with G lanes per pair: its resident CTAs on every SM, or fewer
// for a short work list known on the host.
cudaError_t diag_grid(const DtwJob32 &job, int form, int H, int G, Dtw32Fn1 f, int sm_count,
                      long long *grid_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int bps = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ.mu);
        if (dev < 64) bps = g_occ.blocks[form][H][dev];
        if (bps == 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, f, 128, 0);
            if (e != cudaSuccess) return e;
            if (bps < 1) bps = 1;
            if (dev < 64) g_occ.blocks[form][H][dev] = bps;
        }
    }
    long long grid = (long long)sm_count * bps;
    if (!job.pairs || !job.count) {
        const long long n = job.pairs ? job.n_pairs : job.n_seed;
        const long long groups_per_block = 128 / G;
        const long long need = n > 0 ? (n + groups_per_block - 1) / groups_per_block : 0;
        if (need < grid) grid = need;
    }
    *grid_out = grid;
    return cudaSuccess;
}

}  // namespace

// G lanes per pair and H diagonal pairs per lane with G*H >= W+1 and at most
// G-1 short lanes (H = ceil((W+1)/G)).  A lane needs at least one live pair,
// so H = 1 is allowed only without short lanes.
static bool shape_ok(int W, int g, int *H) {
    const int h = (W + 1 + g - 1) / g;
    if (h > 32) return false;
    if (h == 1 && g * h != W + 1) return false;
    *H = h;
    return true;
}

// Default: the smallest G whose lanes hold the window (fewest shuffles per
// cell); `want` (if valid) overrides it.
bool dtw32_shape(int W, int want, int *G, int *H) {
    if (want >= 1 && want <= 32 && (want & (want - 1)) == 0 && shape_ok(W, want, H)) {
        *G = want;
        return true;
    }
    for (int g = 1; g <= 32; g <<= 1)
        if (shape_ok(W, g, H)) { *G = g; return true; }
    return false;
}

int dtw32_wide_group(int W) {
    int H;
    // (callers check dtw32_rows_ok first: full windows go to the row kernel)
    for (int g = 32; g >= 1; g >>= 1)
        if (shape_ok(W, g, &H)) return g;
    return 0;
}

// Windows up to 1023 use the register kernel; wider ones (up to L-1 with
// L <= NNDTW_MAX_L) the shared-memory band kernel.
bool dtw32_supported(int W) { return W >= 0 && W < NNDTW_MAX_L; }

cudaError_t plan_dtw32(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    // W = 0: the squared Euclidean distance, whatever layout is asked for
    if (job.W == 0) return plan_dtw32_ed(job, sm_count, p);
    // full windows: the row kernels, unless a diagonal group width is asked for
    if (job.group == kRowsGroup + 1 && dtw32_rowsg_ok(job.L, job.W, 16))
        return plan_dtw32_rowsg(job, 16, sm_count, p);
    if (job.group == kRowsGroup + 2 && dtw32_rowsg_ok(job.L, job.W, 8))
        return plan_dtw32_rowsg(job, 8, sm_count, p);
    if ((job.group == 0 || job.group >= kRowsGroup) && dtw32_rows_ok(job.L, job.W))
        return plan_dtw32_rows(job, sm_count, p);
    if ((job.group == 0 || job.group >= kRowsGroup) && dtw32_rowsc_ok(job.L, job.W))
        return plan_dtw32_rowsc(job, sm_count, p);
    int G = 0, H = 0;
    if (!dtw32_shape(job.W, job.group, &G, &H)) return plan_dtw32_wide(job, sm_count, p);
    if (!pick_fn(H, &p->fn1, &p->fnN)) return cudaErrorNotSupported;
    long long grid = 0;
    const cudaError_t e = diag_grid(job, 0, H, G, p->fn1, sm_count, &grid);
    if (e != cudaSuccess) return e;
    p->threads = 128;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = G;
    return cudaSuccess;
}

cudaError_t plan_dtw32_var(const DtwJob32 &job, int sm_count, Dtw32Plan *p) {
    if (!job.pairs || !job.test_off || !job.train_off) return cudaErrorInvalidValue;
    int G = 0, H = 0;
    if (!dtw32_shape(job.W, job.group, &G, &H)) return plan_dtw32_wide(job, sm_count, p);
    if (!pick_var_fn(H, &p->fn1)) return cudaErrorNotSupported;
    p->fnN = nullptr;
    long long grid = 0;
    const cudaError_t e = diag_grid(job, 1, H, G, p->fn1, sm_count, &grid);
    if (e != cudaSuccess) return e;
    p->threads = 128;
    p->smem = 0;
    p->blocks = grid;
    p->lanes = G;
    return cudaSuccess;
}

cudaError_t launch_dtw32(const DtwJob32 &job_in, int sm_count, cudaStream_t s) {
    Dtw32Plan p{};
    cudaError_t e = plan_dtw32(job_in, sm_count, &p);
    if (e != cudaSuccess) return e;
    if (p.blocks <= 0) return cudaSuccess;
    DtwJob32 job = job_in;
    job.lanes = p.lanes;
    p.fn1<<<(unsigned)p.blocks, p.threads, p.smem, s>>>(Src1<DtwJob32>{job});
    return cudaGetLastError();
}

}  // namespace nndtw
