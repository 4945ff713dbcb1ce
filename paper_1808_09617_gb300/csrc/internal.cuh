// Internal declarations shared by the CUDA translation units of libnndtw.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/nndtw.h"

namespace nndtw {

// Sentinels placed outside a series: a query is padded with +PAD and a
// training series with -PAD, so every band cell that falls outside the
// L x L matrix gets delta = (2 PAD)^2 = +inf and never wins a minimum.
template <typename T> struct Pad;
template <> struct Pad<float> { static constexpr float v = 1e30f; };
template <> struct Pad<double> { static constexpr double v = 1e200; };

template <typename T> __host__ __device__ inline T inf_of();
template <> __host__ __device__ inline float inf_of<float>() { return __builtin_huge_valf(); }
template <> __host__ __device__ inline double inf_of<double>() { return __builtin_huge_val(); }

// Ordered key of a (non-negative FP32 distance, index) pair: comparing keys
// as unsigned 64-bit integers compares distances first, then indices, which
// gives the lowest-index tie rule under atomicMin.
__device__ __forceinline__ uint64_t pack_key(float d, uint32_t idx) {
    return (static_cast<uint64_t>(__float_as_uint(d)) << 32) | idx;
}
__device__ __forceinline__ float key_dist(uint64_t k) {
    return __uint_as_float(static_cast<uint32_t>(k >> 32));
}
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return static_cast<uint32_t>(k); }

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ unsigned long long dbits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x));
}

// Rounding margins (Higham, Accuracy and Stability of Numerical Algorithms,
// Lemma 3.1: gamma_n = n u / (1 - n u)).  A floating-point value x_hat of a
// bound or of DTW evaluated with at most n roundings along any chain
// satisfies |x_hat - x| <= gamma_n |x| (all terms are non-negative).
//  lo : multiply a computed value to get a number <= the exact one;
//  hi : multiply a computed value to get a number >= the exact one;
//  abs: absolute slack for terms that underflow to subnormals.
struct Margins {
    float lb_lo, dtw_lo, dtw_hi, abs32;
    double lb_lo64, abs64;
};

Margins make_margins(int L);

// Conservative images of a computed FP32 value x under the margins.
__device__ __forceinline__ float lower32(float x, float lo, float abs_s) {
    return __fsub_rd(__fmul_rd(x, lo), abs_s);
}
__device__ __forceinline__ float upper32(float x, float hi, float abs_s) {
    return __fadd_ru(__fmul_ru(x, hi), abs_s);
}

// Device-side counters (all 64-bit), zeroed at the start of a search.
enum Counter : int {
    C_QUEUE = 0,     // survivors appended by compaction
    C_HEAD,          // next queue entry to claim
    C_CAND,          // completed candidates appended
    C_RECHECK,       // FP64 re-evaluations queued
    C_STARTED,       // DTWs started
    C_ABANDONED,     // DTWs abandoned
    C_CELLS,         // band cells swept
    C_RQUERIES,      // queries with a recheck
    C_SEEDHEAD,      // next seed pair to claim
    C_BAD,           // non-finite input elements found
    C_REVPRUNED,     // pairs dropped by the reverse bound LB_Enhanced(B, A)
    C_QUEUE2,        // survivors of the cascade's second stage (FP32 search)
    C_IMPPRUNED,     // pairs dropped by LB_Enhanced with the LB_Improved bridge
    C_SEEDPAIRS,     // first-candidate pairs listed (unequal-length search)
    C_BADLEN,        // series lengths out of range (unequal-length search)
    C_LIVEPRUNED,    // queued pairs dropped unstarted by their bound against the live best
    C_COUNT
};

// Candidate (a DTW that ran to completion within the margin of the best).
struct Cand {
    int32_t q, t;
    float d;
    int32_t pad;
};
struct Cand64 {
    int32_t q, t;
    double d;
};

// ---- the work of one kernel launch -----------------------------------------
// Every kernel takes its arguments as a job structure, from one of two
// sources: Src1 (one dataset for the whole grid: the single-dataset entry
// points) or SrcN (a batch: CTAs [off[d], off[d+1]) work on dataset d with
// jobs[d], so that one launch serves every dataset of a batch).  A kernel
// reads its job and its CTA index / count within that job once, at the
// start, through get(); the table lives in the launch's parameters
// (__grid_constant__, at most 32 KB), so no device memory holds it.
constexpr int kMaxSets = 64;

template <typename Job> struct Src1 {
    Job job;
    __device__ __forceinline__ const Job &get(int &bid, int &nblk) const {
        bid = (int)blockIdx.x;
        nblk = (int)gridDim.x;
        return job;
    }
};

template <typename Job> struct SrcN {
    int n;
    int off[kMaxSets + 1];
    Job jobs[kMaxSets];
    __device__ __forceinline__ const Job &get(int &bid, int &nblk) const {
        const int b = (int)blockIdx.x;
        int lo = 0, hi = n - 1;   // the last d with off[d] <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        bid = b - off[lo];
        nblk = off[lo + 1] - off[lo];
        return jobs[lo];
    }
};

// Host side: appends dataset jobs with their CTA counts to a SrcN.
template <typename Job> struct SrcNBuilder {
    SrcN<Job> src;
    SrcNBuilder() { src.n = 0; src.off[0] = 0; }
    bool full() const { return src.n == kMaxSets; }
    int blocks() const { return src.off[src.n]; }
    // the caller checks full() first
    void add(const Job &j, int nblocks) {
        if (nblocks <= 0 || src.n >= kMaxSets) return;
        src.jobs[src.n] = j;
        src.off[src.n + 1] = src.off[src.n] + nblocks;
        src.n++;
    }
};

// ---- launchers implemented in the .cu files --------------------------------
template <typename T>
cudaError_t launch_envelopes(const T *train, int64_t N, int L, int W, T *env, cudaStream_t s);
// Second envelopes from envelopes env ([N][L] (U, Lo)): env2[t][i] =
// (max of Lo, min of U) over the window of i, the training side of the
// LB_Improved bridge's second pass.
template <typename T>
cudaError_t launch_second_envelopes(const T *env, int64_t N, int L, int W, T *env2,
                                    cudaStream_t s);

// Envelope work of one set of series (the series themselves, or with env_in
// their envelopes for the second envelopes), its launch shape, and the
// kernel in its two forms (kEnvelopeThreads threads per CTA).
constexpr int kEnvelopeThreads = 256;
template <typename T> struct EnvJob {
    const T *train, *env_in;
    int64_t N;
    int L, W, T_tile, levels;
    T *env;
    // unequal lengths (nullptr: every series has L points): series s is
    // train[off[s] .. off[s+1]), L is the longest length, and its envelope
    // rows i < min(L_s + W, E) are written at env + 2 E s
    const long long *off;
    int E;
};
template <typename T> struct EnvPlan {
    EnvJob<T> job;
    bool one_pass;   // both channels per pass (a kernel variant)
    size_t smem;
    long long blocks;
};
template <typename T> struct EnvFns {
    void (*fn1)(Src1<EnvJob<T>>);
    void (*fnN)(SrcN<EnvJob<T>>);
};
template <typename T>
EnvPlan<T> plan_envelopes(const T *train, const T *env_in, int64_t N, int L, int W, T *env);
template <typename T> EnvFns<T> envelope_fns(bool one_pass);
template <typename T> cudaError_t set_envelope_smem(bool one_pass, size_t smem);

// With seed_keys, also the Euclidean-nearest series of every query; `norms`
// is then scratch for Q + N squared norms.  With ends_out, also the raw sum
// of the two ends and the bands of every pair ([Q][N]): the part of Eq. 7
// that LB_Enhanced(B, A) shares with LB_Enhanced(A, B).  With loo (test ==
// train, leave-one-out), pair (i, i) gets the bound +inf and is never a
// first candidate.
template <typename T>
cudaError_t launch_lb(const T *test, int64_t Q, const T *train, const T *env, int64_t N,
                      int L, int W, int V, bool keogh, bool safe, T lb_lo, T abs_slack,
                      T *lb_out, unsigned long long *seed_keys, T *norms, T *ends_out,
                      bool loo, cudaStream_t s, int64_t q_base = 0, int tile = 0);

// The bound pass (and its squared norms) of one dataset as job structures,
// for the batched search: launch_lb's arguments, its tile shape (a kernel
// variant, as is ed, the fused Euclidean seed; 0 lets the planner choose)
// and launch shape.  The kernel runs kLbThreads threads per CTA, the
// norms 256.
constexpr int kLbThreads = 256;
template <typename T> struct LbJob {
    const T *test;
    int64_t Q;
    const T *train, *env;
    int64_t N;
    int L, W, nb, keogh, safe;
    T lb_lo, abs_slack;
    T *lb_out;
    unsigned long long *seed_keys;
    const T *nq, *nt;
    T *ends_out;
    int loo, qfast, gx;
    int64_t q_base;   // global index of query 0 (leave-one-out over query chunks)
    // W = 0 in the search (FP32, no cascade): the bound is the squared
    // Euclidean distance formed from the norms and dot products, less
    // ed_gamma (sqrt|a|^2 + sqrt|b|^2)^2; no bridge or bands are computed
    int edb;
    T ed_gamma;
};
template <typename T> struct SqnormJob {
    const T *a;
    int64_t na;
    const T *b;
    int64_t nb;
    int L;
    T *out_a, *out_b;
};
template <typename T> struct LbPlan {
    LbJob<T> job;
    SqnormJob<T> sq;
    int tile;    // 1: 32 x 32, 2: 64 x 64, 3: 128 x 64 (queries x training series)
    bool ed;
    size_t smem;
    long long blocks, sq_blocks;
};
template <typename T> struct LbFns {
    void (*fn1)(Src1<LbJob<T>>);
    void (*fnN)(SrcN<LbJob<T>>);
    void (*sq1)(Src1<SqnormJob<T>>);
    void (*sqN)(SrcN<SqnormJob<T>>);
};
template <typename T>
cudaError_t plan_lb(const T *test, int64_t Q, const T *train, const T *env, int64_t N, int L,
                    int W, int V, bool keogh, bool safe, T lb_lo, T abs_slack, T *lb_out,
                    unsigned long long *seed_keys, T *norms, T *ends_out, bool loo,
                    LbPlan<T> *p, int64_t q_base = 0, int tile = 0, bool ed_bound = false);
template <typename T> LbFns<T> lb_fns(int tile, bool ed);
template <typename T> cudaError_t set_lb_smem(int tile, bool ed, size_t smem);

// LB_Enhanced^V (or with keogh, LB_Keogh) of every pair of two ragged sets
// (series k of a set is [off[k], off[k+1]) of its array), unequal lengths
// allowed: +inf where |L_A - L_B| > W (no warping path) or a length lies
// outside [2, max_len] (counted in *bad); env holds the training series'
// envelope rows with stride E (the ragged envelope kernel).  lb_out[Q][N]
// raw or (safe) scaled down by lb_lo and abs_slack; with seed_keys, each
// query's smallest (bound, index) key among its finite bounds is merged in
// with atomicMin (seed_keys must start at all ones).
struct LbVarJob {
    const float *test;
    const long long *test_off;
    int64_t Q;
    const float *train;
    const long long *train_off;
    const float *env;
    int E;
    int64_t N;
    int W, V, max_len, keogh, safe;
    float lb_lo, abs_slack;
    float *lb_out;
    unsigned long long *seed_keys, *bad;
};
cudaError_t launch_lb_var(const LbVarJob &job, cudaStream_t s);
// The pairs (q, key_idx(seed_keys[q])) of the queries with a key, appended
// to pairs (count in *count, which must start at 0).
cudaError_t launch_seed_pairs(const unsigned long long *seed_keys, int64_t Q, uint2 *pairs,
                              unsigned long long *count, int sm_count, cudaStream_t s);

// LB_New (Sec. 2.2.5) of every (query, training series) pair into out[Q][N]
// (raw, or with safe: scaled down by the rounding margin).
template <typename T>
cudaError_t launch_lb_new(const T *test, int64_t Q, const T *train, int64_t N, int L, int W,
                          bool safe, T lb_lo, T lb_abs, T *out, cudaStream_t s);

// FP32 DTW over a work list.  Pairs come from `pairs` ([count] of (q, t)) or,
// when pairs == nullptr, from seed keys (pair p = (p, key_idx(seed_keys[p]))).
struct DtwJob32 {
    const float *test, *train;
    int L, W;
    const uint2 *pairs;                 // or nullptr
    const unsigned long long *seed_keys;// used when pairs == nullptr
    const unsigned long long *count;    // device count of pairs (nullptr: n_pairs)
    long long n_pairs;                  // host count of pairs
    long long n_seed;                   // number of seed pairs (seed mode)
    unsigned long long *head;           // claim counter
    unsigned long long *bsf;            // [Q] packed (dist, idx) keys; nullptr: none
    Cand *cand;                         // completed-candidate list; nullptr: none
    unsigned long long *cand_count;
    float *out;                         // plain mode: out[p] = DTW
    unsigned long long *counters;       // stats (C_STARTED ...), may be nullptr
    float dtw_lo, dtw_hi, abs32;        // margins
    int abandon;                        // 1: abandon against bsf
    int group;                          // lanes per pair (0: library's choice; kRowsGroup: rows)
    int lanes;                          // resolved lanes per pair (set by the launcher)
    // unequal lengths (the *_var plans): series k of test / train is
    // [off[k], off[k+1]) of its array; L is then the longest length
    const long long *test_off, *train_off;
    // live pruning (explicit pairs with bsf; nullptr: none): the pairs' safe
    // bounds lb[q * lb_n + t], tested against the query's best when a pair
    // is due
    const float *lb;
    long long lb_n;
    // work items a group of the diagonal kernel claims at once with dynamic
    // claims (at most its lanes; 0 or 1: one)
    int claim;
};
// How one dataset's FP32 DTW pass is launched: the kernel in its one-dataset
// and batch forms (every FP32 DTW kernel takes a DtwJob32 source), block
// size, dynamic shared memory, CTAs for this dataset's work and the lanes per
// pair to put in the job.  Datasets of a batch whose plans name the same
// kernel share one launch.
using Dtw32Fn1 = void (*)(Src1<DtwJob32>);
using Dtw32FnN = void (*)(SrcN<DtwJob32>);
struct Dtw32Plan {
    Dtw32Fn1 fn1;
    Dtw32FnN fnN;
    int threads;
    size_t smem;
    long long blocks;
    int lanes;
};
cudaError_t plan_dtw32(const DtwJob32 &job, int sm_count, Dtw32Plan *p);
cudaError_t plan_dtw32_wide(const DtwJob32 &job, int sm_count, Dtw32Plan *p);
cudaError_t plan_dtw32_ed(const DtwJob32 &job, int sm_count, Dtw32Plan *p);   // W = 0
cudaError_t plan_dtw32_rows(const DtwJob32 &job, int sm_count, Dtw32Plan *p);
cudaError_t plan_dtw32_rowsg(const DtwJob32 &job, int G, int sm_count, Dtw32Plan *p);
cudaError_t plan_dtw32_rowsc(const DtwJob32 &job, int sm_count, Dtw32Plan *p);
// Unequal lengths (job.test_off / train_off set, explicit pairs): the
// diagonal kernel's VAR form for W <= 1023, the shared-memory band kernel
// beyond.
cudaError_t plan_dtw32_var(const DtwJob32 &job, int sm_count, Dtw32Plan *p);
// One dataset: plan and launch.
cudaError_t launch_dtw32(const DtwJob32 &job, int sm_count, cudaStream_t s);
bool dtw32_rowsg_ok(int L, int W, int G);
bool dtw32_rowsc_ok(int L, int W);   // full window, 2048 < L <= 4096: a CTA per pair
bool dtw32_rows_ok(int L, int W);   // full window and L small enough for the row kernel
constexpr int kRowsGroup = 64;      // DtwJob32::group value selecting the row kernel
// kRowsGroup + 1 / + 2: the row layout with 16 / 8 lanes per pair
bool dtw32_supported(int W);   // window W (<= L-1) fits the FP32 DTW kernel
int dtw32_wide_group(int W);   // widest lanes-per-pair choice for W (latency-bound passes)

// FP64 DTW: same job shape, exact evaluation order.  Inputs are double
// (test/train) or FP32 promoted in-kernel (test32/train32, for the recheck of
// the FP32 search).
struct DtwJob64 {
    const double *test, *train;
    const float *test32, *train32;
    int L, W;
    const uint2 *pairs;                 // or nullptr (seed mode)
    const unsigned long long *seed_keys;
    const unsigned long long *count;    // device count (nullptr: use n_pairs)
    long long n_pairs;                  // host count (pairs or seeds)
    unsigned long long *head;
    unsigned long long *bsf64;          // [Q] double bits; nullptr: none
    Cand64 *cand;
    unsigned long long *cand_count;
    double *out;                        // out[p] = DTW (nullptr: none)
    unsigned long long *counters;
    int abandon;
    // Reverse bound at the start of every pair (nullptr: none):
    // LB_Enhanced(B, A) = ends_bands[q N + t] + the LB_Keogh bridge of the
    // training series against the query's envelope envq ([Q][L] (U, Lo))
    // over [nb, L - nb), scaled down by lb_lo and lb_abs like every bound.
    const double2 *envq;
    const double *ends_bands;
    long long N;
    int nb;
    double lb_lo, lb_abs;
    // With envq: rev tests the reverse bound above; env2 (nullptr: none) the
    // bound with the LB_Improved bridge, lb[q N + t] (the pair's safe
    // LB_Enhanced(A, B)) plus the second pass of the bridge: the LB_Keogh
    // terms of the training series against [min(Lo^A, env2.y), max(U^A,
    // env2.x)] over [nb, L - nb), scaled down like every bound.
    bool rev;
    const double2 *env2;
    const double *lb;
    // unequal lengths: series offsets as in DtwJob32 (L the longest length)
    const long long *test_off, *train_off;
};
cudaError_t launch_dtw64(const DtwJob64 &job, int sm_count, cudaStream_t s);
using Dtw64Fn1 = void (*)(Src1<DtwJob64>);
using Dtw64FnN = void (*)(SrcN<DtwJob64>);
struct Dtw64Plan {
    Dtw64Fn1 fn1;
    Dtw64FnN fnN;
    int threads;
    size_t smem;
    long long blocks;
};
cudaError_t plan_dtw64(const DtwJob64 &job, int sm_count, Dtw64Plan *p);

// The cascade's second stage over a queue of pairs (FP32): with ends, the
// reverse bound LB_Enhanced(B, A); with env2 and lb, LB_Enhanced(A, B) with
// the LB_Improved bridge.  The survivors of in[0 .. *in_count) are appended
// to out (count in *out_count).
// A training element with its gaps to the second envelopes, (B_j -
// env2_j.x, env2_j.y - B_j) rounded down to half precision: the training
// side of the LB_Improved bridge in the FP32 search.
struct __align__(8) BGap {
    float b;
    __half2 g;
};
cudaError_t launch_pack_bgap(const float *train, float *env2, long long n, cudaStream_t s);
struct PackJob {
    const float *train;
    float *env2;
    long long n;   // elements (N * L)
};
struct PackFns {
    void (*fn1)(Src1<PackJob>);
    void (*fnN)(SrcN<PackJob>);
};
PackFns pack_bgap_fns();
long long pack_bgap_blocks(long long n);   // CTAs for n elements

struct CascadeJob {
    const uint2 *in;
    const unsigned long long *in_count;
    const float *train;
    const float2 *envq;    // query envelopes [Q][L] (U, Lo)
    const float *ends;     // [Q][N] ends + bands (raw), or nullptr: no reverse bound
    const BGap *bgap;      // [N][L] training elements and gaps, or nullptr: no
                           // LB_Improved bridge
    const float *lb;       // [Q][N] safe LB_Enhanced(A, B) (with bgap)
    long long N;
    int L, nb;
    const unsigned long long *bsf;
    float lb_lo, lb_abs, dtw_hi, abs32;
    uint2 *out;
    unsigned long long *out_count, *counters;
};
cudaError_t launch_cascade_filter(const CascadeJob &job, long long max_pairs, int sm_count,
                                  cudaStream_t s);
struct CascadeFns {
    void (*fn1)(Src1<CascadeJob>);
    void (*fnN)(SrcN<CascadeJob>);
};
CascadeFns cascade_filter_fns(bool rev, bool imp);          // 256 threads per CTA
long long cascade_filter_blocks(long long max_pairs, int sm_count);

// Adds the second pass of the LB_Improved bridge to every pair's LB_Enhanced
// value in lb[Q][N] (raw, or with safe: both parts scaled down and the sum
// rounded down).
template <typename T>
cudaError_t launch_improved_terms(const T *train, const T *envq, const T *env2, int64_t Q,
                                  int64_t N, int L, int nb, bool safe, T lb_lo, T lb_abs, T *lb,
                                  cudaStream_t s);

int device_sm_count();
void set_last_cuda_error(cudaError_t e);

}  // namespace nndtw
