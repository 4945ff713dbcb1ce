/*
 * nndtw.h -- C ABI of libnndtw.so: exact 1-nearest-neighbour classification
 * under Sakoe-Chiba windowed DTW, pruned by the LB_Enhanced^V lower bound of
 * Tan, Petitjean and Webb, "Elastic bands across the path: a new framework
 * and method to lower bound DTW" (arXiv 1808.09617).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Series are row-major, contiguous: a set of N series of length L is N*L
 *    elements, series t starting at element t*L.  All series of one call have
 *    the same length L (Sec. 2 assumes equal lengths), except in the *_varlen
 *    entry points, which take ragged sets (series of unequal lengths).
 *  - delta(a, b) = (a - b)^2 and every distance and bound is in squared units:
 *    the square root of Eq. 2 is never taken (it does not change the nearest
 *    neighbour).
 *  - W is the integer warping window, |i - j| <= W (Sec. 2.1).  W >= L-1 is
 *    the unconstrained DTW; larger values are treated as L-1.
 *  - V is LB_Enhanced's band count (Sec. 3.1); the number of bands used is
 *    min(floor(L/2), V), as in Algorithm 1.
 *  - Envelopes are interleaved: env[2*(t*L + i)] = U_i, env[2*(t*L + i) + 1]
 *    = Lo_i of series t (Eq. 3-4).
 *  - Pointers named d_* are DEVICE memory owned by the caller; h_* are HOST
 *    memory owned by the caller.  The library never frees or retains them.
 *  - Unless stated, calls are asynchronous on `stream` (a cudaStream_t passed
 *    as void*; NULL is the legacy default stream) and allocate nothing: any
 *    scratch memory is the caller's `d_workspace`.
 *  - Return value: NNDTW_OK (0) or a positive NNDTW_E* code; no exception or
 *    longjmp ever crosses the ABI.  Argument errors are reported before any
 *    work is enqueued.  NNDTW_ECUDA means a CUDA call failed; the CUDA error
 *    string is available from nn_dtw_last_cuda_error().
 *  - Inputs must be finite with magnitude below 1e15 (FP32 entry points) or
 *    1e150 (FP64 entry points); the kernels use +-1e30 / +-1e200 sentinels
 *    outside the series.  NNDTW_CHECK_FINITE makes the search verify this.
 *  - Limits: 2 <= L <= NNDTW_MAX_L, 1 <= N < 2^31 and 0 <= Q < 2^31 for the
 *    search (any N x Q: queries run in chunks, see NNDTW_CHUNK_PAIRS).
 */
#ifndef NNDTW_H
#define NNDTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NNDTW_API __attribute__((visibility("default")))
#else
#define NNDTW_API
#endif

#define NNDTW_MAX_L 8192
/* A search runs its queries in chunks of at most this many (query, training
 * series) pairs, one after another in the same workspace, so that the
 * workspace stays bounded (about 48 bytes per pair of a chunk) whatever Q x N
 * is; results do not depend on the chunking. */
#define NNDTW_CHUNK_PAIRS (1ll << 26)

/* status codes */
#define NNDTW_OK 0
#define NNDTW_EINVAL 1      /* null pointer, size or parameter out of range   */
#define NNDTW_ECUDA 2       /* a CUDA runtime call or kernel launch failed    */
#define NNDTW_ENOSPACE 3    /* workspace smaller than the size function says  */
#define NNDTW_EUNSUPPORTED 4/* valid request this build cannot serve          */
#define NNDTW_ENONFINITE 5  /* NNDTW_CHECK_FINITE found a non-finite input    */

/* flags */
#define NNDTW_LB_KEOGH (1u << 0)     /* lb_enhanced*: compute LB_Keogh instead       */
#define NNDTW_LB_SAFE (1u << 1)      /* lb_enhanced*: write rounding-safe bounds     */
/* lb_enhanced: compute LB_New (Sec. 2.2.5) instead; d_env is then not read
 * and may be NULL */
#define NNDTW_LB_NEW (1u << 18)
#define NNDTW_EXACT_DIST (1u << 2)   /* search: FP64 distance for every query's NN   */
#define NNDTW_NO_PRUNE (1u << 3)     /* search: run DTW on every pair (no LB prune)  */
#define NNDTW_NO_ABANDON (1u << 4)   /* search: no early abandoning inside DTW      */
#define NNDTW_CHECK_FINITE (1u << 5) /* search: reject non-finite or huge inputs     */
#define NNDTW_TIME_STAGES (1u << 6)  /* search: record stage events (see below)      */
#define NNDTW_NO_REVERSE (1u << 7)   /* search: skip the reverse bound LB_Enh(B, A)  */
#define NNDTW_REVERSE (1u << 14)     /* FP32 search: test the reverse bound LB_Enh(B, A) */
/* search: leave-one-out over a training set (test == train, Q == N >= 2):
 * query i never matches training series i (window learning, Sec. 1, 4). */
#define NNDTW_LEAVE_ONE_OUT (1u << 15)
/* search: also test, on the pairs that survive LB_Enhanced^V(A, B), that bound
 * with its LB_Keogh bridge replaced by LB_Improved (the combination Sec. 5
 * proposes; see lb_enhanced_improved).  A tuning choice: it never changes
 * results, and it saves DTW work at the price of one more pass over each
 * surviving pair's training series. */
#define NNDTW_IMPROVED (1u << 16)
/* search: prune with LB_Keogh (Sec. 2.2.3) instead of LB_Enhanced^V, the
 * baseline bound of the paper's study of V (Sec. 4.1); no cascade second
 * stage.  Results never change. */
#define NNDTW_KEOGH_BOUND (1u << 17)
/* search / dtw_windowed: lanes per pair of the FP32 DTW kernel, a tuning
 * choice that never changes results: NNDTW_DTW_GROUP(log2 G) with
 * G = 1, 2, 4, ..., 32; 0 (the default) lets the library choose.  A G that
 * cannot hold the window (more than 64 diagonals per lane) is ignored. */
#define NNDTW_DTW_GROUP(log2g) ((unsigned)((log2g) + 1) << 8)
#define NNDTW_DTW_GROUP_MASK (7u << 8)
/* search / dtw_windowed: for full windows (W >= L-1) sweep DTW by rows, one
 * pair per warp for L <= 2048 and one pair per CTA of 128 threads for L <=
 * 4096 and of 256 threads for L <= 8192
 * (the default for such windows when no NNDTW_DTW_GROUP is given); ignored
 * for other windows.  Combined with
 * NNDTW_DTW_ROWS_LANES16 (L <= 1024) or NNDTW_DTW_ROWS_LANES8 (L <= 512) a
 * pair takes 16 or 8 lanes instead (a tuning choice; results never change;
 * ignored where L is too long). */
/* search: tile shape of the bound pass (queries x training series per CTA),
 * a tuning choice that never changes results: NNDTW_LB_TILE(1) 32 x 32,
 * NNDTW_LB_TILE(2) 64 x 64, NNDTW_LB_TILE(3) 128 x 64; 0 (the default) lets
 * the library choose (64 x 64 when such tiles give every SM two CTAs). */
#define NNDTW_LB_TILE(k) ((unsigned)(k) << 19)
#define NNDTW_LB_TILE_MASK (3u << 19)
#define NNDTW_DTW_ROWS (7u << 8)
#define NNDTW_DTW_ROWS_LANES16 (1u << 12)
#define NNDTW_DTW_ROWS_LANES8 (2u << 12)
#define NNDTW_DTW_ROWS_LANES_MASK (3u << 12)

/* stage indices of nn_dtw_stage_times() */
#define NNDTW_STAGE_ENVELOPES 0 /* S1 (0 when envelopes are supplied)            */
#define NNDTW_STAGE_LB 1        /* S2 bounds of all pairs                        */
#define NNDTW_STAGE_SEED 2      /* S4 DTW of each query's first candidate        */
#define NNDTW_STAGE_COMPACT 3   /* S3 compaction of the surviving pairs          */
#define NNDTW_STAGE_DTW 4       /* S4 DTW of the survivors with early abandoning */
#define NNDTW_STAGE_RECHECK 5   /* S5 FP64 recheck of near ties                  */
#define NNDTW_STAGE_FINAL 6     /* S5 argmin, labels                             */
#define NNDTW_STAGE_TOTAL 7     /* whole call, first to last kernel              */

/* Work counters of one search, filled only when a non-NULL pointer is given;
 * doing so makes the call wait for the stream and makes the DTW kernels count
 * their work with atomics (unless NNDTW_TIME_STAGES is also set, in which case
 * dtw_started, dtw_abandoned, dtw_cells and seed_cells stay 0). */
typedef struct nndtw_stats {
    int64_t pairs;          /* Q * N query x train pairs                        */
    int64_t lb_pruned;      /* pairs whose bound exceeded the query's bound     */
    int64_t dtw_started;    /* DTW computations started (seeds included)        */
    int64_t dtw_abandoned;  /* of those, abandoned early                        */
    int64_t dtw_cells;      /* band cells (i,j) evaluated by the DTW kernels    */
    int64_t rechecked;      /* FP64 re-evaluations of near-tie candidates       */
    int64_t recheck_queries;/* queries that needed at least one                 */
    int64_t seed_cells;     /* of dtw_cells, those of the first-candidate pass  */
    int64_t lb_pruned_reverse; /* survivors dropped by the reverse bound
                                  LB_Enhanced(B, A) when their DTW was due     */
    int64_t lb_pruned_improved;/* survivors dropped by the bound with the
                                  LB_Improved bridge (NNDTW_IMPROVED) then;
                                  a pair both drop counts here only           */
    int64_t lb_pruned_live; /* survivors dropped unstarted when their DTW was
                               due: their bound exceeded the query's best by
                               then (FP32 DTW kernels with live pruning)     */
} nndtw_stats;

/*
 * Upper and lower envelopes of every training series (Sec. 2.2.3, Eq. 3-4):
 *   U_i = max B_j, Lo_i = min B_j over max(1, i-W) <= j <= min(L, i+W).
 * d_train: [N][L]; d_env: [N][L][2] written (U, Lo).  Exact (min/max only).
 * Errors: NNDTW_EINVAL for null pointers, N < 0, L < 1 or L > NNDTW_MAX_L,
 * W < 0.  N == 0 is a no-op.
 */
NNDTW_API int nn_dtw_build_envelopes(const float *d_train, int64_t N, int L, int W, float *d_env,
                           void *stream);
NNDTW_API int nn_dtw_build_envelopes_f64(const double *d_train, int64_t N, int L, int W,
                               double *d_env, void *stream);

/*
 * Second envelopes, the training-series side of the LB_Improved bridge
 * (lb_enhanced_improved): from the envelopes d_env ([N][L][2] (U, Lo), as
 * written by nn_dtw_build_envelopes with the same W),
 *   d_env2[t][i] = (max Lo_j, min U_j) over max(1, i-W) <= j <= min(L, i+W).
 * Exact (min/max only).  Errors as nn_dtw_build_envelopes.
 */
NNDTW_API int nn_dtw_build_second_envelopes(const float *d_env, int64_t N, int L, int W,
                                            float *d_env2, void *stream);
NNDTW_API int nn_dtw_build_second_envelopes_f64(const double *d_env, int64_t N, int L, int W,
                                                double *d_env2, void *stream);

/*
 * LB_Enhanced^V_W(A, B) (Sec. 3.1, Eq. 7; Algorithm 1 with D = +inf) for every
 * query A = test_q and training series B = train_t:
 *   delta(A_1,B_1) + delta(A_L,B_L)
 *   + sum_{i=2..n} [min over the left band L^W_i + min over the right band]
 *   + sum_{i=n+1..L-n} LB_Keogh term of A_i against (U_i, Lo_i),
 * with n = min(floor(L/2), V).  flags & NNDTW_LB_KEOGH computes LB_Keogh
 * (Sec. 2.2.3) instead.  flags & NNDTW_LB_NEW computes LB_New (Sec. 2.2.5)
 * instead, one of the comparison bounds of the paper's tightness study:
 *   delta(A_1,B_1) + delta(A_L,B_L)
 *   + sum_{i=2..L-1} min over max(1,i-W) <= j <= min(L,i+W) of delta(A_i,B_j),
 * O(L (2W+1)) per pair (d_env is not read and may be NULL).
 * flags & NNDTW_LB_SAFE scales each value down by the FP32 (or FP64) rounding
 * margin so that it never exceeds the exact bound; NNDTW_LB_TILE(k) picks the
 * bound pass's tile shape (a tuning choice).
 * d_test: [Q][L]; d_train: [N][L]; d_env: [N][L][2] from
 * nn_dtw_build_envelopes with the same W; d_lb_out: [Q][N], row-major.
 * Errors: NNDTW_EINVAL for null pointers, Q < 0, N < 0, L < 2 or > NNDTW_MAX_L,
 * W < 0, V < 1, or NNDTW_LB_KEOGH together with NNDTW_LB_NEW.
 */
NNDTW_API int lb_enhanced(const float *d_test, int64_t Q, const float *d_train, const float *d_env,
                int64_t N, int L, int W, int V, unsigned flags, float *d_lb_out,
                void *stream);
NNDTW_API int lb_enhanced_f64(const double *d_test, int64_t Q, const double *d_train,
                    const double *d_env, int64_t N, int L, int W, int V, unsigned flags,
                    double *d_lb_out, void *stream);

/*
 * LB_Enhanced^V_W(A, B) with its LB_Keogh bridge replaced by LB_Improved
 * (Sec. 2.2.4, Eq. 5), the combination proposed in Sec. 5: the value of
 * lb_enhanced plus the second pass of LB_Improved over the bridge,
 *   sum_{j=n+1..L-n} LB_Keogh term of B_j against the envelope of A',
 * with A' the projection of A onto B's envelope (Eq. 5) and n =
 * min(floor(L/2), V).  For |i-j| <= W, Lo_i <= B_j <= U_i, so wherever the
 * term is non-zero the window maximum of A' equals max(U^A_j, env2_j.x) and
 * its minimum min(Lo^A_j, env2_j.y): each term is computed against those,
 * with U^A, Lo^A the query's envelopes and env2 the training series'
 * second envelopes.  d_test_env: [Q][L][2] (nn_dtw_build_envelopes on the
 * test set, same W); d_env2: [N][L][2] (nn_dtw_build_second_envelopes);
 * other arguments as lb_enhanced.  flags: NNDTW_LB_SAFE (both parts scaled
 * down, the sum rounded down).  With NNDTW_LB_KEOGH both passes run over the
 * whole series, which is LB_Improved itself (Sec. 2.2.4, Eq. 5):
 *   LB_Keogh(A, B) + sum_{j=1..L} LB_Keogh term of B_j against the envelope
 *   of A' (V is then not used).
 * Errors: those of lb_enhanced, and NNDTW_EINVAL for NNDTW_LB_NEW.
 */
NNDTW_API int lb_enhanced_improved(const float *d_test, const float *d_test_env, int64_t Q,
                                   const float *d_train, const float *d_env, const float *d_env2,
                                   int64_t N, int L, int W, int V, unsigned flags,
                                   float *d_lb_out, void *stream);
NNDTW_API int lb_enhanced_improved_f64(const double *d_test, const double *d_test_env, int64_t Q,
                                       const double *d_train, const double *d_env,
                                       const double *d_env2, int64_t N, int L, int W, int V,
                                       unsigned flags, double *d_lb_out, void *stream);

/*
 * DTW_W(test_q, train_t) (Sec. 2.1, Eq. 1; D(L,L) in squared units) for P
 * explicit pairs, no pruning or abandoning.  d_pairs: [P][2] int32 (q, t);
 * d_out: [P].  The FP32 entry point computes in FP32; the FP64 one evaluates
 * every cell as (a-b)*(a-b) + min(...) with two roundings, in the same order
 * as the plain definition.
 * Errors: NNDTW_EINVAL for null pointers, P < 0, L < 1 or > NNDTW_MAX_L, W < 0.
 * Pair indices are not range-checked: they must address the given arrays.
 */
NNDTW_API int dtw_windowed(const float *d_test, const float *d_train, const int32_t *d_pairs,
                 int64_t P, int L, int W, float *d_out, void *stream);
/* dtw_windowed with flags (NNDTW_DTW_GROUP only). */
NNDTW_API int dtw_windowed_ex(const float *d_test, const float *d_train, const int32_t *d_pairs,
                              int64_t P, int L, int W, unsigned flags, float *d_out, void *stream);
NNDTW_API int dtw_windowed_f64(const double *d_test, const double *d_train, const int32_t *d_pairs,
                     int64_t P, int L, int W, double *d_out, void *stream);

/* Bytes of device workspace that nn_dtw_search (fp64 = 0) or
 * nn_dtw_search_f64 (fp64 = 1) needs for these sizes.  0 on invalid sizes. */
NNDTW_API size_t nn_dtw_workspace_size(int64_t N, int64_t Q, int L, int W, int V, int fp64);

/*
 * Exact 1-NN classification of Q test series against N labelled training
 * series under DTW_W: the lower-bound search of Sec. 4 with LB_Enhanced^V
 * (Algorithm 1) as the bound, cascaded with the reverse bound
 * LB_Enhanced^V(B, A) (the same bound with the series exchanged, over the
 * query's envelope) on the pairs that survive it: by default in the FP64
 * form, with NNDTW_REVERSE in the FP32 form (a tuning choice: it saves DTW
 * work but reads each surviving pair's training series once more);
 * NNDTW_NO_REVERSE leaves it out.  NNDTW_IMPROVED adds, in the same stage,
 * LB_Enhanced^V(A, B) with the LB_Improved bridge (lb_enhanced_improved);
 * the training series' second envelopes are then built into the workspace.
 * For every query q:
 *   d_nn_idx[q]   = argmin_t DTW_W(test_q, train_t), ties to the lowest t;
 *   d_nn_label[q] = d_train_labels[d_nn_idx[q]];
 *   d_nn_dist[q]  = that distance (squared units).
 * The index and label equal those of an exhaustive FP64 evaluation.  The FP32
 * entry point computes bounds and DTW in FP32 with rounding margins and
 * re-evaluates in FP64 the candidates whose FP32 distance is within the
 * margin of the best; d_nn_dist is FP64-exact for those queries (and for all
 * with NNDTW_EXACT_DIST), otherwise the FP32 value.  The FP64 entry point
 * computes everything in FP64 and its distances are exact.
 * In the FP32 form the DTW kernels also drop, unstarted, a queued pair whose
 * bound exceeds its query's best by the time the pair is due (the pruning
 * test against a best the earlier pairs have tightened; not with
 * NNDTW_NO_PRUNE).
 * d_env may be NULL (envelopes are then built into the workspace).
 * Q == 0 is a no-op.  d_workspace must hold nn_dtw_workspace_size() bytes
 * (NNDTW_ENOSPACE otherwise), 256-byte aligned.  stats may be NULL.
 * Errors: NNDTW_EINVAL for null pointers, N < 1, Q < 0, L < 2 or
 * > NNDTW_MAX_L, W < 0, V < 1, N or Q >= 2^31; NNDTW_ENONFINITE (with
 * NNDTW_CHECK_FINITE; the call then waits for the stream).  Searches whose
 * Q x N exceeds NNDTW_CHUNK_PAIRS run their queries in chunks; with
 * NNDTW_TIME_STAGES the stage events then span the whole search but the
 * boundaries between stages are those of the last chunk.
 */
NNDTW_API int nn_dtw_search(const float *d_train, const int32_t *d_train_labels, int64_t N,
                  const float *d_test, int64_t Q, int L, int W, int V,
                  const float *d_env, unsigned flags, int32_t *d_nn_idx,
                  int32_t *d_nn_label, double *d_nn_dist, void *d_workspace,
                  size_t workspace_bytes, nndtw_stats *stats, void *stream);
NNDTW_API int nn_dtw_search_f64(const double *d_train, const int32_t *d_train_labels, int64_t N,
                      const double *d_test, int64_t Q, int L, int W, int V,
                      const double *d_env, unsigned flags, int32_t *d_nn_idx,
                      int32_t *d_nn_label, double *d_nn_dist, void *d_workspace,
                      size_t workspace_bytes, nndtw_stats *stats, void *stream);

/*
 * nn_dtw_search without a workspace argument: the search's scratch memory is
 * a fixed array of NNDTW_NOALLOC_SCRATCH_BYTES inside the library, so the call
 * allocates nothing.  It is meant for callers that cannot allocate device
 * memory themselves: for example code running next to another framework
 * whose caching allocator owns (or has reserved) all device memory, or code
 * on a latency-critical path that must not call cudaMalloc, which can
 * synchronize the device.  The paper has no counterpart to this entry point.
 *  - Limit: sizes for which nn_dtw_workspace_size(N, Q, L, W, V, 0) exceeds
 *    NNDTW_NOALLOC_SCRATCH_BYTES (16 MiB: e.g. 500 x 500 series of length 256
 *    fit) are rejected with NNDTW_ENOSPACE before any work is enqueued.
 *  - The array is part of the library's device image: every GPU that loads
 *    the library holds those 16 MiB until the process exits.
 *  - Every call looks up the array's device address in the current
 *    device's context (cudaGetSymbolAddress); the first call in a context
 *    also loads the library's device code there, so make that first call
 *    before any stream capture.
 *  - All calls share the one array.  Each call clears what must start at
 *    zero, so an earlier call's leftovers do no harm, but calls whose GPU
 *    work overlaps (on different streams or from different host threads on
 *    the same device) race on the array and give wrong results: order them.
 *  - NNDTW_TIME_STAGES is ignored.  Otherwise inputs, outputs, results,
 *    errors and stats are those of nn_dtw_search.
 */
#define NNDTW_NOALLOC_SCRATCH_BYTES (16u << 20)
NNDTW_API int nn_dtw_search_noalloc(const float *d_train, const int32_t *d_train_labels,
                                    int64_t N, const float *d_test, int64_t Q, int L, int W,
                                    int V, const float *d_env, unsigned flags,
                                    int32_t *d_nn_idx, int32_t *d_nn_label, double *d_nn_dist,
                                    nndtw_stats *stats, void *stream);

/*
 * One dataset of a batched search: the arguments of nn_dtw_search for one
 * training set / test set pair.  Device pointers as in nn_dtw_search.
 */
typedef struct nndtw_dataset {
    const float *d_train;          /* [N][L]                                   */
    const int32_t *d_train_labels; /* [N]                                      */
    int64_t N;
    const float *d_test;           /* [Q][L]                                   */
    int64_t Q;
    int L, W, V;
    const float *d_env;            /* [N][L][2] envelopes for W, or NULL      */
    int32_t *d_nn_idx;             /* [Q] outputs                              */
    int32_t *d_nn_label;
    double *d_nn_dist;
    unsigned flags;                /* per-dataset flags, OR-ed with the call's */
} nndtw_dataset;

/*
 * Window learning by leave-one-out 1-NN on a training set (Sec. 1, Sec. 4):
 * for each candidate window h_windows[k] (host array, k < n_windows) the FP32
 * search runs with NNDTW_LEAVE_ONE_OUT (every training series against all the
 * others), all windows at once as one batch, and d_correct[k] (device) gets
 * the number of training series whose leave-one-out nearest neighbour has the
 * same label.  Accuracy = d_correct[k] / N; the paper keeps the window with
 * the highest accuracy (among equal ones this library's reading keeps the
 * smallest window; the choice is left to the caller).  flags: search flags
 * applied to every window (tuning choices, NNDTW_REVERSE, ...).  d_workspace:
 * nn_dtw_learn_window_workspace_size() bytes, 256-byte aligned.  Errors:
 * NNDTW_EINVAL for N < 2, no windows, a negative window, null pointers or
 * invalid sizes; NNDTW_ENOSPACE; NNDTW_ECUDA.  Asynchronous on `stream`.
 */
NNDTW_API size_t nn_dtw_learn_window_workspace_size(int64_t N, int L, const int32_t *h_windows,
                                                    int n_windows, int V);
NNDTW_API int nn_dtw_learn_window(const float *d_train, const int32_t *d_train_labels,
                                  int64_t N, int L, const int32_t *h_windows, int n_windows,
                                  int V, unsigned flags, int64_t *d_correct, void *d_workspace,
                                  size_t workspace_bytes, void *stream);

/* Bytes of device workspace nn_dtw_search_batched needs for these datasets
 * (host array of n descriptors).  0 if any dataset has invalid sizes. */
NNDTW_API size_t nn_dtw_batch_workspace_size(const nndtw_dataset *h_sets, int n);

/*
 * Batched search (the paper's NN-DTW search, Sec. 4, over many independent
 * datasets at once): exactly the results of n separate nn_dtw_search calls.
 * The datasets are searched together, stage by stage, all on `stream`: each
 * stage of the search (envelopes, bounds, first candidates, compaction, the
 * cascade's second stage, DTW, recheck, argmin) is one kernel launch over
 * every dataset of the batch (one per kernel variant where datasets need
 * different ones: tile shapes, DTW layouts), each dataset's CTAs working on
 * its own descriptor, which travels in the launch's parameters; datasets with
 * the most DTW work come first.  Batches of more than 64 datasets run as
 * consecutive groups of 64.  The call allocates nothing, waits for nothing
 * and can be captured in a CUDA graph.  h_sets: host array of n descriptors
 * (read during the call only); d_workspace: nn_dtw_batch_workspace_size()
 * bytes, 256-byte aligned.  flags apply to every dataset.  With
 * NNDTW_TIME_STAGES (at most 64 datasets with Q > 0) the stage events span
 * the whole batch (nn_dtw_stage_times).  Calls are independent of each
 * other: several may run at once on different streams, each with its own
 * workspace.  Errors: NNDTW_EINVAL for invalid descriptors or sizes,
 * NNDTW_ENOSPACE, NNDTW_ECUDA.
 */
NNDTW_API int nn_dtw_search_batched(const nndtw_dataset *h_sets, int n, void *d_workspace,
                                    size_t workspace_bytes, unsigned flags, void *stream);

/* Bytes of device memory nn_dtw_search_host needs (inputs, outputs and the
 * search workspace). 0 on invalid sizes. */
NNDTW_API size_t nn_dtw_host_buffer_size(int64_t N, int64_t Q, int L, int W, int V);

/*
 * nn_dtw_search on HOST buffers: copies h_train, h_train_labels and h_test to
 * the caller's device buffer, runs the FP32 search, copies the results back to
 * h_nn_idx, h_nn_label, h_nn_dist and waits for the stream before returning.
 * Pinned host memory makes the copies faster; pageable memory also works.
 * d_buffer: nn_dtw_host_buffer_size() bytes of device memory, 256-byte
 * aligned.  Same results and errors as nn_dtw_search.
 */
NNDTW_API int nn_dtw_search_host(const float *h_train, const int32_t *h_train_labels, int64_t N,
                       const float *h_test, int64_t Q, int L, int W, int V, unsigned flags,
                       int32_t *h_nn_idx, int32_t *h_nn_label, double *h_nn_dist,
                       void *d_buffer, size_t buffer_bytes, nndtw_stats *stats,
                       void *stream);

/*
 * One dataset of nn_dtw_search_batched_host: the arguments of
 * nn_dtw_search_host for one training set / test set pair (host buffers).
 */
typedef struct nndtw_host_dataset {
    const float *h_train;          /* [N][L]                                   */
    const int32_t *h_train_labels; /* [N]                                      */
    int64_t N;
    const float *h_test;           /* [Q][L]                                   */
    int64_t Q;
    int L, W, V;
    int32_t *h_nn_idx;             /* [Q] outputs                              */
    int32_t *h_nn_label;
    double *h_nn_dist;
    unsigned flags;                /* per-dataset flags, OR-ed with the call's */
} nndtw_host_dataset;

/* Bytes of device memory nn_dtw_search_batched_host needs for these
 * datasets (every dataset's inputs and outputs plus the batched search's
 * workspace).  0 if any dataset has invalid sizes. */
NNDTW_API size_t nn_dtw_batch_host_buffer_size(const nndtw_host_dataset *h_sets, int n);

/*
 * nn_dtw_search_batched on HOST buffers (the batched search of Sec. 4 over
 * many datasets, end to end): copies every dataset's training series, labels
 * and test series into the caller's device buffer (one copy per array, in
 * order on `stream`), runs nn_dtw_search_batched there, copies every
 * dataset's results back to its host arrays and waits for the stream before
 * returning.  Pinned host memory makes the copies asynchronous and faster;
 * pageable memory also works.  d_buffer: nn_dtw_batch_host_buffer_size()
 * bytes of device memory, 256-byte aligned.  Same results and errors as
 * nn_dtw_search_batched (NNDTW_TIME_STAGES is rejected).
 */
NNDTW_API int nn_dtw_search_batched_host(const nndtw_host_dataset *h_sets, int n, void *d_buffer,
                                         size_t buffer_bytes, unsigned flags, void *stream);

/*
 * Series of UNEQUAL lengths within a dataset (Sec. 2: the paper assumes equal
 * lengths for ease of exposition and states that the techniques generalise).
 * A ragged set of n series is one value array d_x and an offset table d_off
 * of n+1 int64 entries (device memory): series k is d_x[d_off[k] ..
 * d_off[k+1]), of length L_k; d_off must be non-decreasing and address d_x.
 * Every length must satisfy 2 <= L_k <= max_len <= NNDTW_MAX_L; max_len only
 * bounds the lengths (and sizes the scratch), it need not be attained.  The
 * reading of the method for A (length L_A) and B (length L_B):
 *  - DTW_W(A, B) is Eq. 1 on the L_A x L_B grid inside |i - j| <= W, ending
 *    at (L_A, L_B); when |L_A - L_B| > W no warping path fits the window and
 *    the distance is +inf.  W >= max_len - 1 is treated as max_len - 1.
 *  - B's envelope (Eq. 3-4) is taken for the rows i of A: U_i, Lo_i = max,
 *    min of B_j over max(1, i-W) <= j <= min(L_B, i+W), i <= L_B + W.
 *  - LB_Keogh sums over the rows of A.  LB_Enhanced^V uses
 *    n = min(floor(min(L_A, L_B)/2), V) bands at each corner: at the start,
 *    band i = the cells (i, j), (j, i), j <= i, inside the window; at the
 *    end, band i = the cells (L_A-i+1, L_B-j+1), (L_A-j+1, L_B-i+1), j <= i,
 *    inside the window; the LB_Keogh bridge covers rows n+1 .. L_A-n.  Both
 *    are +inf when |L_A - L_B| > W.
 *  - The search's first candidate for a query is the series with the
 *    smallest bound (the Euclidean distance needs equal lengths).  A query
 *    with no training series inside the window gets index -1, label -1 and
 *    distance +inf.
 * With all lengths equal every result equals that of the equal-length entry
 * point.  A length outside [2, max_len] makes its series match nothing (the
 * search reports it with NNDTW_CHECK_FINITE, see below).
 */

/* Envelopes of a ragged training set: d_env ([N][max_len][2], row stride
 * max_len) gets (U_i, Lo_i) of series t for its rows i < min(L_t + W,
 * max_len); other rows are not written.  Errors: NNDTW_EINVAL for null
 * pointers, N < 0, max_len outside [2, NNDTW_MAX_L], W < 0. */
NNDTW_API int nn_dtw_build_envelopes_varlen(const float *d_train, const int64_t *d_train_off,
                                            int64_t N, int max_len, int W, float *d_env,
                                            void *stream);

/* LB_Enhanced^V (or, with NNDTW_LB_KEOGH, LB_Keogh) of every query of a
 * ragged test set against every series of a ragged training set, unequal
 * lengths allowed (reading above): d_lb_out [Q][N]; NNDTW_LB_SAFE scales
 * each finite value down by the FP32 rounding margin.  d_env from
 * nn_dtw_build_envelopes_varlen with the same W and max_len.  Errors:
 * NNDTW_EINVAL for null pointers, Q < 0, N < 0, max_len outside
 * [2, NNDTW_MAX_L], W < 0, V < 1, other flags. */
NNDTW_API int lb_enhanced_varlen(const float *d_test, const int64_t *d_test_off, int64_t Q,
                                 const float *d_train, const int64_t *d_train_off,
                                 const float *d_env, int64_t N, int max_len, int W, int V,
                                 unsigned flags, float *d_lb_out, void *stream);

/* FP32 DTW_W of P explicit pairs (d_pairs [P][2] int32 (q, t)) of two ragged
 * sets, unequal lengths allowed (+inf when |L_q - L_t| > W): d_out [P].
 * Pair indices are not range-checked.  Errors: NNDTW_EINVAL for null
 * pointers, P < 0, max_len outside [1, NNDTW_MAX_L], W < 0. */
NNDTW_API int dtw_windowed_varlen(const float *d_test, const int64_t *d_test_off,
                                  const float *d_train, const int64_t *d_train_off,
                                  const int32_t *d_pairs, int64_t P, int max_len, int W,
                                  float *d_out, void *stream);

/* Bytes of device workspace nn_dtw_search_varlen needs.  0 on invalid sizes. */
NNDTW_API size_t nn_dtw_varlen_workspace_size(int64_t N, int64_t Q, int max_len, int W, int V);

/*
 * nn_dtw_search for ragged training and test sets (unequal lengths, reading
 * above): for every query q, d_nn_idx[q] = argmin_t DTW_W(test_q, train_t)
 * with ties to the lowest t, d_nn_label[q] its label and d_nn_dist[q] that
 * distance, as nn_dtw_search computes them (FP32 with rounding margins, an
 * FP64 recheck of near ties, NNDTW_EXACT_DIST); -1, -1, +inf for a query with
 * no training series inside the window.  The training envelopes are built
 * into the workspace.  Flags: NNDTW_EXACT_DIST, NNDTW_NO_PRUNE,
 * NNDTW_NO_ABANDON, NNDTW_KEOGH_BOUND, NNDTW_TIME_STAGES, NNDTW_DTW_GROUP;
 * NNDTW_CHECK_FINITE also checks every value (NNDTW_ENONFINITE) and, after
 * the search, every length (NNDTW_EINVAL if one lies outside [2, max_len]);
 * it makes the call wait for the stream.  NNDTW_REVERSE, NNDTW_IMPROVED and
 * NNDTW_LEAVE_ONE_OUT are rejected (NNDTW_EINVAL).  d_workspace:
 * nn_dtw_varlen_workspace_size() bytes, 256-byte aligned.  Queries run in
 * chunks of at most NNDTW_CHUNK_PAIRS pairs.  Q == 0 is a no-op.  Errors:
 * NNDTW_EINVAL for null pointers, N < 1, Q < 0, max_len outside
 * [2, NNDTW_MAX_L], W < 0, V < 1, N or Q >= 2^31; NNDTW_ENOSPACE;
 * NNDTW_ECUDA.
 */
NNDTW_API int nn_dtw_search_varlen(const float *d_train, const int64_t *d_train_off,
                                   const int32_t *d_train_labels, int64_t N, const float *d_test,
                                   const int64_t *d_test_off, int64_t Q, int max_len, int W,
                                   int V, unsigned flags, int32_t *d_nn_idx,
                                   int32_t *d_nn_label, double *d_nn_dist, void *d_workspace,
                                   size_t workspace_bytes, nndtw_stats *stats, void *stream);

/* Bytes of device memory nn_dtw_search_varlen_host needs for these ragged
 * sets (host offset tables of N+1 and Q+1 entries).  0 on invalid sizes or
 * null tables. */
NNDTW_API size_t nn_dtw_varlen_host_buffer_size(const int64_t *h_train_off, int64_t N,
                                                const int64_t *h_test_off, int64_t Q,
                                                int max_len, int W, int V);

/*
 * nn_dtw_search_varlen on HOST buffers: checks the offset tables on the host
 * (offsets from 0, every length in [2, max_len]; NNDTW_EINVAL otherwise,
 * before any copy), copies the values, offsets and labels to the caller's
 * device buffer, runs the search, copies the results back and waits for the
 * stream.  d_buffer: nn_dtw_varlen_host_buffer_size() bytes, 256-byte
 * aligned.  Same results and errors as nn_dtw_search_varlen.
 */
NNDTW_API int nn_dtw_search_varlen_host(const float *h_train, const int64_t *h_train_off,
                                        const int32_t *h_train_labels, int64_t N,
                                        const float *h_test, const int64_t *h_test_off, int64_t Q,
                                        int max_len, int W, int V, unsigned flags,
                                        int32_t *h_nn_idx, int32_t *h_nn_label,
                                        double *h_nn_dist, void *d_buffer, size_t buffer_bytes,
                                        nndtw_stats *stats, void *stream);

/*
 * Measurement aid, not part of the method.  A search called with
 * NNDTW_TIME_STAGES records CUDA events on its stream at every stage boundary
 * (events created once per thread and device; the call does not wait).  This
 * function waits for the last such search issued by the calling thread and
 * writes its stage times in milliseconds to h_ms[0..7] (NNDTW_STAGE_*).
 * NNDTW_EINVAL if the thread issued no timed search or h_ms is NULL.
 */
NNDTW_API int nn_dtw_stage_times(float *h_ms);

/*
 * Measurement aid, not part of the method: the FP32 CUDA-core rate of the DTW
 * cell update (one subtraction, one three-input minimum, one fused
 * multiply-add per cell, the instruction mix of the FP32 DTW kernel) with
 * independent cells and no memory traffic, over the whole GPU.  Runs `iters`
 * iterations of 16 cells per thread on every SM, waits for the stream and
 * writes the measured cells per second to *h_cells_per_s.  d_sink: device
 * memory of at least nn_dtw_probe_sink_bytes() bytes (receives the results so
 * the work is not optimised away).
 */
NNDTW_API size_t nn_dtw_probe_sink_bytes(void);
NNDTW_API int nn_dtw_probe_cell_rate(void *d_sink, size_t sink_bytes, int iters,
                                     double *h_cells_per_s, void *stream);

/* Measurement aid, not part of the method: the number of kernel launches
 * that the calling thread's last FP32 search call (nn_dtw_search,
 * nn_dtw_search_batched or nn_dtw_search_varlen, and the calls built on
 * them) issued. */
NNDTW_API long long nn_dtw_last_call_launches(void);
/* The same launches by stage: h_counts[k] (k < 7, NNDTW_STAGE_*) counts those
 * issued between stage boundaries k and k+1 (the start of the search counts
 * as stage 0, the cascade's second stage as compaction); h_counts[7] is 0. */
NNDTW_API int nn_dtw_last_call_stage_launches(long long *h_counts);

/* Static description of a status code.  Never NULL. */
NNDTW_API const char *nn_dtw_strerror(int code);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
NNDTW_API const char *nn_dtw_last_cuda_error(void);
/* ABI version (major * 100 + minor). */
NNDTW_API int nn_dtw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NNDTW_H */
