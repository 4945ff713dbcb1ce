// Host orchestration of the NN-DTW search and the C ABI of libnndtw.so.
//
// FP32 search (nn_dtw_search), all on the caller's stream:
//   S1  envelopes of the training set (unless supplied)
//   S2  LB_Enhanced^V for all Q x N pairs, scaled down by the rounding margin,
//       and per query its Euclidean-nearest training series (the first
//       candidate, the paper's starting point of the search, Sec. 4)
//   S4  DTW of that candidate per query, which sets each query's upper bound
//   S3  compaction: pairs whose bound does not exceed the upper bound
//   S4  DTW of the survivors with early abandoning against the live bound;
//       every completed DTW within the margin of the best is recorded
//   S5  candidates within the margin of the final best are re-evaluated in
//       FP64 when a query has two or more; argmin with ties to the lowest
//       index; labels gathered.
// The FP64 search is the same pipeline in FP64, where DTW values are exact
// and no recheck is needed.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace nndtw {

namespace {
thread_local char g_cuda_err[256] = "";
std::mutex g_sm_mu;
int g_sm[64] = {};

constexpr int kSmallThreads = 256;

// ------------------------------------------------------------------ kernels

template <typename T>
__global__ void finite_check_kernel(const T *__restrict__ x, int64_t n, T limit,
                                    unsigned long long *bad) {
    unsigned long long cnt = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T v = x[i];
        if (!(v < limit && v > -limit)) cnt++;
    }
    if (cnt) atomicAdd(bad, cnt);
}

// S3: keep (q, t) iff its safe bound does not exceed the query's upper bound,
// and order the kept pairs by the ratio bound / upper bound (kBuckets buckets,
// counting sort in two passes).  Pairs with a small ratio tend to run their
// DTW to completion, pairs near 1 to be abandoned early, so this order runs
// the long pairs first and leaves short ones for the end of the persistent
// DTW kernel (longest-processing-time-first scheduling), and the pairs most
// likely to lower their query's best come first.  The queue then holds bucket
// 0, bucket 1, ...; within a bucket the order is arbitrary.  64 buckets
// instead of 8 made the batched step 2.9 % faster (its DTW stage 4 %: the
// full-window datasets, whose bounds are weak, find their nearest series
// sooner); 32 gave 2.6 %.
constexpr int kBuckets = 64;

template <typename T> struct UbOf;
template <> struct UbOf<float> {
    float hi, abs_s;
    __device__ float operator()(unsigned long long kb) const {
        return kb == ~0ull ? inf_of<float>() : upper32(key_dist(kb), hi, abs_s);
    }
};
template <> struct UbOf<double> {
    __device__ double operator()(unsigned long long kb) const {
        return __longlong_as_double((long long)kb);
    }
};

// Bucket of a kept pair: kBuckets equal slices of bound / upper bound
// (inv = kBuckets / ub, computed once per query; only the order of the
// queue depends on it).
template <typename T>
__device__ __forceinline__ int bucket_of(T lb, T inv) {
    const int b = (int)(lb * inv);
    return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

// pass 1 (scatter == 0): count the kept pairs of every bucket;
// pass 2 (scatter == 1): write them at bucket offset + position.
// Both passes aggregate per block in shared memory: one global atomic per
// bucket per block-iteration (pass 2) or per block (pass 1).
constexpr int kCompactE = 8;   // pairs per thread per compaction round

template <typename T> struct CompactJob {
    const T *lb;
    int64_t Q, N;
    const unsigned long long *bsf, *seed;
    UbOf<T> ubof;
    int no_prune, gx;   // gx: CTAs along a row; the others stride over the rows
    int finite_only;    // also drop pairs whose bound is +inf (no warping path)
    int scatter;        // 0: count the kept pairs per bucket; 1: write them
    unsigned long long *bcount, *bcursor, *qcount;
    uint2 *queue;
};

template <typename T, typename Src>
__global__ void __launch_bounds__(256)
compact_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const CompactJob<T> &job = src.get(bid, nblk);
    const int scatter = job.scatter;
    const T *__restrict__ lb = job.lb;
    const int64_t Q = job.Q, N = job.N;
    const unsigned long long *__restrict__ bsf = job.bsf;
    const unsigned long long *__restrict__ seed = job.seed;
    const UbOf<T> ubof = job.ubof;
    const int no_prune = job.no_prune, finite_only = job.finite_only;
    unsigned long long *__restrict__ bcount = job.bcount;
    unsigned long long *__restrict__ bcursor = job.bcursor;
    uint2 *__restrict__ queue = job.queue;
    unsigned long long *__restrict__ qcount = job.qcount;
    const int bx = bid % job.gx, by = bid / job.gx, gy = nblk / job.gx;
    __shared__ unsigned long long boff[kBuckets];
    __shared__ unsigned int scount[kBuckets];
    __shared__ unsigned long long sbase[kBuckets];
    __shared__ unsigned long long wsum[kBuckets / 32];
    const int tid = threadIdx.x;
    static_assert(kBuckets % 32 == 0 && kBuckets <= kSmallThreads, "buckets: whole warps");
    if (tid < kBuckets) scount[tid] = 0;
    if (scatter && tid < kBuckets) {
        // bucket offsets: an exclusive prefix sum of the counts, one bucket
        // per thread (inclusive scan per warp, then the warps' totals)
        const unsigned long long c = bcount[tid];
        unsigned long long v = c;
        const int ln = tid & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
            if (ln >= o) v += u;
        }
        if (ln == 31) wsum[tid >> 5] = v;
        boff[tid] = v - c;
    }
    __syncthreads();
    if (scatter && tid < kBuckets) {
        unsigned long long o = 0;
        for (int w = 0; w < (tid >> 5); w++) o += wsum[w];
        boff[tid] += o;
        if (tid == kBuckets - 1 && bid == 0) *qcount = boff[tid] + bcount[tid];
    }
    __syncthreads();
    // each round covers kCompactE * 256 consecutive pairs of a row; element e
    // of thread tid is t0 + e * 256 + tid (coalesced loads)
    constexpr int E = kCompactE;
    for (int64_t q = by; q < Q; q += gy) {
        const T ub = ubof(bsf[q]);
        const T inv = ub > T(0) && ub < inf_of<T>() ? T(kBuckets) / ub : T(0);
        const uint32_t st = key_idx(seed[q]);
        const T *row = lb + q * N;
        for (int64_t t0 = (int64_t)bx * blockDim.x * E; t0 < N;
             t0 += (int64_t)job.gx * blockDim.x * E) {
            unsigned keepm = 0;
            unsigned pos[E];
            int bk[E];
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int64_t t = t0 + (int64_t)e * blockDim.x + tid;
                bool keep = false;
                bk[e] = 0;
                pos[e] = 0;
                if (t < N) {
                    const T v = row[t];
                    // (a leave-one-out pair (q, q) has the bound +inf: never kept)
                    keep = (no_prune ? v < inf_of<T>() : v <= ub) && (uint32_t)t != st &&
                           (!finite_only || v < inf_of<T>());
                    if (keep) bk[e] = bucket_of(v, inv);
                }
                if (keep) {
                    keepm |= 1u << e;
                    pos[e] = atomicAdd(&scount[bk[e]], 1u);
                }
            }
            if (!scatter) continue;
            __syncthreads();
            if (tid < kBuckets) {
                const unsigned int c = scount[tid];
                sbase[tid] = c ? atomicAdd(bcursor + tid, (unsigned long long)c) : 0ull;
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; e++)
                if ((keepm >> e) & 1u)
                    queue[boff[bk[e]] + sbase[bk[e]] + pos[e]] =
                        make_uint2((uint32_t)q, (uint32_t)(t0 + (int64_t)e * blockDim.x + tid));
            __syncthreads();
            if (tid < kBuckets) scount[tid] = 0;
            __syncthreads();
        }
    }
    if (!scatter) {
        __syncthreads();
        if (tid < kBuckets && scount[tid]) atomicAdd(bcount + tid, (unsigned long long)scount[tid]);
    }
}

// S5 (FP32): t is a possible exact argmin iff lower(D_t) <= upper(D_best).
__device__ __forceinline__ bool in_recheck_set(const Cand &e, unsigned long long kb, float lo,
                                               float hi, float abs32) {
    return lower32(e.d, lo, abs32) <= upper32(key_dist(kb), hi, abs32);
}

// The per-query end of one FP32 search: the candidate list, the keys, the
// recheck list and the outputs.
struct FinishJob32 {
    const Cand *cand;
    const unsigned long long *ccount, *bsf;
    float lo, hi, abs32;
    int32_t *rcount;
    int exact;
    uint2 *rlist;
    unsigned long long *counters;     // C_RECHECK (recheck list length), C_RQUERIES
    const double *d64;
    unsigned long long *best64;
    int32_t *bestidx;
    int64_t Q;
    const int32_t *labels;
    int32_t *nn_idx, *nn_label;
    double *nn_dist;
};

template <typename Src>
__global__ void filter32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const FinishJob32 &j = src.get(bid, nblk);
    const long long n = (long long)*j.ccount;
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < n;
         i += (long long)nblk * blockDim.x) {
        const Cand e = j.cand[i];
        if (in_recheck_set(e, j.bsf[e.q], j.lo, j.hi, j.abs32)) atomicAdd(j.rcount + e.q, 1);
    }
}

template <typename Src>
__global__ void collect32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const FinishJob32 &j = src.get(bid, nblk);
    const long long n = (long long)*j.ccount;
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < n;
         i += (long long)nblk * blockDim.x) {
        const Cand e = j.cand[i];
        const unsigned long long kb = j.bsf[e.q];
        if (!in_recheck_set(e, kb, j.lo, j.hi, j.abs32)) continue;
        const int rc = j.rcount[e.q];
        if (!(j.exact || rc >= 2)) continue;
        const unsigned long long slot = atomicAdd(j.counters + C_RECHECK, 1ull);
        j.rlist[slot] = make_uint2((uint32_t)e.q, (uint32_t)e.t);
        if ((uint32_t)e.t == key_idx(kb)) atomicAdd(j.counters + C_RQUERIES, 1ull);
    }
}

template <typename Src>
__global__ void ties32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const FinishJob32 &j = src.get(bid, nblk);
    const long long n = (long long)j.counters[C_RECHECK];
    for (long long i = (long long)bid * blockDim.x + threadIdx.x; i < n;
         i += (long long)nblk * blockDim.x) {
        const uint2 e = j.rlist[i];
        if (dbits(j.d64[i]) == j.best64[e.x]) atomicMin(j.bestidx + e.x, (int32_t)e.y);
    }
}

template <typename Src>
__global__ void finalize32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const FinishJob32 &j = src.get(bid, nblk);
    for (int64_t q = (int64_t)bid * blockDim.x + threadIdx.x; q < j.Q;
         q += (int64_t)nblk * blockDim.x) {
        const unsigned long long kb = j.bsf[q];
        if (kb == ~0ull) {
            // no candidate: no training series has a warping path inside the
            // window (unequal lengths only)
            j.nn_idx[q] = -1;
            j.nn_label[q] = -1;
            j.nn_dist[q] = inf_of<double>();
            continue;
        }
        int32_t idx;
        double dist;
        if (j.exact || j.rcount[q] >= 2) {
            idx = j.bestidx[q];
            dist = __longlong_as_double((long long)j.best64[q]);
        } else {
            idx = (int32_t)key_idx(kb);
            dist = (double)key_dist(kb);
        }
        j.nn_idx[q] = idx;
        j.nn_label[q] = j.labels[idx];
        j.nn_dist[q] = dist;
    }
}

// The search's starting values: counters and bucket tallies 0, query keys
// and FP64 bests all ones (no candidate), recheck tallies 0, tie indices
// INT_MAX (0x7f7f7f7f as written by a byte fill).
struct InitJob32 {
    unsigned long long *counters, *buckets, *bsf, *seed, *best64;
    int32_t *rcount, *bestidx;
    int64_t Q;
};

template <typename Src>
__global__ void init32_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const InitJob32 &j = src.get(bid, nblk);
    const int64_t stride = (int64_t)nblk * blockDim.x;
    const int64_t i0 = (int64_t)bid * blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < C_COUNT; i += stride) j.counters[i] = 0ull;
    for (int64_t i = i0; i < 2 * kBuckets; i += stride) j.buckets[i] = 0ull;
    for (int64_t q = i0; q < j.Q; q += stride) {
        j.bsf[q] = ~0ull;
        j.seed[q] = ~0ull;
        j.best64[q] = ~0ull;
        j.rcount[q] = 0;
        j.bestidx[q] = 0x7f7f7f7f;
    }
}

__global__ void ties64_kernel(const Cand64 *__restrict__ cand, const unsigned long long *ccount,
                              const unsigned long long *__restrict__ bsf64,
                              int32_t *__restrict__ bestidx) {
    const long long n = (long long)*ccount;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Cand64 e = cand[i];
        if (dbits(e.d) == bsf64[e.q]) atomicMin(bestidx + e.q, e.t);
    }
}

__global__ void finalize64_kernel(int64_t Q, const unsigned long long *__restrict__ bsf64,
                                  const int32_t *__restrict__ bestidx,
                                  const int32_t *__restrict__ labels, int32_t *__restrict__ nn_idx,
                                  int32_t *__restrict__ nn_label, double *__restrict__ nn_dist) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t idx = bestidx[q];
        nn_idx[q] = idx;
        nn_label[q] = labels[idx];
        nn_dist[q] = __longlong_as_double((long long)bsf64[q]);
    }
}

// ---------------------------------------------------------------- workspace

long long band_cells(int L, int W) {
    const long long w = W > L - 1 ? L - 1 : W;
    return (long long)L * (2 * w + 1) - w * (w + 1);
}

// CUDA events at the stage boundaries of one search (NNDTW_TIME_STAGES).
// One set of events per thread and device, created on first use and reused;
// the set of the thread's last timed search is read by nn_dtw_stage_times().
struct EventSet {
    cudaEvent_t ev[8] = {};
    bool ready = false;
};
thread_local EventSet t_events[64];
thread_local int t_last_dev = -1;

struct StageTimer {
    bool on = false;
    cudaStream_t s = nullptr;
    EventSet *set = nullptr;
    cudaError_t start(bool enabled, cudaStream_t st) {
        on = enabled;
        s = st;
        if (!on) return cudaSuccess;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        set = &t_events[dev];
        if (!set->ready) {
            for (int i = 0; i < 8; i++) {
                e = cudaEventCreate(&set->ev[i]);
                if (e != cudaSuccess) return e;
            }
            set->ready = true;
        }
        t_last_dev = dev;
        return mark(0);
    }
    cudaError_t mark(int i) {
        if (!on) return cudaSuccess;
        // inside a stream capture the record must be an external graph node
        // so that the event is recorded every time the graph runs
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) return e;
        if (cs == cudaStreamCaptureStatusActive)
            return cudaEventRecordWithFlags(set->ev[i], s, cudaEventRecordExternal);
        return cudaEventRecord(set->ev[i], s);
    }
};

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base(static_cast<char *>(b)) {}
    template <typename P> P *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        P *p = base ? reinterpret_cast<P *>(base + off) : nullptr;
        off += count * sizeof(P);
        return p;
    }
};

struct Layout32 {
    unsigned long long *counters, *bsf, *seed, *best64, *buckets;
    int32_t *rcount, *bestidx;
    float *env, *envq, *env2, *lb, *ends, *norms;
    uint2 *queue, *rlist;
    Cand *cand;
    double *d64;
    size_t bytes;
};

Layout32 layout32(void *base, int64_t N, int64_t Q, int L) {
    Carve c(base);
    Layout32 l;
    const size_t cap = (size_t)Q * (size_t)N + (size_t)Q;
    l.counters = c.take<unsigned long long>(C_COUNT);
    l.buckets = c.take<unsigned long long>(2 * kBuckets);
    l.bsf = c.take<unsigned long long>(Q);
    l.seed = c.take<unsigned long long>(Q);
    l.best64 = c.take<unsigned long long>(Q);
    l.rcount = c.take<int32_t>(Q);
    l.bestidx = c.take<int32_t>(Q);
    l.env = c.take<float>((size_t)N * L * 2);
    l.envq = c.take<float>((size_t)Q * L * 2);
    l.env2 = c.take<float>((size_t)N * L * 2);
    l.lb = c.take<float>((size_t)Q * N);
    l.ends = c.take<float>((size_t)Q * N);
    l.norms = c.take<float>((size_t)Q + (size_t)N);
    l.queue = c.take<uint2>((size_t)Q * N);
    l.cand = c.take<Cand>(cap);
    l.rlist = c.take<uint2>(cap);
    l.d64 = c.take<double>(cap);
    l.bytes = c.off + 256;
    return l;
}

struct Layout64 {
    unsigned long long *counters, *bsf64, *seed, *buckets;
    int32_t *bestidx;
    double *env, *envq, *env2, *lb, *ends, *norms;
    uint2 *queue;
    Cand64 *cand;
    size_t bytes;
};

Layout64 layout64(void *base, int64_t N, int64_t Q, int L) {
    Carve c(base);
    Layout64 l;
    const size_t cap = (size_t)Q * (size_t)N + (size_t)Q;
    l.counters = c.take<unsigned long long>(C_COUNT);
    l.buckets = c.take<unsigned long long>(2 * kBuckets);
    l.bsf64 = c.take<unsigned long long>(Q);
    l.seed = c.take<unsigned long long>(Q);
    l.bestidx = c.take<int32_t>(Q);
    l.env = c.take<double>((size_t)N * L * 2);
    l.envq = c.take<double>((size_t)Q * L * 2);
    l.env2 = c.take<double>((size_t)N * L * 2);
    l.lb = c.take<double>((size_t)Q * N);
    l.ends = c.take<double>((size_t)Q * N);
    l.norms = c.take<double>((size_t)Q + (size_t)N);
    l.queue = c.take<uint2>((size_t)Q * N);
    l.cand = c.take<Cand64>(cap);
    l.bytes = c.off + 256;
    return l;
}

bool search_sizes_ok(int64_t N, int64_t Q, int L, int W, int V) {
    if (N < 1 || Q < 0 || L < 2 || L > NNDTW_MAX_L || W < 0 || V < 1) return false;
    if (N > 0x7fffffffll || Q > 0x7fffffffll) return false;
    return true;
}

// Queries per chunk: a search runs its queries in chunks of at most
// NNDTW_CHUNK_PAIRS (query, training series) pairs, one after another, so
// that its workspace (about 48 bytes per pair of a chunk) never grows with
// Q x N beyond that; each query's search is independent of the others, so the
// results do not depend on the chunking.
int64_t chunk_queries(int64_t N, int64_t Q) {
    const int64_t per = (int64_t)NNDTW_CHUNK_PAIRS / N;
    const int64_t qc = per < 1 ? 1 : per;
    return Q < qc ? Q : qc;
}

unsigned grid_small(long long n) {
    long long g = (n + kSmallThreads - 1) / kSmallThreads;
    long long cap = (long long)device_sm_count() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

dim3 grid_compact(int64_t Q, int64_t N) {
    const long long per_block = (long long)kSmallThreads * kCompactE;
    long long gx = (N + per_block - 1) / per_block;
    if (gx > 64) gx = 64;
    // rows per CTA (it strides over them): enough for about 8192 bounds, so
    // that a CTA on short rows does more than its start-up and barriers, but
    // no fewer CTAs than two per SM while the rows allow (a small search's
    // rows run side by side, not one after another in a CTA)
    const long long per_row = (N + gx - 1) / gx;
    long long rows = per_row > 0 ? 8192 / per_row : 1;
    if (rows > 32) rows = 32;
    const long long min_ctas = 2ll * device_sm_count();
    const long long gy_min = (min_ctas + gx - 1) / gx;
    const long long spread = Q / gy_min;   // rows per CTA with gy_min CTAs
    if (rows > spread) rows = spread;
    if (rows < 1) rows = 1;
    long long gy = (Q + rows - 1) / rows;
    if (gy > 65535) gy = 65535;
    if (gy < 1) gy = 1;
    return dim3((unsigned)gx, (unsigned)gy);
}

#define CK(x)                                                       \
    do {                                                            \
        cudaError_t e_ = (x);                                       \
        if (e_ != cudaSuccess) { set_last_cuda_error(e_); return NNDTW_ECUDA; } \
    } while (0)

// First index of the LB_Keogh bridge of Eq. 7 (the number of bands,
// min(L/2, V), at least 1), as in the bound kernel.
int bridge_start(int L, int V) {
    const int nb = L / 2 < V ? L / 2 : V;
    return nb < 1 ? 1 : nb;
}

void fill_stats(nndtw_stats *st, const unsigned long long *h, int64_t N, int64_t Q, int L,
                int W, bool counted) {
    std::memset(st, 0, sizeof(*st));
    st->pairs = Q * N;
    st->lb_pruned = Q * N - Q - (int64_t)h[C_QUEUE];
    st->rechecked = (int64_t)h[C_RECHECK];
    st->recheck_queries = (int64_t)h[C_RQUERIES];
    if (counted) {
        st->dtw_started = (int64_t)h[C_STARTED];
        st->dtw_abandoned = (int64_t)h[C_ABANDONED];
        st->dtw_cells = (int64_t)h[C_CELLS];
        st->seed_cells = Q * band_cells(L, W);
        st->lb_pruned_reverse = (int64_t)h[C_REVPRUNED];
        st->lb_pruned_improved = (int64_t)h[C_IMPPRUNED];
        st->lb_pruned_live = (int64_t)h[C_LIVEPRUNED];
    }
}

void add_stats(nndtw_stats *t, const nndtw_stats &p) {
    t->pairs += p.pairs;
    t->lb_pruned += p.lb_pruned;
    t->dtw_started += p.dtw_started;
    t->dtw_abandoned += p.dtw_abandoned;
    t->dtw_cells += p.dtw_cells;
    t->rechecked += p.rechecked;
    t->recheck_queries += p.recheck_queries;
    t->seed_cells += p.seed_cells;
    t->lb_pruned_reverse += p.lb_pruned_reverse;
    t->lb_pruned_improved += p.lb_pruned_improved;
    t->lb_pruned_live += p.lb_pruned_live;
}

template <typename T>
int check_finite(const T *x, int64_t n, T limit, unsigned long long *bad, cudaStream_t s) {
    if (n <= 0) return NNDTW_OK;
    finite_check_kernel<T><<<grid_small(n), kSmallThreads, 0, s>>>(x, n, limit, bad);
    CK(cudaGetLastError());
    return NNDTW_OK;
}

int group_from_flags(unsigned flags) {
    const unsigned v = (flags & NNDTW_DTW_GROUP_MASK) >> 8;
    if (v == 7) {
        const unsigned lanes = (flags & NNDTW_DTW_ROWS_LANES_MASK) >> 12;
        return kRowsGroup + (lanes <= 2 ? (int)lanes : 0);
    }
    return v ? 1 << (v - 1) : 0;
}

// ------------------------------------------------------------ FP32 executor
//
// One FP32 search over one dataset or a batch of up to kMaxSets datasets,
// stage by stage on the caller's stream: every stage is one launch over all
// datasets of the batch (one per kernel variant where datasets need
// different ones: tile shapes, DTW layouts), each dataset's CTAs working on
// its own job (SrcN; a single dataset takes the Src1 form).  The datasets'
// workspaces are separate, so no stage of one dataset reads another's data.

struct Set32 {
    const float *train;
    const int32_t *labels;
    int64_t N;
    const float *test;
    int64_t Q;
    int L, W, V;
    const float *env;   // nullptr: built into the workspace
    unsigned flags;
    int32_t *nn_idx, *nn_label;
    double *nn_dist;
    void *ws;           // workspace laid out for q_cap queries, 256-byte aligned
    int64_t q_base;     // index of the first query of this chunk (leave-one-out)
    int64_t q_cap;      // queries the workspace layout holds (Q <= q_cap; the same
                        // for every chunk of a search, so chunks find one layout)
    bool train_ready;   // the training-side data (envelopes, second envelopes,
                        // packed records) is already in the workspace
};

// One kernel (its two forms, block size, largest dynamic shared memory) and
// the datasets it serves in one launch.
template <typename Job> struct Batch {
    void (*fn1)(Src1<Job>) = nullptr;
    void (*fnN)(SrcN<Job>) = nullptr;   // nullptr: no batch form, one launch per dataset
    int threads = 0;
    size_t smem = 0;
    SrcNBuilder<Job> b;
};

// kernel launches issued by the calling thread's last FP32 search call, in
// all and per stage (stage k: between stage boundaries k and k+1 of
// nn_dtw_stage_times)
thread_local long long t_launches = 0;
thread_local long long t_stage_launches[8] = {};
thread_local int t_stage = 0;

void reset_launch_counts() {
    t_launches = 0;
    t_stage = 0;
    for (auto &c : t_stage_launches) c = 0;
}

template <typename Job>
cudaError_t launch_batch(const Batch<Job> &g, cudaStream_t s) {
    const SrcN<Job> &src = g.b.src;
    if (src.n == 0) return cudaSuccess;
    const long long k = (src.n > 1 && g.fnN) ? 1 : src.n;
    t_launches += k;
    t_stage_launches[t_stage] += k;
    if (g.smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(g.fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)g.smem);
        if (e == cudaSuccess && g.fnN)
            e = cudaFuncSetAttribute(g.fnN, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)g.smem);
        if (e != cudaSuccess) return e;
    }
    if (src.n > 1 && g.fnN) {
        g.fnN<<<(unsigned)src.off[src.n], g.threads, g.smem, s>>>(src);
        return cudaGetLastError();
    }
    for (int d = 0; d < src.n; d++) {
        g.fn1<<<(unsigned)(src.off[d + 1] - src.off[d]), g.threads, g.smem, s>>>(
            Src1<Job>{src.jobs[d]});
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Batches keyed by kernel and block size (a handful per stage); a key with
// more than kMaxSets jobs (a stage with two jobs per dataset) gets another
// batch.
template <typename Job> struct Batches {
    std::vector<Batch<Job>> v;
    Batch<Job> &of(void (*fn1)(Src1<Job>), void (*fnN)(SrcN<Job>), int threads) {
        for (auto &g : v)
            if (g.fn1 == fn1 && g.threads == threads && !g.b.full()) return g;
        v.emplace_back();
        Batch<Job> &g = v.back();
        g.fn1 = fn1;
        g.fnN = fnN;
        g.threads = threads;
        return g;
    }
    void add(void (*fn1)(Src1<Job>), void (*fnN)(SrcN<Job>), int threads, size_t smem,
             const Job &job, long long blocks) {
        if (blocks <= 0) return;
        Batch<Job> &g = of(fn1, fnN, threads);
        g.smem = std::max(g.smem, smem);
        g.b.add(job, (int)blocks);
    }
    cudaError_t launch(cudaStream_t s) const {
        for (const auto &g : v) {
            const cudaError_t e = launch_batch(g, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

// Streams on which the variant launches of one stage (bounds, first
// candidates, DTW) run side by side: a few per caller stream and device,
// created on first use and kept, so that calls on different streams never
// share them.  A stage forks from the caller's stream with an event, issues
// its launches round-robin over them and joins back, so the stage events on
// the caller's stream still bracket all of its launches (and a captured
// graph holds the fork and the join).
constexpr int kForkStreams = 8;
struct ForkSet {
    cudaStream_t st[kForkStreams] = {};
    cudaEvent_t fork = nullptr, join[kForkStreams] = {};
};
std::mutex g_fork_mu;
std::vector<std::pair<std::pair<int, cudaStream_t>, ForkSet *>> g_forks;

cudaError_t fork_set(cudaStream_t s, ForkSet **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_fork_mu);
    for (auto &kv : g_forks)
        if (kv.first.first == dev && kv.first.second == s) {
            *out = kv.second;
            return cudaSuccess;
        }
    ForkSet *f = new ForkSet();
    for (int k = 0; k < kForkStreams; k++) {
        e = cudaStreamCreateWithFlags(&f->st[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->join[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    e = cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    g_forks.push_back({{dev, s}, f});
    *out = f;
    return cudaSuccess;
}

// Launches a stage's batches: one batch on the caller's stream, several side
// by side on the fork streams (always joined back, also after an error).
template <typename Job>
cudaError_t launch_forked(const Batches<Job> &g, cudaStream_t s) {
    const int nb = (int)g.v.size();
    if (nb <= 1) return g.launch(s);
    ForkSet *f = nullptr;
    cudaError_t e = fork_set(s, &f);
    if (e != cudaSuccess) return e;
    const int used = nb < kForkStreams ? nb : kForkStreams;
    e = cudaEventRecord(f->fork, s);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < used; k++) {
        e = cudaStreamWaitEvent(f->st[k], f->fork, 0);
        if (e != cudaSuccess) return e;
    }
    cudaError_t first = cudaSuccess;
    for (int b = 0; b < nb && first == cudaSuccess; b++) first = launch_batch(g.v[b], f->st[b % used]);
    for (int k = 0; k < used; k++) {
        e = cudaEventRecord(f->join[k], f->st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, f->join[k], 0);
        if (e != cudaSuccess && first == cudaSuccess) first = e;
    }
    return first;
}

struct Prep32 {
    Layout32 ws;
    int Weff;
    Margins m;
    bool keogh, rev, imp, second, loo, no_prune, exact;
    const float *env;
    unsigned long long *cnt;   // work counters (stats), or nullptr
};

// Blocks for a grid-stride pass over a dataset's candidate lists (at least
// one candidate per query, typically a few): enough threads for about eight
// per query, at most the small-kernel grid.
long long finish_blocks(int64_t Q, int64_t N) {
    const long long by_q = (8 * Q + kSmallThreads - 1) / kSmallThreads;
    const long long cap = grid_small((long long)Q * N + Q);
    return std::max(1ll, std::min(by_q, cap));
}

int run32(const Set32 *sets, int n, bool want_stats, bool timing, nndtw_stats *stats,
          StageTimer &tm, cudaStream_t s) {
    const int sms = device_sm_count();
    t_stage = 0;
    std::vector<Prep32> P(n);
    for (int d = 0; d < n; d++) {
        const Set32 &x = sets[d];
        Prep32 &p = P[d];
        p.ws = layout32(x.ws, x.N, x.q_cap, x.L);
        p.Weff = x.W > x.L - 1 ? x.L - 1 : x.W;
        p.m = make_margins(x.L);
        p.keogh = (x.flags & NNDTW_KEOGH_BOUND) != 0;
        p.no_prune = (x.flags & NNDTW_NO_PRUNE) != 0;
        // the cascade's second stage: the reverse bound (NNDTW_REVERSE) and/or
        // the bound with the LB_Improved bridge (NNDTW_IMPROVED), tuning
        // choices; LB_Keogh as the bound (NNDTW_KEOGH_BOUND) has none
        p.rev = (x.flags & NNDTW_REVERSE) && !p.keogh &&
                !(x.flags & (NNDTW_NO_PRUNE | NNDTW_NO_REVERSE));
        p.imp = (x.flags & NNDTW_IMPROVED) && !p.keogh && !p.no_prune;
        p.second = p.rev || p.imp;
        p.loo = (x.flags & NNDTW_LEAVE_ONE_OUT) != 0;
        p.exact = (x.flags & NNDTW_EXACT_DIST) != 0;
        p.env = x.env ? x.env : p.ws.env;
        // (a later chunk of a search finds the training envelopes it built)
        p.cnt = (want_stats && !timing) ? p.ws.counters : nullptr;
    }
    // Order of the datasets inside a stage's launches: the CTAs of a launch
    // are dispatched roughly in job order, so the datasets with the longest
    // CTAs (bound pass: the longest series; DTW: the most band cells per
    // pair, whose persistent grids drain slowest) go first and the launch
    // ends on short ones.
    std::vector<int> ord_len(n), ord_band(n);
    std::iota(ord_len.begin(), ord_len.end(), 0);
    std::iota(ord_band.begin(), ord_band.end(), 0);
    std::stable_sort(ord_len.begin(), ord_len.end(),
                     [&](int a, int b) { return sets[a].L > sets[b].L; });
    auto band_of = [&](int d) {
        const long long w = 2ll * P[d].Weff + 1;
        return (long long)sets[d].L * (w < sets[d].L ? w : sets[d].L);
    };
    std::stable_sort(ord_band.begin(), ord_band.end(),
                     [&](int a, int b) { return band_of(a) > band_of(b); });

    // starting values of every dataset's counters, keys and tallies
    {
        Batches<InitJob32> g;
        for (int d = 0; d < n; d++) {
            const Layout32 &w = P[d].ws;
            const InitJob32 j{w.counters, w.buckets, w.bsf, w.seed, w.best64, w.rcount, w.bestidx,
                              sets[d].Q};
            g.add(init32_kernel<Src1<InitJob32>>, init32_kernel<SrcN<InitJob32>>, kSmallThreads,
                  0, j, std::min<long long>(grid_small(std::max<int64_t>(sets[d].Q, 64)), 64));
        }
        CK(g.launch(s));
    }
    // optional scan for non-finite inputs (waits for the stream)
    {
        bool any = false;
        for (int d = 0; d < n; d++) {
            if (!(sets[d].flags & NNDTW_CHECK_FINITE)) continue;
            any = true;
            unsigned long long *bad = P[d].ws.counters + C_BAD;
            t_launches += 2;
            t_stage_launches[t_stage] += 2;
            int rc = check_finite<float>(sets[d].train, sets[d].N * sets[d].L, 1e15f, bad, s);
            if (rc) return rc;
            rc = check_finite<float>(sets[d].test, sets[d].Q * sets[d].L, 1e15f, bad, s);
            if (rc) return rc;
        }
        if (any) {
            std::vector<unsigned long long> h(n, 0ull);
            for (int d = 0; d < n; d++)
                if (sets[d].flags & NNDTW_CHECK_FINITE)
                    CK(cudaMemcpyAsync(&h[d], P[d].ws.counters + C_BAD, sizeof(h[d]),
                                       cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int d = 0; d < n; d++)
                if (h[d]) return NNDTW_ENONFINITE;
        }
    }
    // S1: training envelopes (unless supplied) and, for the cascade's second
    // stage, the queries' envelopes; then the second envelopes and the packed
    // training records of the LB_Improved bridge
    {
        Batches<EnvJob<float>> g;
        auto add = [&](const float *src, const float *ein, int64_t cnt, int d, float *out) {
            const EnvPlan<float> ep = plan_envelopes<float>(src, ein, cnt, sets[d].L, P[d].Weff, out);
            const EnvFns<float> f = envelope_fns<float>(ep.one_pass);
            g.add(f.fn1, f.fnN, kEnvelopeThreads, ep.smem, ep.job, ep.blocks);
        };
        for (int d : ord_len) {
            if (!sets[d].env && !sets[d].train_ready)
                add(sets[d].train, nullptr, sets[d].N, d, P[d].ws.env);
            if (P[d].second) add(sets[d].test, nullptr, sets[d].Q, d, P[d].ws.envq);
        }
        CK(g.launch(s));
        Batches<EnvJob<float>> g2;
        Batches<PackJob> gp;
        const PackFns pf = pack_bgap_fns();
        for (int d = 0; d < n; d++) {
            if (!P[d].imp || sets[d].train_ready) continue;
            const EnvPlan<float> ep = plan_envelopes<float>(nullptr, P[d].env, sets[d].N, sets[d].L,
                                                            P[d].Weff, P[d].ws.env2);
            const EnvFns<float> f = envelope_fns<float>(ep.one_pass);
            g2.add(f.fn1, f.fnN, kEnvelopeThreads, ep.smem, ep.job, ep.blocks);
            const long long ne = sets[d].N * sets[d].L;
            gp.add(pf.fn1, pf.fnN, 256, 0, PackJob{sets[d].train, P[d].ws.env2, ne},
                   pack_bgap_blocks(ne));
        }
        CK(g2.launch(s));
        CK(gp.launch(s));
    }
    t_stage = 1;
    CK(tm.mark(1));
    // S2: squared norms, then the safe bounds of all pairs and each query's
    // Euclidean-nearest training series (its first candidate)
    {
        Batches<SqnormJob<float>> gs;
        Batches<LbJob<float>> gl;
        for (int d : ord_len) {
            const Set32 &x = sets[d];
            const Prep32 &p = P[d];
            LbPlan<float> lp{};
            CK(plan_lb<float>(x.test, x.Q, x.train, p.env, x.N, x.L, p.Weff, x.V, p.keogh, true,
                              p.m.lb_lo, p.m.abs32, p.ws.lb, p.ws.seed, p.ws.norms,
                              p.rev ? p.ws.ends : nullptr, p.loo, &lp, x.q_base,
                              (int)((x.flags & NNDTW_LB_TILE_MASK) >> 19),
                              /*ed_bound=*/!p.rev && !p.imp));
            const LbFns<float> f = lb_fns<float>(lp.tile, lp.ed);
            gs.add(f.sq1, f.sqN, 256, 0, lp.sq, lp.sq_blocks);
            gl.add(f.fn1, f.fnN, kLbThreads, lp.smem, lp.job, lp.blocks);
        }
        CK(gs.launch(s));
        CK(launch_forked(gl, s));
    }
    t_stage = 2;
    CK(tm.mark(2));
    // S4 on each query's first candidate (no abandoning): initial upper bounds
    std::vector<DtwJob32> main_jobs(n);
    {
        Batches<DtwJob32> g;
        for (int d : ord_band) {
            const Set32 &x = sets[d];
            const Prep32 &p = P[d];
            DtwJob32 j{};
            j.test = x.test; j.train = x.train; j.L = x.L; j.W = p.Weff;
            j.dtw_lo = p.m.dtw_lo; j.dtw_hi = p.m.dtw_hi; j.abs32 = p.m.abs32;
            j.bsf = p.ws.bsf; j.cand = p.ws.cand; j.cand_count = p.ws.counters + C_CAND;
            j.counters = p.cnt;
            j.group = group_from_flags(x.flags);
            main_jobs[d] = j;
            // one pair per query: latency-bound, so each pair gets the widest group
            j.pairs = nullptr; j.seed_keys = p.ws.seed; j.n_seed = x.Q; j.head = nullptr;
            j.abandon = 0;
            j.group = (dtw32_rows_ok(x.L, p.Weff) || dtw32_rowsc_ok(x.L, p.Weff))
                          ? kRowsGroup : dtw32_wide_group(p.Weff);
            Dtw32Plan pl{};
            CK(plan_dtw32(j, sms, &pl));
            j.lanes = pl.lanes;
            g.add(pl.fn1, pl.fnN, pl.threads, pl.smem, j, pl.blocks);
        }
        CK(launch_forked(g, s));
    }
    t_stage = 3;
    CK(tm.mark(3));
    // S3: compaction against the upper bounds, two passes (count, scatter)
    for (int pass = 0; pass < 2; pass++) {
        Batches<CompactJob<float>> g;
        for (int d = 0; d < n; d++) {
            const Set32 &x = sets[d];
            const Prep32 &p = P[d];
            const dim3 gc = grid_compact(x.Q, x.N);
            CompactJob<float> j{};
            j.lb = p.ws.lb; j.Q = x.Q; j.N = x.N; j.bsf = p.ws.bsf; j.seed = p.ws.seed;
            j.ubof = UbOf<float>{p.m.dtw_hi, p.m.abs32};
            j.no_prune = p.no_prune ? 1 : 0;
            j.gx = (int)gc.x;
            j.scatter = pass;
            j.bcount = p.ws.buckets; j.bcursor = p.ws.buckets + kBuckets;
            j.qcount = p.ws.counters + C_QUEUE; j.queue = p.ws.queue;
            g.add(compact_kernel<float, Src1<CompactJob<float>>>,
                  compact_kernel<float, SrcN<CompactJob<float>>>, kSmallThreads, 0, j,
                  (long long)gc.x * gc.y);
        }
        CK(g.launch(s));
    }
    // the cascade's second stage on the survivors (into the recheck list's
    // storage, which S5 fills only after the DTW pass)
    {
        Batches<CascadeJob> g;
        for (int d = 0; d < n; d++) {
            const Set32 &x = sets[d];
            const Prep32 &p = P[d];
            if (!p.second) continue;
            CascadeJob cj{};
            cj.in = p.ws.queue; cj.in_count = p.ws.counters + C_QUEUE;
            cj.train = x.train; cj.envq = reinterpret_cast<const float2 *>(p.ws.envq);
            cj.ends = p.rev ? p.ws.ends : nullptr;
            cj.bgap = p.imp ? reinterpret_cast<const BGap *>(p.ws.env2) : nullptr;
            cj.lb = p.ws.lb;
            cj.N = x.N; cj.L = x.L; cj.nb = bridge_start(x.L, x.V);
            cj.bsf = p.ws.bsf;
            cj.lb_lo = p.m.lb_lo; cj.lb_abs = p.m.abs32; cj.dtw_hi = p.m.dtw_hi;
            cj.abs32 = p.m.abs32;
            cj.out = p.ws.rlist; cj.out_count = p.ws.counters + C_QUEUE2; cj.counters = p.cnt;
            const CascadeFns f = cascade_filter_fns(p.rev, p.imp);
            g.add(f.fn1, f.fnN, 256, 0, cj, cascade_filter_blocks(x.Q * x.N, sms));
        }
        CK(g.launch(s));
    }
    t_stage = 4;
    CK(tm.mark(4));
    // S4 on the survivors, with early abandoning
    {
        Batches<DtwJob32> g;
        for (int d : ord_band) {
            const Prep32 &p = P[d];
            DtwJob32 j = main_jobs[d];
            j.pairs = p.second ? p.ws.rlist : p.ws.queue; j.seed_keys = nullptr;
            j.count = p.ws.counters + (p.second ? C_QUEUE2 : C_QUEUE);
            j.head = p.ws.counters + C_HEAD;
            if (!p.no_prune) {   // live pruning against the tightening bests
                j.lb = p.ws.lb;
                j.lb_n = sets[d].N;
            }
            j.abandon = (sets[d].flags & NNDTW_NO_ABANDON) ? 0 : 1;
            Dtw32Plan pl{};
            CK(plan_dtw32(j, sms, &pl));
            j.lanes = pl.lanes;
            g.add(pl.fn1, pl.fnN, pl.threads, pl.smem, j, pl.blocks);
        }
        CK(launch_forked(g, s));
    }
    t_stage = 5;
    CK(tm.mark(5));
    // S5: near-tie recheck in FP64 and the final argmin
    std::vector<FinishJob32> fin(n);
    for (int d = 0; d < n; d++) {
        const Set32 &x = sets[d];
        const Prep32 &p = P[d];
        FinishJob32 &j = fin[d];
        j.cand = p.ws.cand; j.ccount = p.ws.counters + C_CAND; j.bsf = p.ws.bsf;
        j.lo = p.m.dtw_lo; j.hi = p.m.dtw_hi; j.abs32 = p.m.abs32;
        j.rcount = p.ws.rcount; j.exact = p.exact ? 1 : 0; j.rlist = p.ws.rlist;
        j.counters = p.ws.counters; j.d64 = p.ws.d64; j.best64 = p.ws.best64;
        j.bestidx = p.ws.bestidx; j.Q = x.Q; j.labels = x.labels;
        j.nn_idx = x.nn_idx; j.nn_label = x.nn_label; j.nn_dist = x.nn_dist;
    }
    auto finish = [&](void (*f1)(Src1<FinishJob32>), void (*fN)(SrcN<FinishJob32>), bool per_q) {
        Batches<FinishJob32> g;
        for (int d = 0; d < n; d++)
            g.add(f1, fN, kSmallThreads, 0, fin[d],
                  per_q ? (long long)grid_small(sets[d].Q) : finish_blocks(sets[d].Q, sets[d].N));
        return g.launch(s);
    };
    CK(finish(filter32_kernel<Src1<FinishJob32>>, filter32_kernel<SrcN<FinishJob32>>, false));
    CK(finish(collect32_kernel<Src1<FinishJob32>>, collect32_kernel<SrcN<FinishJob32>>, false));
    {
        Batches<DtwJob64> g;
        for (int d = 0; d < n; d++) {
            const Set32 &x = sets[d];
            const Prep32 &p = P[d];
            DtwJob64 r{};
            r.test32 = x.test; r.train32 = x.train; r.L = x.L; r.W = p.Weff;
            r.pairs = p.ws.rlist; r.count = p.ws.counters + C_RECHECK; r.head = nullptr;
            r.bsf64 = p.ws.best64; r.out = p.ws.d64; r.abandon = 0;
            Dtw64Plan pl{};
            CK(plan_dtw64(r, sms, &pl));
            // a few pairs per dataset at most unless every query is rechecked
            const long long want = p.exact ? x.Q : std::max<long long>(4, (x.Q + 7) / 8);
            g.add(pl.fn1, pl.fnN, pl.threads, pl.smem, r, std::min(pl.blocks, want));
        }
        CK(launch_forked(g, s));
    }
    CK(finish(ties32_kernel<Src1<FinishJob32>>, ties32_kernel<SrcN<FinishJob32>>, false));
    t_stage = 6;
    CK(tm.mark(6));
    CK(finish(finalize32_kernel<Src1<FinishJob32>>, finalize32_kernel<SrcN<FinishJob32>>, true));
    t_stage = 7;
    CK(tm.mark(7));
    if (stats && n == 1) {
        unsigned long long h[C_COUNT];
        CK(cudaMemcpyAsync(h, P[0].ws.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        fill_stats(stats, h, sets[0].N, sets[0].Q, sets[0].L, P[0].Weff, P[0].cnt != nullptr);
    }
    return NNDTW_OK;
}

// ------------------------------------------------- unequal-length executor
//
// One chunk of queries of the unequal-length search (Sec. 2 generalised),
// on the caller's stream: the stages of run32 over ragged sets.  The first
// candidate of each query is the series with the smallest bound (the
// Euclidean distance is undefined for unequal lengths); pairs without a
// warping path inside the window (|L_A - L_B| > W) have the bound +inf and
// are never kept; a query none of whose pairs has one gets index -1.
struct SetVar {
    const float *train;
    const long long *train_off;
    const int32_t *labels;
    int64_t N;
    const float *test;
    const long long *test_off;   // the chunk's first query's entry (absolute offsets)
    int64_t Q;
    int max_len, W, V;
    unsigned flags;
    int32_t *nn_idx, *nn_label;
    double *nn_dist;
    void *ws;
    int64_t q_cap;
    bool train_ready;   // the training envelopes are already in the workspace
};

int run_var(const SetVar &x, bool want_stats, bool timing, nndtw_stats *stats, StageTimer &tm,
            cudaStream_t s) {
    const int sms = device_sm_count();
    const Layout32 w = layout32(x.ws, x.N, x.q_cap, x.max_len);
    const int Weff = x.W > x.max_len - 1 ? x.max_len - 1 : x.W;
    const Margins m = make_margins(x.max_len);
    const bool exact = (x.flags & NNDTW_EXACT_DIST) != 0;
    unsigned long long *cnt = (want_stats && !timing) ? w.counters : nullptr;
    auto launched = [&](int k) {
        t_launches += k;
        t_stage_launches[t_stage] += k;
    };
    t_stage = 0;
    {
        const InitJob32 j{w.counters, w.buckets, w.bsf, w.seed, w.best64, w.rcount, w.bestidx,
                          x.Q};
        init32_kernel<Src1<InitJob32>><<<std::min<unsigned>(grid_small(std::max<int64_t>(x.Q, 64)),
                                                            64u),
                                         kSmallThreads, 0, s>>>(Src1<InitJob32>{j});
        CK(cudaGetLastError());
        launched(1);
    }
    // S1: the training envelopes, rows up to L_t + W (not past max_len)
    if (!x.train_ready) {
        EnvPlan<float> ep = plan_envelopes<float>(x.train, nullptr, x.N, x.max_len, Weff, w.env);
        ep.job.off = x.train_off;
        ep.job.E = x.max_len;
        CK(set_envelope_smem<float>(ep.one_pass, ep.smem));
        envelope_fns<float>(ep.one_pass).fn1<<<(unsigned)ep.blocks, kEnvelopeThreads, ep.smem, s>>>(
            Src1<EnvJob<float>>{ep.job});
        CK(cudaGetLastError());
        launched(1);
    }
    t_stage = 1;
    CK(tm.mark(1));
    // S2: the safe bounds of all pairs and each query's first candidate
    {
        LbVarJob j{};
        j.test = x.test; j.test_off = x.test_off; j.Q = x.Q;
        j.train = x.train; j.train_off = x.train_off; j.env = w.env; j.E = x.max_len; j.N = x.N;
        j.W = Weff; j.V = x.V; j.max_len = x.max_len;
        j.keogh = (x.flags & NNDTW_KEOGH_BOUND) ? 1 : 0; j.safe = 1;
        j.lb_lo = m.lb_lo; j.abs_slack = m.abs32;
        j.lb_out = w.lb; j.seed_keys = w.seed; j.bad = w.counters + C_BADLEN;
        CK(launch_lb_var(j, s));
        launched(1);
    }
    t_stage = 2;
    CK(tm.mark(2));
    // S4 on each query's first candidate (no abandoning); its pairs are
    // listed in the queue's storage, which the compaction fills afterwards
    DtwJob32 base{};
    base.test = x.test; base.train = x.train; base.L = x.max_len; base.W = Weff;
    base.test_off = x.test_off; base.train_off = x.train_off;
    base.dtw_lo = m.dtw_lo; base.dtw_hi = m.dtw_hi; base.abs32 = m.abs32;
    base.bsf = w.bsf; base.cand = w.cand; base.cand_count = w.counters + C_CAND;
    base.counters = cnt;
    base.group = group_from_flags(x.flags);
    if (base.group >= kRowsGroup) base.group = 0;   // (no row layout for unequal lengths)
    {
        CK(launch_seed_pairs(w.seed, x.Q, w.queue, w.counters + C_SEEDPAIRS, sms, s));
        DtwJob32 j = base;
        j.pairs = w.queue; j.count = w.counters + C_SEEDPAIRS; j.head = w.counters + C_SEEDHEAD;
        j.abandon = 0;
        j.group = dtw32_wide_group(Weff);
        Dtw32Plan pl{};
        CK(plan_dtw32_var(j, sms, &pl));
        j.lanes = pl.lanes;
        if (pl.blocks > 0) {
            pl.fn1<<<(unsigned)pl.blocks, pl.threads, pl.smem, s>>>(Src1<DtwJob32>{j});
            CK(cudaGetLastError());
        }
        launched(2);
    }
    t_stage = 3;
    CK(tm.mark(3));
    // S3: compaction against the upper bounds (pairs with a finite bound only)
    for (int pass = 0; pass < 2; pass++) {
        const dim3 gc = grid_compact(x.Q, x.N);
        CompactJob<float> j{};
        j.lb = w.lb; j.Q = x.Q; j.N = x.N; j.bsf = w.bsf; j.seed = w.seed;
        j.ubof = UbOf<float>{m.dtw_hi, m.abs32};
        j.no_prune = (x.flags & NNDTW_NO_PRUNE) ? 1 : 0;
        j.finite_only = 1;
        j.gx = (int)gc.x;
        j.scatter = pass;
        j.bcount = w.buckets; j.bcursor = w.buckets + kBuckets;
        j.qcount = w.counters + C_QUEUE; j.queue = w.queue;
        compact_kernel<float, Src1<CompactJob<float>>><<<gc.x * gc.y, kSmallThreads, 0, s>>>(
            Src1<CompactJob<float>>{j});
        CK(cudaGetLastError());
        launched(1);
    }
    t_stage = 4;
    CK(tm.mark(4));
    // S4 on the survivors, with early abandoning
    {
        DtwJob32 j = base;
        j.pairs = w.queue; j.count = w.counters + C_QUEUE; j.head = w.counters + C_HEAD;
        j.abandon = (x.flags & NNDTW_NO_ABANDON) ? 0 : 1;
        if (!(x.flags & NNDTW_NO_PRUNE)) {   // live pruning against the tightening bests
            j.lb = w.lb;
            j.lb_n = x.N;
            // the bound-nearest first candidate leaves most queued pairs to be
            // dropped live: claims of 8 wait once per 8 of them
            j.claim = 8;
        }
        Dtw32Plan pl{};
        CK(plan_dtw32_var(j, sms, &pl));
        j.lanes = pl.lanes;
        if (pl.blocks > 0) {
            pl.fn1<<<(unsigned)pl.blocks, pl.threads, pl.smem, s>>>(Src1<DtwJob32>{j});
            CK(cudaGetLastError());
        }
        launched(1);
    }
    t_stage = 5;
    CK(tm.mark(5));
    // S5: near-tie recheck in FP64 and the final argmin
    FinishJob32 f{};
    f.cand = w.cand; f.ccount = w.counters + C_CAND; f.bsf = w.bsf;
    f.lo = m.dtw_lo; f.hi = m.dtw_hi; f.abs32 = m.abs32;
    f.rcount = w.rcount; f.exact = exact ? 1 : 0; f.rlist = w.rlist;
    f.counters = w.counters; f.d64 = w.d64; f.best64 = w.best64;
    f.bestidx = w.bestidx; f.Q = x.Q; f.labels = x.labels;
    f.nn_idx = x.nn_idx; f.nn_label = x.nn_label; f.nn_dist = x.nn_dist;
    const unsigned fb = (unsigned)finish_blocks(x.Q, x.N);
    filter32_kernel<Src1<FinishJob32>><<<fb, kSmallThreads, 0, s>>>(Src1<FinishJob32>{f});
    CK(cudaGetLastError());
    collect32_kernel<Src1<FinishJob32>><<<fb, kSmallThreads, 0, s>>>(Src1<FinishJob32>{f});
    CK(cudaGetLastError());
    {
        DtwJob64 r{};
        r.test32 = x.test; r.train32 = x.train; r.L = x.max_len; r.W = Weff;
        r.test_off = x.test_off; r.train_off = x.train_off;
        r.pairs = w.rlist; r.count = w.counters + C_RECHECK; r.head = nullptr;
        r.bsf64 = w.best64; r.out = w.d64; r.abandon = 0;
        Dtw64Plan pl{};
        CK(plan_dtw64(r, sms, &pl));
        const long long want = exact ? x.Q : std::max<long long>(4, (x.Q + 7) / 8);
        const long long blocks = std::min(pl.blocks, want);
        if (blocks > 0) {
            pl.fn1<<<(unsigned)blocks, pl.threads, pl.smem, s>>>(Src1<DtwJob64>{r});
            CK(cudaGetLastError());
        }
    }
    ties32_kernel<Src1<FinishJob32>><<<fb, kSmallThreads, 0, s>>>(Src1<FinishJob32>{f});
    CK(cudaGetLastError());
    launched(4);
    t_stage = 6;
    CK(tm.mark(6));
    finalize32_kernel<Src1<FinishJob32>><<<grid_small(x.Q), kSmallThreads, 0, s>>>(
        Src1<FinishJob32>{f});
    CK(cudaGetLastError());
    launched(1);
    t_stage = 7;
    CK(tm.mark(7));
    if (stats || (x.flags & NNDTW_CHECK_FINITE)) {
        unsigned long long h[C_COUNT];
        CK(cudaMemcpyAsync(h, w.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if ((x.flags & NNDTW_CHECK_FINITE) && h[C_BADLEN]) return NNDTW_EINVAL;
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            stats->pairs = x.Q * x.N;
            stats->lb_pruned = x.Q * x.N - (int64_t)h[C_SEEDPAIRS] - (int64_t)h[C_QUEUE];
            stats->rechecked = (int64_t)h[C_RECHECK];
            stats->recheck_queries = (int64_t)h[C_RQUERIES];
            if (cnt) {
                stats->dtw_started = (int64_t)h[C_STARTED];
                stats->dtw_abandoned = (int64_t)h[C_ABANDONED];
                stats->dtw_cells = (int64_t)h[C_CELLS];
                stats->lb_pruned_live = (int64_t)h[C_LIVEPRUNED];
            }
        }
    }
    return NNDTW_OK;
}

}  // namespace

// ------------------------------------------------------------------ helpers

void set_last_cuda_error(cudaError_t e) {
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_sm_mu);
    if (dev >= 0 && dev < 64 && g_sm[dev]) return g_sm[dev];
    int n = 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 1;
    if (dev >= 0 && dev < 64) g_sm[dev] = n;
    return n;
}

static double gamma_n(double n, double u) { return n * u / (1.0 - n * u); }

static float round_down_f(double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}
static float round_up_f(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

// The FP32 values of LB and DTW carry a relative error of at most
// gamma_n(u32) with n = (number of rounded operations on the longest chain):
// at most 2L+8 for DTW (a path has at most 2L-1 cells, each one rounding for
// the difference and one for the fused multiply-add) and 2L+16 for the bounds
// (L terms, each a rounded difference and a rounded accumulation, plus the
// band minima).  A further 2^-40 covers the FP64 rounding of the exact values
// the search must reproduce.
Margins make_margins(int L) {
    const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
    const double g_lb = gamma_n(2.0 * L + 16, u32), g_dtw = gamma_n(2.0 * L + 8, u32);
    const double slack = std::ldexp(1.0, -40);
    Margins m;
    m.lb_lo = round_down_f((1.0 - g_lb) * (1.0 - slack));
    m.dtw_lo = round_down_f((1.0 - g_dtw) * (1.0 - slack));
    m.dtw_hi = round_up_f((1.0 + g_dtw) * (1.0 + slack));
    m.abs32 = std::ldexp(1.0f, -126);
    const double g64 = gamma_n(4.0 * L + 32, u64);
    m.lb_lo64 = (1.0 - 2.0 * g64) * (1.0 - 4.0 * u64);
    m.abs64 = std::ldexp(1.0, -1000);
    return m;
}

}  // namespace nndtw

using namespace nndtw;

// ====================================================================== ABI

extern "C" {

int nn_dtw_version(void) { return 106; }

int nn_dtw_stage_times(float *h_ms) {
    if (!h_ms || t_last_dev < 0) return NNDTW_EINVAL;
    EventSet &set = t_events[t_last_dev];
    CK(cudaEventSynchronize(set.ev[7]));
    for (int k = 0; k < 7; k++) CK(cudaEventElapsedTime(&h_ms[k], set.ev[k], set.ev[k + 1]));
    CK(cudaEventElapsedTime(&h_ms[7], set.ev[0], set.ev[7]));
    return NNDTW_OK;
}

const char *nn_dtw_strerror(int code) {
    switch (code) {
        case NNDTW_OK: return "ok";
        case NNDTW_EINVAL: return "invalid argument (null pointer, size or parameter out of range)";
        case NNDTW_ECUDA: return "a CUDA call failed (see nn_dtw_last_cuda_error)";
        case NNDTW_ENOSPACE: return "workspace smaller than nn_dtw_workspace_size()";
        case NNDTW_EUNSUPPORTED: return "request not supported by this build";
        case NNDTW_ENONFINITE: return "non-finite or out-of-range input value";
        default: return "unknown status code";
    }
}

const char *nn_dtw_last_cuda_error(void) { return g_cuda_err; }

long long nn_dtw_last_call_launches(void) { return t_launches; }

int nn_dtw_last_call_stage_launches(long long *h_counts) {
    if (!h_counts) return NNDTW_EINVAL;
    for (int k = 0; k < 8; k++) h_counts[k] = t_stage_launches[k];
    return NNDTW_OK;
}

int nn_dtw_build_envelopes(const float *d_train, int64_t N, int L, int W, float *d_env,
                           void *stream) {
    if (N < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (N == 0) return NNDTW_OK;
    if (!d_train || !d_env) return NNDTW_EINVAL;
    CK(launch_envelopes<float>(d_train, N, L, W, d_env, (cudaStream_t)stream));
    return NNDTW_OK;
}

int nn_dtw_build_envelopes_f64(const double *d_train, int64_t N, int L, int W, double *d_env,
                               void *stream) {
    if (N < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (N == 0) return NNDTW_OK;
    if (!d_train || !d_env) return NNDTW_EINVAL;
    CK(launch_envelopes<double>(d_train, N, L, W, d_env, (cudaStream_t)stream));
    return NNDTW_OK;
}

int nn_dtw_build_second_envelopes(const float *d_env, int64_t N, int L, int W, float *d_env2,
                                  void *stream) {
    if (N < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (N == 0) return NNDTW_OK;
    if (!d_env || !d_env2) return NNDTW_EINVAL;
    CK(launch_second_envelopes<float>(d_env, N, L, W, d_env2, (cudaStream_t)stream));
    return NNDTW_OK;
}

int nn_dtw_build_second_envelopes_f64(const double *d_env, int64_t N, int L, int W,
                                      double *d_env2, void *stream) {
    if (N < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (N == 0) return NNDTW_OK;
    if (!d_env || !d_env2) return NNDTW_EINVAL;
    CK(launch_second_envelopes<double>(d_env, N, L, W, d_env2, (cudaStream_t)stream));
    return NNDTW_OK;
}

int lb_enhanced(const float *d_test, int64_t Q, const float *d_train, const float *d_env,
                int64_t N, int L, int W, int V, unsigned flags, float *d_lb_out, void *stream) {
    if (Q < 0 || N < 0 || L < 2 || L > NNDTW_MAX_L || W < 0 || V < 1) return NNDTW_EINVAL;
    if ((flags & NNDTW_LB_KEOGH) && (flags & NNDTW_LB_NEW)) return NNDTW_EINVAL;
    if (Q == 0 || N == 0) return NNDTW_OK;
    const bool lbnew = (flags & NNDTW_LB_NEW) != 0;
    if (!d_test || !d_train || (!d_env && !lbnew) || !d_lb_out) return NNDTW_EINVAL;
    const Margins m = make_margins(L);
    if (lbnew) {
        CK(launch_lb_new<float>(d_test, Q, d_train, N, L, W, (flags & NNDTW_LB_SAFE) != 0,
                                m.lb_lo, m.abs32, d_lb_out, (cudaStream_t)stream));
        return NNDTW_OK;
    }
    CK(launch_lb<float>(d_test, Q, d_train, d_env, N, L, W, V, (flags & NNDTW_LB_KEOGH) != 0,
                        (flags & NNDTW_LB_SAFE) != 0, m.lb_lo, m.abs32, d_lb_out, nullptr,
                        nullptr, nullptr, false, (cudaStream_t)stream, 0,
                        (int)((flags & NNDTW_LB_TILE_MASK) >> 19)));
    return NNDTW_OK;
}

int lb_enhanced_f64(const double *d_test, int64_t Q, const double *d_train, const double *d_env,
                    int64_t N, int L, int W, int V, unsigned flags, double *d_lb_out,
                    void *stream) {
    if (Q < 0 || N < 0 || L < 2 || L > NNDTW_MAX_L || W < 0 || V < 1) return NNDTW_EINVAL;
    if ((flags & NNDTW_LB_KEOGH) && (flags & NNDTW_LB_NEW)) return NNDTW_EINVAL;
    if (Q == 0 || N == 0) return NNDTW_OK;
    const bool lbnew = (flags & NNDTW_LB_NEW) != 0;
    if (!d_test || !d_train || (!d_env && !lbnew) || !d_lb_out) return NNDTW_EINVAL;
    const Margins m = make_margins(L);
    if (lbnew) {
        CK(launch_lb_new<double>(d_test, Q, d_train, N, L, W, (flags & NNDTW_LB_SAFE) != 0,
                                 m.lb_lo64, m.abs64, d_lb_out, (cudaStream_t)stream));
        return NNDTW_OK;
    }
    CK(launch_lb<double>(d_test, Q, d_train, d_env, N, L, W, V, (flags & NNDTW_LB_KEOGH) != 0,
                         (flags & NNDTW_LB_SAFE) != 0, m.lb_lo64, m.abs64, d_lb_out, nullptr,
                         nullptr, nullptr, false, (cudaStream_t)stream, 0,
                        (int)((flags & NNDTW_LB_TILE_MASK) >> 19)));
    return NNDTW_OK;
}

int lb_enhanced_improved(const float *d_test, const float *d_test_env, int64_t Q,
                         const float *d_train, const float *d_env, const float *d_env2, int64_t N,
                         int L, int W, int V, unsigned flags, float *d_lb_out, void *stream) {
    if (Q < 0 || N < 0 || L < 2 || L > NNDTW_MAX_L || W < 0 || V < 1) return NNDTW_EINVAL;
    if (flags & NNDTW_LB_NEW) return NNDTW_EINVAL;
    if (Q == 0 || N == 0) return NNDTW_OK;
    if (!d_test || !d_test_env || !d_train || !d_env || !d_env2 || !d_lb_out) return NNDTW_EINVAL;
    const int rc = lb_enhanced(d_test, Q, d_train, d_env, N, L, W, V, flags, d_lb_out, stream);
    if (rc != NNDTW_OK) return rc;
    const Margins m = make_margins(L);
    // with NNDTW_LB_KEOGH the first pass is LB_Keogh over the whole series and
    // so is the second: LB_Improved itself (Sec. 2.2.4)
    const int nb = (flags & NNDTW_LB_KEOGH) ? 0 : bridge_start(L, V);
    CK(launch_improved_terms<float>(d_train, d_test_env, d_env2, Q, N, L, nb,
                                    (flags & NNDTW_LB_SAFE) != 0, m.lb_lo, m.abs32, d_lb_out,
                                    (cudaStream_t)stream));
    return NNDTW_OK;
}

int lb_enhanced_improved_f64(const double *d_test, const double *d_test_env, int64_t Q,
                             const double *d_train, const double *d_env, const double *d_env2,
                             int64_t N, int L, int W, int V, unsigned flags, double *d_lb_out,
                             void *stream) {
    if (Q < 0 || N < 0 || L < 2 || L > NNDTW_MAX_L || W < 0 || V < 1) return NNDTW_EINVAL;
    if (flags & NNDTW_LB_NEW) return NNDTW_EINVAL;
    if (Q == 0 || N == 0) return NNDTW_OK;
    if (!d_test || !d_test_env || !d_train || !d_env || !d_env2 || !d_lb_out) return NNDTW_EINVAL;
    const int rc = lb_enhanced_f64(d_test, Q, d_train, d_env, N, L, W, V, flags, d_lb_out, stream);
    if (rc != NNDTW_OK) return rc;
    const Margins m = make_margins(L);
    // with NNDTW_LB_KEOGH the first pass is LB_Keogh over the whole series and
    // so is the second: LB_Improved itself (Sec. 2.2.4)
    const int nb = (flags & NNDTW_LB_KEOGH) ? 0 : bridge_start(L, V);
    CK(launch_improved_terms<double>(d_train, d_test_env, d_env2, Q, N, L, nb,
                                     (flags & NNDTW_LB_SAFE) != 0, m.lb_lo64, m.abs64, d_lb_out,
                                     (cudaStream_t)stream));
    return NNDTW_OK;
}

int dtw_windowed(const float *d_test, const float *d_train, const int32_t *d_pairs, int64_t P,
                 int L, int W, float *d_out, void *stream) {
    return dtw_windowed_ex(d_test, d_train, d_pairs, P, L, W, 0, d_out, stream);
}


int dtw_windowed_ex(const float *d_test, const float *d_train, const int32_t *d_pairs, int64_t P,
                    int L, int W, unsigned flags, float *d_out, void *stream) {
    if (P < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (P == 0) return NNDTW_OK;
    if (!d_test || !d_train || !d_pairs || !d_out) return NNDTW_EINVAL;
    if (!dtw32_supported(W > L - 1 ? L - 1 : W)) return NNDTW_EUNSUPPORTED;
    DtwJob32 j{};
    j.test = d_test; j.train = d_train; j.L = L; j.W = W > L - 1 ? L - 1 : W;
    j.pairs = reinterpret_cast<const uint2 *>(d_pairs);
    j.n_pairs = P;
    j.out = d_out;
    j.group = group_from_flags(flags);
    const Margins m = make_margins(L);
    j.dtw_lo = m.dtw_lo; j.dtw_hi = m.dtw_hi; j.abs32 = m.abs32;
    j.head = nullptr;  // static assignment: pair count known here
    CK(launch_dtw32(j, device_sm_count(), (cudaStream_t)stream));
    return NNDTW_OK;
}

// ------------------------------------------------------- unequal lengths

static bool varlen_sizes_ok(int64_t N, int64_t Q, int max_len, int W, int V) {
    return search_sizes_ok(N, Q, max_len, W, V);
}

int nn_dtw_build_envelopes_varlen(const float *d_train, const int64_t *d_train_off, int64_t N,
                                  int max_len, int W, float *d_env, void *stream) {
    if (N < 0 || max_len < 2 || max_len > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (N == 0) return NNDTW_OK;
    if (!d_train || !d_train_off || !d_env) return NNDTW_EINVAL;
    const int Weff = W > max_len - 1 ? max_len - 1 : W;
    EnvPlan<float> ep = plan_envelopes<float>(d_train, nullptr, N, max_len, Weff, d_env);
    ep.job.off = reinterpret_cast<const long long *>(d_train_off);
    ep.job.E = max_len;
    CK(set_envelope_smem<float>(ep.one_pass, ep.smem));
    envelope_fns<float>(ep.one_pass).fn1<<<(unsigned)ep.blocks, kEnvelopeThreads, ep.smem,
                                           (cudaStream_t)stream>>>(Src1<EnvJob<float>>{ep.job});
    CK(cudaGetLastError());
    return NNDTW_OK;
}

int lb_enhanced_varlen(const float *d_test, const int64_t *d_test_off, int64_t Q,
                       const float *d_train, const int64_t *d_train_off, const float *d_env,
                       int64_t N, int max_len, int W, int V, unsigned flags, float *d_lb_out,
                       void *stream) {
    if (Q < 0 || N < 0 || max_len < 2 || max_len > NNDTW_MAX_L || W < 0 || V < 1)
        return NNDTW_EINVAL;
    if (flags & ~(unsigned)(NNDTW_LB_KEOGH | NNDTW_LB_SAFE)) return NNDTW_EINVAL;
    if (Q == 0 || N == 0) return NNDTW_OK;
    if (!d_test || !d_test_off || !d_train || !d_train_off || !d_env || !d_lb_out)
        return NNDTW_EINVAL;
    if ((double)Q * (double)((N + 63) / 64) > 2147483647.0) return NNDTW_EUNSUPPORTED;
    const Margins m = make_margins(max_len);
    LbVarJob j{};
    j.test = d_test; j.test_off = reinterpret_cast<const long long *>(d_test_off); j.Q = Q;
    j.train = d_train; j.train_off = reinterpret_cast<const long long *>(d_train_off);
    j.env = d_env; j.E = max_len; j.N = N;
    j.W = W > max_len - 1 ? max_len - 1 : W; j.V = V; j.max_len = max_len;
    j.keogh = (flags & NNDTW_LB_KEOGH) ? 1 : 0; j.safe = (flags & NNDTW_LB_SAFE) ? 1 : 0;
    j.lb_lo = m.lb_lo; j.abs_slack = m.abs32; j.lb_out = d_lb_out;
    CK(launch_lb_var(j, (cudaStream_t)stream));
    return NNDTW_OK;
}

int dtw_windowed_varlen(const float *d_test, const int64_t *d_test_off, const float *d_train,
                        const int64_t *d_train_off, const int32_t *d_pairs, int64_t P,
                        int max_len, int W, float *d_out, void *stream) {
    if (P < 0 || max_len < 1 || max_len > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (P == 0) return NNDTW_OK;
    if (!d_test || !d_test_off || !d_train || !d_train_off || !d_pairs || !d_out)
        return NNDTW_EINVAL;
    DtwJob32 j{};
    j.test = d_test; j.train = d_train; j.L = max_len; j.W = W > max_len - 1 ? max_len - 1 : W;
    j.test_off = reinterpret_cast<const long long *>(d_test_off);
    j.train_off = reinterpret_cast<const long long *>(d_train_off);
    j.pairs = reinterpret_cast<const uint2 *>(d_pairs);
    j.n_pairs = P;
    j.out = d_out;
    const Margins m = make_margins(max_len);
    j.dtw_lo = m.dtw_lo; j.dtw_hi = m.dtw_hi; j.abs32 = m.abs32;
    Dtw32Plan pl{};
    CK(plan_dtw32_var(j, device_sm_count(), &pl));
    j.lanes = pl.lanes;
    if (pl.blocks > 0) {
        pl.fn1<<<(unsigned)pl.blocks, pl.threads, pl.smem, (cudaStream_t)stream>>>(
            Src1<DtwJob32>{j});
        CK(cudaGetLastError());
    }
    return NNDTW_OK;
}

size_t nn_dtw_varlen_workspace_size(int64_t N, int64_t Q, int max_len, int W, int V) {
    if (!varlen_sizes_ok(N, Q, max_len, W, V)) return 0;
    return layout32(nullptr, N, chunk_queries(N, Q), max_len).bytes;
}

int nn_dtw_search_varlen(const float *d_train, const int64_t *d_train_off,
                         const int32_t *d_train_labels, int64_t N, const float *d_test,
                         const int64_t *d_test_off, int64_t Q, int max_len, int W, int V,
                         unsigned flags, int32_t *d_nn_idx, int32_t *d_nn_label,
                         double *d_nn_dist, void *d_workspace, size_t workspace_bytes,
                         nndtw_stats *stats, void *stream) {
    if (!varlen_sizes_ok(N, Q, max_len, W, V)) return NNDTW_EINVAL;
    if (flags & (NNDTW_LEAVE_ONE_OUT | NNDTW_REVERSE | NNDTW_IMPROVED)) return NNDTW_EINVAL;
    if (Q == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return NNDTW_OK;
    }
    if (!d_train || !d_train_off || !d_train_labels || !d_test || !d_test_off || !d_nn_idx ||
        !d_nn_label || !d_nn_dist || !d_workspace)
        return NNDTW_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255u) return NNDTW_EINVAL;
    const int64_t qc = chunk_queries(N, Q);
    const Layout32 ws = layout32(d_workspace, N, qc, max_len);
    if (workspace_bytes < ws.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const long long *toff = reinterpret_cast<const long long *>(d_test_off);
    const long long *off = reinterpret_cast<const long long *>(d_train_off);
    reset_launch_counts();
    if (flags & NNDTW_CHECK_FINITE) {
        // value counts from the offset tables' last entries (waits for the stream)
        long long tot[2] = {0, 0};
        CK(cudaMemcpyAsync(&tot[0], off + N, sizeof(long long), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&tot[1], toff + Q, sizeof(long long), cudaMemcpyDeviceToHost, s));
        CK(cudaMemsetAsync(ws.counters + C_BAD, 0, sizeof(unsigned long long), s));
        CK(cudaStreamSynchronize(s));
        if (tot[0] < 0 || tot[1] < 0) return NNDTW_EINVAL;
        int rc = check_finite<float>(d_train, tot[0], 1e15f, ws.counters + C_BAD, s);
        if (rc) return rc;
        rc = check_finite<float>(d_test, tot[1], 1e15f, ws.counters + C_BAD, s);
        if (rc) return rc;
        unsigned long long bad = 0;
        CK(cudaMemcpyAsync(&bad, ws.counters + C_BAD, sizeof(bad), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad) return NNDTW_ENONFINITE;
    }
    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    StageTimer tm;
    CK(tm.start(timing, s));
    nndtw_stats total{};
    for (int64_t q0 = 0; q0 < Q; q0 += qc) {
        const int64_t m = Q - q0 < qc ? Q - q0 : qc;
        SetVar x{};
        x.train = d_train; x.train_off = off; x.labels = d_train_labels; x.N = N;
        x.test = d_test; x.test_off = toff + q0; x.Q = m;
        x.max_len = max_len; x.W = W; x.V = V; x.flags = flags;
        x.nn_idx = d_nn_idx + q0; x.nn_label = d_nn_label + q0; x.nn_dist = d_nn_dist + q0;
        x.ws = d_workspace; x.q_cap = qc; x.train_ready = q0 > 0;
        nndtw_stats part{};
        const int rc = run_var(x, stats != nullptr, timing, stats ? &part : nullptr, tm, s);
        if (rc != NNDTW_OK) return rc;
        if (stats) add_stats(&total, part);
    }
    if (stats) *stats = total;
    return NNDTW_OK;
}

int dtw_windowed_f64(const double *d_test, const double *d_train, const int32_t *d_pairs,
                     int64_t P, int L, int W, double *d_out, void *stream) {
    if (P < 0 || L < 1 || L > NNDTW_MAX_L || W < 0) return NNDTW_EINVAL;
    if (P == 0) return NNDTW_OK;
    if (!d_test || !d_train || !d_pairs || !d_out) return NNDTW_EINVAL;
    DtwJob64 j{};
    j.test = d_test; j.train = d_train; j.L = L; j.W = W > L - 1 ? L - 1 : W;
    j.pairs = reinterpret_cast<const uint2 *>(d_pairs);
    j.n_pairs = P;
    j.out = d_out;
    j.head = nullptr;
    CK(launch_dtw64(j, device_sm_count(), (cudaStream_t)stream));
    return NNDTW_OK;
}

size_t nn_dtw_workspace_size(int64_t N, int64_t Q, int L, int W, int V, int fp64) {
    if (!search_sizes_ok(N, Q, L, W, V)) return 0;
    const int64_t qc = chunk_queries(N, Q);
    return fp64 ? layout64(nullptr, N, qc, L).bytes : layout32(nullptr, N, qc, L).bytes;
}

int nn_dtw_search(const float *d_train, const int32_t *d_train_labels, int64_t N,
                  const float *d_test, int64_t Q, int L, int W, int V, const float *d_env,
                  unsigned flags, int32_t *d_nn_idx, int32_t *d_nn_label, double *d_nn_dist,
                  void *d_workspace, size_t workspace_bytes, nndtw_stats *stats, void *stream) {
    if (!search_sizes_ok(N, Q, L, W, V)) return NNDTW_EINVAL;
    if ((flags & NNDTW_LEAVE_ONE_OUT) && (Q != N || N < 2)) return NNDTW_EINVAL;
    if (Q == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return NNDTW_OK;
    }
    if (!d_train || !d_train_labels || !d_test || !d_nn_idx || !d_nn_label || !d_nn_dist ||
        !d_workspace)
        return NNDTW_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255u) return NNDTW_EINVAL;
    if (!dtw32_supported(W > L - 1 ? L - 1 : W)) return NNDTW_EUNSUPPORTED;
    const int64_t qc = chunk_queries(N, Q);
    if (workspace_bytes < layout32(nullptr, N, qc, L).bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    reset_launch_counts();
    StageTimer tm;
    CK(tm.start(timing, s));
    nndtw_stats total{};
    for (int64_t q0 = 0; q0 < Q; q0 += qc) {
        const int64_t m = Q - q0 < qc ? Q - q0 : qc;
        const Set32 set{d_train, d_train_labels, N, d_test + q0 * L, m, L, W, V, d_env, flags,
                        d_nn_idx + q0, d_nn_label + q0, d_nn_dist + q0, d_workspace, q0, qc,
                        q0 > 0};
        nndtw_stats part{};
        const int rc = run32(&set, 1, stats != nullptr, timing, stats ? &part : nullptr, tm, s);
        if (rc != NNDTW_OK) return rc;
        if (stats) add_stats(&total, part);
    }
    if (stats) *stats = total;
    return NNDTW_OK;
}

int nn_dtw_search_f64(const double *d_train, const int32_t *d_train_labels, int64_t N,
                      const double *d_test_all, int64_t Q_all, int L, int W, int V,
                      const double *d_env, unsigned flags, int32_t *d_nn_idx_all,
                      int32_t *d_nn_label_all, double *d_nn_dist_all, void *d_workspace,
                      size_t workspace_bytes, nndtw_stats *stats, void *stream) {
    if (!search_sizes_ok(N, Q_all, L, W, V)) return NNDTW_EINVAL;
    if ((flags & NNDTW_LEAVE_ONE_OUT) && (Q_all != N || N < 2)) return NNDTW_EINVAL;
    if (Q_all == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return NNDTW_OK;
    }
    if (!d_train || !d_train_labels || !d_test_all || !d_nn_idx_all || !d_nn_label_all ||
        !d_nn_dist_all || !d_workspace)
        return NNDTW_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255u) return NNDTW_EINVAL;
    // queries in chunks of at most NNDTW_CHUNK_PAIRS pairs, one layout for all
    const int64_t qc = chunk_queries(N, Q_all);
    const Layout64 ws = layout64(d_workspace, N, qc, L);
    if (workspace_bytes < ws.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int Weff = W > L - 1 ? L - 1 : W;
    const Margins m = make_margins(L);
    const int sms = device_sm_count();

    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    StageTimer tm;
    CK(tm.start(timing, s));
    if (flags & NNDTW_CHECK_FINITE) {
        CK(cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * C_COUNT, s));
        int rc = check_finite<double>(d_train, N * L, 1e150, ws.counters + C_BAD, s);
        if (rc) return rc;
        rc = check_finite<double>(d_test_all, Q_all * L, 1e150, ws.counters + C_BAD, s);
        if (rc) return rc;
        unsigned long long bad = 0;
        CK(cudaMemcpyAsync(&bad, ws.counters + C_BAD, sizeof(bad), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad) return NNDTW_ENONFINITE;
    }
    const bool keogh = (flags & NNDTW_KEOGH_BOUND) != 0;
    const bool rev = !keogh && !(flags & (NNDTW_NO_PRUNE | NNDTW_NO_REVERSE));
    const bool imp = (flags & NNDTW_IMPROVED) && !keogh && !(flags & NNDTW_NO_PRUNE);
    const double *env = d_env ? d_env : ws.env;
    nndtw_stats total{};
    for (int64_t q0 = 0; q0 < Q_all; q0 += qc) {
        const int64_t Q = Q_all - q0 < qc ? Q_all - q0 : qc;
        const double *d_test = d_test_all + q0 * L;
        int32_t *d_nn_idx = d_nn_idx_all + q0, *d_nn_label = d_nn_label_all + q0;
        double *d_nn_dist = d_nn_dist_all + q0;
        CK(cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * C_COUNT, s));
        CK(cudaMemsetAsync(ws.buckets, 0, sizeof(unsigned long long) * 2 * kBuckets, s));
        CK(cudaMemsetAsync(ws.bsf64, 0x7f, sizeof(unsigned long long) * Q, s));
        CK(cudaMemsetAsync(ws.seed, 0xff, sizeof(unsigned long long) * Q, s));
        CK(cudaMemsetAsync(ws.bestidx, 0x7f, sizeof(int32_t) * Q, s));
        // the training side once, in the first chunk
        if (q0 == 0 && !d_env) CK(launch_envelopes<double>(d_train, N, L, Weff, ws.env, s));
        if (rev || imp) CK(launch_envelopes<double>(d_test, Q, L, Weff, ws.envq, s));
        if (q0 == 0 && imp) CK(launch_second_envelopes<double>(env, N, L, Weff, ws.env2, s));
        CK(tm.mark(1));
        CK(launch_lb<double>(d_test, Q, d_train, env, N, L, Weff, V, keogh, true, m.lb_lo64,
                             m.abs64, ws.lb, ws.seed, ws.norms, rev ? ws.ends : nullptr,
                             (flags & NNDTW_LEAVE_ONE_OUT) != 0, s, q0));
        CK(tm.mark(2));
        unsigned long long *cnt = (stats && !timing) ? ws.counters : nullptr;
        DtwJob64 j{};
        j.test = d_test; j.train = d_train; j.L = L; j.W = Weff;
        j.bsf64 = ws.bsf64; j.cand = ws.cand; j.cand_count = ws.counters + C_CAND;
        j.counters = cnt;
        j.pairs = nullptr; j.seed_keys = ws.seed; j.n_pairs = Q; j.head = nullptr; j.abandon = 0;
        CK(launch_dtw64(j, sms, s));
        CK(tm.mark(3));
        {
            const dim3 gc = grid_compact(Q, N);
            CompactJob<double> cj{};
            cj.lb = ws.lb; cj.Q = Q; cj.N = N; cj.bsf = ws.bsf64; cj.seed = ws.seed;
            cj.ubof = UbOf<double>{};
            cj.no_prune = (flags & NNDTW_NO_PRUNE) ? 1 : 0;
            cj.gx = (int)gc.x;
            cj.bcount = ws.buckets; cj.bcursor = ws.buckets + kBuckets;
            cj.qcount = ws.counters + C_QUEUE; cj.queue = ws.queue;
            for (int pass = 0; pass < 2; pass++) {
                cj.scatter = pass;
                compact_kernel<double, Src1<CompactJob<double>>>
                    <<<gc.x * gc.y, kSmallThreads, 0, s>>>(Src1<CompactJob<double>>{cj});
                CK(cudaGetLastError());
            }
        }
        CK(tm.mark(4));
        j.pairs = ws.queue; j.seed_keys = nullptr; j.count = ws.counters + C_QUEUE;
        j.head = ws.counters + C_HEAD; j.abandon = (flags & NNDTW_NO_ABANDON) ? 0 : 1;
        if (rev || imp) {
            j.envq = reinterpret_cast<const double2 *>(ws.envq);
            j.rev = rev;
            j.ends_bands = ws.ends;
            j.env2 = imp ? reinterpret_cast<const double2 *>(ws.env2) : nullptr;
            j.lb = ws.lb;
            j.N = N;
            j.nb = bridge_start(L, V);
            j.lb_lo = m.lb_lo64;
            j.lb_abs = m.abs64;
        }
        CK(launch_dtw64(j, sms, s));
        CK(tm.mark(5));
        const long long cap = (long long)Q * N + Q;
        ties64_kernel<<<grid_small(cap), kSmallThreads, 0, s>>>(ws.cand, ws.counters + C_CAND,
                                                                ws.bsf64, ws.bestidx);
        CK(cudaGetLastError());
        CK(tm.mark(6));
        finalize64_kernel<<<grid_small(Q), kSmallThreads, 0, s>>>(Q, ws.bsf64, ws.bestidx,
                                                                  d_train_labels, d_nn_idx,
                                                                  d_nn_label, d_nn_dist);
        CK(cudaGetLastError());
        CK(tm.mark(7));
        if (stats) {
            unsigned long long h[C_COUNT];
            CK(cudaMemcpyAsync(h, ws.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            nndtw_stats part{};
            fill_stats(&part, h, N, Q, L, Weff, cnt != nullptr);
            add_stats(&total, part);
        }
    }
    if (stats) *stats = total;
    return NNDTW_OK;
}


size_t nn_dtw_batch_workspace_size(const nndtw_dataset *h_sets, int n) {
    if (!h_sets || n < 0) return 0;
    size_t tot = 256;
    for (int i = 0; i < n; i++) {
        const nndtw_dataset &d = h_sets[i];
        const size_t b = nn_dtw_workspace_size(d.N, d.Q, d.L, d.W, d.V, 0);
        if (b == 0) return 0;
        tot += (b + 255) & ~size_t(255);
    }
    return tot;
}

int nn_dtw_search_batched(const nndtw_dataset *h_sets, int n, void *d_workspace,
                          size_t workspace_bytes, unsigned flags, void *stream) {
    if (n < 0 || (n > 0 && !h_sets)) return NNDTW_EINVAL;
    if (n == 0) return NNDTW_OK;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return NNDTW_EINVAL;
    // round r holds chunk r of every dataset that has one (datasets whose
    // Q x N exceeds NNDTW_CHUNK_PAIRS have several; a dataset's chunks share
    // its workspace, so they run in successive rounds)
    std::vector<std::vector<Set32>> rounds;
    size_t off = 0;
    for (int i = 0; i < n; i++) {
        const nndtw_dataset &d = h_sets[i];
        const size_t b = nn_dtw_workspace_size(d.N, d.Q, d.L, d.W, d.V, 0);
        if (b == 0) return NNDTW_EINVAL;
        const unsigned f = (flags | d.flags) & ~NNDTW_TIME_STAGES;
        if ((f & NNDTW_LEAVE_ONE_OUT) && (d.Q != d.N || d.N < 2)) return NNDTW_EINVAL;
        if (d.Q > 0 && (!d.d_train || !d.d_train_labels || !d.d_test || !d.d_nn_idx ||
                        !d.d_nn_label || !d.d_nn_dist))
            return NNDTW_EINVAL;
        if (!dtw32_supported(d.W > d.L - 1 ? d.L - 1 : d.W)) return NNDTW_EUNSUPPORTED;
        const int64_t qc = d.Q > 0 ? chunk_queries(d.N, d.Q) : 0;
        for (int64_t q0 = 0, r = 0; q0 < d.Q; q0 += qc, r++) {
            const int64_t m = d.Q - q0 < qc ? d.Q - q0 : qc;
            if ((int64_t)rounds.size() <= r) rounds.resize(r + 1);
            rounds[r].push_back(Set32{d.d_train, d.d_train_labels, d.N, d.d_test + q0 * d.L, m,
                                      d.L, d.W, d.V, d.d_env, f, d.d_nn_idx + q0,
                                      d.d_nn_label + q0, d.d_nn_dist + q0,
                                      static_cast<char *>(d_workspace) + off, q0, qc, q0 > 0});
        }
        off += (b + 255) & ~size_t(255);
    }
    if (workspace_bytes < off) return NNDTW_ENOSPACE;
    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    if (timing && (rounds.size() > 1 || (!rounds.empty() && rounds[0].size() > (size_t)kMaxSets)))
        return NNDTW_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    reset_launch_counts();
    StageTimer tm;
    CK(tm.start(timing, s));
    for (auto &sets : rounds) {
        // the datasets with the most DTW work first (the order of the groups
        // of 64 and of the stages run32 does not reorder by a CTA's cost)
        std::stable_sort(sets.begin(), sets.end(), [](const Set32 &a, const Set32 &b) {
            const double wa = (double)a.N * a.Q * band_cells(a.L, a.W);
            const double wb = (double)b.N * b.Q * band_cells(b.L, b.W);
            return wa > wb;
        });
        for (size_t k = 0; k < sets.size(); k += kMaxSets) {
            const int m = (int)std::min<size_t>(kMaxSets, sets.size() - k);
            const int rc = run32(sets.data() + k, m, false, timing, nullptr, tm, s);
            if (rc != NNDTW_OK) return rc;
        }
    }
    return NNDTW_OK;
}

namespace {
struct HostLayout {
    float *train, *test;
    int32_t *labels, *idx, *lab;
    double *dist;
    void *ws;
    size_t ws_bytes, bytes;
};
HostLayout host_layout(void *base, int64_t N, int64_t Q, int L, int W, int V) {
    Carve c(base);
    HostLayout h;
    h.train = c.take<float>((size_t)N * L);
    h.test = c.take<float>((size_t)Q * L);
    h.labels = c.take<int32_t>(N);
    h.idx = c.take<int32_t>(Q);
    h.lab = c.take<int32_t>(Q);
    h.dist = c.take<double>(Q);
    h.ws_bytes = nn_dtw_workspace_size(N, Q, L, W, V, 0);
    h.ws = c.take<unsigned char>(h.ws_bytes);
    h.bytes = c.off + 256;
    return h;
}
}  // namespace

size_t nn_dtw_host_buffer_size(int64_t N, int64_t Q, int L, int W, int V) {
    if (!search_sizes_ok(N, Q, L, W, V)) return 0;
    return host_layout(nullptr, N, Q, L, W, V).bytes;
}

int nn_dtw_search_host(const float *h_train, const int32_t *h_train_labels, int64_t N,
                       const float *h_test, int64_t Q, int L, int W, int V, unsigned flags,
                       int32_t *h_nn_idx, int32_t *h_nn_label, double *h_nn_dist,
                       void *d_buffer, size_t buffer_bytes, nndtw_stats *stats, void *stream) {
    if (!search_sizes_ok(N, Q, L, W, V)) return NNDTW_EINVAL;
    if (Q == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return NNDTW_OK;
    }
    if (!h_train || !h_train_labels || !h_test || !h_nn_idx || !h_nn_label || !h_nn_dist ||
        !d_buffer)
        return NNDTW_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_buffer) & 255u) return NNDTW_EINVAL;
    const HostLayout h = host_layout(d_buffer, N, Q, L, W, V);
    if (buffer_bytes < h.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h.train, h_train, sizeof(float) * N * L, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.test, h_test, sizeof(float) * Q * L, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.labels, h_train_labels, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    int rc = nn_dtw_search(h.train, h.labels, N, h.test, Q, L, W, V, nullptr, flags, h.idx, h.lab,
                           h.dist, h.ws, h.ws_bytes, stats, stream);
    if (rc != NNDTW_OK) return rc;
    CK(cudaMemcpyAsync(h_nn_idx, h.idx, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_nn_label, h.lab, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_nn_dist, h.dist, sizeof(double) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NNDTW_OK;
}

namespace {
// Device buffer of nn_dtw_search_varlen_host: the ragged sets (values and
// offsets), labels, outputs, then the search's workspace.
struct VarHostLayout {
    float *train, *test;
    int64_t *train_off, *test_off;
    int32_t *labels, *idx, *lab;
    double *dist;
    void *ws;
    size_t ws_bytes, bytes;
};
VarHostLayout var_host_layout(void *base, int64_t N, int64_t n_train_values, int64_t Q,
                              int64_t n_test_values, int max_len, int W, int V) {
    Carve c(base);
    VarHostLayout h;
    h.train = c.take<float>((size_t)n_train_values);
    h.test = c.take<float>((size_t)n_test_values);
    h.train_off = c.take<int64_t>((size_t)N + 1);
    h.test_off = c.take<int64_t>((size_t)Q + 1);
    h.labels = c.take<int32_t>(N);
    h.idx = c.take<int32_t>(Q);
    h.lab = c.take<int32_t>(Q);
    h.dist = c.take<double>(Q);
    h.ws_bytes = nn_dtw_varlen_workspace_size(N, Q, max_len, W, V);
    h.ws = c.take<unsigned char>(h.ws_bytes);
    h.bytes = c.off + 256;
    return h;
}

// Offsets start at 0, never decrease, and every length lies in [2, max_len].
bool host_offsets_ok(const int64_t *off, int64_t n, int max_len) {
    if (off[0] != 0) return false;
    for (int64_t k = 0; k < n; k++) {
        const int64_t len = off[k + 1] - off[k];
        if (len < 2 || len > max_len) return false;
    }
    return true;
}
}  // namespace

size_t nn_dtw_varlen_host_buffer_size(const int64_t *h_train_off, int64_t N,
                                      const int64_t *h_test_off, int64_t Q, int max_len, int W,
                                      int V) {
    if (!varlen_sizes_ok(N, Q, max_len, W, V) || !h_train_off || !h_test_off) return 0;
    return var_host_layout(nullptr, N, h_train_off[N], Q, h_test_off[Q], max_len, W, V).bytes;
}

int nn_dtw_search_varlen_host(const float *h_train, const int64_t *h_train_off,
                              const int32_t *h_train_labels, int64_t N, const float *h_test,
                              const int64_t *h_test_off, int64_t Q, int max_len, int W, int V,
                              unsigned flags, int32_t *h_nn_idx, int32_t *h_nn_label,
                              double *h_nn_dist, void *d_buffer, size_t buffer_bytes,
                              nndtw_stats *stats, void *stream) {
    if (!varlen_sizes_ok(N, Q, max_len, W, V)) return NNDTW_EINVAL;
    if (Q == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return NNDTW_OK;
    }
    if (!h_train || !h_train_off || !h_train_labels || !h_test || !h_test_off || !h_nn_idx ||
        !h_nn_label || !h_nn_dist || !d_buffer)
        return NNDTW_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_buffer) & 255u) return NNDTW_EINVAL;
    if (!host_offsets_ok(h_train_off, N, max_len) || !host_offsets_ok(h_test_off, Q, max_len))
        return NNDTW_EINVAL;
    const int64_t nt = h_train_off[N], nq = h_test_off[Q];
    const VarHostLayout h = var_host_layout(d_buffer, N, nt, Q, nq, max_len, W, V);
    if (buffer_bytes < h.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h.train, h_train, sizeof(float) * nt, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.train_off, h_train_off, sizeof(int64_t) * (N + 1),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.test, h_test, sizeof(float) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.test_off, h_test_off, sizeof(int64_t) * (Q + 1),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h.labels, h_train_labels, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    int rc = nn_dtw_search_varlen(h.train, h.train_off, h.labels, N, h.test, h.test_off, Q,
                                  max_len, W, V, flags, h.idx, h.lab, h.dist, h.ws, h.ws_bytes,
                                  stats, stream);
    if (rc != NNDTW_OK) return rc;
    CK(cudaMemcpyAsync(h_nn_idx, h.idx, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_nn_label, h.lab, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_nn_dist, h.dist, sizeof(double) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return NNDTW_OK;
}

namespace {
// Device buffer of nn_dtw_search_batched_host: every dataset's inputs and
// outputs, then the batched search's workspace.
struct HostBatchLayout {
    std::vector<nndtw_dataset> dev;
    size_t ws_off, ws_bytes, bytes;
};
bool host_batch_layout(const nndtw_host_dataset *h, int n, void *base, HostBatchLayout *lay) {
    Carve c(base);
    lay->dev.resize(n);
    for (int i = 0; i < n; i++) {
        const nndtw_host_dataset &x = h[i];
        if (!search_sizes_ok(x.N, x.Q, x.L, x.W, x.V)) return false;
        nndtw_dataset &d = lay->dev[i];
        d = nndtw_dataset{};
        d.d_train = c.take<float>((size_t)x.N * x.L);
        d.d_train_labels = c.take<int32_t>(x.N);
        d.N = x.N;
        d.d_test = c.take<float>((size_t)x.Q * x.L);
        d.Q = x.Q;
        d.L = x.L; d.W = x.W; d.V = x.V;
        d.d_env = nullptr;
        d.d_nn_idx = c.take<int32_t>(x.Q);
        d.d_nn_label = c.take<int32_t>(x.Q);
        d.d_nn_dist = c.take<double>(x.Q);
        d.flags = x.flags;
    }
    lay->ws_bytes = nn_dtw_batch_workspace_size(lay->dev.data(), n);
    if (lay->ws_bytes == 0) return false;
    lay->ws_off = (c.off + 255) & ~size_t(255);
    lay->bytes = lay->ws_off + lay->ws_bytes + 256;
    return true;
}
}  // namespace

size_t nn_dtw_batch_host_buffer_size(const nndtw_host_dataset *h_sets, int n) {
    if (!h_sets || n < 1) return 0;
    HostBatchLayout lay;
    return host_batch_layout(h_sets, n, nullptr, &lay) ? lay.bytes : 0;
}

int nn_dtw_search_batched_host(const nndtw_host_dataset *h_sets, int n, void *d_buffer,
                               size_t buffer_bytes, unsigned flags, void *stream) {
    if (n < 0 || (n > 0 && !h_sets)) return NNDTW_EINVAL;
    if (n == 0) return NNDTW_OK;
    if (!d_buffer || (reinterpret_cast<uintptr_t>(d_buffer) & 255u)) return NNDTW_EINVAL;
    if (flags & NNDTW_TIME_STAGES) return NNDTW_EINVAL;
    for (int i = 0; i < n; i++) {
        const nndtw_host_dataset &x = h_sets[i];
        if (x.Q > 0 && (!x.h_train || !x.h_train_labels || !x.h_test || !x.h_nn_idx ||
                        !x.h_nn_label || !x.h_nn_dist))
            return NNDTW_EINVAL;
    }
    HostBatchLayout lay;
    if (!host_batch_layout(h_sets, n, d_buffer, &lay)) return NNDTW_EINVAL;
    if (buffer_bytes < lay.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n; i++) {
        const nndtw_host_dataset &x = h_sets[i];
        const nndtw_dataset &d = lay.dev[i];
        if (x.Q == 0) continue;
        CK(cudaMemcpyAsync(const_cast<float *>(d.d_train), x.h_train, sizeof(float) * x.N * x.L,
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<int32_t *>(d.d_train_labels), x.h_train_labels,
                           sizeof(int32_t) * x.N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(const_cast<float *>(d.d_test), x.h_test, sizeof(float) * x.Q * x.L,
                           cudaMemcpyHostToDevice, s));
    }
    const int rc = nn_dtw_search_batched(lay.dev.data(), n,
                                         static_cast<char *>(d_buffer) + lay.ws_off, lay.ws_bytes,
                                         flags, stream);
    if (rc != NNDTW_OK) return rc;
    for (int i = 0; i < n; i++) {
        const nndtw_host_dataset &x = h_sets[i];
        const nndtw_dataset &d = lay.dev[i];
        if (x.Q == 0) continue;
        CK(cudaMemcpyAsync(x.h_nn_idx, d.d_nn_idx, sizeof(int32_t) * x.Q, cudaMemcpyDeviceToHost,
                           s));
        CK(cudaMemcpyAsync(x.h_nn_label, d.d_nn_label, sizeof(int32_t) * x.Q,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(x.h_nn_dist, d.d_nn_dist, sizeof(double) * x.Q, cudaMemcpyDeviceToHost,
                           s));
    }
    CK(cudaStreamSynchronize(s));
    return NNDTW_OK;
}

}  // extern "C"
