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
#include <cstdio>
#include <cstring>
#include <mutex>

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
// DTW kernel (longest-processing-time-first scheduling).  The queue then holds
// bucket 0, bucket 1, ...; within a bucket the order is arbitrary.
constexpr int kBuckets = 8;

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

template <typename T>
__global__ void __launch_bounds__(256)
compact_kernel(const T *__restrict__ lb, int64_t Q, int64_t N,
               const unsigned long long *__restrict__ bsf,
               const unsigned long long *__restrict__ seed, UbOf<T> ubof, int no_prune,
               int scatter, unsigned long long *__restrict__ bcount,
               unsigned long long *__restrict__ bcursor, uint2 *__restrict__ queue,
               unsigned long long *__restrict__ qcount) {
    __shared__ unsigned long long boff[kBuckets];
    __shared__ unsigned int scount[kBuckets];
    __shared__ unsigned long long sbase[kBuckets];
    const int tid = threadIdx.x;
    if (tid < kBuckets) {
        scount[tid] = 0;
        if (scatter) {
            unsigned long long o = 0;
            for (int k = 0; k < tid; k++) o += bcount[k];
            boff[tid] = o;
            if (tid == kBuckets - 1 && blockIdx.x == 0 && blockIdx.y == 0)
                *qcount = o + bcount[kBuckets - 1];
        }
    }
    __syncthreads();
    // each round covers kCompactE * 256 consecutive pairs of a row; element e
    // of thread tid is t0 + e * 256 + tid (coalesced loads)
    constexpr int E = kCompactE;
    for (int64_t q = blockIdx.y; q < Q; q += gridDim.y) {
        const T ub = ubof(bsf[q]);
        const T inv = ub > T(0) && ub < inf_of<T>() ? T(kBuckets) / ub : T(0);
        const uint32_t st = key_idx(seed[q]);
        const T *row = lb + q * N;
        for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x * E; t0 < N;
             t0 += (int64_t)gridDim.x * blockDim.x * E) {
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
                    keep = (no_prune ? v < inf_of<T>() : v <= ub) && (uint32_t)t != st;
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

__global__ void filter32_kernel(const Cand *__restrict__ cand, const unsigned long long *ccount,
                                const unsigned long long *__restrict__ bsf, float lo, float hi,
                                float abs32, int32_t *__restrict__ rcount) {
    const long long n = (long long)*ccount;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Cand e = cand[i];
        if (in_recheck_set(e, bsf[e.q], lo, hi, abs32)) atomicAdd(rcount + e.q, 1);
    }
}

__global__ void collect32_kernel(const Cand *__restrict__ cand, const unsigned long long *ccount,
                                 const unsigned long long *__restrict__ bsf, float lo, float hi,
                                 float abs32, const int32_t *__restrict__ rcount, int exact,
                                 uint2 *__restrict__ rlist, unsigned long long *counters) {
    const long long n = (long long)*ccount;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Cand e = cand[i];
        const unsigned long long kb = bsf[e.q];
        if (!in_recheck_set(e, kb, lo, hi, abs32)) continue;
        const int rc = rcount[e.q];
        if (!(exact || rc >= 2)) continue;
        const unsigned long long slot = atomicAdd(counters + C_RECHECK, 1ull);
        rlist[slot] = make_uint2((uint32_t)e.q, (uint32_t)e.t);
        if ((uint32_t)e.t == key_idx(kb)) atomicAdd(counters + C_RQUERIES, 1ull);
    }
}

__global__ void ties32_kernel(const uint2 *__restrict__ rlist, const unsigned long long *rcnt,
                              const double *__restrict__ d64,
                              const unsigned long long *__restrict__ best64,
                              int32_t *__restrict__ bestidx) {
    const long long n = (long long)*rcnt;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint2 e = rlist[i];
        if (dbits(d64[i]) == best64[e.x]) atomicMin(bestidx + e.x, (int32_t)e.y);
    }
}

__global__ void finalize32_kernel(int64_t Q, const unsigned long long *__restrict__ bsf,
                                  const int32_t *__restrict__ rcount,
                                  const unsigned long long *__restrict__ best64,
                                  const int32_t *__restrict__ bestidx, int exact,
                                  const int32_t *__restrict__ labels, int32_t *__restrict__ nn_idx,
                                  int32_t *__restrict__ nn_label, double *__restrict__ nn_dist) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q;
         q += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long kb = bsf[q];
        int32_t idx;
        double dist;
        if (exact || rcount[q] >= 2) {
            idx = bestidx[q];
            dist = __longlong_as_double((long long)best64[q]);
        } else {
            idx = (int32_t)key_idx(kb);
            dist = (double)key_dist(kb);
        }
        nn_idx[q] = idx;
        nn_label[q] = labels[idx];
        nn_dist[q] = dist;
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
    if ((double)N * (double)Q >= 2147483648.0) return false;
    return true;
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
    long long gy = Q < 65535 ? Q : 65535;
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
    }
}

template <typename T>
int check_finite(const T *x, int64_t n, T limit, unsigned long long *bad, cudaStream_t s) {
    if (n <= 0) return NNDTW_OK;
    finite_check_kernel<T><<<grid_small(n), kSmallThreads, 0, s>>>(x, n, limit, bad);
    CK(cudaGetLastError());
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

int nn_dtw_version(void) { return 104; }

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
                        nullptr, nullptr, false, (cudaStream_t)stream));
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
                         nullptr, nullptr, false, (cudaStream_t)stream));
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

static int group_from_flags(unsigned flags) {
    const unsigned v = (flags & NNDTW_DTW_GROUP_MASK) >> 8;
    if (v == 7) {
        const unsigned lanes = (flags & NNDTW_DTW_ROWS_LANES_MASK) >> 12;
        return kRowsGroup + (lanes <= 2 ? (int)lanes : 0);
    }
    return v ? 1 << (v - 1) : 0;
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
    return fp64 ? layout64(nullptr, N, Q, L).bytes : layout32(nullptr, N, Q, L).bytes;
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
    const Layout32 ws = layout32(d_workspace, N, Q, L);
    if (workspace_bytes < ws.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int Weff = W > L - 1 ? L - 1 : W;
    const Margins m = make_margins(L);
    const int sms = device_sm_count();
    const int exact = (flags & NNDTW_EXACT_DIST) ? 1 : 0;

    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    StageTimer tm;
    CK(tm.start(timing, s));
    CK(cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * C_COUNT, s));
    CK(cudaMemsetAsync(ws.buckets, 0, sizeof(unsigned long long) * 2 * kBuckets, s));
    CK(cudaMemsetAsync(ws.bsf, 0xff, sizeof(unsigned long long) * Q, s));
    CK(cudaMemsetAsync(ws.seed, 0xff, sizeof(unsigned long long) * Q, s));
    CK(cudaMemsetAsync(ws.best64, 0xff, sizeof(unsigned long long) * Q, s));
    CK(cudaMemsetAsync(ws.rcount, 0, sizeof(int32_t) * Q, s));
    CK(cudaMemsetAsync(ws.bestidx, 0x7f, sizeof(int32_t) * Q, s));

    if (flags & NNDTW_CHECK_FINITE) {
        int rc = check_finite<float>(d_train, N * L, 1e15f, ws.counters + C_BAD, s);
        if (rc) return rc;
        rc = check_finite<float>(d_test, Q * L, 1e15f, ws.counters + C_BAD, s);
        if (rc) return rc;
        unsigned long long bad = 0;
        CK(cudaMemcpyAsync(&bad, ws.counters + C_BAD, sizeof(bad), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad) return NNDTW_ENONFINITE;
    }

    const float *env = d_env;
    if (!env) {
        CK(launch_envelopes<float>(d_train, N, L, Weff, ws.env, s));
        env = ws.env;
    }
    // the query envelopes, for the reverse bound LB_Enhanced(B, A) (asked for
    // with NNDTW_REVERSE: whether reading every surviving pair's training
    // series once more pays off depends on the data, so the tuner decides)
    // (LB_Keogh as the bound, NNDTW_KEOGH_BOUND, has no second stage)
    const bool keogh = (flags & NNDTW_KEOGH_BOUND) != 0;
    const bool rev = (flags & NNDTW_REVERSE) && !keogh &&
                     !(flags & (NNDTW_NO_PRUNE | NNDTW_NO_REVERSE));
    // and the training series' second envelopes, for the bound with the
    // LB_Improved bridge (asked for with NNDTW_IMPROVED, also a tuning choice)
    const bool imp = (flags & NNDTW_IMPROVED) && !keogh && !(flags & NNDTW_NO_PRUNE);
    if (rev || imp) CK(launch_envelopes<float>(d_test, Q, L, Weff, ws.envq, s));
    if (imp) {
        CK(launch_second_envelopes<float>(env, N, L, Weff, ws.env2, s));
        CK(launch_pack_bgap(d_train, ws.env2, N * L, s));
    }
    CK(tm.mark(1));
    // S2: safe bounds, and per query the Euclidean-nearest series (first candidate)
    CK(launch_lb<float>(d_test, Q, d_train, env, N, L, Weff, V, keogh, true, m.lb_lo, m.abs32,
                        ws.lb, ws.seed, ws.norms, rev ? ws.ends : nullptr,
                        (flags & NNDTW_LEAVE_ONE_OUT) != 0, s));
    CK(tm.mark(2));
    unsigned long long *cnt = (stats && !timing) ? ws.counters : nullptr;
    // S4 on the first candidate of every query: initial upper bounds
    DtwJob32 j{};
    j.test = d_test; j.train = d_train; j.L = L; j.W = Weff;
    j.dtw_lo = m.dtw_lo; j.dtw_hi = m.dtw_hi; j.abs32 = m.abs32;
    j.bsf = ws.bsf; j.cand = ws.cand; j.cand_count = ws.counters + C_CAND;
    j.counters = cnt;
    j.group = group_from_flags(flags);
    j.pairs = nullptr; j.seed_keys = ws.seed; j.n_seed = Q; j.head = nullptr; j.abandon = 0;
    // one pair per query: latency-bound, so spread each pair over the widest group
    const int main_group = j.group;
    j.group = (dtw32_rows_ok(L, Weff) || dtw32_rowsc_ok(L, Weff)) ? kRowsGroup
                                                                : dtw32_wide_group(Weff);
    CK(launch_dtw32(j, sms, s));
    j.group = main_group;
    CK(tm.mark(3));
    // S3: compaction against the upper bounds
    {
        UbOf<float> ubf{m.dtw_hi, m.abs32};
        const int np = (flags & NNDTW_NO_PRUNE) ? 1 : 0;
        for (int pass = 0; pass < 2; pass++) {
            compact_kernel<float><<<grid_compact(Q, N), kSmallThreads, 0, s>>>(
                ws.lb, Q, N, ws.bsf, ws.seed, ubf, np, pass, ws.buckets, ws.buckets + kBuckets,
                ws.queue, ws.counters + C_QUEUE);
            CK(cudaGetLastError());
        }
    }
    // the cascade's second stage on the survivors (into the recheck list's
    // storage, which S5 fills only after the DTW pass)
    const bool second = rev || imp;
    if (second) {
        CascadeJob cj{};
        cj.in = ws.queue; cj.in_count = ws.counters + C_QUEUE;
        cj.train = d_train; cj.envq = reinterpret_cast<const float2 *>(ws.envq);
        cj.ends = rev ? ws.ends : nullptr;
        cj.bgap = imp ? reinterpret_cast<const BGap *>(ws.env2) : nullptr;
        cj.lb = ws.lb;
        cj.N = N; cj.L = L; cj.nb = bridge_start(L, V);
        cj.bsf = ws.bsf;
        cj.lb_lo = m.lb_lo; cj.lb_abs = m.abs32; cj.dtw_hi = m.dtw_hi; cj.abs32 = m.abs32;
        cj.out = ws.rlist; cj.out_count = ws.counters + C_QUEUE2; cj.counters = cnt;
        CK(launch_cascade_filter(cj, Q * N, sms, s));
    }
    CK(tm.mark(4));
    // S4 on the survivors, with early abandoning
    j.pairs = second ? ws.rlist : ws.queue; j.seed_keys = nullptr;
    j.count = ws.counters + (second ? C_QUEUE2 : C_QUEUE);
    j.head = ws.counters + C_HEAD;
    j.abandon = (flags & NNDTW_NO_ABANDON) ? 0 : 1;
    CK(launch_dtw32(j, sms, s));
    CK(tm.mark(5));
    // S5: near-tie recheck in FP64 and the final argmin
    const long long cap = (long long)Q * N + Q;
    const unsigned gs = grid_small(cap);
    filter32_kernel<<<gs, kSmallThreads, 0, s>>>(ws.cand, ws.counters + C_CAND, ws.bsf, m.dtw_lo,
                                                 m.dtw_hi, m.abs32, ws.rcount);
    CK(cudaGetLastError());
    collect32_kernel<<<gs, kSmallThreads, 0, s>>>(ws.cand, ws.counters + C_CAND, ws.bsf,
                                                  m.dtw_lo, m.dtw_hi, m.abs32, ws.rcount, exact,
                                                  ws.rlist, ws.counters);
    CK(cudaGetLastError());
    DtwJob64 r{};
    r.test32 = d_test; r.train32 = d_train; r.L = L; r.W = Weff;
    r.pairs = ws.rlist; r.count = ws.counters + C_RECHECK; r.head = nullptr;
    r.bsf64 = ws.best64; r.out = ws.d64; r.abandon = 0;
    CK(launch_dtw64(r, sms, s));
    ties32_kernel<<<gs, kSmallThreads, 0, s>>>(ws.rlist, ws.counters + C_RECHECK, ws.d64,
                                               ws.best64, ws.bestidx);
    CK(cudaGetLastError());
    CK(tm.mark(6));
    finalize32_kernel<<<grid_small(Q), kSmallThreads, 0, s>>>(
        Q, ws.bsf, ws.rcount, ws.best64, ws.bestidx, exact, d_train_labels, d_nn_idx, d_nn_label,
        d_nn_dist);
    CK(cudaGetLastError());
    CK(tm.mark(7));
    if (stats) {
        unsigned long long h[C_COUNT];
        CK(cudaMemcpyAsync(h, ws.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        fill_stats(stats, h, N, Q, L, Weff, cnt != nullptr);
    }
    return NNDTW_OK;
}

int nn_dtw_search_f64(const double *d_train, const int32_t *d_train_labels, int64_t N,
                      const double *d_test, int64_t Q, int L, int W, int V, const double *d_env,
                      unsigned flags, int32_t *d_nn_idx, int32_t *d_nn_label, double *d_nn_dist,
                      void *d_workspace, size_t workspace_bytes, nndtw_stats *stats,
                      void *stream) {
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
    const Layout64 ws = layout64(d_workspace, N, Q, L);
    if (workspace_bytes < ws.bytes) return NNDTW_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int Weff = W > L - 1 ? L - 1 : W;
    const Margins m = make_margins(L);
    const int sms = device_sm_count();

    const bool timing = (flags & NNDTW_TIME_STAGES) != 0;
    StageTimer tm;
    CK(tm.start(timing, s));
    CK(cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * C_COUNT, s));
    CK(cudaMemsetAsync(ws.buckets, 0, sizeof(unsigned long long) * 2 * kBuckets, s));
    CK(cudaMemsetAsync(ws.bsf64, 0x7f, sizeof(unsigned long long) * Q, s));
    CK(cudaMemsetAsync(ws.seed, 0xff, sizeof(unsigned long long) * Q, s));
    CK(cudaMemsetAsync(ws.bestidx, 0x7f, sizeof(int32_t) * Q, s));
    if (flags & NNDTW_CHECK_FINITE) {
        int rc = check_finite<double>(d_train, N * L, 1e150, ws.counters + C_BAD, s);
        if (rc) return rc;
        rc = check_finite<double>(d_test, Q * L, 1e150, ws.counters + C_BAD, s);
        if (rc) return rc;
        unsigned long long bad = 0;
        CK(cudaMemcpyAsync(&bad, ws.counters + C_BAD, sizeof(bad), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad) return NNDTW_ENONFINITE;
    }
    const double *env = d_env;
    if (!env) {
        CK(launch_envelopes<double>(d_train, N, L, Weff, ws.env, s));
        env = ws.env;
    }
    const bool keogh = (flags & NNDTW_KEOGH_BOUND) != 0;
    const bool rev = !keogh && !(flags & (NNDTW_NO_PRUNE | NNDTW_NO_REVERSE));
    const bool imp = (flags & NNDTW_IMPROVED) && !keogh && !(flags & NNDTW_NO_PRUNE);
    if (rev || imp) CK(launch_envelopes<double>(d_test, Q, L, Weff, ws.envq, s));
    if (imp) CK(launch_second_envelopes<double>(env, N, L, Weff, ws.env2, s));
    CK(tm.mark(1));
    CK(launch_lb<double>(d_test, Q, d_train, env, N, L, Weff, V, keogh, true, m.lb_lo64,
                         m.abs64, ws.lb, ws.seed, ws.norms, rev ? ws.ends : nullptr,
                         (flags & NNDTW_LEAVE_ONE_OUT) != 0, s));
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
        UbOf<double> ubd{};
        const int np = (flags & NNDTW_NO_PRUNE) ? 1 : 0;
        for (int pass = 0; pass < 2; pass++) {
            compact_kernel<double><<<grid_compact(Q, N), kSmallThreads, 0, s>>>(
                ws.lb, Q, N, ws.bsf64, ws.seed, ubd, np, pass, ws.buckets, ws.buckets + kBuckets,
                ws.queue, ws.counters + C_QUEUE);
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
        fill_stats(stats, h, N, Q, L, Weff, cnt != nullptr);
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

}  // extern "C"
