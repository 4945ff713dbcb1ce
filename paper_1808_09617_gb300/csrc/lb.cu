// S2: LB_Enhanced^V_W (Sec. 3.1, Eq. 7 / Algorithm 1 without the abandon
// test) or LB_Keogh (Sec. 2.2.3) for every (query, training series) pair.
//
// Tiling: a CTA of 256 threads owns 16 MR queries x 16 MC training series;
// each thread owns an MR x MC register micro-tile of pairs (queries ty MR + r,
// series in pairs of columns).  MR = MC = 4 (64 x 64 tiles) when the tile
// grid fills the GPU, 2 x 2 (32 x 32) for small problems; 8 x 4 (128 x 64)
// on request (a tuning choice: fewer shared loads per pair-element at half
// the resident CTAs).  The Keogh bridge streams the series in chunks of 32 elements
// staged transposed in shared memory (query values and (U, Lo) envelope
// pairs), so every staged element feeds 4 pairs per thread and 64 per CTA;
// the next chunk is loaded into registers while the current one is used.
// Elements outside the bridge range [n, L-n) are staged as A = 0 with the
// envelope (+inf, -inf), which makes their term exactly 0; the inner loop is
// therefore branch-free: d = A - clamp(A, Lo, U); acc += d * d.
// The band terms need only the first and last n elements of both series
// (the left bands use indices <= n, the right bands >= L-n+1); those are
// staged once per CTA.
//
// Outputs: the bound per pair (raw, or scaled down by the rounding margin)
// and, for the search, per query the packed key (distance, index) of its
// nearest training series in squared Euclidean distance, fused into the same
// pass: the search's first DTW candidate, as in the paper's protocol of
// starting from the candidate nearest in Euclidean distance (Sec. 4).  The
// distance is formed as |a|^2 + |b|^2 - 2 a.b from precomputed squared norms
// (one multiply-add per pair-element); it only picks that first candidate,
// whose exact DTW then bounds the query, so its rounding never changes a
// result.
#include <type_traits>

#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kLC = 32, kThreads = 256, kNBMax = 32;

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

__device__ __forceinline__ float dsq(float a, float b) { float d = a - b; return d * d; }
__device__ __forceinline__ double dsq(double a, double b) {
    double d = __dsub_rn(a, b); return __dmul_rn(d, d);
}
__device__ __forceinline__ float tmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double tmin3(double a, double b, double c) { return fmin(fmin(a, b), c); }

// The distance of a to [l, u] as max(a - u, l - a, 0): the same value as
// a - clamp(a, l, u) up to its sign, with one three-input max instead of a
// max and a min (the min/max pipe issues at half the FP32 rate).
__device__ __forceinline__ float keogh_term(float a, float u, float l, float acc) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a - u), "f"(l - a), "f"(0.f));
    return fmaf(d, d, acc);
}
__device__ __forceinline__ double keogh_term(double a, double u, double l, double acc) {
    double d = a - fmin(fmax(a, l), u);
    return fma(d, d, acc);
}

__device__ __forceinline__ float to_key_float(float x) { return x; }
__device__ __forceinline__ float to_key_float(double x) { return __double2float_rd(x); }

__device__ __forceinline__ float safe_scale(float x, float lo, float abs_s) {
    float v = __fmul_rd(x, lo) - abs_s;
    return v > 0.f ? v : 0.f;
}
__device__ __forceinline__ double safe_scale(double x, double lo, double abs_s) {
    double v = __dmul_rd(x, lo) - abs_s;
    return v > 0.0 ? v : 0.0;
}

// A lower bound of the exact squared Euclidean distance from its value e
// formed as |a|^2 + |b|^2 - 2 a.b: e less g (|a| + |b|)^2, rounded down (g
// bounds the relative rounding of the norms and the dot product).
__device__ __forceinline__ float ed_lower(float e, float na, float nb, float g) {
    const float s = __fadd_ru(__fsqrt_ru(na), __fsqrt_ru(nb));
    return __fsub_rd(e, __fmul_ru(g, __fmul_ru(s, s)));
}

// Four consecutive tile rows of one column into shared memory with vector
// stores: A16 when the destination is 16-byte aligned, else 8-byte stores.
template <bool A16> __device__ __forceinline__ void sts4(float *d, const float (&v)[4]) {
    if (A16) {
        *reinterpret_cast<float4 *>(d) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<float2 *>(d)[0] = make_float2(v[0], v[1]);
        reinterpret_cast<float2 *>(d)[1] = make_float2(v[2], v[3]);
    }
}
template <bool A16> __device__ __forceinline__ void sts4(double *d, const double (&v)[4]) {
    reinterpret_cast<double2 *>(d)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(d)[1] = make_double2(v[2], v[3]);
}
template <bool A16> __device__ __forceinline__ void sts4(float2 *d, const float2 (&v)[4]) {
    reinterpret_cast<float4 *>(d)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    reinterpret_cast<float4 *>(d)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}
template <bool A16> __device__ __forceinline__ void sts4(double2 *d, const double2 (&v)[4]) {
#pragma unroll
    for (int j = 0; j < 4; j++) d[j] = v[j];
}

// The two ends and the V-1 left and right bands of Eq. 7 for one pair:
// element i of A and B is Ap[i], Bp[i] for i < nb, and Ap[last - k],
// Bp[last - k] for the k-th element from the end.  Inlined at each call site
// so that the loads keep the pointers' address space.
template <typename T>
__device__ __forceinline__ T band_terms(const T *Ap, const T *Bp, int last, int nb, int W) {
    T res = dsq(Ap[0], Bp[0]) + dsq(Ap[last], Bp[last]);
    for (int ii = 1; ii < nb; ii++) {
        const int ri = last - ii;
        const T ai = Ap[ii], bi = Bp[ii], ar = Ap[ri], br = Bp[ri];
        T mL = dsq(ai, bi);
        T mR = dsq(ar, br);
        const int jlo = ii - W > 0 ? ii - W : 0;
        for (int jj = jlo; jj < ii; jj++) {
            const int rj = last - jj;
            mL = tmin3(mL, dsq(ai, Bp[jj]), dsq(Ap[jj], bi));
            mR = tmin3(mR, dsq(ar, Bp[rj]), dsq(Ap[rj], br));
        }
        res = res + mL + mR;
    }
    return res;
}

// Shared-memory layout of one stage of chunk tiles: queries [kLC][kQT+4],
// then envelope pairs [kLC][kNT+2], then training values [kLC][kNT+2] when
// the Euclidean seed is fused in.  The row strides keep every row 16-byte
// aligned, so that a thread reads its MR queries, and its column pairs'
// envelopes and values, with vector loads.
constexpr int kPadA = 4, kPadN = 2;
template <typename T, int kQT>
__host__ __device__ constexpr size_t lb_es_offset() {
    return (sizeof(T) * (kLC * (kQT + kPadA)) + 15) / 16 * 16;
}
template <typename T, int kQT, int kNT, bool ED>
__host__ __device__ constexpr size_t lb_stage_bytes() {
    return (lb_es_offset<T, kQT>() + 2 * sizeof(T) * kLC * (kNT + kPadN) +
            (ED ? sizeof(T) * kLC * (kNT + kPadN) : 0) + 15) / 16 * 16;
}

// Vector loads from shared memory: n consecutive values (16-byte aligned).
__device__ __forceinline__ void lds4(float (&d)[4], const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
__device__ __forceinline__ void lds4(double (&d)[4], const double *p) {
    const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
    const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
    d[0] = v0.x; d[1] = v0.y; d[2] = v1.x; d[3] = v1.y;
}
__device__ __forceinline__ void lds2(float (&d)[2], const float *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    d[0] = v.x; d[1] = v.y;
}
__device__ __forceinline__ void lds2(double (&d)[2], const double *p) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    d[0] = v.x; d[1] = v.y;
}
__device__ __forceinline__ void lds2(float2 (&d)[2], const float2 *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    d[0] = make_float2(v.x, v.y); d[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void lds2(double2 (&d)[2], const double2 *p) {
    d[0] = p[0]; d[1] = p[1];
}
template <typename T, int N> __device__ __forceinline__ void ldsn(T (&d)[N], const T *p) {
    if constexpr (N == 8) {
        T lo[4], hi[4];
        lds4(lo, p);
        lds4(hi, p + 4);
#pragma unroll
        for (int k = 0; k < 4; k++) { d[k] = lo[k]; d[4 + k] = hi[k]; }
    } else if constexpr (N == 4) lds4(d, p);
    else if constexpr (N == 2) lds2(d, p);
    else {
#pragma unroll
        for (int k = 0; k < N; k++) d[k] = p[k];
    }
}

// Squared norm of every row of a and of b (one warp per row).
template <typename T, typename Src>
__global__ void sqnorm_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const SqnormJob<T> &job = src.get(bid, nblk);
    const T *__restrict__ a = job.a;
    const T *__restrict__ b = job.b;
    const int64_t na = job.na, nb = job.nb;
    const int L = job.L;
    T *__restrict__ out_a = job.out_a;
    T *__restrict__ out_b = job.out_b;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)nblk * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)bid * blockDim.x + threadIdx.x) >> 5; r < na + nb;
         r += warps) {
        const T *x = r < na ? a + r * L : b + (r - na) * L;
        T acc = T(0);
        for (int i = lane; i < L; i += 32) acc = fma(x[i], x[i], acc);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            if (r < na) out_a[r] = acc;
            else out_b[r - na] = acc;
        }
    }
}

template <typename T, bool ED, int MR, int MC, typename Src>
__global__ void __launch_bounds__(kThreads)
lb_kernel(const __grid_constant__ Src src) {
    int bid, nblk;
    const LbJob<T> &job = src.get(bid, nblk);
    const T *__restrict__ test = job.test;
    const T *__restrict__ train = job.train;
    const T *__restrict__ env = job.env;
    const int64_t Q = job.Q, N = job.N;
    const int L = job.L, W = job.W, nb = job.nb, keogh = job.keogh, safe = job.safe;
    const T lb_lo = job.lb_lo, abs_slack = job.abs_slack;
    T *__restrict__ lb_out = job.lb_out;
    unsigned long long *seed_keys = job.seed_keys;
    const T *__restrict__ nq = job.nq;
    const T *__restrict__ nt = job.nt;
    T *__restrict__ ends_out = job.ends_out;
    const int loo = job.loo, qfast = job.qfast;
    const int64_t q_base = job.q_base;   // global index of query 0 (leave-one-out)
    // the CTA's tile: bx along the fast dimension (gx tiles), by along the other
    const int bx = bid % job.gx, by = bid / job.gx;
    using T2 = typename V2<T>::type;
    constexpr int kQT = 16 * MR, kNT = 16 * MC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // One stage of chunk tiles (the next chunk waits in registers while the
    // current one is used), then the band staging.  Offsets are taken from
    // the shared array itself (not through integer casts), so that every
    // access compiles to a shared-memory load.
    constexpr size_t kEsOff = lb_es_offset<T, kQT>();
    constexpr size_t kStage = lb_stage_bytes<T, kQT, kNT, ED>();
    T *As = reinterpret_cast<T *>(smem_raw);                      // [kLC][kQT+kPadA]
    T2 *Es = reinterpret_cast<T2 *>(smem_raw + kEsOff);           // [kLC][kNT+kPadN], 16-byte aligned
    T *Bs = reinterpret_cast<T *>(Es + kLC * (kNT + kPadN));       // [kLC][kNT+kPadN] (ED only)
    // band staging, rows padded to an odd stride so that the 16 series a
    // warp reads at once fall in distinct banks
    const int bstride = 2 * nb + 1;
    T *Ab = reinterpret_cast<T *>(smem_raw + kStage);              // [kQT][2nb+1]
    T *Bb = Ab + kQT * (nb <= kNBMax ? bstride : 0);               // [kNT][2nb+1]

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // thread (tx, ty) owns the tile's query rows ty MR .. ty MR + MR-1 and the
    // training columns 2 tx, 2 tx + 1 of each group of 32 (MC / 2 groups)
    static_assert(MC % 2 == 0, "training columns come in pairs");
    auto row_of = [&](int r) { return ty * MR + r; };
    auto col_of = [&](int c) { return (c >> 1) * 32 + 2 * tx + (c & 1); };
    // query tiles vary fastest (qfast), so the CTAs resident at one time share
    // a few training tiles (series and envelopes read from DRAM about once)
    const int64_t q0 = (int64_t)(qfast ? bx : by) * kQT;
    const int64_t t0 = (int64_t)(qfast ? by : bx) * kNT;

    T acc[MR][MC], ed[MR][MC];
#pragma unroll
    for (int r = 0; r < MR; r++)
#pragma unroll
        for (int c = 0; c < MC; c++) { acc[r][c] = T(0); ed[r][c] = T(0); }

    // W = 0 in the search: the bound comes from the dot products alone (no
    // envelope is staged, no bridge or band term computed)
    bool ed_only = false;
    if constexpr (ED && std::is_same<T, float>::value) ed_only = job.edb != 0;
    const int mlo = ed_only ? 0 : keogh ? 0 : nb, mhi = ed_only ? 0 : keogh ? L : L - nb;
    const T POS = inf_of<T>();

    const int cbeg = ED ? 0 : (mlo / kLC) * kLC, cend = ED ? L : mhi;
    // Staging of a chunk of kLC elements: thread tid takes groups of four
    // consecutive tile rows at one column (column = group % kLC, so a warp
    // reads 32 consecutive elements of each of four rows: coalesced), loads
    // them into registers one chunk ahead, and writes each group into the
    // transposed tile with vector stores (consecutive columns of a warp land
    // 16 bytes apart modulo 128: no bank conflicts).
    constexpr int kGA = kQT * kLC / 4 / kThreads;   // query groups per thread
    constexpr int kGN = kNT * kLC / 4 / kThreads;   // training groups per thread
    static_assert(kGA * 4 * kThreads == kQT * kLC && kGN * 4 * kThreads == kNT * kLC,
                  "tile groups divide among the threads");
    const T2 *envp = reinterpret_cast<const T2 *>(env);
    T ra[kGA][4], rb[kGN][4];
    T2 re[kGN][4];
    auto load = [&](int c0) {
#pragma unroll
        for (int k = 0; k < kGA; k++) {
            const int g = tid + k * kThreads, col = g % kLC, row4 = (g / kLC) * 4;
            const int i = c0 + col;
            const T *p = test + (q0 + row4) * L + i;
#pragma unroll
            for (int j = 0; j < 4; j++)
                ra[k][j] = (i < L && q0 + row4 + j < Q) ? p[(int64_t)j * L] : T(0);
        }
#pragma unroll
        for (int k = 0; k < kGN; k++) {
            const int g = tid + k * kThreads, col = g % kLC, row4 = (g / kLC) * 4;
            const int i = c0 + col;
            const bool in_bridge = i >= mlo && i < mhi;
            const T2 *pe = envp + (t0 + row4) * L + i;
            const T *pb = train + (t0 + row4) * L + i;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const bool rowok = t0 + row4 + j < N;
                if (rowok && in_bridge) {
                    re[k][j] = pe[(int64_t)j * L];
                } else {
                    re[k][j].x = POS; re[k][j].y = -POS;   // outside the bridge: term 0
                }
                if constexpr (ED) rb[k][j] = (rowok && i < L) ? pb[(int64_t)j * L] : T(0);
            }
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int k = 0; k < kGA; k++) {
            const int g = tid + k * kThreads, col = g % kLC, row4 = (g / kLC) * 4;
            sts4<true>(As + col * (kQT + kPadA) + row4, ra[k]);   // rows 16-byte aligned
        }
#pragma unroll
        for (int k = 0; k < kGN; k++) {
            const int g = tid + k * kThreads, col = g % kLC, row4 = (g / kLC) * 4;
            sts4<true>(Es + col * (kNT + kPadN) + row4, re[k]);
            // (training values: rows of kNT + kPadN, 8-byte aligned in FP32)
            if constexpr (ED) sts4<false>(Bs + col * (kNT + kPadN) + row4, rb[k]);
        }
    };
    if (cbeg < cend) load(cbeg);
    for (int c0 = cbeg; c0 < cend; c0 += kLC) {
        store();
        __syncthreads();
        if (c0 + kLC < cend) load(c0 + kLC);   // in flight while this chunk is used
        if (ed_only) {
#pragma unroll 4
            for (int col = 0; col < kLC; col++) {
                T a[MR], b[MC];
                ldsn<T, MR>(a, As + col * (kQT + kPadA) + ty * MR);
#pragma unroll
                for (int g = 0; g < MC / 2; g++) {
                    T bg[2];
                    lds2(bg, Bs + col * (kNT + kPadN) + g * 32 + 2 * tx);
                    b[2 * g] = bg[0]; b[2 * g + 1] = bg[1];
                }
#pragma unroll
                for (int r = 0; r < MR; r++)
#pragma unroll
                    for (int c = 0; c < MC; c++) ed[r][c] = fma(a[r], b[c], ed[r][c]);
            }
            __syncthreads();
            continue;
        }
#pragma unroll 4
        for (int col = 0; col < kLC; col++) {
            T a[MR];
            T2 e[MC];
            ldsn<T, MR>(a, As + col * (kQT + kPadA) + ty * MR);
#pragma unroll
            for (int g = 0; g < MC / 2; g++) {
                T2 eg[2];
                lds2(eg, Es + col * (kNT + kPadN) + g * 32 + 2 * tx);
                e[2 * g] = eg[0]; e[2 * g + 1] = eg[1];
            }
#pragma unroll
            for (int r = 0; r < MR; r++)
#pragma unroll
                for (int c = 0; c < MC; c++) acc[r][c] = keogh_term(a[r], e[c].x, e[c].y, acc[r][c]);
            if (ED) {
                T b[MC];
#pragma unroll
                for (int g = 0; g < MC / 2; g++) {
                    T bg[2];
                    lds2(bg, Bs + col * (kNT + kPadN) + g * 32 + 2 * tx);
                    b[2 * g] = bg[0]; b[2 * g + 1] = bg[1];
                }
#pragma unroll
                for (int r = 0; r < MR; r++)
#pragma unroll
                    for (int c = 0; c < MC; c++) ed[r][c] = fma(a[r], b[c], ed[r][c]);
            }
        }
        __syncthreads();
    }

    if (!keogh && !ed_only) {
        // stage the first and last nb elements of the tile's series
        const bool staged = nb <= kNBMax;
        if (staged) {
            const int w2 = 2 * nb;
            for (int idx = tid; idx < kQT * w2; idx += kThreads) {
                const int row = idx / w2, m = idx % w2;
                const int i = m < nb ? m : L - w2 + m;
                const int64_t q = q0 + row;
                Ab[row * bstride + m] = q < Q ? test[q * L + i] : T(0);
            }
            for (int idx = tid; idx < kNT * w2; idx += kThreads) {
                const int row = idx / w2, m = idx % w2;
                const int i = m < nb ? m : L - w2 + m;
                const int64_t t = t0 + row;
                Bb[row * bstride + m] = t < N ? train[t * L + i] : T(0);
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < MR; r++) {
            const int64_t q = q0 + row_of(r);
#pragma unroll
            for (int c = 0; c < MC; c++) {
                const int64_t t = t0 + col_of(c);
                // staged copies hold the first nb then the last nb elements
                // (offset of the last nb: L - 2 nb); otherwise read the series
                const T res = staged
                    ? band_terms(Ab + row_of(r) * bstride, Bb + col_of(c) * bstride,
                                 2 * nb - 1, nb, W)
                    : band_terms(test + (q < Q ? q : 0) * L, train + (t < N ? t : 0) * L, L - 1,
                                 nb, W);
                acc[r][c] = res + acc[r][c];
                // the ends and bands alone: they are the same for LB(B, A)
                if (ends_out && q < Q && t < N) ends_out[q * N + t] = res;
            }
        }
    }

    // outputs
#pragma unroll
    for (int r = 0; r < MR; r++) {
        const int64_t q = q0 + row_of(r);
        unsigned long long best = ~0ull;
#pragma unroll
        for (int c = 0; c < MC; c++) {
            const int64_t t = t0 + col_of(c);
            T raw = acc[r][c];
            T sv = safe_scale(raw, lb_lo, abs_slack);
            if constexpr (ED && std::is_same<T, float>::value) {
                if (ed_only && q < Q && t < N) {
                    const T na = nq[q], nb2 = nt[t];
                    T e = na + nb2 - T(2) * ed[r][c];
                    e = e > T(0) ? e : T(0);
                    raw = e;
                    sv = safe_scale(ed_lower(e, na, nb2, job.ed_gamma), lb_lo, abs_slack);
                }
            }
            if (q < Q && t < N) {
                // leave-one-out: a series is never its own candidate
                const bool self = loo && q + q_base == t;
                if (lb_out) lb_out[q * N + t] = self ? POS : (safe ? sv : raw);
                if (ED && !self) {
                    // squared distance from the norms and the dot product
                    // (clamped: rounding may take it slightly below 0)
                    T e = nq[q] + nt[t] - T(2) * ed[r][c];
                    e = e > T(0) ? e : T(0);
                    const unsigned long long k = pack_key(to_key_float(e), (uint32_t)t);
                    best = k < best ? k : best;
                }
            }
        }
        if (ED) {
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off, 16);
                best = o < best ? o : best;
            }
            if (tx == 0 && q < Q && best != ~0ull) atomicMin(seed_keys + q, best);
        }
    }
}

template <typename T, int MR, int MC>
size_t lb_smem(bool ed, bool keogh, int nb) {
    constexpr int kQT = 16 * MR, kNT = 16 * MC;
    size_t smem = ed ? lb_stage_bytes<T, kQT, kNT, true>() : lb_stage_bytes<T, kQT, kNT, false>();
    if (!keogh && nb <= kNBMax) smem += sizeof(T) * (size_t)(kQT + kNT) * (2 * nb + 1);
    return smem;
}

}  // namespace

template <typename T>
cudaError_t plan_lb(const T *test, int64_t Q, const T *train, const T *env, int64_t N, int L,
                    int W, int V, bool keogh, bool safe, T lb_lo, T abs_slack, T *lb_out,
                    unsigned long long *seed_keys, T *norms, T *ends_out, bool loo,
                    LbPlan<T> *p, int64_t q_base, int tile, bool ed_bound) {
    int nb = L / 2 < V ? L / 2 : V;
    if (nb < 1) nb = 1;
    const int Weff = W > L - 1 ? L - 1 : W;
    // 64 x 64 tiles when they give at least two CTAs per SM, else 32 x 32
    const int sms = device_sm_count();
    // tile shape: 64 x 64 when such tiles give at least two CTAs per SM, else
    // 32 x 32, unless the caller asks for one (1: 32 x 32, 2: 64 x 64,
    // 3: 128 x 64)
    p->tile = tile ? tile : (((N + 63) / 64) * ((Q + 63) / 64) < 2ll * sms ? 1 : 2);
    p->ed = seed_keys != nullptr;
    const int kQT = p->tile == 1 ? 32 : p->tile == 2 ? 64 : 128;
    const int kNT = p->tile == 1 ? 32 : 64;
    const long long qt = (Q + kQT - 1) / kQT, nt_tiles = (N + kNT - 1) / kNT;
    LbJob<T> &j = p->job;
    j.test = test; j.Q = Q; j.train = train; j.env = env; j.N = N; j.L = L; j.W = Weff;
    j.nb = nb; j.keogh = keogh ? 1 : 0; j.safe = safe ? 1 : 0; j.lb_lo = lb_lo;
    j.abs_slack = abs_slack; j.lb_out = lb_out; j.seed_keys = seed_keys;
    j.nq = seed_keys ? norms : nullptr; j.nt = seed_keys ? norms + Q : nullptr;
    j.ends_out = keogh ? nullptr : ends_out; j.loo = loo ? 1 : 0; j.q_base = q_base;
    // W = 0: DTW_0 is the squared Euclidean distance and so is the bound
    // (every envelope is the series itself), so in the search the bound is
    // taken from |a|^2 + |b|^2 - 2 a.b, which the fused first-candidate pass
    // forms anyway.  Its rounding error is at most gamma_{L+4} (|a| + |b|)^2
    // (the norms and the dot product are sums of L products, each within
    // gamma_L of its exact value, |a.b| <= |a| |b|, and three more roundings
    // combine them); the margin used is 1 - lb_lo = gamma_{2L+16}, larger.
    j.edb = (ed_bound && std::is_same<T, float>::value && Weff == 0 && seed_keys && safe &&
             !keogh && !j.ends_out) ? 1 : 0;
    j.ed_gamma = T(1) - lb_lo;
    // query tiles vary fastest, so the CTAs resident at one time share a few
    // training tiles
    j.qfast = 1;
    j.gx = (int)qt;
    p->blocks = qt * nt_tiles;
    p->smem = p->tile == 1 ? lb_smem<T, 2, 2>(p->ed, keogh, nb)
            : p->tile == 2 ? lb_smem<T, 4, 4>(p->ed, keogh, nb) : lb_smem<T, 8, 4>(p->ed, keogh, nb);
    p->sq = SqnormJob<T>{test, Q, train, N, L, norms, norms + Q};
    const int64_t rows = Q + N;
    p->sq_blocks = seed_keys ? ((rows + 7) / 8 < 4096 ? (rows + 7) / 8 : 4096) : 0;
    return cudaSuccess;
}

template <typename T, int MR, int MC> void lb_fns_of(bool ed, LbFns<T> *f) {
    f->fn1 = ed ? lb_kernel<T, true, MR, MC, Src1<LbJob<T>>> : lb_kernel<T, false, MR, MC, Src1<LbJob<T>>>;
    f->fnN = ed ? lb_kernel<T, true, MR, MC, SrcN<LbJob<T>>> : lb_kernel<T, false, MR, MC, SrcN<LbJob<T>>>;
}

template <typename T>
LbFns<T> lb_fns(int tile, bool ed) {
    LbFns<T> f;
    if (tile == 1) lb_fns_of<T, 2, 2>(ed, &f);
    else if (tile == 2) lb_fns_of<T, 4, 4>(ed, &f);
    else lb_fns_of<T, 8, 4>(ed, &f);
    f.sq1 = sqnorm_kernel<T, Src1<SqnormJob<T>>>;
    f.sqN = sqnorm_kernel<T, SrcN<SqnormJob<T>>>;
    return f;
}

template <typename T>
cudaError_t set_lb_smem(int tile, bool ed, size_t smem) {
    const LbFns<T> f = lb_fns<T>(tile, ed);
    cudaError_t e = cudaFuncSetAttribute(f.fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f.fnN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

template <typename T>
cudaError_t launch_lb(const T *test, int64_t Q, const T *train, const T *env, int64_t N, int L,
                      int W, int V, bool keogh, bool safe, T lb_lo, T abs_slack, T *lb_out,
                      unsigned long long *seed_keys, T *norms, T *ends_out, bool loo,
                      cudaStream_t s, int64_t q_base, int tile) {
    if (Q <= 0 || N <= 0) return cudaSuccess;
    if (seed_keys && !norms) return cudaErrorInvalidValue;
    LbPlan<T> p{};
    cudaError_t e = plan_lb<T>(test, Q, train, env, N, L, W, V, keogh, safe, lb_lo, abs_slack,
                               lb_out, seed_keys, norms, ends_out, loo, &p, q_base, tile);
    if (e != cudaSuccess) return e;
    const LbFns<T> f = lb_fns<T>(p.tile, p.ed);
    if (p.sq_blocks > 0) {
        // squared norms of the queries (norms[0..Q)) and training series
        // (norms[Q..Q+N)) for the fused Euclidean distance
        f.sq1<<<(unsigned)p.sq_blocks, 256, 0, s>>>(Src1<SqnormJob<T>>{p.sq});
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    e = set_lb_smem<T>(p.tile, p.ed, p.smem);
    if (e != cudaSuccess) return e;
    f.fn1<<<(unsigned)p.blocks, kThreads, p.smem, s>>>(Src1<LbJob<T>>{p.job});
    return cudaGetLastError();
}

template cudaError_t launch_lb<float>(const float *, int64_t, const float *, const float *, int64_t,
                                      int, int, int, bool, bool, float, float, float *,
                                      unsigned long long *, float *, float *, bool,
                                      cudaStream_t, int64_t, int);
template cudaError_t launch_lb<double>(const double *, int64_t, const double *, const double *,
                                       int64_t, int, int, int, bool, bool, double, double,
                                       double *, unsigned long long *, double *, double *,
                                       bool, cudaStream_t, int64_t, int);
template cudaError_t plan_lb<float>(const float *, int64_t, const float *, const float *, int64_t,
                                    int, int, int, bool, bool, float, float, float *,
                                    unsigned long long *, float *, float *, bool,
                                    LbPlan<float> *, int64_t, int, bool);
template LbFns<float> lb_fns<float>(int, bool);
template cudaError_t set_lb_smem<float>(int, bool, size_t);

}  // namespace nndtw
