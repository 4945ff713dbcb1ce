// S1: upper/lower envelopes U, Lo of every training series (Sec. 2.2.3,
// Eq. 3-4): U_i = max B_j and Lo_i = min B_j over the window
// max(1, i-W) <= j <= min(L, i+W).
//
// Method (a block decomposition in the spirit of van Herk / Gil-Werman):
// split the series into aligned tiles of T = 2^floor(log2 W) elements (capped
// at 32, one tile never straddles a warp).  Warp shuffles give, per element,
// the max/min from its tile's start (prefix P) and to its tile's end (suffix
// S).  Every window is at least W+1 > T long, so it covers the end of one
// tile and the start of a later one: U_i = max(S[lo], P[hi], tiles between).
// With T > W/2 at most three tiles lie between; with T = 32 a sparse table
// over tile maxima answers the middle range with two lookups.  min/max are
// exact, so the result is bit-identical to a naive scan.
//
// Series of unequal lengths (offset table off: series s is
// train[off[s] .. off[s+1]), of length L_s <= L): the envelope is taken for
// the rows i < min(L_s + W, E) of a series compared with it (Sec. 2
// generalised), written with a row stride of E; a window then ends at
// min(L_s - 1, i + W), and a window that fits in one tile is a prefix of it
// (starting at 0) or a suffix (ending at L_s - 1).
//
// The same kernel gives the second envelopes used by the LB_Improved bridge:
// fed with a series' envelopes (U, Lo) instead of the series, it takes the
// window maximum of Lo and the window minimum of U.
#include "internal.cuh"

namespace nndtw {
namespace {

constexpr int kEnvThreads = kEnvelopeThreads;

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// Channel 0 is the window maximum of the series (of Lo for the second
// envelopes), channel 1 the window minimum of the series (of U), taken as
// the negated maximum of the negated values (negation is exact).  NP = 2
// computes both channels in one pass over tile prefixes P, suffixes S and
// tile tables M ([NP][L], [NP][L], [NP][levels+1][nt]); NP = 1 runs one
// channel per pass in half the shared memory (the longest FP64 series).
template <typename T, int NP, typename Src>
__global__ void __launch_bounds__(kEnvThreads)
envelope_kernel(const __grid_constant__ Src src) {
    // env_in == nullptr: envelopes of train; else the second envelopes of
    // env_in ([N][L] (U, Lo)): window max of Lo and window min of U
    int bid, nblk;
    const EnvJob<T> &job = src.get(bid, nblk);
    const T *__restrict__ train = job.train;
    const T *__restrict__ env_in = job.env_in;
    const int64_t N = job.N;
    const int L = job.L, W = job.W, T_tile = job.T_tile, levels = job.levels;
    T *__restrict__ env = job.env;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nt = (L + T_tile - 1) / T_tile;
    T *P = reinterpret_cast<T *>(smem_raw);                 // [NP][L]
    T *S = P + (size_t)NP * L;                              // [NP][L]
    T *M = S + (size_t)NP * L;                              // [NP][levels+1][nt]
    const size_t mstride = (size_t)(levels + 1) * nt;

    const int tid = threadIdx.x, lane = tid & 31;
    const int r = lane & (T_tile - 1);
    const T NEG = -inf_of<T>();

    for (int64_t s = bid; s < N; s += nblk) {
        const int64_t x0 = job.off ? (int64_t)job.off[s] : s * (int64_t)L;
        const int Ls = job.off ? (int)(job.off[s + 1] - x0) : L;   // this series' length
        if (Ls < 1 || Ls > L) continue;   // (a ragged length out of range: no envelope)
        const int E = job.off ? job.E : L;                         // output row stride
        const int rows = Ls + W < E ? Ls + W : E;
        const int nts = (Ls + T_tile - 1) / T_tile;
        const T *x = env_in ? nullptr : train + x0;
        const T *ein = env_in ? env_in + s * 2 * (int64_t)L : nullptr;
        T *out = env + s * 2 * (int64_t)E;
        if (W == 0) {
            for (int i = tid; i < Ls; i += kEnvThreads) {
                out[2 * i] = ein ? ein[2 * i + 1] : x[i];
                out[2 * i + 1] = ein ? ein[2 * i] : x[i];
            }
            continue;
        }
        for (int pass = 0; pass < 2 / NP; pass++) {
            // the values whose window maximum channel ch takes
            auto value = [&](int ch, int k) -> T {
                if (ch == 0) return ein ? ein[2 * k + 1] : x[k];
                return -(ein ? ein[2 * k] : x[k]);
            };
            // tile prefix / suffix scans
            for (int base = 0; base < Ls; base += kEnvThreads) {
                const int k = base + tid;
#pragma unroll
                for (int c = 0; c < NP; c++) {
                    const int ch = pass * NP + c;
                    T pm = k < Ls ? value(ch, k) : NEG;
                    T sm = pm;
                    for (int d = 1; d < T_tile; d <<= 1) {
                        const T a = __shfl_up_sync(0xffffffffu, pm, d);
                        const T b = __shfl_down_sync(0xffffffffu, sm, d);
                        if (r >= d) pm = tmax(pm, a);
                        if (r + d < T_tile) sm = tmax(sm, b);
                    }
                    if (k < Ls) {
                        P[(size_t)c * L + k] = pm; S[(size_t)c * L + k] = sm;
                        if (r == 0) M[c * mstride + k / T_tile] = sm;
                    }
                }
            }
            __syncthreads();
            // sparse table over tile maxima (level j covers 2^j tiles)
            for (int j = 1; j <= levels; j++) {
                const int half = 1 << (j - 1);
                const int cnt = nts - (1 << j) + 1;
                for (int idx = tid; idx < NP * cnt; idx += kEnvThreads) {
                    const int c = idx / cnt, t = idx % cnt;
                    const T *pm = M + c * mstride + (size_t)(j - 1) * nt;
                    M[c * mstride + (size_t)j * nt + t] = tmax(pm[t], pm[t + half]);
                }
                __syncthreads();
            }
            for (int i = tid; i < rows; i += kEnvThreads) {
                const int lo = i - W < 0 ? 0 : i - W;
                const int hi = i + W > Ls - 1 ? Ls - 1 : i + W;
                const int a = lo / T_tile + 1, b = hi / T_tile - 1;
                const bool one_tile = lo / T_tile == hi / T_tile;
#pragma unroll
                for (int c = 0; c < NP; c++) {
                    const int ch = pass * NP + c;
                    const T *Pc = P + (size_t)c * L, *Sc = S + (size_t)c * L, *Mc = M + c * mstride;
                    // (one tile: the window is a suffix of the series or a prefix)
                    T u = one_tile ? (hi == Ls - 1 ? Sc[lo] : Pc[hi]) : tmax(Sc[lo], Pc[hi]);
                    if (b >= a) {
                        if (levels == 0) {
                            for (int t = a; t <= b; t++) u = tmax(u, Mc[t]);
                        } else {
                            const int len = b - a + 1;
                            const int j = 31 - __clz(len);
                            const T *mx = Mc + (size_t)j * nt;
                            u = tmax(u, tmax(mx[a], mx[b - (1 << j) + 1]));
                        }
                    }
                    out[2 * i + ch] = ch == 0 ? u : -u;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

template <typename T>
EnvPlan<T> plan_envelopes(const T *train, const T *env_in, int64_t N, int L, int W, T *env) {
    EnvPlan<T> p{};
    const int Weff = W > L - 1 ? L - 1 : W;
    int T_tile = 1, levels = 0;
    if (Weff >= 32) {
        T_tile = 32;
        const int nt = (L + 31) / 32;
        while ((2 << levels) <= nt) levels++;
    } else if (Weff > 0) {
        while (T_tile * 2 <= Weff) T_tile *= 2;
    }
    const int nt = (L + T_tile - 1) / T_tile;
    // both channels in one pass when they fit, else one channel per pass
    const size_t per_channel = sizeof(T) * (2 * (size_t)L + (size_t)(levels + 1) * nt);
    p.one_pass = 2 * per_channel <= 200u * 1024u;
    p.smem = p.one_pass ? 2 * per_channel : per_channel;
    const int sms = device_sm_count();
    p.blocks = N < (int64_t)sms * 8 ? N : (int64_t)sms * 8;
    p.job = EnvJob<T>{train, env_in, N, L, Weff, T_tile, levels, env, nullptr, 0};
    return p;
}

template <typename T>
EnvFns<T> envelope_fns(bool one_pass) {
    EnvFns<T> f;
    if (one_pass) {
        f.fn1 = envelope_kernel<T, 2, Src1<EnvJob<T>>>;
        f.fnN = envelope_kernel<T, 2, SrcN<EnvJob<T>>>;
    } else {
        f.fn1 = envelope_kernel<T, 1, Src1<EnvJob<T>>>;
        f.fnN = envelope_kernel<T, 1, SrcN<EnvJob<T>>>;
    }
    return f;
}

template <typename T>
cudaError_t set_envelope_smem(bool one_pass, size_t smem) {
    const EnvFns<T> f = envelope_fns<T>(one_pass);
    cudaError_t e = cudaFuncSetAttribute(f.fn1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f.fnN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

namespace {
template <typename T>
cudaError_t launch_envelope_kernel(const T *train, const T *env_in, int64_t N, int L, int W,
                                   T *env, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const EnvPlan<T> p = plan_envelopes<T>(train, env_in, N, L, W, env);
    cudaError_t e = set_envelope_smem<T>(p.one_pass, p.smem);
    if (e != cudaSuccess) return e;
    envelope_fns<T>(p.one_pass).fn1<<<(unsigned)p.blocks, kEnvThreads, p.smem, s>>>(
        Src1<EnvJob<T>>{p.job});
    return cudaGetLastError();
}
}  // namespace

template <typename T>
cudaError_t launch_envelopes(const T *train, int64_t N, int L, int W, T *env, cudaStream_t s) {
    return launch_envelope_kernel<T>(train, nullptr, N, L, W, env, s);
}

template <typename T>
cudaError_t launch_second_envelopes(const T *env, int64_t N, int L, int W, T *env2,
                                    cudaStream_t s) {
    return launch_envelope_kernel<T>(nullptr, env, N, L, W, env2, s);
}

template cudaError_t launch_envelopes<float>(const float *, int64_t, int, int, float *,
                                             cudaStream_t);
template cudaError_t launch_envelopes<double>(const double *, int64_t, int, int, double *,
                                              cudaStream_t);
template cudaError_t launch_second_envelopes<float>(const float *, int64_t, int, int, float *,
                                                    cudaStream_t);
template cudaError_t launch_second_envelopes<double>(const double *, int64_t, int, int, double *,
                                                     cudaStream_t);
template EnvPlan<float> plan_envelopes<float>(const float *, const float *, int64_t, int, int,
                                              float *);
template EnvFns<float> envelope_fns<float>(bool);
template cudaError_t set_envelope_smem<float>(bool, size_t);

}  // namespace nndtw
