/*
 * Plain FP64 CPU oracle for exact 1-NN classification under Sakoe-Chiba
 * windowed DTW with the LB_Enhanced^V lower bound
 * (Tan, Petitjean, Webb, "Elastic bands across the path", arXiv 1808.09617).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the bench's
 * CPU-baseline leg use it. It shares no code with the CUDA library.
 *
 * Every routine is written for a reader checking it against the paper by eye:
 * plain loops, no blocking, no fusion, double precision throughout, compiled
 * with -ffp-contract=off so that a*b+c is always two roundings.
 *
 * Conventions (readings of the paper, each listed in the design notes):
 *  - delta(a, b) = (a - b)^2, evaluated as d = a - b; t = d * d.  The paper
 *    calls delta an L2 norm but its Eq. 2 takes a square root over the sum of
 *    deltas and its proofs add deltas directly, so every distance and every
 *    bound here is in squared units (the square root is never taken).
 *  - Series are 0-based arrays in memory; the comments use the paper's
 *    1-based indices.
 *  - W is an integer with 0 <= W; W >= L-1 is the unconstrained DTW.
 *  - Ties in the 1-NN search go to the lowest training index.
 *
 * Parity status: every function below is pinned by the CPU tests against
 * closed forms, brute-force path enumeration, a library sliding-window filter
 * or the paper's theorems; none is "parity unpinned".
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double delta(double a, double b) {
    double d = a - b;
    double t = d * d;
    return t;
}

static double dmin(double x, double y) { return x < y ? x : y; }
static int imax(int x, int y) { return x > y ? x : y; }
static int imin(int x, int y) { return x < y ? x : y; }

/*
 * Upper and lower envelopes of B over window W (Sec. 2.2.3, Eq. 3-4):
 *   U_i = max_{max(1,i-W) <= j <= min(L,i+W)} B_j,
 *   Lo_i = min over the same window.
 * Naive scan of the window, O(L * W).
 */
void oracle_envelope(const double *B, int L, int W, double *U, double *Lo) {
    for (int i = 1; i <= L; i++) {
        int jlo = imax(1, i - W), jhi = imin(L, i + W);
        double u = B[jlo - 1], l = B[jlo - 1];
        for (int j = jlo; j <= jhi; j++) {
            if (B[j - 1] > u) u = B[j - 1];
            if (B[j - 1] < l) l = B[j - 1];
        }
        U[i - 1] = u;
        Lo[i - 1] = l;
    }
}

/*
 * Windowed DTW (Sec. 2.1, Eq. 1 with the warping window of Sec. 2.1):
 *   D(0,0) = 0, D(i,0) = D(0,j) = +inf for i, j >= 1,
 *   D(i,j) = delta(A_i, B_j) + min(D(i-1,j-1), D(i,j-1), D(i-1,j)) for |i-j| <= W,
 *   D(i,j) = +inf for |i-j| > W.
 * Returns D(L,L) (squared units).  If cutoff is finite, the evaluation stops
 * and returns +inf as soon as every cell of a row exceeds cutoff: every
 * warping path crosses every row (continuity) and D never decreases along a
 * path (delta >= 0), so D(L,L) > cutoff then.  Pass +inf for no early
 * abandoning.  Two rows of length L+1 are kept; cells outside the window are
 * +inf.
 */
static double dtw_rows(const double *A, const double *B, int L, int W,
                       double cutoff, double *prev, double *cur) {
    const double INF = INFINITY;
    prev[0] = 0.0;
    for (int j = 1; j <= L; j++) prev[j] = INF;
    for (int i = 1; i <= L; i++) {
        int jlo = imax(1, i - W), jhi = imin(L, i + W);
        cur[jlo - 1] = INF;
        double rowmin = INF;
        for (int j = jlo; j <= jhi; j++) {
            double m = dmin(dmin(prev[j - 1], cur[j - 1]), prev[j]);
            double t = delta(A[i - 1], B[j - 1]);
            cur[j] = t + m;
            if (cur[j] < rowmin) rowmin = cur[j];
        }
        if (jhi + 1 <= L) cur[jhi + 1] = INF;
        if (rowmin > cutoff) return INF;
        double *tmp = prev; prev = cur; cur = tmp;
    }
    return prev[L];
}

double oracle_dtw_abandon(const double *A, const double *B, int L, int W, double cutoff) {
    double *buf = (double *)malloc(sizeof(double) * 2 * (size_t)(L + 1));
    double r = dtw_rows(A, B, L, W, cutoff, buf, buf + (L + 1));
    free(buf);
    return r;
}

double oracle_dtw(const double *A, const double *B, int L, int W) {
    return oracle_dtw_abandon(A, B, L, W, INFINITY);
}

/* Squared Euclidean distance, sum_i delta(A_i, B_i) in index order (DTW_0). */
double oracle_ed(const double *A, const double *B, int L) {
    double s = 0.0;
    for (int i = 0; i < L; i++) s = s + delta(A[i], B[i]);
    return s;
}

/*
 * LB_Keogh (Sec. 2.2.3): sum over i = 1..L of
 *   delta(A_i, U_i) if A_i > U_i, delta(A_i, Lo_i) if A_i < Lo_i, else 0.
 */
double oracle_lb_keogh(const double *A, const double *U, const double *Lo, int L) {
    double res = 0.0;
    for (int i = 0; i < L; i++) {
        if (A[i] > U[i]) res = res + delta(A[i], U[i]);
        else if (A[i] < Lo[i]) res = res + delta(A[i], Lo[i]);
    }
    return res;
}

/*
 * LB_Enhanced^V_W(A, B) by Algorithm 1 of Sec. 3.1, in its order:
 *   res = delta(A_1,B_1) + delta(A_L,B_L); n_bands = min(L/2, V) (integer
 *   division); for i = 2..n_bands the minimum of the left band L_i (cells
 *   (i,j) and (j,i) for max(1,i-W) <= j <= i) and of the mirrored right band
 *   are added; if res >= D the bound returns +inf (abandon); otherwise the
 *   LB_Keogh terms for i = n_bands+1 .. L-n_bands are added.
 * Pass D = +inf for the plain bound of Eq. 7.  Requires L >= 2.
 */
double oracle_lb_enhanced(const double *A, const double *B, const double *U,
                          const double *Lo, int L, int W, int V, double D) {
    /* 1-based accessors: a(i) = A_i, b(i) = B_i */
#define a(i) A[(i) - 1]
#define b(i) B[(i) - 1]
    double res = delta(a(1), b(1)) + delta(a(L), b(L));
    int n_bands = imin(L / 2, V);
    for (int i = 2; i <= n_bands; i++) {
        double minL = delta(a(i), b(i));
        double minR = delta(a(L - i + 1), b(L - i + 1));
        for (int j = imax(1, i - W); j <= i - 1; j++) {
            minL = dmin(minL, delta(a(i), b(j)));
            minL = dmin(minL, delta(a(j), b(i)));
            minR = dmin(minR, delta(a(L - i + 1), b(L - j + 1)));
            minR = dmin(minR, delta(a(L - j + 1), b(L - i + 1)));
        }
        res = res + minL + minR;
    }
    if (res >= D) return INFINITY;
    for (int i = n_bands + 1; i <= L - n_bands; i++) {
        if (a(i) > U[i - 1]) res = res + delta(a(i), U[i - 1]);
        else if (a(i) < Lo[i - 1]) res = res + delta(a(i), Lo[i - 1]);
    }
    return res;
#undef a
#undef b
}

/*
 * LB_Enhanced^V_W(A, B) with its LB_Keogh bridge replaced by LB_Improved, the
 * combination that the conclusion (Sec. 5) proposes.  LB_Improved (Sec. 2.2.4)
 * adds to LB_Keogh(A, B) a second LB_Keogh: that of B against the envelope of
 * A', the projection of A onto B's envelope (Eq. 5).  Here both passes run
 * over the bridge only, i = n_bands+1 .. L-n_bands, so that the bands stay
 * as in Algorithm 1:
 *   res = LB_Enhanced^V_W(A, B)                 (ends, bands, first pass)
 *   A'_i = U_i if A_i > U_i, Lo_i if A_i < Lo_i, A_i otherwise, i = 1..L
 *   (U', Lo') = envelopes of A' over the window W (Eq. 3-4)
 *   res += sum_{j = n_bands+1 .. L-n_bands} LB_Keogh term of B_j against (U'_j, Lo'_j).
 * Requires L >= 2.
 */
double oracle_lb_enhanced_improved(const double *A, const double *B, const double *U,
                                   const double *Lo, int L, int W, int V) {
    double res = oracle_lb_enhanced(A, B, U, Lo, L, W, V, INFINITY);
    const int nb = imin(L / 2, V);   /* n_bands of Algorithm 1 */
    double *Ap = malloc(3 * sizeof(double) * (size_t)L);
    if (!Ap) return NAN;
    double *Up = Ap + L, *Lp = Ap + 2 * L;
    for (int i = 0; i < L; i++) {
        if (A[i] > U[i]) Ap[i] = U[i];
        else if (A[i] < Lo[i]) Ap[i] = Lo[i];
        else Ap[i] = A[i];
    }
    oracle_envelope(Ap, L, W, Up, Lp);
    for (int j = nb + 1; j <= L - nb; j++) {
        if (B[j - 1] > Up[j - 1]) res = res + delta(B[j - 1], Up[j - 1]);
        else if (B[j - 1] < Lp[j - 1]) res = res + delta(B[j - 1], Lp[j - 1]);
    }
    free(Ap);
    return res;
}

/*
 * LB_Improved_W(A, B) (Sec. 2.2.4): LB_Keogh_W(A, B) plus LB_Keogh_W(B, A'),
 * where A' is the projection of A onto B's envelope (Eq. 5) and the second
 * LB_Keogh is taken against the envelope of A' over the same window
 * (Eq. 3-4), both over i = 1..L:
 *   res = LB_Keogh(A against (U, Lo))
 *   A'_i = U_i if A_i > U_i, Lo_i if A_i < Lo_i, A_i otherwise
 *   (U', Lo') = envelopes of A' over W
 *   res += LB_Keogh(B against (U', Lo')).
 */
double oracle_lb_improved(const double *A, const double *B, const double *U,
                          const double *Lo, int L, int W) {
    double res = oracle_lb_keogh(A, U, Lo, L);
    double *Ap = malloc(3 * sizeof(double) * (size_t)L);
    if (!Ap) return NAN;
    double *Up = Ap + L, *Lp = Ap + 2 * L;
    for (int i = 0; i < L; i++) {
        if (A[i] > U[i]) Ap[i] = U[i];
        else if (A[i] < Lo[i]) Ap[i] = Lo[i];
        else Ap[i] = A[i];
    }
    oracle_envelope(Ap, L, W, Up, Lp);
    res = res + oracle_lb_keogh(B, Up, Lp, L);
    free(Ap);
    return res;
}

/*
 * LB_New_W(A, B) (Sec. 2.2.5): the two ends, which every warping path
 * contains (boundary condition), plus, for every i = 2..L-1, the smallest
 * delta(A_i, B_j) over the window max(1, i-W) <= j <= min(L, i+W), since the
 * path pairs A_i with at least one B_j there (continuity):
 *   res = delta(A_1, B_1) + delta(A_L, B_L) + sum_{i=2}^{L-1} min_j delta(A_i, B_j).
 * Naive scan of each window.  Requires L >= 2.
 */
double oracle_lb_new(const double *A, const double *B, int L, int W) {
    double res = delta(A[0], B[0]) + delta(A[L - 1], B[L - 1]);
    for (int i = 2; i <= L - 1; i++) {
        int jlo = imax(1, i - W), jhi = imin(L, i + W);
        double m = INFINITY;
        for (int j = jlo; j <= jhi; j++) m = dmin(m, delta(A[i - 1], B[j - 1]));
        res = res + m;
    }
    return res;
}

/* ------------------------------------------------------------------------ */
/* Threaded drivers over many pairs / queries (plain loops per item).        */

typedef struct {
    const double *test, *train, *U, *Lo;
    const int32_t *labels;
    int64_t Q, N;
    int L, W, V, kind;
    int64_t pair_lo, pair_hi; /* for matrix jobs: flat index range */
    const int32_t *pairs;     /* optional explicit (q, t) list */
    double *out;
    int32_t *nn_idx, *nn_label;
    double *nn_dist;
    int64_t *stats; /* per-thread slot of 3 counters */
    int exclude_self; /* leave-one-out: query q never matches training series q */
} job_t;

static void *lb_matrix_worker(void *p) {
    job_t *j = (job_t *)p;
    for (int64_t f = j->pair_lo; f < j->pair_hi; f++) {
        int64_t q = f / j->N, t = f % j->N;
        const double *A = j->test + q * j->L;
        const double *B = j->train + t * j->L;
        const double *U = j->U + t * j->L, *Lo = j->Lo + t * j->L;
        double v;
        if (j->kind == 1) v = oracle_lb_keogh(A, U, Lo, j->L);
        else if (j->kind == 2) v = oracle_lb_enhanced_improved(A, B, U, Lo, j->L, j->W, j->V);
        else if (j->kind == 3) v = oracle_lb_improved(A, B, U, Lo, j->L, j->W);
        else if (j->kind == 4) v = oracle_lb_new(A, B, j->L, j->W);
        else v = oracle_lb_enhanced(A, B, U, Lo, j->L, j->W, j->V, INFINITY);
        j->out[f] = v;
    }
    return NULL;
}

static void *dtw_pairs_worker(void *p) {
    job_t *j = (job_t *)p;
    for (int64_t f = j->pair_lo; f < j->pair_hi; f++) {
        int64_t q, t;
        if (j->pairs) { q = j->pairs[2 * f]; t = j->pairs[2 * f + 1]; }
        else { q = f / j->N; t = f % j->N; }
        j->out[f] = oracle_dtw(j->test + q * j->L, j->train + t * j->L, j->L, j->W);
    }
    return NULL;
}

/* 1-NN by brute force: argmin over all training series of DTW_W, ties to the
 * lowest index (strict < keeps the first minimum). */
static void *nn_brute_worker(void *p) {
    job_t *j = (job_t *)p;
    for (int64_t q = j->pair_lo; q < j->pair_hi; q++) {
        const double *A = j->test + q * j->L;
        double best = INFINITY;
        int64_t bi = -1;
        for (int64_t t = 0; t < j->N; t++) {
            if (j->exclude_self && t == q) continue;
            double d = oracle_dtw(A, j->train + t * j->L, j->L, j->W);
            if (d < best) { best = d; bi = t; }
        }
        j->nn_idx[q] = (int32_t)bi;
        j->nn_label[q] = j->labels[bi];
        j->nn_dist[q] = best;
    }
    return NULL;
}

/* Stable ordering of training indices by ascending Euclidean distance. */
typedef struct { double key; int64_t idx; } keyed_t;
static int keyed_cmp(const void *x, const void *y) {
    const keyed_t *a = (const keyed_t *)x, *b = (const keyed_t *)y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/*
 * The paper's NN-DTW lower-bound search (Sec. 4): candidates are visited in
 * ascending Euclidean distance to the query, starting from the nearest; each
 * is bounded by LB_Enhanced^V (Algorithm 1) against the current NN distance D
 * and, if not pruned, DTW_W is computed with early abandoning against D.
 * Reading for the lowest-index tie rule: a candidate is pruned or abandoned
 * only when its bound is strictly greater than D, so a candidate whose DTW
 * equals D is still evaluated and wins if its index is lower.  Algorithm 1's
 * "res >= D" test is kept as printed and called with the next double above
 * D, which makes it the strict test "res > D".
 * stats[0] = pairs pruned by the bound, stats[1] = DTWs abandoned,
 * stats[2] = DTWs run to completion.
 */
static void *nn_pruned_worker(void *p) {
    job_t *j = (job_t *)p;
    keyed_t *ord = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)j->N);
    double *rows = (double *)malloc(sizeof(double) * 2 * (size_t)(j->L + 1));
    for (int64_t q = j->pair_lo; q < j->pair_hi; q++) {
        const double *A = j->test + q * j->L;
        for (int64_t t = 0; t < j->N; t++) {
            ord[t].key = oracle_ed(A, j->train + t * j->L, j->L);
            ord[t].idx = t;
        }
        qsort(ord, (size_t)j->N, sizeof(keyed_t), keyed_cmp);
        double D = INFINITY;
        int64_t bi = -1;
        for (int64_t r = 0; r < j->N; r++) {
            int64_t t = ord[r].idx;
            const double *B = j->train + t * j->L;
            double lb = oracle_lb_enhanced(A, B, j->U + t * j->L, j->Lo + t * j->L,
                                           j->L, j->W, j->V, nextafter(D, INFINITY));
            if (lb > D) { j->stats[0]++; continue; }
            double d = dtw_rows(A, B, j->L, j->W, D, rows, rows + (j->L + 1));
            if (isinf(d)) { j->stats[1]++; continue; }
            j->stats[2]++;
            if (d < D || (d == D && t < bi)) { D = d; bi = t; }
        }
        j->nn_idx[q] = (int32_t)bi;
        j->nn_label[q] = j->labels[bi];
        j->nn_dist[q] = D;
    }
    free(rows);
    free(ord);
    return NULL;
}

static void run_threads(void *(*fn)(void *), job_t *base, int64_t total, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > total) nthreads = (int)(total > 0 ? total : 1);
    pthread_t th[256];
    job_t jobs[256];
    int64_t chunk = (total + nthreads - 1) / nthreads;
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = *base;
        jobs[k].pair_lo = (int64_t)k * chunk;
        jobs[k].pair_hi = jobs[k].pair_lo + chunk < total ? jobs[k].pair_lo + chunk : total;
        if (jobs[k].stats) jobs[k].stats = base->stats + 3 * k;
        pthread_create(&th[k], NULL, fn, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
}

/* Envelopes of N series (row-major [N][L]). */
void oracle_envelopes(const double *train, int64_t N, int L, int W, double *U, double *Lo) {
    for (int64_t t = 0; t < N; t++)
        oracle_envelope(train + t * L, L, W, U + t * L, Lo + t * L);
}

/* out[q*N + t] = LB(test_q, train_t); kind 0 = LB_Enhanced^V, 1 = LB_Keogh,
 * 2 = LB_Enhanced^V with the LB_Improved bridge, 3 = LB_Improved, 4 = LB_New. */
void oracle_lb_matrix(const double *test, int64_t Q, const double *train,
                      const double *U, const double *Lo, int64_t N, int L, int W,
                      int V, int kind, double *out, int nthreads) {
    job_t b = {0};
    b.test = test; b.train = train; b.U = U; b.Lo = Lo; b.Q = Q; b.N = N;
    b.L = L; b.W = W; b.V = V; b.kind = kind; b.out = out;
    run_threads(lb_matrix_worker, &b, Q * N, nthreads);
}

/* out[p] = DTW_W(test_{pairs[2p]}, train_{pairs[2p+1]}); pairs == NULL means
 * the full Q x N matrix in row-major order. */
void oracle_dtw_pairs(const double *test, const double *train, int64_t N,
                      const int32_t *pairs, int64_t P, int L, int W, double *out,
                      int nthreads) {
    job_t b = {0};
    b.test = test; b.train = train; b.N = N; b.pairs = pairs; b.L = L; b.W = W;
    b.out = out;
    run_threads(dtw_pairs_worker, &b, P, nthreads);
}

void oracle_nn_brute(const double *train, const int32_t *labels, int64_t N,
                     const double *test, int64_t Q, int L, int W, int32_t *nn_idx,
                     int32_t *nn_label, double *nn_dist, int nthreads) {
    job_t b = {0};
    b.test = test; b.train = train; b.labels = labels; b.Q = Q; b.N = N;
    b.L = L; b.W = W; b.nn_idx = nn_idx; b.nn_label = nn_label; b.nn_dist = nn_dist;
    run_threads(nn_brute_worker, &b, Q, nthreads);
}

/* Leave-one-out 1-NN on a training set (used to learn W, Sec. 1 and 4): the
 * nearest neighbour of each training series among all the others, by brute
 * force, ties to the lowest index. */
void oracle_nn_loo(const double *train, const int32_t *labels, int64_t N, int L, int W,
                   int32_t *nn_idx, int32_t *nn_label, double *nn_dist, int nthreads) {
    job_t b = {0};
    b.test = train; b.train = train; b.labels = labels; b.Q = N; b.N = N;
    b.L = L; b.W = W; b.nn_idx = nn_idx; b.nn_label = nn_label; b.nn_dist = nn_dist;
    b.exclude_self = 1;
    run_threads(nn_brute_worker, &b, N, nthreads);
}

void oracle_nn_pruned(const double *train, const int32_t *labels, const double *U,
                      const double *Lo, int64_t N, const double *test, int64_t Q,
                      int L, int W, int V, int32_t *nn_idx, int32_t *nn_label,
                      double *nn_dist, int64_t *stats3, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int64_t *st = (int64_t *)calloc(3 * 256, sizeof(int64_t));
    job_t b = {0};
    b.test = test; b.train = train; b.labels = labels; b.U = U; b.Lo = Lo;
    b.Q = Q; b.N = N; b.L = L; b.W = W; b.V = V;
    b.nn_idx = nn_idx; b.nn_label = nn_label; b.nn_dist = nn_dist; b.stats = st;
    run_threads(nn_pruned_worker, &b, Q, nthreads);
    stats3[0] = stats3[1] = stats3[2] = 0;
    for (int k = 0; k < 256; k++) {
        stats3[0] += st[3 * k]; stats3[1] += st[3 * k + 1]; stats3[2] += st[3 * k + 2];
    }
    free(st);
}

/* ------------------------------------------------------------------------ */
/* Unequal lengths (Sec. 2: the equal-length exposition generalises).        */
/*
 * Reading: A has L_A points and B has L_B (both >= 2).  DTW is Eq. 1 on the
 * L_A x L_B grid inside the window |i - j| <= W, ending at (L_A, L_B); when
 * |L_A - L_B| > W no warping path fits the window and the distance is +inf.
 * B's envelope is taken for the rows of A (i up to L_B + W); the bounds follow
 * Eq. 7 with the end corner at (L_A, L_B) and n_bands = min(min(L_A, L_B)/2, V).
 * With L_A = L_B every routine below computes what its equal-length
 * counterpart above computes, in the same order.
 */

static int in_window(int i, int j, int W) { return i - j <= W && j - i <= W; }

/* U_i, Lo_i = max, min of B_j over max(1, i-W) <= j <= min(LB, i+W), for
 * i = 1..E (Eq. 3-4 for the rows of a series of up to E points); requires
 * E <= LB + W, so that every window holds at least one point of B. */
void oracle_envelope_var(const double *B, int LB, int W, int E, double *U, double *Lo) {
    for (int i = 1; i <= E; i++) {
        int jlo = imax(1, i - W), jhi = imin(LB, i + W);
        double u = B[jlo - 1], l = B[jlo - 1];
        for (int j = jlo; j <= jhi; j++) {
            if (B[j - 1] > u) u = B[j - 1];
            if (B[j - 1] < l) l = B[j - 1];
        }
        U[i - 1] = u;
        Lo[i - 1] = l;
    }
}

/* DTW_W(A, B) on the LA x LB grid (Eq. 1), row by row over the rows of A, with
 * the same early abandoning as dtw_rows (every path crosses every row of A). */
static double dtw_rows_var(const double *A, int LA, const double *B, int LB, int W,
                           double cutoff, double *prev, double *cur) {
    const double INF = INFINITY;
    if (!in_window(LA, LB, W)) return INF;
    prev[0] = 0.0;
    for (int j = 1; j <= LB; j++) prev[j] = INF;
    for (int i = 1; i <= LA; i++) {
        int jlo = imax(1, i - W), jhi = imin(LB, i + W);
        cur[jlo - 1] = INF;
        double rowmin = INF;
        for (int j = jlo; j <= jhi; j++) {
            double m = dmin(dmin(prev[j - 1], cur[j - 1]), prev[j]);
            double t = delta(A[i - 1], B[j - 1]);
            cur[j] = t + m;
            if (cur[j] < rowmin) rowmin = cur[j];
        }
        if (jhi + 1 <= LB) cur[jhi + 1] = INF;
        if (rowmin > cutoff) return INF;
        double *tmp = prev; prev = cur; cur = tmp;
    }
    return prev[LB];
}

double oracle_dtw_var(const double *A, int LA, const double *B, int LB, int W, double cutoff) {
    double *buf = (double *)malloc(sizeof(double) * 2 * (size_t)(LB + 1));
    double r = dtw_rows_var(A, LA, B, LB, W, cutoff, buf, buf + (LB + 1));
    free(buf);
    return r;
}

/* LB_Keogh over the LA rows of A against B's envelope (U, Lo) for those rows;
 * +inf when |LA - LB| > W (no path). */
double oracle_lb_keogh_var(const double *A, int LA, int LB, const double *U,
                           const double *Lo, int W) {
    if (!in_window(LA, LB, W)) return INFINITY;
    return oracle_lb_keogh(A, U, Lo, LA);
}

/* LB_Enhanced^V_W(A, B) for LA != LB: Algorithm 1's steps with the right bands
 * anchored at the end corner (LA, LB) and every band cell kept only inside
 * the window; the bridge is LB_Keogh over rows n_bands+1 .. LA-n_bands.  D as
 * in oracle_lb_enhanced; +inf when |LA - LB| > W. */
double oracle_lb_enhanced_var(const double *A, int LA, const double *B, int LB,
                              const double *U, const double *Lo, int W, int V, double D) {
    if (!in_window(LA, LB, W)) return INFINITY;
#define a(i) A[(i) - 1]
#define b(j) B[(j) - 1]
    double res = delta(a(1), b(1)) + delta(a(LA), b(LB));
    int n_bands = imin(imin(LA, LB) / 2, V);
    for (int i = 2; i <= n_bands; i++) {
        double minL = delta(a(i), b(i));
        double minR = delta(a(LA - i + 1), b(LB - i + 1));
        for (int j = 1; j <= i - 1; j++) {
            if (in_window(i, j, W)) {
                minL = dmin(minL, delta(a(i), b(j)));
                minL = dmin(minL, delta(a(j), b(i)));
            }
            if (in_window(LA - i + 1, LB - j + 1, W))
                minR = dmin(minR, delta(a(LA - i + 1), b(LB - j + 1)));
            if (in_window(LA - j + 1, LB - i + 1, W))
                minR = dmin(minR, delta(a(LA - j + 1), b(LB - i + 1)));
        }
        res = res + minL + minR;
    }
    if (res >= D) return INFINITY;
    for (int i = n_bands + 1; i <= LA - n_bands; i++) {
        if (a(i) > U[i - 1]) res = res + delta(a(i), U[i - 1]);
        else if (a(i) < Lo[i - 1]) res = res + delta(a(i), Lo[i - 1]);
    }
    return res;
#undef a
#undef b
}

/* Ragged sets: series k is x[off[k] .. off[k+1]); envelope of training
 * series t at env + eoff[t], eoff[t] = off[t] + t * W (L_t + W rows). */
typedef struct {
    const double *test, *train, *U, *Lo;
    const int64_t *toff, *off, *eoff;
    const int32_t *labels;
    int64_t Q, N;
    int W, V, kind;
    int64_t lo, hi;
    double *out;
    int32_t *nn_idx, *nn_label;
    double *nn_dist;
    int64_t *stats;
} vjob_t;

#define VLEN(o, k) ((int)((o)[(k) + 1] - (o)[k]))

static void *lb_matrix_var_worker(void *p) {
    vjob_t *j = (vjob_t *)p;
    for (int64_t f = j->lo; f < j->hi; f++) {
        int64_t q = f / j->N, t = f % j->N;
        const double *A = j->test + j->toff[q], *B = j->train + j->off[t];
        int LA = VLEN(j->toff, q), LB = VLEN(j->off, t);
        const double *U = j->U + j->eoff[t], *Lo = j->Lo + j->eoff[t];
        j->out[f] = j->kind == 1 ? oracle_lb_keogh_var(A, LA, LB, U, Lo, j->W)
                                 : oracle_lb_enhanced_var(A, LA, B, LB, U, Lo, j->W, j->V,
                                                          INFINITY);
    }
    return NULL;
}

static void *dtw_matrix_var_worker(void *p) {
    vjob_t *j = (vjob_t *)p;
    for (int64_t f = j->lo; f < j->hi; f++) {
        int64_t q = f / j->N, t = f % j->N;
        j->out[f] = oracle_dtw_var(j->test + j->toff[q], VLEN(j->toff, q),
                                   j->train + j->off[t], VLEN(j->off, t), j->W, INFINITY);
    }
    return NULL;
}

/* 1-NN by exhaustive DTW, ties to the lowest index; -1 (index and label)
 * when no training series is within the window. */
static void *nn_brute_var_worker(void *p) {
    vjob_t *j = (vjob_t *)p;
    for (int64_t q = j->lo; q < j->hi; q++) {
        const double *A = j->test + j->toff[q];
        int LA = VLEN(j->toff, q);
        double best = INFINITY;
        int64_t bi = -1;
        for (int64_t t = 0; t < j->N; t++) {
            double d = oracle_dtw_var(A, LA, j->train + j->off[t], VLEN(j->off, t), j->W,
                                      INFINITY);
            if (d < best) { best = d; bi = t; }
        }
        j->nn_idx[q] = (int32_t)bi;
        j->nn_label[q] = bi < 0 ? -1 : j->labels[bi];
        j->nn_dist[q] = best;
    }
    return NULL;
}

/* The lower-bound search (Sec. 4) for unequal lengths: candidates in ascending
 * LB_Enhanced order (the Euclidean order is undefined), each bounded by
 * Algorithm 1 against the current D and, if not pruned, its DTW computed with
 * early abandoning; the same strict tests and tie rule as nn_pruned_worker. */
static void *nn_pruned_var_worker(void *p) {
    vjob_t *j = (vjob_t *)p;
    keyed_t *ord = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)j->N);
    int maxlb = 1;
    for (int64_t t = 0; t < j->N; t++) maxlb = imax(maxlb, VLEN(j->off, t));
    double *rows = (double *)malloc(sizeof(double) * 2 * (size_t)(maxlb + 1));
    for (int64_t q = j->lo; q < j->hi; q++) {
        const double *A = j->test + j->toff[q];
        int LA = VLEN(j->toff, q);
        for (int64_t t = 0; t < j->N; t++) {
            ord[t].key = oracle_lb_enhanced_var(A, LA, j->train + j->off[t], VLEN(j->off, t),
                                                j->U + j->eoff[t], j->Lo + j->eoff[t], j->W,
                                                j->V, INFINITY);
            ord[t].idx = t;
        }
        qsort(ord, (size_t)j->N, sizeof(keyed_t), keyed_cmp);
        double D = INFINITY;
        int64_t bi = -1;
        for (int64_t r = 0; r < j->N; r++) {
            int64_t t = ord[r].idx;
            const double *B = j->train + j->off[t];
            int LB = VLEN(j->off, t);
            if (!in_window(LA, LB, j->W)) { j->stats[0]++; continue; }
            double lb = oracle_lb_enhanced_var(A, LA, B, LB, j->U + j->eoff[t],
                                               j->Lo + j->eoff[t], j->W, j->V,
                                               nextafter(D, INFINITY));
            if (lb > D) { j->stats[0]++; continue; }
            double d = dtw_rows_var(A, LA, B, LB, j->W, D, rows, rows + (LB + 1));
            if (isinf(d)) { j->stats[1]++; continue; }
            j->stats[2]++;
            if (d < D || (d == D && t < bi)) { D = d; bi = t; }
        }
        j->nn_idx[q] = (int32_t)bi;
        j->nn_label[q] = bi < 0 ? -1 : j->labels[bi];
        j->nn_dist[q] = D;
    }
    free(rows);
    free(ord);
    return NULL;
}

static void run_vthreads(void *(*fn)(void *), vjob_t *base, int64_t total, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > total) nthreads = (int)(total > 0 ? total : 1);
    pthread_t th[256];
    vjob_t jobs[256];
    int64_t chunk = (total + nthreads - 1) / nthreads;
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = *base;
        jobs[k].lo = (int64_t)k * chunk;
        jobs[k].hi = jobs[k].lo + chunk < total ? jobs[k].lo + chunk : total;
        if (jobs[k].stats) jobs[k].stats = base->stats + 3 * k;
        pthread_create(&th[k], NULL, fn, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
}

/* Envelopes of a ragged training set, L_t + W rows each at eoff[t]. */
void oracle_envelopes_var(const double *train, const int64_t *off, int64_t N, int W,
                          const int64_t *eoff, double *U, double *Lo) {
    for (int64_t t = 0; t < N; t++)
        oracle_envelope_var(train + off[t], VLEN(off, t), W, VLEN(off, t) + W,
                            U + eoff[t], Lo + eoff[t]);
}

/* out[q*N + t] = LB(test_q, train_t): kind 0 = LB_Enhanced^V, 1 = LB_Keogh. */
void oracle_lb_matrix_var(const double *test, const int64_t *toff, int64_t Q,
                          const double *train, const int64_t *off, const double *U,
                          const double *Lo, const int64_t *eoff, int64_t N, int W, int V,
                          int kind, double *out, int nthreads) {
    vjob_t b = {0};
    b.test = test; b.toff = toff; b.Q = Q; b.train = train; b.off = off; b.U = U; b.Lo = Lo;
    b.eoff = eoff; b.N = N; b.W = W; b.V = V; b.kind = kind; b.out = out;
    run_vthreads(lb_matrix_var_worker, &b, Q * N, nthreads);
}

/* out[q*N + t] = DTW_W(test_q, train_t). */
void oracle_dtw_matrix_var(const double *test, const int64_t *toff, int64_t Q,
                           const double *train, const int64_t *off, int64_t N, int W,
                           double *out, int nthreads) {
    vjob_t b = {0};
    b.test = test; b.toff = toff; b.Q = Q; b.train = train; b.off = off; b.N = N; b.W = W;
    b.out = out;
    run_vthreads(dtw_matrix_var_worker, &b, Q * N, nthreads);
}

void oracle_nn_brute_var(const double *train, const int64_t *off, const int32_t *labels,
                         int64_t N, const double *test, const int64_t *toff, int64_t Q, int W,
                         int32_t *nn_idx, int32_t *nn_label, double *nn_dist, int nthreads) {
    vjob_t b = {0};
    b.train = train; b.off = off; b.labels = labels; b.N = N; b.test = test; b.toff = toff;
    b.Q = Q; b.W = W; b.nn_idx = nn_idx; b.nn_label = nn_label; b.nn_dist = nn_dist;
    run_vthreads(nn_brute_var_worker, &b, Q, nthreads);
}

void oracle_nn_pruned_var(const double *train, const int64_t *off, const int32_t *labels,
                          const double *U, const double *Lo, const int64_t *eoff, int64_t N,
                          const double *test, const int64_t *toff, int64_t Q, int W, int V,
                          int32_t *nn_idx, int32_t *nn_label, double *nn_dist,
                          int64_t *stats3, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int64_t *st = (int64_t *)calloc(3 * 256, sizeof(int64_t));
    vjob_t b = {0};
    b.train = train; b.off = off; b.labels = labels; b.U = U; b.Lo = Lo; b.eoff = eoff;
    b.N = N; b.test = test; b.toff = toff; b.Q = Q; b.W = W; b.V = V;
    b.nn_idx = nn_idx; b.nn_label = nn_label; b.nn_dist = nn_dist; b.stats = st;
    run_vthreads(nn_pruned_var_worker, &b, Q, nthreads);
    stats3[0] = stats3[1] = stats3[2] = 0;
    for (int k = 0; k < 256; k++) {
        stats3[0] += st[3 * k]; stats3[1] += st[3 * k + 1]; stats3[2] += st[3 * k + 2];
    }
    free(st);
}
