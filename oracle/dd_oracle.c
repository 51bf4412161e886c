/*
 * dd_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for time-series
 * discord discovery (Polyakov & Zymbler, "Parallel discord discovery in a time
 * series for the Intel Xeon Phi Knights Landing many-core processor",
 * arXiv:1901.00155).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  The product (the CUDA library)
 * shares no code with it and never calls it.
 *
 * Contents (each function cites the passage it follows):
 *   dd_oracle_znorm         Eq. 2 (z-normalisation of the whole series)
 *   dd_oracle_nn_rows       Section 2.1 definitions + Eq. 1: nearest non-self
 *                           match distance of selected subsequences (brute force)
 *   dd_oracle_nn_profile    the same for every subsequence
 *   dd_oracle_discord_brute Section 2.1 "discord" definition: argmax of the
 *                           nearest-neighbour profile ("O1")
 *   dd_oracle_window_stats  per-subsequence mean and centred sum of squares of
 *                           the normalised series (rows of the matrix of Eq. 5)
 *   dd_oracle_breakpoints   SAX breakpoints (text after Eq. 4)
 *   dd_oracle_sax           PAA (Eq. 3) + SAX (Eq. 4) + word hash (Eq. 9)
 *   dd_oracle_index         Freq (Eq. 8), Cand (Eq. 7), Index_Word (Eq. 10)
 *   dd_oracle_hotsax        Algorithms 2-4 (PhiDD: PotentialDiscord followed by
 *                           RefineDiscord) on the CPU ("O2")
 *   dd_oracle_window_mu_sigma, dd_oracle_dist2, dd_oracle_nn_rows_w,
 *   dd_oracle_nn_profile_w  the per-window z-normalised variant (each
 *                           subsequence normalised on its own; one reading of
 *                           Algorithm 2's Znormalize step), brute force
 *
 * Readings of the paper taken here (where it is silent, ambiguous or garbled):
 *   - Distances are plain Euclidean distances between subsequences of the
 *     globally z-normalised series (Eq. 2 normalises the whole series).
 *   - sigma^2 is computed two-pass, (1/m) sum (t - mu)^2, which is the same
 *     quantity as Eq. 2's (1/m) sum t^2 - mu^2 without its cancellation.
 *   - sigma == 0: the normalised series is identically 0.
 *   - Ties in the discord: the total order (nn^2, -index): the smallest index
 *     among equal maxima wins.
 *   - Every subsequence must have at least one non-self match: N >= 2n.
 *   - Algorithm 3's second inner loop is read as also updating the running
 *     minimum (as Algorithm 4 does).
 *   - Eq. 3 (PAA) is read with segment s covering [floor(s n / w),
 *     floor((s+1) n / w)) and the mean over it; Eq. 9 (hash) as the mixed
 *     radix number sum_s letter_s * A^(w-1-s) with 0-based letters.
 *   - PAA input: each subsequence z-normalised on its own (SAX's N(0,1)
 *     assumption, text after Eq. 4) -- mode 0; or the globally normalised
 *     values as they stand -- mode 1.  SAX only orders the search; it never
 *     changes its result.
 *   - Indices are 0-based.
 *   - Per-window variant: window mean and population sigma two-pass in FP64
 *     on the input values; a constant window (centred sum of squares exactly
 *     0) normalises to the zero vector.
 *
 * Parity pins for every function live in tests/ (hand examples, closed forms,
 * invariants, exact integer brute force, O1 == O2).  Nothing here is
 * "parity unpinned".
 *
 * Build: plain C99 + OpenMP, -ffp-contract=off so that x86_64 and aarch64
 * give identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENONFINITE 3

int dd_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check_args(const float* T, int64_t m, int32_t n) {
    if (!T || n < 1 || m < 1) return OR_EINVAL;
    if ((int64_t)n > m) return OR_EINVAL;
    int64_t N = m - n + 1;
    if (N < 2 * (int64_t)n) return OR_EINVAL; /* every row needs a non-self match */
    for (int64_t i = 0; i < m; i++)
        if (!isfinite(T[i])) return OR_ENONFINITE;
    return OR_OK;
}

/* Eq. 2: t^_i = (t_i - mu) / sigma, mu and sigma over the whole series. */
int dd_oracle_znorm(const float* T, int64_t m, double* that, double* mu_out, double* sigma_out) {
    if (!T || m < 1) return OR_EINVAL;
    double s = 0.0;
    for (int64_t i = 0; i < m; i++) s += (double)T[i];
    double mu = s / (double)m;
    double v = 0.0;
    for (int64_t i = 0; i < m; i++) {
        double d = (double)T[i] - mu;
        v += d * d;
    }
    double sigma = sqrt(v / (double)m);
    if (that) {
        for (int64_t i = 0; i < m; i++) that[i] = (sigma > 0.0) ? ((double)T[i] - mu) / sigma : 0.0;
    }
    if (mu_out) *mu_out = mu;
    if (sigma_out) *sigma_out = sigma;
    return OR_OK;
}

/* Eq. 1, squared: sum_k (x_k - y_k)^2 accumulated in k order. */
static double ed2(const double* x, const double* y, int32_t n) {
    double s = 0.0;
    for (int32_t k = 0; k < n; k++) {
        double d = x[k] - y[k];
        s += d * d;
    }
    return s;
}

/* Section 2.1: the nearest non-self match of subsequence i is the minimum of
 * Dist over all j with |i - j| >= n.  Brute force over every j. */
static double nn2_of_row(const double* t, int64_t N, int32_t n, int64_t i, int64_t* arg) {
    double best = INFINITY;
    int64_t barg = -1;
    for (int64_t j = 0; j < N; j++) {
        int64_t d = i > j ? i - j : j - i;
        if (d < n) continue;
        double s = ed2(t + i, t + j, n);
        if (s < best) {
            best = s;
            barg = j;
        }
    }
    if (arg) *arg = barg;
    return best;
}

int dd_oracle_nn_rows(const float* T, int64_t m, int32_t n, const int64_t* rows, int64_t k,
                      double* nn2, int64_t* argnn) {
    int st = check_args(T, m, n);
    if (st) return st;
    int64_t N = m - n + 1;
    for (int64_t r = 0; r < k; r++)
        if (rows[r] < 0 || rows[r] >= N) return OR_EINVAL;
    double* t = (double*)malloc(sizeof(double) * (size_t)m);
    if (!t) return OR_ENOMEM;
    dd_oracle_znorm(T, m, t, NULL, NULL);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < k; r++) {
        int64_t a = -1;
        nn2[r] = nn2_of_row(t, N, n, rows[r], &a);
        if (argnn) argnn[r] = a;
    }
    free(t);
    return OR_OK;
}

int dd_oracle_nn_profile(const float* T, int64_t m, int32_t n, double* nn2) {
    int st = check_args(T, m, n);
    if (st) return st;
    int64_t N = m - n + 1;
    double* t = (double*)malloc(sizeof(double) * (size_t)m);
    if (!t) return OR_ENOMEM;
    dd_oracle_znorm(T, m, t, NULL, NULL);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; i++) nn2[i] = nn2_of_row(t, N, n, i, NULL);
    free(t);
    return OR_OK;
}

/* Section 2.1, discord: the subsequence whose nearest non-self match is the
 * farthest.  Ties: smallest index.  Returns nn^2 (squared distance). */
int dd_oracle_discord_brute(const float* T, int64_t m, int32_t n, int64_t* idx, double* nn2_out) {
    int st = check_args(T, m, n);
    if (st) return st;
    int64_t N = m - n + 1;
    double* nn = (double*)malloc(sizeof(double) * (size_t)N);
    if (!nn) return OR_ENOMEM;
    st = dd_oracle_nn_profile(T, m, n, nn);
    if (st) {
        free(nn);
        return st;
    }
    int64_t best = 0;
    for (int64_t i = 1; i < N; i++)
        if (nn[i] > nn[best]) best = i;
    *idx = best;
    *nn2_out = nn[best];
    free(nn);
    return OR_OK;
}

/* Row i of the subsequence matrix (Eq. 5) over the normalised series: its
 * mean mu_i = (1/n) sum_k t^_{i+k} and its centred sum of squares
 * c_i = sum_k (t^_{i+k} - mu_i)^2.  Direct sums, no prefix sums. */
int dd_oracle_window_stats(const float* T, int64_t m, int32_t n, double* mu_w, double* c_w) {
    if (!T || n < 1 || (int64_t)n > m) return OR_EINVAL;
    int64_t N = m - n + 1;
    double* t = (double*)malloc(sizeof(double) * (size_t)m);
    if (!t) return OR_ENOMEM;
    dd_oracle_znorm(T, m, t, NULL, NULL);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        double s = 0.0;
        for (int32_t k = 0; k < n; k++) s += t[i + k];
        double mu = s / (double)n;
        double c = 0.0;
        for (int32_t k = 0; k < n; k++) {
            double d = t[i + k] - mu;
            c += d * d;
        }
        mu_w[i] = mu;
        c_w[i] = c;
    }
    free(t);
    return OR_OK;
}

/* Standard normal CDF via the C library's erfc: Phi(x) = erfc(-x/sqrt 2)/2. */
static double phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Breakpoints (text after Eq. 4): beta_1 < ... < beta_{A-1} cut N(0,1) into A
 * equiprobable regions, Phi(beta_j) = j / A.  The lower half is found by
 * bisection on Phi; N(0,1) is symmetric, so beta_{A-j} = -beta_j and, for
 * even A, the middle breakpoint is exactly 0. */
int dd_oracle_breakpoints(int32_t A, double* beta) {
    if (A < 2 || A > 64) return OR_EINVAL;
    for (int32_t j = 1; 2 * j < A; j++) {
        double target = (double)j / (double)A;
        double lo = -40.0, hi = 0.0;
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (phi(mid) < target)
                lo = mid;
            else
                hi = mid;
        }
        beta[j - 1] = 0.5 * (lo + hi);
        beta[A - j - 1] = -beta[j - 1];
    }
    if (A % 2 == 0) beta[A / 2 - 1] = 0.0;
    return OR_OK;
}

/* Eq. 3 (PAA) + Eq. 4 (SAX) + Eq. 9 (hash) for every subsequence.
 * paa_mode 0: each subsequence z-normalised on its own before PAA (a constant
 * subsequence becomes all zeros); paa_mode 1: the globally normalised values.
 * Letter s is the j in [0, A) with beta_{j-1} <= paa_s < beta_j (beta_{-1} =
 * -inf, beta_{A-1} = +inf); word code = sum_s letter_s * A^(w-1-s).
 * paa_out (optional): N*w segment values. */
int dd_oracle_sax(const float* T, int64_t m, int32_t n, int32_t w, int32_t A, int32_t paa_mode,
                  int32_t* code, double* paa_out) {
    if (!T || n < 1 || (int64_t)n > m || w < 1 || w > n || A < 2 || A > 64) return OR_EINVAL;
    if (paa_mode != 0 && paa_mode != 1) return OR_EINVAL;
    double dict = pow((double)A, (double)w);
    if (dict > 2147483647.0) return OR_EINVAL;
    int64_t N = m - n + 1;
    double* t = (double*)malloc(sizeof(double) * (size_t)m);
    double* beta = (double*)malloc(sizeof(double) * (size_t)A);
    if (!t || !beta) {
        free(t);
        free(beta);
        return OR_ENOMEM;
    }
    dd_oracle_znorm(T, m, t, NULL, NULL);
    dd_oracle_breakpoints(A, beta);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        const double* x = t + i;
        double mu = 0.0, sd = 1.0;
        if (paa_mode == 0) {
            double s = 0.0;
            for (int32_t k = 0; k < n; k++) s += x[k];
            mu = s / (double)n;
            double v = 0.0;
            for (int32_t k = 0; k < n; k++) {
                double d = x[k] - mu;
                v += d * d;
            }
            sd = sqrt(v / (double)n);
        }
        int32_t h = 0;
        for (int32_t s = 0; s < w; s++) {
            int64_t a = ((int64_t)s * n) / w, b = ((int64_t)(s + 1) * n) / w;
            double acc = 0.0;
            for (int64_t k = a; k < b; k++) acc += x[k];
            double seg = acc / (double)(b - a);
            double v;
            if (paa_mode == 0)
                v = (sd > 0.0) ? (seg - mu) / sd : 0.0;
            else
                v = seg;
            if (paa_out) paa_out[i * w + s] = v;
            int32_t letter = 0;
            while (letter < A - 1 && v >= beta[letter]) letter++;
            h = h * A + letter;
        }
        code[i] = h;
    }
    free(t);
    free(beta);
    return OR_OK;
}

/* Eq. 8: freq_i = number of rows whose word equals row i's word.
 * Eq. 7: Cand = rows whose frequency is the minimum, in ascending order.
 * Eq. 10: Index_Word row h = the rows with word h; stored as CSR buckets
 * (offsets[dict+1], members[N]) with members ascending inside a bucket. */
int dd_oracle_index(const int32_t* code, int64_t N, int32_t dict, int64_t* freq, int64_t* cand,
                    int64_t* ncand, int64_t* offsets, int64_t* members) {
    if (!code || N < 1 || dict < 1) return OR_EINVAL;
    int64_t* cnt = (int64_t*)calloc((size_t)dict, sizeof(int64_t));
    if (!cnt) return OR_ENOMEM;
    for (int64_t i = 0; i < N; i++) {
        if (code[i] < 0 || code[i] >= dict) {
            free(cnt);
            return OR_EINVAL;
        }
        cnt[code[i]]++;
    }
    int64_t fmin = INT64_MAX;
    for (int64_t i = 0; i < N; i++) {
        int64_t f = cnt[code[i]];
        if (freq) freq[i] = f;
        if (f < fmin) fmin = f;
    }
    int64_t nc = 0;
    for (int64_t i = 0; i < N; i++)
        if (cnt[code[i]] == fmin) {
            if (cand) cand[nc] = i;
            nc++;
        }
    if (ncand) *ncand = nc;
    if (offsets) {
        offsets[0] = 0;
        for (int32_t h = 0; h < dict; h++) offsets[h + 1] = offsets[h] + cnt[h];
        if (members) {
            int64_t* fill = (int64_t*)calloc((size_t)dict, sizeof(int64_t));
            if (!fill) {
                free(cnt);
                return OR_ENOMEM;
            }
            for (int64_t i = 0; i < N; i++) {
                int32_t h = code[i];
                members[offsets[h] + fill[h]] = i;
                fill[h]++;
            }
            free(fill);
        }
    }
    free(cnt);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * O2: Algorithms 2-4 on the CPU.
 *
 * best-so-far (bsf) is the pair (dist_bsf, pos_bsf) ordered by (dist, -pos):
 * a row whose full minimum equals dist_bsf replaces pos_bsf only if its index
 * is smaller, so the result is the same whatever order threads finish in and
 * equals the brute force's bit for bit (identical per-pair arithmetic, and the
 * minimum does not depend on visiting order).
 * A row is abandoned as soon as one distance is strictly below dist_bsf; such
 * a row's nearest-neighbour distance is below dist_bsf, so it cannot be the
 * discord.  Reading a stale (smaller) dist_bsf is safe: it only abandons later.
 * ------------------------------------------------------------------------- */
typedef struct {
    double dist;
    int64_t pos;
} bsf_t;

static double bsf_load(const double* p) {
    double v;
#pragma omp atomic read
    v = *p;
    return v;
}

static void bsf_store(double* p, double v) {
#pragma omp atomic write
    *p = v;
}

static int bsf_better(double d, int64_t i, const bsf_t* b) {
    return d > b->dist || (d == b->dist && (b->pos < 0 || i < b->pos));
}

/* Inner loops of Algorithms 3/4 for one row i: first the rows that share i's
 * SAX word (Index_Word row of i's word), then every other row in index order.
 * Returns 1 with *mn = full minimum if the row was not abandoned. */
static int scan_row(const double* t, int64_t N, int32_t n, int64_t i, const int32_t* code,
                    const int64_t* offsets, const int64_t* members, const double* bsf_dist,
                    double* mn, int64_t* evaluated) {
    double best = INFINITY;
    int32_t h = code[i];
    int64_t ev = 0;
    for (int64_t q = offsets[h]; q < offsets[h + 1]; q++) {
        int64_t j = members[q];
        int64_t d = i > j ? i - j : j - i;
        if (d < n) continue;
        double s = ed2(t + i, t + j, n);
        ev++;
        if (s < bsf_load(bsf_dist)) {
            *evaluated += ev;
            return 0;
        }
        if (s < best) best = s;
    }
    for (int64_t j = 0; j < N; j++) {
        if (code[j] == h) continue;
        int64_t d = i > j ? i - j : j - i;
        if (d < n) continue;
        double s = ed2(t + i, t + j, n);
        ev++;
        if (s < bsf_load(bsf_dist)) {
            *evaluated += ev;
            return 0;
        }
        if (s < best) best = s;
    }
    *evaluated += ev;
    *mn = best;
    return 1;
}

int dd_oracle_hotsax(const float* T, int64_t m, int32_t n, int32_t w, int32_t A, int32_t paa_mode,
                     int64_t* idx, double* nn2_out, int64_t* evaluated_pairs) {
    int st = check_args(T, m, n);
    if (st) return st;
    if (w < 1 || w > n || A < 2) return OR_EINVAL;
    double dictd = pow((double)A, (double)w);
    if (dictd > (double)(1 << 24)) return OR_EINVAL;
    int32_t dict = (int32_t)dictd;
    int64_t N = m - n + 1;
    double* t = (double*)malloc(sizeof(double) * (size_t)m);
    int32_t* code = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * (size_t)(dict + 1));
    int64_t* members = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    char* is_cand = (char*)calloc((size_t)N, 1);
    if (!t || !code || !cand || !offsets || !members || !is_cand) {
        st = OR_ENOMEM;
        goto done;
    }
    /* Algorithm 2, preparation stage. */
    dd_oracle_znorm(T, m, t, NULL, NULL);
    st = dd_oracle_sax(T, m, n, w, A, paa_mode, code, NULL);
    if (st) goto done;
    int64_t nc = 0;
    st = dd_oracle_index(code, N, dict, NULL, cand, &nc, offsets, members);
    if (st) goto done;
    for (int64_t q = 0; q < nc; q++) is_cand[cand[q]] = 1;

    bsf_t bsf = {0.0, -1};
    double bsf_dist = 0.0;
    int64_t ev_total = 0;

    /* Algorithm 3 (PotentialDiscord): candidates in ascending order. */
    for (int64_t q = 0; q < nc; q++) {
        int64_t i = cand[q];
        double mn;
        if (scan_row(t, N, n, i, code, offsets, members, &bsf_dist, &mn, &ev_total)) {
            if (bsf_better(mn, i, &bsf)) {
                bsf.dist = mn;
                bsf.pos = i;
                bsf_store(&bsf_dist, mn);
            }
        }
    }
    /* Algorithm 4 (RefineDiscord): every other row, dynamic schedule. */
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ev_total)
    for (int64_t i = 0; i < N; i++) {
        if (is_cand[i]) continue;
        double mn;
        int64_t ev = 0;
        if (scan_row(t, N, n, i, code, offsets, members, &bsf_dist, &mn, &ev)) {
#pragma omp critical(dd_oracle_bsf)
            {
                if (bsf_better(mn, i, &bsf)) {
                    bsf.dist = mn;
                    bsf.pos = i;
                    bsf_store(&bsf_dist, mn);
                }
            }
        }
        ev_total += ev;
    }
    *idx = bsf.pos;
    *nn2_out = bsf.dist;
    if (evaluated_pairs) *evaluated_pairs = ev_total;
    st = OR_OK;
done:
    free(t);
    free(code);
    free(cand);
    free(offsets);
    free(members);
    free(is_cand);
    return st;
}

/* ---------------------------------------------------------------------------
 * Per-window z-normalisation: the variant in which every subsequence is
 * normalised on its own (the usual HOTSAX convention, and one reading of
 * Algorithm 2's Znormalize step) instead of the whole series (Eq. 2).
 *
 * For the subsequence x_i = T[i .. i+n) of the INPUT series (float32 widened
 * exactly to FP64):
 *   mu_i    = (1/n) sum_k x_{i,k}                    (sum in k order)
 *   c_i     = sum_k (x_{i,k} - mu_i)^2               (two-pass, k order)
 *   sigma_i = sqrt(c_i / n)
 *   z_{i,k} = (x_{i,k} - mu_i) / sigma_i, and z_i = 0 when c_i == 0
 * (a constant subsequence becomes the zero vector; the paper is silent on
 * it).  The distance is Eq. 1 on z, squared: sum_k (z_{i,k} - z_{j,k})^2 in k
 * order.  Consequences used by the pins: 0 <= d^2 <= 4n; d^2 = 2n(1 - r_ij)
 * with r_ij the Pearson correlation of two non-constant subsequences; d^2 = n
 * between a constant and a non-constant one; d^2 = 0 between two constant
 * ones; d^2 is unchanged when T is replaced by a*T + b (a != 0).
 * ------------------------------------------------------------------------- */
static void window_mu_sigma(const float* T, int64_t N, int32_t n, double* mu, double* sg) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        double s = 0.0;
        for (int32_t k = 0; k < n; k++) s += (double)T[i + k];
        double mi = s / (double)n;
        double c = 0.0;
        for (int32_t k = 0; k < n; k++) {
            double d = (double)T[i + k] - mi;
            c += d * d;
        }
        mu[i] = mi;
        sg[i] = sqrt(c / (double)n); /* 0 exactly iff c == 0 */
    }
}

static double zval(const float* T, const double* mu, const double* sg, int64_t i, int32_t k) {
    return sg[i] > 0.0 ? ((double)T[i + k] - mu[i]) / sg[i] : 0.0;
}

static double ed2_w(const float* T, const double* mu, const double* sg, int64_t i, int64_t j, int32_t n) {
    double s = 0.0;
    for (int32_t k = 0; k < n; k++) {
        double d = zval(T, mu, sg, i, k) - zval(T, mu, sg, j, k);
        s += d * d;
    }
    return s;
}

static double nn2_of_row_w(const float* T, const double* mu, const double* sg, int64_t N, int32_t n, int64_t i,
                           int64_t* arg) {
    double best = INFINITY;
    int64_t barg = -1;
    for (int64_t j = 0; j < N; j++) {
        int64_t d = i > j ? i - j : j - i;
        if (d < n) continue;
        double s = ed2_w(T, mu, sg, i, j, n);
        if (s < best) {
            best = s;
            barg = j;
        }
    }
    if (arg) *arg = barg;
    return best;
}

/* Window statistics of the input series as defined above: mu_i and sigma_i. */
int dd_oracle_window_mu_sigma(const float* T, int64_t m, int32_t n, double* mu, double* sg) {
    if (!T || !mu || !sg || n < 1 || (int64_t)n > m) return OR_EINVAL;
    for (int64_t i = 0; i < m; i++)
        if (!isfinite(T[i])) return OR_ENONFINITE;
    window_mu_sigma(T, m - n + 1, n, mu, sg);
    return OR_OK;
}

/* Squared distance between subsequences i and j (any i, j in [0, N)).
 * znorm 0: Eq. 1 on the globally normalised series (Eq. 2); znorm 1: per
 * window, as defined above. */
int dd_oracle_dist2(const float* T, int64_t m, int32_t n, int32_t znorm, int64_t i, int64_t j, double* out) {
    if (!T || !out || n < 1 || (int64_t)n > m || (znorm != 0 && znorm != 1)) return OR_EINVAL;
    int64_t N = m - n + 1;
    if (i < 0 || j < 0 || i >= N || j >= N) return OR_EINVAL;
    for (int64_t q = 0; q < m; q++)
        if (!isfinite(T[q])) return OR_ENONFINITE;
    if (znorm == 0) {
        double* t = (double*)malloc(sizeof(double) * (size_t)m);
        if (!t) return OR_ENOMEM;
        dd_oracle_znorm(T, m, t, NULL, NULL);
        *out = ed2(t + i, t + j, n);
        free(t);
        return OR_OK;
    }
    double mu[2], sg[2];
    int64_t idx[2] = {i, j};
    for (int r = 0; r < 2; r++) window_mu_sigma(T + idx[r], 1, n, mu + r, sg + r);
    /* ed2_w on a two-entry table: entry 0 holds row i, entry 1 row j */
    double s = 0.0;
    for (int32_t k = 0; k < n; k++) {
        double a = sg[0] > 0.0 ? ((double)T[i + k] - mu[0]) / sg[0] : 0.0;
        double b = sg[1] > 0.0 ? ((double)T[j + k] - mu[1]) / sg[1] : 0.0;
        double d = a - b;
        s += d * d;
    }
    *out = s;
    return OR_OK;
}

/* Section 2.1 definitions with the per-window distance: nearest non-self
 * match (|i - j| >= n) of selected rows, brute force over every j. */
int dd_oracle_nn_rows_w(const float* T, int64_t m, int32_t n, const int64_t* rows, int64_t k, double* nn2,
                        int64_t* argnn) {
    int st = check_args(T, m, n);
    if (st) return st;
    int64_t N = m - n + 1;
    for (int64_t r = 0; r < k; r++)
        if (rows[r] < 0 || rows[r] >= N) return OR_EINVAL;
    double* mu = (double*)malloc(sizeof(double) * (size_t)N);
    double* sg = (double*)malloc(sizeof(double) * (size_t)N);
    if (!mu || !sg) {
        free(mu);
        free(sg);
        return OR_ENOMEM;
    }
    window_mu_sigma(T, N, n, mu, sg);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < k; r++) {
        int64_t a = -1;
        nn2[r] = nn2_of_row_w(T, mu, sg, N, n, rows[r], &a);
        if (argnn) argnn[r] = a;
    }
    free(mu);
    free(sg);
    return OR_OK;
}

int dd_oracle_nn_profile_w(const float* T, int64_t m, int32_t n, double* nn2) {
    int st = check_args(T, m, n);
    if (st) return st;
    int64_t N = m - n + 1;
    double* mu = (double*)malloc(sizeof(double) * (size_t)N);
    double* sg = (double*)malloc(sizeof(double) * (size_t)N);
    if (!mu || !sg) {
        free(mu);
        free(sg);
        return OR_ENOMEM;
    }
    window_mu_sigma(T, N, n, mu, sg);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; i++) nn2[i] = nn2_of_row_w(T, mu, sg, N, n, i, NULL);
    free(mu);
    free(sg);
    return OR_OK;
}
