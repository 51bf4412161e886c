/*
 * dd.h -- C ABI of the GB300 discord-discovery library (libdd.so).
 *
 * Problem (Polyakov & Zymbler, arXiv:1901.00155, Section 2.1 and Eq. 1-2):
 * given a series T = (t_0 .. t_{m-1}) and a subsequence length n, let
 * N = m - n + 1 and let T_i = (t^_i .. t^_{i+n-1}) be the i-th subsequence of
 * the series z-normalised as a whole (Eq. 2: t^ = (t - mu) / sigma, mu and the
 * population sigma over all m points; sigma == 0 gives t^ == 0).  Two
 * subsequences are a non-self match when |i - j| >= n.  The nearest-neighbour
 * distance of T_i is nn_i = min_{|i-j|>=n} ED(T_i, T_j) (Eq. 1), and the discord
 * is the i maximising nn_i; ties go to the smallest i.  Indices are 0-based
 * (the paper counts from 1).
 *
 * The search follows PhiDD (Algorithms 2-4): SAX words (Eq. 3-4, Eq. 9) order
 * the rows -- the rarest words (Cand, Eq. 7) are searched first
 * (PotentialDiscord, Algorithm 3), then every other row (RefineDiscord,
 * Algorithm 4), each row scanning the rows that share its word (Index_Word,
 * Eq. 10) first and being abandoned as soon as one distance falls below the
 * best-so-far.  The ordering only changes the speed, never the result.
 *
 * Conventions for every entry point
 *   - Device pointers are CUDA device addresses of the current device; the
 *     caller owns them and keeps them valid and unmodified until the call's
 *     work on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Errors are returned as dd_status_t; nothing is printed and nothing
 *     aborts the process.  After DD_ECUDA the plan should be destroyed.
 *   - A plan holds per-(m, n, options) device workspace and serves one call at
 *     a time: a call on a plan whose previous call is still being set up on
 *     another host thread returns DD_EBUSY.  Calls on one plan must be ordered
 *     on one stream (or synchronised by the caller).
 *   - Valid problems need n >= 1 and N >= 2n (m >= 3n - 1), so that every
 *     subsequence has at least one non-self match; otherwise DD_EINVAL.
 *   - A series holding NaN or +-Inf gives DD_ENONFINITE.
 */
#ifndef DD_H_
#define DD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DD_API __attribute__((visibility("default")))
#else
#define DD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_plan_s* dd_plan_t;

typedef enum {
    DD_OK = 0,
    DD_EINVAL = 1,      /* bad sizes, null pointers, bad options */
    DD_ENOMEM = 2,      /* device (or pinned host) allocation failed / workspace too small */
    DD_ENONFINITE = 3,  /* T holds NaN or Inf */
    DD_ETIMEOUT = 4,    /* a bounded device-side wait expired */
    DD_ECUDA = 5,       /* any other CUDA runtime error */
    DD_EBUSY = 6,       /* the plan is in use by another host thread */
    DD_ENOTSUP = 7      /* option combination not supported for these sizes (tensor-core
                           forms for n > 65536; per-window with a tensor-core precision or
                           shards; diagonal-recurrence workspace for N > 2^26), or a wave
                           with more than 2^31 work items (its 32-bit work counter would
                           wrap; the wave stops and the call reports this status) */
} dd_status_t;

/* Arithmetic of the distance tiles.
 *   DD_FP32     direct differences sum_k (x_k - y_k)^2 in FP32 on the CUDA cores
 *               (Eq. 1 squared); nn_distance within ~1e-5 relative.
 *   DD_TC_FP16  Gram tiles <x', y'> of mean-centred rows on the tcgen05 tensor
 *   DD_TC_BF16  cores (FP16 / BF16 operands, FP32 accumulation), a rigorous
 *               error bound per row, and exact FP64 rescoring of every row the
 *               bound cannot rule out: exact index, FP64 distance. */
typedef enum { DD_FP32 = 0, DD_TC_FP16 = 1, DD_TC_BF16 = 2 } dd_precision_t;

typedef struct {
    int32_t precision;     /* dd_precision_t (default DD_FP32) */
    int32_t paa_w;         /* PAA segments per word, Eq. 3 (default 4; min(paa_w, n) is used) */
    int32_t alphabet;      /* SAX alphabet size, Eq. 4 (default 4); alphabet^paa_w <= 4096 */
    int32_t early_abandon; /* 1 = abandon rows against the best-so-far (default); 0 = full scans */
    int32_t paa_mode;      /* 0 = PAA of each subsequence z-normalised on its own (default),
                              1 = PAA of the globally normalised values */
    int32_t phase1_max;    /* at most this many Cand rows run in phase 1 (default 4096) */
    int32_t refine_k;      /* rows with the largest first-wave upper bounds that get a full scan
                              before the other survivors, to raise the best-so-far (default 128).
                              When more than refine_k rows then survive, they also run the
                              time-local wave and refine_k of them, ranked again, a second full
                              scan; 0 = skip both */
    int32_t local_cols;    /* first wave: every row scans the rows of nearest window mean, this many
                              on each side of its tile (default 64: with a 128-row tile, two
                              128-column tiles of the FP32 kernel; FP32 form -- the tensor-core
                              form's first wave is one 128 x 256 band tile per row tile); 0 = no
                              first wave */
    int32_t word_cols;     /* same-word wave (FP32 form): survivors scan this many rows sharing their
                              SAX word (Index_Word, Eq. 10) before their full scans; 0 = skip
                              (default 512) */
    int32_t shard_count;   /* row sharding (multi-GPU, one process per GPU): 0 or 1 = every row.
                              With G > 1 the search considers only the rows of shard shard_index:
                              positions [floor(k N / G), floor((k + 1) N / G)) of the mean-bucketed
                              visit order (every row still scans all columns).  The series' discord
                              is the shard result with the largest nn_distance, ties to the
                              smallest index -- one all-gather of (nn_distance, index) */
    int32_t shard_index;   /* k in [0, G) (default 0) */
    int32_t znorm;         /* 0 = the whole series is z-normalised (Eq. 2; default).
                              1 = every subsequence is z-normalised on its own (window mean and
                              population sigma of the input values, two-pass FP64; a constant
                              subsequence becomes the zero vector), the usual HOTSAX convention.
                              Every window then has mean 0, so the mean-order lower bound of the
                              search is void: per-window plans find the discord from the
                              exhaustive diagonal-recurrence profile (see dd_nn_profile_diag), a
                              rigorous FP32 bound per row and exact FP64 rescoring of every row
                              the bound cannot rule out -- exact index and FP64 distance.
                              Requires DD_FP32 and shard_count <= 1 (else DD_ENOTSUP); the SAX
                              and wave options do not apply */
    int32_t diag;          /* 1 = also hold the workspace of dd_nn_profile_diag (implied by
                              znorm = 1; default 0) */
    int32_t reserved[3];   /* must be zero */
} dd_options_t;

typedef struct {
    int64_t index;          /* 0-based start of the discord (-1 if status != DD_OK) */
    double nn_distance;     /* ED from the discord to its nearest non-self match, on the
                               z-normalised series */
    int32_t status;         /* dd_status_t of the call that produced it */
    int32_t exact;          /* 1: nn_distance is an FP64 rescore (tensor-core forms) */
    int64_t computed_pairs; /* distance pairs evaluated on the GPU by the search */
    int64_t candidates;     /* rows that completed a full scan (FP32) / rows rescored in FP64 (TC) */
} dd_result_t;

/* Read-only device views of a plan's preparation arrays (Section 3.1 data
 * structures), for inspection and testing.  All pointers are device
 * addresses owned by the plan; valid until dd_plan_destroy. */
typedef struct {
    int64_t m, N;
    int32_t n, dict_size;
    const double* stats;       /* [0]=mu [1]=sigma [2]=max|t^| of the series (Eq. 2) */
    const double* P1;          /* [m+1] exclusive prefix sums of t^ (FP64) */
    const double* P2;          /* [m+1] exclusive prefix sums of t^^2 (FP64) */
    const double* mu_w;        /* [N] mean of each subsequence of t^ */
    const double* c_w;         /* [N] centred sum of squares of each subsequence of t^ */
    const int32_t* code;       /* [N] SAX word of each subsequence (Eq. 3, 4, 9) */
    const int32_t* freq_hist;  /* [dict] rows per word (Eq. 8 is freq_i = freq_hist[code_i]) */
    const int32_t* order;      /* [N] row order: words by ascending frequency (then word),
                                  rows ascending inside a word = Index_Word (Eq. 10) */
    const int32_t* word_start; /* [dict] offset of each word's rows in `order` */
    const int32_t* ncand;      /* [1] |Cand| (Eq. 7): Cand = order[0 .. ncand) */
    const float* t32;          /* [m] t^ rounded to FP32 */
} dd_view_t;

/* Per-row error bound of the tensor-core Gram form, for inspection and
 * testing.  The Gram tiles compute, for a row i and a column j, a distance D
 * from FP16/BF16 operands with FP32 accumulation (Eq. 1 squared, rewritten as
 * c_i + c_j + n (mu_i - mu_j)^2 - 2 <x'_i, x'_j> over mean-centred rows); the
 * library proves |D - d^2_ij| <= F_i(D) with
 *     F_i(D) = alpha_i + beta D + gam_i sqrt(max(D, 0) + q2_i),
 * which makes the row's running minimum D_i bracket its nearest-neighbour
 * distance: D_i - F_i(D_i) - gam_i^2 <= nn^2_i <= D_i + F_i(D_i) once every
 * column has been scanned.  The early abandon of Algorithm 4 relies on it.
 * Pointers are device addresses owned by the plan (N floats each, indexed by
 * the original row), filled by each call on a tensor-core plan (dd_prep
 * excluded) and valid until dd_plan_destroy. */
typedef struct {
    int64_t N;
    int32_t precision;   /* dd_precision_t of the plan */
    float beta;          /* relative term, the same for every row */
    const float* alpha;  /* [N] absolute term */
    const float* gam;    /* [N] coefficient of the square-root term */
    const float* q2;     /* [N] offset under the square root */
} dd_bound_view_t;

/* The mean-bucketed row order that the search visits columns in (no
 * counterpart in the paper; it makes the pruning bound d^2(i, j) >= n
 * (mu_i - mu_j)^2 of globally normalised subsequences usable, see Eq. 2 and
 * the rows of Eq. 5), for inspection and testing.  Row i's bin is
 *     clamp(floor((mu_i - lo) / w), 0, bins - 1),  lo = min t^, w = (max t^ - lo) / bins,
 * (mu_i from dd_view_t.mu_w; lo = geom[0] and 1/w = geom[3] below).  The order is a
 * stable counting sort by bin of the rows taken in the order
 * e -> (e * stride) mod N (e = 0, 1, ..., N - 1): sig[p] is the row at
 * position p, sigpos its inverse, binstart[b] the first position of bin b
 * (binstart[bins] = N).  Pointers are device addresses owned by the plan,
 * filled by dd_prep and by every search, valid until dd_plan_destroy. */
typedef struct {
    int64_t N;
    int64_t stride;          /* the stride of the input order, coprime with N */
    int32_t bins;
    const int32_t* sig;      /* [N] row at each position */
    const int32_t* sigpos;   /* [N] position of each row */
    const int32_t* mubin;    /* [N] bin of each row */
    const int32_t* binstart; /* [bins + 1] */
    const double* geom;      /* [4] device: lo, w, 1/sigma, 1/w */
} dd_order_view_t;

/* ---- plans ------------------------------------------------------------- */

/* Fills the defaults listed above. */
DD_API void dd_options_default(dd_options_t* opt);

/* Bytes of device workspace a plan for (m, n, opt) needs (0 if invalid). */
DD_API size_t dd_plan_footprint(int64_t m, int32_t n, const dd_options_t* opt);

/* Creates a plan for series of length m and subsequence length n on the
 * current device.  opt == NULL means defaults.  workspace == NULL: the plan
 * allocates dd_plan_footprint() bytes itself (cudaMalloc) and frees them in
 * dd_plan_destroy; otherwise the caller passes device memory of at least that
 * size (256-byte aligned) that it owns and keeps alive until dd_plan_destroy.
 * Errors: DD_EINVAL (sizes, options), DD_ENOMEM, DD_ECUDA. */
DD_API dd_status_t dd_plan_create(dd_plan_t* plan, int64_t m, int32_t n, const dd_options_t* opt,
                           void* workspace, size_t workspace_bytes);

/* Releases the plan (and its workspace if the plan allocated it). NULL is a no-op. */
DD_API void dd_plan_destroy(dd_plan_t plan);

/* ---- discord search ---------------------------------------------------- */

/* Algorithm 2 (PhiDD) on the device: preparation, PotentialDiscord,
 * RefineDiscord, argmax.  T_dev: m float32 values in device memory.
 * Enqueues everything on `stream`, waits for it, and writes the result to
 * *out (host memory).  Errors: DD_EINVAL, DD_ENONFINITE, DD_ECUDA, DD_EBUSY. */
DD_API dd_status_t dd_find_discord(dd_plan_t plan, const float* T_dev, dd_result_t* out, void* stream);

/* Same work, enqueued only: returns once everything is on `stream`, with no
 * host synchronisation.  out_dev: a dd_result_t in device memory or in
 * pinned (page-locked, mapped) host memory; it is written by the last kernel
 * of the call.  A non-finite series is reported in out_dev->status.
 * Returns DD_EINVAL / DD_EBUSY / DD_ECUDA for launch-time errors only. */
DD_API dd_status_t dd_find_discord_async(dd_plan_t plan, const float* T_dev, dd_result_t* out_dev, void* stream);

/* End-to-end form: T_host is m float32 values in host memory (pinned or
 * pageable).  Copies it to the plan's device buffer, searches, copies the
 * result back, waits.  Errors as dd_find_discord. */
DD_API dd_status_t dd_find_discord_host(dd_plan_t plan, const float* T_host, dd_result_t* out, void* stream);

/* Top-k discords (not in the paper's algorithms; the usual extension of its
 * definition): out[0] is the discord; out[j] is the subsequence with the
 * largest nearest-neighbour distance (ties to the smallest index) among those
 * at least n away from out[0 .. j-1] (|i - out[l].index| >= n).  Nearest
 * neighbours are unchanged: any non-self match counts.  k searches in turn,
 * each excluding the rows near the discords found so far; out holds k
 * results in host memory, and entries past the last possible discord have
 * index -1.  Synchronous on `stream`.  Errors as dd_find_discord, DD_EINVAL
 * for k < 1. */
DD_API dd_status_t dd_find_discords(dd_plan_t plan, const float* T_dev, int32_t k, dd_result_t* out, void* stream);

/* Independent searches over `count` series of possibly different lengths
 * and subsequence lengths (T_dev[k]: m[k] float32 values on the device,
 * n[k]); one options struct for all (NULL = defaults).  Results go to
 * out[k] (host memory); out[k].status reports each series' own error.
 * Runs on a temporary engine (below) with up to 32 workers, longest series
 * first; waits for `stream` first so that the series are ready.  Returns
 * the first error met, DD_OK if every search succeeded.  For the tensor-core
 * forms the fused batch (dd_batch_*, below) searches many series faster. */
DD_API dd_status_t dd_find_discord_batched(int32_t count, const float* const* T_dev, const int64_t* m, const int32_t* n,
                                    const dd_options_t* opt, dd_result_t* out, void* stream);

/* Exhaustive nearest-neighbour profile (no abandon): nn2_dev[i] = squared
 * distance from subsequence i to its nearest non-self match, i in [0, N),
 * computed with the plan's precision (tensor-core forms: the FP32 Gram value,
 * within the per-row bound, not rescored; per-window plans: what
 * dd_nn_profile_diag computes).  nn2_dev: N floats on the device.
 * Enqueued on `stream`, not waited for.  Errors: DD_EINVAL, DD_ECUDA. */
DD_API dd_status_t dd_nn_profile(dd_plan_t plan, const float* T_dev, float* nn2_dev, void* stream);

/* Exhaustive nearest-neighbour distances of selected rows: rows_dev[k]
 * (device int32, k < count <= N) -> nn2_dev[k] (device float).  An entry
 * outside [0, N) gives a non-finite value (NaN; +inf on per-window plans) and
 * is never used as an index (the call still succeeds: the rows are only read
 * on the device).  Per-window plans (znorm = 1): exact FP64 values rounded to
 * float.  Enqueued on `stream`.  Errors: DD_EINVAL (count < 0 or > N, null
 * pointers), DD_ECUDA. */
DD_API dd_status_t dd_nn_rows(dd_plan_t plan, const float* T_dev, const int32_t* rows_dev, int32_t count, float* nn2_dev,
                       void* stream);

/* Exhaustive nearest-neighbour profile by the diagonal recurrence of centred
 * dot products: C(i+1, j+1) = C(i, j) + df_i dg_j + df_j dg_i along every
 * diagonal j - i >= n (O(1) work per pair instead of the O(n) of Eq. 1),
 * FP32, every diagonal re-seeded with a direct dot product every 2048 rows.
 * For each row i it finds an argument j_i (|i - j_i| >= n) whose recurrence
 * distance is minimal up to FP32 rounding, then reports the distance to it
 * computed directly:
 *   global plans (znorm = 0): FP32 direct differences on the normalised
 *     series (Eq. 1 squared, as the FP32 form computes them);
 *   per-window plans (znorm = 1): the exact FP64 per-window distance.
 * So nn2_dev[i] is the distance to a real non-self match, >= the true
 * nearest-neighbour distance (up to that rounding) and above it only where
 * the recurrence's rounding picked a near-tie.  nn2_dev: N floats;
 * nn_index_dev: N int32 arguments, or NULL.  Device memory, enqueued on
 * `stream`.  Needs a plan created with diag = 1 or znorm = 1 (else
 * DD_ENOTSUP); N <= 2^26.  Errors: DD_EINVAL, DD_ENOTSUP, DD_EBUSY, DD_ECUDA. */
DD_API dd_status_t dd_nn_profile_diag(dd_plan_t plan, const float* T_dev, float* nn2_dev, int32_t* nn_index_dev,
                                      void* stream);

/* Runs only the preparation stage of Algorithm 2 (Eq. 2 normalisation,
 * prefix sums, window statistics, PAA/SAX words, Freq, Cand, Index_Word) on
 * `stream` and waits.  Errors: DD_EINVAL, DD_ENONFINITE, DD_ECUDA. */
DD_API dd_status_t dd_prep(dd_plan_t plan, const float* T_dev, void* stream);

/* Device views of the preparation arrays of the last call on the plan. */
DD_API dd_status_t dd_plan_view(dd_plan_t plan, dd_view_t* view);

/* The per-row error-bound terms of a tensor-core plan (dd_bound_view_t).
 * Errors: DD_EINVAL (null arguments), DD_ENOTSUP (an FP32 plan has no Gram
 * bound). */
DD_API dd_status_t dd_plan_bound_view(dd_plan_t plan, dd_bound_view_t* view);

/* The plan's mean-bucketed row order (dd_order_view_t).  Errors: DD_EINVAL
 * (null arguments). */
DD_API dd_status_t dd_plan_order_view(dd_plan_t plan, dd_order_view_t* view);

/* Number of this library's kernels launched by the plan's last call (a graph
 * replay does not count the kernels of conditional waves it skipped).  Reads
 * two device counters: call it after the call has finished. */
DD_API int64_t dd_plan_last_launches(dd_plan_t plan);

/* Per-call measurements of the distance kernels (tracing).  When enabled
 * with dd_plan_set_profiling(plan, 1), the synchronous calls record CUDA
 * events on their stream around every distance-tile launch and fill this
 * struct after the call; asynchronous calls leave it untouched. */
typedef struct {
    int32_t dist_launches;      /* distance-tile kernel launches in the last call */
    int32_t precision;          /* dd_precision_t of those launches */
    double dist_ms;             /* sum of their durations (CUDA events, same stream) */
    int64_t computed_pairs;     /* (row, column) pairs they evaluated */
    double call_ms;             /* whole call: first to last kernel (CUDA events) */
    int64_t reserved[4];
} dd_profile_t;

DD_API dd_status_t dd_plan_set_profiling(dd_plan_t plan, int32_t enable);

/* Synchronous and asynchronous searches are captured once into a CUDA graph
 * and replayed (enable = 1, the default).  enable = 0 enqueues the kernels
 * directly on every call instead -- the same kernels, with the waves that run
 * only when many rows survive checking their own gate on the device.  For
 * per-kernel profilers, which cannot profile the kernels of a graph that
 * holds conditional nodes.  Errors: DD_EINVAL, DD_EBUSY. */
DD_API dd_status_t dd_plan_set_graph(dd_plan_t plan, int32_t enable);

/* Fault injection for tests of the failure handling (no GPU fault is
 * involved).  DD_INJECT_STALL_TC: the plan's next tensor-core distance launch
 * arms its operand stages but issues no copy, so its bounded waits expire
 * (about 2 s); the call then returns DD_ETIMEOUT, the rest of that search is
 * skipped, and the plan stays usable.  Consumed by that launch; with graph
 * capture on, it takes effect only when the graph is captured next, so tests
 * turn capture off (dd_plan_set_graph(plan, 0)).  Errors: DD_EINVAL, DD_EBUSY. */
enum { DD_INJECT_NONE = 0, DD_INJECT_STALL_TC = 1 };
DD_API dd_status_t dd_plan_inject(dd_plan_t plan, int32_t what);
DD_API dd_status_t dd_plan_get_profile(dd_plan_t plan, dd_profile_t* out);

/* Waves of distance tiles of the last call (tracing).  A search runs its
 * rows through a fixed sequence of waves (Algorithm 2): the nearest-mean
 * neighbourhood of every row (LOCAL in the FP32 form, BAND in the tensor-core
 * form), the Cand rows of Algorithm 3 (CAND), the rows with the largest upper
 * bounds (TOP), the columns next to each surviving row in time (TIME: the
 * index-order inner loop of Algorithm 4, direct FP32 differences in both
 * forms), the rows of a word (WORD, FP32 form) and the rest of Algorithm 4
 * (REST); the Gram form ends with direct FP32 full scans of its remaining
 * candidates when there are many (SETTLE); exhaustive calls run EXHAUSTIVE
 * waves. */
typedef enum {
    DD_WAVE_EXHAUSTIVE = 0,
    DD_WAVE_LOCAL = 1,
    DD_WAVE_BAND = 2,
    DD_WAVE_CAND = 3,
    DD_WAVE_TOP = 4,
    DD_WAVE_WORD = 5,
    DD_WAVE_REST = 6,
    DD_WAVE_TIME = 7,
    DD_WAVE_SETTLE = 8,
    DD_WAVE_DIAG = 9   /* every pair by the diagonal recurrence (dd_nn_profile_diag, per-window plans) */
} dd_wave_kind_t;

typedef struct {
    int32_t kind;      /* dd_wave_kind_t */
    int32_t rows;      /* rows in the wave's list */
    int64_t items;     /* work items run (items whose rows were all abandoned, or
                          that no row's lower bound admits, are skipped) */
    int64_t pairs;     /* (row, column) distance pairs evaluated */
    double ms;         /* duration from CUDA events on the call's stream when
                          profiling is enabled (dd_plan_set_profiling), else -1 */
} dd_wave_t;

/* Copies up to `cap` waves of the plan's last call into out[] (host memory)
 * and returns how many waves that call ran (which may exceed cap), or a
 * negative dd_status_t (-DD_EINVAL for a null plan or out with cap > 0,
 * -DD_EBUSY while a call is in flight, -DD_ECUDA).  Reads the plan's
 * device-side counters: call it after the call has finished (synchronous
 * calls, or after synchronising the stream of an asynchronous one). */
DD_API int32_t dd_plan_get_waves(dd_plan_t plan, dd_wave_t* out, int32_t cap);

/* Exhaustive nearest-neighbour profile without any device allocation.
 * The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory at the time of the call -- code running
 * inside a device-memory budget that is already fully handed out to another
 * allocator, or latency-critical loops where an allocation would synchronise
 * the device.  It computes what dd_nn_profile computes in the FP32 form
 * (nn2_dev[i] = squared distance from subsequence i to its nearest non-self
 * match, i in [0, N)), needs no plan, and uses as scratch one fixed array of
 * about 1 MiB inside the library that every GPU loading the library keeps
 * until the process exits.  The caller passes T_dev (m float32 values) and
 * nn2_dev (N floats), both device memory.  Work is enqueued on `stream`.
 *   - m must be at most 262,144; larger series return DD_EINVAL (as do
 *     n < 1, N < 2n and null pointers).
 *   - All calls on a device share the scratch array, and it keeps the last
 *     call's contents: calls whose work overlaps on the GPU (other streams or
 *     host threads) race.  Order them on one stream.
 *   - The first call on a device looks up the scratch address with that
 *     device current; make it before any stream capture.
 *   - A series holding NaN or Inf yields NaN in every output element.
 *   - A CUDA error already pending on the calling thread (cudaPeekAtLastError)
 *     makes the call return DD_ECUDA at once, launching nothing and leaving
 *     that error pending for its owner. */
DD_API dd_status_t dd_nn_profile_static(const float* T_dev, int64_t m, int32_t n, float* nn2_dev, void* stream);

/* Measured peak rate of this device's CUDA-core FMA pipe, for roofline
 * denominators (no counterpart in the paper).  fp64 = 0: FP32 FFMA; fp64 = 1:
 * FP64 DFMA.  Every SM runs independent FMA chains for about 20 ms (CUDA events
 * on `stream`, after a warm-up launch); *fma_per_s receives FMA lane operations
 * per second (two flops each).  Synchronous.  Allocates and frees a 256-byte
 * device buffer.  Errors: DD_EINVAL (bad fp64, null output), DD_ENOMEM,
 * DD_ECUDA. */
DD_API dd_status_t dd_probe_fma_rate(int32_t fp64, double* fma_per_s, void* stream);

/* Static text for a status code. */
DD_API const char* dd_status_string(dd_status_t status);

/* ---- engine: concurrent searches for batches and serving ---------------
 *
 * Not in the paper (which runs one search at a time): a pool of workers,
 * each a host thread with its own CUDA stream, takes requests from one queue
 * and runs them concurrently on the GPU, so that many small searches overlap.
 * Admission is by device memory: every plan lives in a workspace of exactly
 * its footprint (dd_plan_footprint) taken from an engine-owned stream-ordered
 * pool, a host series in a staging buffer of 4 m bytes from the same pool,
 * and a request starts only while the workspaces held by the workers (the
 * resident plans of idle workers included) plus its own fit the engine's
 * budget.  A worker takes the first queued request that fits, so smaller
 * requests pass one that does not -- at most 32 times, after which nothing is
 * admitted past it until it fits.  A worker keeps its last plan and reuses it
 * for requests of the same (m, n), and gives it back when nothing queued fits.
 * Every request uses the engine's options.  A request's result equals that of
 * a plan searching the same series alone. */
typedef struct dd_engine_s* dd_engine_t;

typedef struct {
    int64_t id;          /* the caller's request id */
    dd_result_t result;  /* result.status is the request's own status */
    double queue_ms;     /* submission -> a worker took the request */
    double service_ms;   /* a worker took it -> result on the host (includes
                            the host->device copy of a host series) */
} dd_completion_t;

enum { DD_SERIES_DEVICE = 0, DD_SERIES_HOST = 1 };

/* workers in [1, 64].  The budget is workers x (the largest plan footprint of
 * a series with m <= m_max, n <= n_max, plus m_max floats of staging): the
 * memory a pool of per-worker workspaces of the largest shape would hold.
 * Admission: a request whose plan and staging exceed the whole budget, or a
 * host series longer than m_max, completes with DD_ENOMEM.  (m_max, n_max)
 * must itself be a valid shape.  Errors: DD_EINVAL (bad sizes or options),
 * DD_ENOMEM, DD_ECUDA. */
DD_API dd_status_t dd_engine_create(dd_engine_t* engine, int32_t workers, const dd_options_t* opt, int64_t m_max,
                                    int32_t n_max);

/* The same with an explicit budget of device bytes (0 = the default above). */
DD_API dd_status_t dd_engine_create_budget(dd_engine_t* engine, int32_t workers, const dd_options_t* opt,
                                           int64_t m_max, int32_t n_max, size_t budget_bytes);

/* Queues a search of the m values at T (device memory, or host memory with
 * flags = DD_SERIES_HOST) with subsequence length n.  T must stay valid and
 * unchanged until the request's completion has been polled; a device series
 * must already be complete (the engine's streams are not ordered after the
 * caller's).  Invalid sizes complete with DD_EINVAL.  Returns DD_EINVAL for a
 * null engine or series or bad flags, DD_EBUSY once destruction has begun. */
DD_API dd_status_t dd_engine_submit(dd_engine_t engine, int64_t id, const float* T, int64_t m, int32_t n,
                                    int32_t flags);

/* Moves up to cap finished requests to out[] (host memory), in the order
 * they finished.  When none is ready, waits up to wait_ms milliseconds
 * (negative: until one is; returns 0 at once when no request is
 * outstanding).  Returns how many it moved, or -DD_EINVAL. */
DD_API int32_t dd_engine_poll(dd_engine_t engine, dd_completion_t* out, int32_t cap, int32_t wait_ms);

/* Requests submitted and not yet polled. */
DD_API int64_t dd_engine_outstanding(dd_engine_t engine);

/* Lets running requests finish, drops queued ones, joins the workers and
 * frees everything. */
DD_API void dd_engine_destroy(dd_engine_t engine);

/* ---------------------------------------------------------------- fused batch
 * A batch plan searches many independent series of uneven lengths together:
 * every step of the search (Section 2.1's discord of each series, found by the
 * steps of Algorithms 2-4 with the tensor-core Gram form) is one launch over
 * all series, and the distance tiles of every series are claimed from one
 * device work queue by the persistent tcgen05 kernel.  Series with the same
 * subsequence length n share one set of launches (a group).  Per series:
 * Eq. 2 normalisation of that series alone, the mean-bucketed row order, a band
 * wave (every row tile against the 256 columns around it in that order), full
 * scans of the 128 rows with the largest upper bounds, which fix the series'
 * own best-so-far, scans of the rows whose upper bound still reaches it
 * (abandoned against it, Algorithm 4), and exact FP64 rescoring of every row the
 * per-row error bound cannot rule out.  Each result is that of
 * dd_find_discord on the same series with the same precision: exact index
 * (ties -> smallest), FP64 nn_distance (computed_pairs is 0: pairs are not
 * counted per series).
 *
 * The launches of a call are captured into a CUDA graph, which the next call
 * with the same shapes (count and every (m, n), in order) replays; series
 * pointers are read by the device from a descriptor table, so only the shapes
 * key the graph.  Memory is one device allocation made at creation: capacity
 * max_series series of at most max_values values in total, n <= n_max.  A call
 * beyond that capacity returns DD_ENOMEM; more than 64 distinct n in one call
 * returns DD_ENOTSUP.  Invalid series (as dd_plan_create's sizes, n > n_max, or
 * a null pointer) complete with DD_EINVAL and do not affect the others.  A
 * non-finite series completes with DD_ENONFINITE, a constant one with index 0
 * and distance 0. */
typedef struct dd_batch_s* dd_batch_t;

typedef struct {
    int32_t seg_cols;     /* columns per work item of the full-scan waves: a multiple of 256
                             in [256, 65536] (default 512) */
    int32_t settle_min;   /* a series with more FP64 candidates than this (rows whose Gram
                             bounds overlap the best-so-far) first settles them with direct FP32
                             full scans and their rigorous FP32 bounds (default 4; >= 0) */
    int32_t settle_rows;  /* rows per tile of those FP32 full scans: 32, 64 (default) or 128 (one
                             series' candidates per tile) */
    int32_t reserved[1];  /* must be zero */
} dd_batch_config_t;

DD_API void dd_batch_config_default(dd_batch_config_t* cfg);

/* Device bytes dd_batch_create allocates for this capacity (0 if invalid:
 * max_series in [1, 65536], n_max in [1, 65536], max_values >= 1 and
 * max_values + 384 max_series <= 2^30). */
DD_API size_t dd_batch_footprint(int32_t max_series, int64_t max_values, int32_t n_max);

/* opt: precision DD_TC_FP16 or DD_TC_BF16 (else DD_ENOTSUP), znorm 0, no shards,
 * diag 0; the SAX and wave options do not apply.  cfg may be null (defaults).
 * Errors: DD_EINVAL, DD_ENOTSUP, DD_ENOMEM, DD_ECUDA. */
DD_API dd_status_t dd_batch_create(dd_batch_t* batch, int32_t max_series, int64_t max_values, int32_t n_max,
                                   const dd_options_t* opt, const dd_batch_config_t* cfg);

/* Searches count series (T_dev[k]: m[k] values on the device, complete in
 * stream order on `stream`; m, n, out: host arrays).  Blocking: returns when
 * out[] (host memory) holds every result.  Returns DD_OK or the first
 * non-DD_OK result status; DD_EBUSY if another thread is using the batch. */
DD_API dd_status_t dd_batch_search(dd_batch_t batch, int32_t count, const float* const* T_dev, const int64_t* m,
                                   const int32_t* n, dd_result_t* out, void* stream);

/* The schedule of the group of subsequence length n (cfg null: back to the batch's
 * own), e.g. the one a tuner found fastest for that n.  Takes effect at the next
 * call, which captures a new graph.  DD_EINVAL for a null batch, n < 1 or an
 * invalid cfg; DD_EBUSY while a search runs. */
DD_API dd_status_t dd_batch_set_schedule(dd_batch_t batch, int32_t n, const dd_batch_config_t* cfg);

/* Calls that replayed the captured graph of the previous call's shapes. */
DD_API int64_t dd_batch_graph_replays(dd_batch_t batch);

DD_API void dd_batch_destroy(dd_batch_t batch);

#ifdef __cplusplus
}
#endif
#endif /* DD_H_ */
