/*
 * kmpar.h -- C ABI of the GB300 (sm_103a) k-means|| library.
 *
 * Method: Bahmani, Moseley, Vattani, Kumar, Vassilvitskii, "Scalable K-Means++"
 * (arXiv:1203.6402).  The library runs the data-parallel path of Algorithm 2
 * (Sec. 3.3) on one GPU:
 *
 *   kmpar_init          Alg. 2 steps 1-2  first center uniform over X; psi = phi_X(C)
 *   kmpar_round         Alg. 2 steps 4-5  draw each x with p = min(1, l D^2(x)/phi),
 *                                          C <- C u C', update D^2 and phi
 *   kmpar_set_sampling  Sec. 5.3          or draw exactly floor(l) points per round
 *   kmpar_weight        Alg. 2 step 7     w_c = #points nearest to candidate c
 *   kmpar_recluster     Alg. 2 step 8     weighted k-means++ (Alg. 1, Sec. 4.2) to k
 *   kmpar_lloyd         Sec. 1, Sec. 3.1  Lloyd's iteration to a stable assignment
 *   kmpar_cost          Sec. 3.1          phi_X(C) = sum_x min_i ||x - c_i||^2
 *
 * Conventions (all entry points):
 *   - X is row-major FP32, n rows of d coordinates (row stride d floats), in
 *     DEVICE memory unless a function says otherwise.  It is borrowed: the
 *     caller keeps it alive and unchanged for the life of the context.
 *   - Every call is asynchronous on the context's stream unless it writes to a
 *     host pointer the caller passed (those calls synchronise that stream).
 *   - Errors are returned as kmpar_status; no exception crosses the ABI and no
 *     device trap is used.  kmpar_last_error() gives a one-line reason.
 *   - Nothing is thread-safe per context; distinct contexts are independent.
 *   - Limits: 1 <= d <= 4096, 1 <= n < 2^31, 1 <= k, l > 0, 0 <= rounds,
 *     per-round sample capacity l + 10 sqrt(l) + 64 <= 32768.
 *
 * Fault injection (environment variables, read when the limit applies; for
 * tests of the error paths, none of them is needed in normal use):
 *   KMPAR_ROUND_CAPACITY   lowers the per-round draw capacity (read by kmpar_init
 *                          and kmpar_batch_run)
 *   KMPAR_CTX_LIMIT_BYTES  most device memory one context may hold; a larger
 *                          allocation fails with KMPAR_ERR_OOM (read at every one)
 *   KMPAR_WAIT_CYCLES      clock-cycle budget of each per-draw wait of the
 *                          cooperative reclustering kernel (default ~2 s); a wait
 *                          that runs out returns KMPAR_ERR_TIMEOUT
 *   KMPAR_RECLUSTER_GRID   1: use the cooperative grid form of step 8 at any size
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 * counter = (i_lo, i_hi, round, tag); tag 1 = first center, 2 = round draws,
 * 3 = reclustering draws, 4 = exactly-l round clocks; a uniform double is (a 2^26 + b) / 2^53 with
 * a = word0 >> 5, b = word1 >> 6.  Results are a pure function of
 * (X, k, l, rounds, seed, precision, sampling mode).
 *
 * Ties: an argmin goes to the lowest center number; candidates are numbered in
 * insertion order (initial center 0, then each round's draws in ascending point
 * order).  Decisions whose FP32 values are within the FP32 error bound of one
 * another are re-decided in FP64 with the same formula as the definition
 * (difference form, ascending coordinates, no fused multiply-add).
 */
#ifndef KMPAR_H
#define KMPAR_H

#include <stdint.h>

#if defined(__GNUC__)
#define KMPAR_API __attribute__((visibility("default")))
#else
#define KMPAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kmpar_ctx kmpar_ctx;

typedef enum {
    KMPAR_OK = 0,
    KMPAR_ERR_ARG = 1,              /* an argument is out of range or NULL          */
    KMPAR_ERR_CUDA = 2,             /* a CUDA runtime call or a launch failed       */
    KMPAR_ERR_OOM = 3,              /* device allocation failed                     */
    KMPAR_ERR_CAPACITY = 4,         /* a round drew more points than its capacity   */
    KMPAR_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up           */
    KMPAR_ERR_STATE = 6,            /* call out of order (see each function)        */
    KMPAR_WARN_FEW_CANDIDATES = 7,  /* recluster ran out of positive mass before k  */
    KMPAR_ERR_UNSUPPORTED = 8       /* precision or size not built into this library*/
} kmpar_status;

/* Arithmetic of the distance step.  Every mode stores exact FP32 difference-form
 * distances and takes the same argmin decisions; the modes differ only in how
 * candidates are screened. */
typedef enum {
    KMPAR_FP32 = 0,     /* CUDA-core FP32 difference form for every pair          */
    KMPAR_BF16 = 1,     /* tcgen05 BF16 GEMM-form screening + exact FP32 refine    */
    KMPAR_BF16X3 = 2,   /* tcgen05 split-BF16 (hi/lo, 3 products) screening+refine */
    KMPAR_FP8E4M3 = 3   /* tcgen05 e4m3 screening, per-row power-of-two scales of X
                           and per-tile scales of the centers, + exact FP32 refine */
} kmpar_precision;

/* Counters gathered on the device (kmpar_get_stats synchronises). */
typedef struct {
    int64_t n, m;                 /* points; candidates so far                      */
    int32_t d, k, rounds_done, lloyd_iters;
    int64_t round_added[64];      /* |C'_i| for i = 1..rounds (index i-1)            */
    double  phi[65];              /* psi, then phi after each round                  */
    int64_t sample_near;          /* draws with |u - p| <= 1e-6; exactly-l rounds:
                                     rounds whose last drawn clock has another
                                     within (2d+16) 2^-24 (relative) of it           */
    int64_t sample_refined;       /* draws re-decided with an FP64 D^2                */
    int64_t argmin_fp64;          /* argmin decisions re-decided in FP64              */
    int64_t argmin_wide;          /* screening windows that held more than 2 centers  */
    int64_t recluster_near;       /* reclustering targets within 1e-6 of a boundary   */
    int32_t capacity_overflow;    /* 1 if some round exceeded its capacity            */
    int32_t recluster_warn;       /* 1 if positive mass ran out before k draws        */
    /* with kmpar_set_timing(ctx, 1): CUDA-event time of the distance passes,
     * [0] = round passes (Alg. 2 step 5), [1] = Lloyd assignment passes */
    double  kernel_ms[2];
    int64_t kernel_launches[2];
    int64_t screen_rows;          /* tensor-core passes: rows screened                 */
    int64_t screen_fallback;      /* rows the pair screening left undecided (they go
                                     to the list pass, or, in BF16X3, to the exact
                                     CUDA-core scan)                                 */
    int64_t screen_exact;         /* rows the exact CUDA-core scan decided             */
    int64_t screen_listed;        /* undecided rows of round passes that went to the
                                     exact refine over the lists the screening pass
                                     itself kept (the others took the list pass)     */
    int64_t recluster_snapshots;  /* batched reclustering: D^2 snapshots taken       */
    int64_t lloyd_settled;        /* Lloyd assignments (rows x iterations) that the
                                     bounds between iterations settled without the
                                     tensor pass (tensor modes; same results)        */
} kmpar_stats;

/*
 * Alg. 2 steps 1-2.  Creates a context over X (device, n x d FP32, borrowed),
 * allocates its device buffers, draws the first center i0 = floor(u n) with u
 * from counter (0, 0, 0, 1), and computes D^2(x) = ||x - x_i0||^2 (exact FP32
 * difference form), idx(x) = 0 and psi = sum D^2 (FP64).  k is the number of
 * centers the reclustering produces; ell is the oversampling factor l; rounds is
 * the number of calls to kmpar_round that will follow; stream is a cudaStream_t
 * (NULL = legacy default stream).  On error *out is NULL.  The device buffers
 * come, in stream order, from a memory pool the library keeps per device; memory
 * a destroyed context returned to it is reused without mapping new pages.
 */
KMPAR_API kmpar_status kmpar_init(kmpar_ctx **out, const float *X, int64_t n, int32_t d, int32_t k,
                        double ell, int32_t rounds, uint64_t seed, int32_t precision,
                        void *stream);

/*
 * Alg. 2 steps 4-5, round i (1-based; rounds must be called in order 1..rounds).
 * Draws each x independently with p = min(1, l D^2(x)/phi) (p = 0 if phi = 0),
 * u from counter (x, 0, i, 2); appends the drawn points in ascending order to the
 * candidate set; updates D^2, idx and phi against the new candidates.  n_added
 * and phi (host, nullable) receive |C'_i| and the new phi; passing either
 * synchronises the stream.  KMPAR_ERR_CAPACITY if the round drew more than its
 * capacity (the context is then unusable).
 */
KMPAR_API kmpar_status kmpar_round(kmpar_ctx *ctx, int32_t i, int64_t *n_added, double *phi);

/*
 * Alg. 2 step 7.  Computes w_c = #{x : idx(x) = c} for every candidate c.
 * *m_out (host) receives the number of candidates m; *cand_idx_dev receives a
 * device pointer to m int32 row numbers of X (insertion order) and *w_dev a
 * device pointer to m int64 weights; both are owned by the context and stay valid
 * until kmpar_destroy.  Any out pointer may be NULL.  Synchronises.
 */
KMPAR_API kmpar_status kmpar_weight(kmpar_ctx *ctx, int64_t *m_out, const int32_t **cand_idx_dev,
                          const int64_t **w_dev);

/*
 * Alg. 2 step 8.  Weighted k-means++ over the m candidates: draw t = 0 picks c
 * with probability w_c / sum w; draw t > 0 picks c with probability
 * w_c D^2(c) / sum w D^2, D^2 to the centers drawn so far; a draw uses u from
 * counter (t, 0, 0, 3), target = u * total, and the smallest c whose FP64 prefix
 * sum exceeds the target.  Writes the k chosen rows to centers_dev (device, k x d
 * FP32, caller-owned).  Requires kmpar_weight.  Returns KMPAR_WARN_FEW_CANDIDATES
 * (centers still written, remaining draws repeat the first center) if the mass
 * ran out before k draws.  Synchronises.  Candidate sets that fit one
 * thread-block cluster's shared memory run in a cluster kernel, larger ones in a
 * cooperative grid kernel; setting the environment variable KMPAR_RECLUSTER_GRID
 * to 1 selects the grid kernel for every size (same draws up to reported near
 * ties).  After kmpar_set_recluster(ctx, B) with B > 0, the same law is drawn in
 * batches of up to B draws per D^2 snapshot instead (see kmpar_set_recluster).
 */
KMPAR_API kmpar_status kmpar_recluster(kmpar_ctx *ctx, float *centers_dev);

/*
 * Alg. 2 step 8, second half (optional): Lloyd's iteration on the weighted
 * candidate set from the k centers in centers_dev (device, k x d FP32, updated in
 * place), the reading of step 8 in which weighted k-means++ is followed by local
 * search on the weighted candidates (Sec. 3.3 leaves the reclustering method
 * open).  Each iteration assigns every candidate to its nearest center (the same
 * rule as kmpar_lloyd) and stops if no label changed; otherwise center j becomes
 * sum w_c c / sum w_c over its candidates (FP64 products and sums in ascending
 * candidate order, rounded to FP32 once; a center without candidates keeps its
 * place).  At most max_iter updates; *iters (host, nullable) receives their
 * number.  Requires kmpar_weight.  Synchronises once per iteration.
 */
KMPAR_API kmpar_status kmpar_weighted_lloyd(kmpar_ctx *ctx, float *centers_dev, int32_t max_iter, int32_t *iters);

/*
 * Lloyd's iteration (Sec. 1, Sec. 3.1) on X from the k centers in centers_dev
 * (device, k x d FP32, updated in place).  Each iteration assigns every point to
 * its nearest center (lowest index on ties) and stops if no label changed;
 * otherwise each center becomes the centroid of its cluster (FP64 sums in
 * ascending point order, rounded to FP32; an empty cluster keeps its center).
 * At most max_iter center updates.  labels_dev (device, n int32, nullable)
 * receives the final assignment; *iters (host, nullable) the number of updates;
 * *final_cost (host, nullable) the cost of the final centers; cost_hist (host,
 * nullable, max_iter+1 doubles) the cost of each assignment.  In the tensor modes
 * whose screening adds the center norms in the epilogue (BF16, FP8) with d a
 * multiple of 4, the assignments after the first skip the rows whose distance
 * bounds prove their center unchanged (counted in kmpar_stats.lloyd_settled);
 * every label, distance and center is the one the full assignment gives.
 * Synchronises once per batch of iterations (4, then 8).
 */
KMPAR_API kmpar_status kmpar_lloyd(kmpar_ctx *ctx, float *centers_dev, int32_t max_iter,
                         int32_t *labels_dev, int32_t *iters, double *final_cost,
                         double *cost_hist);

/*
 * Sec. 3.1: phi_X(C) = sum_x min_i ||x - c_i||^2 for X (device, n x d FP32) and
 * C (device, k x d FP32), summed in FP64 over exact FP32 distances.  *phi (host)
 * receives the cost.  Every precision gives this same exact-FP32 value (the
 * CUDA-core pass computes it).  Allocates a small scratch buffer on the stream.
 * Synchronises.
 */
KMPAR_API kmpar_status kmpar_cost(const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                        int32_t precision, double *phi, void *stream);

/*
 * phi_X(C) like kmpar_cost, for callers that cannot allocate device memory when
 * they need it: for instance a host framework that has reserved all of the GPU's
 * memory for its own pool, or a latency-critical loop in which an allocation,
 * which can synchronise the device, is not allowed.  The paper has no
 * counterpart.
 *
 * No allocation: the per-block FP64 partial sums live in a fixed array inside the
 * library (65,539 doubles, about 512 KB, held on every GPU that loads the library
 * until the process exits).  The caller still passes X and C (device) and phi
 * (host).  n is limited to 8,388,608 points (65,536 blocks of 128); larger n
 * returns KMPAR_ERR_ARG with a message in kmpar_last_error(NULL).
 *
 * Every call looks up the array's device address in the current context with
 * cudaGetSymbolAddress (which allocates nothing), so the address is never stale
 * after a device reset or a context switch.  The first call in a process may
 * load the library's device code: make it before any stream capture.  Every
 * call shares the one array,
 * which keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it and must be serialised by the
 * caller.  Synchronises.
 */
KMPAR_API kmpar_status kmpar_cost_noalloc(const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                                          double *phi, void *stream);

/*
 * The whole path in one call: init, rounds 1..r, weight, recluster, Lloyd.
 * flags & KMPAR_HOST_BUFFERS: X, centers_out and labels_out are HOST pointers
 * (copied in and out inside the call); otherwise device pointers.
 * flags & KMPAR_EXACT_SAMPLING: exactly floor(l) draws per round (see
 * kmpar_set_sampling).  (flags >> 8) & 255: updates of kmpar_weighted_lloyd on
 * the candidates after the reclustering (0: none, the default).  (flags >> 16) &
 * 255: the reclustering batch of kmpar_set_recluster (0: one draw at a time).  seed_cost, final_cost and iters are host pointers
 * (nullable).  labels_out is nullable.
 */
#define KMPAR_HOST_BUFFERS 1
#define KMPAR_EXACT_SAMPLING 2
KMPAR_API kmpar_status kmpar_fit(const float *X, int64_t n, int32_t d, int32_t k, double ell, int32_t rounds,
                       uint64_t seed, int32_t precision, int32_t max_iter, float *centers_out,
                       int32_t *labels_out, double *seed_cost, double *final_cost, int32_t *iters,
                       int32_t flags, void *stream);

/*
 * Many independent problems in one call (Alg. 2 steps 1-8 and Lloyd's iteration
 * per problem, Sec. 3.3 applied to each problem separately: the data-parallel
 * pattern of Sec. 3.5 over problems instead of machines).  Problem p owns n rows
 * of d coordinates starting at float x_offset of X (device, row-major); its k
 * seed-then-Lloyd centers go to centers_out + c_offset (device, k x d FP32), its
 * final labels to labels_out + l_offset (device, n int32; labels_out nullable),
 * its candidate row numbers (within the problem) and weights to
 * cand_out + cand_offset and w_out + cand_offset (device; nullable; room for
 * kmpar_batch_cand_capacity(ell, rounds) entries).  Every problem draws from
 * its own seed exactly as kmpar_fit does (same counters, same tie rules); the
 * distances are the exact FP32 difference form on CUDA cores.  Limits: 1 <= d
 * <= 128, 1 <= k <= 512, n < 2^31, 0 <= rounds <= 16, per-round capacity
 * l + 10 sqrt(l) + 64 <= 4096.  results (host, count entries) receive each
 * problem's outcome; a problem whose round overflows its capacity stops there
 * with status KMPAR_ERR_CAPACITY, the others are unaffected.  Work space comes
 * from the library's pool; a problem runs in one thread block, or in a
 * thread-block cluster of 2, 4 or 8 blocks when it has more than 25,000 rows
 * (each block a contiguous range of rows; the cluster combines its sums and its
 * ordered draws in rank order; see kmpar_batch_set_split), largest problems
 * first, one kernel launch per (dimension class, cluster size).  Synchronises.
 */
typedef struct {
    int64_t x_offset;     /* first float of the problem's rows in X               */
    int64_t n;            /* points                                               */
    int32_t d, k;         /* dimension, centers                                   */
    double  ell;          /* oversampling factor l                                */
    int32_t rounds;       /* rounds r                                             */
    int32_t max_iter;     /* Lloyd updates at most                                */
    uint64_t seed;
    int64_t c_offset;     /* first float of the problem's centers in centers_out  */
    int64_t l_offset;     /* first label in labels_out                            */
    int64_t cand_offset;  /* first entry in cand_out / w_out                      */
} kmpar_problem;

typedef struct {
    int64_t m;            /* candidates                                           */
    double  seed_cost;    /* cost of the seed centers (Lloyd's first assignment)  */
    double  final_cost;   /* cost of the final centers                            */
    int32_t iters;        /* Lloyd updates made                                   */
    int32_t status;       /* KMPAR_OK, KMPAR_ERR_CAPACITY or KMPAR_WARN_FEW_CANDIDATES */
    int64_t sample_near;  /* draws with |u - p| <= 1e-6                           */
    int64_t argmin_fp64;  /* argmin decisions re-decided in FP64                  */
    int64_t recluster_near; /* reclustering targets within 1e-6 of a boundary     */
} kmpar_problem_result;

/* Schedule of kmpar_batch_run (process-wide): a problem of more than
 * rows_per_block rows is split over a thread-block cluster of 2, 4 or 8 blocks
 * (default 25,000; 0: never split).  Results do not depend on it beyond the
 * association of FP64 sums.  KMPAR_ERR_ARG for a negative value. */
KMPAR_API kmpar_status kmpar_batch_set_split(int32_t rows_per_block);

/* Candidate slots a problem of oversampling l and r rounds needs in cand_out/w_out. */
KMPAR_API int64_t kmpar_batch_cand_capacity(double ell, int32_t rounds);

KMPAR_API kmpar_status kmpar_batch_run(const float *X, const kmpar_problem *problems, int32_t count,
                                       float *centers_out, int32_t *labels_out, int32_t *cand_out,
                                       int64_t *w_out, kmpar_problem_result *results, void *stream);

/*
 * How Alg. 2 step 4 draws.  KMPAR_SAMPLE_BERNOULLI (the default): every x is
 * drawn independently with p = min(1, l D^2(x)/phi).  KMPAR_SAMPLE_EXACT: the
 * variant of Sec. 5.3 (Fig. 5.1), exactly L = floor(l) points per round without
 * replacement, each successive draw proportional to D^2 among the points not
 * drawn yet (D^2 as at the start of the round); fewer only when fewer than L
 * points have D^2 > 0, and then all of those.  It is computed as the L smallest
 * clocks -ln(u_x) / D^2(x) with u_x from counter (x, 0, round, 4), clocks in
 * FP32 from the stored D^2, equal clocks to the lower x; a round whose L-th clock
 * has another within (2d+16) 2^-24 (relative) of it adds one to sample_near.
 * Call before round 1 (KMPAR_ERR_STATE otherwise).  KMPAR_ERR_ARG for an unknown
 * mode, or l < 1 with KMPAR_SAMPLE_EXACT.  The exact mode allocates 4 n bytes.
 */
#define KMPAR_SAMPLE_BERNOULLI 0
#define KMPAR_SAMPLE_EXACT 1
KMPAR_API kmpar_status kmpar_set_sampling(kmpar_ctx *ctx, int32_t mode);

/*
 * How kmpar_recluster draws the weighted k-means++ sequence (Alg. 2 step 8,
 * Alg. 1 with multiplicities, Sec. 4.2).  batch = 0 (the default): one draw at a
 * time, draw t with u from counter (t, 0, 0, 3) and the inverse CDF of the
 * masses w_j D^2(j) in ascending j.  batch = B in 1..64: the same law drawn in
 * batches: draw 0 as above; then each snapshot S of D^2 fixes the masses
 * w_j S_j, 2B proposals are drawn from them (proposal i with u from counter
 * (p + i, 0, 0, 5), p = 2B x the snapshots before), and in proposal order a
 * proposal j is kept iff v S_j < D(j), v from counter (p + i, 1, 0, 5) and D(j)
 * the smaller of S_j and the distances to the centers kept since the snapshot;
 * a snapshot keeps at most B draws (kmpar_stats.recluster_snapshots counts
 * them).  A draw whose proposals had a target within 1e-6 of the total of a
 * prefix boundary, or v S_j within 1e-4 S_j of D(j), adds one to recluster_near.
 * The batched form allocates d x m floats for a transposed copy of the
 * candidates and ~70 KB.  KMPAR_ERR_ARG for a batch outside 0..64.
 */
KMPAR_API kmpar_status kmpar_set_recluster(kmpar_ctx *ctx, int32_t batch);

/* Device pointers to the context's D^2 (n FP32) and idx (n int32) arrays, valid
 * until the next call on the context; either out pointer may be NULL. */
KMPAR_API kmpar_status kmpar_state(const kmpar_ctx *ctx, const float **D2_dev, const int32_t **idx_dev);

/* Device-side counters (see kmpar_stats).  Synchronises. */
KMPAR_API kmpar_status kmpar_get_stats(kmpar_ctx *ctx, kmpar_stats *out);

/* Writes u(i) for counters (i, 0, round, tag), i = 0..count-1, under key seed,
 * to out_dev (device, count doubles): the generator every draw above uses. */
KMPAR_API kmpar_status kmpar_uniforms(int64_t count, uint32_t round, uint32_t tag, uint64_t seed,
                            double *out_dev, void *stream);

/* Enables (1) or disables (0) CUDA-event timing of the context's distance passes
 * (reported by kmpar_get_stats); off by default. */
KMPAR_API kmpar_status kmpar_set_timing(kmpar_ctx *ctx, int32_t enable);

/* Number of CUDA kernels this library has launched in the process so far. */
KMPAR_API int64_t kmpar_launch_count(void);

/* Waits for the context's stream, then returns the context's buffers to the
 * library's pool (stream-ordered, no device-wide synchronisation).  Device
 * pointers the context handed out (kmpar_weight) are invalid afterwards, and no
 * work on another stream may still read them.  NULL is a no-op. */
KMPAR_API void kmpar_destroy(kmpar_ctx *ctx);

/* Hands the pool memory that no live context uses back to the driver, on every
 * device the library has used.  KMPAR_ERR_CUDA if the driver refuses. */
KMPAR_API kmpar_status kmpar_release_cached_memory(void);
KMPAR_API const char *kmpar_status_string(kmpar_status s);
/* Last error message of ctx, or of the calling thread's last context-free call
 * when ctx is NULL. */
KMPAR_API const char *kmpar_last_error(const kmpar_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* KMPAR_H */
