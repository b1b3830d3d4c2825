/*
 * kpynq.h -- C ABI of the GB300 (sm_103a) work-efficient triangle-inequality
 * K-means library (libkpynq.so).
 *
 * The method is KPynq's (Abstract; Sec. I): K-means whose assignment step runs
 * a "Multi-level Filter" -- a group-level filter and a point-level filter over
 * per-point distance bounds -- before a "Distance Calculator" that evaluates
 * only the point-centroid pairs the filters could not rule out.  The filters
 * discard only evaluations that cannot change a point's nearest centroid, so
 * the result is that of standard (Lloyd) K-means.  The paper gives no formulas;
 * the bound bookkeeping follows the group/point filter scheme of Yinyang
 * K-means, and every reading is stated where it is used.
 *
 * Definitions used by every call:
 *   assignment  a(x) = argmin_k ||x - c_k||^2, ties to the lowest index k.
 *               Labels are exact: equal to the FP64 argmin over the library's
 *               (FP32) centroids, whatever the filters skipped.
 *   update      c_k <- mean of the points assigned to k (FP64 sums); an empty
 *               cluster keeps its centroid.
 *   iteration t assign from C^t, then update to C^{t+1}.  Iteration 0 is a
 *               dense pass over all K centroids; later ones are filtered.
 *   objective   J_t = sum_x ||x - c^t_{a_t(x)}||^2 (FP64).
 *   stop rule   (kmeans_fit) after max_iter iterations, when no label changed,
 *               or when J_{t-1} - J_t < tol * J_{t-1}.
 *
 * Pointers.  Every array argument may be a host or a device pointer; the
 * library asks the CUDA runtime which (cudaPointerGetAttributes).  Device
 * pointers must be on the context's device.  Host input arrays are copied to
 * library-owned device memory; host output arrays are filled by a
 * device-to-host copy before the call returns.  Layouts are row-major and
 * dense: X is N x D float32, centroids K x D float32, labels N int32.
 *
 * Ownership.  A device X is borrowed, not copied: it must stay valid and
 * unchanged until kmeans_destroy.  All other state (bounds, sums, queues) is
 * allocated by kmeans_init and freed by kmeans_destroy.
 *
 * Streams.  All work is ordered on the stream given in kmeans_options (NULL =
 * the legacy default stream).  kmeans_iterate, kmeans_fit and the getters
 * return after that stream has finished their work.
 *
 * Errors.  Every call returns a km_status.  The library never aborts the
 * process; kmeans_last_error gives a message.  A call that fails with
 * KM_ECUDA or KM_ETIMEOUT leaves the context unusable (KM_ESTATE afterwards).
 *
 * Threads.  A context is not thread-safe; distinct contexts are independent.
 */
#ifndef KPYNQ_H
#define KPYNQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KM_API __attribute__((visibility("default")))
#else
#define KM_API
#endif

typedef struct kmeans_ctx kmeans_ctx;

typedef enum {
    KM_OK = 0,
    KM_EINVAL = -1,   /* bad argument: sizes, null pointer, non-finite input */
    KM_ENOMEM = -2,   /* device or host allocation failed */
    KM_ECUDA = -3,    /* a CUDA runtime call or kernel failed */
    KM_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    KM_ESTATE = -5    /* context unusable after an earlier failure */
} km_status;

/* kmeans_options.algo */
enum {
    KM_ALGO_FILTERED = 0, /* group + point filters, survivor distances */
    KM_ALGO_LLOYD = 1     /* plain Lloyd: every distance, every iteration */
};

/* kmeans_options.grouping: how the K centroids form the G groups (labels
 * never depend on it; how much the filters skip does) */
enum {
    KM_GROUP_CONTIGUOUS = 0, /* centroid j -> group floor(j * G / K) */
    KM_GROUP_CLUSTERED = 1   /* groups of nearby centroids: plain Lloyd over the K
                                initial centroids, seeded by their first G rows, 5
                                iterations (FP32, on the device); a centroid joins
                                the group of its nearest centre (lowest index on
                                ties).  Groups left empty are dropped, so fewer
                                than G groups may result; bound rows (kmeans_get_bounds)
                                then hold the remaining groups in the order of
                                their seeds.  Labels and centroids are always in
                                the caller's numbering. */
};

/* kmeans_options.dtype: storage type of X.  init_centroids and every output
 * stay FP32; bfloat16 points are converted exactly to an FP32 copy made at
 * init (so the tensor-core split of X has a zero low half and the oracle's
 * FP64 values are the same numbers). */
enum {
    KM_DTYPE_F32 = 0,  /* X is N x D float */
    KM_DTYPE_BF16 = 1  /* X is N x D bfloat16 (uint16 bit patterns) */
};

typedef struct {
    int32_t algo;        /* KM_ALGO_* */
    int32_t grouping;    /* KM_GROUP_* */
    int32_t validate;    /* nonzero: reject X / init_centroids with NaN or Inf */
    int32_t profile;     /* nonzero: time every kernel with CUDA events (the
                            fit loop then runs launch by launch, not as a
                            graph); see kmeans_get_profile */
    void *stream;        /* cudaStream_t; NULL = legacy default stream */
    int32_t dense;       /* KM_DENSE_*: engine of the dense (all-pairs) passes */
    float dense_switch;  /* a filtered iteration whose global filter leaves more
                            than this fraction of the points runs the dense pass
                            instead (which also makes every bound exact again);
                            0 = library default (0.7 with the tensor-core
                            engine, 0.9 without), >= 1 = never */
    int32_t dtype;       /* KM_DTYPE_*: storage type of X */
    int32_t pad0;        /* must be zero */
    int32_t surv_grab;   /* survivor queue schedule: entries a warp of the D <= 64
                            survivor kernel claims at a time (a multiple of 32 in
                            [32, 1024]; 0 = 32) */
    int32_t pad1;        /* must be zero */
    int64_t reserved[3]; /* must be zero */
} kmeans_options;

/* kmeans_options.dense: how dense passes (iteration 0, plain Lloyd) compute
 * distances.  Both give exact labels. */
enum {
    KM_DENSE_AUTO = 0, /* tensor cores (tcgen05, bfloat16 split in three
                          products, FP32 accumulation) when the shape allows
                          (D = 64 or 128, K <= 256), else FP32 */
    KM_DENSE_FP32 = 1  /* FP32 CUDA cores, direct differences */
};

/* kernel kinds reported by kmeans_get_profile */
enum {
    KM_KERNEL_DENSE = 0,    /* dense assignment (iteration 0, plain Lloyd) */
    KM_KERNEL_MOVES = 1,    /* cluster sums for moved points (dense path) */
    KM_KERNEL_FILTER = 2,   /* global filter + survivor compaction */
    KM_KERNEL_SURVIVOR = 3, /* group/point filter + survivor distances */
    KM_KERNEL_UPDATE = 4,   /* centroid update, drift, objective */
    KM_KERNEL_OTHER = 5,    /* loop control, rebase, bounds export */
    KM_KERNEL_SETTLE = 6,   /* exact settle of the tensor-core pass's near-ties */
    KM_KERNEL_STATS = 7,    /* full recompute of the cluster sums (label sort) */
    KM_KERNEL_PROPOSAL = 8, /* the learned proposal: MLP, centroid table, seeded bounds */
    KM_KERNEL_KINDS = 9
};

/* kmeans_iter_stats.path */
enum {
    KM_PATH_FILTERED = 0,   /* global/group/point filters + survivor distances */
    KM_PATH_DENSE_FP32 = 1, /* every distance, FP32 CUDA cores */
    KM_PATH_DENSE_TC = 2    /* every distance, tensor cores + exact settle */
};

/* Per-iteration statistics (all counts are for that iteration).  A filtered
 * iteration whose global filter leaves more than a set fraction of the points
 * runs the dense pass instead (decided on the device). */
typedef struct {
    int32_t iter;          /* t */
    int32_t done;          /* the stop rule held after this iteration */
    int32_t path;          /* KM_PATH_*: how the assignment was computed */
    int32_t n_settle;      /* rows the tensor-core pass left to the exact settle */
    int64_t n_changed;     /* labels that changed (N at t = 0) */
    int64_t n_survivors;   /* points not kept by the global filter */
    int64_t n_scanned;     /* points still unresolved after tightening u */
    int64_t n_dist;        /* point-centroid distances evaluated: K per point in a dense
                              pass, and at most K per point otherwise (a point the FP32
                              results could not settle counts K, not its scan plus K) */
    int64_t n_recheck;     /* points whose label was settled in FP64 */
    double objective;      /* J_t = J(a_t, C^t) */
    double max_drift;      /* max_k ||c_k^{t+1} - c_k^t|| (rounded up) */
} kmeans_iter_stats;

/* Fill *opt with defaults: filtered algorithm, contiguous groups, no
 * validation, default stream. */
KM_API void kmeans_default_options(kmeans_options *opt);

/*
 * Create a context for one problem and store the initial centroids C^0.
 * X: N x D float32 (host or device; a device X is borrowed).
 * init_centroids: K x D float32 (host or device; copied).
 * Requires 1 <= K <= N < 2^31, 1 <= D <= 4096, 1 <= G <= K, K <= 65535.
 * opt may be NULL (defaults).  On success *out receives the context.
 * Unless profiling, the context's fit graph (kmeans_fit) is recorded here,
 * while the device still works on the copy of X.  Returns when the device
 * work it enqueued has finished (a host X is no longer read afterwards).
 * Errors: KM_EINVAL (bad sizes / null pointers / non-finite data when
 * validating), KM_ENOMEM, KM_ECUDA.  On failure *out is NULL and
 * kmeans_last_error(NULL) describes the failure (per thread).
 */
KM_API int kmeans_init(kmeans_ctx **out, const float *X, int64_t N, int32_t D,
                       int32_t K, int32_t G, const float *init_centroids,
                       const kmeans_options *opt);

/*
 * Run one iteration t: assignment from C^t (dense at t = 0, filtered after;
 * every distance for KM_ALGO_LLOYD), then the centroid update to C^{t+1}
 * with drift.  stats (nullable) receives the iteration's statistics.
 * Blocks until the iteration has finished on the device.
 */
KM_API int kmeans_iterate(kmeans_ctx *ctx, kmeans_iter_stats *stats);

/*
 * Iterate from the current state until the stop rule holds (at most max_iter
 * iterations in this call; tol >= 0), then assign every point to the returned
 * centroids.  Outputs (each nullable; host or device):
 *   labels    N int32   final assignment to the returned centroids
 *   centroids K x D f32 the returned centroids
 *   objective 1 double  J of that pair (FP64)
 *   n_iter    1 int32   iterations performed by this call
 * Without profiling, the loop runs as one CUDA graph whose body repeats
 * under a device-side loop condition set by the stop rule: no host round trip
 * per iteration.
 */
KM_API int kmeans_fit(kmeans_ctx *ctx, int32_t max_iter, double tol,
                      int32_t *labels, float *centroids, double *objective,
                      int32_t *n_iter);

/* Current labels (the last assignment made) into labels[N]. */
KM_API int kmeans_get_labels(kmeans_ctx *ctx, int32_t *labels);

/* Current centroids (those the next assignment will use) into C[K x D]. */
KM_API int kmeans_get_centroids(kmeans_ctx *ctx, float *C);

/* Statistics of iteration t (0 <= t < iterations run so far, at most the
 * last 4096 iterations are kept).  t = -1: the final assignment of the last
 * kmeans_fit (its path, label changes, distances and objective; iter is the
 * number of iterations that fit ran); KM_ESTATE before any fit. */
KM_API int kmeans_get_stats(kmeans_ctx *ctx, int32_t t, kmeans_iter_stats *stats);

/*
 * The per-point bounds, made valid for the current centroids: u[N] (upper
 * bound on ||x - c_a||), lbg[N] (lower bound on the distance to every other
 * centroid) and lb[N x G] (lower bound per centroid group, excluding the
 * point's own centroid).  Each output is nullable.  Only meaningful for
 * KM_ALGO_FILTERED after at least one iteration.
 */
KM_API int kmeans_get_bounds(kmeans_ctx *ctx, float *u, float *lbg, float *lb);

/*
 * Restart from new initial centroids (K x D, host or device): iteration
 * count, bounds, cluster sums, drift tables and statistics are reset; X,
 * sizes, options, device buffers and the recorded fit graph are kept.  Makes
 * no allocation.  Blocks until done.
 */
KM_API int kmeans_reset(kmeans_ctx *ctx, const float *init_centroids);

/*
 * Device time of each kernel kind since the context was created (or since
 * the last kmeans_reset), measured with CUDA events recorded on the
 * context's stream around every launch.  Only collected when
 * kmeans_options.profile is set.  kind: KM_KERNEL_*.  launches / ms nullable.
 */
KM_API int kmeans_get_profile(kmeans_ctx *ctx, int32_t kind, int64_t *launches, double *ms);

/* The grouping in use: grp[k] (nullable, K int32, host or device) = group of
 * centroid k (the caller's numbering), *n_groups (nullable) = the number of
 * groups (G, or fewer for a clustered grouping that left groups empty). */
KM_API int kmeans_get_groups(kmeans_ctx *ctx, int32_t *grp, int32_t *n_groups);

/* Number of iterations run so far on this context. */
KM_API int kmeans_get_iteration(const kmeans_ctx *ctx, int32_t *t);

/*
 * One plain-Lloyd iteration that allocates nothing.  The paper has no
 * counterpart: this entry point is for callers that may not allocate device
 * memory at all -- a host framework that owns every byte of device memory
 * through its own pool, a latency-critical loop in which cudaMalloc/cudaFree
 * would synchronise the device, or a deployment that must reserve all memory
 * at start-up.
 *
 * From centroids C (K x D) it assigns every point of X (N x D) to its nearest
 * centroid (exact, ties to the lowest index) into labels[N], writes the
 * updated centroids (cluster means, an empty cluster keeps its centroid) to
 * C_new (K x D) and J(labels, C) to *objective (FP64): the same results as
 * kmeans_iterate on a KM_ALGO_LLOYD context at the same centroids.  Every
 * pointer must be device memory of the current device; the work is ordered on
 * `stream` (cudaStream_t, NULL = legacy default) and the call returns without
 * waiting for it.
 *
 * Scratch: the cluster sums, counts, a padded copy of C and the control block
 * live in one file-scope static device array of about 1.6 MB, which every GPU
 * that loads the library holds until the process exits.  Hence the limits
 * K <= KM_NOALLOC_MAX_K and D <= KM_NOALLOC_MAX_D (larger sizes: KM_EINVAL).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, and so does the first
 * call after the device's context was made anew (after cudaDeviceReset);
 * make that first call before any stream capture.  Every call shares the one array and clears what
 * it accumulates into, so calls that overlap on the GPU (on different
 * streams, or from threads without ordering) race and give wrong results.
 * No cudaMalloc, cudaFree or allocating library routine is called.  Errors:
 * KM_EINVAL, KM_ECUDA; the message is kmeans_last_error(NULL).
 */
#define KM_NOALLOC_MAX_K 1024
#define KM_NOALLOC_MAX_D 128
KM_API int kmeans_lloyd_step_noalloc(const float *X, int64_t N, int32_t D, const float *C,
                                     int32_t K, int32_t *labels, float *C_new,
                                     double *objective, void *stream);

/* ------------------------------------------------------------------------
 * Sharded iterations: one problem split by rows across processes (one per
 * GPU).  Each process makes a context over its own rows with the same C^0,
 * K, G and options.  An iteration is then
 *   kmeans_shard_assign   this shard's assignment from C^t (the filters and
 *                         the distance calculator of Sec. I, on its rows),
 *                         and its cluster sums about C^t: S (K x D, FP64),
 *                         Q (K, FP64: sum ||x - c_k^t||^2 over its points of
 *                         cluster k), cnt (K) and its number of label changes;
 *   (the caller sums S, Q, cnt and n_changed over the shards: one all-reduce)
 *   kmeans_shard_update   the update from the summed statistics: C^{t+1},
 *                         drift, J_t = sum_k Q_k and the stop rule, the same
 *                         on every shard.
 * The filters' bounds are per point, so they need no exchange; the drift is
 * computed from the same sums on every shard.  stats->done (of the update)
 * says the stop rule holds (no label changed, or a relative decrease of J
 * below tol); the caller stops then, or after its own iteration budget, and
 * makes a final assignment to the returned centroids: one more
 * kmeans_shard_assign, the all-reduce, and kmeans_shard_update with
 * final_pass = 1, which leaves the centroids as they are and writes J of
 * that assignment to *objective.  Labels stay local (kmeans_get_labels).
 * Arrays may be host or device memory.  Errors: KM_EINVAL, KM_ESTATE (an
 * assignment without its update, or the reverse), the codes of
 * kmeans_iterate.
 * ------------------------------------------------------------------------ */
KM_API int kmeans_shard_assign(kmeans_ctx *ctx, double tol, double *S, double *Q, int64_t *cnt,
                               int64_t *n_changed);
KM_API int kmeans_shard_update(kmeans_ctx *ctx, int32_t final_pass, const double *S, const double *Q,
                               const int64_t *cnt, int64_t n_changed, kmeans_iter_stats *stats,
                               double *objective);

/*
 * k-means++ seeding (an initialisation beside the caller's centroids; the
 * paper takes them as given): the first centre is the point floor(u[0] * N),
 * each further centre j a point drawn with probability proportional to
 * D(x)^2, its squared distance to the nearest centre chosen so far
 * (Arthur and Vassilvitskii, SODA 2007), using the uniform u[j] in [0, 1).
 * The draw is exact: D(x)^2 in FP64 (sum over i ascending, no fused
 * multiply-add), weights floor(D(x)^2 * 2^s) as 64-bit integers with 2^s the
 * power of two that puts the largest in [2^31, 2^32), T = floor(u[j] * W)
 * for their sum W, and the centre is the first point whose running weight
 * sum exceeds T (uniform floor(u[j] * N) when W = 0) -- so the same uniforms
 * give the same centres on any implementation.  X: N x D float32, device
 * memory; u: K doubles; centroids: K x D float32 out; indices: K int64 out
 * (nullable); u and the outputs may be host or device memory.  Work on
 * `stream` with stream-ordered scratch (N + N / 1024 doubles); returns after
 * it finished.  Errors: KM_EINVAL, KM_ENOMEM, KM_ECUDA; message in
 * kmeans_last_error(NULL).
 */
KM_API int kmeans_init_kmeanspp(const float *X, int64_t N, int32_t D, int32_t K, const double *u,
                                float *centroids, int64_t *indices, void *stream);

/* Free the context and everything it allocated.  NULL is a no-op. */
KM_API void kmeans_destroy(kmeans_ctx *ctx);

/* Message for the last failure on ctx, or for the calling thread's last
 * failed kmeans_init when ctx is NULL.  Never NULL. */
KM_API const char *kmeans_last_error(const kmeans_ctx *ctx);

/* Kernel launches issued from the host by this library in this process (all
 * contexts; a graph counts its kernels once, when it is recorded). */
KM_API int64_t kmeans_launch_count(void);

/* Kernels of this context that have run on the device, graph replays
 * included, as of the end of the last blocking call. */
KM_API int kmeans_get_kernel_count(const kmeans_ctx *ctx, int64_t *n);

/* ------------------------------------------------------------------------
 * Batched form: many independent problems (uneven N, D, K) fitted by one
 * CUDA graph launch.  Every problem keeps its own context (bounds, sums,
 * loop control); the graph holds one chain per problem (arm -> iteration 0
 * -> while(not done){ iteration } -> final assignment -> objective), so the
 * problems run concurrently and each stops on its own rule.
 * ------------------------------------------------------------------------ */
typedef struct kmeans_batch kmeans_batch;

typedef struct {
    const float *X;               /* N x D row-major, host or device; a device X is borrowed */
    int64_t N;
    int32_t D, K, G;
    const float *init_centroids;  /* K x D, host or device (copied at init) */
} kmeans_problem;

/* Create the contexts of n_problems problems with the options opt (NULL:
 * defaults; profile must be 0; opt->stream is shared by all problems).
 * tune_cache (nullable): path of the autotuner's cache.  When given, each
 * size bucket (D, ceil log2 K, ceil log2 N) takes its settings from the file,
 * or has them chosen by timing short fits (10 iterations) of the bucket's
 * largest problem, one setting at a time: the dense/filtered switch (0.5,
 * 0.7, 0.9, 1 = never), then the dense engine (tensor cores or FP32 CUDA
 * cores, when the tensor cores take the shape), then the survivor queue
 * schedule (32, 64 or 128 entries claimed per warp); the choices are written
 * to the file, one "D logK logN switch dense grab" line per bucket (lines
 * of an older "D logK logN switch" form are read with the defaults for the
 * rest).  Errors: KM_EINVAL (bad arguments), the codes of kmeans_init. */
KM_API int kmeans_batch_init(kmeans_batch **out, int32_t n_problems, const kmeans_problem *problems,
                             const kmeans_options *opt, const char *tune_cache);

/* Fit every problem (at most max_iter >= 1 iterations each, tol as kmeans_fit)
 * with one graph launch; the graph is recorded on the first call and reused
 * while max_iter, tol and the problems' state allow.  All problems must be
 * fresh (after init or kmeans_batch_reset) or all continuing. */
KM_API int kmeans_batch_fit(kmeans_batch *b, int32_t max_iter, double tol);

/* Results of problem i: labels[N], centroids[K x D], objective, iterations
 * run by the last fit (each nullable; host or device memory). */
KM_API int kmeans_batch_get(kmeans_batch *b, int32_t i, int32_t *labels, float *centroids, double *objective,
                            int32_t *n_iter);

/* Restart every problem from its initial centroids (no allocation). */
KM_API int kmeans_batch_reset(kmeans_batch *b);

/* The dense/filtered switch the batch uses for problem i. */
KM_API int kmeans_batch_get_switch(const kmeans_batch *b, int32_t i, float *dense_switch);

/* All tuned settings of problem i (each nullable): the switch, the dense
 * engine (KM_DENSE_*) and the survivor queue schedule (entries per claim). */
KM_API int kmeans_batch_get_tuning(const kmeans_batch *b, int32_t i, float *dense_switch, int32_t *dense,
                                   int32_t *surv_grab);

KM_API void kmeans_batch_destroy(kmeans_batch *b);

/* Message of the last failed batch call (b NULL: of the last failed
 * kmeans_batch_init in this thread). */
KM_API const char *kmeans_batch_last_error(const kmeans_batch *b);

/* ------------------------------------------------------------------------
 * The proposal network on the tensor cores: training and inference.
 *
 * A layered form on top of the filtered method (the paper has no learned
 * component): a multilayer perceptron  D -> hidden -> hidden -> classes  with
 * GELU activations (the exact erf form), trained with softmax cross-entropy
 * (mean over the batch) and Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected
 * moments) on FP32 master weights.  Every matrix product runs on tcgen05 with
 * bfloat16 operands (weights, inputs, activations and backpropagated
 * gradients rounded to bfloat16) and FP32 accumulation; the bias, GELU,
 * softmax, loss, gradient and update arithmetic is FP32.  Parameters are one
 * FP32 vector in the order W1 (hidden x D), b1, W2 (hidden x hidden), b2,
 * W3 (classes x hidden), b3 -- row-major, output index first (z = W a + b).
 * Limits: D <= 256, hidden <= 256, classes <= 512.  All work is ordered on
 * the stream given at creation; every call below returns after it finished.
 * Errors: KM_EINVAL, KM_ENOMEM, KM_ECUDA, KM_ETIMEOUT (a bounded wait in a
 * tensor-core product gave up); message in kmeans_mlp_last_error.
 * ------------------------------------------------------------------------ */
typedef struct kmeans_mlp kmeans_mlp;

/* Create a network on the current device with Xavier-uniform weights
 * (U(-a, a), a = sqrt(6 / (fan_in + fan_out)), from a counter-based
 * generator seeded with `seed`) and zero biases.  On failure *out is NULL
 * and kmeans_mlp_last_error(NULL) has the message. */
KM_API int kmeans_mlp_create(kmeans_mlp **out, int32_t D, int32_t hidden, int32_t classes, uint64_t seed,
                             void *stream);

/* Replace the FP32 master weights (six arrays, host or device) and restart
 * Adam (zero moments, step 0). */
KM_API int kmeans_mlp_set_params(kmeans_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2,
                                 const float *W3, const float *b3);

/* Copy the FP32 master weights out (each pointer nullable; host or device). */
KM_API int kmeans_mlp_get_params(kmeans_mlp *m, float *W1, float *b1, float *W2, float *b2, float *W3, float *b3);

/* One forward and backward pass on a given batch, without an update: X is
 * B x D FP32, y B class indices (device memory), B a multiple of 128.  Writes
 * the gradient of the mean cross-entropy with respect to every parameter to
 * grad (device, the parameter vector's layout) and the mean loss to *loss
 * (nullable). */
KM_API int kmeans_mlp_gradient(kmeans_mlp *m, const float *X, const int32_t *y, int32_t B, double *loss,
                               float *grad);

/* `steps` Adam steps (learning rate lr) on batches of `batch` rows (a
 * multiple of 128) drawn with replacement from the N training rows (X N x D
 * FP32, labels N int32; device memory) by a counter-based generator seeded
 * with `seed`; seed ~0 instead takes rows 0 .. batch-1 in every step (plain
 * full-batch steps, N >= batch).  With K > 0 the labels are centroid indices
 * in [0, K) and the class of a row is its centroid's contiguous group,
 * floor(label * classes / K); with K = 0 they are the classes themselves.
 * One step is recorded once as a CUDA graph and replayed.  *mean_loss and
 * *accuracy (nullable) receive the mean cross-entropy and the fraction of
 * rows whose largest logit was their class, over the rows of all steps. */
KM_API int kmeans_mlp_train(kmeans_mlp *m, const float *X, int64_t N, const int32_t *labels, int32_t K,
                            int64_t steps, int32_t batch, float lr, uint64_t seed, double *mean_loss,
                            double *accuracy);

/* pred[n] = the class with the largest logit (the first on ties) for N rows
 * of X (N x D FP32; X and pred device memory), in chunks of up to 2^17 rows. */
KM_API int kmeans_mlp_predict_net(kmeans_mlp *m, const float *X, int64_t N, int32_t *pred);

KM_API void kmeans_mlp_destroy(kmeans_mlp *m);

/* Message of the last failure on m (m NULL: of the calling thread's last
 * failed kmeans_mlp_create). */
KM_API const char *kmeans_mlp_last_error(const kmeans_mlp *m);

/* Learned group proposal (a layered form on top of the filtered method; the
 * paper has no learned component).  An MLP  D -> hidden -> hidden -> G  with
 * GELU activations (the exact erf form) predicts each point's group as the
 * largest of its G logits, on the tensor cores (the network above).  Weights
 * row-major, output index first: W1 hidden x D, b1 hidden, W2 hidden x
 * hidden, b2 hidden, W3 G x hidden, b3 G (FP32, host or device; copied;
 * hidden <= 256, D <= 256, G <= 512).  With a proposal set, iteration 0 of
 * the filtered method (KM_ALGO_FILTERED only) replaces its dense pass by:
 * the prediction; exact FP32 distances to the predicted group's centroids,
 * giving a label candidate c and u >= d(x, c); group bounds by the triangle
 * inequality, lb_g = min_{c' in g} d(c, c') - u, from a K x G table of
 * centroid distances; then the ordinary filtered assignment (global, group
 * and point filters, distance calculator; Sec. I), so labels are exactly
 * those without a proposal -- a wrong prediction only costs work.  All six
 * pointers NULL: remove the proposal.  Allocates the network, N int32
 * predictions, its chunk buffers and the K x G table.  Errors: KM_EINVAL
 * (Lloyd context, hidden outside [1, 256], D > 256 or G > 512, some pointers
 * NULL), KM_ENOMEM, KM_ECUDA. */
KM_API int kmeans_set_proposal(kmeans_ctx *c, const float *W1, const float *b1, const float *W2, const float *b2,
                               const float *W3, const float *b3, int32_t hidden);

/* The proposal MLP alone: pred[n] = argmax_g logits(X[n]) (first maximum)
 * for N points of dimension D, G classes; weights as above (FP32, rounded to
 * bfloat16 for the tensor-core products).  X and pred are device memory of
 * the current device; the work runs on `stream` (NULL = legacy default) with
 * a temporary network, and the call returns after it finished.  Errors:
 * KM_EINVAL, KM_ENOMEM, KM_ECUDA, KM_ETIMEOUT; message in
 * kmeans_last_error(NULL). */
KM_API int kmeans_mlp_predict(const float *X, int64_t N, int32_t D, const float *W1, const float *b1,
                              const float *W2, const float *b2, const float *W3, const float *b3, int32_t hidden,
                              int32_t classes, int32_t *pred, void *stream);

/* Device self-test of the square-root bounds behind every distance bound
 * (the upper bound u and the lower bounds lb of the filters, Sec. I): the
 * library bounds sqrt(v) by the hardware approximation (sqrt.approx.f32)
 * moved two steps of the bit pattern down / up, which is valid when the
 * approximation is within one step of the correctly rounded root.  This
 * checks lo >= 0 and lo^2 <= v <= hi^2 (squares in FP64, exact) for all 2^31
 * non-negative float bit patterns v on the current device, synchronously
 * (a few milliseconds), and writes the number of failures (0 expected) to
 * *violations.  Allocates 8 bytes of device memory for the duration.  Errors:
 * KM_EINVAL (NULL), KM_ENOMEM, KM_ECUDA; message in kmeans_last_error(NULL). */
KM_API int kmeans_selftest_sqrt(int64_t *violations);

/* Device self-test of the bounded waits: one thread waits on an mbarrier that
 * nothing arrives at, giving up after `polls` bounded try-waits (each returns
 * within a hardware time limit) exactly as the library's kernels do, records
 * the time-out in a control block and returns.  Expected result: KM_ETIMEOUT,
 * with the device still usable afterwards.  Errors: KM_EINVAL (polls outside
 * [1, 65536]), KM_ENOMEM, KM_ECUDA; message in kmeans_last_error(NULL). */
KM_API int kmeans_selftest_timeout(int32_t polls);

/* Testing hook: after `after` more device allocations by contexts (>= 0),
 * every further one fails as out of memory (KM_ENOMEM from the call that
 * made it); a negative value switches the hook off.  Process-wide. */
KM_API void kmeans_debug_fail_alloc(int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* KPYNQ_H */
