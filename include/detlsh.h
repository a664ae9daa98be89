/*
 * detlsh.h -- C-ABI of the GB300 (sm_103a) DET-LSH hot path.
 *
 * DET-LSH (arXiv 2603.24920) answers c^2-k-ANN queries in Euclidean space:
 *   build : K*L Gaussian projections (Eq. 1), dynamic equal-frequency encoding
 *           of each projected coordinate into N_r regions (Sec. III-A, Alg. 1),
 *           and one DE-Tree per projected space (Sec. III-B, Alg. 2);
 *   query : range queries over the L DE-Trees with node lower bounds
 *           (Alg. 3, Sec. IV-C) and the optimised leaf handling of Sec. VI-B2,
 *           inside the c^2-k-ANN loop of Alg. 5 started at the "magic" r_min
 *           of Sec. V-B1, then exact-distance verification and top-k.
 * Every step runs in CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions
 *   - Pointers named "data", "queries", "ids", "dists" may be host or device
 *     memory (the library asks the CUDA driver which); the library copies as
 *     needed.  Accessors named detlsh_get_* write host memory.
 *   - The caller owns every input and output buffer; the library owns the
 *     index (device memory) until detlsh_free.
 *   - Every function returns a detlsh_status.  On error no output is written
 *     and an existing index stays valid.
 *   - An index is immutable after build; detlsh_query may be called from
 *     several host threads on distinct streams.
 *   - "stream" arguments are cudaStream_t values (NULL = legacy default).
 */
#ifndef DETLSH_H
#define DETLSH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DETLSH_OK = 0,
    DETLSH_ERR_INVALID_ARG = -1,     /* a size or parameter is out of range     */
    DETLSH_ERR_NONFINITE_INPUT = -2, /* NaN/Inf in data or queries, or a
                                        projection overflows FP32              */
    DETLSH_ERR_OOM = -3,             /* device or host allocation failed       */
    DETLSH_ERR_CUDA = -4,            /* a CUDA runtime call failed             */
    DETLSH_ERR_CAPACITY = -5,        /* an internal work list overflowed       */
    DETLSH_ERR_NO_DEVICE = -6,       /* no usable CUDA device                  */
    DETLSH_ERR_SCRATCH_LIMIT = -7,   /* the request does not fit the fixed
                                        scratch of detlsh_query_noalloc        */
    DETLSH_ERR_TIMEOUT = -8,         /* a device-side pipeline wait ran past
                                        its limit (the kernel stopped cleanly) */
    DETLSH_ERR_IO = -9,              /* an index file could not be opened,
                                        read or written                        */
    DETLSH_ERR_FORMAT = -10          /* not an index file of this format:
                                        magic, version, byte order, sizes or
                                        checksum                               */
} detlsh_status;

/* Node boxes used by the range query's lower bound (Sec. IV-C). */
enum { DETLSH_BOX_PREFIX = 0, /* regions of the node's iSAX prefix (paper)   */
       DETLSH_BOX_TIGHT = 1 /* min/max code of the node's points           */ };

/* Encoding scheme of the projected coordinates (Sec. III-A). */
enum { DETLSH_ENC_DYNAMIC = 0, /* sampled equal-frequency breakpoints (paper) */
       DETLSH_ENC_STATIC = 1   /* N(0,1) equal-mass breakpoints, ends -inf and
                                  +inf, no sample (the iSAX scheme the paper
                                  compares against)                         */ };

/* Precision of the exact-distance verification step (Alg. 5, top-k). */
enum { DETLSH_PREC_FP32 = 0,        /* FP32 distances over every candidate  */
       DETLSH_PREC_BF16_REFINE = 1  /* BF16 tensor-core scores, then an FP32
                                       re-rank (see rerank_mult)             */ };

/* How Alg. 5 chooses its starting radius r_min (Sec. V-B1). */
enum { DETLSH_RMIN_MAGIC = 0, /* the "magic" r_min: the smallest radius of the
                                 grid c^j (j = -127..127) whose union over the
                                 L trees holds beta*n + k points; condition 1
                                 ends the first round                        */
       DETLSH_RMIN_FIXED = 1, /* a given r_min: Alg. 5 runs its radius loop
                                 r_min c^i (i = 0..253, then unbounded) with
                                 condition 2 (k points of S within c*r)      */
       DETLSH_RMIN_CONTINUOUS = 2 /* the smallest r_min off any grid: the
                                 squared radius is the (beta*n + k)-th
                                 smallest of the points' smallest leaf lower
                                 bound over the trees, so eps and c cancel;
                                 condition 1 ends the first round           */ };

typedef struct detlsh_index detlsh_index;

typedef struct {
    int32_t L;              /* projected spaces = DE-Trees, 1..16 (default 4)      */
    int32_t K;              /* dimensions per projected space, 1..16 (default 16)  */
    int32_t N_r;            /* regions per dimension, power of two in [2,256]
                               (default 256, Sec. III-A)                           */
    int32_t max_size;       /* leaf capacity of Alg. 2, >= 1 (default 64)          */
    uint64_t seed;          /* projection and sample seed                          */
    double sample_frac;     /* breakpoint sample n_s / n, in (0,1] (default 0.1)  */
    int32_t box_mode;       /* DETLSH_BOX_PREFIX (default) or DETLSH_BOX_TIGHT     */
    int32_t keep_bf16;      /* 1: also keep a BF16 copy of the data (default 1)    */
    int32_t keep_projections; /* 1: keep the n x L*K projections (default 0)      */
    int32_t encoding;       /* DETLSH_ENC_DYNAMIC (default) / DETLSH_ENC_STATIC    */
    int32_t tree_group;     /* trees built per pass, 0..L; 0 (default) = as many as
                               fit in half the free device memory.  The trees do
                               not depend on it.                                   */
} detlsh_build_params;

typedef struct {
    double beta;            /* false-positive budget: stop at beta*n + k
                               candidates (Alg. 5; default 0.1, Sec. VI-A)         */
    double c;               /* approximation ratio, 1.1 <= c <= 16 (default 1.5)   */
    int32_t precision;      /* DETLSH_PREC_FP32 (default) / DETLSH_PREC_BF16_REFINE */
    int32_t rerank_mult;    /* BF16 path: 0 (default) = re-rank in FP32 the
                               certified pool (every candidate whose score interval
                               can reach the k best), so the answer equals the
                               FP32 path's exactly; r > 0 = re-rank the r*k best
                               BF16 scores (an approximation)                      */
    int32_t rmin_policy;    /* DETLSH_RMIN_MAGIC (default) / DETLSH_RMIN_FIXED     */
    double r_min;           /* DETLSH_RMIN_FIXED: the starting radius (> 0); the
                               FP32 path only (precision must be FP32)             */
    int32_t per_tree;       /* 0 (default): leaves join S in (LB^2, leaf) order with
                               the budget checked after each leaf (the priority
                               queue of Sec. VI-B2); 1: Alg. 5 as printed, each
                               tree's range query whole, checked after each tree
                               (DETLSH_RMIN_MAGIC only; candidate buffers of n)  */
} detlsh_query_params;

/* Fill *p with the defaults listed above (Sec. V-B1, Sec. VI-A). */
int detlsh_default_build_params(detlsh_build_params *p);
int detlsh_default_query_params(detlsh_query_params *p);

/*
 * Build the index over n points of dimension d (row-major FP32, n*d values).
 * Encoding phase (Sec. III-A, Alg. 1) and indexing phase (Sec. III-B, Alg. 2):
 *   A      : K*L projection vectors, entries N(0,1) (Eq. 1), drawn from seed;
 *   P      : every h_t(o) = a_t . o, the exact dot product rounded once to FP32;
 *   B      : per projected dimension, interior breakpoints = equal-frequency
 *            order statistics of a ~sample_frac sample, ends = min/max of all
 *            n points;
 *   codes  : region index of every projected coordinate (8-bit symbol);
 *   trees  : per projected space, 2^K first-layer nodes split on the most even
 *            dimension while a node holds more than max_size points.
 * Requirements: 1 <= n < 2^31, 1 <= d <= 65536, L*K <= 256.  The data is
 * copied; the caller's buffer may be freed afterwards.
 * Errors: INVALID_ARG, NONFINITE_INPUT, OOM, CUDA, NO_DEVICE.
 */
int detlsh_build(const float *data, int64_t n, int32_t d, int32_t L, int32_t K,
                 int32_t N_r, uint64_t seed, detlsh_index **out);
int detlsh_build_ex(const float *data, int64_t n, int32_t d, const detlsh_build_params *p,
                    void *stream, detlsh_index **out);

/*
 * c^2-k-ANN queries (Alg. 5).  queries: m x d row-major FP32.  For each query:
 * r_min is the smallest radius of the grid r_j = c^j (j = -127..127) whose
 * union over the L range queries holds at least beta*n + k points (magic
 * r_min, Sec. V-B1); Alg. 5 then runs at r_min: trees in order, the leaves of
 * each range query (lower bound <= eps*r, whole leaves, Sec. VI-B2) entering
 * S in ascending lower-bound order (ties: leaf order) until |S| >= beta*n + k;
 * eps^2 = chi^2_{alpha1}(K) with alpha1 = exp(-1/L) (Eq. 2, Lemma 3).
 * Output: ids (int64, m x k) and Euclidean dists (FP32, m x k), ascending,
 * ties by smaller id.  detlsh_query uses beta = 0.1 and FP32 verification.
 * Requirements: m >= 0, 1 <= k <= min(n, 1024).
 * Errors: INVALID_ARG, NONFINITE_INPUT, OOM, CUDA, CAPACITY.
 */
int detlsh_query(const detlsh_index *ix, const float *queries, int64_t m, int32_t k, double c,
                 int64_t *ids, float *dists);
/* As detlsh_query (Alg. 5 from the r_min of Sec. V-B1, verification, top-k),
 * with per-query k (nullable: k_max for all) and parameters (beta, c, precision,
 * the r_min policy of Sec. V-B1 / Alg. 5, the priority order of Sec. VI-B2);
 * rows are k_max wide, padded with id -1 and dist +inf past the query's k. */
int detlsh_query_ex(const detlsh_index *ix, const float *queries, int64_t m,
                    const int32_t *k_per_query, int32_t k_max, const detlsh_query_params *qp,
                    void *stream, int64_t *ids, float *dists);

/*
 * detlsh_query_noalloc -- the same queries and results as detlsh_query_ex
 * (one k for every query, rmin_policy DETLSH_RMIN_MAGIC, per_tree 0 or 1),
 * for callers that cannot allocate device memory while serving: a process
 * whose framework has already claimed nearly all device memory for its own
 * pool, a latency-critical path where cudaMalloc/cudaFree would stall the
 * device, or a deployment that forbids allocation after start-up.  The paper
 * has no counterpart; this entry point only changes where scratch memory
 * comes from.
 *
 * All scratch lives in one fixed 32 MiB device array compiled into the
 * library (every GPU that loads the library holds it until the process
 * exits); the call allocates nothing.  queries (m x d FP32), ids (m x k
 * int64) and dists (m x k FP32) must be device memory owned by the caller,
 * on the index's device, which must be the current device; queries must be
 * 16-byte aligned when d is a multiple of 4 (4-byte aligned otherwise), ids
 * 8-byte and dists 4-byte aligned.
 * Requests that do not fit (the query projections, BF16 query copy and one
 * per-CTA working slot, which grows with the index's leaf count and with
 * beta*n + k, or with n when per_tree = 1) fail with
 * DETLSH_ERR_SCRATCH_LIMIT; smaller batches fit.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every
 * call reuses the same array and clears the part it uses at its start, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  Returns after the results are written.
 * Errors: as detlsh_query_ex (NONFINITE_INPUT before the query kernel runs),
 * plus SCRATCH_LIMIT; INVALID_ARG for host pointers, buffers on another
 * device or misaligned, and for rmin_policy other than DETLSH_RMIN_MAGIC.
 */
int detlsh_query_noalloc(const detlsh_index *ix, const float *queries, int64_t m, int32_t k,
                         const detlsh_query_params *qp, void *stream, int64_t *ids,
                         float *dists);

/*
 * Index files (the index of Sec. III-B, Alg. 2, with the encoding of Sec.
 * III-A, kept between processes).  The paper builds its index in memory and
 * reports its size and build cost (Sec. VI, encoding and indexing); a file
 * lets a serving process answer queries without rebuilding.
 *
 * detlsh_save writes everything the queries and accessors read: the build
 * parameters, eps^2 (Eq. 2), the FP32 data, A (Eq. 1), the breakpoints, the
 * sample ids, the codes, each tree's perm, leaf_begin, leaf boxes and prefix
 * lengths, leaf_of, the leaf-run hulls, and the BF16 copy and projections when
 * the index has them.  Layout: a fixed 672-byte header (magic "DETLSHIX",
 * format version 1, byte-order mark, parameters, per-tree leaf counts and
 * offsets), the arrays in a fixed order, each behind a 16-byte tag and byte
 * count, then a 64-bit checksum of everything before it.  Arrays are in the
 * host's byte order.  The file is written as path + ".tmp" and renamed, so a
 * failed save leaves no partial file under path.  stream orders the
 * device-to-host copies; the call returns when the file is closed.
 * Errors: INVALID_ARG (null index or path), IO, CUDA, OOM (pinned staging).
 *
 * detlsh_load reads such a file into a new index on the current device (the
 * caller frees it with detlsh_free); queries on it return what they return on
 * the saved index.  The header is checked before any device call: a missing
 * or unreadable file gives IO, a file that is not of this format (magic,
 * version, byte order, parameters out of range, inconsistent leaf offsets)
 * gives FORMAT; so do section sizes that disagree with the header, a short
 * file, trailing bytes and a checksum mismatch.  The checksum detects
 * accidental damage, not deliberate tampering: load only files you trust.
 * On error *out is NULL and nothing stays allocated.
 * Errors: INVALID_ARG (null path or out), IO, FORMAT, NO_DEVICE, OOM, CUDA.
 */
int detlsh_save(const detlsh_index *ix, const char *path, void *stream);
int detlsh_load(const char *path, void *stream, detlsh_index **out);

/* Release the index and its device memory.  NULL is accepted. */
int detlsh_free(detlsh_index *ix);

/* Human-readable text of a status code (static storage). */
const char *detlsh_status_string(int status);

/* ---------------------------------------------------------------------------
 * Introspection and parity accessors (host outputs).
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    int32_t d, L, K, N_r, max_size, box_mode, has_bf16;
    int64_t sample_size;        /* points used for the breakpoints           */
    int64_t num_leaves[16];     /* leaves of each DE-Tree                     */
    int64_t max_leaf_size;
    double eps2;                /* eps^2 of Eq. 2                             */
    int64_t device_bytes;       /* device memory held by the index           */
    int64_t projection_fallbacks; /* projections computed by the exact
                                     big-integer path during the build       */
    int32_t encoding;           /* DETLSH_ENC_DYNAMIC / DETLSH_ENC_STATIC     */
} detlsh_info;

int detlsh_get_info(const detlsh_index *ix, detlsh_info *info);
/* Projection vectors A, (L*K) x d, row t = tree*K + dim (Eq. 1). */
int detlsh_get_projection_matrix(const detlsh_index *ix, float *A);
/* Sampled point ids, ascending (sample_size values; the n_s = 0.1 n sample
 * of Sec. III-A). */
int detlsh_get_sample(const detlsh_index *ix, int64_t *ids);
/* Breakpoints, (L*K) x (N_r+1) (Sec. III-A). */
int detlsh_get_breakpoints(const detlsh_index *ix, float *B);
/* Codes, n x (L*K) bytes, point-major (Alg. 1). */
int detlsh_get_codes(const detlsh_index *ix, uint8_t *codes);
/* Projections h(o) of Eq. 1, n x (L*K); only if built with keep_projections. */
int detlsh_get_projections(const detlsh_index *ix, float *P);
/* DE-Tree t (Alg. 2): leaves in canonical order (first-layer key ascending,
 * child 0 before child 1), perm = point ids leaf by leaf (ascending within a
 * leaf), leaf_begin (num_leaves+1), box lo/hi and prefix lengths
 * (num_leaves x K bytes each), leaf_of (n). */
int detlsh_get_tree(const detlsh_index *ix, int32_t t, int64_t *perm, int64_t *leaf_begin,
                    uint8_t *box_lo, uint8_t *box_hi, uint8_t *nbits, int64_t *leaf_of);
/* Squared-radius grid of the magic r_min (Sec. V-B1; eps^2 from Eq. 2):
 * T(j) = fp32(eps^2 c^(2j)), j = -127..127, T(127) = inf. */
int detlsh_get_level_table(const detlsh_index *ix, double c, float *T);
/* Device times (CUDA events on the caller's stream) of the last build and of
 * the last query call on this index, the number of kernels each launched,
 * and the work the last query call did. */
typedef struct {
    float build_ms;            /* whole build                                   */
    float sample_ms;           /* Bernoulli sample + sample projections         */
    float breakpoints_ms;      /* radix sort of the sample columns + extraction */
    float encode_ms;           /* projections of all n points + region codes    */
    float trees_ms;            /* L DE-Tree layouts + leaf-run hulls            */
    float query_ms;            /* whole last query call (device part)           */
    float query_project_ms;    /* query projections                             */
    float query_kernel_ms;     /* the persistent query kernel                   */
    int64_t build_launches;    /* kernels launched by the build                 */
    int64_t query_launches;    /* kernels launched by the last query call       */
    int64_t query_count;       /* queries in the last call                      */
    int64_t query_candidates;  /* sum of |S| over those queries                 */
    int64_t query_leaves;      /* leaves whose bound was computed (expanded)    */
    int64_t query_blocks;      /* leaf-run hulls whose bound was computed       */
    int64_t query_points_visited; /* leaf points visited by the union counts   */
    int64_t query_reranked;    /* rows the BF16 path re-ranked in FP32          */
} detlsh_timings;
int detlsh_get_timings(const detlsh_index *ix, detlsh_timings *t);

/* Exact FP32 projections (Eq. 1) of m rows with the index's A (m x L*K, host
 * or device in/out), the same kernels the build uses. */
int detlsh_project(const detlsh_index *ix, const float *rows, int64_t m, float *out,
                   void *stream);
/* Candidate sets of Alg. 5 for m queries: S (host, m x cap, arrival order
 * unspecified), S_size, j* (radius grid index of r_min) and i* (tree at which
 * |S| reached beta*n + k; -1 when beta*n + k > n and S is every point).
 * Fails with CAPACITY if a set exceeds cap. */
int detlsh_query_candidates(const detlsh_index *ix, const float *queries, int64_t m, int32_t k,
                            const detlsh_query_params *qp, int64_t cap, int64_t *S,
                            int64_t *S_size, int32_t *jstar, int32_t *istar);

/*
 * Queries that can be captured in a CUDA graph (batched serving: the paper has
 * no counterpart; the same Alg. 5 queries and results as detlsh_query_ex).
 *
 * detlsh_query_reserve fixes the query parameters (beta, c, precision,
 * rerank_mult, r_min policy) and the largest batch (m_max queries, k <=
 * k_max) and allocates every buffer the queries need, in buffers of their
 * own.  It is synchronous; call it before any capture, and again whenever the
 * parameters or sizes change (which invalidates graphs captured earlier).
 * Errors: INVALID_ARG (as detlsh_query_ex, or m_max < 1), OOM, CUDA.
 *
 * detlsh_query_async enqueues one batch on `stream` and returns without
 * waiting: it allocates nothing, copies nothing to or from the host and never
 * synchronises, so the call can be captured and the graph replayed with new
 * query contents in the same buffers.  queries (m x d FP32), k_per_query
 * (nullable, m entries), ids (m x k_max) and dists (m x k_max) must be device
 * memory, m <= m_max, k_max <= the reserved k_max.  Errors found on the host
 * (INVALID_ARG: arguments as above or no reservation; CUDA) are returned;
 * errors found on the device (NONFINITE_INPUT for a query holding NaN/Inf,
 * INVALID_ARG for a per-query k outside [1, k_max], CAPACITY) are written to
 * *status (one device int32, 0 = OK) when the batch completes; the outputs of
 * a batch with a non-zero status are unspecified.  Calls on one index must
 * not overlap on the GPU (one stream, or ordered by the caller).
 */
int detlsh_query_reserve(detlsh_index *ix, int64_t m_max, int32_t k_max,
                         const detlsh_query_params *qp);
int detlsh_query_async(const detlsh_index *ix, const float *queries, int64_t m,
                       const int32_t *k_per_query, int32_t k_max, void *stream, int64_t *ids,
                       float *dists, int32_t *status);

/*
 * Tuning of the query kernel (batched serving; the paper has no counterpart:
 * these knobs change how the work of Alg. 3 and Alg. 5 is scheduled on the
 * GPU, never the candidate sets or the answers).
 *   query_ctas_per_sm  persistent query CTAs per SM, 1..5; 0 = as many as fit
 *                      (default 0, i.e. 5 on sm_103a)
 *   expand_runs        runs of 32 leaves each warp tests per chunk of the
 *                      level-ordered range-query expansion, 1..8 (default 4)
 *   visit_chunk        listed leaves laid out per chunk of a flattened point
 *                      visit, 64..512, a multiple of 64 (default 512)
 *   top_hull_min       super-hulls (runs of 32 x 32 leaves) a tree needs before
 *                      its pruned range query starts from the hulls of runs
 *                      of 32 super-hulls, >= 1 (default 1024: trees of about
 *                      a million leaves); not searched by detlsh_autotune
 *   hash_kb            shared memory (KiB) per query CTA for the hash of the
 *                      levels of listed leaves that the union counts, the
 *                      cut and the collection read; 0..160, 0 = the 16 KiB
 *                      projection-LUT region (up to 1,024 leaves; default).
 *                      When more leaves are listed the levels are read from
 *                      the CTA's device scratch instead.  A larger region
 *                      holds 2^b slots of 5 bytes (at most half of them
 *                      used) and leaves fewer CTAs resident per SM; the
 *                      launch takes no more CTAs than fit.
 *   query_scratch_mb   device memory (MiB) for the query CTAs' scratch slots
 *                      (one per concurrent query; a slot holds per-leaf
 *                      arrays of every tree, about 17 bytes per leaf);
 *                      0 = a quarter of the free device memory (default).
 *                      A set budget caps the slots in use.  Fewer slots
 *                      than CTAs limit the queries in flight.  The scratch
 *                      is kept between calls and never shrinks; it is
 *                      replaced by a larger one only for over a quarter
 *                      more slots, within 90% of the free memory plus what
 *                      it holds, and if that allocation fails the call
 *                      runs with the slots held before (or half of them)
 *                      instead of failing.  Not searched by detlsh_autotune.
 * detlsh_set_tuning / detlsh_get_tuning set and read an index's knobs (used
 * by detlsh_query, detlsh_query_ex, detlsh_query_candidates and batches
 * enqueued by detlsh_query_async after the change; detlsh_query_noalloc
 * keeps the defaults).  Errors: INVALID_ARG.
 *
 * detlsh_autotune chooses the knobs for this index on a sample of queries
 * (m x d FP32, host or device; m >= 1) with the query parameters qp and k:
 * starting from the defaults, each knob in turn takes the value with the
 * smallest query-kernel time (CUDA events on stream, best of two runs after
 * a warm-up run), the others held fixed.  The choice is stored in the index
 * and returned in *out (nullable).  With cache_path non-NULL, a text file
 * of one line per key "<key> <ctas_per_sm> <expand_runs> <visit_chunk>
 * <hash_kb> <ms>"
 * is read first: the key names the device and the shape (d, L, K, N_r, n
 * and beta*n + k to the nearest power of two, k, precision, r_min policy);
 * a match is taken without measuring (*from_cache = 1), otherwise the
 * search runs and appends its line.  Blocks until done.
 * Errors: as detlsh_query_ex, and IO when the cache file cannot be written.
 */
typedef struct {
    int32_t query_ctas_per_sm;
    int32_t expand_runs;
    int32_t visit_chunk;
    int32_t top_hull_min;
    int32_t hash_kb;
    int32_t query_scratch_mb;
} detlsh_tuning;
int detlsh_get_tuning(const detlsh_index *ix, detlsh_tuning *t);
int detlsh_set_tuning(detlsh_index *ix, const detlsh_tuning *t);
int detlsh_autotune(detlsh_index *ix, const float *queries, int64_t m, int32_t k,
                    const detlsh_query_params *qp, const char *cache_path, void *stream,
                    detlsh_tuning *out, int32_t *from_cache);

/* (r,c)-ANN query, Alg. 4 of the paper (Sec. V-B), over the range query of
 * Alg. 3 as printed (Sec. IV-C): for each tree in order, nodes whose lower
 * bound exceeds r' = eps*r are pruned, a leaf whose upper bound is within r'
 * gives all its points, and the points of any other reached leaf are tested
 * one by one on their projected distance (FP32, dimensions in order, squared
 * comparison against fp32(eps^2 r^2)).  S is the union over the trees so far;
 * once |S| >= beta*n + 1 the point of S nearest to q is returned (tree_stop =
 * that tree); after all L trees the nearest point of S is returned only if it
 * lies within c*r (FP32 distance), else ids = -1 and dists = +inf (tree_stop
 * = -1).  Nearest = smallest FP32 distance, ties by smaller id.
 *   ix        index built with keep_projections = 1 (the per-point test reads
 *             the stored projections); otherwise DETLSH_ERR_INVALID_ARG
 *   queries   m x d FP32, row-major, host or device
 *   r, beta, c  radius (> 0), false-positive budget (>= 0), ratio (> 1)
 *   ids, dists  m entries each, caller-owned, host or device
 *   tree_stop, S_size  m entries each, nullable
 *   S         m x S_cap ids of S in arrival order (nullable; S_cap >= 1 when
 *             given); entries past min(S_size, S_cap) are unspecified
 * Errors: INVALID_ARG (arguments as above), NONFINITE_INPUT (a query holds NaN
 * or Inf), OOM, CUDA.  Blocks until the results are written. */
int detlsh_rc_ann(const detlsh_index *ix, const float *queries, int64_t m, double r,
                  double beta, double c, int32_t optimised, void *stream, int64_t *ids,
                  float *dists, int32_t *tree_stop, int64_t S_cap, int64_t *S,
                  int64_t *S_size);

#ifdef __cplusplus
}
#endif

#endif /* DETLSH_H */
