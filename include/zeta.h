/*
 * zeta.h -- C ABI of the GB300 controlled-reduction library.
 *
 * Computes the zeta function of a smooth projective hypersurface
 * X = V(f) in P^n over F_p (7 <= p < 50) by controlled reduction in p-adic
 * cohomology (arXiv 2602.24155): (f, p, precision, policy) -> matrix of
 * p^{-1} sigma on H^n_dR(U) -> P(T) = det(1 - T F) in Z[T], with
 * Z(X, T) = P(T)^{(-1)^n} / prod_{i<n} (1 - p^i T)   (paper Sec. 2.1).
 *
 * The long linear recurrence w <- M(y) w mod p^M with M(y) = y A + B
 * (Sec. 3.2, Algorithm 2), driven by a reduction policy (Sec. 4), runs in
 * CUDA kernels for sm_103a; host code in this library prepares the start
 * vectors (Prop. 2.1, Algorithm 1) and finishes with the final
 * Griffiths-Dwork reduction (Sec. 3.3 step (2)) and the characteristic
 * polynomial.  There is no CPU fallback: every entry point that needs the
 * GPU returns ZETA_ERR_DEVICE when no CUDA device is usable.
 *
 * Conventions common to all entry points
 *  - No exceptions cross the ABI; every call returns a zeta_status.
 *  - The caller owns every buffer it passes; the library never frees them.
 *    The context owns its device memory and releases it in zeta_destroy.
 *  - Coefficients of f: C(n+d, n) values in [0, p), monomials of degree d in
 *    n+1 variables in descending lexicographic order of the exponent vector
 *    (x_0 first; for n = 2, d = 2: x0^2, x0x1, x0x2, x1^2, x1x2, x2^2).
 *  - The basis of H^n_dR(U) is the monomial basis of Sec. 2.3: for
 *    m = 1..n the monomials of degree dm-n-1 that are not pivot columns of
 *    the row echelon form over F_p of the image of the Jacobian map M_k
 *    (columns in the order above).  Basis order: m ascending, then monomial
 *    order.  b = dim = ((d-1)^{n+1} + (-1)^{n+1}(d-1)) / d.
 *  - Supported: controlled reduction (Prop. 3.3) with S = {0..n} when
 *    d >= n+1 and S = {n} otherwise (zeta_options.S_mask chooses another
 *    S); step matrices of side s = C(dn, n) <= 512; p^M < 2^60 (the device
 *    keeps residues as two 30-bit limbs, or as at most eight balanced
 *    base-256 digits on the tensor cores).  Other inputs return
 *    ZETA_ERR_UNSUPPORTED or ZETA_ERR_PRECISION.
 *  - Calls are synchronous: they return after the device work has finished.
 *    One context must not be used from two host threads at once.
 */
#ifndef ZETA_H
#define ZETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZETA_OK = 0,
    ZETA_ERR_ARG = 1,          /* null pointer, bad size, coefficient out of range */
    ZETA_ERR_NOT_SMOOTH = 2,   /* the Jacobian criterion fails (Sec. 2.1, Def. 3.1) */
    ZETA_ERR_UNSUPPORTED = 3,  /* p < 7, p >= 50, p | d, p <= n, or d < n+1 */
    ZETA_ERR_PRECISION = 4,    /* p^M would not fit below 2^60 */
    ZETA_ERR_DEVICE = 5,       /* CUDA error or no usable device */
    ZETA_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    ZETA_ERR_OOM = 7,          /* host or device allocation failed */
    ZETA_ERR_INTERNAL = 8      /* an internal consistency check failed */
} zeta_status;

/* Reduction policies (Sec. 4).  Every policy yields the same result. */
typedef enum {
    ZETA_POLICY_PCHUNK = 0,      /* Sec. 4.1: chunks of p on the terms of largest norm, then merge */
    ZETA_POLICY_DEPTH_FIRST = 1, /* Sec. 4.2: greedy v, largest chunk, never merge */
    ZETA_POLICY_VAR_BY_VAR = 2,  /* Sec. 4.3: clear u_n, merge, clear u_{n-1}, ... */
    ZETA_POLICY_LEARNED = 3,     /* p-chunk whose chunk directions are proposed by a trained network
                                    (zeta_options.policy_weights); Algorithm 3 if none is given */
    ZETA_POLICY_COVER = 4        /* p-chunk levels whose destinations are searched so that terms merge
                                    (a search over move 2 of the game of Sec. 3.4; not in the paper) */
} zeta_policy;

/* Which kernel runs the recurrence (every path gives the same result).
 * ZETA_PATH_GEMM: each step M(y) W of Algorithm 2 is an exact fp16 GEMM on
 * the tensor cores (tcgen05, fp32 accumulation in TMEM): residues become L
 * balanced base-256 digits (L = ceil((bits(q) + 2) / 8) <= 8), the rows of
 * M(k-1) and of A are interleaved in one 128-row operand, W's digits form a
 * Toeplitz operand, and a fused epilogue folds the 2L-1 digit diagonals back
 * to residues mod q.  It takes instances with s <= 64 and b <= 16 (plane
 * curves of degree <= 5); others return ZETA_ERR_UNSUPPORTED. */
typedef enum {
    ZETA_PATH_VECTOR = 0,  /* modular matrix-vector steps on the CUDA cores */
    ZETA_PATH_GEMM = 1,    /* exact limb-split modular GEMM steps on the tensor cores */
    ZETA_PATH_AUTO = 2     /* the choice zeta_autotune recorded in the context for the
                              batch's (n, d); ZETA_PATH_VECTOR with default blocks if none */
} zeta_path;

typedef struct {
    uint32_t n, d, p;           /* X in P^n of degree d over F_p */
    const uint32_t *coeffs;     /* host pointer, C(n+d, n) values in [0, p) */
} zeta_hypersurface;

typedef struct {
    zeta_policy policy;
    zeta_path path;
    /* Precision overrides (0 = the rules of Sec. 2.5 as read in the
     * library's documentation).  r_override sets the relative precision r;
     * N_override[m-1] sets the series order N_m.  With overrides smaller
     * than the rules the Frobenius matrix is a truncation and P(T) is not
     * the zeta function; used for small parity cases.  With r_override = r
     * alone, a_i is determined mod p^(r + H(i)), H the Hodge polygon (the
     * slopes n - m of the basis elements of pole order m in increasing
     * order), and mod at most the largest power of p below 2^63: what the
     * Newton height and the unit roots need (relative precision 1 for the
     * height of a cubic fourfold, the unit roots of a quintic surface). */
    uint32_t r_override;
    uint32_t N_override[8];
    uint32_t flags;             /* ZETA_FLAG_* bits */
    /* ZETA_POLICY_LEARNED: host pointer to the network's float weights
     * (layout of zeta_mlp_train) and its hidden width; NULL = Algorithm 3. */
    const float *policy_weights;
    uint32_t policy_hidden;
    /* ZETA_PATH_VECTOR: threads per block of the recurrence kernel (a
     * multiple of 32 in [64, 512]; 0 = the library's choice from s and b). */
    uint32_t block_threads;
    /* The index set S of Prop. 3.3 as a bit mask over x_0..x_n (bit i set =
     * i in S).  0 = automatic: S = {0..n} when d >= n + 1, else S = {n}.
     * f must be S-smooth (Definition 3.1: d_i f for i in S and x_i d_i f
     * for i not in S have no common zero; ZETA_ERR_NOT_SMOOTH otherwise)
     * and |S| <= d (ZETA_ERR_UNSUPPORTED); bits above x_n: ZETA_ERR_ARG.
     * P(T) does not depend on S.  ZETA_POLICY_LEARNED takes S = {0..n}
     * only (ZETA_ERR_UNSUPPORTED). */
    uint32_t S_mask;
} zeta_options;

/* Stop after the unnormalised columns Y (no division by p^(v-m+1), no
 * charpoly): for truncated precisions whose Y is not divisible. */
#define ZETA_FLAG_Y_ONLY 1u
/* Where the setup's right inverses over Z/q are solved (the section of
 * Prop. 3.3 and the final reduction's levels, Sec. 3.3 step (2); Gauss-Jordan
 * with unit pivots, the same matrices either way).  Neither flag: on the
 * device for batches holding an instance with C(dn, n) > 128, on the host
 * otherwise.  Batch calls only (zeta_batch_prepare, zeta_batch). */
#define ZETA_FLAG_HOST_SETUP 2u
#define ZETA_FLAG_DEVICE_SETUP 4u
/* Run every instance of a batch on the whole-GPU executor (one instance at
 * a time, every kernel over all SMs; step matrices in device memory), which
 * instances with C(dn, n) > 512 (cubic fourfolds: 3003) always take, after the
 * batch's persistent launch.  Needs q = p^M < 2^56 and C(dn, n) <= 4096. */
#define ZETA_FLAG_WHOLE_GPU 8u

typedef struct {
    int32_t status;          /* per-instance status (zeta_batch) */
    uint32_t b;              /* dim H^n_dR(U) = deg P */
    uint32_t r;              /* max_m r_m: relative precision of the Frobenius columns */
    uint32_t M;              /* algorithm precision: arithmetic mod p^M */
    uint32_t N[8];           /* series orders N_m, m = 1..n */
    uint32_t s;              /* side of the step matrices, C(dn, n) */
    int32_t eps;             /* sign of the functional equation */
    uint64_t chains;         /* distinct start exponents u after combining terms */
    uint64_t terms;          /* nonzero terms of the Frobenius expansion */
    uint64_t chunks;         /* chunks played (Sec. 3.4 move 1) */
    uint64_t steps;          /* reduction steps: sum of chunk lengths over chains */
    uint64_t column_steps;   /* steps times live columns: one length-s vector advanced one pole order */
    double ms_host_setup;    /* host: basis, section, expansion */
    double ms_device;        /* device: upload + recurrence + download */
    double ms_host_finish;   /* host: final reduction map, normalisation, charpoly */
    double ms_kernel;        /* device time of the recurrence kernel (CUDA events), summed over launches */
    uint64_t kernel_launches;/* launches of the recurrence kernel covered by ms_kernel */
    uint64_t bytes_h2d;      /* bytes copied host -> device (start terms, sections, tables) */
    uint64_t bytes_d2h;      /* bytes copied device -> host (numerators) */
    /* Device latency of the instance inside its persistent launch (batches;
     * per instance only): the times, in ms after the launch's first cluster
     * started, at which a cluster took the instance from the queue and at
     * which its numerators were written back; the instance's result is
     * complete on the device at ms_dev_end.  Recorded by the cluster executor,
     * which runs every batch holding an instance with s > 128 (all of the
     * batch's instances); batches of smaller instances report 0 for both.
     * Instances on the whole-GPU executor (C(dn, n) > 512 or more than 32
     * basis columns) report host-clock times after zeta_batch_run was called:
     * their run's start and its completion. */
    double ms_dev_start;
    double ms_dev_end;
} zeta_stats;

typedef struct zeta_ctx zeta_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL for the legacy default stream; may come from torch).  The
 * context allocates device memory lazily and keeps it for reuse. */
zeta_status zeta_create(zeta_ctx **out, int device, void *cuda_stream);

/* Release every device and host resource of the context.  NULL is allowed. */
zeta_status zeta_destroy(zeta_ctx *ctx);

/* Human-readable text of the last error of this context (never NULL). */
const char *zeta_last_error(const zeta_ctx *ctx);

/* Sizes of an instance without running it (host only, no device needed):
 * b = deg P, r, M (Sec. 2.5), s = C(dn, n).  Any output pointer may be NULL.
 * Returns ZETA_ERR_NOT_SMOOTH for a singular f. */
zeta_status zeta_query(const zeta_hypersurface *hs, const zeta_options *opt,
                       uint32_t *b, uint32_t *r, uint32_t *M, uint32_t *s);

/* Frobenius matrix of one hypersurface.
 *  F_out: caller-owned host buffer of b*b uint64, row-major: column j is
 *         p^{-1} sigma applied to basis element j, in the basis above.
 *         Column j (pole order m) is exact mod p^{r_m + n - m}; entries are
 *         reduced to [0, p^{r_m+n-m}).  r_m (Sec. 2.5) is the least relative
 *         precision of the pole-order-m columns for which every a_i,
 *         i <= b/2, is fixed: r_m = max(1, max_i e_i - G_m(i)) with e_i the
 *         least e with p^e > 2 C(b,i) p^{(n-1)i/2} and G_m(i) = (n - m) + the
 *         i-1 smallest slopes n - m' of the other basis elements.
 *  Y_out: optional (may be NULL) b*b uint64: the unnormalised columns
 *         ((p s_m - 1)! / (n-1)!) p^{1-m} sigma-coordinates mod p^M before
 *         the exact division (a library-independent quantity: it does not
 *         depend on the policy or the kernel path).
 *  st:    optional statistics. */
zeta_status zeta_frobenius(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt,
                           uint64_t *F_out, uint64_t *Y_out, zeta_stats *st);

/* P(T) = det(1 - T F) in Z[T] of one hypersurface (Sec. 2.1; coefficients
 * a_i for i <= b/2 from F, the rest from the functional equation
 * a_{b-i} = eps p^{(n-1)(b-2i)/2} a_i).
 * P_out: caller-owned 2*(b+1) int64: coefficient i is the 128-bit two's
 * complement integer with low word P_out[2i] (read as unsigned) and high
 * word P_out[2i+1]; a_0 = 1. */
zeta_status zeta_charpoly(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt,
                          int64_t *P_out, zeta_stats *st);

/* Many hypersurfaces (any mix of n, d, p; with opt->S_mask = 0 each takes its
 * own default S, so curves, surfaces and threefolds share a launch).  Batches
 * of 256 or more are split into two sub-batches (four from 512, eight from
 * 2048), heaviest
 * instances first (estimated from the precision alone), whose host setup
 * overlaps the device work of the previous one; consecutive sub-batches
 * alternate between the context's stream and a second stream of the context,
 * so that their persistent launches overlap.  Outputs are in input order.
 *  P_out: count * stride * 2 int64; instance i writes b_i+1 coefficients
 *         (two words each, as in zeta_charpoly) at P_out + 2*i*stride
 *         (stride >= max b_i + 1).
 *  per_instance: optional count zeta_stats; status of each instance in
 *         .status (the call returns ZETA_OK if the batch ran, even when some
 *         instances were rejected).
 *  total: optional aggregate statistics. */
zeta_status zeta_batch(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count,
                       const zeta_options *opt, int64_t *P_out, size_t stride,
                       zeta_stats *per_instance, zeta_stats *total);

/* The batch in phases, so that the device part can be timed on its own.
 *  zeta_batch_prepare: host setup of every instance (thread pool) and upload
 *      of the start terms, sections and tables to device memory.  The plan
 *      owns that device memory until zeta_batch_release.
 *  zeta_batch_run: enqueue the recurrence kernels on the context's stream
 *      and return without waiting (inputs already resident); instances on
 *      the whole-GPU executor (C(dn, n) > 512 or more than 32 basis columns)
 *      run to completion before it returns.  May be called again on the same
 *      plan; each run launches again and recomputes the same numerators.
 *  zeta_batch_finish: wait for the stream, read the numerators back, run
 *      the host finish; outputs as in zeta_batch.
 *  zeta_batch_release: free the plan (NULL allowed). */
typedef struct zeta_batch_plan zeta_batch_plan;
zeta_status zeta_batch_prepare(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                               zeta_batch_plan **out);
zeta_status zeta_batch_run(zeta_ctx *ctx, zeta_batch_plan *plan);
zeta_status zeta_batch_finish(zeta_ctx *ctx, zeta_batch_plan *plan, int64_t *P_out, size_t stride,
                              zeta_stats *per_instance, zeta_stats *total);
zeta_status zeta_batch_release(zeta_batch_plan *plan);

/* Autotuner of the batch engine (the paper has no counterpart: its kernels
 * are tuned by hand for one GPU).  Times candidate launch configurations of
 * the recurrence on a sample of the batch (at most `sample` instances, 0 =
 * 16 per SM, so that each candidate runs in its steady state rather than in
 * the tail of a short queue; taken with a constant stride so that the mix of
 * primes is kept):
 * ZETA_PATH_VECTOR with the default block and with 128, 256 and 384 threads
 * per block, and ZETA_PATH_GEMM where the instances allow it (s <= 64,
 * b <= 16).  Every candidate runs the same plans (opt's policy) once; the
 * time is that launch's CUDA-event time; every candidate's
 * P(T) must agree (ZETA_ERR_INTERNAL otherwise).  The fastest is recorded in
 * the context for the sample's (n, d) and used by ZETA_PATH_AUTO.  All
 * instances must share n and d (ZETA_ERR_ARG otherwise).  Host memory only
 * for inputs and `out`; synchronous. */
#define ZETA_TUNE_MAX 8
typedef struct {
    uint32_t n, d;                          /* the class the choice applies to */
    uint32_t sample;                        /* instances timed */
    uint32_t candidates;                    /* entries used below */
    uint32_t cand_path[ZETA_TUNE_MAX];      /* zeta_path of each candidate */
    uint32_t cand_threads[ZETA_TUNE_MAX];   /* block_threads of each candidate (0 = default) */
    double cand_ms[ZETA_TUNE_MAX];          /* mean kernel time per launch */
    uint32_t best;                          /* index of the fastest candidate */
} zeta_tuning;

zeta_status zeta_autotune(zeta_ctx *ctx, const zeta_hypersurface *hs, size_t count, const zeta_options *opt,
                          uint32_t sample, zeta_tuning *out);

/* Kernel-level entry point: Algorithm 2 on `count` independent problems
 * held in DEVICE memory (parity tests of the recurrence kernels).
 *  For problem t: W_t <- M(0) M(1) ... M(k_t - 1) W_t mod q_t with
 *  M(y) = y A_t + B_t; A_t, B_t are s x s row-major at A + t*s*s, B + t*s*s;
 *  W_t is s x c row-major at W + t*s*c (overwritten); k_t = k[t] >= 0;
 *  q_t = q[t] odd in [3, 2^60] with s < 8 q_t (ZETA_ERR_ARG otherwise).
 *  Entries must be reduced mod q_t.
 *  All pointers are device pointers; ZETA_ERR_ARG if s or c exceed the
 *  kernel limits (s <= 512, c <= 32; with ZETA_PATH_GEMM s <= 64, c <= 16).
 *  ZETA_ERR_TIMEOUT if a tensor-core step did not complete within 2 s (the
 *  kernel stops; the context stays usable). */
zeta_status zeta_horner_device(zeta_ctx *ctx, zeta_path path, uint32_t count, uint32_t s, uint32_t c,
                               const uint32_t *k, const uint64_t *A, const uint64_t *B,
                               uint64_t *W, const uint64_t *q);

/* Self-test of the bounded waits (the paper has no counterpart): one block on
 * the CURRENT device waits on a barrier that nothing arrives on, with the same
 * kind of deadline the tensor-core kernels use for their MMA waits, and gives
 * up after limit_ms (1..10000).  Returns ZETA_ERR_TIMEOUT when the wait ran out
 * (the expected outcome) and the time waited in *waited_ms (may be NULL); the
 * context stays usable.  No tensor core, TMEM or global memory beyond an
 * 16-byte status word is touched. */
zeta_status zeta_selftest_wait(zeta_ctx *ctx, uint32_t limit_ms, double *waited_ms);

/* Allocation-free form of zeta_horner_device, for callers that cannot
 * allocate device memory: code running inside another framework's memory
 * pool or a fixed memory budget, plugins that must not call cudaMalloc (or
 * any allocating library routine) after start-up, and code that enqueues
 * work while allocation is forbidden.  The paper has no counterpart; it
 * computes exactly what zeta_horner_device computes (the same block routine
 * for Algorithm 2), with the same arguments minus the context.
 *  - Runs on the CURRENT device, on `cuda_stream` (NULL: legacy default
 *    stream), and returns after the stream has drained.
 *  - Scratch: the step matrices of the problems in flight live in one
 *    file-scope device array of 16 MiB per device (2^21 uint64), which every
 *    GPU that loads the library holds until the process exits.  Limits:
 *    s <= 512, c <= 32, 2 s^2 <= 2^21 - 32 words (one problem's matrices),
 *    2 s c * 8 bytes of shared memory <= 227 KB.  Larger sizes return
 *    ZETA_ERR_ARG before anything is launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it when the lookup succeeds (a failed
 *    lookup is retried by the next call).  cudaDeviceReset on that device
 *    invalidates the cached address: do not call this entry point on a
 *    device after resetting it.
 *  - The call cannot be captured into a CUDA graph: it reads a status word
 *    back into host memory and synchronises the stream before returning.
 *  - Every call shares the array and it keeps the last call's contents; the
 *    matrices are fully written before they are read and the status word is
 *    cleared at the start of each call.  Calls that overlap on the GPU (two
 *    streams, two host threads) race on the array: serialise them.
 *  - Allocates nothing: no cudaMalloc, cudaFree, host heap, or library
 *    allocator.
 *  - Moduli are checked on the device (the host never reads q): a problem
 *    whose q_t is even, outside [3, 2^60], or has s >= 8 q_t is skipped (its
 *    W_t is left unchanged), the other problems are computed, and the call
 *    returns ZETA_ERR_ARG; the next call starts with a cleared status. */
zeta_status zeta_horner_static(void *cuda_stream, uint32_t count, uint32_t s, uint32_t c,
                               const uint32_t *k, const uint64_t *A, const uint64_t *B,
                               uint64_t *W, const uint64_t *q);

/* ---------------------------------------------------------------------------
 * Learned reduction policy (ZETA_POLICY_LEARNED).  The paper closes Sec. 4
 * noting that its policies never inspect U; this network proposes the
 * direction of every chunk of every p-chunk (Sec. 4.1), seeing how many other
 * terms reach each candidate's destination.  Any proposal gives the same
 * Frobenius matrix: only the cost of the reduction game (Sec. 3.4) changes.
 *
 * Network: a candidate (u, v) is a row of ZETA_POLICY_FEATURES floats; score =
 * w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3 with hidden width H (1..128).
 * Parameters, float, in this order: W1 (F x H, row-major), b1 (H), W2 (H x H),
 * b2 (H), w3 (H), b3 (1).  A decision is a group of consecutive rows; the loss
 * is the mean over groups of -log softmax(scores of the group)[label].
 * Buffers are host buffers owned by the caller.
 * ------------------------------------------------------------------------- */
#define ZETA_POLICY_FEATURES 18

/* Number of floats of the parameter vector for hidden width H. */
size_t zeta_mlp_param_count(uint32_t hidden);

/* Glorot-uniform initial weights from a seeded splitmix64 stream (host only). */
zeta_status zeta_mlp_init(uint32_t hidden, uint64_t seed, float *params);

/* Scores of n rows (GPU forward kernel). */
zeta_status zeta_mlp_forward(zeta_ctx *ctx, uint32_t hidden, const float *params, const float *X, size_t n,
                             float *scores);

/* Loss and its gradient with respect to every parameter over all groups
 * (GPU forward and backward kernels); group_off has ngroups+1 row offsets,
 * labels[g] indexes the chosen row of group g. */
zeta_status zeta_mlp_grad(zeta_ctx *ctx, uint32_t hidden, const float *params, const float *X,
                          const uint32_t *group_off, const uint32_t *labels, size_t ngroups, float *grad,
                          float *loss);

/* Adam on mini-batches of batch_groups consecutive groups for `epochs` passes;
 * params updated in place; final_loss (may be NULL) = mean batch loss of the
 * last epoch. */
zeta_status zeta_mlp_train(zeta_ctx *ctx, uint32_t hidden, float *params, const float *X,
                           const uint32_t *group_off, const uint32_t *labels, size_t ngroups, uint32_t epochs,
                           uint32_t batch_groups, float lr, float *final_loss);

/* Training decisions of one instance, generated by the game itself (host
 * only).  The cover game (ZETA_POLICY_COVER) is played with Algorithm 3 and its
 * chunk decisions with two or more legal directions are recorded; for a
 * sample of at most 128 of them, every legal direction is tried in a rollout
 * of the whole game (the same cover game, Algorithm 3 elsewhere) whose cost is
 * the plan's column steps plus 10 per chunk (the measured setup cost of a
 * chunk in column steps).  Each sampled decision is a group of candidate rows
 * (row 0: Algorithm 3's choice) labelled with the cheapest direction (ties to
 * row 0); costs[row] = the row's rollout cost minus the label's.  Two calls:
 * with NULL buffers to read ngroups and ncand, then with buffers of
 * ncand * ZETA_POLICY_FEATURES floats, ngroups+1 offsets, ngroups labels,
 * ncand costs (the calling thread keeps the last instance's result between
 * the two calls, so the rollouts run once).  ZETA_ERR_UNSUPPORTED unless
 * S = {0..n} and n <= 3. */
zeta_status zeta_policy_dataset(const zeta_hypersurface *hs, const zeta_options *opt, size_t *ngroups,
                                size_t *ncand, float *X, uint32_t *group_off, uint32_t *labels, int32_t *costs);

/* Scores of n rows computed on the host: the forward pass the scheduler runs
 * for ZETA_POLICY_LEARNED (the same network as zeta_mlp_forward; float
 * arithmetic in a fixed order).  The scheduler scores a few legal directions
 * per decision between other host work, where a device launch per decision
 * would cost more than the network (a few hundred multiply-adds).  hidden in
 * 1..512; host buffers. */
zeta_status zeta_mlp_forward_host(uint32_t hidden, const float *params, const float *X, size_t n, float *scores);

/* ---------------------------------------------------------------------------
 * Host-only entry points (no device needed): the setup and finishing steps
 * of the path, exposed so that they can be checked in isolation.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t b, s, nv;          /* basis size, C(dn, n), n + 1 */
    uint32_t sec_rows;          /* (n+1) * C(kappa-d+1+n, n): rows (i, nu), i major */
    uint32_t sec_cols;          /* C(kappa+n, n), kappa = (n+1)(d-1)+1-|S| ((n+1)(d-2)+1 for S = {0..n}) */
    uint32_t h_rows;            /* C(dn-1, n): monomials of degree dn-n-1 */
    uint32_t r, M;
    uint64_t q;                 /* p^M */
    uint64_t nchains, nterms;
    /* the reduction game played by opt->policy (Sec. 3.4) */
    uint64_t plan_chunks;       /* move 1 count */
    uint64_t plan_steps;        /* sum of chunk lengths */
    uint64_t plan_column_steps; /* steps times carried columns */
    uint64_t plan_merges;       /* move 2: duplicates combined */
    uint64_t plan_entries;      /* terms processed over all phases */
    uint64_t plan_cap;          /* largest number of merged terms waiting between two phases */
    uint32_t kappa;             /* degree of the section's columns */
    uint32_t S_mask;            /* the index set S used (bit i = i in S) */
} zeta_plan_info;

/* Host setup of one instance (Sec. 2.3-2.5, Prop. 2.1, Alg. 1, Prop. 3.3)
 * and the reduction game of opt->policy (Sec. 3.4, Sec. 4), statistics in info:
 *  sec:        sec_rows x sec_cols uint64 (row-major) -- the section of the
 *              map of J_S in degree kappa over Z/q: column gamma holds G_0..G_n
 *              with sum_i G_i d_i f = x^gamma, G_i a multiple of x_i for i not
 *              in S (rows (i, nu), nu in Homog_{kappa-d+1}; rows (i, nu) with
 *              i not in S and nu_i = 0 are zero).  For S = {0..n}: the section
 *              of M_kappa, nu in Homog_{n(d-2)}.
 *  chain_U:    nchains x nv int32 -- start exponents U (Tweak of
 *              p(beta+alpha+1) - 1 + 1_S), distinct, longest first.
 *  chain_terms:nchains x 2 uint32 -- [begin, end) ranges into the term arrays.
 *  term_rc:    nterms x 2 uint32 -- (row = index of J in Homog_{dn-n}, basis column).
 *  term_coeff: nterms uint64 -- (D_{j,m} C_{j,alpha} mod p^{s_m}) (p s_m - 1)!/(p(m+j) - 1)! mod q.
 *  fin:        b x h_rows uint64 -- the final reduction map (Sec. 3.3 step (2))
 *              from pole-order-n numerators to basis coordinates, mod q.
 * Every buffer may be NULL (then it is not written); call once with NULLs
 * to read the sizes from info. */
zeta_status zeta_plan(const zeta_hypersurface *hs, const zeta_options *opt, zeta_plan_info *info,
                      uint64_t *sec, int32_t *chain_U, uint32_t *chain_terms, uint32_t *term_rc,
                      uint64_t *term_coeff, uint64_t *fin);

/* zeta_plan's sec and fin with the setup's right inverses solved on the
 * device (k_right_inverse: one block per matrix, [A | I] in device memory,
 * Gauss-Jordan over Z/q with unit pivots in column order, the first unit row
 * as pivot; Prop. 3.3 proof, Sec. 3.3 step (2)) and the rest of the setup on
 * the host.  Equal to zeta_plan's word for word: exact arithmetic with the
 * same pivot rule.  sec, fin: host buffers sized as zeta_plan's (either may
 * be NULL); ms_device: the solve kernel's time (CUDA events), may be NULL.
 * ZETA_ERR_UNSUPPORTED when a matrix's C + R words exceed a block's shared
 * memory (about 29 000). */
zeta_status zeta_plan_device(zeta_ctx *ctx, const zeta_hypersurface *hs, const zeta_options *opt, uint64_t *sec,
                             uint64_t *fin, double *ms_device);

/* The index tables the device's step-matrix generation reads for one
 * instance (host only).  The kernel forms, for output row r and input
 * column j of Homog_{dn-n} (monomials omega_r, mu_j),
 *   R_{u,v}[r, j] = sum_i (u_i + e_{r,i}) Sec[secrow[i s + r], rank_kappa(v + e_j - 1)]
 * with e_j = monoS[j] = mu_j + 1 - 1_S, which is Prop. 3.3's
 * x^S sum_i (u_i G_i / x_i + d_i G_i) on monomials for any S; and it adds
 * the pole-order-n numerators at rank_{dn-n-1}(U + e_j - 1).
 *  monoS:  s x nv int32 (the shifted exponents e_j).
 *  secrow: nv x s int32, secrow[i s + r] = row (i, omega_r - 1_S + e_i) of
 *          sec, or -1 where that exponent has a negative entry.
 * Either buffer may be NULL. */
zeta_status zeta_plan_tables(const zeta_hypersurface *hs, const zeta_options *opt, int32_t *monoS,
                             int32_t *secrow);

/* The moves of the plan the host scheduled for one instance (host only, no
 * device): the device executes exactly these.  Two calls: with NULL buffers
 * it returns the counts, then fills caller-owned buffers.
 *  phase_begin: nphases + 1 uint32, entries of phase f are [phase_begin[f],
 *    phase_begin[f+1]).
 *  entries: nentries x (nv + 7) int32: U[nv], chunk_begin, chunk_end (into
 *    chunks), arrival (block of the previous phase whose sum starts W, or -1),
 *    start_chain (chain of zeta_plan whose terms are added, or -1), dest
 *    (block of the next phase the result is added to; -1 = pole order n,
 *    accumulated into the numerators), flags (bit 0: first contribution to its
 *    block: store instead of add), live (bit mask of the columns it carries).
 *  chunks: nchunks x (nv + 1) int32: v[nv], k.
 * Every plan passes the library's move check before it is returned. */
zeta_status zeta_plan_moves(const zeta_hypersurface *hs, const zeta_options *opt, size_t *nphases, size_t *nentries,
                            size_t *nchunks, uint32_t *phase_begin, int32_t *entries, int32_t *chunks);

/* Host finishing steps from accumulated pole-order-n numerators:
 *  H: h_rows x b uint64 mod q -- column j holds the sum over all reduced
 *     terms of column j of the numerators x^U g / x^S (degree dn-n-1).
 *  Outputs as in zeta_frobenius / zeta_charpoly; any may be NULL. */
zeta_status zeta_finish(const zeta_hypersurface *hs, const zeta_options *opt, const uint64_t *H,
                        uint64_t *F_out, uint64_t *Y_out, int64_t *P_out);

#ifdef __cplusplus
}
#endif
#endif /* ZETA_H */
