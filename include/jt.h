/*
 * jt.h -- C ABI of libjt, a GB300 (sm_103a) library that applies the fast
 * discrete Jacobi polynomial transform of Bremer, Pang and Yang, "Fast
 * Algorithms for the Multi-dimensional Jacobi Polynomial Transform"
 * (arXiv:1901.07275).
 *
 * Operators (per axis i, n_i points = n_i degrees, parameters a_i, b_i in (-1,1)):
 *   uniform (Gauss--Jacobi nodes, Sec. 3.1 Eq. tf:transout):  A_i = W_i J_i,
 *     (W_i J_i)[k][j] = sqrt(w_k) P~_j(t_k); A_i is orthogonal;
 *   nonuniform (caller's angles t_k in (0,pi), Sec. 3.1 last paragraph): A_i = J_i,
 *     J_i[k][j] = P~_j(t_k), with P~_j the modified Jacobi function of Eq.
 *     eq:modifiedjac and degrees j = 0..n_i-1.
 *   jt_forward :  f     = (A_0 (x) A_1 (x) ... ) alpha      (Eqs. eq:oneJ, eq:TJ, eq:TJ3)
 *   jt_adjoint :  alpha = (A_0 (x) A_1 (x) ... )^T g        (Eqs. eq:oneJinv, eq:invTJ, eq:invTJ3)
 *   jt_inverse :  the inverse of jt_forward; equals jt_adjoint for uniform axes
 *                 (A_i orthogonal, Sec. 3.1); JT_ENOTSUP if any axis is nonuniform
 *                 (the paper leaves that inverse open, Sec. 5).
 *
 * Each axis is applied as   A x = W V x_V + W Re( sum_k D_{u_k} F D_{v_k} x_G )   (Eq. eq:oneJ):
 * V is the dense block of degrees < nu0 (27), F the row-gathered unnormalised
 * inverse DFT of length L (Eqs. eq:lastJ, eq:permuDFT), u_k, v_k the rank-r factors
 * of the matrix B (Eqs. eq:B, eq:approxA) built at plan creation by the randomised
 * SVD of Algorithm 2.1.  d-dimensional transforms sweep the axes one at a time.
 *
 * Layout: arrays are row-major over (nrhs, n_0, ..., n_{d-1}); the last axis is
 * contiguous and the right-hand-side index is slowest.  JT_FP32 plans take and
 * return float32; JT_SPLIT and JT_FP64_PLAIN plans take and return float64.
 *
 * Memory: alpha, f and g are DEVICE pointers owned by the caller; calls are
 * asynchronous on the given stream (NULL = legacy default stream) and never
 * synchronise.  The plan owns its device tables; all entry points are
 * thread-safe for distinct plans, and a plan is read-only after creation, so
 * concurrent calls on one plan on different streams are safe as long as their
 * output buffers do not overlap -- except for plans that own work buffers, whose
 * calls must be serialised (one stream, or ordered by the caller): JT_FP64_PLAIN
 * plans, and JT_SPLIT plans with an axis longer than 8192 (partial sums of the
 * half-length sweeps).  Such a plan may appear only once in a batch (JT_EINVAL).
 * Input and output may be the same buffer (in-place transform).  No C++ exception
 * crosses this interface.
 */
#ifndef JT_H
#define JT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* jt_stream_t; /* same type as cudaStream_t */

typedef enum {
    JT_OK = 0,
    JT_EINVAL = 1,   /* invalid argument (sizes, parameters outside (-1,1), points outside (0,pi), ...) */
    JT_ENOMEM = 2,   /* host or device allocation failed */
    JT_ENOTSUP = 3,  /* operation not defined for this plan (nonuniform inverse, ...) */
    JT_ECUDA = 4,    /* a CUDA runtime or library call failed */
    JT_ETIMEOUT = 5, /* a bounded device wait expired (jt_plan_check) */
    JT_ENOCONV = 6   /* setup did not converge: rank needed for eps exceeds rank_cap, nodes not found */
} jt_status;

typedef enum {
    JT_FP32 = 0,       /* fused FP32 axis kernels; float32 in/out */
    JT_SPLIT = 1,      /* fused kernels in double-word (hi+lo FP32) arithmetic; float64 in/out */
    JT_FP64_PLAIN = 2  /* unfused FP64 comparison path: the r^d d-dim FFT form (abstract,
                          Sec. 5) with cuFFT Z2Z; float64 in/out */
} jt_precision;

typedef struct {
    int32_t prec;           /* jt_precision */
    int32_t nu0;            /* split degree of Eq. tf:jn, 0..32; default 27 */
    int32_t rank_cap;       /* largest rank allowed per axis; 0 => max(ceil(2 log2 n), 64) */
    int32_t oversample_q;   /* oversampling factor q of Algorithm 2.1; default 3 */
    uint64_t seed;          /* seed of the row/column sampling in Algorithm 2.1 */
    int32_t fft_len_policy; /* 0: L = n if n is a power of two, else the next power of two */
    int32_t autotune;       /* 0: rank splits by the occupancy rule (see jt_plan_set_ksplit);
                               1: jt_batch_create measures them for every member sweep
                               (as jt_plan_tune does) before building the batch */
    int32_t kind;           /* JT_FIRST_KIND (default) or JT_SECOND_KIND */
    int32_t setup_device;   /* 0 (default): the whole setup on the host; 1: the Newton iteration
                               for the nodes, the sampled columns of B (the O(n^2) steps) and
                               the column-pivoted QRs of Algorithm 2.1 in FP64 kernels on the
                               current GPU, the rest on the host.  Same algorithm; tables agree
                               with the host's to rounding. */
} jt_options;

/* Which modified Jacobi functions the transform expands in (Sec. 1, Eqs. eq:jacnonosci,
 * eq:jacnonosci2; the paper notes the transform for Q~ is similar, Sec. 3.1--3.3):
 *   JT_FIRST_KIND   P~_j = M cos(psi)  (the matrix J of every entry point above);
 *   JT_SECOND_KIND  Q~_j = M sin(psi) = -(2/pi) C_j Q_j(cos t) sin(t/2)^{a+1/2} cos(t/2)^{b+1/2},
 *                   Q_j the Jacobi function of the second kind on the cut (Szego 4.62), i.e. the
 *                   imaginary part of the same B o F (Eq. eq:B): A_i = W_i Jq_i (Gauss--Jacobi
 *                   nodes, same weights) or Jq_i (caller's angles).  Forward and adjoint only:
 *                   Jq is not orthogonal, so jt_inverse returns JT_ENOTSUP; JT_FP64_PLAIN
 *                   plans of the second kind are JT_ENOTSUP. */
typedef enum { JT_FIRST_KIND = 0, JT_SECOND_KIND = 1 } jt_kind;

/* Fill *opt with the defaults listed above. */
void jt_options_default(jt_options* opt);

typedef struct jt_plan jt_plan;

/*
 * Create a plan for a d-dimensional transform (d in {1,2,3}).
 *   n[i]      number of points (= number of degrees) on axis i, 1 <= n[i] <= 16384
 *             (<= 8192 for JT_SPLIT)
 *   a[i],b[i] Jacobi parameters, each in (-1, 1) (the method does not apply outside, Sec. 5)
 *   points    NULL, or an array of d host pointers; points[i] == NULL selects the n[i]
 *             Gauss--Jacobi nodes of axis i (uniform); otherwise points[i] holds n[i]
 *             host float64 angles t in (0, pi) (nonuniform axis, W_i = I).
 *   eps       relative accuracy of the low-rank factorisation, in (0, 1): singular values
 *             below eps * sigma_1 are dropped (Sec. 2.1, rank-adaptive wrapper).
 *   opt       NULL for defaults.
 *   stream    stream for the table uploads; the call synchronises it before returning.
 * Setup (nodes, phase data, factorisation) runs on the host in FP64; tables are then
 * uploaded once.  Errors: JT_EINVAL, JT_ENOMEM, JT_ENOCONV, JT_ECUDA; *out is NULL on error.
 */
jt_status jt_plan_create(jt_plan** out, int d, const int64_t* n, const double* a, const double* b,
                         const double* const* points, double eps, const jt_options* opt,
                         jt_stream_t stream);

/* Forward transform of nrhs >= 1 right-hand sides: f = (A_0 (x) ... ) alpha.  alpha and f
 * hold nrhs * prod(n) elements of the plan's I/O type and may alias exactly. */
jt_status jt_forward(jt_plan* plan, const void* alpha, void* f, int64_t nrhs, jt_stream_t stream);

/* Adjoint (transpose): alpha = (A_0 (x) ... )^T g.  Same layout rules as jt_forward. */
jt_status jt_adjoint(jt_plan* plan, const void* g, void* alpha, int64_t nrhs, jt_stream_t stream);

/* Inverse of jt_forward: equal to jt_adjoint when every axis is uniform; JT_ENOTSUP otherwise. */
jt_status jt_inverse(jt_plan* plan, const void* g, void* alpha, int64_t nrhs, jt_stream_t stream);

/*
 * Forward transform of a JT_FP64_PLAIN plan that allocates nothing (the paper has no
 * counterpart; this is a library convenience).  The plain FP64 path needs work buffers
 * beyond its input and output; jt_forward takes them from the plan, this call takes them
 * from one fixed 16 MiB device array compiled into libjt.  It is meant for callers that must
 * not request device memory at call time: a serving loop that cannot risk an allocation
 * failure or the allocator's locks in the middle of a request, or a process whose free device
 * memory is already reserved by another allocator (a framework's caching allocator, for
 * instance).
 *   Same arguments, layout and result as jt_forward (float64 in and out, device pointers).
 *   JT_ENOTSUP for plans of another precision; JT_EINVAL for bad arguments (the element
 *   limit of jt_forward included) or when the plan needs more work space than the array
 *   holds.  With L_a the FFT length of axis a (jt_plan_info: n_a rounded up to a power of
 *   two) and N = prod_a n_a, the plan needs
 *       R(16 prod_a L_a) + R(16 max_a (N / n_a) L_a) + 2 R(8 N)  <=  16 MiB,
 *   R(x) = x rounded up to a multiple of 256 bytes.  512 x 512 fits (12 MiB); 513 x 513 and
 *   1024 x 1024 do not.  No cudaMalloc, cudaFree or allocating library call is made.
 *   The array's device address is looked up when the plan is created, on the plan's device;
 *   that lookup also loads the module, so the device commits the 16 MiB when its first
 *   JT_FP64_PLAIN plan is created (not inside this call) and holds them until exit.
 *   Every call shares the one array, which keeps the last call's contents (each call clears
 *   what it needs at zero itself): calls that overlap on the GPU -- on different streams, or
 *   from different host threads -- race on it and must be serialised by the caller.
 */
jt_status jt_forward_plain_noalloc(jt_plan* plan, const void* alpha, void* f, int64_t nrhs,
                                   jt_stream_t stream);

/*
 * Plan inspection.  For axis in [0, d): *rank = number of rank terms r, *fft_len = L.
 * t_out / w_out (each NULL or n[axis] host float64): the points and the trigonometric
 * Gauss--Jacobi weights w_k (1 for a nonuniform axis).  JT_EINVAL on a bad axis.
 */
jt_status jt_plan_info(const jt_plan* plan, int axis, int* rank, int64_t* fft_len, double* t_out,
                       double* w_out);

/* Transform nrhs right-hand sides held in HOST memory: they pass through the caller's device
 * work area dev_buf (dev_bytes bytes, at least one right-hand side) in chunks of right-hand
 * sides, up to three chunks in flight on three streams the plan owns (forked from and joined
 * back to `stream`), so that the copy to the device of one chunk, the transform of another and
 * the copy back of a third overlap.  direction: 0 forward, 1 adjoint, 2 inverse (the rules of
 * jt_forward, jt_adjoint, jt_inverse).  in_host and out_host hold nrhs * prod(n) elements of
 * the plan's I/O type; page-locked host memory is needed for the copies to overlap.  The call
 * is asynchronous on `stream`: the host arrays must stay valid, and dev_buf untouched, until
 * the stream reaches this point.  Results equal jt_forward / jt_adjoint / jt_inverse on each
 * chunk (each chunk gets the schedule of its own size).  JT_ENOTSUP for JT_FP64_PLAIN plans. */
jt_status jt_transform_host(jt_plan* plan, int direction, const void* in_host, void* out_host, int64_t nrhs,
                            void* dev_buf, size_t dev_bytes, jt_stream_t stream);

/* Dimensions and options of a plan (any output pointer may be NULL): the number of axes,
 * n[0..d-1] (n[d..2] set to 1), the precision, the kind, and whether every axis uses the
 * Gauss--Jacobi nodes (so that jt_inverse is defined for the first kind). */
jt_status jt_plan_shape(const jt_plan* plan, int* d, int64_t* n, int* prec, int* kind, int* all_uniform);

/* Failure detection (no counterpart in the paper).  The FP32 forward sweeps of length up to
 * 512 (not batched, no rank split) wait on bulk copies of their rank tables; every such wait
 * is bounded (about one second), and a
 * kernel whose wait runs out sets a status word of the plan and returns early, leaving its
 * output incomplete instead of hanging.  jt_plan_check synchronises `stream`, then returns
 * JT_ETIMEOUT (and clears the words) if any wait of this plan ran out since the last check,
 * else JT_OK.  JT_EINVAL for a NULL plan, JT_ECUDA if the stream reports an error. */
jt_status jt_plan_check(jt_plan* plan, jt_stream_t stream);

/* Testing hook: with on != 0 the plan's FP32 forward sweeps that stream their tables issue no copy,
 * so their first wait runs out (after about one second) and jt_plan_check reports
 * JT_ETIMEOUT.  on = 0 restores normal operation.  JT_ENOTSUP for other precisions. */
jt_status jt_plan_inject_wait_timeout(jt_plan* plan, int on);

/* Release a plan and its device tables.  NULL is accepted. */
void jt_destroy(jt_plan* plan);

/* ------------------------------------------------------------------------------------
 * Serving helpers (no counterpart in the paper, whose setup runs once per experiment):
 * setting up many plans at once, and saving / loading the result of a plan's setup.
 * ------------------------------------------------------------------------------------ */

/* The arguments of one jt_plan_create call. */
typedef struct {
    int32_t d;
    int64_t n[3];
    double a[3], b[3];
    const double* points[3]; /* per axis as in jt_plan_create (all NULL: Gauss--Jacobi nodes) */
    double eps;
    const jt_options* opt;   /* NULL for defaults */
} jt_plan_desc;

/* Create `count` plans: the host setups run side by side on the host cores, then the tables
 * are uploaded on `stream` (synchronised).  On success out[i] is the plan of descs[i]; on any
 * error every out[i] is NULL, nothing is leaked and the first failing status is returned. */
jt_status jt_plan_create_many(int count, jt_plan** out, const jt_plan_desc* descs, jt_stream_t stream);

/* Serialise the setup of a plan (nodes, weights, bins, factors, dense block: every table
 * jt_plan_create computed, in FP64) into buf, a byte array that jt_plan_load accepts on any
 * little-endian host.  Schedules (jt_plan_set_ksplit / jt_plan_tune) are not saved: they
 * belong to the GPU that measured them.  With buf NULL, *size receives the bytes needed and
 * the call returns JT_OK; with *size too small, *size receives the bytes needed and the call
 * returns JT_EINVAL; otherwise the plan is written and *size set to its length.  The plan is
 * only read. */
jt_status jt_plan_save(const jt_plan* plan, void* buf, size_t* size);

/* Recreate a plan from jt_plan_save bytes without any setup work: the buffer is checked
 * (magic, version, checksum, every size and range; JT_EINVAL before any GPU call if it does
 * not pass), then the tables are uploaded on `stream` (synchronised).  The loaded plan
 * computes bit for bit what the saved one did. */
jt_status jt_plan_load(jt_plan** out, const void* buf, size_t size, jt_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Schedules (no counterpart in the paper, which applies the rank terms one after another
 * on one processor): the rank split of an axis sweep is the number of CTAs (a thread-block
 * cluster, 1, 2, 4 or 8) that share a tile of fibres, each applying a contiguous share of
 * the r rank terms of Eq. eq:oneJ / eq:oneJinv; the partial sums are added in distributed
 * shared memory in a fixed order, so a given split gives reproducible results (different
 * splits agree to rounding).  Splitting shortens the critical path of sweeps with few
 * fibres (large n, few right-hand sides) that cannot fill the GPU otherwise.
 * Order of precedence for a sweep of F fibres: a split measured by jt_plan_tune for F
 * fibres, then one fixed by jt_plan_set_ksplit, then the occupancy rule (double the split,
 * up to 8, while the split tiles fit in one wave and every CTA keeps a rank term).
 * These calls change the plan: do not make them while other calls use the plan.
 * JT_FP64_PLAIN plans have no schedule: JT_ENOTSUP.
 * ------------------------------------------------------------------------------------ */

/* Fix the rank split of axis `axis` (-1: every axis) for `direction` 0 = forward,
 * 1 = adjoint/inverse, -1 = both.  ksplit in {0 (occupancy rule), 1, 2, 4, 8}, else
 * JT_EINVAL.  Drops measured splits of the same axes and directions. */
jt_status jt_plan_set_ksplit(jt_plan* plan, int axis, int direction, int ksplit);

/* Measure, for nrhs right-hand sides, every split in {1, 2, 4, 8} (at most the rank) of
 * every axis sweep in both directions and keep the fastest.  Allocates and frees two
 * scratch arrays of nrhs * prod(n) elements, launches the sweeps on `stream` and
 * synchronises it.  JT_EINVAL if the stream is being captured into a graph. */
jt_status jt_plan_tune(jt_plan* plan, int64_t nrhs, jt_stream_t stream);

/* The rank split the sweep of axis `axis` gets in `direction` (0 forward, 1 adjoint) for
 * nrhs right-hand sides (the launchers may fall back to a smaller cluster if one of that
 * size cannot be resident). */
jt_status jt_plan_schedule(const jt_plan* plan, int axis, int direction, int64_t nrhs, int* ksplit);

/* ------------------------------------------------------------------------------------
 * Batches: many transforms of one precision (JT_FP32 or JT_SPLIT), each with its own plan
 * (any d, n, a, b, points) and number of right-hand sides, executed together.  The axis
 * sweeps are grouped by stage (the s-th sweep of every transform, Sec. 3.2-3.3) and, within
 * a stage, by FFT length, stride kind and rank split; FP32 sweeps of length 16..4096 of one
 * group run as a single kernel launch over all their fibres, other sweeps one launch each.
 * ------------------------------------------------------------------------------------ */
typedef struct jt_batch jt_batch;

/* Build the schedule of a batch of `count` plans (not owned; they must outlive the batch)
 * with nrhs[i] >= 1 right-hand sides each; uploads the job tables on `stream` and
 * synchronises it.  Each member sweep keeps its plan's rank split for that many fibres
 * (see jt_plan_schedule; measured first for plans created with autotune = 1); sweeps with
 * different splits go to different launches.  The launches of one stage are spread over
 * four worker streams that the batch owns, forked from and joined back to the caller's
 * stream on every execution.  JT_EINVAL for mixed precisions, bad arguments, or a JT_SPLIT
 * plan with an axis longer than 8192 listed twice; JT_ENOTSUP for JT_FP64_PLAIN plans. */
jt_status jt_batch_create(jt_batch** out, int count, jt_plan* const* plans, const int64_t* nrhs,
                          jt_stream_t stream);

/* Forward / adjoint transform of every member: in[i], out[i] are device arrays of member i
 * (layout and aliasing rules of jt_forward).  Host arrays `in`, `out` hold count pointers.
 * Only kernel launches are issued (no allocation, copy or synchronisation). */
jt_status jt_batch_forward(jt_batch* batch, const void* const* in, void* const* out, jt_stream_t stream);
jt_status jt_batch_adjoint(jt_batch* batch, const void* const* in, void* const* out, jt_stream_t stream);

/* Release a batch (not its plans).  NULL is accepted. */
void jt_batch_destroy(jt_batch* batch);

/* Static string naming a status code. */
const char* jt_status_string(jt_status s);

/* Measurement helper (no counterpart in the paper): the FP32 arithmetic rate that bounds the
 * axis kernels, measured instead of derived from unit counts.  Launches, on `stream`, a
 * persistent grid of 4 CTAs of 256 threads per SM in which every thread runs 8 independent
 * chains of 16 * iters fused multiply-adds: fma.rn.f32 (paired = 0) or fma.rn.f32x2, two FMAs
 * an instruction (paired = 1).  The caller times the launch (events on `stream`).
 *   sink: device float32 array of at least sink_len >= 1024 * SM-count elements (written);
 *   *flops (host): the launch's floating-point operations, 2 per FMA.
 *   JT_EINVAL for iters < 1, a NULL pointer or a short sink; JT_ECUDA on a launch error. */
jt_status jt_probe_fp32_fma(int paired, int64_t iters, float* sink, int64_t sink_len, double* flops,
                            jt_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Host-side setup of one axis, for inspection and testing of the plan tables.  Runs the
 * same code as jt_plan_create for one axis and touches no GPU.
 *   B-matrix factors (Eqs. eq:B, eq:approxA): the plan stores the row-scaled matrix
 *   W B (W = diag(sqrt(w_k)) for a uniform axis, I otherwise) as sum_k u_k v_k^T with
 *   u_k of length n and v_k of length n - nu0 (plain transpose, not conjugate).
 * ------------------------------------------------------------------------------------ */
typedef struct jt_axis_tables jt_axis_tables;

jt_status jt_axis_tables_create(jt_axis_tables** out, int64_t n, double a, double b,
                                const double* points, double eps, const jt_options* opt);

/* Sizes: rank r, FFT length L, effective nu0 (= min(nu0, n)), and the sampled relative
 * Frobenius error of sum_k u_k v_k^T against W B (any of the pointers may be NULL). */
jt_status jt_axis_tables_info(const jt_axis_tables* t, int* rank, int64_t* fft_len, int* nu0,
                              double* fact_err);

/* Copy the tables to caller-owned host buffers (any may be NULL):
 *   t[n] angles, w[n] trigonometric weights (1 if nonuniform), m[n] FFT bins round(t L / 2 pi),
 *   u[2*r*n] interleaved (re,im) row-major r x n, v[2*r*(n-nu0)] interleaved r x (n-nu0),
 *   vblk[n*nu0] row-major n x nu0 with vblk[k][c] = sqrt(w_k) P~_c(t_k). */
jt_status jt_axis_tables_copy(const jt_axis_tables* t, double* tt, double* w, int32_t* m, double* u,
                              double* v, double* vblk);

/* Evaluate rows of the row-scaled matrix W B exactly (by recurrence), for testing:
 * out[2*(i*(n-nu0)+c)+{0,1}] = (W B)[rows[i]][c]. */
jt_status jt_axis_tables_b_rows(const jt_axis_tables* t, const int64_t* rows, int64_t nrows,
                                double* out);

void jt_axis_tables_destroy(jt_axis_tables* t);

#ifdef __cplusplus
}
#endif

#endif /* JT_H */
