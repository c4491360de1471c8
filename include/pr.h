/*
 * pr.h -- C ABI of the GB300 (sm_103a) IFP1 / IFP2 PageRank library.
 *
 * Method: "Two Parallel PageRank Algorithms via Improving Forward Push"
 * (Zhang, Tang, Yao, Liang; arXiv 2302.03245).  PageRank / personalized
 * PageRank pi solves (I - cP')pi = (1-c)p with P' = P + p d^T (Sec. 2.1,
 * Eq. 1-2).  IFP1 (Alg. 2) and IFP2 (Alg. 3) push residual mass along the
 * out-edges of non-dangling vertices only and normalise the kept mass
 * (Sec. 3.1, Eq. 4); the Power method on P'' (Sec. 4, "SPI") is the baseline.
 *
 * Conventions for every call:
 *  - Every function returns a pr_status; nothing throws across the ABI.  On
 *    any status other than PR_OK, pr_last_error() gives a message (per
 *    calling thread).
 *  - Vertex ids are int32 in [0, n); edge offsets are int32 (m < 2^31 per
 *    graph).  Arrays are plain pointers; "device" means a CUDA device pointer
 *    on the current device, "host" ordinary (pageable or pinned) memory.
 *  - The library owns the device memory it allocates (through the allocator
 *    installed with pr_set_allocator, else cudaMalloc) and never keeps a
 *    pointer to caller memory after a call returns.
 *  - A pr_graph and everything solved on it run on the CUDA stream given at
 *    creation.  One graph must not be used by two host threads at once.
 */
#ifndef PR_H
#define PR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph;   /* opaque: device copy of a graph + solver workspace */
typedef struct pr_server pr_server; /* opaque: continuous-batching request loop */

typedef enum {
    PR_OK = 0,
    PR_EINVAL = 1,   /* invalid argument (message names it) */
    PR_ENOMEM = 2,   /* device or host allocation failed */
    PR_ECUDA = 3,    /* a CUDA call failed (message has the CUDA error) */
    PR_ENOTCONV = 4, /* round/iteration cap reached, or no vertex could be activated;
                        `out` still holds the best-effort result */
    PR_ETIMEOUT = 5, /* a bounded device-side wait ran out (reserved: no kernel of this
                        library waits on another block, rank or flag) */
    PR_EAGAIN = 6,   /* server: over the HBM budget and the queue is full */
    PR_EBUSY = 7,    /* server: request not finished yet */
    PR_ECHECK = 8    /* debug build only: an index or invariant check failed (see
                        pr_debug_report_get); the accesses it guards were skipped */
} pr_status;

typedef enum {
    PR_POWER = 0, /* Power method on P'' (Sec. 4, SPI) -- the baseline */
    PR_IFP1 = 1,  /* Alg. 2 (Sec. 3.2) */
    PR_IFP2 = 2   /* Alg. 3 (Sec. 3.4): no pushes into dangling vertices in phase 1,
                     one pull into each dangling vertex in phase 2 */
} pr_algo;

typedef enum {
    PR_FP64 = 0, /* IEEE double throughout, the paper's arithmetic (Sec. 4 computes
                    in double): residual, reserve, the pushed mass a gather reads
                    per source (pending pushes, Power's pi/deg), the gathered
                    sums, the reductions and the output.  On GB300 the FP64 pipe
                    runs at 1/64 of FP32 */
    PR_FP32 = 1, /* residual, reserve and pushed mass in float; the residual-L1
                    and dangling-mass sums in IEEE double; at the end a
                    correction sweep recomputes the residual from the reserve in
                    IEEE double (r = p + c P~ s - s, s = x/(1-c), from Eq. 4; not
                    in the paper), and IEEE FP64 rounds finish the solve */
    PR_DF64 = 2  /* residual, reserve and pushed mass as double-float pairs
                    (hi + lo floats, 48-bit significand, FP32 instructions); push
                    rounds add into an FP64 inbox with double atomics, folded into
                    the pairs at the next activation; final sums and the output in FP64 */
} pr_prec;

typedef enum {
    PR_MODE_AUTO = 0, /* per round: atomic push when the frontier is small, else CSC pull */
    PR_MODE_PUSH = 1, /* always atomic push over the frontier's out-lists */
    PR_MODE_PULL = 2, /* always deterministic gather over in-lists */
    PR_MODE_LEVELS = 3, /* IFP2 on a graph created with levels: after two synchronous
                          rounds, every round scans the levels in order and a push
                          reaches a higher level in the same round -- the in-round
                          propagation of the asynchronous scans of Sec. 3.2, made
                          deterministic.  The round's residual R counts the pushes
                          still in flight; the stopping rule and the certified bound
                          are those of the other modes.  PR_EINVAL with another
                          algorithm, on a graph without levels, and in
                          pr_solve_batch and the server */
    PR_MODE_ASYNC = 4,  /* IFP1/IFP2 push rounds in the concurrency of Sec. 3.2: the
                          frontier is chosen at the round's start as in the other
                          modes, but each frontier vertex pushes all of its residual
                          at the moment it is processed (an atomic exchange), so mass
                          it received earlier in the same round moves on at once.
                          Fewer rounds; the schedule, and so the rounding and the
                          round count, vary from run to run.  The stopping rule,
                          mass conservation and the certified bound are unchanged.
                          PR_EINVAL with PR_POWER, and in pr_solve_batch and the
                          server */
    PR_MODE_APULL = 5   /* IFP1/IFP2 asynchronous pull rounds, the concurrency of
                          Sec. 3.2 without atomics: a round gathers over every
                          non-dangling row, and each row recomputes what it holds
                          now from the reserves by Eq. 4's identity,
                          r_j = p_j + c sum_{i in S(j)} x_i/((1-c) deg i) - x_j/(1-c),
                          which counts every push committed so far (this round's
                          included when its source committed before the gather read
                          it) and never a push twice; it commits all of r_j when
                          |r_j| > xi_act.  The stop test uses a bound on the
                          residual the round leaves (the commits' pushes counted as
                          possibly not yet taken), so the certified bound holds.
                          Fewer rounds than synchronous ones; the schedule varies
                          from run to run.  With PR_FP32 the recompute cancels to
                          FP32's precision (at most about 1.2e-7/(1-c) of the mass),
                          so FP32 rounds run to a residual of max(eps, ten times
                          that) -- or until the residual stops falling -- and
                          IEEE FP64 rounds continue from the reserve to eps (their
                          first recompute
                          corrects the FP32 rounds, as the FP32 form's correction
                          sweep does; pr_stats.fp64_rounds counts them).  PR_EINVAL
                          with PR_POWER, and in pr_solve_batch and the server */
} pr_mode;

/*
 * Personalization vector p (Sec. 2.1).  nnz < 0: uniform p = e/n.
 * nnz == n and idx == NULL: dense val[n].  Otherwise sparse: val[k] at
 * vertex idx[k], k < nnz, other entries 0.  Entries must be finite and >= 0
 * with a positive sum; p is divided by its sum (the factor is reported in
 * pr_stats.p_scale).  is_device: idx/val are device pointers.
 */
typedef struct {
    int32_t nnz;
    const int32_t *idx;
    const double *val;
    int32_t is_device;
} pr_pvec;

/* Per-solve report. */
typedef struct {
    int32_t rounds;        /* IFP phase-1 rounds (Sec. 3.3.1 "iteration"), or Power iterations */
    int32_t rounds_push;   /* rounds delivered by atomic push */
    int32_t rounds_pull;   /* rounds delivered by in-list gather */
    int32_t fp64_rounds;   /* FP32 form: rounds run in FP64 after the correction sweep */
    int64_t pushes;        /* sum over rounds of |F_t| (active vertices) */
    int64_t edges_pushed;  /* sum over rounds of the active vertices' valid out-edges
                              (the paper's m(t) without the +1, Sec. 3.3.3), plus the
                              IFP2 phase-2 in-edges of dangling vertices */
    int64_t edges_scanned; /* adjacency entries actually read by the delivery kernels */
    double resid_l1;       /* non-dangling residual L1 R at stop (Power: last ||delta||_1) */
    double dangling_mass;  /* sum of the residual on dangling vertices at stop (IFP1) */
    double err_bound;      /* guaranteed L1 distance of `out` from the exact PageRank:
                              IFP1 2cR/(1-c), IFP2 2R/(1-c), Power c*delta/(1-c) */
    double ms;             /* device time of the solve, CUDA events on the graph's stream */
    double p_scale;        /* 1 / sum(p) as given */
    int64_t launches;      /* kernels the solve launched (including those inside CUDA graphs) */
} pr_stats;

/* Kernel kinds of a solve, for pr_kernel_profile. */
enum {
    PR_K_ACTIVATE = 0, /* frontier selection, residual L1, dense pending push */
    PR_K_COMMIT = 1,   /* reserved (the push kernel commits the frontier itself) */
    PR_K_PUSH = 2,     /* push rounds: reserve update + atomic push along out-lists */
    PR_K_PULL = 3,     /* pull rounds: gather along in-lists + next activation */
    PR_K_POWER = 4,    /* Power method iteration */
    PR_K_OTHER = 5,    /* init, correction, phase 2, finalize */
    PR_K_LEVELS = 6,   /* level-ordered rounds (PR_MODE_LEVELS): one round's level launches together */
    PR_K_KINDS = 8
};

/* Per-kernel CUDA-event timing of one solve (opts.profile).  launches[k]
 * counts launches that did work (a round kernel that returned at once because
 * the round used the other delivery mode is not counted); ms[k] is their
 * summed duration. */
typedef struct {
    int32_t launches[PR_K_KINDS];
    double ms[PR_K_KINDS];
} pr_kernel_profile;

/* Tuning and tracing.  Zero-initialise, then set fields; 0 means default. */
typedef struct {
    double xi_act;        /* activation threshold on |r_i| (Alg. 2/3 "h_i > xi");
                             0 => eps / n_nd, which guarantees progress while R > eps */
    int32_t max_rounds;   /* 0 => 100000 */
    int32_t mode;         /* pr_mode */
    double pull_ratio;    /* AUTO: pull when the frontier's out-edges >= pull_ratio * m;
                             0 => the graph's pr_tuning value (0.04 unless set or autotuned) */
    int32_t use_graph;    /* 0 or 1 => rounds run inside a CUDA graph with a device-side
                             while loop (no host sync per round); -1 => host-driven rounds */
    int32_t trace_cap;    /* length of the host trace arrays below (may be 0) */
    double *trace_R;      /* [trace_cap] R_t at the start of round t */
    int64_t *trace_F;     /* [trace_cap] |F_t| */
    int64_t *trace_E;     /* [trace_cap] edges pushed in round t */
    int8_t *trace_mode;   /* [trace_cap] 1 push, 2 pull */
    pr_kernel_profile *profile; /* non-NULL: run the rounds from the host and time every
                                   kernel launch with CUDA events on the graph's stream */
} pr_opts;

/* Static facts about a created graph (the paper's Table 1 columns and more). */
typedef struct {
    int32_t n, n_nd, n_ref, n_d, n_u; /* vertices; non-dangling; non-dangling with in-edges;
                                         dangling; unreferenced (in-degree 0) */
    int64_t m, m_d;                   /* edges; edges into dangling vertices */
    int32_t max_outdeg, max_indeg;
    double ms_preprocess;             /* device time of pr_graph_create (Table 2 analogue) */
    size_t device_bytes;              /* graph storage held on the device */
    int32_t levels;                   /* pr_graph_opts.levels the graph was created with */
    int32_t pad0;
} pr_graph_info;

/*
 * Device memory hooks (optional).  alloc(bytes, stream, ctx) returns a device
 * pointer or NULL; free(ptr, bytes, stream, ctx).  Passing NULL restores
 * cudaMalloc/cudaFree.  Set it before creating graphs; every object frees
 * with the allocator it was allocated with.
 */
typedef void *(*pr_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*pr_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
pr_status pr_set_allocator(pr_alloc_fn alloc, pr_free_fn free_fn, void *ctx);

/*
 * Build the device form of G(V,E) (Sec. 2.1) and run the preprocessing that
 * Alg. 2 and Alg. 3 start with (Sec. 3.4: in IFP2 the edges from a vertex
 * into dangling vertices are marked invalid, so pushes skip them):
 *   out-degree, in-degree, dangling (deg(v) = 0) and unreferenced (no in-link)
 *   classes; vertices are renumbered internally so that every out-list is
 *   [non-dangling targets | dangling targets] and every in-list is
 *   [referenced sources | unreferenced sources], which makes the IFP2 edge
 *   invalidation a per-row prefix; the caller's ids are restored on output.
 *
 * n >= 1, m >= 0.  out_off[n+1] (out_off[0] = 0, non-decreasing,
 * out_off[n] = m) and out_dst[m] (ids in [0, n)) are the out-lists D(v).
 * in_off/in_src (the in-lists S(v)) are optional (NULL): when given they must
 * describe the same edge set and are checked against the out-lists.  A
 * repeated edge is rejected (the adjacency matrix is 0/1, Sec. 2.1); self
 * loops are allowed.  mem_is_device: all four arrays are device pointers,
 * else host.  cuda_stream: the cudaStream_t to run on (NULL = legacy default).
 * The arrays are copied; the caller keeps ownership.  Host arrays are read
 * only within out_off[0..n] and out_dst[0..m): out_off[0] = 0 and out_off[n]
 * = m are checked on the host before the copy, the rest of the checks run on
 * the device on the copies before any kernel indexes by them, and if the
 * device fails before that (no device, no memory) they run on the host.
 * Device memory: the graph itself through the allocator of pr_set_allocator
 * (else cudaMalloc); the temporaries of the build (sort keys, about 16 bytes
 * per edge) through that allocator too when one is installed, else from a
 * stream-ordered pool of the library that keeps up to 2 GiB of them mapped
 * for the next creation on the device.
 * Errors: PR_EINVAL (bad size, offsets, ids, duplicate edge, CSC mismatch;
 * reported ahead of any device error), PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_graph_create(int32_t n, int64_t m, const int32_t *out_off, const int32_t *out_dst,
                          const int32_t *in_off, const int32_t *in_src, int mem_is_device,
                          void *cuda_stream, pr_graph **g);

/*
 * pr_graph_create with options (the in-round propagation of the asynchronous
 * scans of Sec. 3.2 needs an order of the vertices; see PR_MODE_LEVELS).
 * Arguments, ownership and errors as pr_graph_create; opts may be NULL
 * (zero-initialised = defaults); the reserved fields are not read (set them 0).
 *  levels: 0, or L in [1, 16] to prepare level-ordered rounds (PR_MODE_LEVELS):
 *          the non-dangling vertices with in-edges are ranked by
 *          q = floor(2^31 (indeg + 1) / (indeg + outdeg + 2)), ascending (ties
 *          by caller id), and rank r of n_ref gets level floor(r L / n_ref);
 *          inside the referenced class the internal ids run level by level.
 *          Every mode works on such a graph; only PR_MODE_LEVELS needs it.
 *          PR_EINVAL for L outside [0, 16].
 */
typedef struct {
    int32_t levels;
    int32_t reserved[7];
} pr_graph_opts;
pr_status pr_graph_create_ex(int32_t n, int64_t m, const int32_t *out_off, const int32_t *out_dst,
                             const int32_t *in_off, const int32_t *in_src, int mem_is_device, void *cuda_stream,
                             const pr_graph_opts *opts, pr_graph **g);

/* Fill *info for a created graph. */
pr_status pr_graph_get_info(const pr_graph *g, pr_graph_info *info);

/*
 * Launch parameters of a graph's kernels.  They decide how the rounds of
 * Sec. 3.2 / 3.4 map onto the GPU, never what a round computes (the paper has
 * no counterpart: its K CPU threads scan static vertex sets).
 *  pull_thr:     in-degree thresholds of the gather bins, non-increasing, >= 0.
 *                Rows with in-degree above pull_thr[0] get a whole block; above
 *                pull_thr[1..5] they get 32, 16, 8, 4, 2 lanes; the rest 1 lane.
 *                When pull_thr[1] <= 64, IEEE FP64 solves gather the rows at
 *                or below pull_thr[1] by tiles instead: a block stages up to
 *                1024 in-list values of consecutive rows in shared memory and
 *                one thread sums each row there.  Default {4096, 64, 32, 16,
 *                8, 4}.
 *  block_budget: blocks of a dense gather launch, split across the bins in
 *                proportion to their in-list entries (1 .. 16384).
 *  pull_ratio:   the AUTO delivery switch used when a solve passes
 *                pull_ratio = 0: a round pulls when its frontier's out-edges
 *                reach pull_ratio x the valid edges (m, or m - m_d for IFP2).
 *  bin_rows:     (read-only) non-dangling rows per bin, block bin first.
 *  pull_blocks:  (read-only) blocks of a dense gather over the non-dangling rows.
 * pr_graph_set_tuning reads pull_thr, block_budget and pull_ratio (0 keeps the
 * current ratio).  Errors: PR_EINVAL (values; the graph keeps its tuning),
 * PR_ECUDA.
 */
typedef struct {
    int32_t pull_thr[6];
    int32_t block_budget;
    int32_t pad0;
    double pull_ratio;
    int32_t bin_rows[7];
    int32_t pull_blocks;
} pr_tuning;
pr_status pr_graph_get_tuning(const pr_graph *g, pr_tuning *t);
pr_status pr_graph_set_tuning(pr_graph *g, const pr_tuning *t);

/*
 * Autotuner for g's launch parameters (pr_tuning), on g's stream.  It times
 * dense gather rounds (IFP2, state format prec) for a grid of bin thresholds
 * and block budgets and keeps the fastest; then it times atomic push rounds
 * and activation scans against the best gather round and sets pull_ratio at
 * the frontier size where a push round costs as much as a pull round.
 * max_ms bounds the device time of the trial solves (0 = 3000 ms); the best
 * candidate found so far is kept when it runs out.  *t (may be NULL) receives
 * the chosen tuning; report (may be NULL) receives one line per trial, as
 * text, up to report_len bytes.  Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_graph_autotune(pr_graph *g, pr_prec prec, double max_ms, pr_tuning *t, char *report,
                            size_t report_len);

/*
 * Solve PageRank / personalized PageRank on g.
 *  c:   damping factor, 0 < c < 1 (Sec. 2.1).
 *  eps: IFP: stop when the residual L1 over non-dangling vertices R <= eps
 *       (reading of Alg. 2/3 "Management" as an L1 test; activation uses
 *       |r_i| > xi_act).  POWER: stop when ||pi_{k+1} - pi_k||_1 <= eps.
 *  a, prec: pr_algo, pr_prec.   p: personalization (NULL = uniform).
 *  out[n]: the PageRank vector in the caller's vertex ids, sum 1, FP64;
 *       out_is_device selects a device or host pointer.  Written on PR_OK and
 *       PR_ENOTCONV.
 *  st:  optional report.
 * pr_solve_ex adds tuning/tracing options (NULL = defaults).
 * Errors: PR_EINVAL (c, eps, p), PR_ENOTCONV, PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_solve(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                   double *out, int out_is_device, pr_stats *st);
pr_status pr_solve_ex(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                      const pr_opts *opts, double *out, int out_is_device, pr_stats *st);

/*
 * Allocation-free Power-method PageRank.  The paper has no counterpart: this
 * is the library's Power iteration, packaged for callers that cannot
 * allocate device memory -- a framework that owns the whole device
 * memory pool, code on a path where cudaMalloc/cudaFree could synchronise the
 * device, a plug-in that is only handed buffers.  It calls no cudaMalloc,
 * cudaFree or allocating library routine: its working vectors live in one
 * fixed array compiled into this library (about 12.6 MB, held on every GPU
 * that loads the library until the process exits).  Hence:
 *   - n must be at most 524,288; larger n returns PR_EINVAL;
 *   - all calls on a device share that array and the next call overwrites
 *     it: calls that overlap on the GPU (other host threads, other streams)
 *     race, and the caller must serialise them;
 *   - the first call on each device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress); make that first call before
 *     any stream capture.
 * Inputs (device pointers in the caller's vertex ids; not validated, they
 * must describe one valid graph): out_off[n+1] (out-list offsets, giving
 * deg(v)), in_off[n+1] and in_src[m] (in-lists S(v)).  p is uniform.  From
 * pi_0 = e/n it iterates pi_{k+1} = c P pi_k + (c d^T pi_k + (1-c) e^T pi_k) e/n
 * until ||pi_{k+1} - pi_k||_1 <= tol or max_iter iterations, and writes the
 * normalised last iterate to pi[n] (device, owned by the caller).  iters
 * (host, may be NULL) receives the iteration count.  Runs on cuda_stream and
 * synchronises it before returning.
 * Errors: PR_EINVAL (sizes, c, tol, max_iter), PR_ENOTCONV (max_iter reached;
 * pi still written), PR_ECUDA.
 */
pr_status pr_power_noalloc(int32_t n, const int32_t *out_off, const int32_t *in_off, const int32_t *in_src,
                           double c, double tol, int32_t max_iter, double *pi, void *cuda_stream,
                           int32_t *iters);

/*
 * Solve many independent problems at once: IFP1 or IFP2 (Alg. 2 / Alg. 3) on
 * graphs gs[0..count) of any sizes, with damping c[k] and stopping threshold
 * eps[k] (as in pr_solve), uniform personalization (ps may be NULL; any
 * ps[k].nnz >= 0 is rejected), all on gs[0]'s stream and device.  Every
 * problem keeps its own state in one packed device arena; each round phase
 * of all problems is one persistent kernel whose blocks take row tiles of
 * any problem from a device work queue, and the phases run inside a CUDA
 * graph until every problem has stopped.  The arithmetic and stopping rule
 * of each problem are those of pr_solve with the same options (opts may be
 * NULL; traces and profile are ignored).  outs[k][gs[k] n] receives problem
 * k's PageRank (device pointers if outs_are_device, else host).  sts
 * (optional, count entries) gets per-problem reports; ms is the batch time.
 * Errors: PR_EINVAL, PR_ENOTCONV (some problem hit its cap; all outputs are
 * written), PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_solve_batch(pr_graph *const *gs, int32_t count, const double *c, const double *eps, pr_algo a,
                         pr_prec prec, const pr_pvec *ps, const pr_opts *opts, double *const *outs,
                         int outs_are_device, pr_stats *sts);

/*
 * Serving: continuous batching of IFP2 requests (Alg. 3) on resident graphs.
 * A server owns one host thread and a CUDA stream.  The thread admits queued
 * requests while their device memory fits the budget.  On every step it
 * advances all active requests by a few round phases: one persistent kernel
 * per phase takes row tiles of any request from a device work queue.  It
 * finishes the requests that stopped and hands their results back.  A
 * request that arrives while others run joins at the next step.  Arithmetic
 * and stopping rule per request are pr_solve's IFP2 with the default
 * options.
 *
 * pr_server_create: hbm_budget_bytes bounds the device memory of the
 *   admitted requests' states (graphs are the caller's and not counted).
 *   cuda_stream: the stream the server runs on (NULL = legacy default); the
 *   current device is the server's.  *out receives the handle.
 *   Errors: PR_EINVAL (NULL out, zero budget), PR_ENOMEM, PR_ECUDA.
 * pr_server_submit: queue one request on graph g (created on the server's
 *   device; it must stay alive until every ticket on it has been polled
 *   to completion).  c, eps as in pr_solve; prec is PR_DF64 or PR_FP32 (float
 *   rounds, FP64 correction sweep, FP64 rounds: see pr_prec); p is a host pr_pvec
 *   (NULL = uniform; sparse seeds for personalized PageRank), copied.
 *   *ticket receives the request's id.  Thread-safe.  Errors: PR_EINVAL
 *   (arguments, p, a request larger than the whole budget), PR_EAGAIN
 *   (queue full: retry later), PR_ENOMEM.
 * pr_server_poll: PR_EBUSY while the request runs.  Once it has finished:
 *   out[g n] (host or device pointer, may be NULL) receives the PageRank in
 *   the caller's ids (sum 1, FP64) -- the result waits on the device until
 *   this call copies it --, st (may be NULL) the report (ms = submit to
 *   finish), and the ticket is released: PR_OK, or PR_ENOTCONV (round cap reached, or no
 *   vertex left above the activation threshold before R <= eps; out is
 *   written), or the error that stopped the server's thread (PR_ECUDA,
 *   PR_ENOMEM; out is not written).  PR_EINVAL for an unknown or released
 *   ticket.  Thread-safe.
 * pr_server_destroy: stop the thread, drop unfinished requests, free the
 *   server's device memory (NULL is ignored).
 */
pr_status pr_server_create(size_t hbm_budget_bytes, void *cuda_stream, pr_server **out);
pr_status pr_server_submit(pr_server *s, pr_graph *g, double c, double eps, pr_prec prec, const pr_pvec *p,
                           int64_t *ticket);
pr_status pr_server_poll(pr_server *s, int64_t ticket, double *out, pr_stats *st);
void pr_server_destroy(pr_server *s);

/*
 * Server counters since pr_server_create (thread-safe snapshot).  The ms_*
 * fields are host wall time of the server thread per stage, launches and the
 * synchronisations that end them included: admission (allocation, state
 * init, joining a column group), rounds (round launches of groups and of the
 * tile engine, and the stop-flag read), correction (FP32 form), finish
 * (phase 2, normalisation, copy-out).
 */
typedef struct {
    int64_t submitted, finished;      /* requests */
    int64_t steps;                    /* loop iterations that had work */
    int64_t group_launches;           /* column-group round kernels launched */
    int64_t tile_launches;            /* tile-engine phase kernels launched */
    int32_t groups, active;           /* live column groups; requests admitted, not finished */
    double ms_admit, ms_rounds, ms_correct, ms_finish;
    int64_t queued_sum;               /* requests waiting in the queue, summed over steps */
    int64_t running_sum;              /* requests in their rounds (groups and tile engine), summed over steps */
    double ms_tables;                 /* rebuilding and uploading tile tables (part of ms_rounds) */
    double ms_step_max;               /* the longest step */
} pr_server_stats;
pr_status pr_server_get_stats(pr_server *s, pr_server_stats *st);

/*
 * Debug build (libpr_debug.so, compiled with -DPR_DEBUG; the paper has no
 * counterpart).  Its kernels check every index they load from a graph array
 * (in-list sources, out-list targets, frontier entries, the vertex
 * permutation, tile bounds) before using it, and skip the access when it is
 * out of range; after every round of a single solve (synchronous push, pull
 * or asynchronous rounds; not the level-ordered ones) it checks on the device
 * the two invariants of the rounds with a (1-c) reserve: the mass balance
 * (IFP1 sum x + sum r = 1; IFP2 the same plus the mass deferred to phase 2)
 * and the residual identity r = p + c P~ x/(1-c) - x/(1-c) (Sec. 3.1, Eq. 4),
 * each within a tolerance of the state's arithmetic.  A solve or batch whose
 * checks failed returns PR_ECHECK.
 * pr_is_debug_build: 1 in the debug library, 0 in the release one.
 * pr_debug_report_get: the checks run and failed since the last reset, the
 *   first failure (site, value, bound; invariant deviations are scaled by
 *   1e18) and the largest deviations seen; reset != 0 clears it.
 * pr_debug_inject: a test hook: the checks at `site` (0 = none) fail from the
 *   next solve on -- an index check sees half its bound, an invariant check
 *   fails outright -- so the net itself can be tested with no invalid access.
 *   Site 6 instead makes every bounded wait of graph creation's radix sort
 *   (a tile waiting for the counts of the tiles before it) give up at once:
 *   creating a graph whose sorts span more than one tile (over 2048 vertices
 *   or 4096 edges) returns PR_ECUDA, with nothing written outside its
 *   buffers, and creations succeed again once the site is cleared.
 * Both return PR_EINVAL in a release build.
 */
typedef struct {
    int64_t checks, fails;           /* invariant checks run; failed checks of any kind */
    int32_t first_site, pad;         /* 1 in-list source, 2 out-list target, 3 frontier entry,
                                        4 permutation, 5 tile bounds, 16 mass, 17 identity
                                        (6: the sort-wait test hook, never recorded) */
    int64_t first_value, first_bound;
    double max_mass_dev, max_identity_dev;
} pr_debug_report;
int pr_is_debug_build(void);
pr_status pr_debug_report_get(pr_debug_report *out, int reset);
pr_status pr_debug_inject(int32_t site);

/* Release a graph and its workspace (NULL is ignored). */
void pr_destroy(pr_graph *g);

/* Message for the last non-OK status returned to this thread. */
const char *pr_last_error(void);

/* Library version string. */
const char *pr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PR_H */
