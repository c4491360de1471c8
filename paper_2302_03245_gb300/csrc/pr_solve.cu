// pr_solve.cu -- host driver of a solve: workspace, p setup, the round loop
// (IFP1 / IFP2, Alg. 2 / Alg. 3) inside a CUDA-graph while node, the FP64
// correction sweep of the FP32 form, the IFP2 phase-2 pull, the Power-method
// baseline (Sec. 4), normalisation, and pr_solve / pr_solve_ex.
// The kernels and the round state machine are in pr_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pr_kernels.cuh"

namespace pr {

// ------------------------------------------------------------ small kernels
template <typename T>
__global__ void k_init_state(int32_t n, const Ctl *ctl, PVals pv, T *x, T *r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = ST<T>::zero();
        r[i] = ST<T>::p(ctl, pv, i);
    }
}

// dense p in caller ids -> internal ids, scaled
__global__ void k_p_dense(int32_t n, const int32_t *inv, const double *val, double scale, double *p64) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        p64[inv[e]] = val[e] * scale;
}

__global__ void k_p_sparse(int32_t nnz, const int32_t *inv, const int32_t *idx, const double *val, double scale,
                           double *p64) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
        atomicAdd(&p64[inv[idx[k]]], val[k] * scale);
}

// the dense p in the FP32 and double-float formats
__global__ void k_p_formats(int32_t n, const double *p64, float *p32, float2 *pdf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = p64[i];
        p32[i] = (float)v;
        pdf[i] = df_from_d(v);
    }
}

// device-resident p: count bad entries and sum (for validation)
__global__ void k_p_check(int32_t cnt, int32_t n, const int32_t *idx, const double *val, unsigned long long *bad,
                          double *sum) {
    __shared__ double sh[32];
    double s = 0;
    unsigned long long b = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const double v = val[k];
        if (!(v >= 0.0) || !isfinite(v)) b++;
        else s += v;
        if (idx && (idx[k] < 0 || idx[k] >= n)) b++;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(sum, s);
    if (b) atomicAdd(bad, b);
}

// a new run of rounds (after the FP32 phase): the round index continues
__global__ void k_reset_run(Ctl *ctl) {
    ctl->done = 0;
    ctl->status = 0;
    ctl->ticket = 0;
    ctl->mode = MODE_ACT;
    ctl->bin_cnt[0][0] = ctl->bin_cnt[0][1] = ctl->bin_cnt[0][2] = 0;
    ctl->bin_cnt[1][0] = ctl->bin_cnt[1][1] = ctl->bin_cnt[1][2] = 0;
    ctl->want_bins = ctl->policy != MODE_PULL && ctl->policy != POLICY_LEVELS;
    ctl->unref_active = 1;
    ctl->gs_phase = 0;
}

__global__ void k_set_while(const Ctl *ctl, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
}

// Power iteration start: pi_0 = p, q_0 = pi_0 / deg, gamma_0 = c d^T p + (1-c) e^T p.
template <typename T>
__global__ void k_power_init(DevGraph G, Ctl *ctl, Partials P, PVals pv, T *pi, typename ST<T>::V *q) {
    using R = typename ST<T>::R;
    __shared__ double shd[32];
    __shared__ R shr[32];
    R dm = ST<T>::rzero(), tm = ST<T>::rzero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x) {
        const T v = ST<T>::p(ctl, pv, i);
        pi[i] = v;
        if (i < G.n_nd) q[i] = ST<T>::pack(ST<T>::mul(v, ST<T>::invdeg(G, i)));
        else dm = ST<T>::radd(dm, ST<T>::rval(v));
        tm = ST<T>::radd(tm, ST<T>::rval(v));
    }
    const R b2 = block_sum_r<T>(dm, shr), b3 = block_sum_r<T>(tm, shr);
    if (threadIdx.x == 0) {
        store_partial<T>(P.b, b2);
        store_partial<T>(P.c, b3);
    }
    if (!last_block(&ctl->ticket)) return;
    const double sdm = final_sum<T>(P.b, shd);
    const double stm = final_sum<T>(P.c, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        const double gamma = ctl->c * sdm + ctl->one_minus_c * stm;
        ctl->gamma = gamma;
        ctl->gamma_f = (float)gamma;
        ctl->gamma_df = df_from_d(gamma);
        ctl->iter = 0;
        ctl->zsum = stm;
    }
}

// FP32 reserve -> IEEE double state (exactly) and the gather values
// q_u = x_u / ((1-c) deg(u)) of the correction sweep, in double; IFP2's
// dangling residual is p (phase 1 never touches it), IFP1's comes from the sweep
__global__ void k_to_fp64(DevGraph G, const Ctl *ctl, const float *x32, double *x, double *r, double *q, PVals pv,
                          int ifp2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x) {
        const double xv = (double)x32[i];
        x[i] = xv;
        if (i < G.n_nd) q[i] = xv * (G.inv_deg64[i] * ctl->inv_om);
        else if (ifp2) r[i] = ST<double>::p(ctl, pv, i);
    }
}

// FP32 asynchronous pull rounds -> IEEE FP64 ones: the reserve in double and
// the gather values q = x / ((1-c) deg) from it.  The unreferenced
// non-dangling sources get exactly (1-c) p_i, the value they commit in round
// 0 and keep (they receive nothing), so the unreferenced share U the FP64
// rounds gather once agrees with them.  The FP64 rounds recompute every row's
// residual from the reserve (Eq. 4's identity), so the first one does what
// the FP32 form's correction sweep does.
__global__ void k_apull_to_fp64(DevGraph G, const Ctl *ctl, const float *x32, double *x, double *q, PVals pv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x) {
        const bool unref = i >= G.n_ref && i < G.n_nd;
        const double xv = unref ? ctl->one_minus_c * ST<double>::p(ctl, pv, i) : (double)x32[i];
        x[i] = xv;
        if (i < G.n_nd) q[i] = xv * (G.inv_deg64[i] * ctl->inv_om);
    }
}

// the stop threshold of the next run of rounds, with a fresh decision state
// (stall_cap > 0: the run also ends when R stops falling; see Ctl)
__global__ void k_set_stop(Ctl *ctl, double eps, int stall_cap) {
    ctl->eps = eps;
    ctl->done = 0;
    ctl->status = 0;
    ctl->ticket = 0;
    ctl->stall_cap = stall_cap;
    ctl->stall = 0;
    ctl->r_best = 1e300;
}

// q_u = x_u / ((1-c) deg(u)) for the IFP2 phase-2 pull
template <typename T>
__global__ void k_phase2_q(DevGraph G, const Ctl *ctl, const T *x, typename ST<T>::V *q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n_nd; i += gridDim.x * blockDim.x)
        q[i] = ST<T>::pack(ST<T>::mul(x[i], ST<T>::mul(ST<T>::invdeg(G, i), ST<T>::inv_om(ctl))));
}

template <typename T>
__global__ void k_fin_sum(DevGraph G, Ctl *ctl, Partials P, int kind, const T *x, const T *r) {
    using R = typename ST<T>::R;
    __shared__ double shd[32];
    __shared__ R shr[32];
    R s = ST<T>::rzero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x)
        s = ST<T>::radd(s, ST<T>::rval(zval<T>(G, ctl, kind, x, r, i)));
    s = block_sum_r<T>(s, shr);
    if (threadIdx.x == 0) store_partial<T>(P.a, s);
    if (!last_block(&ctl->ticket)) return;
    const double sum = final_sum<T>(P.a, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->zsum = sum;
    }
}

// residual mass on dangling vertices (IFP1 report)
template <typename T>
__global__ void k_dangling_mass(DevGraph G, Ctl *ctl, Partials P, const T *r) {
    using R = typename ST<T>::R;
    __shared__ double shd[32];
    __shared__ R shr[32];
    R s = ST<T>::rzero();
    for (int i = G.n_nd + blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x)
        s = ST<T>::radd(s, ST<T>::rval(r[i]));
    s = block_sum_r<T>(s, shr);
    if (threadIdx.x == 0) store_partial<T>(P.b, s);
    if (!last_block(&ctl->ticket)) return;
    const double sum = final_sum<T>(P.b, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->D = sum;
    }
}

template <typename T>
__global__ void k_fin_write(DevGraph G, const Ctl *ctl, int kind, const T *x, const T *r, double *out) {
    const double inv = 1.0 / ctl->zsum;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x) {
        const int c = PR_IDX(G.perm[i], G.n, DBG_PERM);
        if (c >= 0) out[c] = ST<T>::to_d(zval<T>(G, ctl, kind, x, r, i)) * inv;
    }
}

// ------------------------------------------------------------ debug-build invariants
// After every round of a single solve (debug build), the state (x, r) must
// satisfy what the rounds preserve (Sec. 3.1, Eq. 4, with the (1-c) reserve;
// p sums to 1):
//   mass      IFP1: sum x + sum r = 1.  IFP2: sum x + sum r + Delta = 1, where
//             Delta = sum_i c x_i (deg_i - ndeg_i) / ((1-c) deg_i) is the mass
//             pushed toward dangling vertices and deferred to phase 2;
//   identity  r_j = p_j + c sum_{u in S~(j)} x_u / ((1-c) deg u) - x_j / (1-c),
//             P~ = P (IFP1), P restricted to non-dangling targets (IFP2: a
//             dangling r_j stays p_j).
// Double-float state adds the push-round inbox to r.  One thread per row with a
// serial in-list loop (small graphs only), FP64 atomics into acc[0] (mass) and
// acc[1] (largest identity deviation relative to the row's magnitudes).
#ifdef PR_DEBUG
template <typename T>
__global__ void k_dbg_invariants(DevGraph G, const Ctl *ctl, const T *x, const T *r, const double *din, PVals pv,
                                 int ifp2, double *acc) {
    const double c = ctl->c, om = ctl->one_minus_c;
    double mass = 0.0, dev = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G.n; j += gridDim.x * blockDim.x) {
        const double xj = ST<T>::to_d(x[j]);
        const double rj = ST<T>::to_d(r[j]) + (din ? din[j] : 0.0);
        const double pj = ST<double>::p(ctl, pv, j);
        mass += xj + rj;
        if (ifp2 && j < G.n_nd) {
            const int deg = G.out_off[j + 1] - G.out_off[j];
            mass += c * xj * (double)(deg - G.ndeg[j]) / (om * (double)deg);
        }
        double in = 0.0, mag = 0.0;
        if (!ifp2 || j < G.n_nd) {
            for (int pass = 0; pass < 2; pass++) {
                const int32_t *off = pass ? G.inu_off : G.inr_off;
                const int32_t *src = pass ? G.inu_src : G.inr_src;
                for (int e = off[j]; e < off[j + 1]; e++) {
                    const int u = PR_IDX(src[e], G.n_nd, DBG_IN_SRC);
                    if (u >= 0) in += ST<T>::to_d(x[u]) * G.inv_deg64[u] / om;
                }
            }
        }
        const double want = (ifp2 && j >= G.n_nd) ? pj : pj + c * in - xj / om;
        mag = fabs(pj) + c * in + xj / om + fabs(rj) + 1e-300;
        dev = fmax(dev, fabs(rj - want) / mag);
    }
    atomicAdd(&acc[0], mass);
    atomicMax(reinterpret_cast<unsigned long long *>(&acc[1]), (unsigned long long)__double_as_longlong(dev));
}

// the verdict on one round's sums (one thread): tolerances of the state's
// arithmetic, then the accumulators are cleared for the next round
__global__ void k_dbg_judge(double *acc, double tol_mass, double tol_identity) {
    const double dm = fabs(acc[0] - 1.0), di = acc[1];
    g_pr_dbg.checks++;
    g_pr_dbg.max_mass_dev = fmax(g_pr_dbg.max_mass_dev, dm);
    g_pr_dbg.max_identity_dev = fmax(g_pr_dbg.max_identity_dev, di);
    const bool force = g_pr_dbg.inject == DBG_MASS;
    if (dm > tol_mass || force) dbg_fail(DBG_MASS, (long long)(dm * 1e18), (long long)(tol_mass * 1e18));
    if (di > tol_identity || g_pr_dbg.inject == DBG_IDENTITY)
        dbg_fail(DBG_IDENTITY, (long long)(di * 1e18), (long long)(tol_identity * 1e18));
    acc[0] = 0.0;
    acc[1] = 0.0;
}

// tolerances per state format (p sums to 1; rounds of at most a few hundred)
template <typename T> struct DbgTol;
template <> struct DbgTol<double> {
    static constexpr double mass = 1e-11, identity = 1e-11;
};
template <> struct DbgTol<float2> {
    static constexpr double mass = 1e-10, identity = 1e-9;
};
template <> struct DbgTol<float> {
    static constexpr double mass = 1e-4, identity = 1e-3;
};
#endif

// host side of the debug record of this translation unit
bool dbg_reset_solve(int inject) {
#ifdef PR_DEBUG
    DbgRec z{};
    z.inject = inject;
    return cudaMemcpyToSymbol(g_pr_dbg, &z, sizeof(z)) == cudaSuccess;
#else
    (void)inject;
    return false;
#endif
}
bool dbg_read_solve(DbgRec *out) {
#ifdef PR_DEBUG
    return cudaMemcpyFromSymbol(out, g_pr_dbg, sizeof(*out)) == cudaSuccess;
#else
    (void)out;
    return false;
#endif
}

// ------------------------------------------------------------ profiling
// CUDA-event timing of individual launches (opts.profile): events are
// recorded on the graph's stream around each kernel; afterwards the round
// state machine is replayed on the host from the device trace to charge each
// launch that did work to its kind.
struct Prof {
    pr_kernel_profile *out = nullptr;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int kind;
        size_t e0, e1;
    };
    std::vector<Rec> recs;
    // replay state
    int mode = MODE_ACT, next_round = 0;
    bool finished = false;
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    size_t mark(cudaStream_t s) {
        cudaEvent_t e = next();
        cudaEventRecord(e, s);
        return used - 1;
    }
    void add(int kind, size_t e0, size_t e1) { recs.push_back({kind, e0, e1}); }
    void charge(const Rec &r) {
        float ms = 0;
        cudaEventElapsedTime(&ms, pool[r.e0], pool[r.e1]);
        out->launches[r.kind]++;
        out->ms[r.kind] += ms;
    }
    // modes[k] is the delivery mode of round mode_base + k; the activation of
    // round `last` set the stop flag when `done`
    void settle_rounds(const std::vector<int8_t> &modes, int mode_base, int last, bool done) {
        for (const Rec &r : recs) {
            if (finished) break;
            auto activate = [&]() {
                const int t = next_round;
                if (done && t >= last) {
                    finished = true;
                    return;
                }
                const int k = t - mode_base;
                mode = (k >= 0 && k < (int)modes.size()) ? modes[k] : MODE_PULL;
                next_round = t + 1;
            };
            if ((r.kind == PR_K_PULL || r.kind == PR_K_LEVELS) && mode == MODE_PULL) {
                charge(r);
                activate();
            } else if (r.kind == PR_K_PUSH && mode == MODE_PUSH) {
                charge(r);
                mode = MODE_ACT;
            } else if (r.kind == PR_K_ACTIVATE && mode == MODE_ACT) {
                charge(r);
                activate();
            }
        }
        recs.clear();
        used = 0;
    }
    void settle_power(int last_iter, int first_iter) {
        int it = first_iter;
        for (const Rec &r : recs) {
            if (it < last_iter) charge(r);
            it++;
        }
        recs.clear();
        used = 0;
    }
    ~Prof() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// ------------------------------------------------------------ workspace
struct StateBufs {
    Buf x, r, vbuf, w[2], q;  // round state of one format; q: phase-2 / correction gather values
    Buf din;                  // double-float state: push-round inbox (FP64, zero between rounds)
};

struct Workspace {
    Buf ctl, part, p64, p32, pdf, outbuf, pstage, pstage2, bins, tR, tF, tE, tM;
    Buf dbg;                  // debug build: the invariant sums of a round (2 doubles)
    StateBufs s64, s32, sdf;  // FP64 (reference), FP32, double-float
    Ctl *hctl = nullptr;      // pinned host mirror
    int32_t trace_len = 0;
    uint64_t plan_gen = 0;    // the graph's plan generation the captured graphs were built with
    cudaError_t launch_err = cudaSuccess;  // first failed cudaLaunchKernelEx of a level-ordered round
    cudaStream_t cap_stream = nullptr;
    struct CG {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    } graphs[19];
    void drop_graphs() {
        for (auto &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            g = CG{};
        }
    }
    ~Workspace() {
        drop_graphs();
        if (hctl) cudaFreeHost(hctl);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

void destroy_workspace(pr_graph *g) {
    delete static_cast<Workspace *>(g->ws);
    g->ws = nullptr;
}

static Partials partials_of(Workspace &W) {
    double *d = W.part.as<double>();
    Partials P;
    P.a = d;
    P.b = d + kMaxBlocks;
    P.c = d + 2 * kMaxBlocks;
    P.F = reinterpret_cast<long long *>(d + 3 * kMaxBlocks);
    P.E = P.F + kMaxBlocks;
    P.u = reinterpret_cast<int *>(P.E + kMaxBlocks);
    return P;
}

static Trace trace_of(Workspace &W) {
    Trace t;
    t.R = W.tR.as<double>();
    t.F = W.tF.as<long long>();
    t.E = W.tE.as<long long>();
    t.mode = W.tM.as<int8_t>();
    return t;
}

static PVals pvals_of(Workspace &W) { return PVals{W.p64.as<double>(), W.p32.as<float>(), W.pdf.as<float2>()}; }

// state buffers of one format: x, r (n), vbuf (n_nd), w[2] (n_nd), q (n)
static pr_status alloc_state(StateBufs &S, size_t t_bytes, size_t v_bytes, size_t n, size_t nnd, cudaStream_t s) {
    if (S.q.p) return PR_OK;  // allocated last: present only when all are
    const pr_status st = [&]() -> pr_status {
        PR_TRY(S.x.alloc(t_bytes * n, s));
        PR_TRY(S.r.alloc(t_bytes * n, s));
        PR_TRY(S.vbuf.alloc(t_bytes * nnd, s));
        PR_TRY(S.w[0].alloc(v_bytes * nnd, s));
        PR_TRY(S.w[1].alloc(v_bytes * nnd, s));
        PR_TRY(S.q.alloc(v_bytes * n, s));
        return PR_OK;
    }();
    if (st != PR_OK) {  // leave nothing half-built for the next solve
        for (Buf *b : {&S.x, &S.r, &S.vbuf, &S.w[0], &S.w[1], &S.q}) b->release();
    }
    return st;
}

static pr_status ensure_ws(pr_graph *g, pr_prec prec, int32_t trace_len) {
    cudaStream_t s = g->stream;
    const size_t n = (size_t)g->G.n, nnd = (size_t)std::max(g->G.n_nd, 1);
    if (!g->ws) {
        Workspace *W = new (std::nothrow) Workspace();
        if (!W) return fail(PR_ENOMEM, "host allocation failed");
        const pr_status st = [&]() -> pr_status {
            PR_TRY(W->ctl.alloc(sizeof(Ctl), s));
            PR_TRY(W->part.alloc(sizeof(double) * kMaxBlocks * 6, s));
            PR_TRY(W->p64.alloc(sizeof(double) * n, s));
            PR_TRY(W->p32.alloc(sizeof(float) * n, s));
            PR_TRY(W->pdf.alloc(sizeof(float2) * n, s));
            PR_TRY(W->outbuf.alloc(sizeof(double) * n, s));
            PR_TRY(W->bins.alloc(sizeof(int32_t) * 3 * nnd, s));
            PR_CK(cudaMallocHost(&W->hctl, sizeof(Ctl)));
#ifdef PR_DEBUG
            PR_TRY(W->dbg.alloc(2 * sizeof(double), s));
            PR_CK(cudaMemsetAsync(W->dbg.p, 0, 2 * sizeof(double), s));
#endif
            PR_CK(cudaMemsetAsync(W->ctl.p, 0, sizeof(Ctl), s));
            PR_CK(cudaMemsetAsync(W->part.p, 0, W->part.bytes, s));
            return PR_OK;
        }();
        if (st != PR_OK) {  // the next solve starts over
            g->ws = W;
            destroy_workspace(g);
            return st;
        }
        g->ws = W;
    }
    Workspace &W = *static_cast<Workspace *>(g->ws);
    if (prec == PR_FP64 || prec == PR_FP32) PR_TRY(alloc_state(W.s64, sizeof(double), sizeof(double), n, nnd, s));
    if (prec == PR_FP32) PR_TRY(alloc_state(W.s32, sizeof(float), sizeof(float), n, nnd, s));
    if (prec == PR_DF64) {
        if (!W.sdf.din.p) PR_TRY(W.sdf.din.alloc(sizeof(double) * n, s));
        PR_TRY(alloc_state(W.sdf, sizeof(float2), sizeof(float2), n, nnd, s));
    }
    if (trace_len > W.trace_len) {
        W.drop_graphs();  // the traces are kernel arguments of the captured graphs
        PR_TRY(W.tR.alloc(sizeof(double) * trace_len, s));
        PR_TRY(W.tF.alloc(sizeof(long long) * trace_len, s));
        PR_TRY(W.tE.alloc(sizeof(long long) * trace_len, s));
        PR_TRY(W.tM.alloc(sizeof(int8_t) * trace_len, s));
        W.trace_len = trace_len;
    }
    return PR_OK;
}

static int grid_n(int64_t items, int sms, int per_sm = 8) {
    const int64_t b = (items + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * per_sm));
}

template <typename T> static StateBufs &state_of(Workspace &W);
template <> StateBufs &state_of<double>(Workspace &W) { return W.s64; }
template <> StateBufs &state_of<float>(Workspace &W) { return W.s32; }
template <> StateBufs &state_of<float2>(Workspace &W) { return W.sdf; }

template <typename T> static RoundBuf round_bufs(Workspace &W) {
    StateBufs &S = state_of<T>(W);
    return RoundBuf{S.x.p, S.r.p, S.vbuf.p, {S.w[0].p, S.w[1].p}, W.bins.as<int32_t>(), S.din.as<double>()};
}

// graph-cache keys: 2 per round format (IFP1, IFP2) and one per Power format
template <typename T> static int round_key();
template <> int round_key<float>() { return 0; }
template <> int round_key<double>() { return 2; }
template <> int round_key<float2>() { return 4; }
template <typename T> static int level_key();
template <> int level_key<float>() { return 6; }
template <> int level_key<double>() { return 7; }
template <> int level_key<float2>() { return 8; }
template <typename T> static int power_key();
template <> int power_key<float>() { return 10; }
template <> int power_key<double>() { return 11; }
template <> int power_key<float2>() { return 12; }
template <typename T> static int apull_key();  // 2 per format (IFP1, IFP2)
template <> int apull_key<double>() { return 13; }
template <> int apull_key<float2>() { return 15; }
template <> int apull_key<float>() { return 17; }

// ------------------------------------------------------------ plans
// The plans of a kernel instantiation: the tiled ones where its kernels carry
// gather tiles (UseTiles, pr_kernels.cuh), else the per-row lane bins.
template <typename T> static const Plan &plan_nd_of(const pr_graph *g) {
    return UseTiles<T>::value ? g->plan_nd_t : g->plan_nd;
}
template <typename T> static const Plan &plan_all_of(const pr_graph *g) {
    return UseTiles<T>::value ? g->plan_all_t : g->plan_all;
}
template <typename T> static const Plan &plan_d_of(const pr_graph *g) {
    return UseTiles<T>::value ? g->plan_d_t : g->plan_d;
}

// ------------------------------------------------------------ round loop
constexpr int kRoundLaunches = 3;  // k_round_pull, k_push, k_activate
constexpr int kUnroll = 4;         // rounds per while-loop body

template <typename T, bool IFP2>
static void launch_round(pr_graph *g, Workspace &W, cudaStream_t s, Prof *prof) {
    const DevGraph &G = g->G;
    Ctl *ctl = W.ctl.as<Ctl>();
    const Partials P = partials_of(W);
    const Trace tr = trace_of(W);
    const RoundBuf B = round_bufs<T>(W);
    const int sms = g->num_sms;
    const Plan &PL = IFP2 ? plan_nd_of<T>(g) : plan_all_of<T>(g);
    const int nbt = sms * 4, nbw = sms * 4, nbc = sms * 2;
    const size_t e0 = prof ? prof->mark(s) : 0;
    k_round_pull<T, IFP2><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, P, B, tr);
    const size_t e1 = prof ? prof->mark(s) : 0;
    k_push<T, IFP2><<<nbt + nbw + nbc, kThreads, 0, s>>>(G, ctl, B, nbt, nbw);
    const size_t e2 = prof ? prof->mark(s) : 0;
    k_activate<T, IFP2><<<grid_n(G.n_nd, sms, 8), kThreads, 0, s>>>(G, ctl, P, B, tr);
#ifdef PR_DEBUG
    k_dbg_invariants<T><<<grid_n(G.n, sms, 8), kThreads, 0, s>>>(G, ctl, static_cast<const T *>(B.x),
                                                                 static_cast<const T *>(B.r), B.din, pvals_of(W),
                                                                 IFP2 ? 1 : 0, W.dbg.as<double>());
    k_dbg_judge<<<1, 1, 0, s>>>(W.dbg.as<double>(), DbgTol<T>::mass, DbgTol<T>::identity);
#endif
    if (prof) {
        const size_t e3 = prof->mark(s);
        prof->add(PR_K_PULL, e0, e1);
        prof->add(PR_K_PUSH, e1, e2);
        prof->add(PR_K_ACTIVATE, e2, e3);
    }
}

// One level-ordered round (IFP2, PR_MODE_LEVELS): one k_round_levels launch per
// level in level order, then the rows without in-edges, whose launch takes the
// round's decision over the partial slots of all of them.  Round 0 is the
// activation of p (k_activate); the push kernel never runs in this mode.
template <typename T>
static void launch_round_levels(pr_graph *g, Workspace &W, cudaStream_t s, Prof *prof) {
    const DevGraph &G = g->G;
    Ctl *ctl = W.ctl.as<Ctl>();
    const Partials P = partials_of(W);
    const Trace tr = trace_of(W);
    const RoundBuf B = round_bufs<T>(W);
    // grids padded to whole clusters of kLevelCluster blocks (the long rows'
    // clusters; the padding blocks only take part in the reduction)
    auto grid_of = [](const Plan &PL) { return (PL.nblocks + kLevelCluster - 1) / kLevelCluster * kLevelCluster; };
    int total = grid_of(g->plan_unref);
    for (int l = 0; l < g->levels; l++) total += grid_of(g->plan_lvl[l]);
    // programmatic stream serialization: each level launch may start while the
    // previous one drains (the kernel waits for it before reading anything)
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = kLevelCluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    auto launch = [&](const Plan &PL, LevelLaunch lv) {
        LevelPlan LP{};
        LP.nseg = std::min(PL.nseg, kNumThr + 2);  // a level (cluster rows, block rows, lane bins) or the unreferenced rows
        LP.nblocks = PL.nblocks;
        for (int k = 0; k < LP.nseg; k++) LP.seg[k] = PL.seg[k];
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid_of(PL));
        cfg.blockDim = dim3(kThreads);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_round_levels<T>, G, LP, ctl, P, B, tr, lv);
        if (e != cudaSuccess && W.launch_err == cudaSuccess) W.launch_err = e;
    };
    const size_t e0 = prof ? prof->mark(s) : 0;
    int base = 0;
    for (int l = 0; l < g->levels; l++) {
        launch(g->plan_lvl[l], LevelLaunch{g->level_lo[l], base, total, 0});
        base += grid_of(g->plan_lvl[l]);
    }
    launch(g->plan_unref, LevelLaunch{G.n_ref, base, total, 1});
    const size_t e1 = prof ? prof->mark(s) : 0;
    k_activate<T, true><<<grid_n(G.n_nd, g->num_sms, 8), kThreads, 0, s>>>(G, ctl, P, B, tr);
    if (prof) {
        const size_t e2 = prof->mark(s);
        prof->add(PR_K_LEVELS, e0, e1);
        prof->add(PR_K_ACTIVATE, e1, e2);
    }
}

// Build (once per key) a graph whose while node repeats `body` until ctl->done.
template <typename F>
static pr_status while_graph(Workspace &W, int key, Ctl *ctl, F body, cudaStream_t s) {
    Workspace::CG &cg = W.graphs[key];
    if (!cg.exec) {
        if (!W.cap_stream) PR_CK(cudaStreamCreateWithFlags(&W.cap_stream, cudaStreamNonBlocking));
        PR_CK(cudaGraphCreate(&cg.graph, 0));
        cudaGraphConditionalHandle h;
        PR_CK(cudaGraphConditionalHandleCreate(&h, cg.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        PR_CK(cudaGraphAddNode(&node, cg.graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
        PR_CK(cudaStreamBeginCaptureToGraph(W.cap_stream, bodyg, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
        body(W.cap_stream);
        k_set_while<<<1, 1, 0, W.cap_stream>>>(ctl, h);
        cudaGraph_t captured = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(W.cap_stream, &captured);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (while body)");
        PR_CK(cudaGraphInstantiate(&cg.exec, cg.graph, 0));
    }
    PR_CK(cudaGraphLaunch(cg.exec, s));
    PR_CK(cudaGetLastError());
    return PR_OK;
}

// Rounds until the device stop flag is set: inside a CUDA-graph while node
// (kUnroll rounds per body, no host synchronisation), or host-driven chunks.
template <typename T, bool IFP2>
static pr_status run_rounds(pr_graph *g, Workspace &W, bool use_graph, bool levels, Prof *prof) {
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    auto round = [&](cudaStream_t cs, Prof *pf) {
        if (levels) launch_round_levels<T>(g, W, cs, pf);
        else launch_round<T, IFP2>(g, W, cs, pf);
    };
    W.launch_err = cudaSuccess;
    if (use_graph && !prof) {
        PR_TRY(while_graph(W, levels ? level_key<T>() : round_key<T>() + (IFP2 ? 1 : 0), ctl, [&](cudaStream_t cs) {
            for (int k = 0; k < kUnroll; k++) round(cs, nullptr);
        }, s));
        if (W.launch_err != cudaSuccess) return cuda_fail(W.launch_err, "cudaLaunchKernelEx (level-ordered round)");
        return PR_OK;
    }
    int t0 = 0;
    if (prof) {
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        t0 = W.hctl->round;
        prof->mode = MODE_ACT;
        prof->next_round = t0;
        prof->finished = false;
    }
    int chunk = 2;
    std::vector<int8_t> modes;
    for (;;) {
        for (int k = 0; k < chunk; k++) round(s, prof);
        if (W.launch_err != cudaSuccess) return cuda_fail(W.launch_err, "cudaLaunchKernelEx (level-ordered round)");
        PR_CK(cudaGetLastError());
        PR_CK(cudaMemcpyAsync(&W.hctl->done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->gs_phase, &ctl->gs_phase, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        const int done = W.hctl->done;
        // a level-ordered round that stops has already advanced the round index
        const int last = W.hctl->round - ((done && W.hctl->gs_phase) ? 1 : 0);
        if (prof) {
            const int hi = std::min(last, W.trace_len);
            modes.assign(std::max(hi - t0, 0), 0);
            if (hi > t0) PR_CK(cudaMemcpy(modes.data(), W.tM.as<int8_t>() + t0, hi - t0, cudaMemcpyDeviceToHost));
            prof->settle_rounds(modes, t0, last, done != 0);
        }
        if (done) break;
        chunk = std::min(chunk * 2, 32);
    }
    return PR_OK;
}

// Power: two iterations per body (ping-pong between the x and r buffers and the two w buffers)
template <typename T>
static void launch_power_pair(pr_graph *g, Workspace &W, cudaStream_t s, Prof *prof) {
    using V = typename ST<T>::V;
    const DevGraph &G = g->G;
    Ctl *ctl = W.ctl.as<Ctl>();
    StateBufs &S = state_of<T>(W);
    SweepArgs<T> a{};
    a.pv = pvals_of(W);
    a.P = partials_of(W);
    a.tr = trace_of(W);
    const Plan &PL = plan_all_of<T>(g);
    const size_t m0 = prof ? prof->mark(s) : 0;
    a.val = S.w[0].as<V>();
    a.pi_cur = S.x.as<T>();
    a.pi_next = S.r.as<T>();
    a.q_next = S.w[1].as<V>();
    k_sweep<T, OP_POWER><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
    const size_t m1 = prof ? prof->mark(s) : 0;
    a.val = S.w[1].as<V>();
    a.pi_cur = S.r.as<T>();
    a.pi_next = S.x.as<T>();
    a.q_next = S.w[0].as<V>();
    k_sweep<T, OP_POWER><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
    if (prof) {
        const size_t m2 = prof->mark(s);
        prof->add(PR_K_POWER, m0, m1);
        prof->add(PR_K_POWER, m1, m2);
    }
}

template <typename T>
static pr_status run_power(pr_graph *g, Workspace &W, bool use_graph, Prof *prof) {
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    if (use_graph && !prof)
        return while_graph(W, power_key<T>(), ctl, [&](cudaStream_t cs) { launch_power_pair<T>(g, W, cs, nullptr); },
                           s);
    int chunk = 2, it = 0;
    for (;;) {
        for (int k = 0; k < chunk; k++) launch_power_pair<T>(g, W, s, prof);
        PR_CK(cudaGetLastError());
        PR_CK(cudaMemcpyAsync(&W.hctl->done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->iter, &ctl->iter, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        if (prof) prof->settle_power(W.hctl->iter, it);
        it += 2 * chunk;
        if (W.hctl->done) break;
        chunk = std::min(chunk * 2, 32);
    }
    return PR_OK;
}

// ------------------------------------------------------------ p setup
static pr_status setup_p(pr_graph *g, Workspace &W, const pr_pvec *p, Ctl &h, double *p_scale) {
    cudaStream_t s = g->stream;
    const int32_t n = g->G.n;
    *p_scale = 1.0;
    if (!p || p->nnz < 0) {
        h.p_dense = 0;
        h.pu = 1.0 / (double)n;
        return PR_OK;
    }
    const bool dense = (p->nnz == n && p->idx == nullptr);
    const int32_t cnt = p->nnz;
    if (!dense && (cnt < 0 || cnt > n)) return fail(PR_EINVAL, "p.nnz out of range");
    if (cnt > 0 && !p->val) return fail(PR_EINVAL, "p.val is NULL");
    if (!dense && cnt > 0 && !p->idx) return fail(PR_EINVAL, "p.idx is NULL");
    double sum = 0.0;
    const double *dval = p->val;
    const int32_t *didx = p->idx;
    if (!p->is_device) {
        for (int32_t k = 0; k < cnt; k++) {
            const double v = p->val[k];
            if (!(v >= 0.0) || !std::isfinite(v)) return fail(PR_EINVAL, "p has a negative or non-finite entry");
            if (!dense && (p->idx[k] < 0 || p->idx[k] >= n)) return fail(PR_EINVAL, "p.idx out of range");
            sum += v;
        }
        if (!(sum > 0.0)) return fail(PR_EINVAL, "p sums to zero");
        if (W.pstage.bytes < sizeof(double) * std::max(cnt, 1))
            PR_TRY(W.pstage.alloc(sizeof(double) * std::max(cnt, 1), s));
        PR_CK(cudaMemcpyAsync(W.pstage.p, p->val, sizeof(double) * cnt, cudaMemcpyHostToDevice, s));
        dval = W.pstage.as<double>();
        if (!dense) {
            if (W.pstage2.bytes < sizeof(int32_t) * std::max(cnt, 1))
                PR_TRY(W.pstage2.alloc(sizeof(int32_t) * std::max(cnt, 1), s));
            PR_CK(cudaMemcpyAsync(W.pstage2.p, p->idx, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s));
            didx = W.pstage2.as<int32_t>();
        }
    } else {
        Buf chk;
        PR_TRY(chk.alloc(16, s));
        PR_CK(cudaMemsetAsync(chk.p, 0, 16, s));
        unsigned long long *bad = chk.as<unsigned long long>();
        double *dsum = reinterpret_cast<double *>(bad + 1);
        if (cnt > 0)
            k_p_check<<<grid_n(cnt, g->num_sms), kThreads, 0, s>>>(cnt, n, dense ? nullptr : didx, dval, bad, dsum);
        unsigned long long hb[2];
        PR_CK(cudaMemcpyAsync(hb, chk.p, 16, cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        std::memcpy(&sum, &hb[1], sizeof(double));
        if (hb[0]) return fail(PR_EINVAL, "p has a negative, non-finite or out-of-range entry");
        if (!(sum > 0.0)) return fail(PR_EINVAL, "p sums to zero");
    }
    const double scale = 1.0 / sum;
    *p_scale = scale;
    double *p64 = W.p64.as<double>();
    if (dense) {
        k_p_dense<<<grid_n(n, g->num_sms), kThreads, 0, s>>>(n, g->G.inv, dval, scale, p64);
    } else {
        PR_CK(cudaMemsetAsync(p64, 0, sizeof(double) * n, s));
        if (cnt > 0)
            k_p_sparse<<<grid_n(cnt, g->num_sms), kThreads, 0, s>>>(cnt, g->G.inv, didx, dval, scale, p64);
    }
    k_p_formats<<<grid_n(n, g->num_sms), kThreads, 0, s>>>(n, p64, W.p32.as<float>(), W.pdf.as<float2>());
    h.p_dense = 1;
    h.pu = 0.0;
    return PR_OK;
}

// ------------------------------------------------------------ asynchronous pull rounds
// PR_MODE_APULL: round 0 (every vertex commits p), the unreferenced sources'
// constant share U, then pull rounds until the stop flag, inside a CUDA-graph
// while node (kUnroll rounds per body) or host-driven.  fresh = false: no
// round 0 (the reserve and q are already set), U from the q in place.
template <typename T, bool IFP2>
static pr_status run_apull(pr_graph *g, Workspace &W, bool use_graph, Prof *prof, bool fresh = true) {
    const DevGraph &G = g->G;
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    const Partials P = partials_of(W);
    const Trace tr = trace_of(W);
    RoundBuf B = round_bufs<T>(W);
    B.pv = pvals_of(W);
    const Plan &PL = plan_nd_of<T>(g);
    const int sms = g->num_sms;
    if (fresh) {  // else the rounds continue from a reserve and q already in place
        const size_t e0 = prof ? prof->mark(s) : 0;
        k_apull_init<T, IFP2><<<grid_n(G.n_nd, sms, 8), kThreads, 0, s>>>(G, ctl, P, B, tr);
        if (prof) prof->add(PR_K_ACTIVATE, e0, prof->mark(s));
    }
    k_apull_unref<T><<<grid_n((int64_t)G.n_nd * 32, sms, 8), kThreads, 0, s>>>(G, B);
    auto round = [&](cudaStream_t cs, Prof *pf) {
        const size_t e0 = pf ? pf->mark(cs) : 0;
        k_round_apull<T, IFP2><<<PL.nblocks, kThreads, 0, cs>>>(G, PL, ctl, P, B, tr);
        if (pf) pf->add(PR_K_PULL, e0, pf->mark(cs));
    };
    if (use_graph && !prof)
        return while_graph(W, apull_key<T>() + (IFP2 ? 1 : 0), ctl, [&](cudaStream_t cs) {
            for (int k = 0; k < kUnroll; k++) round(cs, nullptr);
        }, s);
    if (prof) {
        prof->mode = MODE_ACT;
        prof->next_round = 0;
        prof->finished = false;
    }
    int chunk = 2;
    std::vector<int8_t> modes;
    for (;;) {
        for (int k = 0; k < chunk; k++) round(s, prof);
        PR_CK(cudaGetLastError());
        PR_CK(cudaMemcpyAsync(&W.hctl->done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        const int done = W.hctl->done, last = W.hctl->round;
        if (prof) {
            const int hi = std::min(last, W.trace_len);
            modes.assign(std::max(hi, 0), (int8_t)MODE_PULL);
            prof->settle_rounds(modes, 0, last, done != 0);
        }
        if (done) break;
        chunk = std::min(chunk * 2, 32);
    }
    return PR_OK;
}

// IFP1 after asynchronous pull rounds: the residual of every row, dangling ones
// included, from the reserves (the rounds keep only what rows left behind)
template <typename T>
static void apull_final_residual(pr_graph *g, Workspace &W) {
    using V = typename ST<T>::V;
    StateBufs &S = state_of<T>(W);
    SweepArgs<T> a{};
    a.val = S.w[0].as<V>();
    a.r = S.r.as<T>();
    a.x = S.x.as<T>();
    a.pv = pvals_of(W);
    const Plan &PL = plan_all_of<T>(g);
    k_sweep<T, OP_CORRECT><<<PL.nblocks, kThreads, 0, g->stream>>>(g->G, PL, W.ctl.as<Ctl>(), a);
}

// ------------------------------------------------------------ solve
// PR_MODE_APULL with PR_FP32: the FP32 rounds hand over to IEEE FP64 ones at a
// residual kApullF32Margin times the FP32 recompute's own error, which is at
// most about 2 x 2^-24 / (1 - c) of the mass (the rounding of every stored
// x_j / (1 - c) and q_i, summed over the rows; the gathered sums are double):
// 7.9e-6 at c = 0.85.  Should R stop falling first (kApullF32Stall rounds
// without a 1% gain), they hand over then.  Measured on R-MAT scale 22 and
// the scale-24 DAG-heavy graph: the FP32 rounds still fall below 5e-7, and
// handing over at 1e-6 instead of 1e-5 saves 3-5% of the time.
constexpr double kApullF32Margin = 10.0;
constexpr int kApullF32Stall = 8;

template <typename T>
static pr_status ifp_phase1(pr_graph *g, Workspace &W, int algo, bool use_graph, bool levels, Prof *prof) {
    if (algo == PR_IFP2) return run_rounds<T, true>(g, W, use_graph, levels, prof);
    return run_rounds<T, false>(g, W, use_graph, false, prof);
}

// After phase 1 in format T: IFP1 dangling-mass report, IFP2 phase 2, then normalisation.
template <typename T>
static void finish_ifp(pr_graph *g, Workspace &W, int algo, double *dout, int64_t &launches) {
    using V = typename ST<T>::V;
    const DevGraph &G = g->G;
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    StateBufs &S = state_of<T>(W);
    const Partials P = partials_of(W);
    const int gn = grid_n(G.n, g->num_sms, 8);
    if (algo == PR_IFP1) {
        k_dangling_mass<T><<<gn, kThreads, 0, s>>>(G, ctl, P, S.r.as<T>());
        launches += 1;
    }
    if (algo == PR_IFP2 && G.n > G.n_nd) {  // phase 2 (Alg. 3): one pull into every dangling vertex
        k_phase2_q<T><<<grid_n(G.n_nd, g->num_sms, 8), kThreads, 0, s>>>(G, ctl, S.x.as<T>(), S.q.as<V>());
        SweepArgs<T> a{};
        a.val = S.q.as<V>();
        a.r = S.r.as<T>();
        a.pv = pvals_of(W);
        k_sweep<T, OP_PHASE2><<<plan_d_of<T>(g).nblocks, kThreads, 0, s>>>(G, plan_d_of<T>(g), ctl, a);
        launches += 2;
    }
    k_fin_sum<T><<<gn, kThreads, 0, s>>>(G, ctl, P, algo, S.x.as<T>(), S.r.as<T>());
    k_fin_write<T><<<gn, kThreads, 0, s>>>(G, ctl, algo, S.x.as<T>(), S.r.as<T>(), dout);
    launches += 2;
}

template <typename T>
static pr_status solve_power(pr_graph *g, Workspace &W, bool use_graph, Prof *prof, double *dout,
                             int64_t &launches) {
    const DevGraph &G = g->G;
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    StateBufs &S = state_of<T>(W);
    const int gn = grid_n(G.n, g->num_sms, 8);
    k_power_init<T><<<gn, kThreads, 0, s>>>(G, ctl, partials_of(W), pvals_of(W), S.x.as<T>(),
                                           S.w[0].as<typename ST<T>::V>());
    PR_TRY(run_power<T>(g, W, use_graph, prof));
    PR_CK(cudaMemcpyAsync(W.hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaStreamSynchronize(s));
    const T *res = (W.hctl->iter & 1) ? S.r.as<T>() : S.x.as<T>();  // odd iteration count ends in r
    k_fin_sum<T><<<gn, kThreads, 0, s>>>(G, ctl, partials_of(W), PR_POWER, res, res);
    k_fin_write<T><<<gn, kThreads, 0, s>>>(G, ctl, PR_POWER, res, res, dout);
    const int64_t pairs = (W.hctl->iter + 1) / 2 + 1;
    launches += 3 + ((use_graph && !prof) ? pairs * 3 : pairs * 2);
    return PR_OK;
}

static pr_status solve_impl(pr_graph *g, double c, double eps, pr_algo algo, pr_prec prec, const pr_pvec *p,
                            const pr_opts *o, double *out, int out_is_device, pr_stats *st) {
    if (!(c > 0.0 && c < 1.0)) return fail(PR_EINVAL, "c must be in (0, 1)");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PR_EINVAL, "eps must be positive and finite");
    if (algo != PR_POWER && algo != PR_IFP1 && algo != PR_IFP2) return fail(PR_EINVAL, "unknown algorithm");
    if (prec != PR_FP64 && prec != PR_FP32 && prec != PR_DF64) return fail(PR_EINVAL, "unknown precision");
    if (!out) return fail(PR_EINVAL, "out is NULL");
    pr_opts opt{};
    if (o) opt = *o;
    if (opt.max_rounds <= 0) opt.max_rounds = 100000;
    if (opt.pull_ratio <= 0) opt.pull_ratio = g->pull_ratio;
    if (opt.mode < 0 || opt.mode > PR_MODE_APULL) return fail(PR_EINVAL, "unknown mode");
    if (opt.mode == PR_MODE_ASYNC && algo == PR_POWER) return fail(PR_EINVAL, "PR_MODE_ASYNC runs IFP1 and IFP2");
    const bool apull = opt.mode == PR_MODE_APULL;
    if (apull && algo == PR_POWER) return fail(PR_EINVAL, "PR_MODE_APULL runs IFP1 and IFP2");
    const bool levels = opt.mode == PR_MODE_LEVELS;
    if (levels && algo != PR_IFP2) return fail(PR_EINVAL, "PR_MODE_LEVELS runs IFP2 only");
    if (levels && g->levels <= 0) return fail(PR_EINVAL, "PR_MODE_LEVELS needs a graph created with levels");
    if (opt.xi_act < 0) return fail(PR_EINVAL, "xi_act must be >= 0");
    const bool use_graph = opt.use_graph >= 0;  // 0 = default (on); -1 = host-driven rounds
    Prof prof_obj;
    Prof *prof = nullptr;
    if (opt.profile) {
        std::memset(opt.profile, 0, sizeof(*opt.profile));
        prof_obj.out = opt.profile;
        prof = &prof_obj;
    }
    PR_TRY(ensure_ws(g, prec, opt.max_rounds + 2));
    Workspace &W = *static_cast<Workspace *>(g->ws);
    if (W.plan_gen != g->plan_gen) {  // the captured launches carry the old plans
        W.drop_graphs();
        W.plan_gen = g->plan_gen;
    }
    cudaStream_t s = g->stream;
    const DevGraph &G = g->G;
    Ctl h{};
    double p_scale = 1.0;
    PR_TRY(setup_p(g, W, p, h, &p_scale));
    const int64_t m_valid = algo == PR_IFP2 ? (G.m - g->info.m_d) : G.m;
    h.c = c;
    h.one_minus_c = 1.0 - c;
    h.eps = eps;
    h.xi = opt.xi_act > 0 ? opt.xi_act : eps / (double)std::max(G.n_nd, 1);
    h.pull_edges = opt.pull_ratio * (double)std::max<int64_t>(m_valid, 1);
    h.algo = algo;
    h.policy = opt.mode;
    h.max_rounds = opt.max_rounds;
    h.trace_cap = W.trace_len;
    fill_formats(h);
    // in-list entries one pull round reads (IFP2: non-dangling rows only)
    h.scan_ref = algo == PR_IFP2 ? g->scan_nd_ref : G.m_ref;
    h.scan_unref = algo == PR_IFP2 ? g->scan_nd_unref : G.m_unref;
    h.mode = MODE_ACT;
    h.want_bins = opt.mode == PR_MODE_AUTO || opt.mode == PR_MODE_PUSH || opt.mode == PR_MODE_ASYNC;
    h.unref_active = 1;
    h.gs_phase = 0;
    *W.hctl = h;
    Ctl *ctl = W.ctl.as<Ctl>();
    PR_CK(cudaMemcpyAsync(ctl, W.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    PR_CK(cudaEventCreate(&e0));
    PR_CK(cudaEventCreate(&e1));
    PR_CK(cudaEventRecord(e0, s));
    const int gn = grid_n(G.n, g->num_sms, 8);
    const PVals pv = pvals_of(W);
    double *dout = out_is_device ? out : W.outbuf.as<double>();
    int fp64_rounds = 0;
    int64_t launches = 0;
    auto count_rounds = [&](int first_round) -> pr_status {
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->gs_phase, &ctl->gs_phase, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        // a stop in a level-ordered round counts that round (round = t + 1)
        const int64_t acts = W.hctl->round - first_round + (W.hctl->gs_phase ? 0 : 1);
        const int64_t bodies = (acts + kUnroll - 1) / kUnroll;
        const int per_round = levels ? g->levels + 2 : kRoundLaunches;
        launches += (use_graph && !prof) ? bodies * (kUnroll * per_round + 1) : acts * per_round;
        return PR_OK;
    };
    // asynchronous pull rounds: launches of round 0, the unreferenced share, the
    // rounds (kUnroll per graph body) and the finish
    auto apull_launches = [&](int first_round = 0) -> pr_status {
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        const int64_t rr = std::max(W.hctl->round - first_round - (first_round ? 0 : 1), 0);
        launches += 2 + ((use_graph && !prof) ? ((rr + kUnroll - 1) / kUnroll + 1) * (kUnroll + 1) : rr);
        return PR_OK;
    };
    if (algo == PR_POWER) {
        if (prec == PR_FP64) PR_TRY(solve_power<double>(g, W, use_graph, prof, dout, launches));
        else if (prec == PR_FP32) PR_TRY(solve_power<float>(g, W, use_graph, prof, dout, launches));
        else PR_TRY(solve_power<float2>(g, W, use_graph, prof, dout, launches));
    } else if (apull && prec == PR_FP64) {
        k_init_state<double><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.s64.x.as<double>(), W.s64.r.as<double>());
        if (algo == PR_IFP2) PR_TRY((run_apull<double, true>(g, W, use_graph, prof)));
        else PR_TRY((run_apull<double, false>(g, W, use_graph, prof)));
        PR_TRY(apull_launches());
        if (algo == PR_IFP1) {
            apull_final_residual<double>(g, W);
            launches += 1;
        }
        finish_ifp<double>(g, W, algo, dout, launches);
        launches += 1;
    } else if (apull && prec == PR_FP32) {
        // FP32 asynchronous pull rounds down to max(eps, the hand-over point),
        // where the recompute's cancellation in FP32 is still well below the
        // residual; then IEEE FP64 asynchronous pull rounds from the reserve to eps
        k_init_state<float><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.s32.x.as<float>(), W.s32.r.as<float>());
        const double handover = kApullF32Margin * 2.0 * std::ldexp(1.0, -24) / (1.0 - c);
        k_set_stop<<<1, 1, 0, s>>>(ctl, std::max(eps, handover), kApullF32Stall);
        if (algo == PR_IFP2) PR_TRY((run_apull<float, true>(g, W, use_graph, prof)));
        else PR_TRY((run_apull<float, false>(g, W, use_graph, prof)));
        PR_TRY(apull_launches());
        const int32_t r32_rounds = W.hctl->round;
        double *x64 = W.s64.x.as<double>(), *r64 = W.s64.r.as<double>();
        k_init_state<double><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, x64, r64);
        k_apull_to_fp64<<<gn, kThreads, 0, s>>>(G, ctl, W.s32.x.as<float>(), x64, W.s64.w[0].as<double>(), pv);
        k_set_stop<<<1, 1, 0, s>>>(ctl, eps, 0);
        if (algo == PR_IFP2) PR_TRY((run_apull<double, true>(g, W, use_graph, prof, false)));
        else PR_TRY((run_apull<double, false>(g, W, use_graph, prof, false)));
        PR_TRY(apull_launches(r32_rounds));
        fp64_rounds = W.hctl->round - r32_rounds;
        if (algo == PR_IFP1) {
            apull_final_residual<double>(g, W);
            launches += 1;
        }
        finish_ifp<double>(g, W, algo, dout, launches);
        launches += 5;  // the two inits, the conversion, the two stop settings
    } else if (apull) {  // double-float
        PR_CK(cudaMemsetAsync(W.sdf.din.p, 0, sizeof(double) * G.n, s));
        k_init_state<float2><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.sdf.x.as<float2>(), W.sdf.r.as<float2>());
        if (algo == PR_IFP2) PR_TRY((run_apull<float2, true>(g, W, use_graph, prof)));
        else PR_TRY((run_apull<float2, false>(g, W, use_graph, prof)));
        PR_TRY(apull_launches());
        if (algo == PR_IFP1) {
            apull_final_residual<float2>(g, W);
            launches += 1;
        }
        finish_ifp<float2>(g, W, algo, dout, launches);
        launches += 1;
    } else if (prec == PR_FP64) {
        k_init_state<double><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.s64.x.as<double>(), W.s64.r.as<double>());
        PR_TRY(ifp_phase1<double>(g, W, algo, use_graph, levels, prof));
        PR_TRY(count_rounds(0));
        finish_ifp<double>(g, W, algo, dout, launches);
        launches += 1;
    } else if (prec == PR_DF64) {
        PR_CK(cudaMemsetAsync(W.sdf.din.p, 0, sizeof(double) * G.n, s));
        k_init_state<float2><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.sdf.x.as<float2>(), W.sdf.r.as<float2>());
        PR_TRY(ifp_phase1<float2>(g, W, algo, use_graph, levels, prof));
        PR_TRY(count_rounds(0));
        if (algo == PR_IFP1 && G.n > G.n_nd) {  // pushes into dangling rows still in the inbox
            k_fold_inbox<<<gn, kThreads, 0, s>>>(W.sdf.r.as<float2>(), W.sdf.din.as<double>(), G.n_nd, G.n);
            launches += 1;
        }
        finish_ifp<float2>(g, W, algo, dout, launches);
        launches += 1;
    } else {  // FP32 rounds, then the IEEE FP64 correction sweep and FP64 rounds to the end
        k_init_state<float><<<gn, kThreads, 0, s>>>(G.n, ctl, pv, W.s32.x.as<float>(), W.s32.r.as<float>());
        PR_TRY(ifp_phase1<float>(g, W, algo, use_graph, levels, prof));
        PR_TRY(count_rounds(0));
        const int32_t r32_rounds = W.hctl->round;
        double *x64 = W.s64.x.as<double>(), *r64 = W.s64.r.as<double>();
        k_to_fp64<<<gn, kThreads, 0, s>>>(G, ctl, W.s32.x.as<float>(), x64, r64, W.s64.q.as<double>(), pv,
                                          algo == PR_IFP2);
        SweepArgs<double> a{};
        a.val = W.s64.q.as<double>();
        a.r = r64;
        a.x = x64;
        a.pv = pv;
        const Plan &PL = algo == PR_IFP2 ? plan_nd_of<double>(g) : plan_all_of<double>(g);
        k_reset_run<<<1, 1, 0, s>>>(ctl);
        k_sweep<double, OP_CORRECT><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
        PR_TRY(ifp_phase1<double>(g, W, algo, use_graph, levels, prof));
        PR_TRY(count_rounds(r32_rounds));
        fp64_rounds = W.hctl->round - r32_rounds;
        finish_ifp<double>(g, W, algo, dout, launches);
        launches += 4;  // init, to FP64, reset, correction sweep
    }
    PR_CK(cudaEventRecord(e1, s));
    if (!out_is_device) PR_CK(cudaMemcpyAsync(out, dout, sizeof(double) * G.n, cudaMemcpyDeviceToHost, s));
    PR_CK(cudaMemcpyAsync(W.hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaStreamSynchronize(s));
    PR_CK(cudaGetLastError());
    float ms = 0;
    PR_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const Ctl &hc = *W.hctl;
    if (opt.trace_cap > 0) {
        const int32_t nrec = std::min<int32_t>(opt.trace_cap, W.trace_len);
        if (opt.trace_R) PR_CK(cudaMemcpy(opt.trace_R, W.tR.p, sizeof(double) * nrec, cudaMemcpyDeviceToHost));
        if (opt.trace_F) PR_CK(cudaMemcpy(opt.trace_F, W.tF.p, sizeof(long long) * nrec, cudaMemcpyDeviceToHost));
        if (opt.trace_E) PR_CK(cudaMemcpy(opt.trace_E, W.tE.p, sizeof(long long) * nrec, cudaMemcpyDeviceToHost));
        if (opt.trace_mode) PR_CK(cudaMemcpy(opt.trace_mode, W.tM.p, nrec, cudaMemcpyDeviceToHost));
    }
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->ms = ms;
        st->p_scale = p_scale;
        st->launches = launches;
        if (algo == PR_POWER) {
            st->rounds = hc.iter;
            st->resid_l1 = hc.delta;
            st->err_bound = c * hc.delta / (1.0 - c);
            st->edges_scanned = (int64_t)hc.iter * G.m;
        } else {
            st->rounds = hc.round;
            st->rounds_push = hc.rounds_push;
            st->rounds_pull = hc.rounds_pull;
            st->fp64_rounds = fp64_rounds;
            st->pushes = hc.pushes;
            st->edges_pushed = hc.edges_pushed + (algo == PR_IFP2 ? g->info.m_d : 0);
            st->edges_scanned = hc.edges_scanned + (algo == PR_IFP2 ? g->info.m_d : 0);
            st->resid_l1 = hc.R;
            st->dangling_mass = algo == PR_IFP1 ? hc.D : 0.0;
            st->err_bound = (algo == PR_IFP1 ? 2.0 * c * hc.R : 2.0 * hc.R) / (1.0 - c);
        }
    }
    if (hc.status == 1) return fail(PR_ENOTCONV, "round/iteration cap reached before the stopping test held");
    if (hc.status == 2) return fail(PR_ENOTCONV, "no vertex above xi_act while the residual is above eps");
    return PR_OK;
}

// ------------------------------------------------------------ debug record (host)
// The records of the translation units are collected after every single and
// batched solve into one report; pr_debug_inject names a site that the next
// solves force to fail (a test of the net itself, with no invalid access).
static std::mutex g_dbg_mu;
static pr_debug_report g_dbg_acc{};
static int g_dbg_inject = 0;

#ifdef PR_DEBUG
static void dbg_merge(const DbgRec &d) {
    g_dbg_acc.checks += (int64_t)d.checks;
    if (d.fails && !g_dbg_acc.fails) {
        g_dbg_acc.first_site = d.site;
        g_dbg_acc.first_value = d.value;
        g_dbg_acc.first_bound = d.bound;
    }
    g_dbg_acc.fails += (int64_t)d.fails;
    g_dbg_acc.max_mass_dev = std::max(g_dbg_acc.max_mass_dev, d.max_mass_dev);
    g_dbg_acc.max_identity_dev = std::max(g_dbg_acc.max_identity_dev, d.max_identity_dev);
}
#endif

int dbg_injected() {
    std::lock_guard<std::mutex> lock(g_dbg_mu);
    return g_dbg_inject;
}

void dbg_begin(cudaStream_t s) {
#ifdef PR_DEBUG
    cudaStreamSynchronize(s);
    std::lock_guard<std::mutex> lock(g_dbg_mu);
    dbg_reset_solve(g_dbg_inject);
    dbg_reset_batch(g_dbg_inject);
    dbg_reset_group(g_dbg_inject);
#else
    (void)s;
#endif
}

pr_status dbg_end(cudaStream_t s, const char *what, pr_status st) {
#ifdef PR_DEBUG
    cudaStreamSynchronize(s);
    DbgRec a{}, b{}, c{};
    std::lock_guard<std::mutex> lock(g_dbg_mu);
    dbg_read_solve(&a);
    dbg_read_batch(&b);
    dbg_read_group(&c);
    dbg_merge(a);
    dbg_merge(b);
    dbg_merge(c);
    const unsigned long long fails = a.fails + b.fails + c.fails;
    if (fails) {
        const DbgRec &f = a.fails ? a : (b.fails ? b : c);
        return fail(PR_ECHECK, std::string(what) + ": debug check failed at site " + std::to_string(f.site) +
                                   " (value " + std::to_string(f.value) + ", bound " + std::to_string(f.bound) +
                                   "; " + std::to_string(fails) + " failures)");
    }
#else
    (void)s;
    (void)what;
#endif
    return st;
}

}  // namespace pr

using namespace pr;

extern "C" int pr_is_debug_build(void) {
#ifdef PR_DEBUG
    return 1;
#else
    return 0;
#endif
}

extern "C" pr_status pr_debug_report_get(pr_debug_report *out, int reset) {
    if (!out) return fail(PR_EINVAL, "pr_debug_report_get: out is NULL");
    if (!pr_is_debug_build()) return fail(PR_EINVAL, "pr_debug_report_get: not a debug build (PR_DEBUG)");
    std::lock_guard<std::mutex> lock(g_dbg_mu);
    *out = g_dbg_acc;
    if (reset) g_dbg_acc = pr_debug_report{};
    return PR_OK;
}

extern "C" pr_status pr_debug_inject(int32_t site) {
    if (!pr_is_debug_build()) return fail(PR_EINVAL, "pr_debug_inject: not a debug build (PR_DEBUG)");
    if (site < 0) return fail(PR_EINVAL, "pr_debug_inject: site must be >= 0");
    std::lock_guard<std::mutex> lock(g_dbg_mu);
    g_dbg_inject = site;
    return PR_OK;
}

extern "C" pr_status pr_solve_ex(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                                 const pr_opts *opts, double *out, int out_is_device, pr_stats *st) {
    if (!g) return fail(PR_EINVAL, "graph is NULL");
    dbg_begin(g->stream);
    pr_status s = solve_impl(g, c, eps, a, prec, p, opts, out, out_is_device, st);
    if (s == PR_ECUDA) {
        cudaStreamSynchronize(g->stream);
        cudaGetLastError();
    }
    if (s == PR_OK || s == PR_ENOTCONV) s = dbg_end(g->stream, "pr_solve", s);
    return s;
}

extern "C" pr_status pr_solve(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                              double *out, int out_is_device, pr_stats *st) {
    return pr_solve_ex(g, c, eps, a, prec, p, nullptr, out, out_is_device, st);
}
