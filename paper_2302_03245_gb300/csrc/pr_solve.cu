// pr_solve.cu -- the IFP1 / IFP2 round loop (Alg. 2, Alg. 3), the IFP2
// phase-2 pull, the FP64 correction sweep of the FP32 form, the Power-method
// baseline (Sec. 4), normalisation, and pr_solve / pr_solve_ex.
//
// Round semantics (synchronous snapshot rounds; Sec. 3.3.1 counts one
// "iteration" as one scan over all vertices), with a (1-c) reserve, which
// does not change the normalised result (Sec. 3.1 after Eq. 4):
//
//   R_t = sum_{i non-dangling} |r_i|            stop when R_t <= eps
//   F_t = { i non-dangling : |r_i| > xi_act }   snapshot before any push
//   i in F_t:  x_i += (1-c) r_i,  r_i = 0,  w_i = c r_i / deg(i)
//   j:         r_j += sum_{i in S(j) & F_t} w_i  (IFP2: non-dangling j only)
//
// One round is four kernels on one stream:
//   k_activate  reads r, computes R_t, |F_t|, edges, the dense w and (when a
//               sparse round is expected) the frontier bins; its last block
//               takes the stop decision and the push/pull choice.
//   k_commit    push rounds only: x_i += (1-c) r_i, r_i = 0 over the frontier.
//   k_push      push rounds only: atomicAdd of w_i along the out-list prefix
//               (all targets for IFP1, the non-dangling prefix for IFP2).
//   k_rows      pull rounds only: each row j commits its own activation
//               (the same |r_j| > xi_act test on the same r_j) and gathers w
//               over its in-list; deterministic.
// Nothing in a round runs on the host: the stop flag lives in device memory,
// every kernel returns at once when it is set, and the rounds are replayed
// inside a CUDA graph whose while-node re-reads the flag.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pr_internal.cuh"

namespace pr {

enum { MODE_PUSH = 1, MODE_PULL = 2 };
enum { OP_ROUND = 0, OP_POWER = 1, OP_CORRECT = 2, OP_PHASE2 = 3 };

struct Ctl {
    // parameters (host-written per solve)
    double c, one_minus_c, eps, xi, pull_edges, pu;
    int32_t algo, policy, max_rounds, p_dense;
    int64_t scan_ref, scan_unref;  // in-list entries read by one pull round
    int32_t trace_cap, pad0;
    // evolving state (device-written)
    int32_t round, cur, done, status, mode, bins_ok, want_bins, unref_active;
    uint32_t ticket, pad1;
    uint32_t bin_cnt[2][3];
    double R, D;
    long long F, E;
    long long pushes, edges_pushed, edges_scanned;
    int32_t rounds_push, rounds_pull;
    // power / finalize
    double gamma, delta, zsum;
    int32_t iter, pad2;
};

struct Partials {
    double *a, *b, *c;   // [kMaxBlocks] each
    long long *F, *E;    // [kMaxBlocks]
    int *u;              // [kMaxBlocks]
};

struct Trace {
    double *R;
    long long *F, *E;
    int8_t *mode;
};

// CUDA-event timing of individual launches (opts.profile): events are
// recorded on the graph's stream around each kernel; a launch is charged to
// its kind only if its round actually used it (decided after the fact from
// the device trace).
struct Prof {
    pr_kernel_profile *out = nullptr;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int kind, round;
        size_t e0, e1;
    };
    std::vector<Rec> recs;
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
    void add(int kind, int round, size_t e0, size_t e1) { recs.push_back({kind, round, e0, e1}); }
    // charge the recorded launches (after a synchronize); keep(kind, round) says which did work
    template <typename F> void settle(F keep) {
        for (const Rec &r : recs) {
            if (!keep(r.kind, r.round)) continue;
            float ms = 0;
            cudaEventElapsedTime(&ms, pool[r.e0], pool[r.e1]);
            out->launches[r.kind]++;
            out->ms[r.kind] += ms;
        }
        recs.clear();
        used = 0;
    }
    ~Prof() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// ------------------------------------------------------------ helpers
template <typename T> __device__ __forceinline__ T inv_deg(const DevGraph &G, int i);
template <> __device__ __forceinline__ double inv_deg<double>(const DevGraph &G, int i) {
    return G.inv_deg64[i];
}
template <> __device__ __forceinline__ float inv_deg<float>(const DevGraph &G, int i) {
    return G.inv_deg32[i];
}

// |r_i| > xi_act, evaluated identically wherever an activation is decided
template <typename T> __device__ __forceinline__ bool is_active(T v, double xi) {
    return (double)(v < T(0) ? -v : v) > xi;
}

__device__ __forceinline__ double pval(const Ctl *ctl, const double *p64, int j) {
    return ctl->p_dense ? p64[j] : ctl->pu;
}

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum (fixed tree: deterministic); result valid in thread 0
template <typename V> __device__ __forceinline__ V block_sum(V v, V *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    V r = V(0);
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : V(0);
        r = warp_sum(r);
    }
    return r;
}

// last-block election: every block calls with its partials already stored
__device__ __forceinline__ bool last_block(uint32_t *ticket) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// ------------------------------------------------------------ init
template <typename T>
__global__ void k_init_state(int32_t n, const Ctl *ctl, const double *p64, T *x, T *r) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] = T(0);
        r[i] = (T)pval(ctl, p64, i);
    }
}

// dense p in caller ids -> internal ids, scaled
__global__ void k_p_dense(int32_t n, const int32_t *inv, const double *val, double scale, double *p64) {
    int stride = gridDim.x * blockDim.x;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) p64[inv[e]] = val[e] * scale;
}

__global__ void k_p_sparse(int32_t nnz, const int32_t *inv, const int32_t *idx, const double *val,
                           double scale, double *p64) {
    int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
        atomicAdd(&p64[inv[idx[k]]], val[k] * scale);
}

// device-resident p: count bad entries and sum (for validation)
__global__ void k_p_check(int32_t cnt, int32_t n, const int32_t *idx, const double *val,
                          unsigned long long *bad, double *sum) {
    __shared__ double sh[32];
    double s = 0;
    unsigned long long b = 0;
    int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += stride) {
        double v = val[k];
        if (!(v >= 0.0) || !isfinite(v)) b++;
        else s += v;
        if (idx && (idx[k] < 0 || idx[k] >= n)) b++;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(sum, s);
    if (b) atomicAdd(bad, b);
}

__global__ void k_reset_run(Ctl *ctl) {
    ctl->done = 0;
    ctl->status = 0;
    ctl->ticket = 0;
    ctl->bin_cnt[0][0] = ctl->bin_cnt[0][1] = ctl->bin_cnt[0][2] = 0;
    ctl->bin_cnt[1][0] = ctl->bin_cnt[1][1] = ctl->bin_cnt[1][2] = 0;
    ctl->want_bins = ctl->policy != MODE_PULL;
    ctl->unref_active = 1;
}

__global__ void k_set_while(const Ctl *ctl, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
}

// ------------------------------------------------------------ activate
// Reads r over non-dangling vertices: R_t, |F_t|, edges, dense w, bins.
template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_activate(DevGraph G, Ctl *ctl, Partials P, const T *r,
                                                      T *w, int32_t *bins, Trace tr) {
    if (ctl->done) return;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    const double xi = ctl->xi;
    const T cT = (T)ctl->c;
    const int want = ctl->want_bins;
    const int t = ctl->round;
    uint32_t *bcnt = ctl->bin_cnt[t & 1];
    const int n_nd = G.n_nd;
    const int lane = threadIdx.x & 31;
    double Rl = 0;
    long long Fl = 0, El = 0;
    int ul = 0;
    for (int base = blockIdx.x * blockDim.x; base < n_nd; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        bool act = false;
        int pd = 0;
        if (i < n_nd) {
            const T v = r[i];
            Rl += (double)(v < T(0) ? -v : v);
            act = is_active(v, xi);
            pd = IFP2 ? G.ndeg[i] : (G.out_off[i + 1] - G.out_off[i]);
            w[i] = act ? v * (cT * inv_deg<T>(G, i)) : T(0);
            if (act) {
                Fl++;
                El += pd;
                ul |= (i >= G.n_ref);
            }
        }
        if (want) {  // warp-aggregated append into the three degree bins
            const int bin = pd <= kWarpRowMin ? 0 : (pd <= kCtaRowMin ? 1 : 2);
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const unsigned mask = __ballot_sync(0xffffffffu, act && bin == b);
                if (!mask) continue;
                unsigned pos0 = 0;
                const int leader = __ffs(mask) - 1;
                if (lane == leader) pos0 = atomicAdd(&bcnt[b], (unsigned)__popc(mask));
                pos0 = __shfl_sync(0xffffffffu, pos0, leader);
                if (act && bin == b)
                    bins[(size_t)b * n_nd + pos0 + __popc(mask & ((1u << lane) - 1u))] = i;
            }
        }
    }
    const double Rb = block_sum(Rl, shd);
    const long long Fb = block_sum(Fl, shl);
    const long long Eb = block_sum(El, shl);
    const int ub = __syncthreads_or(ul);
    if (threadIdx.x == 0) {
        P.a[blockIdx.x] = Rb;
        P.F[blockIdx.x] = Fb;
        P.E[blockIdx.x] = Eb;
        P.u[blockIdx.x] = ub;
    }
    if (!last_block(&ctl->ticket)) return;
    // deterministic final reduction over the block partials
    double R = 0;
    long long F = 0, E = 0;
    int u = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        R += __ldcg(&P.a[k]);
        F += __ldcg(&P.F[k]);
        E += __ldcg(&P.E[k]);
        u |= __ldcg(&P.u[k]);
    }
    R = block_sum(R, shd);
    F = block_sum(F, shl);
    E = block_sum(E, shl);
    u = __syncthreads_or(u);
    if (threadIdx.x != 0) return;
    ctl->ticket = 0;
    ctl->R = R;
    ctl->F = F;
    ctl->E = E;
    if (t < ctl->trace_cap) tr.R[t] = R;
    uint32_t *nxt = ctl->bin_cnt[(t + 1) & 1];
    nxt[0] = nxt[1] = nxt[2] = 0;
    if (R <= ctl->eps) {
        ctl->done = 1;
        ctl->status = 0;
        return;
    }
    if (t >= ctl->max_rounds) {
        ctl->done = 1;
        ctl->status = 1;
        return;
    }
    if (F == 0) {
        ctl->done = 1;
        ctl->status = 2;
        return;
    }
    int mode;
    if (ctl->policy == MODE_PUSH) mode = MODE_PUSH;
    else if (ctl->policy == MODE_PULL) mode = MODE_PULL;
    else mode = (want && (double)E < ctl->pull_edges) ? MODE_PUSH : MODE_PULL;
    ctl->mode = mode;
    ctl->cur = t;
    ctl->round = t + 1;
    ctl->unref_active = u;
    ctl->pushes += F;
    ctl->edges_pushed += E;
    if (mode == MODE_PULL) {
        ctl->edges_scanned += ctl->scan_ref + (u ? ctl->scan_unref : 0);
        ctl->rounds_pull++;
    } else {
        ctl->edges_scanned += E;
        ctl->rounds_push++;
    }
    if (t < ctl->trace_cap) {
        tr.F[t] = F;
        tr.E[t] = E;
        tr.mode[t] = (int8_t)mode;
    }
    if (ctl->policy == 0) ctl->want_bins = (double)E < 2.0 * ctl->pull_edges;
}

// ------------------------------------------------------------ push rounds
template <typename T>
__global__ void k_commit(const Ctl *ctl, const int32_t *bins, int32_t n_nd, T *x, T *r) {
    if (ctl->done || ctl->mode != MODE_PUSH) return;
    const uint32_t *cnt = ctl->bin_cnt[ctl->cur & 1];
    const uint32_t c0 = cnt[0], c1 = cnt[1], c2 = cnt[2];
    const uint32_t total = c0 + c1 + c2;
    const T om = (T)ctl->one_minus_c;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        int i;
        if (k < c0) i = bins[k];
        else if (k < c0 + c1) i = bins[(size_t)n_nd + (k - c0)];
        else i = bins[(size_t)2 * n_nd + (k - c0 - c1)];
        const T v = r[i];
        x[i] += om * v;
        r[i] = T(0);
    }
}

template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_push(DevGraph G, const Ctl *ctl, const int32_t *bins,
                                                  const T *w, T *r, int nb_thread, int nb_warp) {
    if (ctl->done || ctl->mode != MODE_PUSH) return;
    const uint32_t *cnt = ctl->bin_cnt[ctl->cur & 1];
    const int n_nd = G.n_nd;
    const int b = blockIdx.x;
    if (b < nb_thread) {
        const uint32_t c0 = cnt[0];
        for (uint32_t k = b * blockDim.x + threadIdx.x; k < c0; k += nb_thread * blockDim.x) {
            const int i = bins[k];
            const T wi = w[i];
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            for (int e = e0; e < e1; e++) atomicAdd(&r[G.out_dst[e]], wi);
        }
    } else if (b < nb_thread + nb_warp) {
        const uint32_t c1 = cnt[1];
        const int lane = threadIdx.x & 31;
        const int wpb = blockDim.x >> 5;
        for (uint32_t k = (b - nb_thread) * wpb + (threadIdx.x >> 5); k < c1; k += nb_warp * wpb) {
            const int i = bins[(size_t)n_nd + k];
            const T wi = w[i];
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            for (int e = e0 + lane; e < e1; e += 32) atomicAdd(&r[G.out_dst[e]], wi);
        }
    } else {
        const uint32_t c2 = cnt[2];
        const int nb_cta = gridDim.x - nb_thread - nb_warp;
        for (uint32_t k = b - nb_thread - nb_warp; k < c2; k += nb_cta) {
            const int i = bins[(size_t)2 * n_nd + k];
            const T wi = w[i];
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&r[G.out_dst[e]], wi);
        }
    }
}

// ------------------------------------------------------------ row kernels
template <typename T> struct RowArgs {
    const T *val;        // gathered per source
    T *r;                // ROUND / CORRECT / PHASE2 output residual
    T *x;                // ROUND reserve; CORRECT reads x
    const T *pi_cur;     // POWER
    T *pi_next, *q_next; // POWER
    const double *p64;
    Partials P;
    Trace tr;
};

// sum of val[src[e]] over e in [off[j] + start, off[j+1]) stepping by `step`;
// in-list entries are streamed once (evict-first), gathered values go through
// the read-only cache (they are not written during the kernel)
template <typename T>
__device__ __forceinline__ T row_sum(const int32_t *__restrict__ off, const int32_t *__restrict__ src, int j,
                                     const T *__restrict__ val, int start, int step) {
    const int a = __ldg(&off[j]), b = __ldg(&off[j + 1]);
    T acc0 = T(0), acc1 = T(0);
    int e = a + start;
    for (; e + step < b; e += 2 * step) {
        acc0 += __ldg(&val[__ldcs(&src[e])]);
        acc1 += __ldg(&val[__ldcs(&src[e + step])]);
    }
    if (e < b) acc0 += __ldg(&val[__ldcs(&src[e])]);
    return acc0 + acc1;
}

template <typename T, int OP>
__device__ __forceinline__ void row_epilogue(const DevGraph &G, const Ctl *ctl, RowArgs<T> &a, int j,
                                             T acc, double &s1, double &s2, double &s3) {
    if (OP == OP_ROUND) {
        T base;
        if (j < G.n_nd) {
            const T v = a.r[j];
            if (is_active(v, ctl->xi)) {
                a.x[j] += (T)ctl->one_minus_c * v;
                base = T(0);
            } else {
                base = v;
            }
        } else {
            base = a.r[j];
        }
        a.r[j] = base + acc;
    } else if (OP == OP_POWER) {
        const T y = (T)ctl->c * acc + (T)(ctl->gamma * pval(ctl, a.p64, j));
        const T old = a.pi_cur[j];
        s1 += fabs((double)y - (double)old);
        if (j >= G.n_nd) s2 += (double)y;
        s3 += (double)y;
        a.pi_next[j] = y;
        a.q_next[j] = j < G.n_nd ? y * inv_deg<T>(G, j) : T(0);
    } else if (OP == OP_CORRECT) {
        // r = p + c P~ s - s with s = x / (1-c)   (exact residual of the current reserve)
        const double s = (double)a.x[j] / ctl->one_minus_c;
        a.r[j] = (T)(pval(ctl, a.p64, j) + ctl->c * (double)acc - s);
    } else {  // OP_PHASE2: r_d = p_d + c sum_{u in S(d)} x_u / ((1-c) deg(u))
        a.r[j] = (T)(pval(ctl, a.p64, j) + ctl->c * (double)acc);
    }
}

// rows of a segment handled by groups of LANES threads; the loop bound is
// uniform across the block so the width-LANES shuffles always see full warps
template <typename T, int OP, int LANES>
__device__ __forceinline__ void rows_lanes(const DevGraph &G, const Seg &S, int lb, Ctl *ctl, RowArgs<T> &a,
                                           bool use_unref, double &s1, double &s2, double &s3) {
    constexpr int GPB = kThreads / LANES;
    const int grp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    for (int base = S.lo + lb * GPB; base < S.hi; base += S.nblk * GPB) {
        const int j = base + grp;
        T acc = T(0);
        if (j < S.hi) {
            acc = row_sum<T>(G.inr_off, G.inr_src, j, a.val, lane, LANES);
            if (use_unref) acc += row_sum<T>(G.inu_off, G.inu_src, j, a.val, lane, LANES);
        }
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LANES);
        if (j < S.hi && lane == 0) row_epilogue<T, OP>(G, ctl, a, j, acc, s1, s2, s3);
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) k_rows(DevGraph G, Plan PL, Ctl *ctl, RowArgs<T> a) {
    // the loop kernels stop with the device flag; the one-shot sweeps
    // (FP64 correction, IFP2 phase 2) run after the flag is set
    if ((OP == OP_ROUND || OP == OP_POWER) && ctl->done) return;
    if (OP == OP_ROUND && ctl->mode != MODE_PULL) return;
    const bool use_unref = (OP == OP_ROUND) ? (ctl->unref_active != 0) : true;
    int s = 0;
    while (s + 1 < PL.nseg && (int)blockIdx.x >= PL.seg[s + 1].blk0) s++;
    const Seg S = PL.seg[s];
    const int lb = blockIdx.x - S.blk0;
    double s1 = 0, s2 = 0, s3 = 0;
    __shared__ double shd[32];
    __shared__ T sht[32];
    switch (S.lanes) {
        case 1: rows_lanes<T, OP, 1>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        case 2: rows_lanes<T, OP, 2>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        case 4: rows_lanes<T, OP, 4>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        case 8: rows_lanes<T, OP, 8>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        case 16: rows_lanes<T, OP, 16>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        case 32: rows_lanes<T, OP, 32>(G, S, lb, ctl, a, use_unref, s1, s2, s3); break;
        default:
            for (int j = S.lo + lb; j < S.hi; j += S.nblk) {
                T acc = row_sum<T>(G.inr_off, G.inr_src, j, a.val, threadIdx.x, blockDim.x);
                if (use_unref) acc += row_sum<T>(G.inu_off, G.inu_src, j, a.val, threadIdx.x, blockDim.x);
                acc = block_sum(acc, sht);
                if (threadIdx.x == 0) row_epilogue<T, OP>(G, ctl, a, j, acc, s1, s2, s3);
            }
    }
    if (OP != OP_POWER) return;
    // Power: ||pi_{k+1} - pi_k||_1, d^T pi_{k+1}, e^T pi_{k+1}
    const double b1 = block_sum(s1, shd);
    const double b2 = block_sum(s2, shd);
    const double b3 = block_sum(s3, shd);
    if (threadIdx.x == 0) {
        a.P.a[blockIdx.x] = b1;
        a.P.b[blockIdx.x] = b2;
        a.P.c[blockIdx.x] = b3;
    }
    if (!last_block(&ctl->ticket)) return;
    double d = 0, dm = 0, tm = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        d += __ldcg(&a.P.a[k]);
        dm += __ldcg(&a.P.b[k]);
        tm += __ldcg(&a.P.c[k]);
    }
    d = block_sum(d, shd);
    dm = block_sum(dm, shd);
    tm = block_sum(tm, shd);
    if (threadIdx.x != 0) return;
    ctl->ticket = 0;
    const int it = ctl->iter + 1;
    ctl->iter = it;
    ctl->delta = d;
    ctl->zsum = tm;
    ctl->gamma = ctl->c * dm + ctl->one_minus_c * tm;  // Eq. 1: c d^T pi + (1-c) e^T pi
    if (it < ctl->trace_cap) a.tr.R[it] = d;
    if (d <= ctl->eps) {
        ctl->done = 1;
        ctl->status = 0;
    } else if (it >= ctl->max_rounds) {
        ctl->done = 1;
        ctl->status = 1;
    }
}

// Power iteration start: pi_0 = p, q_0 = pi_0 / deg, gamma_0 from d^T p and e^T p.
template <typename T>
__global__ void k_power_init(DevGraph G, Ctl *ctl, Partials P, const double *p64, T *pi, T *q) {
    __shared__ double shd[32];
    double dm = 0, tm = 0;
    const int n = G.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T v = (T)pval(ctl, p64, i);
        pi[i] = v;
        q[i] = i < G.n_nd ? v * inv_deg<T>(G, i) : T(0);
        if (i >= G.n_nd) dm += (double)v;
        tm += (double)v;
    }
    const double b2 = block_sum(dm, shd), b3 = block_sum(tm, shd);
    if (threadIdx.x == 0) {
        P.b[blockIdx.x] = b2;
        P.c[blockIdx.x] = b3;
    }
    if (!last_block(&ctl->ticket)) return;
    dm = 0;
    tm = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        dm += __ldcg(&P.b[k]);
        tm += __ldcg(&P.c[k]);
    }
    dm = block_sum(dm, shd);
    tm = block_sum(tm, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->gamma = ctl->c * dm + ctl->one_minus_c * tm;
        ctl->iter = 0;
        ctl->zsum = tm;
    }
}

// ------------------------------------------------------------ FP32 -> FP64
// x64 = x32; q64_u = x64_u / ((1-c) deg(u)); IFP2: r64_d = p_d (dangling untouched in phase 1)
template <typename T>
__global__ void k_to64(DevGraph G, const Ctl *ctl, const T *x32, double *x64, double *r64, double *q64,
                       const double *p64, int ifp2) {
    const int n = G.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double xv = (double)x32[i];
        x64[i] = xv;
        if (i < G.n_nd) q64[i] = xv / ctl->one_minus_c * G.inv_deg64[i];
        else if (ifp2) r64[i] = pval(ctl, p64, i);
    }
}

// q64_u = x_u / ((1-c) deg(u)) for the IFP2 phase-2 pull
__global__ void k_phase2_q(DevGraph G, const Ctl *ctl, const double *x64, double *q64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n_nd; i += gridDim.x * blockDim.x)
        q64[i] = x64[i] / ctl->one_minus_c * G.inv_deg64[i];
}

// ------------------------------------------------------------ finalize
// IFP1: z = x + (1-c) r (Alg. 2 pibar + h);  IFP2: z = x (non-dangling), (1-c) r (dangling)
// (Alg. 3 pibar);  POWER: z = pi.  pi = z / sum z, scattered back to caller ids.
template <typename T>
__device__ __forceinline__ double zval(const DevGraph &G, const Ctl *ctl, int kind, const T *x, const T *r,
                                       int i) {
    if (kind == PR_IFP1) return (double)x[i] + ctl->one_minus_c * (double)r[i];
    if (kind == PR_IFP2) return i < G.n_nd ? (double)x[i] : ctl->one_minus_c * (double)r[i];
    return (double)x[i];
}

template <typename T>
__global__ void k_fin_sum(DevGraph G, Ctl *ctl, Partials P, int kind, const T *x, const T *r) {
    __shared__ double shd[32];
    double s = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x)
        s += zval(G, ctl, kind, x, r, i);
    s = block_sum(s, shd);
    if (threadIdx.x == 0) P.a[blockIdx.x] = s;
    if (!last_block(&ctl->ticket)) return;
    s = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) s += __ldcg(&P.a[k]);
    s = block_sum(s, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->zsum = s;
    }
}

// dangling residual mass (IFP1 report)
__global__ void k_dangling_mass(DevGraph G, Ctl *ctl, Partials P, const double *r) {
    __shared__ double shd[32];
    double s = 0;
    for (int i = G.n_nd + blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x)
        s += r[i];
    s = block_sum(s, shd);
    if (threadIdx.x == 0) P.b[blockIdx.x] = s;
    if (!last_block(&ctl->ticket)) return;
    s = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) s += __ldcg(&P.b[k]);
    s = block_sum(s, shd);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->D = s;
    }
}

template <typename T>
__global__ void k_fin_write(DevGraph G, const Ctl *ctl, int kind, const T *x, const T *r, double *out) {
    const double inv = 1.0 / ctl->zsum;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += gridDim.x * blockDim.x)
        out[G.perm[i]] = zval(G, ctl, kind, x, r, i) * inv;
}

// ------------------------------------------------------------ workspace
struct Workspace {
    Buf ctl, part, p64, x64, r64, w64, w64b, x32, r32, w32, w32b, bins, tR, tF, tE, tM, outbuf, pstage,
        pstage2;
    Ctl *hctl = nullptr;  // pinned host mirror
    int32_t trace_len = 0;
    cudaStream_t cap_stream = nullptr;
    // cached CUDA graphs of the round loop, per (precision, algo, policy)
    struct G {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int key = -1;
    } graphs[12];
    ~Workspace() {
        for (auto &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
        }
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

static pr_status ensure_ws(pr_graph *g, bool fp32, int32_t trace_len) {
    cudaStream_t s = g->stream;
    if (!g->ws) {
        Workspace *W = new (std::nothrow) Workspace();
        if (!W) return fail(PR_ENOMEM, "host allocation failed");
        g->ws = W;
        const size_t n = (size_t)g->G.n, nnd = (size_t)std::max(g->G.n_nd, 1);
        PR_TRY(W->ctl.alloc(sizeof(Ctl), s));
        PR_TRY(W->part.alloc(sizeof(double) * kMaxBlocks * 6, s));
        PR_TRY(W->p64.alloc(sizeof(double) * n, s));
        PR_TRY(W->x64.alloc(sizeof(double) * n, s));
        PR_TRY(W->r64.alloc(sizeof(double) * n, s));
        PR_TRY(W->w64.alloc(sizeof(double) * n, s));
        PR_TRY(W->w64b.alloc(sizeof(double) * n, s));
        PR_TRY(W->bins.alloc(sizeof(int32_t) * 3 * nnd, s));
        PR_TRY(W->outbuf.alloc(sizeof(double) * n, s));
        PR_CK(cudaMallocHost(&W->hctl, sizeof(Ctl)));
        PR_CK(cudaMemsetAsync(W->ctl.p, 0, sizeof(Ctl), s));
        PR_CK(cudaMemsetAsync(W->part.p, 0, W->part.bytes, s));
    }
    Workspace &W = *static_cast<Workspace *>(g->ws);
    if (fp32 && !W.x32.p) {
        const size_t n = (size_t)g->G.n;
        PR_TRY(W.x32.alloc(sizeof(float) * n, s));
        PR_TRY(W.r32.alloc(sizeof(float) * n, s));
        PR_TRY(W.w32.alloc(sizeof(float) * n, s));
        PR_TRY(W.w32b.alloc(sizeof(float) * n, s));
    }
    if (trace_len > W.trace_len) {
        // traces change device pointers: drop cached graphs
        for (auto &cg : W.graphs) {
            if (cg.exec) cudaGraphExecDestroy(cg.exec);
            if (cg.graph) cudaGraphDestroy(cg.graph);
            cg = Workspace::G{};
        }
        PR_TRY(W.tR.alloc(sizeof(double) * trace_len, s));
        PR_TRY(W.tF.alloc(sizeof(long long) * trace_len, s));
        PR_TRY(W.tE.alloc(sizeof(long long) * trace_len, s));
        PR_TRY(W.tM.alloc(sizeof(int8_t) * trace_len, s));
        W.trace_len = trace_len;
    }
    return PR_OK;
}

static int grid_n(int64_t items, int sms, int per_sm = 8) {
    int64_t b = (items + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * per_sm));
}

// ------------------------------------------------------------ round launch
struct RoundBufs {
    void *x, *r, *w;
};

// one round = 4 launches (activate, commit, push, pull)
constexpr int kRoundLaunches = 4;
constexpr int kUnroll = 4;  // rounds per while-loop body

template <typename T, bool IFP2>
static void launch_round(pr_graph *g, Workspace &W, T *x, T *r, T *w, cudaStream_t s, Prof *prof = nullptr,
                         int round = 0) {
    const DevGraph &G = g->G;
    Ctl *ctl = W.ctl.as<Ctl>();
    Partials P = partials_of(W);
    Trace tr = trace_of(W);
    const int sms = g->num_sms;
    const int ga = grid_n(G.n_nd, sms, 8);
    size_t e0 = prof ? prof->mark(s) : 0;
    k_activate<T, IFP2><<<ga, kThreads, 0, s>>>(G, ctl, P, r, w, W.bins.as<int32_t>(), tr);
    size_t e1 = prof ? prof->mark(s) : 0;
    k_commit<T><<<sms * 4, kThreads, 0, s>>>(ctl, W.bins.as<int32_t>(), G.n_nd, x, r);
    size_t e2 = prof ? prof->mark(s) : 0;
    const int nbt = sms * 4, nbw = sms * 4, nbc = sms * 2;
    k_push<T, IFP2><<<nbt + nbw + nbc, kThreads, 0, s>>>(G, ctl, W.bins.as<int32_t>(), w, r, nbt, nbw);
    size_t e3 = prof ? prof->mark(s) : 0;
    RowArgs<T> a{};
    a.val = w;
    a.r = r;
    a.x = x;
    const Plan &PL = IFP2 ? g->plan_nd : g->plan_all;
    k_rows<T, OP_ROUND><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
    if (prof) {
        size_t e4 = prof->mark(s);
        prof->add(PR_K_ACTIVATE, round, e0, e1);
        prof->add(PR_K_COMMIT, round, e1, e2);
        prof->add(PR_K_PUSH, round, e2, e3);
        prof->add(PR_K_PULL, round, e3, e4);
    }
}

// Run rounds until the device stop flag is set.  With a CUDA graph: a while
// node whose body holds `unroll` rounds and a kernel that copies !done into
// the loop condition -- no host synchronisation per round.
template <typename T, bool IFP2>
static pr_status run_rounds(pr_graph *g, Workspace &W, T *x, T *r, T *w, bool use_graph, int key,
                            Prof *prof) {
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    const int unroll = kUnroll;
    if (use_graph && !prof) {
        Workspace::G &cg = W.graphs[key];
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
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            PR_CK(cudaStreamBeginCaptureToGraph(W.cap_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < unroll; k++) launch_round<T, IFP2>(g, W, x, r, w, W.cap_stream);
            k_set_while<<<1, 1, 0, W.cap_stream>>>(ctl, h);
            cudaGraph_t captured = nullptr;
            cudaError_t ce = cudaStreamEndCapture(W.cap_stream, &captured);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (round loop)");
            PR_CK(cudaGraphInstantiate(&cg.exec, cg.graph, 0));
            cg.key = key;
        }
        PR_CK(cudaGraphLaunch(cg.exec, s));
        PR_CK(cudaGetLastError());
        return PR_OK;
    }
    // host-driven chunks: every kernel returns at once after the stop flag is set
    int t = 0;
    if (prof) {
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        t = W.hctl->round;
    }
    int chunk = 2;
    std::vector<int8_t> modes;
    for (;;) {
        const int t0 = t;
        for (int k = 0; k < chunk; k++) launch_round<T, IFP2>(g, W, x, r, w, s, prof, t++);
        PR_CK(cudaGetLastError());
        PR_CK(cudaMemcpyAsync(&W.hctl->done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (prof) {
            const int hi = std::min(t, W.trace_len);
            modes.assign(std::max(hi - t0, 0), 0);
            if (hi > t0) PR_CK(cudaMemcpyAsync(modes.data(), W.tM.as<int8_t>() + t0, hi - t0, cudaMemcpyDeviceToHost, s));
        }
        PR_CK(cudaStreamSynchronize(s));
        const int done = W.hctl->done, last = W.hctl->round;  // rounds < last delivered
        if (prof) {
            prof->settle([&](int kind, int rd) {
                if (kind == PR_K_ACTIVATE) return rd <= last && !(done && rd > last);
                if (rd >= last || rd - t0 >= (int)modes.size()) return false;
                const int md = modes[rd - t0];
                return kind == PR_K_PULL ? md == MODE_PULL : md == MODE_PUSH;
            });
        }
        if (done) break;
        chunk = std::min(chunk * 2, 32);
    }
    return PR_OK;
}

// Power loop: two iterations per body (ping-pong buffers), same while-node scheme.
template <typename T>
static void launch_power_pair(pr_graph *g, Workspace &W, T *piA, T *qA, T *piB, T *qB, cudaStream_t s,
                              size_t *mark0 = nullptr, Prof *prof = nullptr, int it = 0) {
    const DevGraph &G = g->G;
    Ctl *ctl = W.ctl.as<Ctl>();
    RowArgs<T> a{};
    a.p64 = W.p64.as<double>();
    a.P = partials_of(W);
    a.tr = trace_of(W);
    const Plan &PL = g->plan_all;
    a.val = qA;
    a.pi_cur = piA;
    a.pi_next = piB;
    a.q_next = qB;
    k_rows<T, OP_POWER><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
    size_t m1 = prof ? prof->mark(s) : 0;
    a.val = qB;
    a.pi_cur = piB;
    a.pi_next = piA;
    a.q_next = qA;
    k_rows<T, OP_POWER><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
    if (prof) {
        size_t m2 = prof->mark(s);
        prof->add(PR_K_POWER, it, *mark0, m1);
        prof->add(PR_K_POWER, it + 1, m1, m2);
    }
}

template <typename T>
static pr_status run_power(pr_graph *g, Workspace &W, T *piA, T *qA, T *piB, T *qB, bool use_graph, int key,
                           Prof *prof) {
    cudaStream_t s = g->stream;
    Ctl *ctl = W.ctl.as<Ctl>();
    if (use_graph && !prof) {
        Workspace::G &cg = W.graphs[key];
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
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            PR_CK(cudaStreamBeginCaptureToGraph(W.cap_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
            launch_power_pair<T>(g, W, piA, qA, piB, qB, W.cap_stream);
            k_set_while<<<1, 1, 0, W.cap_stream>>>(ctl, h);
            cudaGraph_t captured = nullptr;
            cudaError_t ce = cudaStreamEndCapture(W.cap_stream, &captured);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (power loop)");
            PR_CK(cudaGraphInstantiate(&cg.exec, cg.graph, 0));
            cg.key = key;
        }
        PR_CK(cudaGraphLaunch(cg.exec, s));
        PR_CK(cudaGetLastError());
        return PR_OK;
    }
    int chunk = 2, it = 0;
    for (;;) {
        for (int k = 0; k < chunk; k++) {
            size_t e0 = prof ? prof->mark(s) : 0;
            launch_power_pair<T>(g, W, piA, qA, piB, qB, s, prof ? &e0 : nullptr, prof, it);
            it += 2;
        }
        PR_CK(cudaGetLastError());
        PR_CK(cudaMemcpyAsync(&W.hctl->done, &ctl->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&W.hctl->iter, &ctl->iter, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        const int last = W.hctl->iter;  // iterations 1..last ran
        if (prof) prof->settle([&](int kind, int i) { return i < last; });
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
        if (!W.pstage.p || W.pstage.bytes < sizeof(double) * std::max(cnt, 1))
            PR_TRY(W.pstage.alloc(sizeof(double) * std::max(cnt, 1), s));
        PR_CK(cudaMemcpyAsync(W.pstage.p, p->val, sizeof(double) * cnt, cudaMemcpyHostToDevice, s));
        dval = W.pstage.as<double>();
        if (!dense) {
            if (!W.pstage2.p || W.pstage2.bytes < sizeof(int32_t) * std::max(cnt, 1))
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
    h.p_dense = 1;
    h.pu = 0.0;
    return PR_OK;
}

// ------------------------------------------------------------ solve
template <typename T>
static pr_status ifp_phase1(pr_graph *g, Workspace &W, int algo, T *x, T *r, T *w, bool use_graph, int keybase,
                            Prof *prof) {
    if (algo == PR_IFP2) return run_rounds<T, true>(g, W, x, r, w, use_graph, keybase + 1, prof);
    return run_rounds<T, false>(g, W, x, r, w, use_graph, keybase, prof);
}

static pr_status solve_impl(pr_graph *g, double c, double eps, pr_algo algo, pr_prec prec, const pr_pvec *p,
                            const pr_opts *o, double *out, int out_is_device, pr_stats *st) {
    if (!(c > 0.0 && c < 1.0)) return fail(PR_EINVAL, "c must be in (0, 1)");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PR_EINVAL, "eps must be positive and finite");
    if (algo != PR_POWER && algo != PR_IFP1 && algo != PR_IFP2) return fail(PR_EINVAL, "unknown algorithm");
    if (prec != PR_FP64 && prec != PR_FP32) return fail(PR_EINVAL, "unknown precision");
    if (!out) return fail(PR_EINVAL, "out is NULL");
    pr_opts opt{};
    if (o) opt = *o;
    if (opt.max_rounds <= 0) opt.max_rounds = 100000;
    if (opt.pull_ratio <= 0) opt.pull_ratio = 0.04;
    if (opt.mode < 0 || opt.mode > 2) return fail(PR_EINVAL, "unknown mode");
    if (opt.xi_act < 0) return fail(PR_EINVAL, "xi_act must be >= 0");
    const bool use_graph = opt.use_graph >= 0;  // 0 = default (on); -1 = host-driven rounds
    Prof prof_obj;
    Prof *prof = nullptr;
    if (opt.profile) {
        std::memset(opt.profile, 0, sizeof(*opt.profile));
        prof_obj.out = opt.profile;
        prof = &prof_obj;
    }
    const bool fp32 = prec == PR_FP32;
    const int32_t trace_len = opt.max_rounds + 2;
    PR_TRY(ensure_ws(g, fp32, trace_len));
    Workspace &W = *static_cast<Workspace *>(g->ws);
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
    // in-list entries one pull round reads (IFP2: non-dangling rows only)
    {
        int32_t hv[4] = {0, 0, 0, 0};
        PR_CK(cudaMemcpyAsync(&hv[0], G.inr_off + G.n_nd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaMemcpyAsync(&hv[1], G.inu_off + G.n_nd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        h.scan_ref = algo == PR_IFP2 ? hv[0] : G.m_ref;
        h.scan_unref = algo == PR_IFP2 ? hv[1] : G.m_unref;
    }
    h.want_bins = opt.mode != MODE_PULL;
    h.unref_active = 1;
    *W.hctl = h;
    Ctl *ctl = W.ctl.as<Ctl>();
    PR_CK(cudaMemcpyAsync(ctl, W.hctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    PR_CK(cudaEventCreate(&e0));
    PR_CK(cudaEventCreate(&e1));
    PR_CK(cudaEventRecord(e0, s));
    const int sms = g->num_sms;
    const int gn = grid_n(G.n, sms, 8);
    Partials P = partials_of(W);
    double *x64 = W.x64.as<double>(), *r64 = W.r64.as<double>(), *w64 = W.w64.as<double>(),
           *w64b = W.w64b.as<double>(), *p64 = W.p64.as<double>();
    const double *fin_x = x64, *fin_r = r64;
    int fin_kind = algo;
    int fp64_rounds = 0;
    if (algo == PR_POWER) {
        if (fp32) {
            float *pa = W.x32.as<float>(), *pb = W.r32.as<float>(), *qa = W.w32.as<float>(), *qb = W.w32b.as<float>();
            k_power_init<float><<<gn, kThreads, 0, s>>>(G, ctl, P, p64, pa, qa);
            PR_TRY(run_power<float>(g, W, pa, qa, pb, qb, use_graph, 10, prof));
            // result: iteration parity picks the buffer; widen to FP64 for the finalize
            PR_CK(cudaMemcpyAsync(W.hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            PR_CK(cudaStreamSynchronize(s));
            const float *res = (W.hctl->iter & 1) ? pb : pa;
            k_to64<float><<<gn, kThreads, 0, s>>>(G, ctl, res, x64, r64, w64, p64, 0);
        } else {
            k_power_init<double><<<gn, kThreads, 0, s>>>(G, ctl, P, p64, x64, w64);
            PR_TRY(run_power<double>(g, W, x64, w64, r64, w64b, use_graph, 11, prof));
            PR_CK(cudaMemcpyAsync(W.hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            PR_CK(cudaStreamSynchronize(s));
            if (W.hctl->iter & 1) fin_x = r64;
        }
        fin_kind = PR_POWER;
    } else if (fp32) {
        float *x = W.x32.as<float>(), *r = W.r32.as<float>(), *w = W.w32.as<float>();
        k_init_state<float><<<gn, kThreads, 0, s>>>(G.n, ctl, p64, x, r);
        PR_TRY(ifp_phase1<float>(g, W, algo, x, r, w, use_graph, 0, prof));
        // FP64 correction sweep: r = p + c P~ s - s from the FP32 reserve, then FP64 rounds
        k_to64<float><<<gn, kThreads, 0, s>>>(G, ctl, x, x64, r64, w64, p64, algo == PR_IFP2);
        RowArgs<double> a{};
        a.val = w64;
        a.r = r64;
        a.x = x64;
        a.p64 = p64;
        const Plan &PL = algo == PR_IFP2 ? g->plan_nd : g->plan_all;
        k_reset_run<<<1, 1, 0, s>>>(ctl);
        k_rows<double, OP_CORRECT><<<PL.nblocks, kThreads, 0, s>>>(G, PL, ctl, a);
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        const int32_t r32_rounds = W.hctl->round;
        PR_TRY(ifp_phase1<double>(g, W, algo, x64, r64, w64, use_graph, 2, prof));
        PR_CK(cudaMemcpyAsync(&W.hctl->round, &ctl->round, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        fp64_rounds = W.hctl->round - r32_rounds;
    } else {
        k_init_state<double><<<gn, kThreads, 0, s>>>(G.n, ctl, p64, x64, r64);
        PR_TRY(ifp_phase1<double>(g, W, algo, x64, r64, w64, use_graph, 2, prof));
    }
    if (algo == PR_IFP1) k_dangling_mass<<<gn, kThreads, 0, s>>>(G, ctl, P, r64);
    if (algo == PR_IFP2) {  // phase 2 (Alg. 3): one pull into every dangling vertex
        k_phase2_q<<<grid_n(G.n_nd, sms, 8), kThreads, 0, s>>>(G, ctl, x64, w64);
        RowArgs<double> a{};
        a.val = w64;
        a.r = r64;
        a.p64 = p64;
        if (G.n > G.n_nd) k_rows<double, OP_PHASE2><<<g->plan_d.nblocks, kThreads, 0, s>>>(G, g->plan_d, ctl, a);
    }
    k_fin_sum<double><<<gn, kThreads, 0, s>>>(G, ctl, P, fin_kind, fin_x, fin_r);
    double *dout = out_is_device ? out : W.outbuf.as<double>();
    k_fin_write<double><<<gn, kThreads, 0, s>>>(G, ctl, fin_kind, fin_x, fin_r, dout);
    PR_CK(cudaEventRecord(e1, s));
    if (!out_is_device)
        PR_CK(cudaMemcpyAsync(out, dout, sizeof(double) * G.n, cudaMemcpyDeviceToHost, s));
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
        // launches: rounds run inside a while node execute whole bodies of kUnroll rounds
        // (+1 condition kernel); host-driven chunks launch every round they enqueue.
        int64_t L = 0;
        const int64_t act = (algo == PR_POWER ? hc.iter : hc.round) + 1;  // incl. the stopping one
        if (algo == PR_POWER) {
            const int64_t pairs = (hc.iter + 2) / 2;
            L = 1 + pairs * 2 + (use_graph && !prof ? pairs : 0) + 2;
        } else {
            const int64_t bodies = (act + kUnroll - 1) / kUnroll;
            L = (use_graph && !prof) ? bodies * (kUnroll * kRoundLaunches + 1) : act * kRoundLaunches;
            L += 1 + 2 + (algo == PR_IFP2 ? 2 : 1) + (fp32 ? 3 : 0);
        }
        st->launches = L;
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

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_solve_ex(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                                 const pr_opts *opts, double *out, int out_is_device, pr_stats *st) {
    if (!g) return fail(PR_EINVAL, "graph is NULL");
    pr_status s = solve_impl(g, c, eps, a, prec, p, opts, out, out_is_device, st);
    if (s == PR_ECUDA) {
        cudaStreamSynchronize(g->stream);
        cudaGetLastError();
    }
    return s;
}

extern "C" pr_status pr_solve(pr_graph *g, double c, double eps, pr_algo a, pr_prec prec, const pr_pvec *p,
                              double *out, int out_is_device, pr_stats *st) {
    return pr_solve_ex(g, c, eps, a, prec, p, nullptr, out, out_is_device, st);
}
