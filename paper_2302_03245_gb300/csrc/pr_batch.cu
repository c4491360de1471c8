// pr_batch.cu -- pr_solve_batch: many independent IFP1 / IFP2 solves (Alg. 2 /
// Alg. 3) of graphs of uneven size in one persistent kernel per round phase.
//
// Every problem k (graph + personalization + c, eps) keeps its own control
// block and state (x, r, w, bins) in one packed device arena, addressed by
// int64 offsets.  Its rows are cut into tiles along the graph's pull plan
// (in-degree bins, so a tile has one lanes-per-row setting); the tiles of all
// problems form one static table.  A round phase is one launch of
// k_batch_phase: its blocks take tiles from a device work queue (an atomic
// counter over the table), so small and large problems share the GPU with no
// per-problem launches.  For each tile the block performs the problem's
// pending action -- activation, fused pull + next activation, or atomic push
// (each tile pushes its share of the frontier) -- and the last tile of a
// problem to finish takes that problem's stop decision and push/pull choice
// exactly as in the single-graph solver.  The phases run inside a CUDA-graph
// while node until no problem is active.  The one-shot stages (init, FP64
// correction, phase 2, normalisation) are tiled the same way.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pr_group.cuh"
#include "pr_kernels.cuh"

// requests of one graph in flight before new ones join a column group (a
// group round gathers K columns at once; with few columns live, separate
// tile rounds cost less)
#ifndef PR_GROUP_MIN_INFLIGHT
#define PR_GROUP_MIN_INFLIGHT 2
#endif
// column groups per (graph, format) at most.  Every group round is a full pass
// over the graph's in-lists, so more groups on a graph do not serve more
// requests per second: they only stretch every step.  Requests beyond the
// free columns wait in the queue (continuous batching: they join as columns
// free up) instead of running alone in the tile engine, where each costs a
// full pass per round.
#ifndef PR_SERVER_MAX_GROUPS
#define PR_SERVER_MAX_GROUPS 4
#endif

namespace pr {

struct Tile {
    int32_t prob, lo, hi, lanes;  // rows [lo, hi) of problem `prob`; lanes per row (0: block per row)
};

struct BProb {
    DevGraph G;
    RoundBuf B;                  // state in the round format
    Ctl *ctl;
    int32_t t0, nt;              // round tiles [t0, t0 + nt)
    int32_t v0, nv;              // vertex tiles
    int32_t d0, nd;              // dangling-row tiles
    PVals pv;
    double *qc;                  // FP32 form: gather values x_u / ((1-c) deg u) of the correction
    void *q;                     // phase-2 gather values
    double *out;                 // normalised result (device)
};

struct BCtl {
    uint32_t head, exit_ticket;
    int32_t active, pad;
};

struct BSlots {  // per-tile partials of the round reductions
    double *R;
    long long *F, *E;
    int *u;
};

// -------------------------------------------------------------- device helpers
// The block claims tile after tile from the queue; returns -1 when it is empty.
__device__ __forceinline__ int claim_tile(BCtl *bc, int ntiles) {
    __shared__ int s_tile;
    __syncthreads();
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&bc->head, 1u);
    __syncthreads();
    const int t = s_tile;
    return t < ntiles ? t : -1;
}

// the last block of the grid to leave resets the queue for the next launch
__device__ __forceinline__ void leave_queue(BCtl *bc) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bc->exit_ticket, 1u) == gridDim.x - 1) {
            bc->head = 0;
            bc->exit_ticket = 0;
            __threadfence();
        }
    }
}

// true in the block that finished the last of the problem's `count` tiles
__device__ __forceinline__ bool last_tile(Ctl *ctl, int count) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1u) == (unsigned)(count - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Each push tile handles its share (worker w of nw) of every frontier bin.
template <typename T, bool IFP2>
__device__ __forceinline__ void push_worker(const DevGraph &G, const Ctl *ctl, const RoundBuf &B, int w, int nw) {
    const uint32_t *cnt = (ctl->cur & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
    const int n_nd = G.n_nd;
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    const T *vbuf = static_cast<const T *>(B.vbuf);
    const T cT = ST<T>::c(ctl);
    for (int b = 0; b < 3; b++) {
        const int c = (int)cnt[b];
        const int ch = (c + nw - 1) / nw;
        const int lo = min(w * ch, c), hi = min(lo + ch, c);
        const int32_t *bins = B.bins + (size_t)b * n_nd;
        if (b == 0) {  // a thread per vertex
            for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
                const int i = PR_IDX(bins[k], n_nd, DBG_BIN);
                if (i < 0) continue;
                const T v = vbuf[i];
                push_commit<T>(ctl, x, r, i, v);
                const T wi = ST<T>::mul(v, ST<T>::mul(cT, ST<T>::invdeg(G, i)));
                const int e0 = G.out_off[i];
                const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
                for (int e = e0; e < e1; e++) {
                    const int t = PR_IDX(G.out_dst[e], IFP2 ? n_nd : G.n, DBG_OUT_DST);
                    if (t >= 0) ST<T>::push_to(r, B.din, t, wi);
                }
            }
        } else {  // a warp (bin 1) or the block (bin 2) per vertex
            const int lanes = b == 1 ? 32 : (int)blockDim.x;
            const int gid = b == 1 ? (int)(threadIdx.x >> 5) : 0;
            const int ngrp = b == 1 ? (int)(blockDim.x >> 5) : 1;
            const int lane = b == 1 ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
            for (int k = lo + gid; k < hi; k += ngrp) {
                const int i = PR_IDX(bins[k], n_nd, DBG_BIN);  // the same for the whole group
                if (i < 0) continue;
                const T v = vbuf[i];
                if (lane == 0) push_commit<T>(ctl, x, r, i, v);
                const T wi = ST<T>::mul(v, ST<T>::mul(cT, ST<T>::invdeg(G, i)));
                const int e0 = G.out_off[i];
                const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
                push_list<T, IFP2>(G, r, B.din, e0, e1, wi, lane, lanes);
            }
        }
    }
}

// -------------------------------------------------------------- the phase kernel
template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_batch_phase(const BProb *probs, const Tile *tiles, int ntiles,
                                                         BCtl *bc, BSlots sl) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ A sha[32];
    __shared__ R shr[32];
    const Trace no_trace{nullptr, nullptr, nullptr, nullptr};
    for (;;) {
        const int tile = claim_tile(bc, ntiles);
        if (tile < 0) break;
        const Tile tl = tiles[tile];
        const BProb &P = probs[tl.prob];
        Ctl *ctl = P.ctl;
        if (ctl->done) continue;
        const int mode = ctl->mode;
        const int t = ctl->round;
        const int want = ctl->want_bins;
        uint32_t *bcnt = (t & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
        R Rl = ST<T>::rzero();
        long long Fl = 0, El = 0;
        int ul = 0;
        if (mode == MODE_PULL) {
            const V *wprev = static_cast<const V *>((t & 1) ? P.B.w[0] : P.B.w[1]);
            V *wnext = static_cast<V *>((t & 1) ? P.B.w[1] : P.B.w[0]);
            const Seg S{tl.lo, tl.hi, tl.lanes, 0, 1};
            round_segment<T, IFP2>(P.G, S, 0, ctl, P.B, wprev, wnext, ctl->unref_active != 0, want, bcnt, Rl, Fl,
                                   El, ul, sha);
        } else if (mode == MODE_ACT) {
            V *w = static_cast<V *>((t & 1) ? P.B.w[1] : P.B.w[0]);
            activate_range<T, IFP2>(P.G, ctl, P.B, w, tl.lo, min(tl.hi, P.G.n_nd), 0, blockDim.x, want, bcnt, Rl,
                                    Fl, El, ul);
        } else {
            push_worker<T, IFP2>(P.G, ctl, P.B, tile - P.t0, P.nt);
        }
        if (mode != MODE_PUSH) {
            const R Rb = block_sum_r<T>(Rl, shr);
            const long long Fb = block_sum(Fl, shl);
            const long long Eb = block_sum(El, shl);
            const int ub = __syncthreads_or(ul);
            if (threadIdx.x == 0) {
                memcpy(reinterpret_cast<char *>(sl.R) + 8 * (size_t)tile, &Rb, 8);
                sl.F[tile] = Fb;
                sl.E[tile] = Eb;
                sl.u[tile] = ub;
            }
        }
        if (!last_tile(ctl, P.nt)) continue;
        if (mode == MODE_PUSH) {  // frontier delivered: the activation is next
            if (threadIdx.x == 0) {
                ctl->ticket = 0;
                ctl->mode = MODE_ACT;
            }
            continue;
        }
        double Rs = 0.0;
        long long F = 0, E = 0;
        int u = 0;
        for (int k = P.t0 + threadIdx.x; k < P.t0 + P.nt; k += blockDim.x) {
            R v;
            const unsigned long long bits = __ldcg(reinterpret_cast<const unsigned long long *>(sl.R) + k);
            memcpy(&v, &bits, 8);
            Rs += ST<T>::r_to_d(v);
            F += __ldcg(&sl.F[k]);
            E += __ldcg(&sl.E[k]);
            u |= __ldcg(&sl.u[k]);
        }
        Rs = block_sum(Rs, shd);
        F = block_sum(F, shl);
        E = block_sum(E, shl);
        u = __syncthreads_or(u);
        if (threadIdx.x == 0) {
            round_decision(ctl, t, Rs, F, E, u, want, no_trace);
            if (ctl->done) atomicSub(&bc->active, 1);
        }
    }
    leave_queue(bc);
}

__global__ void k_batch_set_while(const BCtl *bc, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, bc->active > 0 ? 1u : 0u);
}

// -------------------------------------------------------------- one-shot stages
// (each tile once; a block per tile, grid-stride over the tile list)
template <typename T>
__global__ void k_batch_init(const BProb *probs, const Tile *vt, int nvt) {
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        T *x = static_cast<T *>(P.B.x);
        T *r = static_cast<T *>(P.B.r);
        double *din = P.B.din;
        for (int i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x) {
            x[i] = ST<T>::zero();
            r[i] = ST<T>::p(P.ctl, P.pv, i);
            if (din) din[i] = 0.0;
        }
    }
}

// FP32 reserve -> IEEE double state (exactly), and the gather values
// q_u = x_u / ((1-c) deg(u)) of the correction sweep in double; IFP2's dangling
// residual is p (phase 1 never touches it), IFP1's comes from the sweep
template <bool IFP2>
__global__ void k_batch_to_fp64(const BProb *probs, const BProb *probs64, const Tile *vt, int nvt) {
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        const BProb &Q = probs64[tl.prob];
        const float *x32 = static_cast<const float *>(P.B.x);
        double *x = static_cast<double *>(Q.B.x);
        double *r = static_cast<double *>(Q.B.r);
        for (int i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x) {
            const double xv = (double)x32[i];
            x[i] = xv;
            if (i < P.G.n_nd) Q.qc[i] = xv * (P.G.inv_deg64[i] * P.ctl->inv_om);
            else if (IFP2) r[i] = P.ctl->p_dense ? P.pv.p64[i] : P.ctl->pu;
        }
    }
}

// correction sweep r = p + c P~ s - s (IEEE double) over the round tiles, into
// the FP64 state
__global__ void __launch_bounds__(kThreads) k_batch_correct(const BProb *probs64, const Tile *tiles, int ntiles) {
    using A = typename GT<double>::A;
    __shared__ A sha[32];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        const BProb &Q = probs64[tl.prob];
        SweepArgs<double> a{};
        a.val = Q.qc;
        a.r = static_cast<double *>(Q.B.r);
        a.x = static_cast<const double *>(Q.B.x);
        a.pv = Q.pv;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        const Seg S{tl.lo, tl.hi, tl.lanes, 0, 1};
        sweep_segment<double, OP_CORRECT>(Q.G, S, 0, Q.ctl, a, s1, s2, s3, sha);
    }
}

// double-float inboxes folded into r (IFP1 dangling rows: pushed into, never activated)
__global__ void k_batch_fold(const BProb *probs, const Tile *vt, int nvt) {
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        float2 *r = static_cast<float2 *>(P.B.r);
        for (int i = max(tl.lo, P.G.n_nd) + (int)threadIdx.x; i < tl.hi; i += blockDim.x)
            ST<float2>::fold(r, P.B.din, i);
    }
}

__global__ void k_batch_reset(const BProb *probs, int count, BCtl *bc) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        Ctl *ctl = probs[k].ctl;
        ctl->done = 0;
        ctl->status = 0;
        ctl->ticket = 0;
        ctl->mode = MODE_ACT;
        ctl->bin_cnt[0][0] = ctl->bin_cnt[0][1] = ctl->bin_cnt[0][2] = 0;
        ctl->bin_cnt[1][0] = ctl->bin_cnt[1][1] = ctl->bin_cnt[1][2] = 0;
        ctl->want_bins = ctl->policy != MODE_PULL;
        ctl->unref_active = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bc->active = count;
        bc->head = 0;
        bc->exit_ticket = 0;
    }
}

// IFP2 phase 2 (Alg. 3): q_u = x_u / ((1-c) deg(u)), then one pull into every dangling vertex
template <typename T>
__global__ void k_batch_phase2_q(const BProb *probs, const Tile *vt, int nvt) {
    using V = typename ST<T>::V;
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        const T *x = static_cast<const T *>(P.B.x);
        V *q = static_cast<V *>(P.q);
        const int hi = min(tl.hi, P.G.n_nd);
        for (int i = tl.lo + threadIdx.x; i < hi; i += blockDim.x)
            q[i] = ST<T>::pack(ST<T>::mul(x[i], ST<T>::mul(ST<T>::invdeg(P.G, i), ST<T>::inv_om(P.ctl))));
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_batch_phase2(const BProb *probs, const Tile *dt, int ndt) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    __shared__ A sha[32];
    for (int k = blockIdx.x; k < ndt; k += gridDim.x) {
        const Tile tl = dt[k];
        const BProb &P = probs[tl.prob];
        SweepArgs<T> a{};
        a.val = static_cast<const V *>(P.q);
        a.r = static_cast<T *>(P.B.r);
        a.pv = P.pv;
        R s1 = ST<T>::rzero(), s2 = ST<T>::rzero(), s3 = ST<T>::rzero();
        const Seg S{tl.lo, tl.hi, tl.lanes, 0, 1};
        sweep_segment<T, OP_PHASE2>(P.G, S, 0, P.ctl, a, s1, s2, s3, sha);
    }
}

// normaliser per problem (vertex tiles; the problem's last tile adds them up)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_batch_fin_sum(const BProb *probs, const Tile *vt, int nvt, int kind,
                                                           double *slots) {
    using R = typename ST<T>::R;
    __shared__ double shd[32];
    __shared__ R shr[32];
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        const T *x = static_cast<const T *>(P.B.x);
        const T *r = static_cast<const T *>(P.B.r);
        R s = ST<T>::rzero();
        for (int i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x)
            s = ST<T>::radd(s, ST<T>::rval(zval<T>(P.G, P.ctl, kind, x, r, i)));
        s = block_sum_r<T>(s, shr);
        if (threadIdx.x == 0) slots[k] = ST<T>::r_to_d(s);
        if (!last_tile(P.ctl, P.nv)) continue;
        double sum = 0.0;
        for (int q = P.v0 + threadIdx.x; q < P.v0 + P.nv; q += blockDim.x) sum += __ldcg(&slots[q]);
        sum = block_sum(sum, shd);
        if (threadIdx.x == 0) {
            P.ctl->ticket = 0;
            P.ctl->zsum = sum;
        }
    }
}

template <typename T>
__global__ void k_batch_fin_write(const BProb *probs, const Tile *vt, int nvt, int kind) {
    for (int k = blockIdx.x; k < nvt; k += gridDim.x) {
        const Tile tl = vt[k];
        const BProb &P = probs[tl.prob];
        const T *x = static_cast<const T *>(P.B.x);
        const T *r = static_cast<const T *>(P.B.r);
        const double inv = 1.0 / P.ctl->zsum;
        for (int i = tl.lo + threadIdx.x; i < tl.hi; i += blockDim.x) {
            const int c = PR_IDX(P.G.perm[i], P.G.n, DBG_PERM);
            if (c >= 0) P.out[c] = ST<T>::to_d(zval<T>(P.G, P.ctl, kind, x, r, i)) * inv;
        }
    }
}

// -------------------------------------------------------------- host side
namespace {

constexpr int kVertexTile = 4096;   // rows per elementwise tile
constexpr int kEdgeTile = 16384;    // target in-list entries per round tile

// rows per tile for a lanes-per-row setting (rows have in-degree <= 2 * lanes below 32)
int tile_rows(int lanes) {
    if (lanes == 0) return 1;
    if (lanes >= 32) return 64;
    return std::max(kThreads / lanes, kEdgeTile / (2 * lanes));
}

void cut_plan(const Plan &PL, int prob, std::vector<Tile> &out) {
    for (int s = 0; s < PL.nseg; s++) {
        const Seg &S = PL.seg[s];
        const int step = tile_rows(S.lanes);
        for (int lo = S.lo; lo < S.hi; lo += step) out.push_back(Tile{prob, lo, std::min(lo + step, S.hi), S.lanes});
    }
}

void cut_rows(int lo, int hi, int prob, std::vector<Tile> &out) {
    for (int a = lo; a < hi; a += kVertexTile) out.push_back(Tile{prob, a, std::min(a + kVertexTile, hi), 1});
}

struct Arena {  // bump allocator over one device buffer (256-byte aligned slices)
    Buf buf;
    size_t used = 0;
    size_t take(size_t bytes) {
        const size_t at = used;
        used += (bytes + 255) & ~(size_t)255;
        return at;
    }
    template <typename X> X *at(size_t off) const { return reinterpret_cast<X *>(static_cast<char *>(buf.p) + off); }
};

struct StateOffsets {
    size_t x, r, vbuf, w0, w1, bins, q;
    size_t din;  // double-float state: push-round inbox (FP64); else unused
};

StateOffsets take_state(Arena &A, size_t n, size_t nnd, size_t t_bytes, size_t v_bytes, bool inbox) {
    StateOffsets o{};
    o.x = A.take(t_bytes * n);
    o.r = A.take(t_bytes * n);
    o.vbuf = A.take(t_bytes * nnd);
    o.w0 = A.take(v_bytes * nnd);
    o.w1 = A.take(v_bytes * nnd);
    o.bins = A.take(sizeof(int32_t) * 3 * nnd);
    o.q = A.take(v_bytes * n);
    o.din = inbox ? A.take(sizeof(double) * n) : 0;
    return o;
}

RoundBuf round_buf(const Arena &A, const StateOffsets &o) {
    return RoundBuf{A.at<char>(o.x), A.at<char>(o.r), A.at<char>(o.vbuf), {A.at<char>(o.w0), A.at<char>(o.w1)},
                    A.at<int32_t>(o.bins), o.din ? A.at<double>(o.din) : nullptr};
}

template <typename T, bool IFP2>
pr_status run_batch_rounds(cudaStream_t s, cudaStream_t cap, const BProb *d_probs, const Tile *d_tiles,
                           int ntiles, BCtl *bc, BSlots sl, int grid, cudaGraphExec_t *exec, cudaGraph_t *graph) {
    // a while node: kUnrollB phases per body, then the active-problem test
    constexpr int kUnrollB = 4;
    PR_CK(cudaGraphCreate(graph, 0));
    cudaGraphConditionalHandle h;
    PR_CK(cudaGraphConditionalHandleCreate(&h, *graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    PR_CK(cudaGraphAddNode(&node, *graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    PR_CK(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < kUnrollB; k++)
        k_batch_phase<T, IFP2><<<grid, kThreads, 0, cap>>>(d_probs, d_tiles, ntiles, bc, sl);
    k_batch_set_while<<<1, 1, 0, cap>>>(bc, h);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &captured);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture (batch while body)");
    PR_CK(cudaGraphInstantiate(exec, *graph, 0));
    PR_CK(cudaGraphLaunch(*exec, s));
    PR_CK(cudaGetLastError());
    return PR_OK;
}

struct GraphGuard {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~GraphGuard() {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

template <typename T>
pr_status batch_rounds(bool ifp2, cudaStream_t s, cudaStream_t cap, const BProb *d_probs, const Tile *d_tiles,
                       int ntiles, BCtl *bc, BSlots sl, int grid) {
    GraphGuard gg;
    if (ifp2) PR_TRY(run_batch_rounds<T, true>(s, cap, d_probs, d_tiles, ntiles, bc, sl, grid, &gg.e, &gg.g));
    else PR_TRY(run_batch_rounds<T, false>(s, cap, d_probs, d_tiles, ntiles, bc, sl, grid, &gg.e, &gg.g));
    PR_CK(cudaStreamSynchronize(s));  // the graph is destroyed on return
    return PR_OK;
}

}  // namespace

static pr_status solve_batch_impl(pr_graph *const *gs, int32_t count, const double *c, const double *eps,
                                  pr_algo algo, pr_prec prec, const pr_pvec *ps, const pr_opts *o,
                                  double *const *outs, int outs_are_device, pr_stats *sts) {
    if (!gs || count < 1) return fail(PR_EINVAL, "pr_solve_batch: no graphs");
    if (!c || !eps || !outs) return fail(PR_EINVAL, "pr_solve_batch: c, eps and outs are required");
    if (algo != PR_IFP1 && algo != PR_IFP2) return fail(PR_EINVAL, "pr_solve_batch: algo must be IFP1 or IFP2");
    if (prec != PR_FP64 && prec != PR_FP32 && prec != PR_DF64) return fail(PR_EINVAL, "unknown precision");
    pr_opts opt{};
    if (o) opt = *o;
    if (opt.max_rounds <= 0) opt.max_rounds = 100000;
    if (opt.mode == PR_MODE_LEVELS || opt.mode == PR_MODE_ASYNC || opt.mode == PR_MODE_APULL)
        return fail(PR_EINVAL, "PR_MODE_LEVELS, PR_MODE_ASYNC and PR_MODE_APULL run in pr_solve only");
    if (opt.mode < 0 || opt.mode > 2) return fail(PR_EINVAL, "unknown mode");
    for (int k = 0; k < count; k++) {
        if (!gs[k]) return fail(PR_EINVAL, "pr_solve_batch: graph " + std::to_string(k) + " is NULL");
        if (!(c[k] > 0.0 && c[k] < 1.0)) return fail(PR_EINVAL, "pr_solve_batch: c out of (0, 1)");
        if (!(eps[k] > 0.0) || !std::isfinite(eps[k])) return fail(PR_EINVAL, "pr_solve_batch: eps must be > 0");
        if (!outs[k]) return fail(PR_EINVAL, "pr_solve_batch: outs[k] is NULL");
        if (ps && ps[k].nnz >= 0) return fail(PR_EINVAL, "pr_solve_batch: only uniform p is supported");
        if (gs[k]->device != gs[0]->device) return fail(PR_EINVAL, "pr_solve_batch: graphs on different devices");
    }
    const bool ifp2 = algo == PR_IFP2;
    cudaStream_t s = gs[0]->stream;
    const int sms = gs[0]->num_sms;
    // tiles
    std::vector<Tile> rt, vt, dt;
    std::vector<BProb> hp(count), hp64;
    for (int k = 0; k < count; k++) {
        pr_graph *g = gs[k];
        hp[k].t0 = (int32_t)rt.size();
        cut_plan(ifp2 ? g->plan_nd : g->plan_all, k, rt);
        hp[k].nt = (int32_t)rt.size() - hp[k].t0;
        if (hp[k].nt == 0) {  // a graph with no rows still needs one tile for its decisions
            rt.push_back(Tile{k, 0, 0, 1});
            hp[k].nt = 1;
        }
        hp[k].v0 = (int32_t)vt.size();
        cut_rows(0, g->G.n, k, vt);
        hp[k].nv = (int32_t)vt.size() - hp[k].v0;
        hp[k].d0 = (int32_t)dt.size();
        cut_plan(g->plan_d, k, dt);
        hp[k].nd = (int32_t)dt.size() - hp[k].d0;
    }
    // arena: control blocks, per-problem state, outputs, tiles, slots
    const bool fp32 = prec == PR_FP32;
    const size_t tb = prec == PR_FP64 ? sizeof(double) : (prec == PR_FP32 ? sizeof(float) : sizeof(float2));
    const size_t vb = prec == PR_FP32 ? sizeof(float) : sizeof(float2);
    Arena A;
    const size_t off_ctl = A.take(sizeof(Ctl) * count);
    const size_t off_bc = A.take(sizeof(BCtl));
    std::vector<StateOffsets> so(count), so64(fp32 ? count : 0);
    std::vector<size_t> off_out(count), off_qc(count);
    for (int k = 0; k < count; k++) {
        const size_t n = gs[k]->G.n, nnd = std::max(gs[k]->G.n_nd, 1);
        so[k] = take_state(A, n, nnd, tb, vb, prec == PR_DF64);
        if (fp32) {
            so64[k] = take_state(A, n, nnd, sizeof(double), sizeof(double), false);
            off_qc[k] = A.take(sizeof(double) * n);
        }
        off_out[k] = outs_are_device ? 0 : A.take(sizeof(double) * n);
    }
    const size_t off_probs = A.take(sizeof(BProb) * count);
    const size_t off_probs64 = fp32 ? A.take(sizeof(BProb) * count) : 0;
    const size_t off_rt = A.take(sizeof(Tile) * rt.size());
    const size_t off_vt = A.take(sizeof(Tile) * vt.size());
    const size_t off_dt = A.take(sizeof(Tile) * std::max<size_t>(dt.size(), 1));
    const size_t nslot = std::max(rt.size(), vt.size());
    const size_t off_sR = A.take(sizeof(double) * nslot);
    const size_t off_sF = A.take(sizeof(long long) * nslot);
    const size_t off_sE = A.take(sizeof(long long) * nslot);
    const size_t off_su = A.take(sizeof(int) * nslot);
    PR_TRY(A.buf.alloc(A.used, s));
    Ctl *d_ctl = A.at<Ctl>(off_ctl);
    BCtl *bc = A.at<BCtl>(off_bc);
    // control blocks and problem descriptors
    std::vector<Ctl> hc(count);
    for (int k = 0; k < count; k++) {
        pr_graph *g = gs[k];
        Ctl &h = hc[k];
        std::memset(&h, 0, sizeof(h));
        const int64_t m_valid = ifp2 ? (g->G.m - g->info.m_d) : g->G.m;
        h.c = c[k];
        h.one_minus_c = 1.0 - c[k];
        h.eps = eps[k];
        h.xi = opt.xi_act > 0 ? opt.xi_act : eps[k] / (double)std::max(g->G.n_nd, 1);
        h.pull_edges = (opt.pull_ratio > 0 ? opt.pull_ratio : g->pull_ratio) * (double)std::max<int64_t>(m_valid, 1);
        h.pu = 1.0 / (double)g->G.n;
        h.algo = algo;
        h.policy = opt.mode;
        h.max_rounds = opt.max_rounds;
        h.trace_cap = 0;
        h.scan_ref = ifp2 ? g->scan_nd_ref : g->G.m_ref;
        h.scan_unref = ifp2 ? g->scan_nd_unref : g->G.m_unref;
        h.mode = MODE_ACT;
        h.want_bins = opt.mode != MODE_PULL;
        h.unref_active = 1;
        fill_formats(h);
        BProb &P = hp[k];
        P.G = g->G;
        P.B = round_buf(A, so[k]);
        P.ctl = d_ctl + k;
        P.pv = PVals{nullptr, nullptr, nullptr};
        P.q = A.at<char>(so[k].q);
        P.out = outs_are_device ? outs[k] : A.at<double>(off_out[k]);
        if (fp32) {
            P.qc = A.at<double>(off_qc[k]);
        }
    }
    if (fp32) {
        hp64 = hp;
        for (int k = 0; k < count; k++) {
            hp64[k].B = round_buf(A, so64[k]);
            hp64[k].q = A.at<char>(so64[k].q);
        }
    }
    BCtl hbc{0, 0, count, 0};
    PR_CK(cudaMemcpyAsync(d_ctl, hc.data(), sizeof(Ctl) * count, cudaMemcpyHostToDevice, s));
    PR_CK(cudaMemcpyAsync(bc, &hbc, sizeof(BCtl), cudaMemcpyHostToDevice, s));
    const BProb *d_probs = A.at<BProb>(off_probs);
    PR_CK(cudaMemcpyAsync(A.at<BProb>(off_probs), hp.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice, s));
    const BProb *d_probs64 = fp32 ? A.at<BProb>(off_probs64) : nullptr;
    if (fp32)
        PR_CK(cudaMemcpyAsync(A.at<BProb>(off_probs64), hp64.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice,
                              s));
    const Tile *d_rt = A.at<Tile>(off_rt), *d_vt = A.at<Tile>(off_vt), *d_dt = A.at<Tile>(off_dt);
    PR_CK(cudaMemcpyAsync(A.at<Tile>(off_rt), rt.data(), sizeof(Tile) * rt.size(), cudaMemcpyHostToDevice, s));
    PR_CK(cudaMemcpyAsync(A.at<Tile>(off_vt), vt.data(), sizeof(Tile) * vt.size(), cudaMemcpyHostToDevice, s));
    if (!dt.empty())
        PR_CK(cudaMemcpyAsync(A.at<Tile>(off_dt), dt.data(), sizeof(Tile) * dt.size(), cudaMemcpyHostToDevice, s));
    BSlots sl{A.at<double>(off_sR), A.at<long long>(off_sF), A.at<long long>(off_sE), A.at<int>(off_su)};
    const int nrt = (int)rt.size(), nvt = (int)vt.size(), ndt = (int)dt.size();
    const int grid = sms * 6;  // persistent: about the resident capacity
    const int sgrid = (int)std::min<int64_t>(std::max(nvt, 1), (int64_t)sms * 16);
    cudaStream_t cap = nullptr;
    PR_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } cap_guard{cap};
    cudaEvent_t e0, e1;
    PR_CK(cudaEventCreate(&e0));
    PR_CK(cudaEventCreate(&e1));
    PR_CK(cudaEventRecord(e0, s));
    int kind = algo;
    std::vector<int32_t> r32_rounds(count, 0);
    if (prec == PR_FP64) {
        k_batch_init<double><<<sgrid, kThreads, 0, s>>>(d_probs, d_vt, nvt);
        PR_TRY(batch_rounds<double>(ifp2, s, cap, d_probs, d_rt, nrt, bc, sl, grid));
    } else if (prec == PR_DF64) {
        k_batch_init<float2><<<sgrid, kThreads, 0, s>>>(d_probs, d_vt, nvt);
        PR_TRY(batch_rounds<float2>(ifp2, s, cap, d_probs, d_rt, nrt, bc, sl, grid));
    } else {
        k_batch_init<float><<<sgrid, kThreads, 0, s>>>(d_probs, d_vt, nvt);
        PR_TRY(batch_rounds<float>(ifp2, s, cap, d_probs, d_rt, nrt, bc, sl, grid));
        std::vector<Ctl> mid(count);
        PR_CK(cudaMemcpyAsync(mid.data(), d_ctl, sizeof(Ctl) * count, cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        for (int k = 0; k < count; k++) r32_rounds[k] = mid[k].round;
        if (ifp2) k_batch_to_fp64<true><<<sgrid, kThreads, 0, s>>>(d_probs, d_probs64, d_vt, nvt);
        else k_batch_to_fp64<false><<<sgrid, kThreads, 0, s>>>(d_probs, d_probs64, d_vt, nvt);
        k_batch_correct<<<(int)std::min<int64_t>(nrt, (int64_t)sms * 16), kThreads, 0, s>>>(d_probs64, d_rt, nrt);
        k_batch_reset<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(d_probs64, count, bc);
        PR_TRY(batch_rounds<double>(ifp2, s, cap, d_probs64, d_rt, nrt, bc, sl, grid));
    }
    // phase 2 and normalisation in the final format
    const BProb *d_fin = fp32 ? d_probs64 : d_probs;
    const int dgrid = (int)std::min<int64_t>(std::max(ndt, 1), (int64_t)sms * 16);
    if (prec == PR_FP64 || fp32) {
        if (ifp2 && ndt) {
            k_batch_phase2_q<double><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt);
            k_batch_phase2<double><<<dgrid, kThreads, 0, s>>>(d_fin, d_dt, ndt);
        }
        k_batch_fin_sum<double><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt, kind, sl.R);
        k_batch_fin_write<double><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt, kind);
    } else {
        if (ifp2 && ndt) {
            k_batch_phase2_q<float2><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt);
            k_batch_phase2<float2><<<dgrid, kThreads, 0, s>>>(d_fin, d_dt, ndt);
        }
        if (!ifp2) k_batch_fold<<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt);
        k_batch_fin_sum<float2><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt, kind, sl.R);
        k_batch_fin_write<float2><<<sgrid, kThreads, 0, s>>>(d_fin, d_vt, nvt, kind);
    }
    PR_CK(cudaEventRecord(e1, s));
    for (int k = 0; k < count && !outs_are_device; k++)
        PR_CK(cudaMemcpyAsync(outs[k], hp[k].out, sizeof(double) * gs[k]->G.n, cudaMemcpyDeviceToHost, s));
    PR_CK(cudaMemcpyAsync(hc.data(), d_ctl, sizeof(Ctl) * count, cudaMemcpyDeviceToHost, s));
    PR_CK(cudaStreamSynchronize(s));
    PR_CK(cudaGetLastError());
    float ms = 0;
    PR_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bool all_ok = true;
    for (int k = 0; k < count; k++) {
        const Ctl &h = hc[k];
        if (h.status != 0) all_ok = false;
        if (!sts) continue;
        pr_stats &st = sts[k];
        std::memset(&st, 0, sizeof(st));
        st.rounds = h.round;
        st.rounds_push = h.rounds_push;
        st.rounds_pull = h.rounds_pull;
        st.fp64_rounds = fp32 ? h.round - r32_rounds[k] : 0;
        st.pushes = h.pushes;
        st.edges_pushed = h.edges_pushed + (ifp2 ? gs[k]->info.m_d : 0);
        st.edges_scanned = h.edges_scanned + (ifp2 ? gs[k]->info.m_d : 0);
        st.resid_l1 = h.R;
        st.err_bound = (algo == PR_IFP1 ? 2.0 * h.c * h.R : 2.0 * h.R) / (1.0 - h.c);
        st.ms = ms;
        st.p_scale = 1.0;
    }
    if (!all_ok) return fail(PR_ENOTCONV, "pr_solve_batch: a problem hit the round cap or stalled");
    return PR_OK;
}

}  // namespace pr

using namespace pr;

extern "C" pr_status pr_solve_batch(pr_graph *const *gs, int32_t count, const double *c, const double *eps,
                                    pr_algo a, pr_prec prec, const pr_pvec *ps, const pr_opts *opts,
                                    double *const *outs, int outs_are_device, pr_stats *sts) {
    cudaStream_t st0 = (gs && count > 0 && gs[0]) ? gs[0]->stream : nullptr;
    dbg_begin(st0);
    pr_status s = solve_batch_impl(gs, count, c, eps, a, prec, ps, opts, outs, outs_are_device, sts);
    if (s == PR_ECUDA && st0) {
        cudaStreamSynchronize(st0);
        cudaGetLastError();
    }
    if (s == PR_OK || s == PR_ENOTCONV) s = dbg_end(st0, "pr_solve_batch", s);
    return s;
}

namespace pr {
// host side of the debug record of this translation unit (batches, server)
bool dbg_reset_batch(int inject) {
#ifdef PR_DEBUG
    DbgRec z{};
    z.inject = inject;
    return cudaMemcpyToSymbol(g_pr_dbg, &z, sizeof(z)) == cudaSuccess;
#else
    (void)inject;
    return false;
#endif
}
bool dbg_read_batch(DbgRec *out) {
#ifdef PR_DEBUG
    return cudaMemcpyFromSymbol(out, g_pr_dbg, sizeof(*out)) == cudaSuccess;
#else
    (void)out;
    return false;
#endif
}
}  // namespace pr

// ============================================================== serving
// pr_server: continuous batching of IFP2 requests (full PageRank or
// personalized PageRank) on resident graphs.  A host thread owns the stream
// and loops: admit queued requests while the device-memory budget allows
// (each request gets its own state block); run a few round phases of every
// active request with k_batch_phase over their tile table; read back which
// requests stopped; finish those (FP64 correction for the FP32 form, IFP2
// phase 2, normalisation) with the batched stage kernels, copy their results
// to the host and release their memory.  New requests join at the next step,
// while the others continue.
namespace pr {

// Compact status of the active requests (one D2H copy per step).
struct ReqStat {
    int32_t done, status, round, pad;
};

__global__ void k_gather_status(const BProb *probs, int count, ReqStat *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const Ctl *c = probs[k].ctl;
        out[k] = ReqStat{c->done, c->status, c->round, 0};
    }
}

__global__ void k_gather_ctls(Ctl *const *ctls, int count, ReqStat *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const Ctl *c = ctls[k];
        out[k] = ReqStat{c->done, c->status, c->round, 0};
    }
}

// r = p for one request: zero everywhere, then the seeds (or uniform)
template <typename T>
__global__ void k_req_init(int32_t n, T *x, T *r, double pu, const int32_t *idx, const double *val, int nnz,
                           const int32_t *inv, double *p64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = ST<T>::zero();
        r[i] = nnz < 0 ? ST<T>::pack_from_d(pu) : ST<T>::zero();
        if (p64) p64[i] = nnz < 0 ? pu : 0.0;
    }
}

template <typename T>
__global__ void k_req_seeds(T *r, const int32_t *idx, const double *val, int nnz, const int32_t *inv, double *p64) {
    // one thread: seeds may repeat; they are few (personalization on 1-64 vertices)
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int k = 0; k < nnz; k++) {
        const int i = inv[idx[k]];
        r[i] = ST<T>::add(r[i], ST<T>::pack_from_d(val[k]));
        if (p64) p64[i] += val[k];
    }
}

}  // namespace pr

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace pr {
namespace {

// parallel seeding (seeds may repeat): r[inv[idx[k]]] += val[k]
template <typename T>
__global__ void k_req_seed_par(T *r, const int32_t *idx, const double *val, int nnz, const int32_t *inv,
                               double *p64) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int i = inv[idx[k]];
        ST<T>::atomic_add(&r[i], ST<T>::pack_from_d(val[k]));
        if (p64) atomicAdd(&p64[i], val[k]);
    }
}

struct SReq {
    int64_t ticket = 0;
    pr_graph *g = nullptr;
    double c = 0.85, eps = 1e-6;
    pr_prec prec = PR_DF64;
    int32_t nnz = -1;               // < 0: uniform p
    std::vector<int32_t> idx;
    std::vector<double> val;
    double p_scale = 1.0;
    int stage = 0;                  // 0 queued, 1 rounds, 2 FP64 rounds after correction, 3 done
    pr_status status = PR_OK;
    size_t bytes = 0;
    void *mem = nullptr;            // one stream-ordered allocation
    StateOffsets s_main{}, s64{};  // s64: FP32 requests after the FP64 correction
    size_t off_ctl = 0, off_out = 0, off_qc = 0, off_p64 = 0, off_sidx = 0, off_sval = 0;
    int32_t rounds_first = 0;
    void *group = nullptr;          // column group holding the request's rounds (nullptr: tile engine)
    int gcol = -1;
    double *dout = nullptr;         // normalised result (device, own allocation: outlives the state)
    size_t out_bytes = 0;
    pr_stats st{};
    std::chrono::steady_clock::time_point t_submit;
    template <typename X> X *at(size_t off) const { return reinterpret_cast<X *>(static_cast<char *>(mem) + off); }
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// device bytes of a request and the offsets of its arrays
size_t layout(SReq &q) {
    const size_t n = q.g->G.n, nnd = std::max(q.g->G.n_nd, 1);
    size_t used = 0;
    auto take = [&](size_t b) {
        const size_t at = used;
        used += align256(b);
        return at;
    };
    const bool fp32 = q.prec == PR_FP32;
    const size_t tb = fp32 ? sizeof(float) : sizeof(float2), vb = fp32 ? sizeof(float) : sizeof(float2);
    auto state = [&](size_t t_bytes, size_t v_bytes) {
        StateOffsets o{};
        o.x = take(t_bytes * n);
        o.r = take(t_bytes * n);
        o.vbuf = take(t_bytes * nnd);
        o.w0 = take(v_bytes * nnd);
        o.w1 = take(v_bytes * nnd);
        o.bins = take(sizeof(int32_t) * 3 * nnd);
        o.q = take(v_bytes * n);
        if (t_bytes == sizeof(float2)) o.din = take(sizeof(double) * n);  // double-float state only
        return o;
    };
    q.off_ctl = take(sizeof(Ctl));
    q.s_main = state(tb, vb);
    if (fp32) {
        q.s64 = state(sizeof(double), sizeof(double));
        q.off_qc = take(sizeof(double) * n);
        q.off_p64 = take(sizeof(double) * n);
    }
    q.off_sidx = take(sizeof(int32_t) * std::max(q.nnz, 1));
    q.off_sval = take(sizeof(double) * std::max(q.nnz, 1));
    return used;
}

RoundBuf req_buf(const SReq &q, const StateOffsets &o) {
    return RoundBuf{q.at<char>(o.x), q.at<char>(o.r), q.at<char>(o.vbuf), {q.at<char>(o.w0), q.at<char>(o.w1)},
                    q.at<int32_t>(o.bins), o.din ? q.at<double>(o.din) : nullptr};
}

}  // namespace

struct ServerImpl {
    // K requests on one graph whose rounds share every gather (pr_group.cu)
    struct Group {
        pr_graph *g = nullptr;
        int fmt = 0;  // 0: float state, 1: double-float
        void *mem = nullptr;
        size_t bytes = 0;
        GroupDev D{};
        SReq *col[8] = {};
        int32_t next_launch = 0;
        int live() const {
            int c = 0;
            for (int k = 0; k < group_columns(fmt); k++) c += col[k] != nullptr;
            return c;
        }
    };
    std::vector<Group *> groups;
    pr_server_stats stats{};  // written by the server thread under mu
    using Clock = std::chrono::steady_clock;
    void add_ms(double pr_server_stats::*field, Clock::time_point t0) {
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        std::lock_guard<std::mutex> lock(mu);
        stats.*field += ms;
    }
    std::unordered_map<uint64_t, int> inflight;  // requests per graph (uid), submitted and not finished
    int32_t group_min_rows = 1 << 14;            // smaller graphs run in the tile engine
    Buf d_gctl, d_gstat;
    cudaStream_t s = nullptr;
    cudaStream_t ps = nullptr;  // copies of results to callers (pr_server_poll)
    // The server's own memory pool.  It keeps what it has reserved until the
    // server is destroyed: with the device's default pool, memory freed by a
    // finished request went back to the driver at the next synchronisation and
    // every admission mapped it again, a cost that grew with the requests in flight.
    cudaMemPool_t pool = nullptr;
    int device = 0, sms = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool stop = false;
    int64_t next_ticket = 1;
    size_t queue_cap = 1 << 16;
    std::deque<SReq *> queue;
    std::unordered_map<int64_t, SReq *> reqs;
    // [0] FP32 requests in their FP32 rounds, [1] double-float requests, [2] FP32
    // requests in their FP64 rounds after the correction
    std::vector<SReq *> act[3];
    // per-graph tile templates (prob index filled in when a table is built)
    struct Tiles {
        std::vector<Tile> round, vert, dang;
        uint64_t plan_gen = 0;  // the graph's plans they were cut from
    };
    std::unordered_map<uint64_t, Tiles> tiles;  // by pr_graph::uid
    // device tables of the current step (grow-only)
    Buf d_probs[3], d_tiles[3], d_bc[3], d_slots, d_stat, d_fprobs, d_ftiles, d_fdtiles, d_fvtiles;
    int ntiles[3] = {0, 0, 0};
    bool dirty[3] = {true, true, true};
    pr_status loop_error = PR_OK;
    std::string loop_msg;

    const Tiles &tiles_of(pr_graph *g) {
        auto it = tiles.find(g->uid);
        if (it != tiles.end() && it->second.plan_gen == g->plan_gen) return it->second;
        if (it != tiles.end()) tiles.erase(it);  // retuned since: cut again
        Tiles T;
        T.plan_gen = g->plan_gen;
        cut_plan(g->plan_nd, 0, T.round);
        if (T.round.empty()) T.round.push_back(Tile{0, 0, 0, 1});
        cut_rows(0, g->G.n, 0, T.vert);
        cut_plan(g->plan_d, 0, T.dang);
        return tiles.emplace(g->uid, std::move(T)).first->second;
    }

    // table entry of a request in the state of act[fmt]: 0 the FP32 rounds, 1 a
    // double-float request, 2 the FP64 rounds of an FP32 request after correction
    BProb prob_of(SReq *q, int fmt) {
        BProb P{};
        P.G = q->g->G;
        P.ctl = q->at<Ctl>(q->off_ctl);
        const StateOffsets &o = fmt == 2 ? q->s64 : q->s_main;
        P.B = req_buf(*q, o);
        P.q = q->at<char>(o.q);
        P.out = q->dout;
        if (q->prec == PR_FP32) {
            P.qc = q->at<double>(q->off_qc);
            P.pv = PVals{q->at<double>(q->off_p64), nullptr, nullptr};
        }
        return P;
    }

    // copy a problem table and its tiles to the device; returns the tile count
    pr_status upload(const std::vector<SReq *> &set, int fmt, int which, Buf &dp, Buf &dt,
                     std::vector<BProb> &hp, std::vector<Tile> &ht) {
        hp.clear();
        ht.clear();
        for (size_t k = 0; k < set.size(); k++) {
            BProb P = prob_of(set[k], fmt);
            const Tiles &T = tiles_of(set[k]->g);
            const std::vector<Tile> &src = which == 0 ? T.round : (which == 1 ? T.vert : T.dang);
            const int base = (int)ht.size();
            for (Tile t : src) {
                t.prob = (int32_t)k;
                ht.push_back(t);
            }
            if (which == 0) {
                P.t0 = base;
                P.nt = (int)src.size();
            } else if (which == 1) {
                P.v0 = base;
                P.nv = (int)src.size();
            } else {
                P.d0 = base;
                P.nd = (int)src.size();
            }
            hp.push_back(P);
        }
        const size_t pb = sizeof(BProb) * std::max<size_t>(hp.size(), 1), tb = sizeof(Tile) * std::max<size_t>(ht.size(), 1);
        if (dp.bytes < pb) PR_TRY(dp.alloc_async(pb * 2, s, pool));
        if (dt.bytes < tb) PR_TRY(dt.alloc_async(tb * 2, s, pool));
        if (!hp.empty()) PR_CK(cudaMemcpyAsync(dp.p, hp.data(), sizeof(BProb) * hp.size(), cudaMemcpyHostToDevice, s));
        if (!ht.empty()) PR_CK(cudaMemcpyAsync(dt.p, ht.data(), sizeof(Tile) * ht.size(), cudaMemcpyHostToDevice, s));
        return PR_OK;
    }

    pr_status admit_one(SReq *q) {
        q->bytes = layout(*q);
        q->out_bytes = sizeof(double) * (size_t)q->g->G.n;
        PR_CK(cudaMallocFromPoolAsync(&q->mem, q->bytes, pool, s));
        PR_CK(cudaMallocFromPoolAsync(reinterpret_cast<void **>(&q->dout), q->out_bytes, pool, s));
        const DevGraph &G = q->g->G;
        Ctl h{};
        h.c = q->c;
        h.one_minus_c = 1.0 - q->c;
        h.eps = q->eps;
        h.xi = q->eps / (double)std::max(G.n_nd, 1);
        h.pull_edges = q->g->pull_ratio * (double)std::max<int64_t>(G.m - q->g->info.m_d, 1);
        h.pu = q->nnz < 0 ? 1.0 / (double)G.n : 0.0;
        h.p_dense = (q->prec == PR_FP32 && q->nnz >= 0) ? 1 : 0;
        h.algo = PR_IFP2;
        h.policy = 0;
        h.max_rounds = 100000;
        h.scan_ref = q->g->scan_nd_ref;
        h.scan_unref = q->g->scan_nd_unref;
        h.mode = MODE_ACT;
        h.want_bins = 1;
        h.unref_active = 1;
        fill_formats(h);
        PR_CK(cudaMemcpyAsync(q->at<Ctl>(q->off_ctl), &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        for (const StateOffsets *o : {&q->s_main, &q->s64})  // double-float inboxes start empty
            if (o->din) PR_CK(cudaMemsetAsync(q->at<char>(o->din), 0, sizeof(double) * G.n, s));
        double *p64 = q->prec == PR_FP32 ? q->at<double>(q->off_p64) : nullptr;
        const int grid = (int)std::min<int64_t>((G.n + kThreads - 1) / kThreads, (int64_t)sms * 8);
        const int32_t *sidx = q->at<int32_t>(q->off_sidx);
        const double *sval = q->at<double>(q->off_sval);
        if (q->nnz > 0) {
            PR_CK(cudaMemcpyAsync(q->at<int32_t>(q->off_sidx), q->idx.data(), sizeof(int32_t) * q->nnz,
                                  cudaMemcpyHostToDevice, s));
            PR_CK(cudaMemcpyAsync(q->at<double>(q->off_sval), q->val.data(), sizeof(double) * q->nnz,
                                  cudaMemcpyHostToDevice, s));
        }
        const double pu = 1.0 / (double)G.n;
        if (q->prec == PR_FP32) {
            float *x = q->at<float>(q->s_main.x), *r = q->at<float>(q->s_main.r);
            k_req_init<float><<<grid, kThreads, 0, s>>>(G.n, x, r, pu, sidx, sval, q->nnz, G.inv, p64);
            if (q->nnz > 0) k_req_seed_par<float><<<8, kThreads, 0, s>>>(r, sidx, sval, q->nnz, G.inv, p64);
        } else {
            float2 *x = q->at<float2>(q->s_main.x), *r = q->at<float2>(q->s_main.r);
            k_req_init<float2><<<grid, kThreads, 0, s>>>(G.n, x, r, pu, sidx, sval, q->nnz, G.inv, p64);
            if (q->nnz > 0) k_req_seed_par<float2><<<8, kThreads, 0, s>>>(r, sidx, sval, q->nnz, G.inv, p64);
        }
        PR_CK(cudaGetLastError());
        return PR_OK;
    }

    // FP32 requests that stopped: the IEEE FP64 correction, then FP64 rounds
    pr_status correct(const std::vector<SReq *> &set) {
        std::vector<BProb> hp;
        std::vector<Tile> hv, hr;
        PR_TRY(upload(set, 0, 1, d_fprobs, d_fvtiles, hp, hv));
        // the same problems with their round tiles (a second table in d_fdtiles)
        std::vector<BProb> hp2;
        PR_TRY(upload(set, 0, 0, d_fprobs, d_ftiles, hp2, hr));
        // merge: vertex tile indices in hp, round tile indices in hp2 (same order)
        for (size_t k = 0; k < hp.size(); k++) {
            hp[k].t0 = hp2[k].t0;
            hp[k].nt = hp2[k].nt;
        }
        PR_CK(cudaMemcpyAsync(d_fprobs.p, hp.data(), sizeof(BProb) * hp.size(), cudaMemcpyHostToDevice, s));
        std::vector<BProb> h64 = hp;
        for (size_t k = 0; k < set.size(); k++) {
            h64[k].B = req_buf(*set[k], set[k]->s64);
            h64[k].q = set[k]->at<char>(set[k]->s64.q);
        }
        Buf dfp;
        PR_TRY(dfp.alloc_async(sizeof(BProb) * h64.size(), s, pool));
        PR_CK(cudaMemcpyAsync(dfp.p, h64.data(), sizeof(BProb) * h64.size(), cudaMemcpyHostToDevice, s));
        const int nv = (int)hv.size(), nr = (int)hr.size();
        const int g1 = (int)std::min<int64_t>(std::max(nv, 1), (int64_t)sms * 16);
        const int g2 = (int)std::min<int64_t>(std::max(nr, 1), (int64_t)sms * 16);
        const BProb *dp = d_fprobs.as<BProb>();
        k_batch_to_fp64<true><<<g1, kThreads, 0, s>>>(dp, dfp.as<BProb>(), d_fvtiles.as<Tile>(), nv);
        k_batch_correct<<<g2, kThreads, 0, s>>>(dfp.as<BProb>(), d_ftiles.as<Tile>(), nr);
        Buf bcb;
        PR_TRY(bcb.alloc_async(sizeof(BCtl), s, pool));
        k_batch_reset<<<((int)set.size() + kThreads - 1) / kThreads, kThreads, 0, s>>>(dfp.as<BProb>(), (int)set.size(),
                                                                                     bcb.as<BCtl>());
        PR_CK(cudaStreamSynchronize(s));
        PR_CK(cudaGetLastError());
        return PR_OK;
    }

    // stopped requests: phase 2, normalisation, release; per state format
    // (1 double-float, 2 FP64 after the correction of an FP32 request)
    pr_status finish(const std::vector<SReq *> &set, const std::vector<int> &fmt) {
        for (int f = 1; f <= 2; f++) {
            std::vector<SReq *> part;
            for (size_t k = 0; k < set.size(); k++)
                if (fmt[k] == f) part.push_back(set[k]);
            if (!part.empty()) PR_TRY(finish_fmt(part, f));
        }
        return PR_OK;
    }

    pr_status finish_fmt(const std::vector<SReq *> &set, int fmt) {
        std::vector<BProb> hp;
        std::vector<Tile> hv, hd;
        // per-request format: build the table by hand
        for (size_t k = 0; k < set.size(); k++) {
            BProb P = prob_of(set[k], fmt);
            const Tiles &T = tiles_of(set[k]->g);
            P.v0 = (int)hv.size();
            for (Tile t : T.vert) {
                t.prob = (int32_t)k;
                hv.push_back(t);
            }
            P.nv = (int)T.vert.size();
            P.d0 = (int)hd.size();
            for (Tile t : T.dang) {
                t.prob = (int32_t)k;
                hd.push_back(t);
            }
            P.nd = (int)T.dang.size();
            hp.push_back(P);
        }
        if (d_fprobs.bytes < sizeof(BProb) * hp.size()) PR_TRY(d_fprobs.alloc_async(sizeof(BProb) * hp.size() * 2, s, pool));
        if (d_fvtiles.bytes < sizeof(Tile) * std::max<size_t>(hv.size(), 1))
            PR_TRY(d_fvtiles.alloc_async(sizeof(Tile) * std::max<size_t>(hv.size(), 1) * 2, s, pool));
        if (d_fdtiles.bytes < sizeof(Tile) * std::max<size_t>(hd.size(), 1))
            PR_TRY(d_fdtiles.alloc_async(sizeof(Tile) * std::max<size_t>(hd.size(), 1) * 2, s, pool));
        PR_CK(cudaMemcpyAsync(d_fprobs.p, hp.data(), sizeof(BProb) * hp.size(), cudaMemcpyHostToDevice, s));
        PR_CK(cudaMemcpyAsync(d_fvtiles.p, hv.data(), sizeof(Tile) * hv.size(), cudaMemcpyHostToDevice, s));
        if (!hd.empty()) PR_CK(cudaMemcpyAsync(d_fdtiles.p, hd.data(), sizeof(Tile) * hd.size(), cudaMemcpyHostToDevice, s));
        const int nv = (int)hv.size(), nd = (int)hd.size();
        if (d_slots.bytes < sizeof(double) * std::max(nv, 1)) PR_TRY(d_slots.alloc_async(sizeof(double) * std::max(nv, 1) * 2, s, pool));
        const int g1 = (int)std::min<int64_t>(std::max(nv, 1), (int64_t)sms * 16);
        const int g2 = (int)std::min<int64_t>(std::max(nd, 1), (int64_t)sms * 16);
        const BProb *dp = d_fprobs.as<BProb>();
        if (fmt == 2) {
            k_batch_phase2_q<double><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv);
            if (nd) k_batch_phase2<double><<<g2, kThreads, 0, s>>>(dp, d_fdtiles.as<Tile>(), nd);
            k_batch_fin_sum<double><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv, PR_IFP2, d_slots.as<double>());
            k_batch_fin_write<double><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv, PR_IFP2);
        } else {
            k_batch_phase2_q<float2><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv);
            if (nd) k_batch_phase2<float2><<<g2, kThreads, 0, s>>>(dp, d_fdtiles.as<Tile>(), nd);
            k_batch_fin_sum<float2><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv, PR_IFP2, d_slots.as<double>());
            k_batch_fin_write<float2><<<g1, kThreads, 0, s>>>(dp, d_fvtiles.as<Tile>(), nv, PR_IFP2);
        }
        std::vector<Ctl> hc(set.size());
        for (size_t k = 0; k < set.size(); k++)  // results stay on the device until polled
            PR_CK(cudaMemcpyAsync(&hc[k], set[k]->at<Ctl>(set[k]->off_ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        PR_CK(cudaGetLastError());
        const auto now = std::chrono::steady_clock::now();
        for (size_t k = 0; k < set.size(); k++) {
            SReq *q = set[k];
            const Ctl &h = hc[k];
            std::memset(&q->st, 0, sizeof(q->st));
            q->st.rounds = h.round;
            q->st.rounds_push = h.rounds_push;
            q->st.rounds_pull = h.rounds_pull;
            q->st.fp64_rounds = q->prec == PR_FP32 ? h.round - q->rounds_first : 0;
            q->st.pushes = h.pushes;
            q->st.edges_pushed = h.edges_pushed + q->g->info.m_d;
            q->st.edges_scanned = h.edges_scanned + q->g->info.m_d;
            q->st.resid_l1 = h.R;
            q->st.err_bound = 2.0 * h.R / (1.0 - h.c);
            q->st.ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
            q->st.p_scale = q->p_scale;
            q->status = h.status == 0 ? PR_OK : PR_ENOTCONV;
            PR_CK(cudaFreeAsync(q->mem, s));
            q->mem = nullptr;
        }
        return PR_OK;
    }

    bool any_active() const {
        if (!act[0].empty() || !act[1].empty() || !act[2].empty()) return true;
        for (const Group *G : groups)
            if (G->live()) return true;
        return false;
    }

    // put a just-admitted request into a column group of its graph when the
    // graph is large and has at least PR_GROUP_MIN_INFLIGHT requests in
    // flight; false: tile engine
    bool try_group(SReq *q) {
        if (q->g->G.n_nd < group_min_rows) return false;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (inflight[q->g->uid] < PR_GROUP_MIN_INFLIGHT) return false;
        }
        const int fmt = q->prec == PR_FP32 ? 0 : 1;
        const int K = group_columns(fmt);
        Group *G = nullptr;
        int col = -1;
        for (Group *gr : groups) {
            if (gr->g != q->g || gr->fmt != fmt) continue;
            for (int k = 0; k < K && col < 0; k++)
                if (!gr->col[k]) col = k;
            if (col >= 0) {
                G = gr;
                break;
            }
        }
        if (!G) {
            int ng = 0;
            for (const Group *gr : groups) ng += gr->g == q->g && gr->fmt == fmt;
            if (ng >= PR_SERVER_MAX_GROUPS) return false;
            const size_t gb = group_bytes(q->g, fmt);
            {
                std::lock_guard<std::mutex> lock(mu);
                if (used + gb > budget) return false;
                used += gb;
            }
            G = new (std::nothrow) Group();
            void *mem = nullptr;
            if (!G || cudaMallocFromPoolAsync(&mem, gb, pool, s) != cudaSuccess) {
                cudaGetLastError();
                delete G;
                std::lock_guard<std::mutex> lock(mu);
                used -= gb;
                return false;
            }
            G->g = q->g;
            G->fmt = fmt;
            G->mem = mem;
            G->bytes = gb;
            group_layout(q->g, fmt, mem, G->D);
            for (int k = 0; k < 8; k++) {
                G->D.ctl[k] = nullptr;
                G->D.join[k] = -1;
            }
            if (cudaMemsetAsync(G->D.ticket, 0, sizeof(uint32_t), s) != cudaSuccess) {
                cudaGetLastError();
                cudaFreeAsync(mem, s);
                delete G;
                std::lock_guard<std::mutex> lock(mu);
                used -= gb;
                return false;
            }
            groups.push_back(G);
            col = 0;
        }
        G->col[col] = q;
        G->D.ctl[col] = q->at<Ctl>(q->off_ctl);
        G->D.join[col] = G->next_launch;
        if (group_load(q->g, G->D, fmt, col, q->at<char>(q->s_main.x), q->at<char>(q->s_main.r), s) != PR_OK) {
            G->col[col] = nullptr;
            G->D.ctl[col] = nullptr;
            G->D.join[col] = -1;
            return false;
        }
        q->group = G;
        q->gcol = col;
        return true;
    }

    void release_group_if_empty(Group *G) {
        if (G->live()) return;
        cudaFreeAsync(G->mem, s);
        {
            std::lock_guard<std::mutex> lock(mu);
            used -= G->bytes;
        }
        groups.erase(std::find(groups.begin(), groups.end(), G));
        delete G;
    }

    // a few rounds of every group, then its finished columns leave: FP32
    // requests go on to the correction, double-float requests to the finish
    pr_status step_groups(int phases) {
        std::vector<std::pair<Group *, int>> cols;
        std::vector<Ctl *> ptrs;
        const auto t_rounds = Clock::now();
        int64_t launched = 0;
        for (Group *G : groups) {
            if (!G->live()) continue;
            for (int k = 0; k < phases; k++) PR_TRY(group_round(G->g, G->D, G->fmt, G->next_launch++, s));
            launched += phases;
            for (int k = 0; k < group_columns(G->fmt); k++)
                if (G->col[k]) {
                    cols.emplace_back(G, k);
                    ptrs.push_back(G->D.ctl[k]);
                }
        }
        if (cols.empty()) return PR_OK;
        const int cnt = (int)cols.size();
        if (d_gctl.bytes < sizeof(Ctl *) * cnt) PR_TRY(d_gctl.alloc_async(sizeof(Ctl *) * cnt * 2, s, pool));
        if (d_gstat.bytes < sizeof(ReqStat) * cnt) PR_TRY(d_gstat.alloc_async(sizeof(ReqStat) * cnt * 2, s, pool));
        PR_CK(cudaMemcpyAsync(d_gctl.p, ptrs.data(), sizeof(Ctl *) * cnt, cudaMemcpyHostToDevice, s));
        k_gather_ctls<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, s>>>(d_gctl.as<Ctl *>(), cnt,
                                                                           d_gstat.as<ReqStat>());
        std::vector<ReqStat> hs(cnt);
        PR_CK(cudaMemcpyAsync(hs.data(), d_gstat.p, sizeof(ReqStat) * cnt, cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        PR_CK(cudaGetLastError());
        add_ms(&pr_server_stats::ms_rounds, t_rounds);
        {
            std::lock_guard<std::mutex> lock(mu);
            stats.group_launches += launched;
        }
        std::vector<SReq *> to_correct, to_finish;
        std::vector<int> fin_fmt;
        std::vector<Group *> touched;
        for (int i = 0; i < cnt; i++) {
            if (!hs[i].done) continue;
            Group *G = cols[i].first;
            const int k = cols[i].second;
            SReq *q = G->col[k];
            PR_TRY(group_extract(G->g, G->D, G->fmt, k, q->at<char>(q->s_main.x), q->at<char>(q->s_main.r), s));
            G->col[k] = nullptr;
            G->D.ctl[k] = nullptr;
            G->D.join[k] = -1;
            q->group = nullptr;
            q->gcol = -1;
            touched.push_back(G);
            if (q->prec == PR_FP32) {
                q->rounds_first = hs[i].round;
                to_correct.push_back(q);
            } else {
                to_finish.push_back(q);
                fin_fmt.push_back(1);
            }
        }
        if (!to_correct.empty()) {
            const auto t0 = Clock::now();
            PR_TRY(correct(to_correct));
            add_ms(&pr_server_stats::ms_correct, t0);
            for (SReq *q : to_correct) {
                q->stage = 2;
                act[2].push_back(q);
            }
            dirty[2] = true;
        }
        if (!to_finish.empty()) {
            const auto t0 = Clock::now();
            PR_TRY(finish(to_finish, fin_fmt));
            add_ms(&pr_server_stats::ms_finish, t0);
            complete(to_finish);
        }
        for (Group *G : touched)
            if (std::find(groups.begin(), groups.end(), G) != groups.end()) release_group_if_empty(G);
        return PR_OK;
    }

    // finished requests: results are on the host; free their budget share
    void complete(const std::vector<SReq *> &done) {
        std::lock_guard<std::mutex> lock(mu);
        stats.finished += (int64_t)done.size();
        for (SReq *q : done) {
            q->stage = 3;
            used -= q->bytes;
            auto it = inflight.find(q->g->uid);
            if (it != inflight.end() && --it->second <= 0) inflight.erase(it);
        }
        cv.notify_all();
    }

    pr_status step_once() {
        const auto t_step = Clock::now();
        const pr_status st = step_body();
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t_step).count();
        std::lock_guard<std::mutex> lock(mu);
        stats.ms_step_max = std::max(stats.ms_step_max, ms);
        return st;
    }

    pr_status step_body() {
        // admit
        std::vector<SReq *> adm;
        {
            std::lock_guard<std::mutex> lock(mu);
            stats.queued_sum += (int64_t)queue.size();
            // free group columns per (graph, format), counting the groups that may still be made
            std::unordered_map<uint64_t, int> free_cols;
            auto key_of = [](const SReq *q) { return (q->g->uid << 1) | (q->prec == PR_FP32 ? 0u : 1u); };
            auto cols_of = [&](const SReq *q) -> int & {
                const uint64_t key = key_of(q);
                auto it = free_cols.find(key);
                if (it != free_cols.end()) return it->second;
                const int fmt = q->prec == PR_FP32 ? 0 : 1, K = group_columns(fmt);
                int freec = 0, ng = 0;
                for (const Group *G : groups)
                    if (G->g == q->g && G->fmt == fmt) {
                        ng++;
                        freec += K - G->live();
                    }
                freec += std::max(0, PR_SERVER_MAX_GROUPS - ng) * K;
                return free_cols.emplace(key, freec).first->second;
            };
            for (auto it = queue.begin(); it != queue.end();) {
                SReq *q = *it;
                const size_t need = layout(*q) + sizeof(double) * (size_t)q->g->G.n;
                if (used + need > budget && (any_active() || !adm.empty())) break;
                // a request headed for a column group waits for a free column
                const bool grouped = q->g->G.n_nd >= group_min_rows && inflight[q->g->uid] >= PR_GROUP_MIN_INFLIGHT;
                if (grouped && (any_active() || !adm.empty())) {
                    int &fc = cols_of(q);
                    if (fc <= 0) {
                        ++it;
                        continue;
                    }
                    fc--;
                }
                it = queue.erase(it);
                used += need;
                adm.push_back(q);
            }
        }
        const auto t_adm = Clock::now();
        for (SReq *q : adm) {
            PR_TRY(admit_one(q));
            q->stage = 1;
            if (try_group(q)) continue;
            const int f = q->prec == PR_FP32 ? 0 : 1;
            act[f].push_back(q);
            dirty[f] = true;
        }
        if (!adm.empty()) add_ms(&pr_server_stats::ms_admit, t_adm);
        {
            int64_t running = (int64_t)(act[0].size() + act[1].size() + act[2].size());
            for (const Group *G : groups) running += G->live();
            std::lock_guard<std::mutex> lock(mu);
            stats.steps++;
            stats.running_sum += running;
        }
        // a few rounds of every request, per state format (groups first)
        constexpr int kPhases = 4;
        PR_TRY(step_groups(kPhases));
        if (act[0].empty() && act[1].empty() && act[2].empty()) return PR_OK;
        std::vector<BProb> hp;
        std::vector<Tile> ht;
        for (int f = 0; f < 3; f++) {
            if (act[f].empty()) continue;
            if (dirty[f]) {
                const auto t_tab = Clock::now();
                PR_TRY(upload(act[f], f, 0, d_probs[f], d_tiles[f], hp, ht));
                add_ms(&pr_server_stats::ms_tables, t_tab);
                ntiles[f] = (int)ht.size();
                if (!d_bc[f].p) PR_TRY(d_bc[f].alloc_async(sizeof(BCtl), s, pool));
                PR_CK(cudaMemsetAsync(d_bc[f].p, 0, sizeof(BCtl), s));
                const size_t sb = (sizeof(double) * 2 + sizeof(long long) * 2) * std::max(ntiles[f], 1);
                if (d_slots.bytes < sb) PR_TRY(d_slots.alloc_async(sb * 2, s, pool));
                dirty[f] = false;
            }
            const int nt = ntiles[f];
            double *base = d_slots.as<double>();
            BSlots sl{base, reinterpret_cast<long long *>(base + nt), reinterpret_cast<long long *>(base + 2 * nt),
                      reinterpret_cast<int *>(base + 3 * nt)};
            const int grid = sms * 6;
            const auto t_tile = Clock::now();
            {
                std::lock_guard<std::mutex> lock(mu);
                stats.tile_launches += kPhases;
            }
            for (int k = 0; k < kPhases; k++) {
                if (f == 0)
                    k_batch_phase<float, true><<<grid, kThreads, 0, s>>>(d_probs[f].as<BProb>(), d_tiles[f].as<Tile>(),
                                                                         nt, d_bc[f].as<BCtl>(), sl);
                else if (f == 1)
                    k_batch_phase<float2, true><<<grid, kThreads, 0, s>>>(d_probs[f].as<BProb>(), d_tiles[f].as<Tile>(),
                                                                          nt, d_bc[f].as<BCtl>(), sl);
                else
                    k_batch_phase<double, true><<<grid, kThreads, 0, s>>>(d_probs[f].as<BProb>(), d_tiles[f].as<Tile>(),
                                                                          nt, d_bc[f].as<BCtl>(), sl);
            }
            // which requests stopped
            const int cnt = (int)act[f].size();
            if (d_stat.bytes < sizeof(ReqStat) * cnt) PR_TRY(d_stat.alloc_async(sizeof(ReqStat) * cnt * 2, s, pool));
            k_gather_status<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, s>>>(d_probs[f].as<BProb>(), cnt,
                                                                                 d_stat.as<ReqStat>());
            std::vector<ReqStat> hs(cnt);
            PR_CK(cudaMemcpyAsync(hs.data(), d_stat.p, sizeof(ReqStat) * cnt, cudaMemcpyDeviceToHost, s));
            PR_CK(cudaStreamSynchronize(s));
            PR_CK(cudaGetLastError());
            add_ms(&pr_server_stats::ms_rounds, t_tile);
            std::vector<SReq *> keep, to_correct, to_finish;
            std::vector<int> fin_fmt;
            for (int k = 0; k < cnt; k++) {
                SReq *q = act[f][k];
                if (!hs[k].done) {
                    keep.push_back(q);
                } else if (f == 0 && q->prec == PR_FP32) {
                    q->rounds_first = hs[k].round;
                    to_correct.push_back(q);
                } else {
                    to_finish.push_back(q);
                    fin_fmt.push_back(f);
                }
            }
            if (keep.size() != act[f].size()) {
                act[f].swap(keep);
                dirty[f] = true;
            }
            if (!to_correct.empty()) {
                const auto t0 = Clock::now();
                PR_TRY(correct(to_correct));
                add_ms(&pr_server_stats::ms_correct, t0);
                for (SReq *q : to_correct) {
                    q->stage = 2;
                    act[2].push_back(q);
                }
                dirty[2] = true;
            }
            if (!to_finish.empty()) {
                const auto t0 = Clock::now();
                PR_TRY(finish(to_finish, fin_fmt));
                add_ms(&pr_server_stats::ms_finish, t0);
                complete(to_finish);
            }
        }
        return PR_OK;
    }

    void loop() {
        cudaSetDevice(device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lock(mu);
                cv.wait_for(lock, std::chrono::milliseconds(5),
                            [&] { return stop || !queue.empty() || any_active(); });
                if (stop) return;
                if (queue.empty() && !any_active()) continue;
            }
            const pr_status st = step_once();
            if (st != PR_OK) {
                std::lock_guard<std::mutex> lock(mu);
                loop_error = st;
                loop_msg = pr_last_error();
                // fail every pending request; the server stays usable for polling
                std::vector<SReq *> failed;
                for (int f = 0; f < 3; f++) {
                    for (SReq *q : act[f]) failed.push_back(q);
                    act[f].clear();
                    dirty[f] = true;
                }
                for (Group *G : groups) {
                    for (int k = 0; k < 8; k++)
                        if (G->col[k]) failed.push_back(G->col[k]);
                    cudaFreeAsync(G->mem, s);
                    used -= G->bytes;
                    delete G;
                }
                groups.clear();
                for (SReq *q : failed) {
                    q->stage = 3;
                    q->status = st;
                    q->group = nullptr;
                    if (q->mem) cudaFreeAsync(q->mem, s);
                    if (q->dout) cudaFreeAsync(q->dout, s);
                    q->mem = nullptr;
                    q->dout = nullptr;
                    used -= q->bytes + q->out_bytes;
                    q->out_bytes = 0;
                    auto it = inflight.find(q->g->uid);
                    if (it != inflight.end() && --it->second <= 0) inflight.erase(it);
                }
                cv.notify_all();
            }
        }
    }
};

}  // namespace pr

struct pr_server {
    pr::ServerImpl impl;
};

using namespace pr;

extern "C" pr_status pr_server_create(size_t hbm_budget_bytes, void *cuda_stream, pr_server **out) {
    if (!out) return fail(PR_EINVAL, "pr_server_create: out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes == 0) return fail(PR_EINVAL, "pr_server_create: budget must be > 0");
    pr_server *S = new (std::nothrow) pr_server();
    if (!S) return fail(PR_ENOMEM, "host allocation failed");
    ServerImpl &I = S->impl;
    I.budget = hbm_budget_bytes;
    I.s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&I.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&I.sms, cudaDevAttrMultiProcessorCount, I.device);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "pr_server_create");
    }
    e = cudaStreamCreateWithFlags(&I.ps, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "pr_server_create (copy stream)");
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = I.device;
    e = cudaMemPoolCreate(&I.pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(I.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        if (I.pool) cudaMemPoolDestroy(I.pool);
        cudaStreamDestroy(I.ps);
        delete S;
        return cuda_fail(e, "pr_server_create (memory pool)");
    }
    I.th = std::thread([&I] { I.loop(); });
    *out = S;
    return PR_OK;
}

extern "C" pr_status pr_server_submit(pr_server *S, pr_graph *g, double c, double eps, pr_prec prec,
                                      const pr_pvec *p, int64_t *ticket) {
    if (!S || !g || !ticket) return fail(PR_EINVAL, "pr_server_submit: NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(PR_EINVAL, "c must be in (0, 1)");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(PR_EINVAL, "eps must be positive and finite");
    if (prec != PR_FP32 && prec != PR_DF64) return fail(PR_EINVAL, "pr_server_submit: prec must be FP32 or DF64");
    ServerImpl &I = S->impl;
    SReq *q = new (std::nothrow) SReq();
    if (!q) return fail(PR_ENOMEM, "host allocation failed");
    q->g = g;
    q->c = c;
    q->eps = eps;
    q->prec = prec;
    q->t_submit = std::chrono::steady_clock::now();
    const int32_t n = g->G.n;
    if (p && p->nnz >= 0) {
        if (p->is_device) {
            delete q;
            return fail(PR_EINVAL, "pr_server_submit: p must be in host memory");
        }
        const bool dense = p->nnz == n && p->idx == nullptr;
        double sum = 0.0;
        for (int32_t k = 0; k < p->nnz; k++) {
            const double v = p->val[k];
            const int32_t i = dense ? k : p->idx[k];
            if (!(v >= 0.0) || !std::isfinite(v) || i < 0 || i >= n) {
                delete q;
                return fail(PR_EINVAL, "pr_server_submit: bad personalization entry");
            }
            if (v > 0.0) {
                q->idx.push_back(i);
                q->val.push_back(v);
                sum += v;
            }
        }
        if (!(sum > 0.0)) {
            delete q;
            return fail(PR_EINVAL, "p sums to zero");
        }
        for (double &v : q->val) v /= sum;
        q->p_scale = 1.0 / sum;
        q->nnz = (int32_t)q->idx.size();
    }
    const size_t need = layout(*q);
    if (need > I.budget) {
        delete q;
        return fail(PR_EINVAL, "pr_server_submit: one request needs more device memory than the budget");
    }
    std::lock_guard<std::mutex> lock(I.mu);
    if (I.queue.size() >= I.queue_cap) {
        delete q;
        return fail(PR_EAGAIN, "pr_server_submit: queue full");
    }
    q->ticket = I.next_ticket++;
    I.reqs[q->ticket] = q;
    I.queue.push_back(q);
    I.inflight[g->uid]++;
    I.stats.submitted++;
    *ticket = q->ticket;
    I.cv.notify_all();
    return PR_OK;
}

extern "C" pr_status pr_server_poll(pr_server *S, int64_t ticket, double *out, pr_stats *st) {
    if (!S) return fail(PR_EINVAL, "pr_server_poll: NULL server");
    ServerImpl &I = S->impl;
    SReq *q = nullptr;
    std::string msg;
    {
        std::lock_guard<std::mutex> lock(I.mu);
        auto it = I.reqs.find(ticket);
        if (it == I.reqs.end()) return fail(PR_EINVAL, "pr_server_poll: unknown ticket");
        if (it->second->stage != 3) return PR_EBUSY;
        q = it->second;
        I.reqs.erase(it);
        msg = I.loop_msg;
    }
    // the result was completed (and the server's stream synchronised) before
    // the request was marked done: copy it on the copy stream, outside the lock
    const pr_status status = q->status;
    pr_status ret = status;
    if (q->dout) {
        int old = -1;
        cudaGetDevice(&old);
        if (old != I.device) cudaSetDevice(I.device);
        cudaError_t e = cudaSuccess;
        if (out && (status == PR_OK || status == PR_ENOTCONV))
            e = cudaMemcpyAsync(out, q->dout, q->out_bytes, cudaMemcpyDefault, I.ps);
        if (e == cudaSuccess) e = cudaFreeAsync(q->dout, I.ps);
        if (e == cudaSuccess) e = cudaStreamSynchronize(I.ps);
        if (old >= 0 && old != I.device) cudaSetDevice(old);
        if (e != cudaSuccess) ret = cuda_fail(e, "pr_server_poll (result copy)");
        std::lock_guard<std::mutex> lock(I.mu);
        I.used -= q->out_bytes;
    }
    if (st && (status == PR_OK || status == PR_ENOTCONV)) *st = q->st;
    delete q;
    if (ret == PR_ECUDA) return ret;
    if (status != PR_OK) return fail(status, msg.empty() ? "request did not converge" : msg);
    return PR_OK;
}

extern "C" pr_status pr_server_get_stats(pr_server *S, pr_server_stats *out) {
    if (!S || !out) return fail(PR_EINVAL, "pr_server_get_stats: NULL argument");
    ServerImpl &I = S->impl;
    std::lock_guard<std::mutex> lock(I.mu);
    *out = I.stats;
    int live = 0;
    for (const ServerImpl::Group *G : I.groups) live += G->live() > 0;
    out->groups = live;
    out->active = (int32_t)(I.stats.submitted - I.stats.finished - (int64_t)I.queue.size());
    return PR_OK;
}

extern "C" void pr_server_destroy(pr_server *S) {
    if (!S) return;
    ServerImpl &I = S->impl;
    {
        std::lock_guard<std::mutex> lock(I.mu);
        I.stop = true;
    }
    I.cv.notify_all();
    if (I.th.joinable()) I.th.join();
    cudaStreamSynchronize(I.s);
    for (ServerImpl::Group *G : I.groups) {
        cudaFreeAsync(G->mem, I.s);
        delete G;
    }
    I.groups.clear();
    for (auto &kv : I.reqs) {
        if (kv.second->mem) cudaFreeAsync(kv.second->mem, I.s);
        if (kv.second->dout) cudaFreeAsync(kv.second->dout, I.s);
        delete kv.second;
    }
    for (Buf *b : {&I.d_gctl, &I.d_gstat, &I.d_slots, &I.d_stat, &I.d_fprobs, &I.d_ftiles, &I.d_fdtiles,
                   &I.d_fvtiles})
        b->release();
    for (int f = 0; f < 3; f++) {
        I.d_probs[f].release();
        I.d_tiles[f].release();
        I.d_bc[f].release();
    }
    cudaStreamSynchronize(I.s);
    cudaStreamSynchronize(I.ps);
    if (I.ps) cudaStreamDestroy(I.ps);
    if (I.pool) cudaMemPoolDestroy(I.pool);  // every allocation from it has been freed above
    delete S;
}
