// pr_group.cu -- column groups: K IFP2 solves on the same graph advanced by one
// gather per round.
//
// Requests served on one resident graph (personalized PageRank with different
// seeds, or different damping factors) run the same rounds over the same
// in-lists.  A group keeps K of them side by side: x[i][k], r[i][k] and the
// pending push w[i][k] of column k are contiguous for a vertex, so the K
// columns of one in-list entry's source are one 32-byte sector, read by two
// lanes with 16-byte loads (K = 8 for float state, 4 for double-float).  Each column keeps its own parameters,
// round counter and stopping decision; the arithmetic of a column is that of
// a pull round of the single solve (Alg. 3, synchronous snapshot rounds):
//   commit of round t-1 (x += (1-c) r, r = 0 where |r| > xi),
//   delivery r_j += sum_{i in S(j)} w_{t-1}[i],
//   activation of round t on the new r_j (w_t = c r_j / deg_j where |r_j| > xi),
// with R_t = sum |r_j| over the non-dangling rows for the stop test.  A column
// whose first round this is (its state was just loaded) skips the commit,
// which makes that round the plain activation of the single solve.
#include <algorithm>

#include "pr_internal.cuh"
#include "pr_kernels.cuh"
#include "pr_group.cuh"

namespace pr {
namespace {

template <typename T> struct GK {
    static constexpr int K = 32 / (int)sizeof(typename ST<T>::V);
};

// per-column parameters read once per block
template <typename T, int K> struct ColParams {
    T c[K], om[K], xi[K];
    int act[K], fresh[K];
    int any;
    int use_unref;  // some column's previous round was its first (see k_group_round)
};

// Thread layout: a vertex's K columns are 32 bytes; a lane loads 16 of them
// (CPL = 16 / sizeof(V) columns), so a "slot" of LPE = K / CPL = 2 lanes reads
// one in-list entry: both lanes load the source id (one broadcast) and one
// 16-byte half each of the source's sector.  A row is served by max(LANES, 2)
// lanes (LANES from the graph's pull bins), i.e. by one or more slots, whose
// sums are combined by shuffles across slots.  A lane keeps the partial R, F,
// E of its own CPL columns.
template <typename V> struct Cols {
    static constexpr int CPL = 16 / (int)sizeof(V);
};
template <typename V> struct Half {
    V v[Cols<V>::CPL];
};
template <typename V> __device__ __forceinline__ Half<V> load_half(const V *__restrict__ w, size_t at) {
    static_assert(sizeof(Half<V>) == 16, "half a vertex's columns is 16 bytes");
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(w + at));
    Half<V> h;
    memcpy(&h, &a, 16);
    return h;
}

template <typename T, int K>
__device__ __forceinline__ void column_epilogue(const DevGraph &G, const ColParams<T, K> &P, T *x, T *r,
                                                typename ST<T>::V *wnext, int j, int k, T in,
                                                typename ST<T>::R &Rl, int &Fl, int &El) {
    const size_t at = (size_t)j * K + k;
    const T v = r[at];
    T base = v;
    if (!P.fresh[k] && ST<T>::gt(ST<T>::absv(v), P.xi[k])) {  // commit of round t-1
        x[at] = ST<T>::add(x[at], ST<T>::mul(P.om[k], v));
        base = ST<T>::zero();
    }
    const T rn = ST<T>::add(base, in);
    r[at] = rn;
    Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(rn)));
    const bool act = ST<T>::gt(ST<T>::absv(rn), P.xi[k]);
    wnext[at] = ST<T>::pack(act ? ST<T>::mul(rn, ST<T>::mul(P.c[k], ST<T>::invdeg(G, j))) : ST<T>::zero());
    if (act) {
        Fl += 1;
        El += G.ndeg[j];
    }
}

// this lane's CPL columns summed over the in-list entries e = off[j] + slot,
// + nslots, ... of row j, U entries in flight, in entry order
template <typename T, int K, int U>
__device__ __forceinline__ void slot_sum(const int32_t *__restrict__ off, const int32_t *__restrict__ src, int nsrc, int j,
                                         const typename ST<T>::V *__restrict__ w, int part, int slot, int nslots,
                                         typename GT<typename ST<T>::V>::A *acc) {
    using V = typename ST<T>::V;
    constexpr int CPL = Cols<V>::CPL;
    const int b = __ldg(&off[j + 1]);
    for (int e = __ldg(&off[j]) + slot; e < b; e += U * nslots) {
        int idx[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int ee = e + u * nslots;
            idx[u] = ee < b ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (idx[u] >= 0) {
                const Half<V> h = load_half(w, (size_t)idx[u] * K + part * CPL);
#pragma unroll
                for (int c = 0; c < CPL; c++) acc[c] = GT<V>::add(acc[c], h.v[c]);
            }
        }
    }
}

template <typename T, int K, int LANES>
__device__ __forceinline__ void group_rows(const DevGraph &G, const Seg &S, int lb, const ColParams<T, K> &P, T *x,
                                           T *r, const typename ST<T>::V *wprev, typename ST<T>::V *wnext,
                                           typename ST<T>::R *Rl, int *Fl, int *El) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    constexpr int CPL = Cols<V>::CPL;
    constexpr int LPE = K / CPL;                // lanes per in-list entry
    constexpr int L = LANES > LPE ? LANES : LPE;  // lanes per row
    constexpr int NS = L / LPE;                 // slots per row
    constexpr int RPB = kThreads / L;           // rows per block pass
    constexpr int U = LANES >= 2 && NS == 1 ? 8 : 4;
    const int part = threadIdx.x % LPE;
    const int slot = (threadIdx.x % L) / LPE;
    const int grp = threadIdx.x / L;
    // the plan sized this segment's blocks for LANES lanes per row: spread its
    // rows over the same blocks with L lanes each
    const int stride = S.nblk * RPB;
    for (int base = S.lo + lb * RPB; base < S.hi; base += stride) {
        const int j = base + grp;
        A acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; c++) acc[c] = GT<V>::zero();
        if (j < S.hi) {
            slot_sum<T, K, U>(G.inr_off, G.inr_src, G.n_nd, j, wprev, part, slot, NS, acc);
            if (P.use_unref) slot_sum<T, K, U>(G.inu_off, G.inu_src, G.n_nd, j, wprev, part, slot, NS, acc);
        }
#pragma unroll
        for (int o = L / 2; o >= LPE; o >>= 1)
#pragma unroll
            for (int c = 0; c < CPL; c++) acc[c] = GT<V>::add(acc[c], GT<V>::shfl_xor(acc[c], o, L));
        if (j < S.hi && slot == 0) {
#pragma unroll
            for (int c = 0; c < CPL; c++) {
                const int k = part * CPL + c;
                if (P.act[k])
                    column_epilogue<T, K>(G, P, x, r, wnext, j, k, ST<T>::from_acc(acc[c]), Rl[c], Fl[c], El[c]);
            }
        }
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads, 5) k_group_round(DevGraph G, Plan PL, GroupDev D, int32_t launch_id) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    constexpr int CPL = Cols<V>::CPL;
    constexpr int LPE = K / CPL;
    static_assert(K * sizeof(V) == 32 && LPE * CPL == K, "one 32-byte sector per vertex, 16 bytes per lane");
    __shared__ ColParams<T, K> P;
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        const Ctl *c = D.ctl[k];
        const int act = c != nullptr && D.join[k] >= 0 && D.join[k] <= launch_id && !c->done;
        P.act[k] = act;
        P.fresh[k] = act && D.join[k] == launch_id;
        if (c) {
            P.c[k] = ST<T>::c(c);
            P.om[k] = ST<T>::om(c);
            P.xi[k] = ST<T>::xi(c);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // Unreferenced sources (no in-edges) push only in a column's first
        // round: their residual is never refilled.  Their in-list segment is
        // read in the round after some column's first round, and skipped in
        // every other round (it holds zeros there).
        int any = 0, unref = 0;
        for (int k = 0; k < K; k++) {
            any |= P.act[k];
            unref |= P.act[k] && D.join[k] == launch_id - 1;
        }
        P.any = any;
        P.use_unref = unref;
    }
    __syncthreads();
    if (!P.any) return;  // every block returns: no column is running
    T *x = static_cast<T *>(D.x);
    T *r = static_cast<T *>(D.r);
    const V *wprev = static_cast<const V *>((launch_id & 1) ? D.w[0] : D.w[1]);
    V *wnext = static_cast<V *>((launch_id & 1) ? D.w[1] : D.w[0]);
    int s = 0;
    while (s + 1 < PL.nseg && (int)blockIdx.x >= PL.seg[s + 1].blk0) s++;
    const Seg S = PL.seg[s];
    const int lb = blockIdx.x - S.blk0;
    const int part = threadIdx.x % LPE;  // this lane's columns: part * CPL + c
    R Rl[CPL];
    int Fl[CPL], El[CPL];
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        Rl[c] = ST<T>::rzero();
        Fl[c] = 0;
        El[c] = 0;
    }
    switch (S.lanes) {
        case 1: group_rows<T, K, 1>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        case 2: group_rows<T, K, 2>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        case 4: group_rows<T, K, 4>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        case 8: group_rows<T, K, 8>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        case 16: group_rows<T, K, 16>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        case 32: group_rows<T, K, 32>(G, S, lb, P, x, r, wprev, wnext, Rl, Fl, El); break;
        default: {  // one block per row: kThreads / LPE slots
            __shared__ A sha[kThreads / 32][K];
            const int slot = threadIdx.x / LPE;
            for (int j = S.lo + lb; j < S.hi; j += S.nblk) {
                A acc[CPL];
#pragma unroll
                for (int c = 0; c < CPL; c++) acc[c] = GT<V>::zero();
                slot_sum<T, K, 4>(G.inr_off, G.inr_src, G.n_nd, j, wprev, part, slot, kThreads / LPE, acc);
                if (P.use_unref)
                    slot_sum<T, K, 4>(G.inu_off, G.inu_src, G.n_nd, j, wprev, part, slot, kThreads / LPE, acc);
#pragma unroll
                for (int o = 16; o >= LPE; o >>= 1)
#pragma unroll
                    for (int c = 0; c < CPL; c++) acc[c] = GT<V>::add(acc[c], GT<V>::shfl_xor(acc[c], o, 32));
                __syncthreads();
                if ((threadIdx.x & 31) < LPE)
#pragma unroll
                    for (int c = 0; c < CPL; c++) sha[threadIdx.x >> 5][part * CPL + c] = acc[c];
                __syncthreads();
                if ((int)threadIdx.x < LPE) {
#pragma unroll
                    for (int c = 0; c < CPL; c++) {
                        const int k = part * CPL + c;
                        if (!P.act[k]) continue;
                        A t = GT<V>::zero();
                        for (int w = 0; w < kThreads / 32; w++) t = GT<V>::add(t, sha[w][k]);
                        column_epilogue<T, K>(G, P, x, r, wnext, j, k, ST<T>::from_acc(t), Rl[c], Fl[c], El[c]);
                    }
                }
            }
        }
    }
    // block partials per column: a column's lanes are LPE apart; fold the higher
    // lanes of each warp, then one slot per warp in shared memory
    __shared__ R shr[kThreads / 32][K];
    __shared__ int shf[kThreads / 32][K], she[kThreads / 32][K];
#pragma unroll
    for (int o = 16; o >= LPE; o >>= 1)
#pragma unroll
        for (int c = 0; c < CPL; c++) {
            Rl[c] = ST<T>::radd(Rl[c], ST<T>::rshfl(Rl[c], o));
            Fl[c] += __shfl_down_sync(0xffffffffu, Fl[c], o);
            El[c] += __shfl_down_sync(0xffffffffu, El[c], o);
        }
    const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln < LPE)
#pragma unroll
        for (int c = 0; c < CPL; c++) {
            shr[wid][part * CPL + c] = Rl[c];
            shf[wid][part * CPL + c] = Fl[c];
            she[wid][part * CPL + c] = El[c];
        }
    __syncthreads();
    if (threadIdx.x < K) {
        const int k = threadIdx.x;
        R rv = ST<T>::rzero();
        long long fv = 0, ev = 0;
        for (int w = 0; w < kThreads / 32; w++) {
            rv = ST<T>::radd(rv, shr[w][k]);
            fv += shf[w][k];
            ev += she[w][k];
        }
        const size_t at = (size_t)blockIdx.x * K + k;
        memcpy(reinterpret_cast<char *>(D.slot_r) + 8 * at, &rv, 8);
        D.slot_f[at] = fv;
        D.slot_e[at] = ev;
    }
    if (!last_block(D.ticket)) return;
    // the last block: column totals over all blocks (fixed order) and the decisions
    __shared__ double shd[32];
    __shared__ long long shl[32];
    for (int k = 0; k < K; k++) {
        if (!P.act[k]) continue;  // uniform across the block
        double Rs = 0.0;
        long long F = 0, E = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const size_t at = (size_t)b * K + k;
            R v;
            const unsigned long long bits = __ldcg(reinterpret_cast<const unsigned long long *>(D.slot_r) + at);
            memcpy(&v, &bits, 8);
            Rs += ST<T>::r_to_d(v);
            F += __ldcg(&D.slot_f[at]);
            E += __ldcg(&D.slot_e[at]);
        }
        Rs = block_sum(Rs, shd);
        F = block_sum(F, shl);
        E = block_sum(E, shl);
        if (threadIdx.x == 0) {
            Ctl *c = D.ctl[k];
            const int t = c->round;
            c->R = Rs;
            c->F = F;
            c->E = E;
            if (Rs <= c->eps) {
                c->done = 1;
                c->status = 0;
            } else if (t >= c->max_rounds) {
                c->done = 1;
                c->status = 1;
            } else if (F == 0) {
                c->done = 1;
                c->status = 2;
            } else {
                c->round = t + 1;
                c->cur = t;
                c->pushes += F;
                c->edges_pushed += E;
                c->edges_scanned += c->scan_ref + c->scan_unref;
                c->rounds_pull++;
            }
        }
    }
    if (threadIdx.x == 0) *D.ticket = 0;
}

// column k <- (x, r) of one solve (caller vertex order is not involved: both
// are in the graph's internal order); both pending-push buffers of the column
// are cleared so its first round delivers nothing
template <typename T, int K>
__global__ void k_group_load(int32_t n, int32_t n_nd, GroupDev D, int k, const T *__restrict__ x0,
                             const T *__restrict__ r0) {
    using V = typename ST<T>::V;
    T *x = static_cast<T *>(D.x);
    T *r = static_cast<T *>(D.r);
    V *w0 = static_cast<V *>(D.w[0]);
    V *w1 = static_cast<V *>(D.w[1]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[(size_t)i * K + k] = x0[i];
        r[(size_t)i * K + k] = r0[i];
        if (i < n_nd) {
            w0[(size_t)i * K + k] = GT<V>::zero();
            w1[(size_t)i * K + k] = GT<V>::zero();
        }
    }
}

template <typename T, int K>
__global__ void k_group_extract(int32_t n, GroupDev D, int k, T *__restrict__ x0, T *__restrict__ r0) {
    const T *x = static_cast<const T *>(D.x);
    const T *r = static_cast<const T *>(D.r);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x0[i] = x[(size_t)i * K + k];
        r0[i] = r[(size_t)i * K + k];
    }
}

int grid_rows(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sms * 8)); }

}  // namespace

int group_columns(int fmt) { return fmt == 0 ? GK<float>::K : GK<float2>::K; }

size_t group_bytes(const pr_graph *g, int fmt) {
    const size_t n = g->G.n, nnd = std::max(g->G.n_nd, 1);
    const size_t row = 32;  // K values of one vertex, either format
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return a(row * n) * 2 + a(row * nnd) * 2 + a((size_t)kMaxBlocks * 8 * 24) + 256;
}

void group_layout(const pr_graph *g, int fmt, void *base, GroupDev &D) {
    const size_t n = g->G.n, nnd = std::max(g->G.n_nd, 1);
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *p = static_cast<char *>(base);
    D.x = p;
    p += a(32 * n);
    D.r = p;
    p += a(32 * n);
    D.w[0] = p;
    p += a(32 * nnd);
    D.w[1] = p;
    p += a(32 * nnd);
    D.slot_r = reinterpret_cast<double *>(p);
    D.slot_f = reinterpret_cast<long long *>(p + (size_t)kMaxBlocks * 8 * 8);
    D.slot_e = reinterpret_cast<long long *>(p + (size_t)kMaxBlocks * 8 * 16);
    p += a((size_t)kMaxBlocks * 8 * 24);
    D.ticket = reinterpret_cast<uint32_t *>(p);
    (void)fmt;
}

pr_status group_round(const pr_graph *g, const GroupDev &D, int fmt, int32_t launch_id, cudaStream_t s) {
    const Plan &PL = g->plan_nd;
    if (g->G.n_nd == 0) return PR_OK;
    if (fmt == 0) k_group_round<float, 8><<<PL.nblocks, kThreads, 0, s>>>(g->G, PL, D, launch_id);
    else k_group_round<float2, 4><<<PL.nblocks, kThreads, 0, s>>>(g->G, PL, D, launch_id);
    PR_CK(cudaGetLastError());
    return PR_OK;
}

pr_status group_load(const pr_graph *g, const GroupDev &D, int fmt, int col, const void *x, const void *r,
                     cudaStream_t s) {
    const int grid = grid_rows(g->G.n, std::max(g->num_sms, 1));
    if (fmt == 0)
        k_group_load<float, 8><<<grid, kThreads, 0, s>>>(g->G.n, g->G.n_nd, D, col, static_cast<const float *>(x),
                                                          static_cast<const float *>(r));
    else
        k_group_load<float2, 4><<<grid, kThreads, 0, s>>>(g->G.n, g->G.n_nd, D, col, static_cast<const float2 *>(x),
                                                           static_cast<const float2 *>(r));
    PR_CK(cudaGetLastError());
    return PR_OK;
}

pr_status group_extract(const pr_graph *g, const GroupDev &D, int fmt, int col, void *x, void *r, cudaStream_t s) {
    const int grid = grid_rows(g->G.n, std::max(g->num_sms, 1));
    if (fmt == 0)
        k_group_extract<float, 8><<<grid, kThreads, 0, s>>>(g->G.n, D, col, static_cast<float *>(x),
                                                             static_cast<float *>(r));
    else
        k_group_extract<float2, 4><<<grid, kThreads, 0, s>>>(g->G.n, D, col, static_cast<float2 *>(x),
                                                              static_cast<float2 *>(r));
    PR_CK(cudaGetLastError());
    return PR_OK;
}

}  // namespace pr

namespace pr {
// host side of the debug record of this translation unit (column groups)
bool dbg_reset_group(int inject) {
#ifdef PR_DEBUG
    DbgRec z{};
    z.inject = inject;
    return cudaMemcpyToSymbol(g_pr_dbg, &z, sizeof(z)) == cudaSuccess;
#else
    (void)inject;
    return false;
#endif
}
bool dbg_read_group(DbgRec *out) {
#ifdef PR_DEBUG
    return cudaMemcpyFromSymbol(out, g_pr_dbg, sizeof(*out)) == cudaSuccess;
#else
    (void)out;
    return false;
#endif
}
}  // namespace pr
