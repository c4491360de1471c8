// pr_kernels.cuh -- device code of the IFP1 / IFP2 rounds (Alg. 2, Alg. 3),
// the Power-method iteration (Sec. 4), the FP64 correction sweep, the IFP2
// phase-2 pull and the normalisation.
//
// Round semantics: synchronous snapshot rounds (Sec. 3.3.1 counts one
// "iteration" as one scan over all vertices) with a (1-c) reserve, which does
// not change the normalised result (Sec. 3.1, after Eq. 4):
//
//   R_t = sum_{i non-dangling} |r_i|            stop when R_t <= eps
//   F_t = { i non-dangling : |r_i| > xi_act }   snapshot before any push
//   i in F_t:  x_i += (1-c) r_i,  r_i = 0,  w_i = c r_i / deg(i)
//   j:         r_j += sum_{i in S(j) & F_t} w_i  (IFP2: non-dangling j only)
//
// Kernels and the state machine (ctl->mode names the pending action):
//   k_activate    (mode ACT or PUSH): activation of round t = ctl->round from r:
//                 R_t, |F_t|, edges, w_t (and the frontier bins + snapshot v
//                 when an atomic-push delivery is expected); its last block
//                 takes the stop decision and picks the delivery of round t.
//   k_round_pull  (mode PULL): delivers round t-1 by gathering w_{t-1} along
//                 every in-list (each row commits its own activation: the
//                 same |r_j| > xi_act test on the same r_j), then takes round
//                 t's activation decision for the same row -- one kernel per
//                 round, deterministic.
//   k_push        (mode PUSH): delivers round t-1 from the frontier bins:
//                 x_i += (1-c) v_i, r_i -= v_i, and an atomic add of
//                 c v_i/deg(i) along the out-list (IFP2: its non-dangling
//                 prefix).  The subtraction is order-independent, so the
//                 commit needs no separate pass; k_activate follows.
// A round is [k_round_pull, k_push, k_activate]; kernels whose mode is not
// pending return at once, and all of them return once ctl->done is set.
//
// Number formats.  GB300's FP64 pipe retires a warp instruction in about 64
// cycles of one SM sub-partition, even when a single lane executes it, so
// the state type T is one of
//   double  -- IEEE FP64 throughout (the paper's arithmetic, PR_FP64): state,
//              pushed mass, gathers, sums;
//   float   -- FP32 state (PR_FP32), with FP64 scalars; its correction sweep
//              and the rounds after it run in IEEE FP64;
//   float2  -- double-float (hi, lo) pairs, value hi + lo, 48-bit significand,
//              arithmetic on FP32 instructions only (PR_DF64).
// The FP32 and double-float forms gather float / double-float values; their
// residual-L1 and other sums run in double-float with a final FP64 sum.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include <cmath>

#include "pr_debug.cuh"
#include "pr_internal.cuh"

namespace pr {

enum { MODE_ACT = 0, MODE_PUSH = 1, MODE_PULL = 2 };
constexpr int POLICY_LEVELS = 3;  // PR_MODE_LEVELS: level-ordered pull rounds
constexpr int POLICY_ASYNC = 4;   // PR_MODE_ASYNC: push rounds that take r_i at push time
constexpr int POLICY_APULL = 5;   // PR_MODE_APULL: pull rounds that recompute r_j from the reserves

struct Ctl {
    // parameters (host-written per solve), in every format the kernels use
    double c, one_minus_c, eps, xi, pull_edges, pu, inv_om;
    float c_f, om_f, xi_f, pu_f, inv_om_f, pad5;
    float2 c_df, om_df, xi_df, pu_df, inv_om_df;
    int32_t algo, policy, max_rounds, p_dense;
    int64_t scan_ref, scan_unref;  // in-list entries read by one pull round
    int32_t trace_cap, pad0;
    // evolving state (device-written)
    int32_t round;         // next round to activate
    int32_t cur;           // round awaiting delivery
    int32_t done, status, mode, want_bins, unref_active, pad3;
    uint32_t ticket, pad1;
    uint32_t bin_cnt[2][3];
    double R, D;
    long long F, E;
    long long pushes, edges_pushed, edges_scanned;
    int32_t rounds_push, rounds_pull;
    // power / finalize
    double gamma, delta, zsum;
    float gamma_f, pad4;
    float2 gamma_df, zinv_df;
    int32_t iter, pad2;
    // level-ordered rounds: the kind of the next pull round (0 synchronous,
    // 1 the first level-ordered round, 2 level-ordered, 3 commit only: the
    // round cap stops the run at the start of the first level-ordered round)
    int32_t gs_phase, pad6;
    // asynchronous pull rounds that hand over to another precision: the run
    // also ends once R has not fallen below 0.99 of its best for stall_cap
    // rounds (0: never)
    int32_t stall_cap, stall;
    double r_best;
};

struct Partials {
    double *a, *b, *c;   // [kMaxBlocks] each (double-float sums reuse the 8-byte slots)
    long long *F, *E;    // [kMaxBlocks]
    int *u;              // [kMaxBlocks]
};

struct Trace {
    double *R;
    long long *F, *E;
    int8_t *mode;
};

// personalization in each format (dense) -- one of them is used by a kernel
struct PVals {
    const double *p64;
    const float *p32;
    const float2 *pdf;
};

// ------------------------------------------------------------ double-float
// value = hi + lo with |lo| <= ulp(hi)/2 (Dekker 1971; Knuth TAOCP 4.2.2)
__host__ __device__ __forceinline__ float2 df_from_d(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);  // exact error of the high product
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_abs(float2 a) { return a.x < 0.f ? df_neg(a) : a; }
__device__ __forceinline__ bool df_gt(float2 a, float2 b) { return a.x > b.x || (a.x == b.x && a.y > b.y); }
__device__ __forceinline__ double df_to_d(float2 a) { return (double)a.x + (double)a.y; }

// atomic a += v on a double-float pair (64-bit compare-and-swap loop)
__device__ __forceinline__ void df_atomic_add(float2 *a, float2 v) {
    unsigned long long *p = reinterpret_cast<unsigned long long *>(a);
    unsigned long long old = *p, assumed;
    do {
        assumed = old;
        float2 cur;
        memcpy(&cur, &assumed, 8);
        const float2 nv = df_add(cur, v);
        unsigned long long nb;
        memcpy(&nb, &nv, 8);
        old = atomicCAS(p, assumed, nb);
    } while (old != assumed);
}

// ------------------------------------------------------------ gathered element types
template <typename V> struct GT;
template <> struct GT<double> {
    using A = double;
    static __device__ __forceinline__ A zero() { return 0.0; }
    static __device__ __forceinline__ A add(A a, double v) { return a + v; }
    static __device__ __forceinline__ A shfl_down(A a, int o, int w) { return __shfl_down_sync(0xffffffffu, a, o, w); }
    static __device__ __forceinline__ A shfl_xor(A a, int o, int w) { return __shfl_xor_sync(0xffffffffu, a, o, w); }
};
template <> struct GT<float> {
    using A = float;
    static __device__ __forceinline__ A zero() { return 0.f; }
    static __device__ __forceinline__ A add(A a, float v) { return a + v; }
    static __device__ __forceinline__ A shfl_down(A a, int o, int w) { return __shfl_down_sync(0xffffffffu, a, o, w); }
    static __device__ __forceinline__ A shfl_xor(A a, int o, int w) { return __shfl_xor_sync(0xffffffffu, a, o, w); }
};
template <> struct GT<float2> {
    using A = float2;
    static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ A add(A a, float2 v) { return df_add(a, v); }
    static __device__ __forceinline__ A shfl_down(A a, int o, int w) {
        return make_float2(__shfl_down_sync(0xffffffffu, a.x, o, w), __shfl_down_sync(0xffffffffu, a.y, o, w));
    }
    static __device__ __forceinline__ A shfl_xor(A a, int o, int w) {
        return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o, w), __shfl_xor_sync(0xffffffffu, a.y, o, w));
    }
};

// ------------------------------------------------------------ state traits
// R: the accumulator of sums (residual L1, Power deltas, normaliser)
template <typename T> struct ST;
template <> struct ST<double> {
    using V = double;  // pushed mass gathered and summed in IEEE double
    using R = double;
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double absv(double a) { return fabs(a); }
    static __device__ __forceinline__ bool gt(double a, double b) { return a > b; }
    static __device__ __forceinline__ double c(const Ctl *k) { return k->c; }
    static __device__ __forceinline__ double om(const Ctl *k) { return k->one_minus_c; }
    static __device__ __forceinline__ double xi(const Ctl *k) { return k->xi; }
    static __device__ __forceinline__ double gamma(const Ctl *k) { return k->gamma; }
    static __device__ __forceinline__ double inv_om(const Ctl *k) { return k->inv_om; }
    static __device__ __forceinline__ double p(const Ctl *k, const PVals &P, int j) {
        return k->p_dense ? P.p64[j] : k->pu;
    }
    static __device__ __forceinline__ double invdeg(const DevGraph &G, int i) { return G.inv_deg64[i]; }
    static __device__ __forceinline__ double from_acc(double a) { return a; }
    static __device__ __forceinline__ double pack(double v) { return v; }
    static __device__ __forceinline__ double to_d(double v) { return v; }
    static __device__ __forceinline__ double pack_from_d(double v) { return v; }
    static __device__ __forceinline__ R rval(double v) { return v; }
    static __device__ __forceinline__ R radd(R a, R b) { return a + b; }
    static __device__ __forceinline__ R rzero() { return 0.0; }
    static __device__ __forceinline__ R rshfl(R a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ double r_to_d(R a) { return a; }
    static __device__ __forceinline__ void atomic_add(double *a, double v) { atomicAdd(a, v); }
    // push-round delivery, the pushing vertex's own subtraction, and the read of
    // r_i at the activation that follows a push round (see ST<float2>)
    static __device__ __forceinline__ void push_to(double *r, double *, int j, double w) { atomicAdd(&r[j], w); }
    static __device__ __forceinline__ void commit_sub(double *r, int i, double v) { atomicAdd(&r[i], -v); }
    static __device__ __forceinline__ double fold(double *r, double *, int i) { return r[i]; }
    // asynchronous push rounds: all of r_i at this moment, leaving 0
    static __device__ __forceinline__ double take(double *r, double *, int i) {
        return __longlong_as_double(
            (long long)atomicExch(reinterpret_cast<unsigned long long *>(&r[i]), 0ull));
    }
};
template <> struct ST<float> {
    using V = float;
    using R = double;  // the residual-L1 and other sums of FP32 state run in IEEE double
    static __device__ __forceinline__ float zero() { return 0.f; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float absv(float a) { return fabsf(a); }
    static __device__ __forceinline__ bool gt(float a, float b) { return a > b; }
    static __device__ __forceinline__ float c(const Ctl *k) { return k->c_f; }
    static __device__ __forceinline__ float om(const Ctl *k) { return k->om_f; }
    static __device__ __forceinline__ float xi(const Ctl *k) { return k->xi_f; }
    static __device__ __forceinline__ float gamma(const Ctl *k) { return k->gamma_f; }
    static __device__ __forceinline__ float inv_om(const Ctl *k) { return k->inv_om_f; }
    static __device__ __forceinline__ float p(const Ctl *k, const PVals &P, int j) {
        return k->p_dense ? P.p32[j] : k->pu_f;
    }
    static __device__ __forceinline__ float invdeg(const DevGraph &G, int i) { return G.inv_deg32[i]; }
    static __device__ __forceinline__ float from_acc(float a) { return a; }
    static __device__ __forceinline__ float pack(float v) { return v; }
    static __device__ __forceinline__ double to_d(float v) { return (double)v; }
    static __device__ __forceinline__ float pack_from_d(double v) { return (float)v; }
    static __device__ __forceinline__ R rval(float v) { return (double)v; }
    static __device__ __forceinline__ R radd(R a, R b) { return a + b; }
    static __device__ __forceinline__ R rzero() { return 0.0; }
    static __device__ __forceinline__ R rshfl(R a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ double r_to_d(R a) { return a; }
    static __device__ __forceinline__ void atomic_add(float *a, float v) { atomicAdd(a, v); }
    static __device__ __forceinline__ void push_to(float *r, double *, int j, float w) { atomicAdd(&r[j], w); }
    static __device__ __forceinline__ void commit_sub(float *r, int i, float v) { atomicAdd(&r[i], -v); }
    static __device__ __forceinline__ float fold(float *r, double *, int i) { return r[i]; }
    static __device__ __forceinline__ float take(float *r, double *, int i) { return atomicExch(&r[i], 0.f); }
};
template <> struct ST<float2> {
    using V = float2;
    using R = float2;
    static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return df_add(a, b); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return df_mul(a, b); }
    static __device__ __forceinline__ float2 neg(float2 a) { return df_neg(a); }
    static __device__ __forceinline__ float2 absv(float2 a) { return df_abs(a); }
    static __device__ __forceinline__ bool gt(float2 a, float2 b) { return df_gt(a, b); }
    static __device__ __forceinline__ float2 c(const Ctl *k) { return k->c_df; }
    static __device__ __forceinline__ float2 om(const Ctl *k) { return k->om_df; }
    static __device__ __forceinline__ float2 xi(const Ctl *k) { return k->xi_df; }
    static __device__ __forceinline__ float2 gamma(const Ctl *k) { return k->gamma_df; }
    static __device__ __forceinline__ float2 inv_om(const Ctl *k) { return k->inv_om_df; }
    static __device__ __forceinline__ float2 p(const Ctl *k, const PVals &P, int j) {
        return k->p_dense ? P.pdf[j] : k->pu_df;
    }
    static __device__ __forceinline__ float2 invdeg(const DevGraph &G, int i) { return G.inv_degdf[i]; }
    static __device__ __forceinline__ float2 from_acc(float2 a) { return a; }
    static __device__ __forceinline__ float2 pack(float2 v) { return v; }
    static __device__ __forceinline__ double to_d(float2 v) { return df_to_d(v); }
    static __device__ __forceinline__ float2 pack_from_d(double v) { return df_from_d(v); }
    static __device__ __forceinline__ R rval(float2 v) { return v; }
    static __device__ __forceinline__ R radd(R a, R b) { return df_add(a, b); }
    static __device__ __forceinline__ R rzero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ R rshfl(R a, int o) { return GT<float2>::shfl_down(a, o, 32); }
    static __device__ __forceinline__ double r_to_d(R a) { return df_to_d(a); }
    static __device__ __forceinline__ void atomic_add(float2 *a, float2 v) { df_atomic_add(a, v); }
    // A push round adds into an FP64 inbox with the L2's native double atomics:
    // a double-float compare-and-swap loop serialises on vertices that many
    // frontier vertices push into.  The double sum keeps more than the pair's
    // 48 significant bits.  Nothing else writes r during a push round, so the
    // pushing vertex subtracts its snapshot from r directly, and the activation
    // that follows every push round folds the inbox into r.
    static __device__ __forceinline__ void push_to(float2 *, double *din, int j, float2 w) {
        atomicAdd(&din[j], df_to_d(w));
    }
    static __device__ __forceinline__ void commit_sub(float2 *r, int i, float2 v) { r[i] = df_add(r[i], df_neg(v)); }
    static __device__ __forceinline__ float2 fold(float2 *r, double *din, int i) {
        const double d = din[i];
        if (d == 0.0) return r[i];
        const float2 v = df_add(r[i], df_from_d(d));
        r[i] = v;
        din[i] = 0.0;
        return v;
    }
    // asynchronous push rounds: r_i (written only by vertex i itself in a push
    // round) plus everything its inbox has received so far, leaving both 0
    static __device__ __forceinline__ float2 take(float2 *r, double *din, int i) {
        const double d = __longlong_as_double(
            (long long)atomicExch(reinterpret_cast<unsigned long long *>(&din[i]), 0ull));
        const float2 v = df_add(r[i], df_from_d(d));
        r[i] = make_float2(0.f, 0.f);
        return v;
    }
};

// |v| > xi_act, evaluated identically wherever an activation is decided.
// FP32: xi_f is the largest float <= xi, so the test equals (double)|v| > xi.
// FP64: non-negative doubles are ordered like their bit patterns, so |v| > xi
// (xi >= 0) is an integer comparison, off the FP64 pipe.
template <typename T> __device__ __forceinline__ bool is_active(T v, const Ctl *ctl) {
    if constexpr (std::is_same<T, double>::value) {
        return (__double_as_longlong(v) & 0x7fffffffffffffffll) > __double_as_longlong(ctl->xi);
    } else {
        return ST<T>::gt(ST<T>::absv(v), ST<T>::xi(ctl));
    }
}


// ------------------------------------------------------------ reductions
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

// block-wide sum of an ST<T>::R accumulator
template <typename T> __device__ __forceinline__ typename ST<T>::R block_sum_r(typename ST<T>::R v,
                                                                             typename ST<T>::R *sh) {
    using R = typename ST<T>::R;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ST<T>::radd(v, ST<T>::rshfl(v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    R r = ST<T>::rzero();
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : ST<T>::rzero();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = ST<T>::radd(r, ST<T>::rshfl(r, o));
    }
    return r;
}

// block-wide sum of a gathered accumulator
template <typename V> __device__ __forceinline__ typename GT<V>::A block_sum_gt(typename GT<V>::A v,
                                                                              typename GT<V>::A *sh) {
    using A = typename GT<V>::A;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = GT<V>::add(v, GT<V>::shfl_down(v, o, 32));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    A r = GT<V>::zero();
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : GT<V>::zero();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = GT<V>::add(r, GT<V>::shfl_down(r, o, 32));
    }
    return r;
}

// last-block election: every block calls with its partials already stored
__device__ __forceinline__ bool last_block(uint32_t *ticket) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// the last block's FP64 sum of the blocks' R partials (stored in 8-byte slots)
template <typename T> __device__ __forceinline__ double final_sum(const double *slots, double *shd) {
    using R = typename ST<T>::R;
    const unsigned long long *p = reinterpret_cast<const unsigned long long *>(slots);
    double s = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        R v;
        const unsigned long long bits = __ldcg(p + k);
        memcpy(&v, &bits, 8);
        s += ST<T>::r_to_d(v);
    }
    return block_sum(s, shd);
}

template <typename T> __device__ __forceinline__ void store_partial(double *slots, typename ST<T>::R v) {
    memcpy(reinterpret_cast<char *>(slots) + 8 * (size_t)blockIdx.x, &v, 8);
}

// A gathered value: through the read-only (non-coherent) path when the array
// is not written during the kernel (NC), else a plain load (asynchronous pull
// rounds read values that other rows of the same launch update).
template <bool NC, typename V> __device__ __forceinline__ V ldv(const V *p) {
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// Gathers of in-list sums.  A lane sums val[src[e]] over its entries
// e = off[j] + start, + step, ... < off[j+1] strictly in that order (one
// accumulator per row), so the result does not depend on how the loads are
// batched.  The loads are batched U at a time: U in-list entries first (they
// stream from HBM once, evict-first), then the U gathered values (read-only
// path; L2-resident in practice), so that U dependent load pairs per row are
// in flight instead of one.
template <typename V, int U, bool NC = true>
__device__ __forceinline__ void row_acc_u(const int32_t *__restrict__ src, int nsrc, const V *__restrict__ val, int &e,
                                          int b, int step, typename GT<V>::A &acc) {
    int idx[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int ee = e + u * step;
        idx[u] = ee < b ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
        if (idx[u] >= 0) acc = GT<V>::add(acc, ldv<NC>(&val[idx[u]]));
    e += U * step;
}

// one row, all of a block's threads (start = threadIdx.x, step = blockDim.x)
template <typename V, bool NC = true>
__device__ __forceinline__ typename GT<V>::A row_sum(const int32_t *__restrict__ off,
                                                     const int32_t *__restrict__ src, int nsrc, int j,
                                                     const V *__restrict__ val, int start, int step) {
    using A = typename GT<V>::A;
    const int b = __ldg(&off[j + 1]);
    int e = __ldg(&off[j]) + start;
    A acc = GT<V>::zero();
    while (e < b) row_acc_u<V, 8, NC>(src, nsrc, val, e, b, step, acc);
    return acc;
}

// The sums of ROWS rows at once (rows js[r], valid[r]), U entries per row per
// step: the in-list entry loads and then the gathers of all rows are in flight
// together.
template <typename V, int ROWS, int U, bool NC = true>
__device__ __forceinline__ void row_sums(const int32_t *__restrict__ off, const int32_t *__restrict__ src, int nsrc,
                                         const int *js, const bool *valid, const V *__restrict__ val, int start,
                                         int step, typename GT<V>::A *acc) {
    int e[ROWS], b[ROWS];
    bool any = false;
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        acc[r] = GT<V>::zero();
        e[r] = 0;
        b[r] = 0;
        if (valid[r]) {
            e[r] = __ldg(&off[js[r]]) + start;
            b[r] = __ldg(&off[js[r] + 1]);
        }
        any |= e[r] < b[r];
    }
    while (any) {
        int idx[ROWS][U];
#pragma unroll
        for (int r = 0; r < ROWS; r++)
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int ee = e[r] + u * step;
                idx[r][u] = ee < b[r] ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
            }
        any = false;
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
#pragma unroll
            for (int u = 0; u < U; u++)
                if (idx[r][u] >= 0) acc[r] = GT<V>::add(acc[r], ldv<NC>(&val[idx[r][u]]));
            e[r] += U * step;
            any |= e[r] < b[r];
        }
    }
}

// rows in flight per lane group: short rows (few lanes) interleave more of them
template <int LANES> struct RowsInFlight {
    static constexpr int value = LANES <= 2 ? 4 : (LANES <= 16 ? 2 : 1);
};
// entries per row per step: with the default thresholds a row below 32 lanes
// has at most 4 * LANES entries (two steps; 1- and 2-lane rows interleave 4
// rows instead, within the register cap); warp rows run up to 128 entries per
// lane
#ifndef PR_U_SMALL
#define PR_U_SMALL 1
#endif
#ifndef PR_U_MID
#define PR_U_MID 2
#endif
#ifndef PR_U_WARP
#define PR_U_WARP 8
#endif
template <int LANES> struct EntriesInFlight {
    static constexpr int value = LANES <= 2 ? PR_U_SMALL : (LANES < 32 ? PR_U_MID : PR_U_WARP);
};

// ------------------------------------------------------------ gather tiles
// Single solves in IEEE FP64 gather short rows by tiles.  The tiles' shared
// memory is reserved by every launch of a kernel that contains them and
// shrinks L1, where the lane bins keep their hottest gathered values: measured
// on R-MAT scale 22, tiles speed up the FP64 kernels (heavier row epilogues)
// and slow down the FP32 and double-float ones, so only the FP64
// instantiations carry them.  PR_PULL_TILES=0 removes them everywhere.
#ifndef PR_PULL_TILES
#define PR_PULL_TILES 1
#endif
template <typename T> struct UseTiles {
    static constexpr bool value = PR_PULL_TILES && std::is_same<T, double>::value;
};
// rows per warp batch of the double-precision warp rows (see kWarpBatch)
#ifndef PR_WARP_BATCH
#define PR_WARP_BATCH 4
#endif
// A tile's pending values (in-list order) and its rows' entry offsets relative
// to the tile's first entry, in shared memory.
template <typename V> struct TileSmem {
    V val[kTileE];
    int32_t off[kTileRows + 1];
};
// the row state a tile's epilogues start from, fetched while the gathers fly
template <typename T> struct TileRows {
    T v[kTileRows];
};

// The shared memory of a double-precision segment's gather tiles.
template <typename T, typename V> struct SegSmem {
    struct {
        TileSmem<V> sm;
        TileRows<T> rs;
    } tile;
};

// Stages tile t: every thread first loads its kTileE / kThreads in-list
// entries (coalesced, evict-first), then gathers their values (independent
// loads), then the row offsets are copied.  Rows [ra, rb) of the tile.
template <typename V, typename T = float, bool NC = true>
__device__ __forceinline__ void tile_load(const DevGraph &G, int t, const V *__restrict__ val, TileSmem<V> &sm,
                                          int &ra, int &rb, const T *rowv = nullptr, TileRows<T> *rs = nullptr) {
    constexpr int U = kTileE / kThreads;
    constexpr int RU = (kTileRows + kThreads - 1) / kThreads;
    ra = __ldg(&G.tile_row[t]);
    rb = __ldg(&G.tile_row[t + 1]);
#ifdef PR_DEBUG
    if (ra < 0 || rb < ra || rb > G.n || rb - ra > kTileRows) {  // an empty tile: nothing is read
        dbg_fail(DBG_TILE_ROW, ra, rb);
        ra = rb = 0;
    }
#endif
    T pre[RU];
    if (rs) {  // the rows' state, in flight with the in-list loads and gathers below
#pragma unroll
        for (int k = 0; k < RU; k++) {
            const int i = (int)threadIdx.x + k * kThreads;
            if (i < rb - ra) pre[k] = rowv[ra + i];
        }
    }
    const int ea = __ldg(&G.inr_off[ra]);
    const int ne = __ldg(&G.inr_off[rb]) - ea;
    int idx[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int k = (int)threadIdx.x + u * kThreads;
        idx[u] = k < ne ? PR_IDX(__ldcs(&G.inr_src[ea + k]), G.n_nd, DBG_IN_SRC) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
        if (idx[u] >= 0) sm.val[threadIdx.x + u * kThreads] = ldv<NC>(&val[idx[u]]);
    for (int i = threadIdx.x; i <= rb - ra; i += kThreads) sm.off[i] = __ldg(&G.inr_off[ra + i]) - ea;
    if (rs) {
#pragma unroll
        for (int k = 0; k < RU; k++) {
            const int i = (int)threadIdx.x + k * kThreads;
            if (i < rb - ra) rs->v[i] = pre[k];
        }
    }
    __syncthreads();
}

// sum of tile row i (entries in order, as one lane sums a row)
template <typename V>
__device__ __forceinline__ typename GT<V>::A tile_row_sum(const TileSmem<V> &sm, int i) {
    typename GT<V>::A acc = GT<V>::zero();
    const int e1 = sm.off[i + 1];
    for (int e = sm.off[i]; e < e1; e++) acc = GT<V>::add(acc, sm.val[e]);
    return acc;
}

// ------------------------------------------------------------ IEEE double warp rows
// GB300's FP64 pipe takes as long for a warp instruction whatever lanes are
// active (measured: one lane costs as much as 32).  A row served by a whole
// warp pays each FP64 instruction of its lane reduction and of its epilogue
// (run by one lane) for one row.  So double-precision warp rows go through in
// batches of kWarpBatch rows per warp: every row's 32 lanes sum their entries
// (lane l: entries l, l + 32, ... in order, kWarpU loads in flight), one
// reduce-scatter over the warp finishes all the batch's rows with every lane
// adding (warp_batch_sums64), and lane k runs row k's epilogue, so each FP64
// instruction after the gather serves kWarpBatch rows.  Measured on R-MAT
// scale 22 (IEEE FP64 pull round): batches of 2, 4 and 8 rows take 0.213,
// 0.205 and 0.242 ms (8 rows run short of registers).
constexpr int kWarpBatch = PR_WARP_BATCH;  // 1 turns the batches off (shuffle-reduced lane bins)
static_assert(kWarpBatch <= 32, "a lane finishes each row of a batch");

// lane's share of row j's sum: entries off[j] + lane, + 32, ... in order,
// kWarpU of them per step.  The next step's in-list entries are loaded before
// this step's values are added, so a busy FP64 pipe does not hold back the
// loads; the adds of the last, partial step stop where the row ends (a
// warp-uniform bound; lanes past the end add an exact 0.0).  Measured on
// R-MAT scale 22, IEEE FP64 pull round: 0.254 ms with the shuffle-reduced
// lane bins, 0.226 ms with batches of 4 rows, 0.207 ms with batches of 4 and
// this pipelining (8 entries per step spill at the 40-register cap), 0.205 ms
// with the batch's reduce-scatter instead of partials parked in shared memory.
constexpr int kWarpU = 4;
template <bool NC = true>
__device__ __forceinline__ double warp_row_part64(const int32_t *__restrict__ off, const int32_t *__restrict__ src,
                                                  int nsrc, int j, const double *__restrict__ val, int lane) {
    const int b = __ldg(&off[j + 1]);
    double acc = 0.0;
    int base = __ldg(&off[j]);
    int idx[kWarpU];
#pragma unroll
    for (int u = 0; u < kWarpU; u++) {
        const int ee = base + lane + 32 * u;
        idx[u] = ee < b ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
    }
    while (base < b) {
        double v[kWarpU];
#pragma unroll
        for (int u = 0; u < kWarpU; u++) v[u] = idx[u] >= 0 ? ldv<NC>(&val[idx[u]]) : 0.0;
        const int nu = min(kWarpU, (b - base + 31) >> 5);  // steps holding an entry of some lane
        base += 32 * kWarpU;
#pragma unroll
        for (int u = 0; u < kWarpU; u++) {
            const int ee = base + lane + 32 * u;
            idx[u] = ee < b ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
        }
#pragma unroll
        for (int u = 0; u < kWarpU; u++)
            if (u < nu) acc += v[u];
    }
    return acc;
}

// The sums of rows j0 .. j0 + kWarpBatch - 1 (those below hi) by one warp: lane
// k < kWarpBatch returns row j0 + k's sum.  off2/src2: an optional second
// in-list segment, added to each lane's share before the reduction.  Every
// lane keeps its share of every row of the batch; a reduce-scatter then halves
// the rows a lane holds at each exchange (partner lane ^ 16, ^ 8, ...) until
// each group of 32 / kWarpBatch lanes holds one row, which a butterfly over
// the group finishes.  All 32 lanes add in every step: kWarpBatch - 1 + log2(32
// / kWarpBatch) double adds per batch, against 2 per row plus 7 for one lane
// per row when each row is reduced on its own.  The order of the additions is
// fixed, so the sums do not depend on scheduling.
template <bool NC = true>
__device__ __forceinline__ double warp_batch_sums64(const int32_t *off, const int32_t *src, const int32_t *off2,
                                                    const int32_t *src2, int nsrc, int j0, int hi, const double *val,
                                                    int lane) {
    static_assert((kWarpBatch & (kWarpBatch - 1)) == 0, "a power of two of rows per batch");
    constexpr int kGroup = 32 / kWarpBatch;  // lanes that end up holding one row
    double a[kWarpBatch];
#pragma unroll
    for (int k = 0; k < kWarpBatch; k++) {
        const int j = j0 + k;
        a[k] = 0.0;
        if (j < hi) {  // warp-uniform
            a[k] = warp_row_part64<NC>(off, src, nsrc, j, val, lane);
            if (off2) a[k] += warp_row_part64<NC>(off2, src2, nsrc, j, val, lane);
        }
    }
    // reduce-scatter: after the exchange with lane ^ o a lane keeps the upper
    // half of its rows when (lane & o), else the lower half
#pragma unroll
    for (int o = 16, cnt = kWarpBatch; cnt > 1; o >>= 1, cnt >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < cnt / 2; i++) {
            const double send = upper ? a[i] : a[i + cnt / 2];
            const double keep = upper ? a[i + cnt / 2] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    // lane l now holds part of row l / kGroup; finish it over its group
#pragma unroll
    for (int o = kGroup / 2; o > 0; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
    return __shfl_sync(0xffffffffu, a[0], (lane % kWarpBatch) * kGroup);
}

// ------------------------------------------------------------ round decision
// Executed by thread 0 of the last block of an activation (round t).
__device__ __forceinline__ void round_decision(Ctl *ctl, int t, double R, long long F, long long E, int u,
                                               int want, const Trace &tr) {
    ctl->ticket = 0;
    ctl->R = R;
    ctl->F = F;
    ctl->E = E;
    if (t < ctl->trace_cap) tr.R[t] = R;
    uint32_t *nxt = ((t + 1) & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
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
    if (ctl->policy == MODE_PUSH || ctl->policy == POLICY_ASYNC) mode = MODE_PUSH;
    else if (ctl->policy == MODE_PULL || ctl->policy == POLICY_LEVELS) mode = MODE_PULL;
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

struct RoundBuf {
    void *x, *r, *vbuf;  // T arrays
    void *w[2];          // ST<T>::V arrays; w[t & 1] written by the activation of round t
    int32_t *bins;
    double *din;         // [n] push-round inbox of double-float state (zero between rounds); else unused
    PVals pv;            // asynchronous pull rounds: p at every row
};

// activation of one non-dangling vertex i with residual v (round t):
// pending push w_t[i], snapshot v for a push delivery, frontier counters
template <typename T, bool IFP2>
__device__ __forceinline__ bool activate_one(const DevGraph &G, const Ctl *ctl, int i, T v, int want,
                                             typename ST<T>::V *w, T *vbuf, int &pd, long long &F, long long &E,
                                             int &u) {
    const bool act = is_active(v, ctl);
    pd = IFP2 ? G.ndeg[i] : (G.out_off[i + 1] - G.out_off[i]);
    w[i] = ST<T>::pack(act ? ST<T>::mul(v, ST<T>::mul(ST<T>::c(ctl), ST<T>::invdeg(G, i))) : ST<T>::zero());
    if (act) {
        F++;
        E += pd;
        u |= (i >= G.n_ref);
        if (want) vbuf[i] = v;
    }
    return act;
}

// warp-aggregated append of active vertices into the three out-degree bins
__device__ __forceinline__ void bins_append(bool act, int pd, int i, uint32_t *bcnt, int32_t *bins, int n_nd) {
    const int lane = threadIdx.x & 31;
    const int bin = pd <= kWarpRowMin ? 0 : (pd <= kCtaRowMin ? 1 : 2);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const unsigned mask = __ballot_sync(0xffffffffu, act && bin == b);
        if (!mask) continue;
        unsigned pos0 = 0;
        const int leader = __ffs(mask) - 1;
        if (lane == leader) pos0 = atomicAdd(&bcnt[b], (unsigned)__popc(mask));
        pos0 = __shfl_sync(0xffffffffu, pos0, leader);
        if (act && bin == b) bins[(size_t)b * n_nd + pos0 + __popc(mask & ((1u << lane) - 1u))] = i;
    }
}

// ------------------------------------------------------------ k_push
template <typename T>
__device__ __forceinline__ void push_commit(const Ctl *ctl, T *x, T *r, int i, T v) {
    x[i] = ST<T>::add(x[i], ST<T>::mul(ST<T>::om(ctl), v));
    ST<T>::commit_sub(r, i, v);
}

// The mass a frontier vertex pushes, decided by one thread (lane 0 or thread
// 0) and its reserve committed there.  Synchronous rounds: the activation's
// snapshot v_i, subtracted from r_i.  Asynchronous rounds (PR_MODE_ASYNC, the
// concurrency of Sec. 3.2): all of r_i at this moment, taken atomically, so
// mass that reached i earlier in the same round moves on now.
template <typename T>
__device__ __forceinline__ T push_mass(const Ctl *ctl, bool async, T *x, T *r, double *din, const T *vbuf, int i) {
    T v;
    if (async) {
        v = ST<T>::take(r, din, i);
        x[i] = ST<T>::add(x[i], ST<T>::mul(ST<T>::om(ctl), v));
    } else {
        v = vbuf[i];
        push_commit<T>(ctl, x, r, i, v);
    }
    return v;
}

// The pushes of one out-list [e0, e1) by `lanes` threads (this one is `lane`),
// one target per load and atomic.  (Four targets per 16-byte load, after the
// unaligned head, measured slower: a lane then issues four atomics in a row,
// and a 50-entry row keeps 13 lanes busy instead of 32; asynchronous rounds on
// R-MAT scale 22 in double-float took 31.6 ms instead of 27.8.)
template <typename T, bool IFP2>
__device__ __forceinline__ void push_list(const DevGraph &G, T *r, double *din, int e0, int e1, T wi, int lane,
                                          int lanes) {
    [[maybe_unused]] const int bound = IFP2 ? G.n_nd : G.n;  // the debug build's index check
    for (int e = e0 + lane; e < e1; e += lanes) {
        const int t = PR_IDX(G.out_dst[e], bound, DBG_OUT_DST);
        if (t >= 0) ST<T>::push_to(r, din, t, wi);
    }
}

__device__ __forceinline__ double shfl0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ float shfl0(float v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ float2 shfl0(float2 v) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, 0), __shfl_sync(0xffffffffu, v.y, 0));
}

template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_push(DevGraph G, const Ctl *ctl, RoundBuf B, int nb_thread,
                                                  int nb_warp) {
    if (ctl->done || ctl->mode != MODE_PUSH) return;
    const uint32_t *cnt = (ctl->cur & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
    const int n_nd = G.n_nd;
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    const T *vbuf = static_cast<const T *>(B.vbuf);
    const int32_t *bins = B.bins;
    const T cT = ST<T>::c(ctl);
    const bool async = ctl->policy == POLICY_ASYNC;
    const int b = blockIdx.x;
    if (b < nb_thread) {
        const uint32_t c0 = cnt[0];
        for (uint32_t k = b * blockDim.x + threadIdx.x; k < c0; k += nb_thread * blockDim.x) {
            const int i = PR_IDX(bins[k], n_nd, DBG_BIN);
            if (i < 0) continue;
            const T v = push_mass<T>(ctl, async, x, r, B.din, vbuf, i);
            const T wi = ST<T>::mul(v, ST<T>::mul(cT, ST<T>::invdeg(G, i)));
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            for (int e = e0; e < e1; e++) {
                const int t = PR_IDX(G.out_dst[e], IFP2 ? n_nd : G.n, DBG_OUT_DST);
                if (t >= 0) ST<T>::push_to(r, B.din, t, wi);
            }
        }
    } else if (b < nb_thread + nb_warp) {
        const uint32_t c1 = cnt[1];
        const int lane = threadIdx.x & 31;
        const int wpb = blockDim.x >> 5;
        for (uint32_t k = (b - nb_thread) * wpb + (threadIdx.x >> 5); k < c1; k += nb_warp * wpb) {
            const int i = PR_IDX(bins[(size_t)n_nd + k], n_nd, DBG_BIN);  // the same for the whole warp
            if (i < 0) continue;
            T v = ST<T>::zero();
            if (lane == 0) v = push_mass<T>(ctl, async, x, r, B.din, vbuf, i);
            v = shfl0(v);
            const T wi = ST<T>::mul(v, ST<T>::mul(cT, ST<T>::invdeg(G, i)));
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            push_list<T, IFP2>(G, r, B.din, e0, e1, wi, lane, 32);
        }
    } else {
        const uint32_t c2 = cnt[2];
        const int nb_cta = gridDim.x - nb_thread - nb_warp;
        __shared__ T vsh;
        for (uint32_t k = b - nb_thread - nb_warp; k < c2; k += nb_cta) {
            const int i = PR_IDX(bins[(size_t)2 * n_nd + k], n_nd, DBG_BIN);  // the same for the whole block
            if (i < 0) continue;
            if (threadIdx.x == 0) vsh = push_mass<T>(ctl, async, x, r, B.din, vbuf, i);
            __syncthreads();
            const T v = vsh;
            __syncthreads();  // vsh is rewritten by the next vertex
            const T wi = ST<T>::mul(v, ST<T>::mul(cT, ST<T>::invdeg(G, i)));
            const int e0 = G.out_off[i];
            const int e1 = IFP2 ? e0 + G.ndeg[i] : G.out_off[i + 1];
            push_list<T, IFP2>(G, r, B.din, e0, e1, wi, threadIdx.x, blockDim.x);
        }
    }
}

// ------------------------------------------------------------ k_round_pull
// commit + update + next activation of row j (run by one lane per row)
// v: r_j as the row starts (prefetched by the caller)
template <typename T, bool IFP2>
__device__ __forceinline__ bool pull_row_epilogue_v(const DevGraph &G, const Ctl *ctl, const RoundBuf &B,
                                                    typename ST<T>::V *wnext, int j, T v, T in, int want, int &pd,
                                                    typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul) {
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    if (j >= G.n_nd) {  // dangling vertex (IFP1): receives, never pushes
        r[j] = ST<T>::add(v, in);
        return false;
    }
    T base_v = v;
    if (is_active(v, ctl)) {  // commit of round t-1 (decided on this same r_j)
        x[j] = ST<T>::add(x[j], ST<T>::mul(ST<T>::om(ctl), v));
        base_v = ST<T>::zero();
    }
    const T rn = ST<T>::add(base_v, in);
    r[j] = rn;
    Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(rn)));
    return activate_one<T, IFP2>(G, ctl, j, rn, want, wnext, static_cast<T *>(B.vbuf), pd, Fl, El, ul);
}

template <typename T, bool IFP2>
__device__ __forceinline__ bool pull_row_epilogue(const DevGraph &G, const Ctl *ctl, const RoundBuf &B,
                                                  typename ST<T>::V *wnext, int j, T in, int want, int &pd,
                                                  typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul) {
    return pull_row_epilogue_v<T, IFP2>(G, ctl, B, wnext, j, static_cast<const T *>(B.r)[j], in, want, pd, Rl, Fl,
                                        El, ul);
}

// ------------------------------------------------------------ asynchronous pull rounds
// PR_MODE_APULL (the asynchronous scans of Sec. 3.2, in pull form).  The state
// is the reserve x and, per non-dangling source i, q_i = x_i / ((1-c) deg i)
// (w[0], updated in place), with U_j = sum of q_i over j's unreferenced
// in-neighbours (w[1]; they push once, in round 0).  A row recomputes what it
// holds now from Eq. 4's identity,
//   r_j = p_j + c (sum_{i in S(j), referenced} q_i + U_j) - x_j / (1-c),
// which counts every push made so far -- this round's included, whenever the
// source has committed before the gather reads it -- and never a push twice.
// If |r_j| > xi_act it commits: x_j += (1-c) r_j, q_j follows, r_j = 0.  The
// round's R is a bound on the residual the round leaves: what rows left
// behind, plus c |r_j| ndeg_j / deg_j for every commit, whose pushes may have
// reached their targets after those gathered.  IFP2's dangling rows are never
// touched (phase 2 fills them); IFP1's get their residual at the end.
template <typename T, bool IFP2>
__device__ __forceinline__ bool apull_row_epilogue(const DevGraph &G, const Ctl *ctl, const RoundBuf &B, int j,
                                                   T xj, T in, int &pd, typename ST<T>::R &Rl, long long &Fl,
                                                   long long &El) {
    using V = typename ST<T>::V;
    static_assert(std::is_same<V, T>::value, "gathered values in the state's format");
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    V *q = static_cast<V *>(B.w[0]);
    const V *U = static_cast<const V *>(B.w[1]);
    const T inflow = ST<T>::mul(ST<T>::c(ctl), ST<T>::add(in, U[j]));
    const T rj = ST<T>::add(ST<T>::add(ST<T>::p(ctl, B.pv, j), inflow), ST<T>::neg(ST<T>::mul(xj, ST<T>::inv_om(ctl))));
    pd = IFP2 ? G.ndeg[j] : (G.out_off[j + 1] - G.out_off[j]);
    if (is_active(rj, ctl)) {
        const T xn = ST<T>::add(xj, ST<T>::mul(ST<T>::om(ctl), rj));
        x[j] = xn;
        r[j] = ST<T>::zero();
        q[j] = ST<T>::mul(xn, ST<T>::mul(ST<T>::invdeg(G, j), ST<T>::inv_om(ctl)));
        const T share = ST<T>::mul(ST<T>::c(ctl), ST<T>::mul(ST<T>::pack_from_d((double)G.ndeg[j]), ST<T>::invdeg(G, j)));
        Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::mul(ST<T>::absv(rj), share)));
        Fl++;
        El += pd;
        return true;
    }
    r[j] = rj;
    Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(rj)));
    return false;
}

// the epilogue of a gathered row: synchronous rounds (EPI 0) or asynchronous
// pull rounds (EPI 1; pre = x_j, no frontier bins)
template <typename T, bool IFP2, int EPI>
__device__ __forceinline__ bool row_epilogue(const DevGraph &G, const Ctl *ctl, const RoundBuf &B,
                                             typename ST<T>::V *wnext, int j, T pre, T in, int want, int &pd,
                                             typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul) {
    if constexpr (EPI == 0) return pull_row_epilogue_v<T, IFP2>(G, ctl, B, wnext, j, pre, in, want, pd, Rl, Fl, El, ul);
    else return apull_row_epilogue<T, IFP2>(G, ctl, B, j, pre, in, pd, Rl, Fl, El);
}
// the row state an epilogue starts from: r_j (synchronous), x_j (asynchronous pull)
template <typename T, int EPI>
__device__ __forceinline__ const T *epi_state(const RoundBuf &B) {
    return static_cast<const T *>(EPI == 0 ? B.r : B.x);
}

// Rows of a plan segment handled by groups of LANES threads, ROWS rows per
// group at a time; the loop bound is uniform across the block so the
// width-LANES shuffles always see full warps.
template <typename T, bool IFP2, int LANES, int EPI = 0>
__device__ __forceinline__ void round_rows(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                           const RoundBuf &B, const typename ST<T>::V *wprev,
                                           typename ST<T>::V *wnext, bool use_unref, int want, uint32_t *bcnt,
                                           typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    constexpr int GPB = kThreads / LANES;
    constexpr int ROWS = RowsInFlight<LANES>::value;
    const int grp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    const int stride = S.nblk * GPB;
    for (int base = S.lo + lb * GPB; base < S.hi; base += ROWS * stride) {
        int js[ROWS];
        bool valid[ROWS];
        A acc[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            js[r] = base + r * stride + grp;
            valid[r] = js[r] < S.hi;
        }
        row_sums<V, ROWS, EntriesInFlight<LANES>::value, EPI == 0>(G.inr_off, G.inr_src, G.n_nd, js, valid, wprev, lane,
                                                                   LANES, acc);
        if (use_unref) {
            A extra[ROWS];
            row_sums<V, ROWS, EntriesInFlight<LANES>::value, EPI == 0>(G.inu_off, G.inu_src, G.n_nd, js, valid, wprev,
                                                                       lane, LANES, extra);
#pragma unroll
            for (int r = 0; r < ROWS; r++) acc[r] = GT<V>::add(acc[r], extra[r]);
        }
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
#pragma unroll
            for (int o = LANES / 2; o > 0; o >>= 1) acc[r] = GT<V>::add(acc[r], GT<V>::shfl_down(acc[r], o, LANES));
            bool act = false;
            int pd = 0;
            if (valid[r] && lane == 0)
                act = row_epilogue<T, IFP2, EPI>(G, ctl, B, wnext, js[r], epi_state<T, EPI>(B)[js[r]],
                                                 ST<T>::from_acc(acc[r]), want, pd, Rl, Fl, El, ul);
            if (want) bins_append(act, pd, js[r], bcnt, B.bins, G.n_nd);
        }
    }
}

// Double-precision warp rows of a pull round's segment, in batches of
// kWarpBatch rows per warp (batch i of the segment goes to warp i mod the
// segment's warps); lane k finishes row k of a batch.
template <bool IFP2, int EPI = 0>
__device__ __forceinline__ void round_warp_rows64(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                                  const RoundBuf &B, const double *wprev, double *wnext,
                                                  bool use_unref, int want, uint32_t *bcnt, double &Rl, long long &Fl,
                                                  long long &El, int &ul) {
    constexpr int WPB = kThreads / 32;
    const int lane = threadIdx.x & 31;
    const int nbatch = (S.hi - S.lo + kWarpBatch - 1) / kWarpBatch;
    for (int bt = lb * WPB + (int)(threadIdx.x >> 5); bt < nbatch; bt += S.nblk * WPB) {
        const int j0 = S.lo + bt * kWarpBatch;
        const double sum = warp_batch_sums64<EPI == 0>(G.inr_off, G.inr_src, use_unref ? G.inu_off : nullptr,
                                                       G.inu_src, G.n_nd, j0, S.hi, wprev, lane);
        const int j = j0 + lane;
        bool act = false;
        int pd = 0;
        if (lane < kWarpBatch && j < S.hi)
            act = row_epilogue<double, IFP2, EPI>(G, ctl, B, wnext, j, epi_state<double, EPI>(B)[j], sum, want, pd,
                                                  Rl, Fl, El, ul);
        if (want) bins_append(act, pd, j, bcnt, B.bins, G.n_nd);
    }
}

// The gather tiles of a pull round's segment: block lb takes tiles lb, lb +
// nblk, ...; one thread per row sums it from shared memory (plus the
// unreferenced sources' segment from global memory while it can be nonzero)
// and runs the row's epilogue.
template <typename T, bool IFP2, int EPI = 0>
__device__ __forceinline__ void round_tiles(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                            const RoundBuf &B, const typename ST<T>::V *wprev,
                                            typename ST<T>::V *wnext, bool use_unref, int want, uint32_t *bcnt,
                                            typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul,
                                            TileSmem<typename ST<T>::V> &sm, TileRows<T> &rs) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    for (int t = S.t0 + lb; t < S.t0 + S.nt; t += S.nblk) {
        int ra, rb;
        tile_load<V, T, EPI == 0>(G, t, wprev, sm, ra, rb, epi_state<T, EPI>(B), &rs);
        const int nrow = rb - ra;
        for (int base = 0; base < nrow; base += kThreads) {
            const int i = base + (int)threadIdx.x;
            const int j = ra + i;
            bool act = false;
            int pd = 0;
            if (i < nrow) {
                A acc = tile_row_sum<V>(sm, i);
                if (use_unref) acc = GT<V>::add(acc, row_sum<V, EPI == 0>(G.inu_off, G.inu_src, G.n_nd, j, wprev, 0, 1));
                act = row_epilogue<T, IFP2, EPI>(G, ctl, B, wnext, j, rs.v[i], ST<T>::from_acc(acc), want, pd, Rl,
                                                 Fl, El, ul);
            }
            if (want) bins_append(act, pd, j, bcnt, B.bins, G.n_nd);
        }
        __syncthreads();  // the next tile reuses the shared arrays
    }
}

// One segment (or tile) of a pull round: rows [S.lo, S.hi) with S.lanes threads per
// row (0: the whole block per row); block lb of S.nblk.
template <typename T, bool IFP2, int EPI = 0>
__device__ __forceinline__ void round_segment(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                              const RoundBuf &B, const typename ST<T>::V *wprev,
                                              typename ST<T>::V *wnext, bool use_unref, int want, uint32_t *bcnt,
                                              typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul,
                                              typename GT<typename ST<T>::V>::A *sha) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    if constexpr (std::is_same<T, double>::value) {
        __shared__ SegSmem<T, V> smu;
        if (UseTiles<T>::value && S.lanes == kTileLanes) {
            round_tiles<T, IFP2, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul,
                                      smu.tile.sm, smu.tile.rs);
            return;
        }
        if (kWarpBatch > 1 && S.lanes == 32) {
            round_warp_rows64<IFP2, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul);
            return;
        }
    }
    switch (S.lanes) {
        case 1: round_rows<T, IFP2, 1, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        case 2: round_rows<T, IFP2, 2, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        case 4: round_rows<T, IFP2, 4, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        case 8: round_rows<T, IFP2, 8, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        case 16: round_rows<T, IFP2, 16, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        case 32: round_rows<T, IFP2, 32, EPI>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul); break;
        default:  // one block per row
            for (int j = S.lo + lb; j < S.hi; j += S.nblk) {
                A acc = row_sum<V, EPI == 0>(G.inr_off, G.inr_src, G.n_nd, j, wprev, threadIdx.x, blockDim.x);
                if (use_unref)
                    acc = GT<V>::add(acc, row_sum<V, EPI == 0>(G.inu_off, G.inu_src, G.n_nd, j, wprev, threadIdx.x,
                                                               blockDim.x));
                acc = block_sum_gt<V>(acc, sha);
                if (threadIdx.x == 0) {
                    int pd = 0;
                    const bool act = row_epilogue<T, IFP2, EPI>(G, ctl, B, wnext, j, epi_state<T, EPI>(B)[j],
                                                                ST<T>::from_acc(acc), want, pd, Rl, Fl, El, ul);
                    if (want && act) {
                        const int bin = pd <= kWarpRowMin ? 0 : (pd <= kCtaRowMin ? 1 : 2);
                        const unsigned pos = atomicAdd(&bcnt[bin], 1u);
                        B.bins[(size_t)bin * G.n_nd + pos] = j;
                    }
                }
            }
    }
}

// Activation of rows [lo, hi) (non-dangling ids), stepping by `step` from
// lo + first: the trip count is uniform across each warp.
template <typename T, bool IFP2>
__device__ __forceinline__ void activate_range(const DevGraph &G, const Ctl *ctl, const RoundBuf &B,
                                               typename ST<T>::V *w, int lo, int hi, int first, int step, int want,
                                               uint32_t *bcnt, typename ST<T>::R &Rl, long long &Fl, long long &El,
                                               int &ul) {
    T *r = static_cast<T *>(B.r);
    T *vbuf = static_cast<T *>(B.vbuf);
    for (int base = lo + first; base < hi; base += step) {
        const int i = base + (int)threadIdx.x;
        bool act = false;
        int pd = 0;
        if (i < hi) {
            const T v = ST<T>::fold(r, B.din, i);  // the previous round was a push round
            Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(v)));
            act = activate_one<T, IFP2>(G, ctl, i, v, want, w, vbuf, pd, Fl, El, ul);
        }
        if (want) bins_append(act, pd, i, bcnt, B.bins, G.n_nd);
    }
}

// ------------------------------------------------------------ k_activate
template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_activate(DevGraph G, Ctl *ctl, Partials P, RoundBuf B, Trace tr) {
    using R = typename ST<T>::R;
    using V = typename ST<T>::V;
    if (ctl->done || ctl->mode == MODE_PULL) return;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ R shr[32];
    const int want = ctl->want_bins;
    const int t = ctl->round;
    uint32_t *bcnt = (t & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
    V *w = static_cast<V *>((t & 1) ? B.w[1] : B.w[0]);
    const int n_nd = G.n_nd;
    R Rl = ST<T>::rzero();
    long long Fl = 0, El = 0;
    int ul = 0;
    activate_range<T, IFP2>(G, ctl, B, w, 0, n_nd, blockIdx.x * blockDim.x, gridDim.x * blockDim.x, want, bcnt, Rl,
                            Fl, El, ul);
    const R Rb = block_sum_r<T>(Rl, shr);
    const long long Fb = block_sum(Fl, shl);
    const long long Eb = block_sum(El, shl);
    const int ub = __syncthreads_or(ul);
    if (threadIdx.x == 0) {
        store_partial<T>(P.a, Rb);
        P.F[blockIdx.x] = Fb;
        P.E[blockIdx.x] = Eb;
        P.u[blockIdx.x] = ub;
    }
    if (!last_block(&ctl->ticket)) return;
    const double Rsum = final_sum<T>(P.a, shd);
    long long F = 0, E = 0;
    int u = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        F += __ldcg(&P.F[k]);
        E += __ldcg(&P.E[k]);
        u |= __ldcg(&P.u[k]);
    }
    F = block_sum(F, shl);
    E = block_sum(E, shl);
    u = __syncthreads_or(u);
    if (threadIdx.x == 0) round_decision(ctl, t, Rsum, F, E, u, want, tr);
}

// resident blocks per SM the dense pull round is compiled for: 6 caps it at 40
// registers without spills (48 warps per SM), which measured 18% faster per
// launch than the uncapped 48 registers (5 blocks) on R-MAT scale 22
#ifndef PR_PULL_MIN_BLOCKS
#define PR_PULL_MIN_BLOCKS 6
#endif

template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads, PR_PULL_MIN_BLOCKS) k_round_pull(DevGraph G, Plan PL, Ctl *ctl, Partials P,
                                                                            RoundBuf B, Trace tr) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    if (ctl->done || ctl->mode != MODE_PULL) return;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ A sha[32];
    __shared__ R shr[32];
    const int t = ctl->round;  // activation of round t; delivery of round t - 1
    const int want = ctl->want_bins;
    const bool use_unref = ctl->unref_active != 0;
    uint32_t *bcnt = (t & 1) ? ctl->bin_cnt[1] : ctl->bin_cnt[0];
    const V *wprev = static_cast<const V *>((t & 1) ? B.w[0] : B.w[1]);  // written by round t - 1
    V *wnext = static_cast<V *>((t & 1) ? B.w[1] : B.w[0]);
    int s = 0;
    while (s + 1 < PL.nseg && (int)blockIdx.x >= PL.seg[s + 1].blk0) s++;
    const Seg S = PL.seg[s];
    const int lb = blockIdx.x - S.blk0;
    R Rl = ST<T>::rzero();
    long long Fl = 0, El = 0;
    int ul = 0;
    round_segment<T, IFP2>(G, S, lb, ctl, B, wprev, wnext, use_unref, want, bcnt, Rl, Fl, El, ul, sha);
    const R Rb = block_sum_r<T>(Rl, shr);
    const long long Fb = block_sum(Fl, shl);
    const long long Eb = block_sum(El, shl);
    const int ub = __syncthreads_or(ul);
    if (threadIdx.x == 0) {
        store_partial<T>(P.a, Rb);
        P.F[blockIdx.x] = Fb;
        P.E[blockIdx.x] = Eb;
        P.u[blockIdx.x] = ub;
    }
    if (!last_block(&ctl->ticket)) return;
    const double Rsum = final_sum<T>(P.a, shd);
    long long F = 0, E = 0;
    int u = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        F += __ldcg(&P.F[k]);
        E += __ldcg(&P.E[k]);
        u |= __ldcg(&P.u[k]);
    }
    F = block_sum(F, shl);
    E = block_sum(E, shl);
    u = __syncthreads_or(u);
    if (threadIdx.x == 0) round_decision(ctl, t, Rsum, F, E, u, want, tr);
}

// ------------------------------------------------------------ asynchronous pull rounds
// The decision after round t of PR_MODE_APULL (thread 0 of the last block):
// R is the bound on the residual the round left, F and E its commits.
__device__ __forceinline__ void apull_decision(Ctl *ctl, int t, double R, long long F, long long E, const Trace &tr) {
    ctl->ticket = 0;
    ctl->R = R;
    ctl->F = F;
    ctl->E = E;
    if (t < ctl->trace_cap) {
        tr.R[t] = R;
        tr.F[t] = F;
        tr.E[t] = E;
        tr.mode[t] = (int8_t)MODE_PULL;
    }
    ctl->pushes += F;
    ctl->edges_pushed += E;
    if (t > 0) {
        ctl->edges_scanned += ctl->scan_ref;
        ctl->rounds_pull++;
    }
    ctl->cur = t;
    ctl->round = t + 1;
    ctl->mode = MODE_PULL;
    if (R <= ctl->eps) {
        ctl->done = 1;
        ctl->status = 0;
    } else if (F == 0) {
        ctl->done = 1;
        ctl->status = 2;
    } else if (t + 1 >= ctl->max_rounds) {
        ctl->done = 1;
        ctl->status = 1;
    } else if (ctl->stall_cap > 0) {  // a hand-over run: R stopped falling, hand over now
        if (R < 0.99 * ctl->r_best) {
            ctl->r_best = R;
            ctl->stall = 0;
        } else if (++ctl->stall >= ctl->stall_cap) {
            ctl->done = 1;
            ctl->status = 0;
        }
    }
}

// the block partials of R, F, E, and the last block's decision
template <typename T>
__device__ __forceinline__ void apull_reduce(Ctl *ctl, const Partials &P, const Trace &tr, int t,
                                             typename ST<T>::R Rl, long long Fl, long long El,
                                             typename ST<T>::R *shr, double *shd, long long *shl) {
    using R = typename ST<T>::R;
    const R Rb = block_sum_r<T>(Rl, shr);
    const long long Fb = block_sum(Fl, shl);
    const long long Eb = block_sum(El, shl);
    if (threadIdx.x == 0) {
        store_partial<T>(P.a, Rb);
        P.F[blockIdx.x] = Fb;
        P.E[blockIdx.x] = Eb;
    }
    if (!last_block(&ctl->ticket)) return;
    const double Rsum = final_sum<T>(P.a, shd);
    long long F = 0, E = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        F += __ldcg(&P.F[k]);
        E += __ldcg(&P.E[k]);
    }
    F = block_sum(F, shl);
    E = block_sum(E, shl);
    if (threadIdx.x == 0) apull_decision(ctl, t, Rsum, F, E, tr);
}

// Round 0: every non-dangling vertex holds p_i and commits it if above xi_act;
// q_i = x_i / ((1-c) deg i) for all of them (0 when nothing is committed).
template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads) k_apull_init(DevGraph G, Ctl *ctl, Partials P, RoundBuf B, Trace tr) {
    using R = typename ST<T>::R;
    using V = typename ST<T>::V;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ R shr[32];
    if (ctl->done) return;
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    V *q = static_cast<V *>(B.w[0]);
    R Rl = ST<T>::rzero();
    long long Fl = 0, El = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n_nd; i += gridDim.x * blockDim.x) {
        const T v = r[i];
        if (is_active(v, ctl)) {
            const T xn = ST<T>::mul(ST<T>::om(ctl), v);
            x[i] = xn;
            r[i] = ST<T>::zero();
            q[i] = ST<T>::mul(xn, ST<T>::mul(ST<T>::invdeg(G, i), ST<T>::inv_om(ctl)));
            const T share = ST<T>::mul(ST<T>::c(ctl), ST<T>::mul(ST<T>::pack_from_d((double)G.ndeg[i]), ST<T>::invdeg(G, i)));
            Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::mul(ST<T>::absv(v), share)));
            Fl++;
            El += IFP2 ? G.ndeg[i] : (G.out_off[i + 1] - G.out_off[i]);
        } else {
            q[i] = ST<T>::zero();
            Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(v)));
        }
    }
    apull_reduce<T>(ctl, P, tr, 0, Rl, Fl, El, shr, shd, shl);
}

// U_j = sum of q_i over the unreferenced in-neighbours of non-dangling row j:
// they hold p and nothing else, commit in round 0 and never again.  A warp per
// row, lanes in entry order, a fixed shuffle tree.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apull_unref(DevGraph G, RoundBuf B) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    const V *q = static_cast<const V *>(B.w[0]);
    V *U = static_cast<V *>(B.w[1]);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < G.n_nd; j += warps) {
        A acc = row_sum<V>(G.inu_off, G.inu_src, G.n_nd, j, q, lane, 32);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = GT<V>::add(acc, GT<V>::shfl_down(acc, o, 32));
        if (lane == 0) U[j] = ST<T>::from_acc(acc);
    }
}

// One asynchronous pull round over the non-dangling rows (the IFP2 plan): the
// referenced in-neighbours' q by the plan's gathers, then apull_row_epilogue.
template <typename T, bool IFP2>
__global__ void __launch_bounds__(kThreads, PR_PULL_MIN_BLOCKS) k_round_apull(DevGraph G, Plan PL, Ctl *ctl, Partials P,
                                                                             RoundBuf B, Trace tr) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    if (ctl->done) return;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ A sha[32];
    __shared__ R shr[32];
    const int t = ctl->round;
    int s = 0;
    while (s + 1 < PL.nseg && (int)blockIdx.x >= PL.seg[s + 1].blk0) s++;
    const Seg S = PL.seg[s];
    const int lb = blockIdx.x - S.blk0;
    R Rl = ST<T>::rzero();
    long long Fl = 0, El = 0;
    int ul = 0;
    round_segment<T, IFP2, 1>(G, S, lb, ctl, B, static_cast<const V *>(B.w[0]), nullptr, false, 0, nullptr, Rl, Fl,
                              El, ul, sha);
    apull_reduce<T>(ctl, P, tr, t, Rl, Fl, El, shr, shd, shl);
}

// ------------------------------------------------------------ level-ordered rounds (IFP2)
// One launch serves one level's rows (plan of the level); the launches of a
// round run in level order, the rows without in-edges last, and the last
// launch takes the round's decision over the partial slots of all of them.
// a level's plan: its lane bins only (a kernel argument of 150 bytes instead
// of the full plan's 2.6 KB)
struct LevelPlan {
    Seg seg[kNumThr + 2];    // the cluster rows, the other block rows, then the lane bins
    int32_t nseg, nblocks;   // nblocks: blocks with work; the grid is padded to whole clusters
};

struct LevelLaunch {
    int32_t split;       // sources below this id belong to lower levels
    int32_t slot_base;   // this launch's first partial slot
    int32_t slot_total;  // slots of the whole round (read by the deciding launch)
    int32_t decide;      // the round's last launch
};

// sums of a row's pending pushes: sources of lower levels pushed in this round
// (wcur; in the first level-ordered round also in the previous one, which was
// synchronous and delivered nothing in-round), the others in the previous
// round (wprev).  Each lane adds its entries in order; ROWS rows and U entries
// per row are in flight at once, as in row_sums.
template <typename V, int ROWS, int U>
__device__ __forceinline__ void level_row_sums(const int32_t *__restrict__ off, const int32_t *__restrict__ src,
                                               int nsrc, const int *js, const bool *valid, const V *__restrict__ wcur,
                                               const V *__restrict__ wprev, int split, bool both, int start,
                                               int step, typename GT<V>::A *acc) {
    int e[ROWS], b[ROWS];
    bool any = false;
#pragma unroll
    for (int r = 0; r < ROWS; r++) {
        e[r] = 0;
        b[r] = 0;
        if (valid[r]) {
            e[r] = __ldg(&off[js[r]]) + start;
            b[r] = __ldg(&off[js[r] + 1]);
        }
        any |= e[r] < b[r];
    }
    while (any) {
        int idx[ROWS][U];
#pragma unroll
        for (int r = 0; r < ROWS; r++)
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int ee = e[r] + u * step;
                idx[r][u] = ee < b[r] ? PR_IDX(__ldcs(&src[ee]), nsrc, DBG_IN_SRC) : -1;
            }
        any = false;
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int i = idx[r][u];
                if (i < 0) continue;
                if (i < split) {
                    acc[r] = GT<V>::add(acc[r], __ldg(&wcur[i]));
                    if (both) acc[r] = GT<V>::add(acc[r], __ldg(&wprev[i]));
                } else {
                    acc[r] = GT<V>::add(acc[r], __ldg(&wprev[i]));
                }
            }
            e[r] += U * step;
            any |= e[r] < b[r];
        }
    }
}

// a level-ordered row: [deferred commit of the synchronous round before] +
// delivery + activation committed at once; R counts the residual left and the
// pushes into the row's own or lower levels (in flight until the next round)
template <typename T>
__device__ __forceinline__ void level_row_epilogue(const DevGraph &G, const Ctl *ctl, const RoundBuf &B,
                                                   typename ST<T>::V *wcur, int j, T in, bool deferred,
                                                   typename ST<T>::R &Rl, long long &Fl, long long &El) {
    T *x = static_cast<T *>(B.x);
    T *r = static_cast<T *>(B.r);
    T v = r[j];
    if (deferred && is_active(v, ctl)) {  // commit of the synchronous round's activation
        x[j] = ST<T>::add(x[j], ST<T>::mul(ST<T>::om(ctl), v));
        v = ST<T>::zero();
    }
    const T rn = ST<T>::add(v, in);
    if (is_active(rn, ctl)) {
        x[j] = ST<T>::add(x[j], ST<T>::mul(ST<T>::om(ctl), rn));
        r[j] = ST<T>::zero();
        const T w = ST<T>::mul(rn, ST<T>::mul(ST<T>::c(ctl), ST<T>::invdeg(G, j)));
        wcur[j] = ST<T>::pack(w);
        Fl++;
        El += G.ndeg[j];
        Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::mul(ST<T>::absv(w), ST<T>::pack_from_d((double)G.gs_back[j]))));
    } else {
        r[j] = rn;
        wcur[j] = ST<T>::pack(ST<T>::zero());
        Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(rn)));
    }
}

// Rows of one level's plan segment, LANES threads per row, ROWS rows per lane
// group at a time (as round_rows).  Phase 0: a synchronous round (deferred
// commit); phases 1 and 2: level-ordered.  The segment of unreferenced
// sources is read only in the synchronous round: from the level-ordered
// rounds on, those sources have nothing left to push.
template <typename T, int LANES>
__device__ __forceinline__ void level_rows(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                           const RoundBuf &B, const typename ST<T>::V *wprev,
                                           typename ST<T>::V *wcur, int phase, int split,
                                           typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    constexpr int GPB = kThreads / LANES;
    constexpr int ROWS = RowsInFlight<LANES>::value;
    constexpr int U = EntriesInFlight<LANES>::value;
    const int grp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    const int stride = S.nblk * GPB;
    const bool both = phase == 1;
    for (int base = S.lo + lb * GPB; base < S.hi; base += ROWS * stride) {
        int js[ROWS];
        bool valid[ROWS];
        A acc[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            js[r] = base + r * stride + grp;
            valid[r] = js[r] < S.hi;
            acc[r] = GT<V>::zero();
        }
        level_row_sums<V, ROWS, U>(G.inr_off, G.inr_src, G.n_nd, js, valid, wcur, wprev, split, both, lane, LANES, acc);
        if (phase == 0)
            level_row_sums<V, ROWS, U>(G.inu_off, G.inu_src, G.n_nd, js, valid, wcur, wprev, split, both, lane, LANES, acc);
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
#pragma unroll
            for (int o = LANES / 2; o > 0; o >>= 1) acc[r] = GT<V>::add(acc[r], GT<V>::shfl_down(acc[r], o, LANES));
            if (valid[r] && lane == 0) {
                if (phase == 0) {
                    int pd = 0;
                    pull_row_epilogue<T, true>(G, ctl, B, wcur, js[r], ST<T>::from_acc(acc[r]), 0, pd, Rl, Fl, El,
                                               ul);
                } else {
                    level_row_epilogue<T>(G, ctl, B, wcur, js[r], ST<T>::from_acc(acc[r]), phase == 1, Rl, Fl, El);
                }
            }
        }
    }
}

// A row with more than kClusterRowMin in-list entries, served by a cluster of
// kLevelCluster blocks: block q of the cluster sums the entries q * 256 +
// tid, stepping 8 * 256 (in entry order per thread), and the cluster's rank-0
// block adds the blocks' sums in rank order through distributed shared memory
// and runs the row's epilogue.  Every block of a cluster takes this path or
// none does: the segment starts and ends on cluster boundaries (checked when
// the plan is built, and here, together with the launch's cluster size).
template <typename T>
__device__ __forceinline__ void level_cluster_row(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                                  const RoundBuf &B, const typename ST<T>::V *wprev,
                                                  typename ST<T>::V *wcur, int phase, int split,
                                                  typename ST<T>::R &Rl, long long &Fl, long long &El, int &ul,
                                                  typename GT<typename ST<T>::V>::A *sha) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    if (cl.num_blocks() != kLevelCluster || S.blk0 % kLevelCluster != 0 || S.nblk % kLevelCluster != 0) return;
    __shared__ A part;
    const int rank = (int)cl.block_rank();
    const int j = S.lo + lb / kLevelCluster;
    const bool ok = j < S.hi;
    A acc = GT<V>::zero();
    const int start = rank * (int)blockDim.x + (int)threadIdx.x, step = kLevelCluster * (int)blockDim.x;
    level_row_sums<V, 1, 8>(G.inr_off, G.inr_src, G.n_nd, &j, &ok, wcur, wprev, split, phase == 1, start, step, &acc);
    if (phase == 0)
        level_row_sums<V, 1, 8>(G.inu_off, G.inu_src, G.n_nd, &j, &ok, wcur, wprev, split, false, start, step, &acc);
    acc = block_sum_gt<V>(acc, sha);
    if (threadIdx.x == 0) part = acc;
    cl.sync();
    if (rank == 0 && threadIdx.x == 0 && ok) {
        A tot = GT<V>::zero();
        for (int q = 0; q < kLevelCluster; q++) tot = GT<V>::add(tot, *cl.map_shared_rank(&part, q));
        if (phase == 0) {
            int pd = 0;
            pull_row_epilogue<T, true>(G, ctl, B, wcur, j, ST<T>::from_acc(tot), 0, pd, Rl, Fl, El, ul);
        } else {
            level_row_epilogue<T>(G, ctl, B, wcur, j, ST<T>::from_acc(tot), phase == 1, Rl, Fl, El);
        }
    }
    cl.sync();  // the other blocks' shared memory is read above: they stay until rank 0 is done
}

// the decision after a round of level launches (t = the round just run)
__device__ __forceinline__ void level_decision(Ctl *ctl, int t, int phase, double R, long long F, long long E,
                                               int u, const Trace &tr) {
    if (phase == 0) {  // a synchronous round: R is its start-of-round residual
        round_decision(ctl, t, R, F, E, u, 0, tr);
        // a cap at round t + 1 stops at its start: that round only commits
        if (!ctl->done) ctl->gs_phase = t + 1 >= ctl->max_rounds ? 3 : 1;
        return;
    }
    if (phase == 3) {
        ctl->ticket = 0;
        ctl->done = 1;
        ctl->status = 1;
        return;
    }
    // a level-ordered round ran whole: its pushes stand, R is the residual
    // left after it (in flight included)
    ctl->ticket = 0;
    ctl->R = R;
    ctl->F = F;
    ctl->E = E;
    if (t < ctl->trace_cap) {
        tr.R[t] = R;
        tr.F[t] = F;
        tr.E[t] = E;
        tr.mode[t] = (int8_t)MODE_PULL;
    }
    ctl->pushes += F;
    ctl->edges_pushed += E;
    ctl->edges_scanned += ctl->scan_ref + ctl->scan_unref;
    ctl->rounds_pull++;
    ctl->round = t + 1;
    ctl->cur = t;
    if (R <= ctl->eps) {
        ctl->done = 1;
        ctl->status = 0;
    } else if (F == 0) {
        ctl->done = 1;
        ctl->status = 2;
    } else if (t + 1 >= ctl->max_rounds) {
        ctl->done = 1;
        ctl->status = 1;
    } else {
        ctl->gs_phase = 2;
        ctl->unref_active = 0;
    }
}

// the level kernel reads two pending-push arrays per row: at 6 blocks per SM
// (40 registers) it spills, at 5 (48 registers) it does not
#ifndef PR_LEVEL_MIN_BLOCKS
#define PR_LEVEL_MIN_BLOCKS 5
#endif

// Launched with programmatic stream serialization: the launch of the next
// level may begin while this one drains; griddepcontrol.wait holds every
// thread until the previous launch has completed and its writes are visible,
// and nothing is read before it.  Without the launch attribute both
// instructions are no-ops.
template <typename T>
__global__ void __launch_bounds__(kThreads, PR_LEVEL_MIN_BLOCKS) k_round_levels(DevGraph G, LevelPlan PL, Ctl *ctl,
                                                                              Partials P, RoundBuf B, Trace tr,
                                                                              LevelLaunch lv) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (ctl->done || ctl->mode != MODE_PULL) return;
    __shared__ double shd[32];
    __shared__ long long shl[32];
    __shared__ A sha[32];
    __shared__ R shr[32];
    const int t = ctl->round;
    const int phase = ctl->gs_phase;
    const V *wprev = static_cast<const V *>((t & 1) ? B.w[0] : B.w[1]);  // written by round t - 1
    V *wcur = static_cast<V *>((t & 1) ? B.w[1] : B.w[0]);
    const int split = phase ? lv.split : 0;
    R Rl = ST<T>::rzero();
    long long Fl = 0, El = 0;
    int ul = 0;
    if (phase >= 1 && phase <= 2 && lv.decide && PL.nseg > 0) {
        // the rows without in-edges: from the first level-ordered round on they
        // receive nothing and hold at most a residual below xi_act (round 1
        // committed what round 0 activated), so they only add |r| to R
        const T *r = static_cast<const T *>(B.r);
        for (int j = PL.seg[0].lo + blockIdx.x * blockDim.x + threadIdx.x; j < PL.seg[PL.nseg - 1].hi;
             j += gridDim.x * blockDim.x)
            Rl = ST<T>::radd(Rl, ST<T>::rval(ST<T>::absv(r[j])));
    } else if (phase == 3 && PL.nseg > 0) {  // commit of the synchronous round's activation, nothing else
        T *x = static_cast<T *>(B.x);
        T *r = static_cast<T *>(B.r);
        for (int j = PL.seg[0].lo + blockIdx.x * blockDim.x + threadIdx.x; j < PL.seg[PL.nseg - 1].hi;
             j += gridDim.x * blockDim.x) {
            const T v = r[j];
            if (is_active(v, ctl)) {
                x[j] = ST<T>::add(x[j], ST<T>::mul(ST<T>::om(ctl), v));
                r[j] = ST<T>::zero();
            }
        }
    } else if (PL.nseg > 0 && (int)blockIdx.x < PL.nblocks) {  // blocks past nblocks pad the last cluster
        int lo = 0, hi = PL.nseg - 1;  // the last segment with blk0 <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (PL.seg[mid].blk0 <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        const Seg S = PL.seg[lo];
        const int lb = blockIdx.x - S.blk0;
        switch (S.lanes) {
            case kClusterLanes:
                level_cluster_row<T>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul, sha);
                break;
            case 1: level_rows<T, 1>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            case 2: level_rows<T, 2>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            case 4: level_rows<T, 4>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            case 8: level_rows<T, 8>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            case 16: level_rows<T, 16>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            case 32: level_rows<T, 32>(G, S, lb, ctl, B, wprev, wcur, phase, split, Rl, Fl, El, ul); break;
            default:
                for (int j = S.lo + lb; j < S.hi; j += S.nblk) {
                    const bool ok = true;
                    A acc = GT<V>::zero();
                    level_row_sums<V, 1, 8>(G.inr_off, G.inr_src, G.n_nd, &j, &ok, wcur, wprev, split, phase == 1,
                                            threadIdx.x, blockDim.x, &acc);
                    if (phase == 0)
                        level_row_sums<V, 1, 8>(G.inu_off, G.inu_src, G.n_nd, &j, &ok, wcur, wprev, split, false,
                                                threadIdx.x, blockDim.x, &acc);
                    acc = block_sum_gt<V>(acc, sha);
                    if (threadIdx.x == 0) {
                        if (phase == 0) {
                            int pd = 0;
                            pull_row_epilogue<T, true>(G, ctl, B, wcur, j, ST<T>::from_acc(acc), 0, pd, Rl, Fl, El,
                                                       ul);
                        } else {
                            level_row_epilogue<T>(G, ctl, B, wcur, j, ST<T>::from_acc(acc), phase == 1, Rl, Fl, El);
                        }
                    }
                }
        }
    }
    const R Rb = block_sum_r<T>(Rl, shr);
    const long long Fb = block_sum(Fl, shl);
    const long long Eb = block_sum(El, shl);
    const int ub = __syncthreads_or(ul);
    const int slot = lv.slot_base + blockIdx.x;
    if (threadIdx.x == 0) {
        memcpy(reinterpret_cast<char *>(P.a) + 8 * (size_t)slot, &Rb, 8);
        P.F[slot] = Fb;
        P.E[slot] = Eb;
        P.u[slot] = ub;
    }
    if (!lv.decide || !last_block(&ctl->ticket)) return;
    const unsigned long long *pa = reinterpret_cast<const unsigned long long *>(P.a);
    double Rs = 0.0;
    long long F = 0, E = 0;
    int u = 0;
    for (int k = threadIdx.x; k < lv.slot_total; k += blockDim.x) {
        R v;
        const unsigned long long bits = __ldcg(pa + k);
        memcpy(&v, &bits, 8);
        Rs += ST<T>::r_to_d(v);
        F += __ldcg(&P.F[k]);
        E += __ldcg(&P.E[k]);
        u |= __ldcg(&P.u[k]);
    }
    Rs = block_sum(Rs, shd);
    F = block_sum(F, shl);
    E = block_sum(E, shl);
    u = __syncthreads_or(u);
    if (threadIdx.x == 0) level_decision(ctl, t, phase, Rs, F, E, u, tr);
}

// ------------------------------------------------------------ sweeps: Power, correction, phase 2
// resident blocks per SM the sweeps are compiled for (as the pull round: the
// gathers are latency-bound, so warps in flight matter more than registers).
// The double-float Power sweep keeps 5: at 6 (40 registers) it spills 384
// bytes and measured 2% slower, while the FP32 and FP64 sweeps gained 9% and
// 7% at 6.
#ifndef PR_SWEEP_MIN_BLOCKS
#define PR_SWEEP_MIN_BLOCKS 6
#endif
template <typename T, int OP> struct SweepMinBlocks {
    static constexpr int value = (std::is_same<T, float2>::value && OP == 1) ? 5 : PR_SWEEP_MIN_BLOCKS;
};
enum { OP_POWER = 1, OP_CORRECT = 2, OP_PHASE2 = 3 };

template <typename T> struct SweepArgs {
    const typename ST<T>::V *val;  // gathered per source
    T *r;                          // CORRECT / PHASE2 output residual
    const T *x;                    // CORRECT reads the reserve
    const T *pi_cur;               // POWER
    T *pi_next;                    // POWER
    typename ST<T>::V *q_next;     // POWER
    PVals pv;
    Partials P;
    Trace tr;
};

// the row value an epilogue starts from: Power's pi_k, the correction's
// reserve, phase 2's residual (prefetched by the tile path)
template <typename T, int OP>
__device__ __forceinline__ T sweep_row_state(const SweepArgs<T> &a, int j) {
    if constexpr (OP == OP_POWER) return a.pi_cur[j];
    else if constexpr (OP == OP_CORRECT) return a.x[j];
    else return a.r[j];
}
template <typename T, int OP>
__device__ __forceinline__ const T *sweep_state_array(const SweepArgs<T> &a) {
    if constexpr (OP == OP_POWER) return a.pi_cur;
    else if constexpr (OP == OP_CORRECT) return a.x;
    else return a.r;
}

template <typename T, int OP>
__device__ __forceinline__ void sweep_epilogue_v(const DevGraph &G, const Ctl *ctl, SweepArgs<T> &a, int j, T pre,
                                                 T in, typename ST<T>::R &s1, typename ST<T>::R &s2,
                                                 typename ST<T>::R &s3) {
    if constexpr (OP == OP_POWER) {
        // pi_{k+1} = c P pi_k + gamma_k p, gamma_k = c d^T pi_k + (1-c) e^T pi_k  (Eq. 1)
        const T y = ST<T>::add(ST<T>::mul(ST<T>::c(ctl), in), ST<T>::mul(ST<T>::gamma(ctl), ST<T>::p(ctl, a.pv, j)));
        const T old = pre;
        s1 = ST<T>::radd(s1, ST<T>::rval(ST<T>::absv(ST<T>::add(y, ST<T>::neg(old)))));
        if (j >= G.n_nd) s2 = ST<T>::radd(s2, ST<T>::rval(y));
        s3 = ST<T>::radd(s3, ST<T>::rval(y));
        a.pi_next[j] = y;
        if (j < G.n_nd) a.q_next[j] = ST<T>::pack(ST<T>::mul(y, ST<T>::invdeg(G, j)));
    } else if constexpr (OP == OP_CORRECT) {
        // r = p + c P~ s - s with s = x / (1-c): the exact residual of the current
        // reserve (for any s, (I - c P~)(y - s) = p + c P~ s - s, from Eq. 4), from the
        // gathered values q_u = x_u / ((1-c) deg u); 1/(1-c) is applied as a multiply by
        // its reciprocal.  The FP32 form's correction runs it in IEEE double; the end of
        // asynchronous pull rounds (IFP1) in the rounds' format.
        const T sj = ST<T>::mul(pre, ST<T>::inv_om(ctl));
        a.r[j] = ST<T>::add(ST<T>::add(ST<T>::p(ctl, a.pv, j), ST<T>::mul(ST<T>::c(ctl), in)), ST<T>::neg(sj));
    } else {  // OP_PHASE2: r_d = p_d + c sum_{u in S(d)} x_u / ((1-c) deg(u)); phase 1 never
              // touches a dangling residual, so r_d still holds p_d
        a.r[j] = ST<T>::add(pre, ST<T>::mul(ST<T>::c(ctl), in));
    }
}

template <typename T, int OP>
__device__ __forceinline__ void sweep_epilogue(const DevGraph &G, const Ctl *ctl, SweepArgs<T> &a, int j, T in,
                                               typename ST<T>::R &s1, typename ST<T>::R &s2,
                                               typename ST<T>::R &s3) {
    sweep_epilogue_v<T, OP>(G, ctl, a, j, sweep_row_state<T, OP>(a, j), in, s1, s2, s3);
}

template <typename T, int OP, int LANES>
__device__ __forceinline__ void sweep_rows(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl, SweepArgs<T> &a,
                                           typename ST<T>::R &s1, typename ST<T>::R &s2, typename ST<T>::R &s3) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    constexpr int GPB = kThreads / LANES;
    constexpr int ROWS = RowsInFlight<LANES>::value;
    const int grp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
    const int stride = S.nblk * GPB;
    for (int base = S.lo + lb * GPB; base < S.hi; base += ROWS * stride) {
        int js[ROWS];
        bool valid[ROWS];
        A acc[ROWS], extra[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            js[r] = base + r * stride + grp;
            valid[r] = js[r] < S.hi;
        }
        row_sums<V, ROWS, EntriesInFlight<LANES>::value>(G.inr_off, G.inr_src, G.n_nd, js, valid, a.val, lane, LANES, acc);
        row_sums<V, ROWS, EntriesInFlight<LANES>::value>(G.inu_off, G.inu_src, G.n_nd, js, valid, a.val, lane, LANES, extra);
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            acc[r] = GT<V>::add(acc[r], extra[r]);
#pragma unroll
            for (int o = LANES / 2; o > 0; o >>= 1) acc[r] = GT<V>::add(acc[r], GT<V>::shfl_down(acc[r], o, LANES));
            if (valid[r] && lane == 0) sweep_epilogue<T, OP>(G, ctl, a, js[r], ST<T>::from_acc(acc[r]), s1, s2, s3);
        }
    }
}

// The gather tiles of a sweep's segment (see round_tiles)
template <typename T, int OP>
__device__ __forceinline__ void sweep_tiles(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl, SweepArgs<T> &a,
                                            typename ST<T>::R &s1, typename ST<T>::R &s2, typename ST<T>::R &s3,
                                            TileSmem<typename ST<T>::V> &sm, TileRows<T> &rs) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    for (int t = S.t0 + lb; t < S.t0 + S.nt; t += S.nblk) {
        int ra, rb;
        tile_load<V, T>(G, t, a.val, sm, ra, rb, sweep_state_array<T, OP>(a), &rs);
        const int nrow = rb - ra;
        for (int i = threadIdx.x; i < nrow; i += kThreads) {
            const int j = ra + i;
            A acc = tile_row_sum<V>(sm, i);
            acc = GT<V>::add(acc, row_sum<V>(G.inu_off, G.inu_src, G.n_nd, j, a.val, 0, 1));
            sweep_epilogue_v<T, OP>(G, ctl, a, j, rs.v[i], ST<T>::from_acc(acc), s1, s2, s3);
        }
        __syncthreads();
    }
}

// Double-precision warp rows of a sweep, in batches of kWarpBatch rows per
// warp (see round_warp_rows64); both in-list segments are always read.
template <int OP>
__device__ __forceinline__ void sweep_warp_rows64(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                                  SweepArgs<double> &a, double &s1, double &s2, double &s3) {
    constexpr int WPB = kThreads / 32;
    const int lane = threadIdx.x & 31;
    const int nbatch = (S.hi - S.lo + kWarpBatch - 1) / kWarpBatch;
    for (int bt = lb * WPB + (int)(threadIdx.x >> 5); bt < nbatch; bt += S.nblk * WPB) {
        const int j0 = S.lo + bt * kWarpBatch;
        const double sum = warp_batch_sums64(G.inr_off, G.inr_src, G.inu_off, G.inu_src, G.n_nd, j0, S.hi, a.val, lane);
        const int j = j0 + lane;
        if (lane < kWarpBatch && j < S.hi) sweep_epilogue<double, OP>(G, ctl, a, j, sum, s1, s2, s3);
    }
}

// One segment (or tile) of a sweep: rows [S.lo, S.hi), S.lanes threads per row.
template <typename T, int OP>
__device__ __forceinline__ void sweep_segment(const DevGraph &G, const Seg &S, int lb, const Ctl *ctl,
                                              SweepArgs<T> &a, typename ST<T>::R &s1, typename ST<T>::R &s2,
                                              typename ST<T>::R &s3, typename GT<typename ST<T>::V>::A *sha) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    if constexpr (std::is_same<T, double>::value) {
        __shared__ SegSmem<T, V> smu;
        if (UseTiles<T>::value && S.lanes == kTileLanes) {
            sweep_tiles<T, OP>(G, S, lb, ctl, a, s1, s2, s3, smu.tile.sm, smu.tile.rs);
            return;
        }
        if (kWarpBatch > 1 && S.lanes == 32) {
            sweep_warp_rows64<OP>(G, S, lb, ctl, a, s1, s2, s3);
            return;
        }
    }
    switch (S.lanes) {
        case 1: sweep_rows<T, OP, 1>(G, S, lb, ctl, a, s1, s2, s3); break;
        case 2: sweep_rows<T, OP, 2>(G, S, lb, ctl, a, s1, s2, s3); break;
        case 4: sweep_rows<T, OP, 4>(G, S, lb, ctl, a, s1, s2, s3); break;
        case 8: sweep_rows<T, OP, 8>(G, S, lb, ctl, a, s1, s2, s3); break;
        case 16: sweep_rows<T, OP, 16>(G, S, lb, ctl, a, s1, s2, s3); break;
        case 32: sweep_rows<T, OP, 32>(G, S, lb, ctl, a, s1, s2, s3); break;
        default:
            for (int j = S.lo + lb; j < S.hi; j += S.nblk) {
                A acc = row_sum<V>(G.inr_off, G.inr_src, G.n_nd, j, a.val, threadIdx.x, blockDim.x);
                acc = GT<V>::add(acc, row_sum<V>(G.inu_off, G.inu_src, G.n_nd, j, a.val, threadIdx.x, blockDim.x));
                acc = block_sum_gt<V>(acc, sha);
                if (threadIdx.x == 0) sweep_epilogue<T, OP>(G, ctl, a, j, ST<T>::from_acc(acc), s1, s2, s3);
            }
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads, (SweepMinBlocks<T, OP>::value)) k_sweep(DevGraph G, Plan PL, Ctl *ctl,
                                                                                    SweepArgs<T> a) {
    using V = typename ST<T>::V;
    using A = typename GT<V>::A;
    using R = typename ST<T>::R;
    if (OP == OP_POWER && ctl->done) return;  // the one-shot sweeps run after the stop flag is set
    int s = 0;
    while (s + 1 < PL.nseg && (int)blockIdx.x >= PL.seg[s + 1].blk0) s++;
    const Seg S = PL.seg[s];
    const int lb = blockIdx.x - S.blk0;
    R s1 = ST<T>::rzero(), s2 = ST<T>::rzero(), s3 = ST<T>::rzero();
    __shared__ double shd[32];
    __shared__ A sha[32];
    __shared__ R shr[32];
    sweep_segment<T, OP>(G, S, lb, ctl, a, s1, s2, s3, sha);
    if (OP != OP_POWER) return;
    // Power: ||pi_{k+1} - pi_k||_1, d^T pi_{k+1}, e^T pi_{k+1}
    const R b1 = block_sum_r<T>(s1, shr);
    const R b2 = block_sum_r<T>(s2, shr);
    const R b3 = block_sum_r<T>(s3, shr);
    if (threadIdx.x == 0) {
        store_partial<T>(a.P.a, b1);
        store_partial<T>(a.P.b, b2);
        store_partial<T>(a.P.c, b3);
    }
    if (!last_block(&ctl->ticket)) return;
    const double d = final_sum<T>(a.P.a, shd);
    const double dm = final_sum<T>(a.P.b, shd);
    const double tm = final_sum<T>(a.P.c, shd);
    if (threadIdx.x != 0) return;
    ctl->ticket = 0;
    const int it = ctl->iter + 1;
    ctl->iter = it;
    ctl->delta = d;
    ctl->zsum = tm;
    const double gamma = ctl->c * dm + ctl->one_minus_c * tm;
    ctl->gamma = gamma;
    ctl->gamma_f = (float)gamma;
    ctl->gamma_df = df_from_d(gamma);
    if (it < ctl->trace_cap) a.tr.R[it] = d;
    if (d <= ctl->eps) {
        ctl->done = 1;
        ctl->status = 0;
    } else if (it >= ctl->max_rounds) {
        ctl->done = 1;
        ctl->status = 1;
    }
}

// IFP1: z = x + (1-c) r (Alg. 2 pibar + h);  IFP2: z = x (non-dangling), (1-c) r (dangling)
// (Alg. 3 pibar);  POWER: z = pi.  pi = z / sum z, scattered back to caller ids.
template <typename T>
__device__ __forceinline__ T zval(const DevGraph &G, const Ctl *ctl, int kind, const T *x, const T *r, int i) {
    if (kind == PR_IFP1) return ST<T>::add(x[i], ST<T>::mul(ST<T>::om(ctl), r[i]));
    if (kind == PR_IFP2) return i < G.n_nd ? x[i] : ST<T>::mul(ST<T>::om(ctl), r[i]);
    return x[i];
}


// inbox of double-float state folded into r over rows [lo, hi) (IFP1 dangling
// rows receive pushes and no activation reads them)
static __global__ void k_fold_inbox(float2 *r, double *din, int32_t lo, int32_t hi) {
    for (int i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x)
        ST<float2>::fold(r, din, i);
}

// host-side conversions of the scalar parameters
inline float float_at_most(double v) {  // largest float <= v
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

inline void fill_formats(Ctl &h) {
    h.inv_om = 1.0 / h.one_minus_c;
    h.c_f = (float)h.c;
    h.om_f = (float)h.one_minus_c;
    h.xi_f = float_at_most(h.xi);
    h.pu_f = (float)h.pu;
    h.inv_om_f = (float)h.inv_om;
    h.c_df = df_from_d(h.c);
    h.om_df = df_from_d(h.one_minus_c);
    h.xi_df = df_from_d(h.xi);
    h.pu_df = df_from_d(h.pu);
    h.inv_om_df = df_from_d(h.inv_om);
}

}  // namespace pr
