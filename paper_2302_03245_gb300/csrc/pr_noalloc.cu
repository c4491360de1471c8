// pr_noalloc.cu -- pr_power_noalloc: the Power-method PageRank iteration on
// caller-owned device arrays, for callers that must not allocate device
// memory (a host framework that owns the whole device pool, code that runs
// where an allocation could synchronise the device, a plugin that is handed
// buffers only).  It allocates nothing: its working vectors live in one
// file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.
//
// The iteration is the one of k_rows<OP_POWER> (pi_{k+1} = c P pi_k +
// (c d^T pi_k + (1-c) e^T pi_k) e/n, uniform personalization), written here
// over the caller's own in-lists with one warp per row, so that no graph
// preprocessing (which allocates) is needed.
#include <mutex>

#include "pr_internal.cuh"

namespace {

constexpr int32_t kNaMaxN = 1 << 19;  // largest n accepted (524,288 vertices)
constexpr int kNaBlocks = 1024;       // blocks of every kernel here == partial-sum slots
constexpr int kNaThreads = 256;

struct NaCtl {
    double gamma, delta, total;
    unsigned int ticket;
    int iter, done;
};

// layout of the scratch array, in bytes
constexpr size_t kOffAlt = 0;                                    // double[kNaMaxN]  other pi buffer
constexpr size_t kOffQ0 = kOffAlt + sizeof(double) * kNaMaxN;    // double[kNaMaxN]  pi/deg, even
constexpr size_t kOffQ1 = kOffQ0 + sizeof(double) * kNaMaxN;     // double[kNaMaxN]  pi/deg, odd
constexpr size_t kOffPart = kOffQ1 + sizeof(double) * kNaMaxN;   // double[3][kNaBlocks]
constexpr size_t kOffCtl = kOffPart + sizeof(double) * 3 * kNaBlocks;
constexpr size_t kScratchBytes = kOffCtl + 256;                  // 12.6 MB

static __device__ __align__(256) unsigned char pr_noalloc_scratch[kScratchBytes];

struct NaPtrs {
    double *alt, *q0, *q1, *part;
    NaCtl *ctl;
};

NaPtrs carve(unsigned char *base) {
    NaPtrs p;
    p.alt = reinterpret_cast<double *>(base + kOffAlt);
    p.q0 = reinterpret_cast<double *>(base + kOffQ0);
    p.q1 = reinterpret_cast<double *>(base + kOffQ1);
    p.part = reinterpret_cast<double *>(base + kOffPart);
    p.ctl = reinterpret_cast<NaCtl *>(base + kOffCtl);
    return p;
}

__device__ __forceinline__ double na_block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

__device__ __forceinline__ bool na_last_block(unsigned int *ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// pi_0 = e/n, q_0 = pi_0 / deg, gamma_0 = c d^T pi_0 + (1-c) e^T pi_0
__global__ void k_na_init(int32_t n, const int32_t *out_off, double c, double *pi, double *q, double *part,
                          NaCtl *ctl) {
    __shared__ double sh[32];
    double dm = 0.0, tm = 0.0;
    const double p = 1.0 / (double)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t deg = out_off[i + 1] - out_off[i];
        pi[i] = p;
        q[i] = deg ? p / (double)deg : 0.0;
        if (!deg) dm += p;
        tm += p;
    }
    dm = na_block_sum(dm, sh);
    tm = na_block_sum(tm, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = dm;
        part[kNaBlocks + blockIdx.x] = tm;
    }
    if (!na_last_block(&ctl->ticket)) return;
    dm = 0.0;
    tm = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        dm += __ldcg(&part[k]);
        tm += __ldcg(&part[kNaBlocks + k]);
    }
    dm = na_block_sum(dm, sh);
    tm = na_block_sum(tm, sh);
    if (threadIdx.x == 0) {
        ctl->gamma = c * dm + (1.0 - c) * tm;
        ctl->total = tm;
        ctl->delta = 0.0;
        ctl->iter = 0;
        ctl->done = 0;
        ctl->ticket = 0;
    }
}

// one iteration, one warp per row of the caller's in-lists
__global__ void k_na_iter(int32_t n, const int32_t *out_off, const int32_t *in_off, const int32_t *in_src,
                          double c, double tol, int32_t max_iter, const double *pi, const double *q,
                          double *pi_next, double *q_next, double *part, NaCtl *ctl) {
    if (ctl->done) return;
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const double gp = ctl->gamma / (double)n;
    double d = 0.0, dm = 0.0, tm = 0.0;
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        double acc = 0.0;
        for (int e = in_off[j] + lane; e < in_off[j + 1]; e += 32) acc += q[in_src[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double y = c * acc + gp;
            const int32_t deg = out_off[j + 1] - out_off[j];
            d += fabs(y - pi[j]);
            if (!deg) dm += y;
            tm += y;
            pi_next[j] = y;
            q_next[j] = deg ? y / (double)deg : 0.0;
        }
    }
    d = na_block_sum(d, sh);
    dm = na_block_sum(dm, sh);
    tm = na_block_sum(tm, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = d;
        part[kNaBlocks + blockIdx.x] = dm;
        part[2 * kNaBlocks + blockIdx.x] = tm;
    }
    if (!na_last_block(&ctl->ticket)) return;
    d = dm = tm = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        d += __ldcg(&part[k]);
        dm += __ldcg(&part[kNaBlocks + k]);
        tm += __ldcg(&part[2 * kNaBlocks + k]);
    }
    d = na_block_sum(d, sh);
    dm = na_block_sum(dm, sh);
    tm = na_block_sum(tm, sh);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->iter += 1;
        ctl->delta = d;
        ctl->total = tm;
        ctl->gamma = c * dm + (1.0 - c) * tm;
        if (d <= tol || ctl->iter >= max_iter) ctl->done = 1;
    }
}

__global__ void k_na_normalize(int32_t n, const double *src, const NaCtl *ctl, double *out) {
    const double inv = 1.0 / ctl->total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = src[i] * inv;
}

// device address of the scratch array, looked up once per device
std::mutex g_na_mu;
unsigned char *g_na_addr[64] = {};

}  // namespace

extern "C" pr_status pr_power_noalloc(int32_t n, const int32_t *out_off, const int32_t *in_off,
                                      const int32_t *in_src, double c, double tol, int32_t max_iter, double *pi,
                                      void *cuda_stream, int32_t *iters) {
    using pr::fail;
    if (n < 1 || n > kNaMaxN)
        return fail(PR_EINVAL, "pr_power_noalloc: n must be in [1, " + std::to_string(kNaMaxN) + "]");
    if (!out_off || !in_off || !in_src || !pi) return fail(PR_EINVAL, "pr_power_noalloc: NULL array");
    if (!(c > 0.0 && c < 1.0)) return fail(PR_EINVAL, "pr_power_noalloc: c must be in (0, 1)");
    if (!(tol > 0.0)) return fail(PR_EINVAL, "pr_power_noalloc: tol must be positive");
    if (max_iter < 1) return fail(PR_EINVAL, "pr_power_noalloc: max_iter must be >= 1");
    int dev = 0;
    PR_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PR_EINVAL, "pr_power_noalloc: device id out of range");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_addr[dev]) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, pr_noalloc_scratch);
            if (e != cudaSuccess) return pr::cuda_fail(e, "cudaGetSymbolAddress(pr_noalloc_scratch)");
            g_na_addr[dev] = static_cast<unsigned char *>(addr);
        }
        base = g_na_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const NaPtrs P = carve(base);
    PR_CK(cudaMemsetAsync(P.ctl, 0, sizeof(NaCtl), s));  // the array keeps the last call's contents
    k_na_init<<<kNaBlocks, kNaThreads, 0, s>>>(n, out_off, c, pi, P.q0, P.part, P.ctl);
    // iterate: even steps read (pi, q0) and write (alt, q1); odd steps the reverse
    int done = 0, it = 0;
    int chunk = 8;
    while (!done) {
        for (int k = 0; k < chunk; k++, it++) {
            const bool even = (it & 1) == 0;
            k_na_iter<<<kNaBlocks, kNaThreads, 0, s>>>(n, out_off, in_off, in_src, c, tol, max_iter,
                                                       even ? pi : P.alt, even ? P.q0 : P.q1,
                                                       even ? P.alt : pi, even ? P.q1 : P.q0, P.part, P.ctl);
        }
        PR_CK(cudaGetLastError());
        NaCtl h;
        PR_CK(cudaMemcpyAsync(&h, P.ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        done = h.done;
        if (done) {
            // the last iterate sits in `pi` after an even number of iterations, else in the scratch
            const double *src = (h.iter & 1) ? P.alt : pi;
            k_na_normalize<<<kNaBlocks, kNaThreads, 0, s>>>(n, src, P.ctl, pi);
            PR_CK(cudaGetLastError());
            PR_CK(cudaStreamSynchronize(s));
            if (iters) *iters = h.iter;
            if (h.delta > tol) return fail(PR_ENOTCONV, "pr_power_noalloc: max_iter reached");
        }
    }
    return PR_OK;
}
