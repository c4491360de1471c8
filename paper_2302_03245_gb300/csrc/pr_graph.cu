// pr_graph.cu -- error state, device allocator, and pr_graph_create: the
// preprocessing that Alg. 2 and Alg. 3 start with (Sec. 3.4), on the GPU.
//
// From the caller's out-lists this builds, on the device:
//   * out-degree / in-degree, the dangling (deg = 0) and unreferenced
//     (in-degree 0) classes (Sec. 2.1);
//   * an internal vertex numbering [referenced non-dangling | unreferenced
//     non-dangling | dangling], each class sorted by in-degree (descending);
//   * sorted internal out-lists, whose non-dangling targets form a prefix of
//     length ndeg[i] -- the IFP2 edge invalidation of Sec. 3.4 is then a
//     per-row length, no edge is moved or deleted;
//   * in-lists split into a "ref" segment (sources with in-edges) and an
//     "unref" segment (unreferenced sources), both sorted.
// Sorting uses CUB's device radix sort; everything else is hand-written.

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cstring>
#include <thread>
#include <vector>

#include "pr_debug.cuh"
#include "pr_internal.cuh"
#include "pr_sort.cuh"

namespace pr {

// ------------------------------------------------------------ error state
static thread_local std::string t_err;
void set_error(const std::string &msg) { t_err = msg; }
pr_status fail(pr_status st, const std::string &msg) {
    t_err = msg;
    return st;
}
pr_status cuda_fail(cudaError_t e, const char *what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PR_ECUDA;
}

// ------------------------------------------------------------ allocator
static pr_alloc_fn g_alloc = nullptr;
static pr_free_fn g_free = nullptr;
static void *g_ctx = nullptr;

void *dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (g_alloc) return g_alloc(bytes, (void *)s, g_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (g_free) g_free(p, bytes, (void *)s, g_ctx);
    else cudaFree(p);
}

// A buffer remembers the allocator that made it, so a later pr_set_allocator
// does not hand it to the wrong free function.
pr_status Buf::alloc(size_t nbytes, cudaStream_t stream) {
    release();
    s = stream;
    if (nbytes == 0) nbytes = 16;
    if (g_alloc) {
        p = g_alloc(nbytes, (void *)stream, g_ctx);
        ffn = g_free;
        fctx = g_ctx;
    } else {
        if (cudaMalloc(&p, nbytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        ffn = nullptr;
        fctx = nullptr;
    }
    if (!p) return fail(PR_ENOMEM, "device allocation of " + std::to_string(nbytes) + " bytes failed");
    bytes = nbytes;
    return PR_OK;
}

void Buf::release() {
    if (p) {
        if (stream_ordered) cudaFreeAsync(p, s);
        else if (ffn) ffn(p, bytes, (void *)s, fctx);
        else cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    stream_ordered = false;
}

pr_status Buf::alloc_async(size_t nbytes, cudaStream_t stream, cudaMemPool_t pool) {
    release();
    s = stream;
    if (nbytes == 0) nbytes = 16;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, nbytes, pool, stream) : cudaMallocAsync(&p, nbytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return fail(PR_ENOMEM, "device allocation of " + std::to_string(nbytes) + " bytes failed");
    }
    bytes = nbytes;
    ffn = nullptr;
    fctx = nullptr;
    stream_ordered = true;
    return PR_OK;
}

// ------------------------------------------------------------ kernels
static __global__ void k_validate(int32_t n, int64_t m, const int32_t *off, const int32_t *dst,
                                  unsigned long long *bad) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i <= n; i += stride) {
        int32_t o = off[i];
        if (i == 0 && o != 0) atomicAdd(&bad[0], 1ULL);
        if (i == n && (int64_t)o != m) atomicAdd(&bad[0], 1ULL);
        if (i < n && off[i + 1] < o) atomicAdd(&bad[0], 1ULL);
        if (o < 0 || (int64_t)o > m) atomicAdd(&bad[0], 1ULL);
    }
    for (int64_t e = tid; e < m; e += stride) {
        int32_t d = dst[e];
        if (d < 0 || d >= n) atomicAdd(&bad[1], 1ULL);
    }
}

static __global__ void k_indeg(int64_t m, const int32_t *dst, int32_t *indeg) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(&indeg[dst[e]], 1);
}

// Level of every non-dangling vertex with in-edges (level-ordered rounds):
// ranked by q = floor(2^31 (indeg + 1) / (indeg + outdeg + 2)) < 2^31,
// ascending, ties by id (the key packs q << B | id); the others sort after
// them (all ones in the 31 + B bits sorted).
static __global__ void k_level_keys(int32_t n, const int32_t *off, const int32_t *indeg, int B, uint64_t *keys,
                                    unsigned int *n_ref) {
    __shared__ unsigned int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    unsigned int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t deg = off[i + 1] - off[i], id = indeg[i];
        if (deg > 0 && id > 0) {
            const uint64_t q = ((uint64_t)(id + 1) << 31) / (uint64_t)(id + deg + 2);
            keys[i] = (q << B) | (uint64_t)(uint32_t)i;
            c++;
        } else {
            keys[i] = ~0ULL;
        }
    }
    if (c) atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0 && cnt) atomicAdd(n_ref, cnt);
}

// rank r of n_ref (sorted keys) -> level floor(r L / n_ref)
static __global__ void k_assign_levels(const uint64_t *sorted, int32_t n_ref, int32_t L, int B, int32_t *level) {
    const uint64_t id_mask = (1ULL << B) - 1;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_ref; r += gridDim.x * blockDim.x)
        level[(int32_t)(sorted[r] & id_mask)] = (int32_t)(((int64_t)r * L) / n_ref);
}

// valid out-edges of each non-dangling row into its own or a lower level (the
// pushes a level-ordered round leaves for the next round); rows without
// in-edges are scanned last, so all their pushes wait
static __global__ void k_level_back(int32_t n_ref, int32_t n_nd, const int32_t *out_off, const int32_t *out_dst,
                                    const int32_t *ndeg, const int32_t *lo, int32_t L, int32_t *back) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_nd; j += gridDim.x * blockDim.x) {
        if (j >= n_ref) {
            back[j] = ndeg[j];
            continue;
        }
        int a = 0, b = L - 1;  // the level of row j: the last l with lo[l] <= j
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (lo[mid] <= j) a = mid;
            else b = mid - 1;
        }
        const int32_t end = lo[a + 1];
        int32_t x = out_off[j], y = out_off[j] + ndeg[j];  // valid targets, ascending
        while (x < y) {
            const int32_t mid = x + ((y - x) >> 1);
            if (out_dst[mid] < end) x = mid + 1;
            else y = mid;
        }
        back[j] = x - out_off[j];
    }
}

// class 0: deg>0 & indeg>0, class 1: deg>0 & indeg==0, class 2: deg==0.
// key = class << (LB + IB) | level << IB | (2^IB - 1 - indeg), with indeg <=
// m < 2^IB and LB = 4 level bits on level-ordered graphs (else 0): a stable
// sort on the low 2 + LB + IB bits orders by class, level, in-degree
// descending, then id.
static __global__ void k_vertex_keys(int32_t n, const int32_t *off, const int32_t *indeg, const int32_t *level,
                                     int IB, int LB, uint64_t *keys, int32_t *vals, unsigned int *class_cnt) {
    __shared__ unsigned int cnt[3];
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned int local[3] = {0, 0, 0};
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int32_t deg = off[i + 1] - off[i];
        int32_t id = indeg[i];
        uint32_t cls = deg == 0 ? 2u : (id == 0 ? 1u : 0u);
        const uint64_t lev = (cls == 0 && level) ? (uint64_t)level[i] : 0;  // level-ordered graphs
        keys[i] = ((uint64_t)cls << (LB + IB)) | (lev << IB) | (((1ULL << IB) - 1) - (uint64_t)(uint32_t)id);
        vals[i] = i;
        local[cls]++;
    }
    for (int k = 0; k < 3; k++)
        if (local[k]) atomicAdd(&cnt[k], local[k]);
    __syncthreads();
    if (threadIdx.x < 3 && cnt[threadIdx.x]) atomicAdd(&class_cnt[threadIdx.x], cnt[threadIdx.x]);
}

static __global__ void k_invert(int32_t n, const int32_t *perm, int32_t *inv) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) inv[perm[i]] = i;
}

// Edge keys in internal ids, packed as src << (B+1) | flag << B | dst, with
// flag = (src >= n_ref): the source is unreferenced.  off/ent are caller
// lists: row v holds the entries ent[off[v] .. off[v+1]), and row_is_src says
// whether the row is the source end (out-lists) or the target end (in-lists).
// With pos (the internal out-list offsets), entry e of row v is written to
// pos[inv[v]] + (e - off[v]), which groups the keys by internal source;
// without it, to index e.  With counts, the keys' digits of a radix sort on
// bits [cbegin, cend) are counted on the way (radix_count_key).
//
// A warp takes chunks of 32 * kEdgeChunk consecutive entries, lane l the
// entries base + l + 32 j.  A lane finds the row of its first entry by binary
// search and then walks forward through the offsets, about one cached offset
// read per entry (a binary search per entry cost 0.8 ms on 47M edges); a walk
// that passes more than kWalk rows (a run of empty rows) finishes by binary
// search.  The offsets are validated before this runs: off[0] = 0,
// non-decreasing, off[n] = m.
constexpr int kEdgeChunk = 16;
constexpr int kWalk = 4;
static __global__ void k_edge_keys(int32_t n, int64_t m, const int32_t *off, const int32_t *ent,
                                   const int32_t *inv, int B, int32_t n_ref, int row_is_src,
                                   const int32_t *pos, uint64_t *keys, int cbegin, int cend, uint32_t *counts) {
    __shared__ uint32_t h[kRadixMaxPasses][kRadixDigits];
    if (counts) {
        for (int k = threadIdx.x; k < kRadixMaxPasses * kRadixDigits; k += blockDim.x) (&h[0][0])[k] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t chunk = 32 * kEdgeChunk;
    for (int64_t base = warp * chunk; base < m; base += nwarps * chunk) {
        int64_t e = base + lane;
        if (e >= m) break;
        int32_t lo = 0, hi = n;  // the last row with off[row] <= e (off[n] = m > e)
        while (hi - lo > 1) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if ((int64_t)off[mid] <= e) lo = mid;
            else hi = mid;
        }
        int32_t row = lo;
        for (int j = 0; j < kEdgeChunk && e < m; j++, e += 32) {
            for (int w = 0; (int64_t)off[row + 1] <= e; w++) {
                if (w == kWalk) {  // off[row + 1] <= e < off[n]: search (row + 1, n)
                    lo = row + 1;
                    hi = n;
                    while (hi - lo > 1) {
                        const int32_t mid = lo + ((hi - lo) >> 1);
                        if ((int64_t)off[mid] <= e) lo = mid;
                        else hi = mid;
                    }
                    row = lo;
                    break;
                }
                row++;
            }
            const uint64_t r = (uint64_t)inv[row], c = (uint64_t)inv[ent[e]];
            const uint64_t src = row_is_src ? r : c, dst = row_is_src ? c : r;
            const uint64_t key = (src << (B + 1)) | ((src >= (uint64_t)n_ref ? 1ULL : 0ULL) << B) | dst;
            keys[pos ? (int64_t)pos[r] + (e - (int64_t)off[row]) : e] = key;
            if (counts) radix_count_key(h, key, cbegin, cend);
        }
    }
    if (counts) {
        __syncthreads();
        radix_count_flush(h, cbegin, cend, counts);
    }
}

// One pass over the keys sorted by (flag, dst, src): the source of entry e
// goes to inr_src[e] (e < m_ref, referenced sources) or inu_src[e - m_ref];
// each run of equal (flag, dst) adds its length to cnt[flag * (n + 1) + dst]
// (its first entry adds -e, its last e + 1); equal neighbours are repeated
// edges; the digits of the sort on the source bits [B+1, 2B+1) are counted
// (radix_count_key).
static __global__ void k_in_lists(int64_t m, const uint64_t *keys, int B, int32_t n, int64_t m_ref,
                                  int32_t *inr_src, int32_t *inu_src, int32_t *cnt, unsigned long long *dups,
                                  uint32_t *counts) {
    __shared__ uint32_t h[kRadixMaxPasses][kRadixDigits];
    for (int k = threadIdx.x; k < kRadixMaxPasses * kRadixDigits; k += blockDim.x) (&h[0][0])[k] = 0;
    __syncthreads();
    const uint64_t low_mask = (1ULL << (B + 1)) - 1, id_mask = (1ULL << B) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint64_t k = keys[e], f = k & low_mask;
        const int32_t src = (int32_t)((k >> (B + 1)) & id_mask);
        if (e < m_ref) inr_src[e] = src;
        else inu_src[e - m_ref] = src;
        int32_t *row = cnt + (int64_t)(f >> B) * (n + 1) + (int64_t)(f & id_mask);
        if (e == 0 || (keys[e - 1] & low_mask) != f) atomicAdd(row, (int32_t)-e);
        if (e + 1 == m || (keys[e + 1] & low_mask) != f) atomicAdd(row, (int32_t)(e + 1));
        c += e > 0 && keys[e - 1] == k;
        radix_count_key(h, k, B + 1, 2 * B + 1);
    }
    if (c) atomicAdd(dups, c);
    __syncthreads();
    radix_count_flush(h, B + 1, 2 * B + 1, counts);
}

// a field of every key: col[e] = (keys[e] >> shift) & mask
static __global__ void k_field(int64_t m, const uint64_t *keys, int shift, uint64_t mask, int32_t *col) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride)
        col[e] = (int32_t)((keys[e] >> shift) & mask);
}

// positions where two key arrays differ
static __global__ void k_count_diff(int64_t m, const uint64_t *a, const uint64_t *b, unsigned long long *cnt) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride) c += a[e] != b[e];
    if (c) atomicAdd(cnt, c);
}

// deg[i] = out-degree of internal vertex i (caller vertex perm[i]); deg[n] = 0.
// Its exclusive sum is the internal out-list offsets.
static __global__ void k_new_degrees(int32_t n, const int32_t *off, const int32_t *perm, int32_t *deg) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride)
        deg[i] = i < n ? off[perm[i] + 1] - off[perm[i]] : 0;
}

static __global__ void k_vertex_arrays(int32_t n_nd, const int32_t *off, const int32_t *dst,
                                       int32_t *ndeg, double *inv64, float *inv32, float2 *invdf) {
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nd; i += stride) {
        int32_t a = off[i], b = off[i + 1];
        int32_t lo = a, hi = b;  // first target >= n_nd
        while (lo < hi) {
            int32_t mid = lo + ((hi - lo) >> 1);
            if (dst[mid] < n_nd) lo = mid + 1;
            else hi = mid;
        }
        ndeg[i] = lo - a;
        double inv = 1.0 / (double)(b - a);
        inv64[i] = inv;
        inv32[i] = (float)inv;
        const float inv_hi = __double2float_rn(inv);
        invdf[i] = make_float2(inv_hi, __double2float_rn(inv - (double)inv_hi));
    }
}

// m_d, n_u and the maximum out- and in-degrees (block-aggregated)
static __global__ void k_degree_facts(int32_t n, int32_t n_nd, const int32_t *perm, const int32_t *indeg_ext,
                                      const int32_t *off_int, unsigned int *n_u,
                                      int *maxes, unsigned long long *m_d) {
    __shared__ unsigned int s_u;
    __shared__ int s_max[2];
    __shared__ unsigned long long s_md;
    if (threadIdx.x == 0) {
        s_u = 0;
        s_max[0] = s_max[1] = 0;
        s_md = 0;
    }
    __syncthreads();
    unsigned int u = 0;
    int mo = 0, mi = 0;
    unsigned long long md = 0;
    int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int32_t id = indeg_ext[perm[i]];
        int32_t od = off_int[i + 1] - off_int[i];
        if (i >= n_nd) md += (unsigned long long)id;
        u += id == 0;
        mo = max(mo, od);
        mi = max(mi, id);
    }
    if (u) atomicAdd(&s_u, u);
    if (md) atomicAdd(&s_md, md);
    atomicMax(&s_max[0], mo);
    atomicMax(&s_max[1], mi);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_u) atomicAdd(n_u, s_u);
        if (s_md) atomicAdd(m_d, s_md);
        atomicMax(&maxes[0], s_max[0]);
        atomicMax(&maxes[1], s_max[1]);
    }
}

// bins[k] = number of rows in [lo, hi) (in-degree sorted descending) with indeg > thr[k]
// range blockIdx.x [lo, hi): the first row whose in-degree (ref + unref
// segments) is <= thr[k]; the rows of a range are sorted by in-degree, descending
static __global__ void k_bin_bounds(const int32_t *inr_off, const int32_t *inu_off, const int32_t *lo,
                                    const int32_t *hi, const int32_t *thr, int nthr, int32_t *bounds) {
    const int k = threadIdx.x;
    if (k >= nthr) return;
    int32_t a = lo[blockIdx.x], b = hi[blockIdx.x];
    while (a < b) {
        int32_t mid = a + ((b - a) >> 1);
        const int32_t d = (inr_off[mid + 1] - inr_off[mid]) + (inu_off[mid + 1] - inu_off[mid]);
        if (d > thr[k]) a = mid + 1;
        else b = mid;
    }
    bounds[blockIdx.x * nthr + k] = a;
}

// edges of the ref+unref in-list segments in [lo, hi) of rows (for block budgets)
static __global__ void k_range_edges(const int32_t *inr_off, const int32_t *inu_off, const int32_t *rows,
                                     int nrows, long long *edges) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    edges[k] = (long long)inr_off[rows[k]] + inu_off[rows[k]];
}

static int grid_for(int64_t items, int num_sms) {
    int64_t b = (items + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

static int bits_for(int32_t n) {
    int B = 1;
    while (B < 31 && ((int64_t)1 << B) < (int64_t)n) B++;
    return B;
}

// ------------------------------------------------------------ gather tiles
// in-list offsets at the first and last tiled row of each range
static __global__ void k_tile_ends(const int32_t *inr_off, const int32_t *lo, const int32_t *hi, int nr,
                                   int32_t *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    out[2 * k] = lo[k] < hi[k] ? inr_off[lo[k]] : 0;
    out[2 * k + 1] = lo[k] < hi[k] ? inr_off[hi[k] - 1] : 0;
}

// unit position of row j of a tiled range (entries before it plus kTileW per row)
__device__ __forceinline__ long long tile_unit(const int32_t *inr_off, int32_t lo, int32_t e_lo, int32_t j) {
    return (long long)(inr_off[j] - e_lo) + (long long)kTileW * (j - lo);
}

// tab[t] = first row of tile t, tab[nt] = hi: rows whose first unit lies in
// [t U, (t+1) U) form tile t; a row spans fewer than U units, so every tile
// index up to the last row's gets exactly one first row
static __global__ void k_tile_marks(const int32_t *inr_off, int32_t lo, int32_t hi, int32_t *tab) {
    const int32_t e_lo = inr_off[lo];
    for (int32_t j = lo + blockIdx.x * blockDim.x + threadIdx.x; j < hi; j += gridDim.x * blockDim.x) {
        const long long t = tile_unit(inr_off, lo, e_lo, j) / kTileU;
        const bool first = j == lo || tile_unit(inr_off, lo, e_lo, j - 1) / kTileU != t;
        if (first) tab[t] = j;
        if (j == hi - 1) tab[t + 1] = hi;
    }
}

// ------------------------------------------------------------ plans
// Blocks go to segments in proportion to their work (in-list entries + 2 per
// row), at most as many as the segment has row groups, within a budget of
// block_budget + one per segment (< kMaxBlocks).
struct RangeSpec {
    int32_t lo, hi, lanes;
    long long edges;
    int32_t t0 = 0, nt = 0;  // gather tiles (lanes == kTileLanes)
};

static Plan make_plan(const RangeSpec *r, int nr, int budget) {
    Plan P{};
    double total = 0;
    for (int k = 0; k < nr; k++)
        if (r[k].hi > r[k].lo) total += (double)r[k].edges + 2.0 * (r[k].hi - r[k].lo);
    int blk = 0;
    for (int k = 0; k < nr && P.nseg < kMaxSeg; k++) {
        if (r[k].hi <= r[k].lo) continue;
        const int64_t rows = r[k].hi - r[k].lo;
        const double work = (double)r[k].edges + 2.0 * rows;
        const int64_t groups_per_block = r[k].lanes > 0 ? kThreads / r[k].lanes : 1;
        const int64_t need = r[k].lanes == kTileLanes ? r[k].nt : (rows + groups_per_block - 1) / groups_per_block;
        int64_t nb = (int64_t)(budget * (work / std::max(total, 1.0)) + 0.5);
        nb = std::max<int64_t>(1, std::min(nb, need));
        if (r[k].lanes == kClusterLanes) nb = rows * kLevelCluster;  // one cluster per row, whatever the budget
        Seg &sg = P.seg[P.nseg++];
        sg.lo = r[k].lo;
        sg.hi = r[k].hi;
        sg.lanes = r[k].lanes;
        sg.blk0 = blk;
        sg.nblk = (int32_t)nb;
        sg.t0 = r[k].t0;
        sg.nt = r[k].nt;
        blk += (int)nb;
    }
    P.nblocks = std::max(blk, 1);
    return P;
}

// rows [lo, hi) of one class split at bounds[0..5] into block / 32 / 16 / 8 / 4 / 2 / 1 lanes
static int class_ranges(int32_t lo, int32_t hi, const int32_t *bounds, const long long *e_lo,
                        const long long *e_b, long long e_hi, RangeSpec *out) {
    static const int lanes[kNumThr + 1] = {0, 32, 16, 8, 4, 2, 1};
    int32_t a = lo;
    long long ea = *e_lo;
    for (int k = 0; k <= kNumThr; k++) {
        const int32_t b = k < kNumThr ? bounds[k] : hi;
        const long long eb = k < kNumThr ? e_b[k] : e_hi;
        out[k] = RangeSpec{a, b, lanes[k], eb - ea, 0, 0};
        a = b;
        ea = eb;
    }
    return kNumThr + 1;
}

void build_plans(pr_graph *g) {
    const int32_t n_nd = g->G.n_nd, n_ref = g->G.n_ref;
    const int nr = g->nranges;  // referenced ranges (levels), then the dangling range
    std::vector<RangeSpec> ref, d, lvl[kMaxLevels], ref_t, d_t;
    // level-ordered rounds: every row above kClusterRowMin in-list entries gets
    // a block cluster, unless all levels' clusters together would take more
    // than half the partial-sum slots; then the clusters per level are halved
    // until they fit (the rows are sorted by in-degree: the longest keep theirs)
    int32_t max_rows = kMaxBlocks / kLevelCluster;
    auto cluster_total = [&](int32_t cap) {
        long long t = 0;
        for (int k = 0; k + 1 < nr && g->levels; k++)
            t += (long long)std::min(cap, std::max(0, g->cl_hi[k] - g->range_lo[k])) * kLevelCluster;
        return t;
    };
    while (max_rows > 1 && cluster_total(max_rows) > kMaxBlocks / 2) max_rows /= 2;
    const long long cluster_blocks = g->levels ? cluster_total(max_rows) : 0;
    for (int k = 0; k < nr; k++) {
        const long long *E = &g->range_edges[(size_t)k * (kNumThr + 2)];
        RangeSpec rs[kNumThr + 1];
        class_ranges(g->range_lo[k], g->range_hi[k], &g->bounds[(size_t)k * kNumThr], &E[0], &E[1], E[kNumThr + 1],
                     rs);
        // the tiled variant: the block and warp bins, then the short rows as tiles
        std::vector<RangeSpec> tiled;
        if (g->tile_nt[k] > 0) {
            tiled.push_back(rs[0]);
            tiled.push_back(rs[1]);
            RangeSpec t{g->tile_lo[k], g->range_hi[k], kTileLanes, 0, g->tile_t0[k], g->tile_nt[k]};
            for (int c = 2; c <= kNumThr; c++) t.edges += rs[c].edges;
            tiled.push_back(t);
        } else {
            tiled.assign(rs, rs + kNumThr + 1);
        }
        for (int c = 0; c <= kNumThr; c++) {
            const RangeSpec &r = rs[c];
            if (k < nr - 1) {
                ref.push_back(r);
                if (!g->levels) continue;
                // the longest rows by clusters (first in the plan), then one block
                // per row down to kLevelBlockRowMin entries, then warps
                const int32_t bh = std::max(rs[0].hi, g->lb_hi[k]);  // end of the level's block rows
                if (c == 0) {
                    const int32_t ch = std::min(g->cl_hi[k], r.lo + max_rows);
                    lvl[k].push_back(RangeSpec{r.lo, ch, kClusterLanes, r.edges, 0, 0});
                    lvl[k].push_back(RangeSpec{ch, bh, 0, r.edges, 0, 0});
                } else if (c == 1) {
                    lvl[k].push_back(RangeSpec{bh, r.hi, 32, r.edges, 0, 0});
                } else {
                    lvl[k].push_back(r);
                }
            } else {
                d.push_back(r);
            }
        }
        for (const RangeSpec &r : tiled) (k < nr - 1 ? ref_t : d_t).push_back(r);
    }
    // unreferenced rows (no in-edges): one lane each; their in-lists are empty
    const long long e_ref_end = g->range_edges[(size_t)(nr - 2) * (kNumThr + 2) + kNumThr + 1];
    const long long e_nd = g->range_edges[(size_t)(nr - 1) * (kNumThr + 2)];
    const RangeSpec unref{n_ref, n_nd, 1, e_nd - e_ref_end, 0, 0};
    std::vector<RangeSpec> nd = ref, all = ref, nd_t = ref_t, all_t = ref_t;
    nd.push_back(unref);
    all.push_back(unref);
    all.insert(all.end(), d.begin(), d.end());
    nd_t.push_back(unref);
    all_t.push_back(unref);
    all_t.insert(all_t.end(), d_t.begin(), d_t.end());
    g->plan_nd = make_plan(nd.data(), (int)nd.size(), g->block_budget);
    g->plan_d = make_plan(d.data(), (int)d.size(), g->block_budget);
    g->plan_all = make_plan(all.data(), (int)all.size(), g->block_budget);
    g->plan_nd_t = make_plan(nd_t.data(), (int)nd_t.size(), g->block_budget);
    g->plan_d_t = make_plan(d_t.data(), (int)d_t.size(), g->block_budget);
    g->plan_all_t = make_plan(all_t.data(), (int)all_t.size(), g->block_budget);
    // level-ordered rounds launch one level at a time, and a latency-bound
    // gather needs the whole GPU's resident warps: every level gets the full
    // block budget (capped so the round's launches fit the partial-sum slots);
    // a small level is limited by its row groups in make_plan
    if (g->levels) {
        // what the cluster segments and the padding to whole clusters leave,
        // shared by the L + 1 launches (make_plan adds at most 1 per segment);
        // and no more than kLevelRoundBlocks / (L + 1): a level launch is short,
        // and more blocks than that measured slower (their scheduling and the
        // round's final reduction over all slots grow with them)
        const long long left = kMaxBlocks - cluster_blocks - (long long)kLevelCluster * (g->levels + 1);
        const long long round_blocks = std::min<long long>(left, kLevelRoundBlocks);
        // the round's lane-bin blocks go to the levels in proportion to their
        // work (R-MAT's hubs crowd the middle levels), at least 32 each, and no
        // level more than twice the block budget
        auto work_of = [](const std::vector<RangeSpec> &v) {
            double w = 0;
            for (const RangeSpec &r : v)
                if (r.hi > r.lo && r.lanes != kClusterLanes) w += (double)r.edges + 2.0 * (r.hi - r.lo);
            return w;
        };
        const std::vector<RangeSpec> u{unref};
        double wsum = work_of(u);
        for (int l = 0; l < g->levels; l++) wsum += work_of(lvl[l]);
        const long long spare = round_blocks - (long long)(g->levels + 1) * (kNumThr + 3 + 32);
        auto budget_of = [&](const std::vector<RangeSpec> &v) {
            const double share = wsum > 0 ? work_of(v) / wsum : 0.0;
            const long long b = 32 + (long long)(std::max<long long>(spare, 0) * share);
            return (int)std::min<long long>(b, 2LL * g->block_budget);
        };
        for (int l = 0; l < g->levels; l++)
            g->plan_lvl[l] = make_plan(lvl[l].data(), (int)lvl[l].size(), budget_of(lvl[l]));
        g->plan_unref = make_plan(u.data(), 1, budget_of(u));
    }
}

pr_status set_bins(pr_graph *g, const int32_t *thr, int32_t budget, cudaStream_t s) {
    const int32_t n = g->G.n, n_nd = g->G.n_nd, n_ref = g->G.n_ref;
    for (int k = 0; k < kNumThr; k++) {
        if (thr[k] < 0 || (k > 0 && thr[k] > thr[k - 1]))
            return fail(PR_EINVAL, "pull thresholds must be >= 0 and non-increasing");
    }
    if (budget < 1 || budget > kMaxBlocks / 2) return fail(PR_EINVAL, "block budget out of range");
    // the ranges: the referenced class (or its levels), then the dangling class
    int32_t lo[kMaxLevels + 1], hi[kMaxLevels + 1];
    int nr = 0;
    if (g->levels) {
        for (int l = 0; l < g->levels; l++) {
            lo[nr] = g->level_lo[l];
            hi[nr++] = g->level_lo[l + 1];
        }
    } else {
        lo[nr] = 0;
        hi[nr++] = n_ref;
    }
    lo[nr] = n_nd;
    hi[nr++] = n;
    Buf small, ebuf;
    const size_t rows_n = (size_t)nr * (kNumThr + 2);
    PR_TRY(small.alloc(sizeof(int32_t) * (8 + 2 * (kMaxLevels + 1) + nr * kNumThr + rows_n), s));
    PR_TRY(ebuf.alloc(sizeof(long long) * rows_n, s));
    int32_t *d_thr = small.as<int32_t>();           // [6]
    int32_t *d_lo = d_thr + 8;                      // [nr]
    int32_t *d_hi = d_lo + (kMaxLevels + 1);        // [nr]
    int32_t *d_bounds = d_hi + (kMaxLevels + 1);    // [nr * 6]
    int32_t *d_rows = d_bounds + nr * kNumThr;      // [nr * 8]
    long long *d_edges = ebuf.as<long long>();      // [nr * 8]
    PR_CK(cudaMemcpyAsync(d_thr, thr, sizeof(int32_t) * kNumThr, cudaMemcpyHostToDevice, s));
    PR_CK(cudaMemcpyAsync(d_lo, lo, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
    PR_CK(cudaMemcpyAsync(d_hi, hi, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
    k_bin_bounds<<<nr, 32, 0, s>>>(g->inr_off.as<int32_t>(), g->inu_off.as<int32_t>(), d_lo, d_hi, d_thr, kNumThr,
                                   d_bounds);
    std::vector<int32_t> b((size_t)nr * kNumThr);
    PR_CK(cudaMemcpyAsync(b.data(), d_bounds, sizeof(int32_t) * b.size(), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaStreamSynchronize(s));
    std::vector<int32_t> rows(rows_n);
    for (int k = 0; k < nr; k++) {
        rows[(size_t)k * (kNumThr + 2)] = lo[k];
        for (int t = 0; t < kNumThr; t++) rows[(size_t)k * (kNumThr + 2) + 1 + t] = b[(size_t)k * kNumThr + t];
        rows[(size_t)k * (kNumThr + 2) + kNumThr + 1] = hi[k];
    }
    std::vector<long long> edges(rows_n);
    PR_CK(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int32_t) * rows_n, cudaMemcpyHostToDevice, s));
    k_range_edges<<<(int)((rows_n + 31) / 32), 32, 0, s>>>(g->inr_off.as<int32_t>(), g->inu_off.as<int32_t>(),
                                                           d_rows, (int)rows_n, d_edges);
    PR_CK(cudaMemcpyAsync(edges.data(), d_edges, sizeof(long long) * rows_n, cudaMemcpyDeviceToHost, s));
    PR_CK(cudaStreamSynchronize(s));
    PR_CK(cudaGetLastError());
    // gather tiles over the short rows (in-degree <= thr[1] <= kTileDeg) of each range
    int32_t t_lo[kMaxLevels + 1], t_nt[kMaxLevels + 1] = {}, t_t0[kMaxLevels + 1] = {};
    const bool tiled = thr[1] <= kTileDeg;
    for (int k = 0; k < nr; k++) t_lo[k] = tiled ? b[(size_t)k * kNumThr + 1] : hi[k];
    Buf tiles;
    {
        int32_t *d_tlo = d_lo;  // [nr]: the range starts were consumed by k_bin_bounds (stream synchronized)
        PR_CK(cudaMemcpyAsync(d_tlo, t_lo, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
        int32_t *d_ends = d_rows;  // [2 nr] (the class rows were consumed above)
        k_tile_ends<<<1, 32, 0, s>>>(g->inr_off.as<int32_t>(), d_tlo, d_hi, nr, d_ends);
        std::vector<int32_t> ends(2 * (size_t)nr);
        PR_CK(cudaMemcpyAsync(ends.data(), d_ends, sizeof(int32_t) * ends.size(), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        int32_t total = 0;
        for (int k = 0; k < nr; k++) {
            if (t_lo[k] >= hi[k]) continue;
            const long long u_last = (long long)(ends[2 * k + 1] - ends[2 * k]) + (long long)kTileW * (hi[k] - 1 - t_lo[k]);
            t_nt[k] = (int32_t)(u_last / kTileU + 1);
            t_t0[k] = total;
            total += t_nt[k] + 1;
        }
        PR_TRY(tiles.alloc(sizeof(int32_t) * std::max(total, 1), s));
        for (int k = 0; k < nr; k++) {
            if (!t_nt[k]) continue;
            const int rows = hi[k] - t_lo[k];
            const int grid = std::max(1, std::min((rows + kThreads - 1) / kThreads, g->num_sms * 8));
            k_tile_marks<<<grid, kThreads, 0, s>>>(g->inr_off.as<int32_t>(), t_lo[k], hi[k],
                                                   tiles.as<int32_t>() + t_t0[k]);
        }
        PR_CK(cudaGetLastError());
    }
    // level-ordered rounds: per level, the rows above kClusterRowMin entries
    // (clusters) and above kLevelBlockRowMin (one block each), both within the
    // rows the tuning gives a block or a warp ([lo, bounds[1]))
    int32_t cl_hi[kMaxLevels + 1], lb_hi[kMaxLevels + 1];
    for (int k = 0; k < nr; k++) cl_hi[k] = lb_hi[k] = lo[k];
    if (g->levels) {
        const int32_t lthr[2] = {kClusterRowMin, kLevelBlockRowMin};
        std::vector<int32_t> b1(nr), out(2 * (size_t)nr);
        for (int k = 0; k < nr; k++) b1[k] = b[(size_t)k * kNumThr + 1];
        PR_CK(cudaMemcpyAsync(d_thr, lthr, sizeof(lthr), cudaMemcpyHostToDevice, s));
        PR_CK(cudaMemcpyAsync(d_lo, lo, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
        PR_CK(cudaMemcpyAsync(d_hi, b1.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, s));
        k_bin_bounds<<<nr, 32, 0, s>>>(g->inr_off.as<int32_t>(), g->inu_off.as<int32_t>(), d_lo, d_hi, d_thr, 2,
                                       d_bounds);
        PR_CK(cudaMemcpyAsync(out.data(), d_bounds, sizeof(int32_t) * out.size(), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        PR_CK(cudaGetLastError());
        for (int k = 0; k < nr; k++) {
            cl_hi[k] = out[2 * (size_t)k];
            lb_hi[k] = out[2 * (size_t)k + 1];
        }
    }
    // plans are built into a scratch copy first: the graph keeps its bins on failure
    pr_graph *T = new (std::nothrow) pr_graph();
    if (!T) return fail(PR_ENOMEM, "host allocation failed");
    T->G = g->G;
    T->levels = g->levels;
    for (int l = 0; l <= kMaxLevels; l++) T->level_lo[l] = g->level_lo[l];
    for (int k = 0; k < nr; k++) {
        T->cl_hi[k] = cl_hi[k];
        T->lb_hi[k] = lb_hi[k];
    }
    T->nranges = nr;
    for (int k = 0; k < nr; k++) {
        T->range_lo[k] = lo[k];
        T->range_hi[k] = hi[k];
    }
    for (size_t k = 0; k < b.size(); k++) T->bounds[k] = b[k];
    for (size_t k = 0; k < rows_n; k++) T->range_edges[k] = edges[k];
    T->block_budget = budget;
    for (int k = 0; k < nr; k++) {
        T->tile_lo[k] = t_lo[k];
        T->tile_nt[k] = t_nt[k];
        T->tile_t0[k] = t_t0[k];
    }
    build_plans(T);
    bool ok = T->plan_all.nblocks <= kMaxBlocks && T->plan_nd.nblocks <= kMaxBlocks &&
              T->plan_all_t.nblocks <= kMaxBlocks && T->plan_nd_t.nblocks <= kMaxBlocks;
    // one level-ordered round's launches share the slots; each grid is padded
    // to whole clusters
    auto padded = [](int nb) { return (nb + kLevelCluster - 1) / kLevelCluster * kLevelCluster; };
    int lvl_blocks = T->levels ? padded(T->plan_unref.nblocks) : 0;
    for (int l = 0; l < T->levels; l++) {
        lvl_blocks += padded(T->plan_lvl[l].nblocks);
        // a cluster segment must start and end on cluster boundaries (it is the first segment)
        const Plan &PL = T->plan_lvl[l];
        for (int q = 0; q < PL.nseg; q++)
            if (PL.seg[q].lanes == kClusterLanes &&
                (PL.seg[q].blk0 % kLevelCluster != 0 || PL.seg[q].nblk % kLevelCluster != 0))
                ok = false;
    }
    ok = ok && lvl_blocks <= kMaxBlocks;
    if (!ok) {
        delete T;
        return fail(PR_EINVAL, "pull plan exceeds the partial-sum slots");
    }
    for (int k = 0; k < kNumThr; k++) g->thr[k] = thr[k];
    g->nranges = nr;
    for (int k = 0; k <= kMaxLevels; k++) {
        g->range_lo[k] = T->range_lo[k];
        g->range_hi[k] = T->range_hi[k];
    }
    for (size_t k = 0; k < sizeof(g->bounds) / sizeof(g->bounds[0]); k++) g->bounds[k] = T->bounds[k];
    for (size_t k = 0; k < sizeof(g->range_edges) / sizeof(g->range_edges[0]); k++)
        g->range_edges[k] = T->range_edges[k];
    g->block_budget = budget;
    g->plan_nd = T->plan_nd;
    g->plan_d = T->plan_d;
    g->plan_all = T->plan_all;
    g->plan_nd_t = T->plan_nd_t;
    g->plan_d_t = T->plan_d_t;
    g->plan_all_t = T->plan_all_t;
    for (int k = 0; k <= kMaxLevels; k++) {
        g->tile_lo[k] = T->tile_lo[k];
        g->tile_nt[k] = T->tile_nt[k];
        g->tile_t0[k] = T->tile_t0[k];
    }
    g->tile_row.swap(tiles);  // the old table is released when `tiles` leaves scope (stream synchronized)
    g->G.tile_row = g->tile_row.as<int32_t>();
    for (int l = 0; l < kMaxLevels; l++) g->plan_lvl[l] = T->plan_lvl[l];
    for (int k = 0; k <= kMaxLevels; k++) {
        g->cl_hi[k] = T->cl_hi[k];
        g->lb_hi[k] = T->lb_hi[k];
    }
    g->plan_unref = T->plan_unref;
    g->plan_gen++;
    delete T;
    return PR_OK;
}

}  // namespace pr

using namespace pr;

// ------------------------------------------------------------ ABI
extern "C" const char *pr_last_error(void) { return t_err.c_str(); }

extern "C" const char *pr_version(void) { return "pr-gb300 0.1 (sm_103a)"; }

extern "C" pr_status pr_set_allocator(pr_alloc_fn alloc, pr_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(PR_EINVAL, "pr_set_allocator: alloc and free must both be set or both NULL");
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = ctx;
    return PR_OK;
}

extern "C" pr_status pr_graph_get_info(const pr_graph *g, pr_graph_info *info) {
    if (!g || !info) return fail(PR_EINVAL, "pr_graph_get_info: NULL argument");
    *info = g->info;
    return PR_OK;
}

extern "C" void pr_destroy(pr_graph *g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    destroy_workspace(g);
    delete g;
}

// The first index in [0, count) where bad(k) holds, or count.  Chunks are
// scanned by up to 16 host threads; inside a chunk, blocks of 4096 indices are
// OR-reduced without an early exit (a loop the compiler vectorises), and only
// a block that holds a bad index is searched for the first one.  The
// element-by-element loop with an early exit took about 3 ms on a 47M-entry
// edge array with 16 threads; this one runs at memory speed.
template <typename F> static int64_t first_bad(int64_t count, F bad) {
    const int64_t kChunk = 1 << 20, kBlock = 4096;
    const int nt = (int)std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()), 16,
                                           (count + kChunk - 1) / kChunk});
    auto scan = [&](int64_t lo, int64_t hi) {
        for (int64_t b = lo; b < hi; b += kBlock) {
            const int64_t e = std::min(hi, b + kBlock);
            unsigned any = 0;
            for (int64_t k = b; k < e; k++) any |= (unsigned)bad(k);
            if (any)
                for (int64_t k = b; k < e; k++)
                    if (bad(k)) return k;
        }
        return count;
    };
    if (nt <= 1) return scan(0, count);
    std::vector<int64_t> found(nt, count);
    std::vector<std::thread> th;
    const int64_t per = (count + nt - 1) / nt;
    for (int t = 0; t < nt; t++) {
        auto part = [&, t]() { found[t] = scan(std::min(count, t * per), std::min(count, (t + 1) * per)); };
        try {
            th.emplace_back(part);
        } catch (...) {  // no thread to be had: scan this part here
            part();
        }
    }
    for (auto &x : th) x.join();
    return *std::min_element(found.begin(), found.end());
}

// The checks of one host CSR (or CSC) pair: "" when they hold, else the message.
static std::string check_host_lists(int32_t n, int64_t m, const int32_t *off, const int32_t *dst) {
    if (off[0] != 0) return "out_off[0] must be 0";
    const int64_t i = first_bad(n, [&](int64_t k) { return off[k + 1] < off[k]; });
    if (i < n) return "out_off is not non-decreasing at row " + std::to_string(i);
    if ((int64_t)off[n] != m) return "out_off[n] != m";
    // one unsigned compare covers both ends: a negative id wraps above n
    const int64_t e = first_bad(m, [&](int64_t k) { return (uint32_t)dst[k] >= (uint32_t)n; });
    if (e < m) return "out_dst[" + std::to_string(e) + "] out of range";
    return "";
}

static bool allocator_hooked() { return g_alloc != nullptr; }

// Temporaries of graph creation without an allocator hook: one stream-ordered
// pool per device, owned by the library.  Freed temporaries are reused without
// the device-wide synchronisation that cudaFree takes, and up to
// kCreationCache bytes of them stay mapped for the next creation (mapping new
// device memory is a large part of a creation's cost); above that the pool
// returns memory at the stream synchronisations.
constexpr uint64_t kCreationCache = 2ull << 30;
static cudaMemPool_t creation_pool(int dev) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = kCreationCache;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

namespace {
pr_status create_impl(int32_t n, int64_t m, const int32_t *out_off, const int32_t *out_dst,
                      const int32_t *in_off, const int32_t *in_src, int mem_is_device,
                      cudaStream_t s, int32_t levels, pr_graph *g) {
    int dev = 0;
    PR_CK(cudaGetDevice(&dev));
    int sms = 0;
    PR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g->device = dev;
    g->num_sms = sms;
    g->stream = s;
    Scratch sc;  // the hook, when one is installed, serves the temporaries too
    if (!allocator_hooked()) {
        sc.pool = creation_pool(dev);
        if (!sc.pool) return fail(PR_ECUDA, "cannot create the memory pool of graph creation");
    }
    cudaEvent_t e0, e1;
    PR_CK(cudaEventCreate(&e0));
    PR_CK(cudaEventCreate(&e1));
    PR_CK(cudaEventRecord(e0, s));

    // caller arrays on the device
    Buf c_off, c_dst, c_ioff, c_isrc;
    const int32_t *d_off = out_off, *d_dst = out_dst, *d_ioff = in_off, *d_isrc = in_src;
    if (!mem_is_device) {
        PR_TRY(sc.get(c_off, sizeof(int32_t) * (n + 1), s));
        PR_TRY(sc.get(c_dst, sizeof(int32_t) * m, s));
        PR_CK(cudaMemcpyAsync(c_off.p, out_off, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
        if (m) PR_CK(cudaMemcpyAsync(c_dst.p, out_dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
        d_off = c_off.as<int32_t>();
        d_dst = c_dst.as<int32_t>();
        if (in_off) {
            PR_TRY(sc.get(c_ioff, sizeof(int32_t) * (n + 1), s));
            PR_TRY(sc.get(c_isrc, sizeof(int32_t) * m, s));
            PR_CK(cudaMemcpyAsync(c_ioff.p, in_off, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
            if (m) PR_CK(cudaMemcpyAsync(c_isrc.p, in_src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
            d_ioff = c_ioff.as<int32_t>();
            d_isrc = c_isrc.as<int32_t>();
        }
    }
    // small device scratch: [0..1] validation, [2] dup count, [3] m_d, class counts, facts
    Buf scratch;
    PR_TRY(sc.get(scratch, 256, s));
    PR_CK(cudaMemsetAsync(scratch.p, 0, 256, s));
    unsigned long long *bad = scratch.as<unsigned long long>();         // [0],[1]
    unsigned long long *dups = bad + 2;                                 // [2]
    unsigned long long *m_d = bad + 3;                                  // [3]
    unsigned int *class_cnt = reinterpret_cast<unsigned int *>(bad + 4);// 3 entries
    unsigned int *fact_cnt = class_cnt + 4;                             // 5 entries
    int *maxes = reinterpret_cast<int *>(fact_cnt + 6);                 // 2 entries
    int *sort_err = reinterpret_cast<int *>(bad + 12);                  // radix_sort's flag

    // waits for the stream; PR_ECUDA if a radix sort so far gave up (its output is incomplete)
    auto sort_check = [&]() -> pr_status {
        int h = 0;
        PR_CK(cudaMemcpyAsync(&h, sort_err, sizeof(h), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        return h ? fail(PR_ECUDA, "graph creation: a radix sort pass gave up waiting for an earlier tile") : PR_OK;
    };
    const int gm = grid_for(std::max<int64_t>(m, n + 1), sms), gn = grid_for(n + 1, sms);
    {  // the caller's lists, on the device (host arrays: the copies), before any kernel indexes by them
        k_validate<<<gm, kThreads, 0, s>>>(n, m, d_off, d_dst, bad);
        if (d_ioff) k_validate<<<gm, kThreads, 0, s>>>(n, m, d_ioff, d_isrc, bad);
        unsigned long long hb[2];
        PR_CK(cudaMemcpyAsync(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
        PR_CK(cudaStreamSynchronize(s));
        if (hb[0]) return fail(PR_EINVAL, "offsets are not a valid CSR/CSC offset array");
        if (hb[1]) return fail(PR_EINVAL, "an edge endpoint is outside [0, n)");
    }
    const int B = bits_for(n);
    // degrees and classes
    Buf indeg;
    PR_TRY(sc.get(indeg, sizeof(int32_t) * n, s));
    PR_CK(cudaMemsetAsync(indeg.p, 0, sizeof(int32_t) * n, s));
    if (m) k_indeg<<<gm, kThreads, 0, s>>>(m, d_dst, indeg.as<int32_t>());
    Buf vk, vk2, vv2;
    PR_TRY(sc.get(vk, sizeof(uint64_t) * n, s));
    PR_TRY(sc.get(vk2, sizeof(uint64_t) * n, s));
    Buf level;
    if (levels > 0) {  // levels of the referenced class (level-ordered rounds)
        PR_TRY(sc.get(level, sizeof(int32_t) * n, s));
        unsigned int *lvl_cnt = class_cnt + 3;
        k_level_keys<<<gn, kThreads, 0, s>>>(n, d_off, indeg.as<int32_t>(), B, vk.as<uint64_t>(), lvl_cnt);
        PR_TRY(radix_sort(vk.as<uint64_t>(), nullptr, n, 0, 31 + B, vk2.as<uint64_t>(), nullptr, nullptr, sort_err, sc,
                          s));
        unsigned int h_ref = 0;
        PR_CK(cudaMemcpyAsync(&h_ref, lvl_cnt, sizeof(h_ref), cudaMemcpyDeviceToHost, s));
        PR_TRY(sort_check());
        if (h_ref)
            k_assign_levels<<<grid_for(h_ref, sms), kThreads, 0, s>>>(vk.as<uint64_t>(), (int32_t)h_ref, levels, B,
                                                                    level.as<int32_t>());
    }
    // the renumbering: a stable sort of the vertex keys, carrying the ids
    PR_TRY(g->perm.alloc(sizeof(int32_t) * n, s));
    PR_TRY(sc.get(vv2, sizeof(int32_t) * n, s));
    {
        const int IB = bits_for(m + 1), LB = levels > 0 ? 4 : 0;
        k_vertex_keys<<<gn, kThreads, 0, s>>>(n, d_off, indeg.as<int32_t>(),
                                              levels > 0 ? level.as<int32_t>() : nullptr, IB, LB, vk.as<uint64_t>(),
                                              g->perm.as<int32_t>(), class_cnt);
        PR_TRY(radix_sort(vk.as<uint64_t>(), g->perm.as<int32_t>(), n, 0, 2 + LB + IB, vk2.as<uint64_t>(),
                          vv2.as<int32_t>(), nullptr, sort_err, sc, s));
    }
    vk.release();
    vk2.release();
    vv2.release();
    level.release();
    unsigned int hc[3];
    PR_CK(cudaMemcpyAsync(hc, class_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
    PR_TRY(sort_check());  // perm is complete before anything indexes by it
    PR_TRY(g->inv.alloc(sizeof(int32_t) * n, s));
    k_invert<<<gn, kThreads, 0, s>>>(n, g->perm.as<int32_t>(), g->inv.as<int32_t>());
    const int32_t n_ref = (int32_t)hc[0], n_nd = (int32_t)(hc[0] + hc[1]);
    g->levels = levels;
    for (int l = 0; l <= levels; l++)  // level l holds the ranks [ceil(l n_ref / L), ceil((l+1) n_ref / L))
        g->level_lo[l] = (int32_t)(((int64_t)l * n_ref + levels - 1) / levels);

    // Edges in internal ids.  The keys (k_edge_keys) pack src << (B+1) |
    // flag << B | dst; the caller's rows are written to their internal rows,
    // so the keys arrive grouped by src.  A stable sort on the low B+1 bits
    // then orders them by (flag, dst, src): the in-lists, referenced sources
    // first.  A second stable sort, on the src bits, orders them by (src, dst)
    // (the flag is a function of src): the out-lists.  Each sort covers B+1 or
    // B bits, where one sort of whole keys covers 2B.
    const uint64_t id_mask = (1ULL << B) - 1;
    PR_TRY(g->out_off.alloc(sizeof(int32_t) * (n + 1), s));
    PR_TRY(g->out_dst.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    {
        Buf deg;
        PR_TRY(sc.get(deg, sizeof(int32_t) * (n + 1), s));
        k_new_degrees<<<gn, kThreads, 0, s>>>(n, d_off, g->perm.as<int32_t>(), deg.as<int32_t>());
        PR_TRY(scan_i32(deg.as<int32_t>(), g->out_off.as<int32_t>(), n + 1, nullptr, sc, s));
    }
    Buf ek, ek2, dc;
    PR_TRY(sc.get(ek, sizeof(uint64_t) * std::max<int64_t>(m, 1), s));
    PR_TRY(sc.get(ek2, sizeof(uint64_t) * std::max<int64_t>(m, 1), s));
    PR_TRY(sc.get(dc, sizeof(uint32_t) * 2 * kRadixMaxPasses * kRadixDigits, s));  // digit counts of the two sorts
    PR_CK(cudaMemsetAsync(dc.p, 0, sizeof(uint32_t) * 2 * kRadixMaxPasses * kRadixDigits, s));
    uint32_t *counts_in = dc.as<uint32_t>(), *counts_out = counts_in + kRadixMaxPasses * kRadixDigits;
    uint64_t *keys = ek.as<uint64_t>(), *alt = ek2.as<uint64_t>();
    if (m)
        k_edge_keys<<<gm, kThreads, 0, s>>>(n, m, d_off, d_dst, g->inv.as<int32_t>(), B, n_ref, 1,
                                            g->out_off.as<int32_t>(), keys, 0, B + 1, counts_in);
    // in-lists: sorted by (flag, dst, src), the first m_ref keys are the
    // edges from referenced sources (internal ids below n_ref: the first
    // out_off[n_ref] out-list entries)
    bool swapped = false;
    PR_TRY(radix_sort(keys, nullptr, m, 0, B + 1, alt, nullptr, counts_in, sort_err, sc, s, &swapped));
    if (swapped) std::swap(keys, alt);
    int32_t h_mref = 0;
    PR_CK(cudaMemcpyAsync(&h_mref, g->out_off.as<int32_t>() + n_ref, sizeof(h_mref), cudaMemcpyDeviceToHost, s));
    PR_TRY(sort_check());  // the keys are complete before their fields index anything
    const int64_t m_ref = h_mref, m_unref = m - m_ref;
    PR_TRY(g->inr_off.alloc(sizeof(int32_t) * (n + 1), s));
    PR_TRY(g->inu_off.alloc(sizeof(int32_t) * (n + 1), s));
    PR_TRY(g->inr_src.alloc(sizeof(int32_t) * std::max<int64_t>(m_ref, 1), s));
    PR_TRY(g->inu_src.alloc(sizeof(int32_t) * std::max<int64_t>(m_unref, 1), s));
    {
        Buf cnt;
        PR_TRY(sc.get(cnt, sizeof(int32_t) * 2 * (size_t)(n + 1), s));
        PR_CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * 2 * (size_t)(n + 1), s));
        int32_t *cnt_ref = cnt.as<int32_t>(), *cnt_unref = cnt_ref + (n + 1);
        if (m)
            k_in_lists<<<gm, kThreads, 0, s>>>(m, keys, B, n, m_ref, g->inr_src.as<int32_t>(),
                                               g->inu_src.as<int32_t>(), cnt_ref, dups, counts_out);
        PR_TRY(scan_i32(cnt_ref, g->inr_off.as<int32_t>(), n + 1, nullptr, sc, s));
        PR_TRY(scan_i32(cnt_unref, g->inu_off.as<int32_t>(), n + 1, nullptr, sc, s));
    }
    // out-lists (offsets from the scan above)
    PR_TRY(radix_sort(keys, nullptr, m, B + 1, 2 * B + 1, alt, nullptr, counts_out, sort_err, sc, s, &swapped));
    if (swapped) std::swap(keys, alt);
    if (m) k_field<<<gm, kThreads, 0, s>>>(m, keys, 0, id_mask, g->out_dst.as<int32_t>());
    // optional caller in-lists: the same edge set?  Their keys, sorted whole,
    // must equal the out-list keys, which are now in ascending order.
    if (d_ioff) {
        Buf ck;
        PR_TRY(sc.get(ck, sizeof(uint64_t) * std::max<int64_t>(m, 1), s));
        uint64_t *ckeys = ck.as<uint64_t>();
        if (m)
            k_edge_keys<<<gm, kThreads, 0, s>>>(n, m, d_ioff, d_isrc, g->inv.as<int32_t>(), B, n_ref, 0, nullptr,
                                                ckeys, 0, 0, nullptr);
        PR_TRY(radix_sort(ckeys, nullptr, m, 0, 2 * B + 1, alt, nullptr, nullptr, sort_err, sc, s, &swapped));
        if (swapped) ckeys = alt;  // alt is free: the out-list keys are in keys
        if (m) k_count_diff<<<gm, kThreads, 0, s>>>(m, keys, ckeys, bad + 1);
        unsigned long long hb = 0;
        PR_CK(cudaMemcpyAsync(&hb, bad + 1, sizeof(hb), cudaMemcpyDeviceToHost, s));
        PR_TRY(sort_check());
        if (hb) return fail(PR_EINVAL, "in_off/in_src do not describe the same edges as out_off/out_dst");
    }
    ek.release();
    ek2.release();
    // the degree facts
    k_degree_facts<<<gn, kThreads, 0, s>>>(n, n_nd, g->perm.as<int32_t>(), indeg.as<int32_t>(),
                                           g->out_off.as<int32_t>(), fact_cnt, maxes, m_d);
    // per-vertex arrays
    PR_TRY(g->ndeg.alloc(sizeof(int32_t) * std::max(n_nd, 1), s));
    PR_TRY(g->inv_deg64.alloc(sizeof(double) * std::max(n_nd, 1), s));
    PR_TRY(g->inv_deg32.alloc(sizeof(float) * std::max(n_nd, 1), s));
    PR_TRY(g->inv_degdf.alloc(sizeof(float2) * std::max(n_nd, 1), s));
    if (n_nd)
        k_vertex_arrays<<<grid_for(n_nd, sms), kThreads, 0, s>>>(
            n_nd, g->out_off.as<int32_t>(), g->out_dst.as<int32_t>(), g->ndeg.as<int32_t>(),
            g->inv_deg64.as<double>(), g->inv_deg32.as<float>(), g->inv_degdf.as<float2>());
    if (levels > 0) {
        Buf d_lo;
        PR_TRY(d_lo.alloc(sizeof(int32_t) * (kMaxLevels + 1), s));
        PR_CK(cudaMemcpyAsync(d_lo.p, g->level_lo, sizeof(int32_t) * (levels + 1), cudaMemcpyHostToDevice, s));
        PR_TRY(g->gs_back.alloc(sizeof(int32_t) * std::max(n_nd, 1), s));
        if (n_nd)
            k_level_back<<<grid_for(n_nd, sms), kThreads, 0, s>>>(n_ref, n_nd, g->out_off.as<int32_t>(),
                                                                  g->out_dst.as<int32_t>(), g->ndeg.as<int32_t>(),
                                                                  d_lo.as<int32_t>(), levels,
                                                                  g->gs_back.as<int32_t>());
        PR_CK(cudaStreamSynchronize(s));  // d_lo is freed at the end of this scope
    }
    int32_t hnd[2] = {0, 0};
    PR_CK(cudaMemcpyAsync(&hnd[0], g->inr_off.as<int32_t>() + n_nd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaMemcpyAsync(&hnd[1], g->inu_off.as<int32_t>() + n_nd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    unsigned int hu = 0;
    int hm[2];
    unsigned long long hmd = 0;
    PR_CK(cudaMemcpyAsync(&hu, fact_cnt, sizeof(hu), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaMemcpyAsync(hm, maxes, sizeof(hm), cudaMemcpyDeviceToHost, s));
    PR_CK(cudaMemcpyAsync(&hmd, m_d, sizeof(hmd), cudaMemcpyDeviceToHost, s));
    unsigned long long hdup = 0;
    PR_CK(cudaMemcpyAsync(&hdup, dups, sizeof(hdup), cudaMemcpyDeviceToHost, s));
    PR_TRY(sort_check());
    if (hdup) return fail(PR_EINVAL, std::to_string(hdup) + " repeated edge(s): the adjacency is 0/1");

    DevGraph &G = g->G;
    G.n = n;
    G.n_nd = n_nd;
    G.n_ref = n_ref;
    G.m = m;
    G.m_ref = m_ref;
    G.m_unref = m_unref;
    G.out_off = g->out_off.as<int32_t>();
    G.out_dst = g->out_dst.as<int32_t>();
    G.ndeg = g->ndeg.as<int32_t>();
    G.inv_deg64 = g->inv_deg64.as<double>();
    G.inv_deg32 = g->inv_deg32.as<float>();
    G.inv_degdf = g->inv_degdf.as<float2>();
    G.inr_off = g->inr_off.as<int32_t>();
    G.inr_src = g->inr_src.as<int32_t>();
    G.inu_off = g->inu_off.as<int32_t>();
    G.inu_src = g->inu_src.as<int32_t>();
    G.perm = g->perm.as<int32_t>();
    G.inv = g->inv.as<int32_t>();
    G.gs_back = levels > 0 ? g->gs_back.as<int32_t>() : nullptr;
    g->scan_nd_ref = hnd[0];
    g->scan_nd_unref = hnd[1];
    g->pull_ratio = 0.04;
    PR_TRY(set_bins(g, kDefaultThr, sms * 16, s));
    PR_CK(cudaEventRecord(e1, s));
    PR_CK(cudaEventSynchronize(e1));
    float ms = 0;
    PR_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);

    pr_graph_info &I = g->info;
    I.n = n;
    I.n_nd = n_nd;
    I.n_ref = n_ref;
    I.n_d = n - n_nd;
    I.n_u = (int32_t)hu;
    I.m = m;
    I.m_d = (int64_t)hmd;
    I.max_outdeg = hm[0];
    I.max_indeg = hm[1];
    I.ms_preprocess = ms;
    I.levels = levels;
    I.device_bytes = g->out_off.bytes + g->out_dst.bytes + g->ndeg.bytes + g->inv_deg64.bytes +
                     g->inv_deg32.bytes + g->inv_degdf.bytes + g->inr_off.bytes + g->inr_src.bytes + g->inu_off.bytes +
                     g->inu_src.bytes + g->perm.bytes + g->inv.bytes + g->gs_back.bytes;
    return PR_OK;
}
}  // namespace

extern "C" pr_status pr_graph_create_ex(int32_t n, int64_t m, const int32_t *out_off,
                                     const int32_t *out_dst, const int32_t *in_off,
                                     const int32_t *in_src, int mem_is_device, void *cuda_stream,
                                     const pr_graph_opts *opts, pr_graph **g) {
    if (!g) return fail(PR_EINVAL, "pr_graph_create: g is NULL");
    *g = nullptr;
    if (n < 1) return fail(PR_EINVAL, "n must be >= 1");
    if (m < 0 || m >= ((int64_t)1 << 31)) return fail(PR_EINVAL, "m must be in [0, 2^31)");
    if (!out_off || (m > 0 && !out_dst)) return fail(PR_EINVAL, "out_off/out_dst missing");
    if (!in_off && in_src) return fail(PR_EINVAL, "in_src given without in_off");
    if (in_off && m > 0 && !in_src) return fail(PR_EINVAL, "in_off given without in_src");
    const int32_t levels = opts ? opts->levels : 0;
    if (levels < 0 || levels > kMaxLevels) return fail(PR_EINVAL, "levels must be in [0, 16]");
    if (!mem_is_device) {
        // the two ends first, on the host: the copies read m entries, so off[n] = m must hold before they start
        if (out_off[0] != 0 || (int64_t)out_off[n] != m) return fail(PR_EINVAL, "out_off must run from 0 to m");
        if (in_off && (in_off[0] != 0 || (int64_t)in_off[n] != m))
            return fail(PR_EINVAL, "in_off must run from 0 to m");
    }
    pr_graph *G = new (std::nothrow) pr_graph();
    if (!G) return fail(PR_ENOMEM, "host allocation failed");
    static std::atomic<uint64_t> serial{0};
    G->uid = ++serial;
#ifdef PR_DEBUG
    dbg_reset_sort(dbg_injected());  // the radix sort's test hook (DBG_SORT_WAIT)
#endif
    pr_status st = create_impl(n, m, out_off, out_dst, in_off, in_src, mem_is_device,
                               (cudaStream_t)cuda_stream, levels, G);
    if (!allocator_hooked()) {  // keep at most kCreationCache bytes of freed temporaries mapped
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            if (cudaMemPool_t pool = creation_pool(dev)) cudaMemPoolTrimTo(pool, kCreationCache);
        cudaGetLastError();
    }
    if (st != PR_OK && st != PR_EINVAL && !mem_is_device) {
        // the device failed before it could check the lists (no device, no memory): check
        // host arrays here, so that invalid arguments are reported as such on any machine
        std::string e = check_host_lists(n, m, out_off, out_dst);
        if (e.empty() && in_off) e = check_host_lists(n, m, in_off, in_src);
        if (!e.empty()) st = fail(PR_EINVAL, e);
    }
    if (st != PR_OK) {
        std::string msg = pr_last_error();
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        cudaGetLastError();
        delete G;
        set_error(msg);
        return st;
    }
    *g = G;
    return PR_OK;
}

extern "C" pr_status pr_graph_create(int32_t n, int64_t m, const int32_t *out_off, const int32_t *out_dst,
                                     const int32_t *in_off, const int32_t *in_src, int mem_is_device,
                                     void *cuda_stream, pr_graph **g) {
    return pr_graph_create_ex(n, m, out_off, out_dst, in_off, in_src, mem_is_device, cuda_stream, nullptr, g);
}
