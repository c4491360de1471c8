// pr_sort.cu -- the library's own scans and sorts for graph creation (no
// library sort or scan on the path):
//   scan_i32       exclusive prefix sum of int32 counts (three passes: tile
//                  sums, one block scans them, tiles add their base);
//   radix_sort     stable LSD radix sort of 64-bit keys with optional int32
//                  values, 8-bit digits: per tile a digit histogram, one scan
//                  of all histograms (digit-major), then a stable scatter in
//                  which every key's rank among equal digits of its tile comes
//                  from warp matches and per-warp counts;
//   sort_rows      each row of a CSR-like int32 array sorted ascending: rows
//                  of up to kSmallRow entries by one thread (insertion sort),
//                  longer rows by one block each (the same stable LSD scheme,
//                  in place through a scratch copy of the row).
// All three are deterministic: results do not depend on scheduling.
#include <algorithm>

#include "pr_internal.cuh"
#include "pr_sort.cuh"

namespace pr {

namespace {

constexpr int kScanTile = 2048;   // int32 per scan tile (256 threads x 8)
constexpr int kSortTile = 2048;   // keys per radix tile (8 rounds of 256)
constexpr int kDigits = 256;
constexpr int kWarps = kThreads / 32;

// exclusive block scan of one int per thread (block of kThreads); returns the
// block total in *total (all threads)
__device__ __forceinline__ int block_exscan(int v, int *sh, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kWarps ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kWarps) sh[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int before = wid ? sh[wid - 1] : 0;
    *total = sh[kWarps - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_tile_sums(const int32_t *in, int64_t n, int32_t *sums) {
    __shared__ int sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int v = 0;
    for (int k = 0; k < kScanTile / kThreads; k++) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) v += in[i];
    }
    int total;
    block_exscan(v, sh, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block: exclusive scan of the tile sums in place (any count, chunk by chunk)
__global__ void __launch_bounds__(kThreads) k_scan_sums(int32_t *sums, int64_t nt, int32_t *grand) {
    __shared__ int sh[32];
    int carry = 0;
    for (int64_t c = 0; c < nt; c += kThreads) {
        const int64_t i = c + threadIdx.x;
        const int v = i < nt ? sums[i] : 0;
        int total;
        const int ex = block_exscan(v, sh, &total);
        if (i < nt) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && grand) *grand = carry;
}

// each thread scans a contiguous run of 8, the block scans the runs' totals
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const int32_t *in, int64_t n, const int32_t *sums,
                                                        int32_t *out) {
    __shared__ int sh[32];
    constexpr int R = kScanTile / kThreads;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * R;
    int v[R], t = 0;
#pragma unroll
    for (int k = 0; k < R; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    int total;
    int run = block_exscan(t, sh, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < R; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------ radix sort
__device__ __forceinline__ int digit_of(uint64_t k, int shift, int nbits) {
    return (int)((k >> shift) & ((1ull << nbits) - 1ull));
}

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint64_t *keys, int64_t n, int shift, int nbits,
                                                        int64_t ntiles, int32_t *hist) {
    __shared__ int h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kThreads) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&h[digit_of(keys[i], shift, nbits)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << nbits); d += kThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// The stable scatter of one tile: the tile's keys in rounds of kThreads (key
// r * kThreads + t is thread t's in round r); a key's destination is the
// digit's global base for this tile + the keys of that digit in earlier
// rounds + those of earlier warps in this round + those of earlier lanes of
// its warp (a warp match).
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint64_t *keys, const int32_t *vals, int64_t n,
                                                           int shift, int nbits, int64_t ntiles,
                                                           const int32_t *offs, uint64_t *keys_out,
                                                           int32_t *vals_out) {
    __shared__ int run[kDigits];
    __shared__ int wcnt[kWarps][kDigits];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kDigits; d += kThreads)
        run[d] = d < (1 << nbits) ? offs[(int64_t)d * ntiles + blockIdx.x] : 0;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortTile / kThreads; r++) {
        for (int k = threadIdx.x; k < kWarps * kDigits; k += kThreads) (&wcnt[0][0])[k] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)r * kThreads + threadIdx.x;
        const bool ok = i < n;
        const uint64_t key = ok ? keys[i] : 0;
        const int d = ok ? digit_of(key, shift, nbits) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const int wrank = __popc(same & lt);
        if (ok && wrank == 0) wcnt[wid][d] = __popc(same);
        __syncthreads();
        int before = 0;
        if (ok)
            for (int w = 0; w < wid; w++) before += wcnt[w][d];
        const int pos = ok ? run[d] + before + wrank : 0;
        __syncthreads();  // every thread has read run[] for this round
        for (int dd = threadIdx.x; dd < kDigits; dd += kThreads) {
            int t = 0;
#pragma unroll
            for (int w = 0; w < kWarps; w++) t += wcnt[w][dd];
            run[dd] += t;
        }
        if (ok) {
            keys_out[pos] = key;
            if (vals) vals_out[pos] = vals[i];
        }
        __syncthreads();  // wcnt[] and run[] are read above before the next round rewrites them
    }
}

// ------------------------------------------------------------ row sorts
constexpr int kSmallRow = 32;

// rows of at most kSmallRow entries: one thread each, insertion sort in place
__global__ void k_rows_small(int32_t *data, const int32_t *off, int32_t nrows) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrows; j += gridDim.x * blockDim.x) {
        const int a = off[j], b = off[j + 1];
        if (b - a < 2 || b - a > kSmallRow) continue;
        for (int e = a + 1; e < b; e++) {
            const int32_t v = data[e];
            int k = e - 1;
            while (k >= a && data[k] > v) {
                data[k + 1] = data[k];
                k--;
            }
            data[k + 1] = v;
        }
    }
}

// rows above kSmallRow entries: flag (1) or not (0), for the compaction
__global__ void k_rows_big_flag(const int32_t *off, int32_t nrows, int32_t *flag) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrows; j += gridDim.x * blockDim.x)
        flag[j] = off[j + 1] - off[j] > kSmallRow;
}

__global__ void k_rows_big_list(const int32_t *flag, const int32_t *pos, int32_t nrows, int32_t *list) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrows; j += gridDim.x * blockDim.x)
        if (flag[j]) list[pos[j]] = j;
}

// One block per long row: stable LSD radix sort of its entries (values in
// [0, 2^bits)) by 8-bit digits, ping-ponging between the row and its place in
// a scratch array of the same layout; an odd pass count ends with a copy back.
__global__ void __launch_bounds__(kThreads) k_rows_big(int32_t *data, int32_t *scratch, const int32_t *off,
                                                      const int32_t *list, const int32_t *count, int bits) {
    __shared__ int hist[kDigits];
    __shared__ int run[kDigits];
    __shared__ int wcnt[kWarps][kDigits];
    __shared__ int sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nbig = *count;
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int j = list[q];
        const int a = off[j], len = off[j + 1] - a;
        int32_t *src = data + a, *dst = scratch + a;
        int passes = 0;
        for (int shift = 0; shift < bits; shift += 8, passes++) {
            const int nb = bits - shift < 8 ? bits - shift : 8;
            const int mask = (1 << nb) - 1;
            for (int d = threadIdx.x; d < kDigits; d += kThreads) hist[d] = 0;
            __syncthreads();
            for (int e = threadIdx.x; e < len; e += kThreads) atomicAdd(&hist[(src[e] >> shift) & mask], 1);
            __syncthreads();
            int total;
            const int ex = block_exscan(hist[threadIdx.x], sh, &total);  // kThreads == kDigits
            run[threadIdx.x] = ex;
            for (int r = 0; r * kThreads < len; r++) {
                for (int k = threadIdx.x; k < kWarps * kDigits; k += kThreads) (&wcnt[0][0])[k] = 0;
                __syncthreads();
                const int e = r * kThreads + threadIdx.x;
                const bool ok = e < len;
                const int32_t v = ok ? src[e] : 0;
                const int d = ok ? (v >> shift) & mask : -1;
                const unsigned same = __match_any_sync(0xffffffffu, d);
                const int wrank = __popc(same & lt);
                if (ok && wrank == 0) wcnt[wid][d] = __popc(same);
                __syncthreads();
                int before = 0;
                if (ok)
                    for (int w = 0; w < wid; w++) before += wcnt[w][d];
                const int pos = ok ? run[d] + before + wrank : 0;
                __syncthreads();
                {
                    int t = 0;
#pragma unroll
                    for (int w = 0; w < kWarps; w++) t += wcnt[w][threadIdx.x];
                    run[threadIdx.x] += t;
                }
                if (ok) dst[pos] = v;
                __syncthreads();  // wcnt[] and run[] are read above before the next round rewrites them
            }
            __syncthreads();
            int32_t *t = src;
            src = dst;
            dst = t;
        }
        if (passes & 1)  // the sorted row is in the scratch array
            for (int e = threadIdx.x; e < len; e += kThreads) data[a + e] = scratch[a + e];
        __syncthreads();
    }
}

int grid_of(int64_t items, int sms, int per_sm = 8) {
    const int64_t b = (items + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * per_sm));
}

}  // namespace

static_assert(kThreads == kDigits, "the block scans of the sorts give one digit per thread");

pr_status scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, cudaStream_t s) {
    if (n <= 0) {
        if (total) PR_CK(cudaMemsetAsync(total, 0, sizeof(int32_t), s));
        return PR_OK;
    }
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    Buf sums;
    PR_TRY(sums.alloc(sizeof(int32_t) * nt, s));
    k_scan_tile_sums<<<(unsigned)nt, kThreads, 0, s>>>(in, n, sums.as<int32_t>());
    k_scan_sums<<<1, kThreads, 0, s>>>(sums.as<int32_t>(), nt, total);
    k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(in, n, sums.as<int32_t>(), out);
    PR_CK(cudaGetLastError());
    return PR_OK;
}

pr_status radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int begin_bit, int end_bit, uint64_t *keys_alt,
                     int32_t *vals_alt, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return PR_OK;
    if (n > INT32_MAX) return fail(PR_EINVAL, "radix_sort: more than 2^31 keys");
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    Buf hist;
    PR_TRY(hist.alloc(sizeof(int32_t) * kDigits * ntiles, s));
    uint64_t *ka = keys, *kb = keys_alt;
    int32_t *va = vals, *vb = vals_alt;
    int passes = 0;
    for (int shift = begin_bit; shift < end_bit; shift += 8, passes++) {
        const int nb = std::min(8, end_bit - shift);
        const int64_t nh = ((int64_t)1 << nb) * ntiles;
        k_radix_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(ka, n, shift, nb, ntiles, hist.as<int32_t>());
        PR_TRY(scan_i32(hist.as<int32_t>(), hist.as<int32_t>(), nh, nullptr, s));
        k_radix_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(ka, va, n, shift, nb, ntiles, hist.as<int32_t>(), kb,
                                                             vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {  // the result is in the alternate buffers
        PR_CK(cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        if (vals) PR_CK(cudaMemcpyAsync(vals, vals_alt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    PR_CK(cudaGetLastError());
    return PR_OK;
}

pr_status sort_rows(int32_t *data, const int32_t *off, int32_t nrows, int64_t m, int bits, int sms, cudaStream_t s) {
    if (nrows <= 0 || m <= 1) return PR_OK;
    k_rows_small<<<grid_of(nrows, sms), kThreads, 0, s>>>(data, off, nrows);
    Buf flag, pos, list, scratch, cnt;
    PR_TRY(flag.alloc(sizeof(int32_t) * nrows, s));
    PR_TRY(pos.alloc(sizeof(int32_t) * nrows, s));
    PR_TRY(list.alloc(sizeof(int32_t) * nrows, s));
    PR_TRY(cnt.alloc(sizeof(int32_t), s));
    k_rows_big_flag<<<grid_of(nrows, sms), kThreads, 0, s>>>(off, nrows, flag.as<int32_t>());
    PR_TRY(scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), nrows, cnt.as<int32_t>(), s));
    k_rows_big_list<<<grid_of(nrows, sms), kThreads, 0, s>>>(flag.as<int32_t>(), pos.as<int32_t>(), nrows,
                                                             list.as<int32_t>());
    PR_TRY(scratch.alloc(sizeof(int32_t) * m, s));
    k_rows_big<<<sms * 4, kThreads, 0, s>>>(data, scratch.as<int32_t>(), off, list.as<int32_t>(), cnt.as<int32_t>(),
                                            bits);
    PR_CK(cudaGetLastError());
    PR_CK(cudaStreamSynchronize(s));  // the scratch buffers are released on return
    return PR_OK;
}

}  // namespace pr
