// pr_sort.cu -- the library's own scans and sorts for graph creation (no
// library sort or scan on the path):
//   scan_i32       exclusive prefix sum of int32 counts (three passes: tile
//                  sums, one block scans them, tiles add their base);
//   radix_sort     stable LSD radix sort of 64-bit keys with optional int32
//                  values, 8-bit digits: the digit counts of all passes from
//                  one read of the keys, then one kernel per pass that orders
//                  each tile by digit in shared memory (warp ballots and
//                  per-warp counts give the ranks), finds the tile's global
//                  offsets by decoupled look-back and writes every digit's run
//                  of the tile as one contiguous piece.
// The results do not depend on scheduling.

#include <algorithm>

#include "pr_debug.cuh"
#include "pr_internal.cuh"
#include "pr_sort.cuh"

namespace pr {

namespace {

constexpr int kScanTile = 2048;   // int32 per scan tile (256 threads x 8)
constexpr int kDigits = kRadixDigits;
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
// Stable LSD radix sort with 8-bit digits, one kernel per digit pass (the
// "one-sweep" arrangement): the digit counts of every pass come from one read
// of the keys before the first pass; in a pass each tile ranks its keys in
// shared memory and finds how many keys of each digit the tiles before it
// hold by looking back through their published counts (decoupled look-back),
// so no per-pass histogram kernel or scan is needed.
__device__ __forceinline__ int digit_of(uint64_t k, int shift, int nbits) {
    return (int)((k >> shift) & ((1ull << nbits) - 1ull));
}

constexpr int kMaxPasses = kRadixMaxPasses;
// digit counts of every pass, one read of the keys
__global__ void __launch_bounds__(kThreads) k_radix_counts(const uint64_t *keys, int64_t n, int begin_bit,
                                                          int end_bit, uint32_t *counts) {
    __shared__ uint32_t h[kMaxPasses][kDigits];
    for (int k = threadIdx.x; k < kMaxPasses * kDigits; k += kThreads) (&h[0][0])[k] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        radix_count_key(h, keys[i], begin_bit, end_bit);
    __syncthreads();
    radix_count_flush(h, begin_bit, end_bit, counts);
}

// per pass (block p): exclusive sum over the digits, in place
__global__ void __launch_bounds__(kThreads) k_radix_starts(uint32_t *counts) {
    __shared__ int sh[32];
    uint32_t *c = counts + (size_t)blockIdx.x * kDigits;
    int total;
    const int ex = block_exscan((int)c[threadIdx.x], sh, &total);
    c[threadIdx.x] = (uint32_t)ex;
}

// A tile's published count of one digit: bits [0, 32) the count, bit 32 set
// when the count is the tile's own (aggregate), bit 33 when it includes every
// earlier tile (inclusive), bits [40, 48) the pass it belongs to (so the
// words of the previous pass read as not yet published).
constexpr unsigned long long kStAgg = 1ull << 32, kStIncl = 1ull << 33;
constexpr int kSpinLimit = 1 << 20;  // look-back polls without progress before a tile gives up
constexpr int kLookBack = 8;         // status words read per look-back step
constexpr int kMatchEvery = 3;       // ranking rounds that use the warp match instruction (0: none)

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st_status(unsigned long long *p, unsigned long long v) {
    *(volatile unsigned long long *)p = v;
}

// One digit pass over tiles of R * kThreads keys.  A block takes the next
// tile number from a counter (so every earlier tile belongs to a block that
// has already started) and ranks the tile's keys: warp w holds the keys
// w * R * 32 + r * 32 + lane in registers and, in order of r, ranks each among
// the equal digits of its segment (the lanes with equal digits come from one
// ballot per digit bit; one of them reads and advances the warp's running
// count of the digit).  The warps' counts, summed per digit in warp order, and
// a block scan over the digits give the tile's own digit-sorted order.  Thread
// d publishes the tile's count of digit d, looks back through the earlier
// tiles' words until it meets an inclusive one, and publishes its inclusive
// count.  The keys, placed in the tile's order in shared memory, then go out
// with consecutive threads writing consecutive keys, so each digit's run of
// the tile is one contiguous piece.  A look-back that polls kSpinLimit times
// without progress sets *err and the tile writes nothing.
template <int R, bool VALS>
__global__ void __launch_bounds__(kThreads, 3) k_radix_pass(const uint64_t *keys, const int32_t *vals, int64_t n,
                                                        int shift, int nbits, const uint32_t *starts,
                                                        unsigned long long *status, int epoch,
                                                        unsigned int *tile_ctr, int *err, uint64_t *keys_out,
                                                        int32_t *vals_out) {
    constexpr int T = R * kThreads;
    __shared__ uint64_t skeys[T];
    __shared__ int32_t svals[VALS ? T : 1];
    __shared__ int whist[kWarps][kDigits];
    __shared__ int lstart[kDigits];
    __shared__ int64_t gbase[kDigits];
    __shared__ int sh[32];
    __shared__ unsigned int s_tile;
    __shared__ int s_bad;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_ctr, 1u);
        s_bad = 0;
    }
    for (int k = threadIdx.x; k < kWarps * kDigits; k += kThreads) (&whist[0][0])[k] = 0;
    __syncthreads();
    const unsigned int t = s_tile;
    const int64_t base = (int64_t)t * T;
    uint64_t key[R];
    int dig[R], rank[R];
    int32_t val[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t i = base + wid * (R * 32) + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? keys[i] : 0;
        dig[r] = ok ? digit_of(key[r], shift, nbits) : -1;
        if (VALS) val[r] = ok ? vals[i] : 0;
    }
    const unsigned lt = (1u << lane) - 1u;
    const bool full = base + T <= n;  // every key of the tile is valid (all tiles but the last)
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int d = dig[r];
        // The lanes holding the same digit.  Rounds r with r % kMatchEvery == 0
        // take the warp match instruction, the others one ballot per digit bit:
        // the two run on different pipes, so mixing them spreads the load.
        unsigned same;
        if (kMatchEvery > 0 && r % kMatchEvery == 0) {
            same = __match_any_sync(0xffffffffu, d);
        } else {
            same = full ? 0xffffffffu : ~(__ballot_sync(0xffffffffu, d < 0) ^ (d < 0 ? 0xffffffffu : 0u));
#pragma unroll
            for (int b = 0; b < 8; b++) {  // digits above nbits are 0 on every lane
                const unsigned m = 0u - ((unsigned)(d >> b) & 1u);
                same &= ~(__ballot_sync(0xffffffffu, m != 0) ^ m);
            }
        }
        const int leader = __ffs(same) - 1;
        int before = 0;
        if (d >= 0 && lane == leader) {  // one lane per digit reads and advances the warp's count
            before = whist[wid][d];
            whist[wid][d] = before + __popc(same);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[r] = before + __popc(same & lt);
        __syncwarp();
    }
    __syncthreads();
    {  // thread d = digit d
        const int d = threadIdx.x;
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const int c = whist[w][d];
            whist[w][d] = tot;
            tot += c;
        }
        int total;
        lstart[d] = block_exscan(tot, sh, &total);
        const unsigned long long E = (unsigned long long)(epoch & 0xFF) << 40;
        unsigned long long *mine = status + (size_t)t * kDigits + d;
        uint32_t excl = 0;
        if (t == 0) {
            st_status(mine, E | kStIncl | (uint32_t)tot);
        } else {
            st_status(mine, E | kStAgg | (uint32_t)tot);
            // Look back kLookBack words at a time (independent loads); tile 0
            // always publishes an inclusive word, so the walk ends there at the
            // latest.
            int64_t j = (int64_t)t - 1;
            int spins = 0;
            bool ok = true;
#ifdef PR_DEBUG
            // test hook of the debug build: every wait runs out at its first poll
            const int spin_limit = g_pr_dbg.inject == DBG_SORT_WAIT ? 0 : kSpinLimit;
#else
            constexpr int spin_limit = kSpinLimit;
#endif
            while (true) {
                if (spins >= spin_limit) {
                    ok = false;
                    s_bad = 1;
                    break;
                }
                unsigned long long v[kLookBack];
#pragma unroll
                for (int w = 0; w < kLookBack; w++) v[w] = j - w >= 0 ? ld_status(status + (size_t)(j - w) * kDigits + d) : 0;
                int used = 0;
                bool incl = false;
#pragma unroll
                for (int w = 0; w < kLookBack; w++) {
                    if (used < w || incl) break;  // an earlier word was not ready, or the walk is over
                    if (((v[w] >> 40) & 0xFF) != (unsigned long long)(epoch & 0xFF) || !(v[w] & (kStAgg | kStIncl)))
                        break;
                    excl += (uint32_t)v[w];
                    used++;
                    incl = (v[w] & kStIncl) != 0;
                }
                if (incl) break;
                j -= used;
                if (used == 0) {
                    ++spins;
                    __nanosleep(32);
                }
            }
            // (a tile that gave up leaves its aggregate: later tiles look past it)
            if (ok) st_status(mine, E | kStIncl | (uint32_t)(excl + (uint32_t)tot));
        }
        gbase[d] = (int64_t)starts[d] + excl;
    }
    __syncthreads();
    if (s_bad) {  // every thread sees the same flag after the barrier
        if (threadIdx.x == 0) atomicExch(err, 1);
        return;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int d = dig[r];
        if (d < 0) continue;
        const int pos = lstart[d] + whist[wid][d] + rank[r];
        skeys[pos] = key[r];
        if (VALS) svals[pos] = val[r];
    }
    __syncthreads();
    const int cnt = (int)(n - base < T ? n - base : T);
    if (cnt == T) {  // a full tile: independent iterations, unrolled
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int p = r * kThreads + threadIdx.x;
            const uint64_t k = skeys[p];
            const int d = digit_of(k, shift, nbits);
            const int64_t g = gbase[d] + (p - lstart[d]);
            keys_out[g] = k;
            if (VALS) vals_out[g] = svals[p];
        }
    } else {
        for (int p = threadIdx.x; p < cnt; p += kThreads) {
            const uint64_t k = skeys[p];
            const int d = digit_of(k, shift, nbits);
            const int64_t g = gbase[d] + (p - lstart[d]);
            keys_out[g] = k;
            if (VALS) vals_out[g] = svals[p];
        }
    }
}

}  // namespace

static_assert(kThreads == kDigits, "the block scans of the sorts give one digit per thread");

// host side of this translation unit's debug record (only the test hook is read)
bool dbg_reset_sort(int inject) {
#ifdef PR_DEBUG
    DbgRec z{};
    z.inject = inject;
    return cudaMemcpyToSymbol(g_pr_dbg, &z, sizeof(z)) == cudaSuccess;
#else
    (void)inject;
    return false;
#endif
}

pr_status scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, const Scratch &sc, cudaStream_t s) {
    if (n <= 0) {
        if (total) PR_CK(cudaMemsetAsync(total, 0, sizeof(int32_t), s));
        return PR_OK;
    }
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    Buf sums;
    PR_TRY(sc.get(sums, sizeof(int32_t) * nt, s));
    k_scan_tile_sums<<<(unsigned)nt, kThreads, 0, s>>>(in, n, sums.as<int32_t>());
    k_scan_sums<<<1, kThreads, 0, s>>>(sums.as<int32_t>(), nt, total);
    k_scan_tiles<<<(unsigned)nt, kThreads, 0, s>>>(in, n, sums.as<int32_t>(), out);
    PR_CK(cudaGetLastError());
    return PR_OK;
}

pr_status radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int begin_bit, int end_bit, uint64_t *keys_alt,
                     int32_t *vals_alt, uint32_t *counts, int *err, const Scratch &sc, cudaStream_t s,
                     bool *in_alt) {
    if (in_alt) *in_alt = false;
    if (n <= 1 || end_bit <= begin_bit) return PR_OK;
    if (n > INT32_MAX) return fail(PR_EINVAL, "radix_sort: more than 2^31 keys");
    const int npass = (end_bit - begin_bit + 7) / 8;
    if (npass > kMaxPasses) return fail(PR_EINVAL, "radix_sort: more than 64 bits");
    // keys only: 16 per thread; with values: 8 (shared memory)
    const int T = (vals ? 8 : 16) * kThreads;
    const int64_t ntiles = (n + T - 1) / T;
    Buf own, status;
    PR_TRY(sc.get(own, sizeof(uint32_t) * (kMaxPasses * kDigits + kMaxPasses), s));
    PR_TRY(sc.get(status, sizeof(unsigned long long) * kDigits * ntiles, s));
    unsigned int *ctr = own.as<uint32_t>() + kMaxPasses * kDigits;
    PR_CK(cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * kMaxPasses, s));
    PR_CK(cudaMemsetAsync(status.p, 0, sizeof(unsigned long long) * kDigits * ntiles, s));
    uint32_t *cnt = counts;
    if (!cnt) {
        cnt = own.as<uint32_t>();
        PR_CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kMaxPasses * kDigits, s));
        int dev = 0, sms = 0;
        PR_CK(cudaGetDevice(&dev));
        PR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t cg = std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sms * 4);
        k_radix_counts<<<(unsigned)cg, kThreads, 0, s>>>(keys, n, begin_bit, end_bit, cnt);
    }
    k_radix_starts<<<npass, kThreads, 0, s>>>(cnt);
    uint64_t *ka = keys, *kb = keys_alt;
    int32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < npass; p++) {
        const int shift = begin_bit + 8 * p;
        const int nb = std::min(8, end_bit - shift);
        unsigned long long *st = status.as<unsigned long long>();
        // the pass number tags the status words, so one zeroing serves every pass
        if (vals)
            k_radix_pass<8, true><<<(unsigned)ntiles, kThreads, 0, s>>>(ka, va, n, shift, nb, cnt + p * kDigits, st,
                                                                       p + 1, ctr + p, err, kb, vb);
        else
            k_radix_pass<16, false><<<(unsigned)ntiles, kThreads, 0, s>>>(ka, nullptr, n, shift, nb,
                                                                         cnt + p * kDigits, st, p + 1, ctr + p, err,
                                                                         kb, nullptr);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if ((npass & 1) && in_alt && !vals) {  // the caller takes the result from keys_alt
        *in_alt = true;
    } else if (npass & 1) {  // the result is in the alternate buffers
        PR_CK(cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        if (vals) PR_CK(cudaMemcpyAsync(vals, vals_alt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    PR_CK(cudaGetLastError());
    return PR_OK;
}

}  // namespace pr
