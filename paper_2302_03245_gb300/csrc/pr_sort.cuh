// pr_sort.cuh -- the library's own scan and sort used by graph creation
// (pr_sort.cu).  Device pointers, the stream's order; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pr_internal.cuh"

namespace pr {

// Where the temporaries of graph creation come from: a stream-ordered pool
// (freed with cudaFreeAsync, no device-wide synchronisation) when `pool` is
// set, else Buf::alloc (the installed allocator hook, or cudaMalloc).
struct Scratch {
    cudaMemPool_t pool = nullptr;
    pr_status get(Buf &b, size_t bytes, cudaStream_t s) const {
        return pool ? b.alloc_async(bytes, s, pool) : b.alloc(bytes, s);
    }
};

// out[i] = in[0] + ... + in[i-1] for i < n (in == out allowed); *total (device,
// optional) = the sum of all n
pr_status scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, const Scratch &sc, cudaStream_t s);

constexpr int kRadixDigits = 256;  // 8-bit digits
constexpr int kRadixMaxPasses = 8;

// The digit counts a radix sort needs, gathered by a kernel that already reads
// every key: each key adds its digit of every pass of a sort on
// [begin_bit, end_bit) to a block histogram h in shared memory (zeroed, then
// a __syncthreads before the first call); radix_count_flush (every thread of
// the block, after a __syncthreads) adds h to the device counts.
__device__ __forceinline__ void radix_count_key(uint32_t (*h)[kRadixDigits], uint64_t key, int begin_bit,
                                                int end_bit) {
    for (int shift = begin_bit, p = 0; shift < end_bit; shift += 8, p++) {
        const int nb = end_bit - shift < 8 ? end_bit - shift : 8;
        atomicAdd(&h[p][(int)((key >> shift) & ((1ull << nb) - 1ull))], 1u);
    }
}
__device__ __forceinline__ void radix_count_flush(uint32_t (*h)[kRadixDigits], int begin_bit, int end_bit,
                                                  uint32_t *counts) {
    const int n = (end_bit - begin_bit + 7) / 8 * kRadixDigits;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t c = (&h[0][0])[k];
        if (c) atomicAdd(&counts[k], c);
    }
}

// Stable ascending sort of keys (with vals, if not NULL) by bits
// [begin_bit, end_bit), at most 64; keys_alt / vals_alt: scratch of the same
// sizes.  The result is in keys / vals, except that a sort of keys alone
// with in_alt given may leave it in keys_alt (then *in_alt = true) instead of
// copying it back.  counts: NULL, or the digit counts of
// every pass (kRadixMaxPasses x kRadixDigits, device) that the caller gathered
// with radix_count_key over exactly these keys; they are overwritten.  *err
// (device int, set by the caller to 0 and read at its next synchronisation)
// becomes nonzero if a pass gave up waiting for an earlier tile; the result is
// then incomplete.
pr_status radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int begin_bit, int end_bit, uint64_t *keys_alt,
                     int32_t *vals_alt, uint32_t *counts, int *err, const Scratch &sc, cudaStream_t s,
                     bool *in_alt = nullptr);

}  // namespace pr
