// pr_sort.cuh -- the library's own scan and sorts used by graph creation
// (pr_sort.cu).  Device pointers, the stream's order; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pr_internal.cuh"

namespace pr {

// out[i] = in[0] + ... + in[i-1] for i < n (in == out allowed); *total (device,
// optional) = the sum of all n
pr_status scan_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total, cudaStream_t s);

// Stable ascending sort of keys (with vals, if not NULL) by bits
// [begin_bit, end_bit); keys_alt / vals_alt: scratch of the same sizes.  The
// result is in keys / vals.
pr_status radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int begin_bit, int end_bit, uint64_t *keys_alt,
                     int32_t *vals_alt, cudaStream_t s);

// Every row [off[j], off[j+1]) of data (values in [0, 2^bits)) sorted ascending;
// m = off[nrows].  Synchronises the stream before returning.
pr_status sort_rows(int32_t *data, const int32_t *off, int32_t nrows, int64_t m, int bits, int sms, cudaStream_t s);

}  // namespace pr
