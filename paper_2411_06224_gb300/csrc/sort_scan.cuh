// Hand-written device primitives of the hash assembly: stable LSD radix sort
// of (uint64 key, uint32 value) pairs and the exclusive scan of int32
// (sort_scan.cu).  Both run on the given stream; temp is caller-provided
// device memory of at least the stated size.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

size_t radix_sort_temp_bytes(int64_t n);
// keys_out / vals_out receive the pairs sorted by the key's bits [0, end_bit),
// stable; the inputs are left as they are (they must not alias the outputs).
int radix_sort_pairs(cudaStream_t st, const uint64_t* k_in, uint64_t* k_out, const uint32_t* v_in, uint32_t* v_out,
                     int64_t n, int end_bit, void* temp, size_t temp_bytes);

size_t scan_temp_bytes(int64_t n);
// out[i] = sum of in[0..i-1]; in and out may be the same array; n < 2^31.
int exclusive_scan_i32(cudaStream_t st, const int32_t* in, int32_t* out, int64_t n, void* temp, size_t temp_bytes);

}  // namespace gs
