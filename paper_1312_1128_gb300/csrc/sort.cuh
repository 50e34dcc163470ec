// sort.cuh -- device-wide scan and radix sort used by the tree build and ray grouping.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

void note_launch();  // defined in api.cu

namespace lens {

size_t scan_temp_bytes(int64_t n);
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, void* tmp,
                        cudaStream_t s);

template <typename K> size_t radix_sort_temp_bytes(int64_t n);
// err: the device error word (DERR_INDEX if a bounds check in a pass failed).
template <typename K>
void radix_sort_pairs(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, int begin_bit,
                      int end_bit, void* tmp, cudaStream_t s, K** kres, uint32_t** vres, uint32_t* err);

}  // namespace lens
