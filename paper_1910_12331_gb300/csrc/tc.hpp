// tc.hpp -- the tensor-core (tcgen05) MTTKRP path: bf16 split planes of X and
// of the factors, and its launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace cpgn {

// Handle-owned cache of the bf16 high/low planes of X, keyed by the X
// pointer, its shape and the caller's version stamp.
struct SplitCache {
    void* planes = nullptr;   // device: [2][total] bf16 (high plane, then low plane)
    size_t bytes = 0;
    const void* key_ptr = nullptr;
    uint64_t key_version = 0;
    int64_t key_total = -1;
    int key_dtype = -1;
    void* fac = nullptr;      // device: split factor planes (small)
    size_t fac_bytes = 0;
};

size_t split_cache_bytes(const cp_desc* d);
// Kernels one tensor-core MTTKRP call launches (before it runs: counts the split if the cache misses).
int tc_launch_count(const SplitCache& c, const cp_desc* d, const Shape& s);
void split_cache_free(SplitCache& c);
// All-mode MTTKRP on tensor cores (bf16x3): M zeroed by the caller.
// status: device word that receives CP_ERR_TIMEOUT if a bounded wait expires.
cp_status tc_mttkrp_all(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                        Ptrs<double> M, int* status, cudaStream_t st);
// Single mode n (ALS) on tensor cores: M.p[n] zeroed by the caller.
cp_status tc_mttkrp_mode(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                         Ptrs<double> M, int n, int* status, cudaStream_t st);

// All-mode MTTKRP of a tensor given directly as bf16 planes [2][s1][mid][pitch],
// pitch = tc_row_pitch(s_N) (used for the residual tensor).
cp_status tc_mttkrp_planes(SplitCache& c, const void* planes, const Shape& s, Ptrs<const double> A, Ptrs<double> M,
                           int* status, cudaStream_t st);
int64_t tc_row_pitch(int64_t sN);

}  // namespace cpgn
