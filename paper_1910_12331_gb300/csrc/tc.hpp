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
    void* planes = nullptr;   // device: bf16 planes in PlaneTiling layout
    size_t bytes = 0;
    const void* key_ptr = nullptr;
    uint64_t key_version = 0;
    int64_t key_total = -1;
    int key_dtype = -1;
    void* fac = nullptr;      // device: split factor planes (small)
    size_t fac_bytes = 0;
};

size_t split_cache_bytes(const cp_desc* d);
// Device workspace (partials, operand planes) one tensor-core MTTKRP call needs, on a GPU with `sms` SMs.
size_t tc_workspace_bytes(const Shape& s, int sms);
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

// Layout of the bf16 planes the tensor-core MTTKRP reads.  X (s_1 x mid x
// s_N) is cut into tiles of 128 rows i (block b) x 64 columns k (chunk c) of
// one slice m.  A tile holds its hi plane then its lo plane, each
// rows(b) x 64 bf16 in 128-byte rows whose 16-byte pieces are permuted by the
// 128-byte swizzle (piece j of row r stored at piece j ^ (r mod 8)), i.e. the
// exact byte image of the tensor cores' K-major operand, so that one linear
// bulk copy per plane lands it in shared memory.  rows(b) = 128 except for the
// last block (its valid rows rounded up to 8).  Tiles are stored in the order
// the MTTKRP visits them: block b, then chunk pair g = c / 2, then slice m,
// then c within the pair, so that each CTA reads one sequential stream.  Rows
// i >= s_1 and columns k >= s_N inside a tile are zero.
struct PlaneTiling {
    int64_t s1, mid, sN;
    int nib, nch, rows_last;
    __host__ __device__ static PlaneTiling of(const Shape& s) {
        PlaneTiling t;
        t.s1 = s.dims[0];
        t.mid = s.mid;
        t.sN = s.dims[s.N - 1];
        t.nib = (int)((t.s1 + 127) / 128);
        t.nch = (int)((t.sN + 63) / 64);
        t.rows_last = (int)(((t.s1 - (int64_t)(t.nib - 1) * 128) + 7) / 8 * 8);
        return t;
    }
    __host__ __device__ int rows(int b) const { return b == nib - 1 ? rows_last : 128; }
    // rows of the padded i range: all rows that exist in some tile
    __host__ __device__ int64_t rows_padded() const { return (int64_t)(nib - 1) * 128 + rows_last; }
    // element offset of tile (b, c, m)
    __host__ __device__ int64_t tile(int b, int c, int64_t m) const {
        const int g = c >> 1, ncg = nch - 2 * g < 2 ? nch - 2 * g : 2;
        return (int64_t)b * nch * mid * (2 * 128 * 64) +
               ((int64_t)(2 * g) * mid + m * ncg + (c & 1)) * (2 * (int64_t)rows(b) * 64);
    }
    // element offset of X[i, m, k] in plane 0 (hi) or 1 (lo)
    __host__ __device__ int64_t elem(int64_t i, int64_t m, int64_t k, int plane) const {
        const int b = (int)(i >> 7), r = (int)(i & 127), kk = (int)(k & 63);
        return tile(b, (int)(k >> 6), m) + ((int64_t)plane * rows(b) + r) * 64 + ((((kk >> 3) ^ (r & 7)) << 3) | (kk & 7));
    }
    __host__ __device__ int64_t total() const { return tile(nib - 1, 0, 0) + (int64_t)nch * mid * 2 * rows_last * 64; }
};

// All-mode MTTKRP of a tensor given directly as bf16 planes in PlaneTiling
// layout (used for the residual tensor).
cp_status tc_mttkrp_planes(SplitCache& c, const void* planes, const Shape& s, Ptrs<const double> A, Ptrs<double> M,
                           int* status, cudaStream_t st);

}  // namespace cpgn
