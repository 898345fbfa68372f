// common.cuh -- shared device-side definitions of the CP-GN CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cpgn.h"

namespace cpgn {

constexpr int kMaxN = CP_MAX_ORDER;

// Shape of a problem as kernels see it.  Packed factor-like buffers store
// A^(1), ..., A^(N) back to back, each row-major s_n x R; row offsets are in
// rows (multiply by R for element offsets).
struct Shape {
    int N;
    int R;
    int64_t dims[kMaxN];
    int64_t roff[kMaxN + 1];   // first packed row of each mode; roff[N] = total rows
    int64_t mid;               // prod_{n=2}^{N-1} s_n (1 for N = 2)
    int64_t total;             // prod_n s_n
};

// A set of per-mode device pointers (factors, outputs) passed by value.
template <typename T>
struct Ptrs {
    T* p[kMaxN];
};

// Device-side statistics of one call; zeroed before and read back after.
struct DevStats {
    double gnorm2[kMaxN];   // ||G^(n)||_F^2
    double mnorm2[kMaxN];   // ||M^(n)||_F^2
    double vnorm2[kMaxN];   // ||V^(n)||_F^2
    double anorm2[kMaxN];   // ||A^(n)||_F^2 after the update
    double res_num;         // sum (x - x~)^2 (after the update)
    double res_den;         // sum x^2
    double eres_num;        // sum (x - x~)^2 at the entry point (residual gradient)
    double eres_den;
    double cg_rnorm;        // final sum_n ||R^(n)||_F
    double slope;           // <G, V> (Armijo line search)
    double dot_part[64];    // its block partials
    int cg_iters;
    int status;             // cp_status raised on the device
    int stopped;            // stationarity test held: no CG iteration, V = 0
    int pad;
};

// State of a bounded-spin grid barrier; zeroed before every persistent launch.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int abort;
    int pad;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_s32(const int* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ unsigned int atom_add_release_u32(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid, on one
// monotonic arrival counter (zeroed before the launch): the k-th barrier is
// complete when the counter reaches k * nblocks.  Thread 0 of each block
// publishes the block's writes (block barrier, fence, release add) and polls
// with acquire loads; the abort flag is read every 32nd poll, so that a poll costs one L2
// round trip.  Every wait is bounded by `limit` polls: on expiry the barrier
// records CP_ERR_TIMEOUT, raises the abort flag and returns false; a block
// waiting in any barrier sees the flag within 32 polls and returns false too,
// so that every block leaves the kernel.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status, unsigned int nblocks, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned int old = atom_add_release_u32(&bar->count, 1u);
        const unsigned int target = (old / nblocks + 1u) * nblocks;
        long long polls = 0;
        while ((int)(ld_acquire_u32(&bar->count) - target) < 0) {
            if (++polls > limit) {
                set_status(status, CP_ERR_TIMEOUT);
                atomicExch(&bar->abort, 1);
                ok = 0;
                break;
            }
            if ((polls & 31) == 0 && ld_volatile_s32(&bar->abort)) {
                ok = 0;
                break;
            }
            if (polls > 256) __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in every thread.  `scratch` holds
// at least blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += scratch[w];
    __syncthreads();
    return t;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

}  // namespace cpgn
