// k_mttkrp_tc.cu -- all-mode MTTKRP on tcgen05 tensor cores (sm_103a), bf16x3.
//
// Arithmetic.  Every operand value v is split into bf16 parts v = v_hi + v_lo
// (+ O(2^-17 |v|)); a product is formed as x_hi*b_hi + x_hi*b_lo + x_lo*b_hi,
// each term exact in the FP32 tensor-core accumulator (the split of
// Henry, Tang and Heinecke, "Leveraging the bfloat16 artificial intelligence
// datatype for higher-precision computations", ARITH 2019).  Accumulation is
// FP32; the cross-block reductions and the outputs are FP64.
//
// Algorithm (Section 2.2's dimension tree, evaluated in one pass over X).  X is
// viewed as s_1 x mid x s_N.  For every slice m of the middle modes, with
// w_m[r] = prod_{middle q} a^(q)_{i_q(m) r}:
//   GEMM-Y  Y_m = X(:, m, :) A^(N)                  (M = i rows, K = k)
//   GEMM-Z  Z   = X(:, m, :)^T (A^(1) * w_m)        (M = k rows, K = i)
// GEMM-Z folds w_m into its B operand, so its TMEM accumulator sums over all
// slices of a work unit and directly holds a partial M^(N).  Y_m is read out
// per slice: M^(1) += w_m * Y_m (registers) and c_m = colsum(A^(1) * Y_m)
// feeds the middle modes.  Both GEMMs read the same shared-memory tile of X:
// K-major for GEMM-Y and MN-major for GEMM-Z.
//
// Kernel structure: persistent, one CTA per SM, 6 warps.
//   warp 0      TMA producer: X tiles (128 i x 128 k, both planes) and the
//               matching B_Y tile of A^(N), 2-stage ring, mbarrier complete_tx.
//   warp 1      TMEM allocator and single-thread tcgen05.mma issuer.
//   warps 2..5  epilogue: build B_Z = (A^(1) * w_m) planes in shared memory,
//               read Y_m from TMEM (double-buffered), accumulate M^(1),
//               reduce c_m, and at the end of a unit read the M^(N) partial.
// A work unit is (i-block of 128 rows, k-group of <= 512 columns, slice range).
// Units write FP32 partials to workspace; a finalize kernel reduces them in a
// fixed order into the FP64 outputs (no atomics, deterministic).
// Every mbarrier wait is bounded: on expiry the CTA records CP_ERR_TIMEOUT,
// raises a CTA-local abort flag, drains what it issued (bounded) and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kernels.hpp"
#include "tc.hpp"

namespace cpgn {

namespace tc {

constexpr int kThreads = 192;           // 6 warps
constexpr int kStages = 2;
constexpr int kBI = 128;                // rows of an i-block (MMA M of GEMM-Y)
constexpr int kKC = 128;                // columns of a k-chunk (MMA M of GEMM-Z)
constexpr int kRT = 64;                 // rank columns per launch (MMA N)
constexpr int kChunksPerGroup = 4;      // k-group = 512 columns
constexpr uint32_t kXSub = 32 * 1024;   // one 64-column sub-tile of X, both planes
constexpr uint32_t kXPlane = 16 * 1024; // one plane of a sub-tile (128 rows x 128 B)
constexpr uint32_t kBYSub = 16 * 1024;  // one 64-column sub-tile of B_Y, both planes
constexpr uint32_t kBYPlane = 8 * 1024;
constexpr uint32_t kStageBytes = 2 * kXSub + 2 * kBYSub;  // 96 KB
constexpr uint32_t kBZBytes = 32 * 1024;
constexpr uint32_t kDynSmem = kStages * kStageBytes + kBZBytes + 1024;  // + alignment slack
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitLimit = 1LL << 26;

struct Params {
    int N;
    int R;              // columns of this rank tile (<= 64)
    int64_t s1, mid, sN;
    int nib, nkg, nsplit, nunits;
    const float* A1f;   // [s1][64] rows of A^(1) (rank tile), FP32, zero padded
    const float* midf;  // middle factors [rows][64], FP32
    int64_t midoff[kMaxN];
    int64_t middim[kMaxN];
    float* P_Y1;        // [nunits][128][64]
    float* P_Z;         // [nunits][512][64]
    float* P_c;         // [nib * nkg][mid][64]
    int* status;
    long long* trace;   // event timestamps of block 0 (trace builds only), else null
};

// Optional event trace of block 0 (compiled in with -DCPGN_TC_TRACE): slot
// ev * 1024 + idx receives clock64() at event ev, occurrence idx.
#ifdef CPGN_TC_TRACE
#define TC_TRACE(ev, idx)                                                                  \
    do {                                                                                   \
        if (p.trace && blockIdx.x == 0 && (idx) < 1024) p.trace[(ev) * 1024 + (idx)] = clock64(); \
    } while (0)
#else
#define TC_TRACE(ev, idx) \
    do {                  \
    } while (0)
#endif

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase.  Returns false (and raises the CTA abort
// flag and the global status) when the limit expires or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (i > 256) __nanosleep(32);
    }
    *abort_flag = 1;
    atomicCAS(status, 0, CP_ERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor, 128-byte swizzle, version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor: D F32, A/B BF16, M = 128, N = 64, A K- or MN-major, B K-major.
__device__ __forceinline__ uint32_t idesc_bf16(bool a_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) | ((uint32_t)(kRT >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Column of the value v[j] held by `lane` after butterfly_reduce64 (2 per lane).
__device__ __forceinline__ int butterfly_col(int lane, int j) {
    return ((lane >> 4) & 1) * 32 + ((lane >> 3) & 1) * 16 + ((lane >> 2) & 1) * 8 + ((lane >> 1) & 1) * 4 +
           (lane & 1) * 2 + j;
}
// Reduce 64 per-lane values over the 32 lanes of a warp; lane ends with the
// sums of columns butterfly_col(lane, 0) and butterfly_col(lane, 1) in v[0], v[1].
__device__ __forceinline__ void butterfly_reduce64(float* v, int lane) {
#pragma unroll
    for (int off = 16, w = 32; off >= 1; off >>= 1, w >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < w; ++j) {
            const float send = upper ? v[j] : v[j + w];
            const float keep = upper ? v[j + w] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

__device__ __forceinline__ void named_sync_epi() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__host__ __device__ __forceinline__ int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

struct Unit {
    int b, kg;
    int64_t m0, m1;
};
__device__ __forceinline__ Unit unit_of(const Params& p, int u) {
    Unit r;
    const int j = u % p.nsplit;
    const int bk = u / p.nsplit;
    r.b = bk / p.nkg;
    r.kg = bk % p.nkg;
    r.m0 = (int64_t)j * p.mid / p.nsplit;
    r.m1 = (int64_t)(j + 1) * p.mid / p.nsplit;
    return r;
}

__global__ void __launch_bounds__(kThreads, 1)
    mttkrp_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBY, Params p) {
    extern __shared__ __align__(1024) unsigned char dsmem[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages];
    __shared__ __align__(8) uint64_t bar_bz_full, bar_bz_empty, bar_dy_full[2], bar_dy_empty[2], bar_dz_full,
        bar_dz_empty, bar_drain;
    __shared__ int dec_s;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;
    __shared__ float w_s[2][kRT];
    __shared__ float red_s[4][kRT];

    unsigned char* base = (unsigned char*)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    const uint32_t s_stage0 = sbase;
    const uint32_t s_bz = sbase + kStages * kStageBytes;
    unsigned char* bz_gen = base + kStages * kStageBytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_bz_full), 128);
        mbar_init(smem_u32(&bar_bz_empty), 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bar_dy_full[s]), 1);
            mbar_init(smem_u32(&bar_dy_empty[s]), 128);
        }
        mbar_init(smem_u32(&bar_dz_full), 1);
        mbar_init(smem_u32(&bar_dz_empty), 128);
        mbar_init(smem_u32(&bar_drain), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t t_dy0 = tmem, t_dz = tmem + 2 * kRT;
    const int G = gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < p.nunits && ok; u += G) {
                const Unit U = unit_of(p, u);
                const int c0 = U.kg * kChunksPerGroup;
                const int c1 = (int)imin(c0 + kChunksPerGroup, (p.sN + kKC - 1) / kKC);
                for (int64_t m = U.m0; m < U.m1 && ok; ++m)
                    for (int c = c0; c < c1; ++c, ++it) {
                        const int s = it % kStages;
                        const uint32_t ph = (it / kStages) & 1;
                        if (!(ok = mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1, &abort_s, p.status))) break;
                        TC_TRACE(0, it);
                        const uint32_t fb = smem_u32(&bar_full[s]);
                        mbar_expect_tx(fb, kStageBytes);
                        const uint32_t st = s_stage0 + s * kStageBytes;
                        tma_load_4d(st, &tmX, c * kKC, (int)m, U.b * kBI, 0, fb);
                        tma_load_4d(st + kXSub, &tmX, c * kKC + 64, (int)m, U.b * kBI, 0, fb);
                        tma_load_2d(st + 2 * kXSub, &tmBY, c * kKC, 0, fb);
                        tma_load_2d(st + 2 * kXSub + kBYSub, &tmBY, c * kKC + 64, 0, fb);
                    }
            }
            // drain: every issued stage must have landed before the CTA may exit
            for (int k = (it > kStages ? it - kStages : 0); k < it; ++k)
                mbar_wait(smem_u32(&bar_full[k % kStages]), (k / kStages) & 1, &abort_s, p.status);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA
        if (lane == 0) {
            const uint32_t id_y = idesc_bf16(false), id_z = idesc_bf16(true);
            int it = 0;
            int64_t t = 0;  // slice counter
            int v = 0;      // unit counter
            bool ok = true;
            for (int u = blockIdx.x; u < p.nunits && ok; u += G, ++v) {
                const Unit U = unit_of(p, u);
                const int c0 = U.kg * kChunksPerGroup;
                const int c1 = (int)imin(c0 + kChunksPerGroup, (p.sN + kKC - 1) / kKC);
                const int ivalid = (int)imin(kBI, p.s1 - (int64_t)U.b * kBI);
                const int zsteps = (ivalid + 15) / 16;
                bool zfirst[kChunksPerGroup] = {true, true, true, true};
                // the epilogue must have read the previous unit's M^(N) partial
                if (!(ok = mbar_wait(smem_u32(&bar_dz_empty), (v & 1) ^ 1, &abort_s, p.status))) break;
                for (int64_t m = U.m0; m < U.m1 && ok; ++m, ++t) {
                    const int buf = (int)(t & 1);
                    const uint32_t dph = (uint32_t)((t >> 1) & 1);
                    if (!(ok = mbar_wait(smem_u32(&bar_dy_empty[buf]), dph ^ 1, &abort_s, p.status))) break;
                    tc_fence_after();
                    const uint32_t t_dy = t_dy0 + buf * kRT;
                    bool yfirst = true;
                    for (int c = c0; c < c1; ++c, ++it) {
                        const int s = it % kStages;
                        if (!(ok = mbar_wait(smem_u32(&bar_full[s]), (it / kStages) & 1, &abort_s, p.status))) break;
                        TC_TRACE(1, it);
                        tc_fence_after();
                        const uint32_t st = s_stage0 + s * kStageBytes;
                        // GEMM-Y: D_Y(128 i x 64 r) += X(i, k) * B_Y(k, r), k in this chunk
                        const int kvalid = (int)imin(kKC, p.sN - (int64_t)c * kKC);
                        const int ysteps = (kvalid + 15) / 16;
                        for (int ks = 0; ks < ysteps; ++ks) {
                            const int sub = ks >> 2, kk = ks & 3;
                            const uint32_t xa = st + sub * kXSub + kk * 32;
                            const uint32_t ba = st + 2 * kXSub + sub * kBYSub + kk * 32;
                            const uint64_t xh = sdesc(xa, 16, 1024), xl = sdesc(xa + kXPlane, 16, 1024);
                            const uint64_t bh = sdesc(ba, 16, 1024), bl = sdesc(ba + kBYPlane, 16, 1024);
                            tc_mma(t_dy, xh, bh, id_y, yfirst ? 0 : 1);
                            tc_mma(t_dy, xh, bl, id_y, 1);
                            tc_mma(t_dy, xl, bh, id_y, 1);
                            yfirst = false;
                        }
                        // GEMM-Z needs this slice's B_Z = A^(1) * w_m
                        if (c == c0) {
                            if (!(ok = mbar_wait(smem_u32(&bar_bz_full), (uint32_t)(t & 1), &abort_s, p.status))) break;
                            TC_TRACE(2, (int)t);
                            tc_fence_after();
                        }
                        // GEMM-Z: D_Z[c](128 k x 64 r) += X(i, k)^T * B_Z(i, r), i in this block
                        const uint32_t t_z = t_dz + (c - c0) * kRT;
                        for (int ks = 0; ks < zsteps; ++ks) {
                            const uint32_t xa = st + ks * 2048;
                            const uint32_t ba = s_bz + (ks >> 2) * 16384 + (ks & 3) * 32;
                            const uint64_t xh = sdesc(xa, kXSub, 1024), xl = sdesc(xa + kXPlane, kXSub, 1024);
                            const uint64_t bh = sdesc(ba, 16, 1024), bl = sdesc(ba + 8192, 16, 1024);
                            tc_mma(t_z, xh, bh, id_z, zfirst[c - c0] ? 0 : 1);
                            tc_mma(t_z, xh, bl, id_z, 1);
                            tc_mma(t_z, xl, bh, id_z, 1);
                            zfirst[c - c0] = false;
                        }
                        tc_commit(smem_u32(&bar_empty[s]));
                        TC_TRACE(3, it);
                    }
                    if (!ok) break;
                    tc_commit(smem_u32(&bar_dy_full[buf]));
                    tc_commit(smem_u32(&bar_bz_empty));
                }
                if (ok) tc_commit(smem_u32(&bar_dz_full));
            }
            // drain: every issued MMA must have completed before TMEM is freed
            tc_commit(smem_u32(&bar_drain));
            mbar_wait(smem_u32(&bar_drain), 0, &abort_s, p.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;           // TMEM lane quadrant of this warp
        const int row = q * 32 + lane;    // row within the i-block / k-chunk
        const int et = threadIdx.x - 64;  // 0..127
        // bounded wait with a decision shared by all 128 epilogue threads, so that
        // they leave together and no named barrier is left waiting
        auto epi_wait = [&](uint32_t bar, uint32_t parity) -> bool {
            mbar_wait(bar, parity, &abort_s, p.status);
            named_sync_epi();
            if (et == 0) dec_s = abort_s;
            named_sync_epi();
            return dec_s == 0;
        };
        float a1r[kRT];
        float m1acc[kRT];
        int64_t t = 0;
        int v = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < p.nunits && ok; u += G, ++v) {
            const Unit U = unit_of(p, u);
            const int64_t gi = (int64_t)U.b * kBI + row;
            const bool rowok = gi < p.s1;
#pragma unroll
            for (int r = 0; r < kRT; ++r) {
                a1r[r] = rowok ? p.A1f[gi * kRT + r] : 0.0f;
                m1acc[r] = 0.0f;
            }
            float* Pc = p.P_c + (int64_t)(U.b * p.nkg + U.kg) * p.mid * kRT;
            const int64_t nsl = U.m1 - U.m0;
            const int64_t t0 = t;
            for (int64_t j = 0; j <= nsl && ok; ++j) {
                if (j < nsl) {
                    // ---- w_m and B_Z(m) = A^(1)(block) * w_m, bf16 hi/lo, K-major swizzled
                    const int64_t tt = t0 + j, m = U.m0 + j;
                    const int wb = (int)(tt & 1);
                    if (!(ok = epi_wait(smem_u32(&bar_bz_empty), (uint32_t)((tt & 1) ^ 1)))) break;
                    if (et == 0) TC_TRACE(4, (int)tt);
                    if (et < kRT) {
                        float w = 1.0f;
                        int64_t rem = m;
                        for (int qq = p.N - 2; qq >= 1; --qq) {
                            const int64_t iq = rem % p.middim[qq];
                            rem /= p.middim[qq];
                            w *= p.midf[(p.midoff[qq] + iq) * kRT + et];
                        }
                        w_s[wb][et] = w;
                    }
                    named_sync_epi();
                    {
                        const int i = row;  // K index of B_Z
                        unsigned char* sub = bz_gen + (i >> 6) * 16384;
                        const int ii = i & 63;
#pragma unroll 8
                        for (int r = 0; r < kRT; ++r) {
                            const float pv = a1r[r] * w_s[wb][r];
                            const __nv_bfloat16 hi = __float2bfloat16_rn(pv);
                            const __nv_bfloat16 lo = __float2bfloat16_rn(pv - __bfloat162float(hi));
                            const uint32_t off = r * 128 + ((((ii >> 3) ^ (r & 7)) & 7) << 4) + (ii & 7) * 2;
                            *reinterpret_cast<__nv_bfloat16*>(sub + off) = hi;
                            *reinterpret_cast<__nv_bfloat16*>(sub + 8192 + off) = lo;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(smem_u32(&bar_bz_full));
                    if (et == 0) TC_TRACE(5, (int)tt);
                }
                if (j > 0) {
                    // ---- epilogue of the previous slice: Y_m
                    const int64_t tp = t0 + j - 1, m = U.m0 + j - 1;
                    const int buf = (int)(tp & 1);
                    if (!(ok = epi_wait(smem_u32(&bar_dy_full[buf]), (uint32_t)((tp >> 1) & 1)))) break;
                    if (et == 0) TC_TRACE(6, (int)tp);
                    tc_fence_after();
                    float y[kRT];
                    const uint32_t ta = t_dy0 + buf * kRT + ((uint32_t)(q * 32) << 16);
#pragma unroll
                    for (int jj = 0; jj < kRT; jj += 16) tmem_ld16(ta + jj, y + jj);
                    tc_fence_before();
                    mbar_arrive(smem_u32(&bar_dy_empty[buf]));
#pragma unroll
                    for (int r = 0; r < kRT; ++r) {
                        m1acc[r] = fmaf(w_s[buf][r], y[r], m1acc[r]);
                        y[r] *= a1r[r];
                    }
                    if (p.N >= 3) {
                        butterfly_reduce64(y, lane);
                        red_s[q][butterfly_col(lane, 0)] = y[0];
                        red_s[q][butterfly_col(lane, 1)] = y[1];
                        named_sync_epi();
                        if (et < kRT) {
                            const float cm = red_s[0][et] + red_s[1][et] + red_s[2][et] + red_s[3][et];
                            Pc[m * kRT + et] = cm;
                        }
                        named_sync_epi();
                    }
                    if (et == 0) TC_TRACE(7, (int)tp);
                }
            }
            t = t0 + nsl;
            if (!ok) break;
            // ---- unit end: M^(1) partial from registers, M^(N) partial from TMEM
            float* py = p.P_Y1 + ((int64_t)u * kBI + row) * kRT;
#pragma unroll
            for (int r = 0; r < kRT; r += 4)
                *reinterpret_cast<float4*>(py + r) = make_float4(m1acc[r], m1acc[r + 1], m1acc[r + 2], m1acc[r + 3]);
            if (!(ok = epi_wait(smem_u32(&bar_dz_full), (uint32_t)(v & 1)))) break;
            tc_fence_after();
            const int c0 = U.kg * kChunksPerGroup;
            const int c1 = (int)imin(c0 + kChunksPerGroup, (p.sN + kKC - 1) / kKC);
            for (int c = c0; c < c1; ++c) {
                float z[kRT];
                const uint32_t ta = t_dz + (c - c0) * kRT + ((uint32_t)(q * 32) << 16);
#pragma unroll
                for (int j = 0; j < kRT; j += 16) tmem_ld16(ta + j, z + j);
                float* pz = p.P_Z + ((int64_t)u * (kChunksPerGroup * kKC) + (c - c0) * kKC + row) * kRT;
#pragma unroll
                for (int r = 0; r < kRT; r += 4)
                    *reinterpret_cast<float4*>(pz + r) = make_float4(z[r], z[r + 1], z[r + 2], z[r + 3]);
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&bar_dz_empty));
        }
        (void)et;
    }
    // ---- teardown: every role has left its loop (all waits are bounded)
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------ preparation
// X -> bf16 planes [2][s1][mid][sNp] (hi, lo), zero in the padding columns.
// Four consecutive columns per thread, 8-byte stores; FP32 arithmetic for FP32
// input (x - hi is exact), FP64 only for FP64 input.
template <typename TX>
__device__ __forceinline__ void split1(TX x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    if constexpr (sizeof(TX) == 4) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    } else {
        hi = __double2bfloat16(x);
        lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    }
}

template <typename TX>
__global__ void split_x_kernel(const TX* __restrict__ X, __nv_bfloat16* __restrict__ planes, int64_t rows, int64_t sN,
                               int64_t sNp) {
    const int64_t q4 = sNp / 4;  // sNp is a multiple of 8
    const int64_t total4 = rows * q4, total = rows * sNp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rr = e / q4, k = (e - rr * q4) * 4;
        const TX* xr = X + rr * sN;
        __nv_bfloat16 hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split1<TX>(k + u < sN ? xr[k + u] : (TX)0, hi[u], lo[u]);
        uint2 vh, vl;
        vh.x = (uint32_t)__bfloat16_as_ushort(hi[0]) | ((uint32_t)__bfloat16_as_ushort(hi[1]) << 16);
        vh.y = (uint32_t)__bfloat16_as_ushort(hi[2]) | ((uint32_t)__bfloat16_as_ushort(hi[3]) << 16);
        vl.x = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
        vl.y = (uint32_t)__bfloat16_as_ushort(lo[2]) | ((uint32_t)__bfloat16_as_ushort(lo[3]) << 16);
        *reinterpret_cast<uint2*>(planes + rr * sNp + k) = vh;
        *reinterpret_cast<uint2*>(planes + total + rr * sNp + k) = vl;
    }
}

// B_Y planes [128][sNp]: rows 0..63 = hi of A^(N)[:, r0 + r]^T, rows 64..127 = lo.
__global__ void split_by_kernel(const double* __restrict__ AN, int R, int r0, int64_t sN, int64_t sNp,
                                __nv_bfloat16* __restrict__ BY) {
    const int64_t total = (int64_t)kRT * sNp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / sNp);
        const int64_t k = e % sNp;
        const double a = (k < sN && r0 + r < R) ? AN[k * R + r0 + r] : 0.0;
        const __nv_bfloat16 hi = __double2bfloat16(a);
        BY[e] = hi;
        BY[total + e] = __double2bfloat16(a - (double)__bfloat162float(hi));
    }
}

// FP32 copy of rows of a factor for columns r0..r0+63 (zero padded): out[rows][64]
__global__ void factor_f32_kernel(const double* __restrict__ A, int R, int r0, int64_t rows, float* __restrict__ out) {
    const int64_t total = rows * kRT;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kRT;
        const int r = (int)(e % kRT);
        out[e] = (r0 + r < R) ? (float)A[i * R + r0 + r] : 0.0f;
    }
}

// Reduce the unit partials into the FP64 outputs (fixed order), columns
// r0..r0+Rt-1.  Block = 8 output rows of one mode; thread (row t/32, columns
// 2*(t%32) + {0,1}); the partials are visited in a fixed order with coalesced
// 256-byte row loads.
constexpr int kFinRows = 8;
__global__ void finalize_kernel(Params p, Ptrs<double> M, Ptrs<const double> A, int R, int r0, int Rt,
                                int64_t sNfull, unsigned mode_mask) {
    const int N = p.N;
    const int n = blockIdx.y;
    if (!(mode_mask & (1u << n))) return;
    const int64_t sn = n == 0 ? p.s1 : (n == N - 1 ? p.sN : p.middim[n]);
    const int64_t i = (int64_t)blockIdx.x * kFinRows + (threadIdx.x >> 5);
    if (i >= sn) return;
    const int c0 = 2 * (threadIdx.x & 31);
    double acc0 = 0.0, acc1 = 0.0;
    if (n == 0) {
        const int b = (int)(i / kBI);
        for (int kg = 0; kg < p.nkg; ++kg)
            for (int j = 0; j < p.nsplit; ++j) {
                const int u = (b * p.nkg + kg) * p.nsplit + j;
                const float2 v = *reinterpret_cast<const float2*>(p.P_Y1 + ((int64_t)u * kBI + (i % kBI)) * kRT + c0);
                acc0 += v.x;
                acc1 += v.y;
            }
    } else if (n == N - 1) {
        const int kg = (int)(i / (kChunksPerGroup * kKC));
        for (int b = 0; b < p.nib; ++b)
            for (int j = 0; j < p.nsplit; ++j) {
                const int u = (b * p.nkg + kg) * p.nsplit + j;
                const float2 v = *reinterpret_cast<const float2*>(
                    p.P_Z + ((int64_t)u * (kChunksPerGroup * kKC) + (i % (kChunksPerGroup * kKC))) * kRT + c0);
                acc0 += v.x;
                acc1 += v.y;
            }
    } else {
        // middle mode n: sum over the slices m whose index in mode n is i
        const int64_t sub = p.mid / p.middim[n];
        for (int64_t t = 0; t < sub; ++t) {
            int64_t rem = t, m = 0, mult = 1;
            double lo0 = 1.0, lo1 = 1.0;
            for (int q = N - 2; q >= 1; --q) {
                int64_t iq;
                if (q == n) {
                    iq = i;
                } else {
                    iq = rem % p.middim[q];
                    rem /= p.middim[q];
                    if (c0 < Rt) lo0 *= A.p[q][iq * R + r0 + c0];
                    if (c0 + 1 < Rt) lo1 *= A.p[q][iq * R + r0 + c0 + 1];
                }
                m += iq * mult;
                mult *= p.middim[q];
            }
            double cs0 = 0.0, cs1 = 0.0;
            for (int bk = 0; bk < p.nib * p.nkg; ++bk) {
                const float2 v = *reinterpret_cast<const float2*>(p.P_c + ((int64_t)bk * p.mid + m) * kRT + c0);
                cs0 += v.x;
                cs1 += v.y;
            }
            acc0 += cs0 * lo0;
            acc1 += cs1 * lo1;
        }
    }
    if (c0 < Rt) M.p[n][i * R + r0 + c0] = acc0;
    if (c0 + 1 < Rt) M.p[n][i * R + r0 + c0 + 1] = acc1;
    (void)sNfull;
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        cudaGetLastError();
    });
    return fn;
}

static int64_t pad8(int64_t v) { return (v + 7) / 8 * 8; }
#ifdef CPGN_TC_TRACE
long long* tc_trace_ptr = nullptr;
#endif

}  // namespace tc

using namespace tc;

size_t split_cache_bytes(const cp_desc* d) {
    int64_t rows = 1;
    for (int n = 0; n + 1 < d->order; ++n) rows *= d->dims[n];
    return (size_t)(2 * rows * pad8(d->dims[d->order - 1]) * sizeof(__nv_bfloat16));
}

int tc_launch_count(const SplitCache& c, const cp_desc* d, const Shape& s) {
    const bool hit = c.planes && c.key_ptr != nullptr && c.key_version == d->x_version && c.key_total == s.total &&
                     c.key_dtype == (int)d->x_dtype;
    const int tiles = (s.R + kRT - 1) / kRT;
    return (hit ? 0 : 1) + tiles * (2 + (s.N - 2) + 2);
}

void split_cache_free(SplitCache& c) {
    if (c.planes) cudaFree(c.planes);
    if (c.fac) cudaFree(c.fac);
    c = SplitCache{};
}

static cp_status ensure_buf(void*& p, size_t& cur, size_t need) {
    if (cur >= need) return CP_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cur = 0;
    if (cudaMalloc(&p, need) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_NOMEM;
    }
    cur = need;
    return CP_OK;
}

// Launch geometry of one tensor-core MTTKRP over the shape.
struct TcGeom {
    int nib, nkg, nsplit, nunits, grid;
};
static TcGeom tc_geom(const Shape& s, int sms) {
    TcGeom g;
    g.nib = (int)((s.dims[0] + kBI - 1) / kBI);
    const int64_t chunks = (s.dims[s.N - 1] + kKC - 1) / kKC;
    g.nkg = (int)((chunks + kChunksPerGroup - 1) / kChunksPerGroup);
    const int pairs = g.nib * g.nkg;
    g.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(s.mid, (sms + pairs - 1) / pairs));
    g.nunits = pairs * g.nsplit;
    g.grid = std::min(g.nunits, sms);
    return g;
}

int64_t tc_row_pitch(int64_t sN) { return pad8(sN); }

// bf16 planes of X, cached by pointer / size / version.
static cp_status tc_split_x(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, int sms,
                            cudaStream_t st) {
    const int N = s.N;
    const int64_t sN = s.dims[N - 1], sNp = pad8(sN), rows = s.dims[0] * s.mid;
    const size_t pbytes = (size_t)2 * rows * sNp * sizeof(__nv_bfloat16);
    const bool hit = c.planes && c.key_ptr == X && c.key_version == d->x_version && c.key_total == s.total &&
                     c.key_dtype == (int)d->x_dtype && c.bytes >= pbytes;
    if (hit) return CP_OK;
    if (c.bytes < pbytes) {
        if (c.planes) cudaFree(c.planes);
        c.planes = nullptr;
        c.bytes = 0;
        if (cudaMalloc(&c.planes, pbytes) != cudaSuccess) {
            cudaGetLastError();
            return CP_ERR_NOMEM;
        }
        c.bytes = pbytes;
    }
    const int blocks = sms * 8;
    if (d->x_dtype == CP_F32)
        split_x_kernel<float><<<blocks, 256, 0, st>>>((const float*)X, (__nv_bfloat16*)c.planes, rows, sN, sNp);
    else
        split_x_kernel<double><<<blocks, 256, 0, st>>>((const double*)X, (__nv_bfloat16*)c.planes, rows, sN, sNp);
    c.key_ptr = X;
    c.key_version = d->x_version;
    c.key_total = s.total;
    c.key_dtype = (int)d->x_dtype;
    return CP_OK;
}

// MTTKRP on planes [2][s1][mid][sNp] that are already in device memory.
static cp_status tc_main(SplitCache& c, const void* planes, const Shape& s, Ptrs<const double> A, Ptrs<double> M,
                         unsigned mode_mask, int* status, cudaStream_t st) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return CP_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int N = s.N, R = s.R;
    const int64_t s1 = s.dims[0], sN = s.dims[N - 1], mid = s.mid, sNp = pad8(sN);
    // ---- workspace: factor planes and unit partials
    const TcGeom g = tc_geom(s, sms);
    int64_t midrows = 0;
    Params p{};
    p.N = N;
    p.s1 = s1;
    p.mid = mid;
    p.sN = sN;
    p.nib = g.nib;
    p.nkg = g.nkg;
    p.nsplit = g.nsplit;
    p.nunits = g.nunits;
    for (int q = 1; q + 1 < N; ++q) {
        p.midoff[q] = midrows;
        p.middim[q] = s.dims[q];
        midrows += s.dims[q];
    }
    const size_t by_b = (size_t)2 * kRT * sNp * sizeof(__nv_bfloat16);
    const size_t a1_b = (size_t)s1 * kRT * sizeof(float);
    const size_t mid_b = (size_t)std::max<int64_t>(midrows, 1) * kRT * sizeof(float);
    const size_t py_b = (size_t)g.nunits * kBI * kRT * sizeof(float);
    const size_t pz_b = (size_t)g.nunits * kChunksPerGroup * kKC * kRT * sizeof(float);
    const size_t pc_b = (size_t)g.nib * g.nkg * mid * kRT * sizeof(float);
    const size_t off_a1 = (by_b + 255) / 256 * 256;
    const size_t off_mid = off_a1 + (a1_b + 255) / 256 * 256;
    const size_t off_py = off_mid + (mid_b + 255) / 256 * 256;
    const size_t off_pz = off_py + (py_b + 255) / 256 * 256;
    const size_t off_pc = off_pz + (pz_b + 255) / 256 * 256;
    const size_t total_b = off_pc + pc_b;
    if (ensure_buf(c.fac, c.fac_bytes, total_b) != CP_OK) return CP_ERR_NOMEM;
    unsigned char* wb = (unsigned char*)c.fac;
    __nv_bfloat16* BY = (__nv_bfloat16*)wb;
    p.A1f = (const float*)(wb + off_a1);
    p.midf = (const float*)(wb + off_mid);
    p.P_Y1 = (float*)(wb + off_py);
    p.P_Z = (float*)(wb + off_pz);
    p.P_c = (float*)(wb + off_pc);
    p.status = status;
    p.trace = nullptr;
#ifdef CPGN_TC_TRACE
    {
        static long long* trace_buf = nullptr;
        if (!trace_buf) cudaMalloc(&trace_buf, 8 * 1024 * sizeof(long long));
        cudaMemsetAsync(trace_buf, 0, 8 * 1024 * sizeof(long long), st);
        p.trace = trace_buf;
        tc_trace_ptr = trace_buf;
    }
#endif
    // ---- tensor maps
    CUtensorMap tmX, tmBY;
    {
        cuuint64_t dims[4] = {(cuuint64_t)sNp, (cuuint64_t)mid, (cuuint64_t)s1, 2};
        cuuint64_t strides[3] = {(cuuint64_t)(sNp * 2), (cuuint64_t)(mid * sNp * 2), (cuuint64_t)(s1 * mid * sNp * 2)};
        cuuint32_t box[4] = {64, 1, (cuuint32_t)kBI, 2};
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(planes), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return CP_ERR_UNSUPPORTED;
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)sNp, 128};
        cuuint64_t strides[1] = {(cuuint64_t)(sNp * 2)};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t es[2] = {1, 1};
        if (enc(&tmBY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, BY, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return CP_ERR_UNSUPPORTED;
    }
    static bool attr_set[64] = {};
    if (dev >= 64 || !attr_set[dev]) {
        if (cudaFuncSetAttribute(mttkrp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem) !=
            cudaSuccess) {
            cudaGetLastError();
            return CP_ERR_UNSUPPORTED;
        }
        if (dev < 64) attr_set[dev] = true;
    }
    for (int r0 = 0; r0 < R; r0 += kRT) {
        const int Rt = std::min(kRT, R - r0);
        p.R = Rt;
        split_by_kernel<<<sms, 256, 0, st>>>(A.p[N - 1], R, r0, sN, sNp, BY);
        factor_f32_kernel<<<sms, 256, 0, st>>>(A.p[0], R, r0, s1, (float*)p.A1f);
        for (int q = 1; q + 1 < N; ++q)
            factor_f32_kernel<<<64, 256, 0, st>>>(A.p[q], R, r0, s.dims[q], (float*)p.midf + p.midoff[q] * kRT);
        mttkrp_tc_kernel<<<g.grid, kThreads, kDynSmem, st>>>(tmX, tmBY, p);
        if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
        int64_t mx = 0;
        for (int n = 0; n < N; ++n) mx = std::max<int64_t>(mx, s.dims[n] * Rt);
        int64_t mrows = 0;
        for (int n = 0; n < N; ++n) mrows = std::max<int64_t>(mrows, s.dims[n]);
        dim3 fg((unsigned)((mrows + kFinRows - 1) / kFinRows), N);
        finalize_kernel<<<fg, 32 * kFinRows, 0, st>>>(p, M, A, R, r0, Rt, sN, mode_mask);
        if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
    }
    return CP_OK;
}

static cp_status tc_run(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                        Ptrs<double> M, unsigned mode_mask, int* status, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cp_status r = tc_split_x(c, d, s, X, sms, st);
    if (r != CP_OK) return r;
    return tc_main(c, c.planes, s, A, M, mode_mask, status, st);
}

cp_status tc_mttkrp_all(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                        Ptrs<double> M, int* status, cudaStream_t st) {
    return tc_run(c, d, s, X, A, M, (1u << s.N) - 1u, status, st);
}

cp_status tc_mttkrp_mode(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                         Ptrs<double> M, int n, int* status, cudaStream_t st) {
    return tc_run(c, d, s, X, A, M, 1u << n, status, st);
}

cp_status tc_mttkrp_planes(SplitCache& c, const void* planes, const Shape& s, Ptrs<const double> A, Ptrs<double> M,
                           int* status, cudaStream_t st) {
    return tc_main(c, planes, s, A, M, (1u << s.N) - 1u, status, st);
}

}  // namespace cpgn

#ifdef CPGN_TC_TRACE
// trace builds only: device pointer of the last trace buffer (8 x 1024 int64)
extern "C" int cpgn_tc_trace_copy(long long* host) {
    if (!cpgn::tc::tc_trace_ptr) return 1;
    return cudaMemcpy(host, cpgn::tc::tc_trace_ptr, 8 * 1024 * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess;
}
#endif
