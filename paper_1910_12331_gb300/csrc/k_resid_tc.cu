// k_resid_tc.cu -- the residual tensor E = X - [[A^(1), ..., A^(N)]] with the
// reconstruction on tcgen05 tensor cores (sm_103a), written as bf16 high/low
// planes (PlaneTiling) for the tensor-core MTTKRP and/or in FP64, with
// sum E^2 and sum X^2.  Used for R <= 64; larger ranks take the CUDA-core
// kernel of k_resid.cu.
//
// Why: the gradient G^(n) = -E_(n) P^(n) of Eq. (2.3) needs E to far better
// than FP32's 2^-24 when E is small; see k_resid.cu.
//
// Arithmetic: error-free splitting of a matrix product into slice products on
// fixed grids (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), with bf16 slices and the tensor
// core's FP32 accumulation:
//   X is viewed as the (s_1 mid) x s_N matrix of its rows (i, m), m indexing
//   the middle modes, and [[A]][(i, m), k] = sum_r u_r v_kr with
//   u_r = a^(1)_ir w_m[r] (w_m: the product of the middle factors' rows) and
//   v_kr = a^(N)_kr.  Row (i, m) of u is scaled by the power of two
//   sigma >= max_r |u_r|, row k of v by tau_k >= max_r |v_kr|, and every scaled
//   value is cut into five pieces on the grids 2^-8, 2^-16, ..., 2^-40 (round
//   to nearest on each grid; the remainder goes on to the next).  A piece on
//   grid 2^-8s is an integer of at most 8 significant bits times 2^-8s, exact
//   in bf16; |piece s| <= 2^(9 - 8s) for s >= 2.  The product of pieces s and t
//   is an integer of at most 16 bits on the grid 2^-8(s+t).  The piece pairs
//   with s + t = L <= 6 (15 pairs) are accumulated in four TMEM accumulators:
//     L = 2, 3, 4, one each: every sum of a level over r < 64 stays below 2^23
//       units of its grid, so the FP32 accumulation is exact;
//     L = 5 and 6 together: magnitudes below 2^-16 R, so each of the at most
//       36 accumulating MMAs rounds by at most 2^-41 sigma tau.
//   The pairs with s + t >= 7 and the remainders beyond the fifth piece are
//   below 2^-39.5 per rank term.  The epilogue forms (h, l) = the exact
//   double-float sum of levels 2 and 3 plus the FP32 sum of the rest (rounding
//   below 2^-40 R), scales back by sigma tau (powers of two) and subtracts from
//   x: error below 2^-38.5 R sigma tau in all.
//
// Kernel: persistent, one CTA per SM, 20 warps.  A run is 128 consecutive rows
// (i, m); a step is one 64-column chunk c of k (the last chunk's MMAs are
// only as wide as its columns, rounded up to 16).
//   warp 0      producer: the step's pieces of v (5 x 8 KB, one bulk copy,
//               precomputed once per call, pre-swizzled), its tau_k and (FP32
//               X, s_N a multiple of 4) the 128 x 64 X tile by two 2-D tensor
//               copies, into one of two slots.
//   warp 1      TMEM allocator and MMA issuer (one thread): 15 piece pairs x
//               K/16 MMAs (M = 128, N = 64) into the four accumulators of one
//               of two TMEM buffers (4 x 64 columns each).
//   warps 4-19  workers: build the pieces of u for a run (5 x 16 KB), then per
//               step drain the four accumulators (lane = row, 16 columns per
//               warp in two groups of 8), form E and write it.
// Every mbarrier wait is bounded (CP_ERR_TIMEOUT, CTA abort flag, drain).
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "kernels.hpp"
#include "tc.hpp"
#include "tc_ptx.cuh"

namespace cpgn {

namespace rtc {

using namespace tcx;

constexpr int kSlices = 5;                         // pieces per value
constexpr int kAcc = 4;                            // accumulators: L = 2, 3, 4 and L = 5 + 6
constexpr int kBI = 128;                           // rows (i, m) of a run (M)
constexpr int kKC = 64;                            // columns k of a step (N, at most)
constexpr int kRT = 64;                            // rank columns (K), zero padded
constexpr uint32_t kASlice = kBI * 128;            // 128 rows x 64 bf16, K-major, 128-byte swizzle
constexpr uint32_t kBSlice = kKC * 128;            // 64 rows x 64 bf16
constexpr uint32_t kABytes = kSlices * kASlice;    // 80 KB
constexpr uint32_t kBBytes = kSlices * kBSlice;    // 40 KB per step
constexpr uint32_t kXBox = kBI * 32 * 4;           // 128 rows x 32 FP32 of X, 128-byte swizzle (one tensor copy)
constexpr uint32_t kXTile = 2 * kXBox;             // a step's 64 columns
constexpr uint32_t kPayload = kABytes + 2 * kBBytes + 2 * kXTile;
constexpr int kWorkWarps = 16;
constexpr int kWork = 32 * kWorkWarps;
constexpr int kThreads = 128 + kWork;
constexpr uint32_t kTmemCols = 512;                // 2 buffers x 4 accumulators x 64 columns
constexpr uint32_t kDBuf = kAcc * kKC;             // TMEM columns of one buffer

// Accumulator of level L = s + t.
__host__ __device__ constexpr int acc_of_level(int L) { return L <= 4 ? L - 2 : 3; }

struct Params {
    int N, R;
    int64_t s1, mid, sN;
    int64_t rows;        // s1 * mid rows (i, m), row f = i * mid + m
    int64_t runs;        // ceil(rows / 128)
    int nck;             // 64-column chunks of k
    PlaneTiling pt;
    const void* X;
    int x_f64;
    int x_tma;           // X tiles come by tensor copy (FP32, s_N % 4 == 0), else the workers load X
    const float2* A1df;  // [s1][64] (hi, lo) of A^(1), zero padded
    const float2* Wdf;   // [mid][64] (hi, lo) of w_m, zero padded
    const unsigned char* Vsl;  // [nck][5][64][128 B] pieces of a^(N)_kr / tau_k, swizzled
    const float* tau;    // [nck * 64]
    __nv_bfloat16* planes;  // bf16 planes of E (PlaneTiling), or null
    double* E64;            // E in FP64, C-contiguous like X, or null
    DevStats* stats;
    int* status;
};

struct SmemCtl {
    uint64_t a_full, a_empty, b_full[2], b_empty[2], d_full[2], d_empty[2], x_full[2], x_empty[2], drain;
    uint32_t tmem_base;
    int abort_flag;
    float sig[2][kBI];      // sigma of each row of a run, by run parity
    double red[2][kWorkWarps];
    alignas(16) float tau_s[2][kKC];  // tau_k of a step, with its X tile
};
constexpr uint32_t kDynSmem = kPayload + (uint32_t)sizeof(SmemCtl);
static_assert(kDynSmem <= 227 * 1024, "shared memory above the per-block limit");

// Smallest power of two >= v for finite v > 0 (FP32 / FP64 bit patterns).
__host__ __device__ __forceinline__ float pow2_ceil_f(float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    u = (u + 0x007fffffu) & 0xff800000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}
__device__ __forceinline__ double pow2_ceil_d(double v) {
    const unsigned long long u = (__double_as_longlong(v) + 0x000fffffffffffffull) & 0xfff0000000000000ull;
    return __longlong_as_double((long long)u);
}
// 1 / p for a power of two p in the normal range (exact)
__device__ __forceinline__ float pow2_inv(float p) {
    return __uint_as_float((uint32_t)(254u << 23) - __float_as_uint(p));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}
// Byte offset of element (row, col) in a K-major operand tile with rows of
// 64 bf16 (128 bytes) and the 128-byte swizzle: 16-byte piece j of row r is
// stored at piece j ^ (r mod 8); 8-row groups are 1024 bytes apart.
__host__ __device__ __forceinline__ uint32_t sw128(int row, int col) {
    return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
           (uint32_t)((((col >> 3) ^ (row & 7)) << 4) | ((col & 7) << 1));
}
__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Pieces of one scaled double-float value (|h + l| <= 1) on the grids 2^-8s.
__device__ __forceinline__ void cut5(float h, float l, float* pc) {
    pc[0] = rintf(h * 0x1p8f) * 0x1p-8f;
    h -= pc[0];
    pc[1] = rintf(h * 0x1p16f) * 0x1p-16f;
    h -= pc[1];
    pc[2] = rintf(h * 0x1p24f) * 0x1p-24f;
    h -= pc[2];
    float hh, ll;
    two_sum(h, l, hh, ll);  // the low part joins below 2^-24
    pc[3] = rintf(hh * 0x1p32f) * 0x1p-32f;
    hh = (hh - pc[3]) + ll;
    pc[4] = rintf(hh * 0x1p40f) * 0x1p-40f;
}

__global__ void __launch_bounds__(kThreads, 1) recon_tc_kernel(const __grid_constant__ CUtensorMap tmX, Params p) {
    extern __shared__ __align__(1024) unsigned char dsmem[];
    if (smem_u32(dsmem) & 1023u) {
        if (threadIdx.x == 0) atomicCAS(p.status, 0, CP_ERR_UNSUPPORTED);
        return;
    }
    SmemCtl& C = *reinterpret_cast<SmemCtl*>(dsmem + kPayload);
    volatile int* abort_s = &C.abort_flag;
    const uint32_t sA = smem_u32(dsmem), sB = sA + kABytes, sX = sB + 2 * kBBytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&C.a_full), kWork);
        mbar_init(smem_u32(&C.a_empty), 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&C.b_full[s]), 1);
            mbar_init(smem_u32(&C.b_empty[s]), 1);
            mbar_init(smem_u32(&C.d_full[s]), 1);
            mbar_init(smem_u32(&C.d_empty[s]), kWork);
            mbar_init(smem_u32(&C.x_full[s]), 1);
            mbar_init(smem_u32(&C.x_empty[s]), kWork);
        }
        mbar_init(smem_u32(&C.drain), 1);
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&C.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = C.tmem_base;
    const int64_t J0 = (int64_t)blockIdx.x * p.runs / gridDim.x;
    const int64_t J1 = (int64_t)(blockIdx.x + 1) * p.runs / gridDim.x;
    const int ksteps = (p.R + 15) / 16;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int64_t tt = 0;
            bool ok = true;
            for (int64_t j = J0; j < J1 && ok; ++j) {
                for (int c = 0; c < p.nck; ++c, ++tt) {
                    const int slot = (int)(tt & 1);
                    const uint32_t pe = (uint32_t)(((tt >> 1) & 1) ^ 1);
                    if (!(ok = mbar_wait(smem_u32(&C.b_empty[slot]), pe, abort_s, p.status))) break;
                    const uint32_t fb = smem_u32(&C.b_full[slot]);
                    mbar_expect_tx(fb, kBBytes);
                    bulk_load(sB + slot * kBBytes, p.Vsl + (size_t)c * kBBytes, kBBytes, fb);
                    // the step's tau_k and (tensor copy) X tile, released by the workers; a box
                    // that starts at or beyond s_N is not loaded (its columns are masked)
                    if (!(ok = mbar_wait(smem_u32(&C.x_empty[slot]), pe, abort_s, p.status))) break;
                    const uint32_t fx = smem_u32(&C.x_full[slot]);
                    const int nbox = p.x_tma ? ((int64_t)c * kKC + 32 < p.sN ? 2 : 1) : 0;
                    mbar_expect_tx(fx, (uint32_t)nbox * kXBox + kKC * 4u);
                    bulk_load(smem_u32(&C.tau_s[slot][0]), p.tau + (size_t)c * kKC, kKC * 4u, fx);
                    for (int hb = 0; hb < nbox; ++hb)
                        tma_load_2d(sX + slot * kXTile + hb * kXBox, &tmX, c * kKC + hb * 32, (int)(j * kBI), fx);
                }
            }
            for (int64_t k = (tt > 2 ? tt - 2 : 0); k < tt; ++k) {
                mbar_drain(smem_u32(&C.b_full[k & 1]), (uint32_t)((k >> 1) & 1), p.status);
                mbar_drain(smem_u32(&C.x_full[k & 1]), (uint32_t)((k >> 1) & 1), p.status);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int64_t tt = 0;
            int jr = 0;
            bool ok = true;
            for (int64_t j = J0; j < J1 && ok; ++j, ++jr) {
                if (!(ok = mbar_wait(smem_u32(&C.a_full), (uint32_t)(jr & 1), abort_s, p.status))) break;
                for (int c = 0; c < p.nck; ++c, ++tt) {
                    const int slot = (int)(tt & 1);
                    const uint32_t ph = (uint32_t)((tt >> 1) & 1);
                    if (!(ok = mbar_wait(smem_u32(&C.d_empty[slot]), ph ^ 1, abort_s, p.status))) break;
                    if (!(ok = mbar_wait(smem_u32(&C.b_full[slot]), ph, abort_s, p.status))) break;
                    tc_fence_after();
                    const int64_t left = p.sN - (int64_t)c * kKC;
                    const int nstep = left >= kKC ? kKC : (int)((left + 15) / 16 * 16);
                    const uint32_t id = idesc_bf16(nstep, false, false);
                    const uint32_t dbase = tmem + slot * kDBuf;
                    const uint64_t a0 = sdesc(sA, 16, 1024), b0 = sdesc(sB + slot * kBBytes, 16, 1024);
                    // K-step outermost, then level, then piece pair (the order of the
                    // reconstruction's bit-stability tests)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        if (ks >= ksteps) break;
#pragma unroll
                        for (int L = 2; L <= kSlices + 1; ++L) {
#pragma unroll
                            for (int sp = 1; sp <= kSlices; ++sp) {
                                const int t = L - sp;
                                if (t < 1 || t > kSlices) continue;
                                const int a = acc_of_level(L);
                                // the first MMA into an accumulator in a step overwrites it
                                const bool first = ks == 0 && sp == 1 && (a < 3 || L == 5);
                                const uint64_t ao = (uint64_t)(((sp - 1) * kASlice + ks * 32) >> 4);
                                const uint64_t bo = (uint64_t)(((t - 1) * kBSlice + ks * 32) >> 4);
                                tc_mma(dbase + a * kKC, a0 + ao, b0 + bo, id, first ? 0 : 1);
                            }
                        }
                    }
                    tc_commit(smem_u32(&C.b_empty[slot]));
                    tc_commit(smem_u32(&C.d_full[slot]));
                    if (c == p.nck - 1) tc_commit(smem_u32(&C.a_empty));
                }
            }
            tc_commit(smem_u32(&C.drain));
            mbar_drain(smem_u32(&C.drain), 0, p.status);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ------------------------------------------------------------ workers
        const int wk = warp - 4;
        const int q = warp & 3;              // TMEM lane quadrant of this warp
        const int cg = wk >> 2;              // 16-column group of a step
        const int row = q * 32 + lane;       // TMEM lane = row of the run
        const int et = wk * 32 + lane;       // 0 .. kWork - 1
        bool ok = true;
        float eh = 0.f, el = 0.f, xh = 0.f, xl = 0.f;

        // pieces of u for run j: eight lanes per row (8 rank columns = one 16-byte
        // piece each), four rows per warp and pass, two passes
        auto build = [&](int64_t j, int jr) {
            if (ok) ok = mbar_wait(smem_u32(&C.a_empty), (uint32_t)((jr & 1) ^ 1), abort_s, p.status);
            if (!ok) return;
            const int c8 = lane & 7;
#pragma unroll 1
            for (int pass = 0; pass < kBI / (4 * kWorkWarps); ++pass) {
                const int brow = pass * (4 * kWorkWarps) + wk * 4 + (lane >> 3);
                const int64_t f = j * kBI + brow;
                float2 v[8];
                float mx = 0.f;
                if (f < p.rows) {
                    const int64_t i = f / p.mid, m = f - i * p.mid;
                    const float4* asrc = reinterpret_cast<const float4*>(p.A1df + (size_t)i * kRT + c8 * 8);
                    const float4* wsrc = reinterpret_cast<const float4*>(p.Wdf + (size_t)m * kRT + c8 * 8);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 a4 = __ldg(asrc + u), w4 = __ldg(wsrc + u);
                        v[2 * u] = df_mul(make_float2(a4.x, a4.y), make_float2(w4.x, w4.y));
                        v[2 * u + 1] = df_mul(make_float2(a4.z, a4.w), make_float2(w4.z, w4.w));
                        mx = fmaxf(mx, fmaxf(fabsf(v[2 * u].x), fabsf(v[2 * u + 1].x)));
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = make_float2(0.f, 0.f);
                }
                // sigma >= max_r |u_r| over the row's eight lanes (hi parts; the low
                // parts stay inside the 2^-24 slack of the first piece)
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
                const float sg = pow2_ceil_f(fmaxf(mx, 0x1p-100f));
                if (c8 == 0) C.sig[jr & 1][brow] = sg;
                const float inv = pow2_inv(sg);
                float pc[8][kSlices];
#pragma unroll
                for (int u = 0; u < 8; ++u) cut5(v[u].x * inv, v[u].y * inv, pc[u]);
                const uint32_t off = sw128(brow, c8 * 8);
#pragma unroll
                for (int sl = 0; sl < kSlices; ++sl) {
                    uint4 q4;
                    q4.x = bf2(pc[0][sl], pc[1][sl]);
                    q4.y = bf2(pc[2][sl], pc[3][sl]);
                    q4.z = bf2(pc[4][sl], pc[5][sl]);
                    q4.w = bf2(pc[6][sl], pc[7][sl]);
                    *reinterpret_cast<uint4*>(dsmem + sl * kASlice + off) = q4;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&C.a_full));
        };

        int64_t tt = 0;
        int jr = 0;
        if (J0 < J1) build(J0, 0);
        for (int64_t j = J0; j < J1; ++j, ++jr) {
            const int64_t f = j * kBI + row;  // this thread's row (i, m) of X
            const bool live = f < p.rows;
            const int64_t i = live ? f / p.mid : 0;
            const int64_t m = live ? f - i * p.mid : 0;
            const int b = (int)(i >> 7), r = (int)(i & 127);
            const int rows_b = p.pt.rows(b);
            for (int c = 0; c < p.nck; ++c, ++tt) {
                // the next run's pieces of u go in while this run's last step drains
                if (c == p.nck - 1 && j + 1 < J1) build(j + 1, jr + 1);
                if (!ok) continue;
                const int slot = (int)(tt & 1);
                const uint32_t ph = (uint32_t)((tt >> 1) & 1);
                if (!(ok = mbar_wait(smem_u32(&C.x_full[slot]), ph, abort_s, p.status))) continue;
                if (!(ok = mbar_wait(smem_u32(&C.d_full[slot]), ph, abort_s, p.status))) continue;
                tc_fence_after();
                // sigma of this run: written by another worker before its a_full arrival,
                // which the MMAs behind d_full waited for
                const float sg = C.sig[jr & 1][row];
                const int64_t tb = live && p.planes ? p.pt.tile(b, c, m) : 0;
                float e2 = 0.f, x2 = 0.f;
#pragma unroll 1
                for (int sgp = 0; sgp < 2; ++sgp) {
                    const int cc = cg * 16 + sgp * 8;  // first column of this group inside the chunk
                    const int64_t k0 = (int64_t)c * kKC + cc;
                    uint32_t d0[8], d1[8], d2[8], d3[8];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + slot * kDBuf + cc;
                    tmem_ld8x4_wait(ta, ta + kKC, ta + 2 * kKC, ta + 3 * kKC, d0, d1, d2, d3);
                    float it[8], xv[8];
                    {
                        const float4 t0 = *reinterpret_cast<const float4*>(&C.tau_s[slot][cc]);
                        const float4 t1 = *reinterpret_cast<const float4*>(&C.tau_s[slot][cc + 4]);
                        it[0] = t0.x, it[1] = t0.y, it[2] = t0.z, it[3] = t0.w;
                        it[4] = t1.x, it[5] = t1.y, it[6] = t1.z, it[7] = t1.w;
                    }
                    const bool full = live && k0 + 8 <= p.sN;  // every column of the group is in X
                    if (p.x_tma) {
                        // box cc / 32, 128-byte rows; 16-byte piece j of row r at piece j ^ (r mod 8)
                        const unsigned char* xr = dsmem + (kABytes + 2 * kBBytes) + slot * kXTile +
                                                  (cc >> 5) * kXBox + row * 128;
                        const int j0 = (cc & 31) >> 2;
                        const float4 x0 = *reinterpret_cast<const float4*>(xr + ((j0 ^ (row & 7)) << 4));
                        const float4 x1 = *reinterpret_cast<const float4*>(xr + (((j0 + 1) ^ (row & 7)) << 4));
                        xv[0] = x0.x, xv[1] = x0.y, xv[2] = x0.z, xv[3] = x0.w;
                        xv[4] = x1.x, xv[5] = x1.y, xv[6] = x1.z, xv[7] = x1.w;
                    } else if (!p.x_f64) {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            xv[u] = (live && k0 + u < p.sN) ? __ldg(reinterpret_cast<const float*>(p.X) + f * p.sN + k0 + u)
                                                            : 0.f;
                    }
                    if (sgp == 1) {  // every read of this step's slot is done
                        mbar_arrive(smem_u32(&C.x_empty[slot]));
                        tc_fence_before();
                        mbar_arrive(smem_u32(&C.d_empty[slot]));
                    }
                    float ev[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const int64_t k = k0 + w;
                        const bool valid = full || (live && k < p.sN);
                        // levels 2 and 3 exactly as (h, l); levels 4..6 join l
                        float h, l;
                        two_sum(__uint_as_float(d0[w]), __uint_as_float(d1[w]), h, l);
                        l += __uint_as_float(d2[w]) + __uint_as_float(d3[w]);
                        const float tk = it[w];
                        float e = 0.f;
                        if (p.x_f64) {  // X in FP64: the subtraction in FP64
                            const double xd = valid ? reinterpret_cast<const double*>(p.X)[f * p.sN + k] : 0.0;
                            const double st = (double)sg * (double)tk;
                            const double ed = (xd - (double)h * st) - (double)l * st;
                            if (valid && p.E64) p.E64[f * p.sN + k] = ed;
                            e = valid ? (float)ed : 0.f;
                            xv[w] = (float)xd;
                        } else if (valid) {
                            // x - h sigma tau is exact near the optimum (Sterbenz); the scalings
                            // by powers of two are exact
                            const float hs = (h * sg) * tk, ls = (l * sg) * tk;
                            e = (xv[w] - hs) - ls;
                            if (p.E64) p.E64[f * p.sN + k] = ((double)xv[w] - (double)hs) - (double)ls;
                        }
                        ev[w] = e;
                        const float xm = valid ? xv[w] : 0.f;  // columns beyond s_N may hold stale data
                        e2 = fmaf(e, e, e2);
                        x2 = fmaf(xm, xm, x2);
                    }
                    if (live && p.planes) {
                        // 8 columns = one 16-byte piece of the row in each plane
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int u = 0; u < 8; u += 2) {
                            const __nv_bfloat162 hi2 = __floats2bfloat162_rn(ev[u], ev[u + 1]);
                            const float2 hf = __bfloat1622float2(hi2);
                            const __nv_bfloat162 lo2 = __floats2bfloat162_rn(ev[u] - hf.x, ev[u + 1] - hf.y);
                            hw[u >> 1] = *reinterpret_cast<const uint32_t*>(&hi2);
                            lw[u >> 1] = *reinterpret_cast<const uint32_t*>(&lo2);
                        }
                        const int pos = (((cc >> 3) ^ (r & 7)) << 3);
                        *reinterpret_cast<uint4*>(p.planes + tb + (int64_t)r * 64 + pos) =
                            make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(p.planes + tb + ((int64_t)rows_b + r) * 64 + pos) =
                            make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                float s1, s2;
                two_sum(eh, e2, s1, s2);
                eh = s1;
                el += s2;
                two_sum(xh, x2, s1, s2);
                xh = s1;
                xl += s2;
            }
        }
        // sum E^2 and sum X^2 over the workers (FP64 across threads, fixed order)
        double num = warp_sum((double)eh + (double)el), den = warp_sum((double)xh + (double)xl);
        if (lane == 0) {
            C.red[0][wk] = num;
            C.red[1][wk] = den;
        }
        named_sync(1, kWork);
        if (et == 0) {
            double a = 0.0, bsum = 0.0;
            for (int w = 0; w < kWorkWarps; ++w) {
                a += C.red[0][w];
                bsum += C.red[1][w];
            }
            atomicAdd(&p.stats->eres_num, a);
            atomicAdd(&p.stats->eres_den, bsum);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ------------------------------------------------------------ preparation
__device__ __forceinline__ float2 split_df(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

// A1df rows (s1 x 64, zero padded) and Wdf rows w_m = prod_{middle q} a^(q)_{i_q(m) r}
__global__ void recon_prep_rows(Shape s, Ptrs<const double> A, float2* A1df, float2* Wdf) {
    const int R = s.R, N = s.N;
    const int64_t na = s.dims[0] * kRT, nw = s.mid * kRT;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nw; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < na) {
            const int64_t i = e / kRT;
            const int r = (int)(e - i * kRT);
            A1df[e] = r < R ? split_df(A.p[0][i * R + r]) : make_float2(0.f, 0.f);
        } else {
            const int64_t f = e - na, m = f / kRT;
            const int r = (int)(f - m * kRT);
            double w = r < R ? 1.0 : 0.0;
            int64_t t = m;
            for (int qq = N - 2; qq >= 1 && r < R; --qq) {
                const int64_t iq = t % s.dims[qq];
                t /= s.dims[qq];
                w *= A.p[qq][iq * R + r];
            }
            Wdf[f] = split_df(w);
        }
    }
}

// Pieces of v_kr = a^(N)_kr / tau_k (one warp per k; lanes r and r + 32),
// exact in FP64, stored as the swizzled K-major image of each 64-row chunk.
__global__ void recon_prep_v(Shape s, const double* AN, int nck, unsigned char* Vsl, float* tau) {
    const int R = s.R;
    const int64_t sN = s.dims[s.N - 1];
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= (int64_t)nck * kKC) return;
    double v[2];
    double mx = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        v[h] = (k < sN && r < R) ? AN[k * R + r] : 0.0;
        mx = fmax(mx, fabs(v[h]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double t = mx > 0.0 ? pow2_ceil_d(mx) : 1.0;
    if (lane == 0) tau[k] = (float)t;
    const int c = (int)(k / kKC), kk = (int)(k - (int64_t)c * kKC);
    unsigned char* img = Vsl + (size_t)c * kBBytes;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = lane + 32 * h;
        // exact scalings by powers of two: multiplications by their exact reciprocals
        double x = v[h] * __longlong_as_double((2046LL << 52) - __double_as_longlong(t));  // 1 / t, t = 2^k
#pragma unroll
        for (int sl = 1; sl <= kSlices; ++sl) {
            // 2^(8 sl) and 2^(-8 sl) from their bit patterns
            const double g = __longlong_as_double((long long)(1023 + 8 * sl) << 52);
            const double gi = __longlong_as_double((long long)(1023 - 8 * sl) << 52);
            const double pc = rint(x * g) * gi;
            x -= pc;
            *reinterpret_cast<__nv_bfloat16*>(img + (size_t)(sl - 1) * kBSlice + sw128(kk, r)) =
                __float2bfloat16_rn((float)pc);
        }
    }
}

// The padding rows of the last i-block of every plane tile (rows s1 .. rounded
// up to 8) are never rows of X: zero, so that the MTTKRP of the planes reads
// finite values there.
__global__ void zero_pad_rows(PlaneTiling pt, int64_t s1, __nv_bfloat16* planes) {
    const int b = pt.nib - 1;
    const int r0 = (int)(s1 - (int64_t)b * 128), nr = pt.rows_last - r0;
    const int64_t per_tile = 2LL * nr * 64;
    const int64_t total = (int64_t)pt.nch * pt.mid * per_tile;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / per_tile, w = e - t * per_tile;
        const int c = (int)(t / pt.mid);
        const int64_t m = t - (int64_t)c * pt.mid;
        const int plane = (int)(w / (nr * 64)), rr = (int)(w % (nr * 64)) / 64, col = (int)(w % 64);
        planes[pt.tile(b, c, m) + ((int64_t)plane * pt.rows_last + r0 + rr) * 64 + col] = __float2bfloat16_rn(0.f);
    }
}

struct Layout {
    size_t a1, w, v, tau, total;
};
inline Layout layout_of(const Shape& s) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const int nck = (int)((s.dims[s.N - 1] + kKC - 1) / kKC);
    Layout l;
    l.a1 = 0;
    l.w = up((size_t)s.dims[0] * kRT * sizeof(float2));
    l.v = l.w + up((size_t)s.mid * kRT * sizeof(float2));
    l.tau = l.v + up((size_t)nck * kBBytes);
    l.total = l.tau + up((size_t)nck * kKC * sizeof(float));
    return l;
}

}  // namespace rtc

bool resid_tc_supported(const Shape& s) {
    return s.R <= rtc::kRT && s.N >= 2 && s.dims[0] * s.mid <= 0x7fffffffLL;
}

size_t resid_tc_scratch_bytes(const Shape& s) { return rtc::layout_of(s).total; }

int launch_resid_split_tc(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, void* planes,
                          double* E64, void* scratch, DevStats* stats, int* status, cudaStream_t st,
                          int reserve_sms) {
    using namespace rtc;
    static bool attr_set[64] = {};
    static int sms_of[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(recon_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (dev < 64) {
            attr_set[dev] = true;
            sms_of[dev] = sms;
        }
    }
    const int sms = dev < 64 ? sms_of[dev] : 148;
    const PlaneTiling pt = PlaneTiling::of(s);
    const Layout l = layout_of(s);
    unsigned char* sc = (unsigned char*)scratch;
    Params p;
    p.N = s.N;
    p.R = s.R;
    p.s1 = s.dims[0];
    p.mid = s.mid;
    p.sN = s.dims[s.N - 1];
    p.rows = p.s1 * p.mid;
    p.runs = (p.rows + kBI - 1) / kBI;
    p.nck = (int)((p.sN + kKC - 1) / kKC);
    p.pt = pt;
    p.X = X;
    p.x_f64 = xdt == CP_F64;
    p.A1df = (const float2*)(sc + l.a1);
    p.Wdf = (const float2*)(sc + l.w);
    p.Vsl = sc + l.v;
    p.tau = (const float*)(sc + l.tau);
    p.planes = (__nv_bfloat16*)planes;
    p.E64 = E64;
    p.stats = stats;
    p.status = status;
    int launched = 3;
    if (planes && pt.rows_last > (int)(p.s1 - (int64_t)(pt.nib - 1) * 128)) {
        zero_pad_rows<<<64, 256, 0, st>>>(pt, p.s1, (__nv_bfloat16*)planes);
        ++launched;
    }
    recon_prep_rows<<<256, 256, 0, st>>>(s, A, (float2*)(sc + l.a1), (float2*)(sc + l.w));
    const int64_t nk = (int64_t)p.nck * kKC;
    recon_prep_v<<<(unsigned)((nk * 32 + 255) / 256), 256, 0, st>>>(s, A.p[s.N - 1], p.nck, sc + l.v,
                                                                    (float*)(sc + l.tau));
    // X tiles by tensor copy: FP32 X viewed as the (s_1 mid) x s_N matrix of its rows,
    // box 32 x 128, 128-byte swizzle, zero fill outside the tensor
    CUtensorMap tmX;
    memset(&tmX, 0, sizeof(tmX));
    p.x_tma = 0;
    EncodeTiledFn enc = tc_encode_fn();
    if (enc && xdt == CP_F32 && p.sN % 4 == 0 && ((uintptr_t)X & 15u) == 0) {
        cuuint64_t dims[2] = {(cuuint64_t)p.sN, (cuuint64_t)p.rows};
        cuuint64_t strides[1] = {(cuuint64_t)p.sN * 4};
        cuuint32_t box[2] = {32, (cuuint32_t)kBI};
        cuuint32_t es[2] = {1, 1};
        p.x_tma = enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    // one CTA per SM (a CTA's shared memory fills an SM), less the SMs reserved for work beside it:
    // a CTA that had to wait for one of them would finish its static share of the runs late
    const int grid = (int)std::min<int64_t>(std::max(1, sms - std::max(0, reserve_sms)), p.runs);
    recon_tc_kernel<<<grid, kThreads, kDynSmem, st>>>(tmX, p);
    return launched;
}

}  // namespace cpgn
