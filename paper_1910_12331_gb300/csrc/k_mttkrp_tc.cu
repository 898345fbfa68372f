// k_mttkrp_tc.cu -- all-mode MTTKRP on tcgen05 tensor cores (sm_103a), bf16 split products.
//
// Arithmetic.  Every operand value v is split into bf16 parts v = v_hi + v_lo
// (+ O(2^-17 |v|)); products are sums of bf16 x bf16 terms, each exact in the
// FP32 tensor-core accumulator (the split of Henry, Tang and Heinecke,
// "Leveraging the bfloat16 artificial intelligence datatype for
// higher-precision computations", ARITH 2019).  GEMM-Y forms
// x_hi*b_hi + x_lo*b_hi + x_hi*b_lo (bf16x3) with two MMAs per K-step, the B
// operand stacking [b_hi; b_lo] in its N rows for the x_hi product.  GEMM-Z
// stacks hi and lo in both operands (A rows 2r, 2r+1 = hi, lo of column r;
// B columns = [x_hi | x_lo]) and so forms all four products (bf16x4) in one
// MMA per K-step.  Accumulation is FP32; the partials are reduced in FP64.
//
// Algorithm (Section 2.2's dimension tree, one pass over X).  X is viewed as
// s_1 x mid x s_N.  For a slice m of the middle modes,
// w_m[r] = prod_{middle q} a^(q)_{i_q(m) r}.  A step (b, g, m) covers the 128
// rows i of block b and the 128 columns k of group g (two 64-column chunks):
//   GEMM-Y     D_Y[i][r]    = sum_k X[i,m,k] a^(N)_{kr}              (Y_m, partial over k)
//   GEMM-Z^T   D_Z[c][r][k] += sum_i (a^(1)_{ir} w_m[r]) X[i,m,k]    (M^(N), per chunk c)
// GEMM-Z folds w_m into its A operand (B_Z, rebuilt per step), so D_Z
// accumulates in TMEM over the steps of a segment (at most kLmax steps of one
// (b, g) run).  D_Y is read out per step: M^(1)[i] += w_m * D_Y[i]
// (registers, per run) and c_m = sum_i a^(1)_{ir} D_Y[i][r] feeds the middle
// modes.  Both GEMMs read the same shared-memory X chunk: GEMM-Y as a K-major
// A operand, GEMM-Z as an MN-major B operand.
//
// Kernel: persistent, one CTA per SM, 12 warps; CTA g owns a contiguous range
// of steps in (b, g, m) order (m fastest).
//   warp 0      producer: the step's X chunk tiles (128 i x 64 k, both planes,
//               32 KB each, stored pre-swizzled so that linear bulk copies land
//               them) into one of two step slots, and the step's B_Z =
//               split(a^(1)(block b) * w_m)^T (32 KB, built for every (b, m)
//               by bz_prep_kernel in the same pre-swizzled form) into one of
//               two B_Z buffers; the w_m rows a few steps ahead; at each run
//               start the group's B_Y = [hi; lo] a^(N)^T (2 x 16 KB by TMA,
//               resident for the run).
//   warp 1      TMEM allocator and GEMM-Y issuer (one thread).
//   warp 2      GEMM-Z issuer (one thread).
//   warp 3      idle.
//   warps 4-11  workers, two per TMEM lane quadrant: drain D_Y
//               (double-buffered in TMEM) into M^(1) and c_m, and D_Z at
//               segment end.  One code path per sub-partition keeps the hot
//               instruction footprint small.
// Partials go to workspace in FP32 and a finalize kernel reduces them in a
// fixed order into the FP64 outputs (no atomics, deterministic).
// Every mbarrier wait is bounded: on expiry the CTA records CP_ERR_TIMEOUT,
// raises a CTA-local abort flag, drains what it issued (bounded) and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kernels.hpp"
#include "tc.hpp"
#include "tc_ptx.cuh"

namespace cpgn {

namespace tc {

using namespace tcx;

constexpr int kWQ = 2;                   // worker warps per TMEM lane quadrant
constexpr int kWork = 128 * kWQ;         // worker threads
constexpr int kThreads = 128 + kWork;    // four role warps + the workers
constexpr int kWCols = 64 / kWQ;         // rank columns of D_Y / D_Z per worker warp
constexpr int kStages = 4;               // X chunk tiles in flight
constexpr int kBI = 128;                 // rows of an i-block (M of GEMM-Y, K of GEMM-Z)
constexpr int kKC = 64;                  // columns of a chunk
constexpr int kGroup = 2;                // chunks per step
constexpr int kRT = 64;                  // rank columns per launch
constexpr int kLmax = 32;                // steps per segment at most (bounds the FP32 TMEM chains)
constexpr uint32_t kTile = 32 * 1024;    // X chunk tile [plane][128 i][64 k] bf16
constexpr uint32_t kXPlane = 16 * 1024;  // one plane of a tile
constexpr uint32_t kOpSub = 16 * 1024;   // 128 rows x 64 bf16 of a K-major operand
constexpr uint32_t kBYBytes = kGroup * kOpSub;  // B_Y: [chunk][128 rows: r hi, r lo][64 k]
constexpr uint32_t kBZBytes = 2 * kOpSub;       // B_Z: [i / 64][128 rows: 2r hi, 2r+1 lo][64 i]
constexpr uint32_t kPayload = kStages * kTile + kBYBytes + 2 * kBZBytes;  // 1024-aligned operand buffers
constexpr int kWRing = 6;                // w_m rows in flight (shared by builders and epilogue)
constexpr int kWAhead = 3;               // the producer loads w_m this many steps ahead of its X loads
constexpr uint32_t kTmemCols = 512;      // D_Y x2 (128 columns each) + D_Z x2 chunks (128 each)
constexpr CUtensorMapL2promotion kL2Promo = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;

struct Params {
    int N;
    int R;              // columns of this rank tile (<= 64)
    const unsigned char* planes;  // bf16 planes of X in PlaneTiling layout
    PlaneTiling pt;
    int64_t s1, mid, sN;
    int nib, nch, ngr;  // i-blocks, 64-column chunks, groups of two chunks
    int64_t steps;      // nib * ngr * mid
    int smax;           // segment slots per CTA
    int64_t middim[kMaxN];  // s_q of the middle modes (index q)
    const float* A1f;   // [s1][64] rows of A^(1) (rank tile), FP32, zero padded
    const float* W;     // [mid][64] w_m (rank tile), FP32, zero padded
    const unsigned char* BZ;  // [nib][mid] B_Z tiles of the rank tile (kBZBytes each, pre-swizzled)
    float* P_Y1;        // [slot][128 i][64 r]        M^(1) partial of a run (when seg[slot].y)
    float* P_Z;         // [slot][2 chunks][64 r][64 k]  M^(N) partial of a segment
    float* P_c;         // [nib][ngr][mid][64]        c_m partial of a step
    int4* seg;          // [slot]: (b, g, y, 0) of the segment in a slot; b = -1 if unused
    int* status;
};

// Barriers, flags and small arrays, placed after the operand buffers in the
// one dynamic shared-memory region (the kernel uses no static shared memory,
// so the region starts on the 1024-byte boundary the swizzled operands need;
// the kernel checks this and reports CP_ERR_UNSUPPORTED otherwise).
struct SmemCtl {
    uint64_t full[2], empty[2];  // per step slot (two chunk stages each)
    uint64_t bz_full[2], bz_empty[2], dy_full[2], dy_empty[2];
    uint64_t by_full, by_empty, dz_full, dz_empty, drain[2];
    uint64_t w_full[kWRing], w_empty[kWRing];
    uint32_t tmem_base;
    int abort_flag;
    int dec[2];
    alignas(16) float red[4][kRT];       // per-warp column sums of the epilogue
    alignas(16) float wring[kWRing][kRT];  // w_m rows, filled by bulk copies
};
constexpr uint32_t kDynSmem = kPayload + (uint32_t)sizeof(SmemCtl);
static_assert(kDynSmem <= 227 * 1024, "shared memory above the per-block limit");


// Sum 16 per-lane values over the 32 lanes of a warp.  Afterwards lane l holds
// in v[0] the warp total of column butterfly16_col(l) (lanes l and l^1 agree).
__device__ __forceinline__ void butterfly16(float* v, int lane) {
#pragma unroll
    for (int off = 16, w = 8; off >= 2; off >>= 1, w >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < w; ++j) {
            const float send = upper ? v[j] : v[j + w];
            const float keep = upper ? v[j + w] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ int butterfly16_col(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Step (b, g, m) of linear index t = (b * ngr + g) * mid + m.  Decoded once
// per role; the loops then advance it without divisions.
struct StepId {
    int b, g;
    int64_t m;
    __device__ __forceinline__ void next(const Params& p) {
        if (++m == p.mid) {
            m = 0;
            if (++g == p.ngr) {
                g = 0;
                ++b;
            }
        }
    }
};
__device__ __forceinline__ StepId step_of(const Params& p, int64_t t) {
    StepId r;
    r.m = t % p.mid;
    const int64_t bg = t / p.mid;
    r.g = (int)(bg % p.ngr);
    r.b = (int)(bg / p.ngr);
    return r;
}
// Segment bookkeeping shared by the MMA issuer and the epilogue: a run is a
// maximal range of steps with fixed (b, g) inside the CTA's range; a segment
// is at most kLmax consecutive steps of one run.
struct SegTrack {
    int zs = -1, zl = 0;
    // call once per step, in order; returns (run_start, seg_start)
    __device__ __forceinline__ void enter(int64_t t, int64_t T0, int64_t m, bool& run_start, bool& seg_start) {
        run_start = t == T0 || m == 0;
        seg_start = run_start || zl == kLmax;
        if (seg_start) {
            ++zs;
            zl = 0;
        }
        ++zl;
    }
};
__device__ __forceinline__ bool run_last(const Params& p, int64_t t, int64_t T1, int64_t m) {
    return t + 1 == T1 || m + 1 == p.mid;
}

__global__ void __launch_bounds__(kThreads, 1)
    mttkrp_tc_kernel(const __grid_constant__ CUtensorMap tmBY, Params p) {
    extern __shared__ __align__(1024) unsigned char dsmem[];
    if (smem_u32(dsmem) & 1023u) {  // block-uniform: nothing has been issued yet
        if (threadIdx.x == 0) atomicCAS(p.status, 0, CP_ERR_UNSUPPORTED);
        return;
    }
    unsigned char* base = dsmem;
    SmemCtl& C = *reinterpret_cast<SmemCtl*>(base + kPayload);
    volatile int* abort_s = &C.abort_flag;
    const uint32_t sbase = smem_u32(base);
    const uint32_t s_stage0 = sbase;
    const uint32_t s_by = sbase + kStages * kTile;
    const uint32_t s_bz0 = s_by + kBYBytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Rows of the last i-block beyond its tile's rows are never copied in; they
    // must hold finite values (they meet zero rows of B_Z and unused rows of D_Y).
    for (int e = threadIdx.x; e < (int)(kStages * kTile / 16); e += kThreads)
        reinterpret_cast<uint4*>(base)[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&C.full[s]), 1);
            mbar_init(smem_u32(&C.empty[s]), 2);  // released by both MMA issuers
            mbar_init(smem_u32(&C.drain[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&C.bz_full[s]), 1);
            mbar_init(smem_u32(&C.bz_empty[s]), 1);
            mbar_init(smem_u32(&C.dy_full[s]), 1);
            mbar_init(smem_u32(&C.dy_empty[s]), kWork);
        }
        for (int s = 0; s < kWRing; ++s) {
            mbar_init(smem_u32(&C.w_full[s]), 1);
            mbar_init(smem_u32(&C.w_empty[s]), kWork);
        }
        mbar_init(smem_u32(&C.by_full), 1);
        mbar_init(smem_u32(&C.by_empty), 1);
        mbar_init(smem_u32(&C.dz_full), 1);
        mbar_init(smem_u32(&C.dz_empty), kWork);
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
    const uint32_t t_dy0 = tmem, t_dz0 = tmem + 256;
    const int64_t T0 = (int64_t)blockIdx.x * p.steps / gridDim.x;
    const int64_t T1 = (int64_t)(blockIdx.x + 1) * p.steps / gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            bool ok = true;
            int yg = -1;
            int64_t it = 0;
            StepId sp = step_of(p, T0), wsp = sp;  // wsp: the next step whose w_m row is loaded
            int64_t wl = 0;                         // w_m rows loaded so far
            for (int64_t t = T0; t < T1 && ok; ++t, sp.next(p)) {
                for (; ok && wl <= (t - T0) + kWAhead && T0 + wl < T1; ++wl, wsp.next(p)) {
                    const int ws = (int)(wl % kWRing);
                    if (!(ok = mbar_wait(smem_u32(&C.w_empty[ws]), (uint32_t)(((wl / kWRing) & 1) ^ 1), abort_s,
                                         p.status)))
                        break;
                    const uint32_t wb = smem_u32(&C.w_full[ws]);
                    mbar_expect_tx(wb, kRT * sizeof(float));
                    bulk_load(smem_u32(&C.wring[ws][0]), p.W + wsp.m * kRT, kRT * sizeof(float), wb);
                }
                if (!ok) break;
                if (t == T0 || sp.m == 0) {  // run start: the group's B_Y (both chunks; missing ones read as zero)
                    ++yg;
                    if (!(ok = mbar_wait(smem_u32(&C.by_empty), (uint32_t)((yg & 1) ^ 1), abort_s, p.status)))
                        break;
                    const uint32_t fb = smem_u32(&C.by_full);
                    mbar_expect_tx(fb, kBYBytes);
                    for (int cc = 0; cc < kGroup; ++cc)
                        tma_load_2d(s_by + cc * kOpSub, &tmBY, (sp.g * kGroup + cc) * kKC, 0, fb);
                }
                // the step's chunks go to the two stages of step slot tt & 1
                const int nc = (int)imin(kGroup, p.nch - sp.g * kGroup);
                const uint32_t pbytes = (uint32_t)p.pt.rows(sp.b) * 128u;  // one plane of a tile
                const int slot = (int)(it & 1);
                if (!(ok = mbar_wait(smem_u32(&C.empty[slot]), (uint32_t)(((it >> 1) & 1) ^ 1), abort_s, p.status)))
                    break;
                const uint32_t fb = smem_u32(&C.full[slot]);
                mbar_expect_tx(fb, 2 * nc * pbytes);
                for (int cc = 0; cc < nc; ++cc) {
                    const unsigned char* src = p.planes + 2 * p.pt.tile(sp.b, sp.g * kGroup + cc, sp.m);
                    const uint32_t dst = s_stage0 + (2 * slot + cc) * kTile;
                    bulk_load(dst, src, pbytes, fb);
                    bulk_load(dst + kXPlane, src + pbytes, pbytes, fb);
                }
                // the step's B_Z, once the GEMM-Z MMAs two steps back have released its buffer
                if (!(ok = mbar_wait(smem_u32(&C.bz_empty[slot]), (uint32_t)(((it >> 1) & 1) ^ 1), abort_s,
                                     p.status)))
                    break;
                const uint32_t fz = smem_u32(&C.bz_full[slot]);
                mbar_expect_tx(fz, kBZBytes);
                bulk_load(s_bz0 + slot * kBZBytes, p.BZ + ((size_t)sp.b * p.mid + sp.m) * kBZBytes, kBZBytes, fz);
                ++it;
            }
            // every issued copy must have landed before the CTA may exit
            for (int64_t k = (it > 2 ? it - 2 : 0); k < it; ++k) {
                mbar_drain(smem_u32(&C.full[k & 1]), (uint32_t)((k >> 1) & 1), p.status);
                mbar_drain(smem_u32(&C.bz_full[k & 1]), (uint32_t)((k >> 1) & 1), p.status);
            }
            for (int64_t k = (wl > kWRing ? wl - kWRing : 0); k < wl; ++k)
                mbar_drain(smem_u32(&C.w_full[k % kWRing]), (uint32_t)((k / kWRing) & 1), p.status);
            if (yg >= 0) mbar_drain(smem_u32(&C.by_full), (uint32_t)(yg & 1), p.status);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ GEMM-Y issuer
        // (also the TMEM allocator).  D_Y[i][0:64] += X_hi B_hi + X_lo B_hi,
        // D_Y[i][64:128] += X_hi B_lo over both chunks of a step.  Descriptors
        // are a base descriptor plus the K-step's byte offset / 16 (the 14-bit
        // address field cannot carry: shared memory is below 256 KB).
        if (lane == 0) {
            const uint32_t id_y128 = idesc_bf16(128, false, false), id_y64 = idesc_bf16(64, false, false);
            bool ok = true;
            int yg = -1;
            StepId sp = step_of(p, T0);
            for (int64_t t = T0, tt = 0; t < T1 && ok; ++t, ++tt, sp.next(p)) {
                if (t == T0 || sp.m == 0) {
                    ++yg;
                    if (!(ok = mbar_wait(smem_u32(&C.by_full), (uint32_t)(yg & 1), abort_s, p.status))) break;
                }
                const int slot = (int)(tt & 1), db = slot;
                const uint32_t ph = (uint32_t)((tt >> 1) & 1);
                // K-steps of 16 columns in each chunk of the step (0 for a missing second chunk)
                const int64_t k0 = (int64_t)sp.g * kGroup * kKC;
                const int ys0 = (int)((imin(kKC, p.sN - k0) + 15) / 16);
                const int ys1 = p.sN > k0 + kKC ? (int)((imin(kKC, p.sN - k0 - kKC) + 15) / 16) : 0;
                if (!(ok = mbar_wait(smem_u32(&C.dy_empty[db]), ph ^ 1, abort_s, p.status))) break;
                if (!(ok = mbar_wait(smem_u32(&C.full[slot]), ph, abort_s, p.status))) break;
                tc_fence_after();
                const uint32_t t_dy = t_dy0 + db * 128;
                const uint64_t dx0 = sdesc(s_stage0 + (2 * slot) * kTile, 16, 1024), dby0 = sdesc(s_by, 16, 1024);
#pragma unroll
                for (int cc = 0; cc < kGroup; ++cc) {
                    const int ysteps = cc == 0 ? ys0 : ys1;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        if (ks < ysteps) {
                            const uint64_t xo = (uint64_t)((cc * kTile + ks * 32) >> 4);
                            const uint64_t bo = (uint64_t)((cc * kOpSub + ks * 32) >> 4);
                            tc_mma(t_dy, dx0 + xo, dby0 + bo, id_y128, (cc | ks) != 0);
                            tc_mma(t_dy, dx0 + xo + (kXPlane >> 4), dby0 + bo, id_y64, 1);
                        }
                    }
                }
                tc_commit(smem_u32(&C.dy_full[db]));
                tc_commit(smem_u32(&C.empty[slot]));
                if (run_last(p, t, T1, sp.m)) tc_commit(smem_u32(&C.by_empty));
            }
            // every issued MMA must have completed before TMEM is freed
            tc_commit(smem_u32(&C.drain[0]));
            mbar_drain(smem_u32(&C.drain[0]), 0, p.status);
        }
        __syncwarp();
    } else if (warp == 2) {
        // ------------------------------------------------------ GEMM-Z issuer
        // D_Z[rho][n] += sum_i B_Z[rho][i] [X_hi c0 | X_lo c0 | X_hi c1 | X_lo c1][i][n]:
        // one N = 256 MMA per K-step covers both chunks (the two stages of a
        // step slot are adjacent, so the four 64-column atoms are 16 KB apart).
        if (lane == 0) {
            const uint32_t id_z = idesc_bf16(256, false, true);
            bool ok = true;
            SegTrack seg;
            bool zfirst = true;
            StepId sp = step_of(p, T0);
            for (int64_t t = T0, tt = 0; t < T1 && ok; ++t, ++tt, sp.next(p)) {
                bool run_start, seg_start;
                seg.enter(t, T0, sp.m, run_start, seg_start);
                if (seg_start) {
                    // the epilogue must have read the previous segment's D_Z
                    if (!(ok = mbar_wait(smem_u32(&C.dz_empty), (uint32_t)((seg.zs & 1) ^ 1), abort_s, p.status)))
                        break;
                    zfirst = true;
                }
                const int slot = (int)(tt & 1), db = slot;
                const uint32_t ph = (uint32_t)((tt >> 1) & 1);
                const int zsteps = (int)((imin(kBI, p.s1 - (int64_t)sp.b * kBI) + 15) / 16);
                if (!(ok = mbar_wait(smem_u32(&C.full[slot]), ph, abort_s, p.status))) break;
                if (!(ok = mbar_wait(smem_u32(&C.bz_full[db]), ph, abort_s, p.status))) break;
                tc_fence_after();
                const uint64_t dbz = sdesc(s_bz0 + db * kBZBytes, 16, 1024);
                const uint64_t dxz = sdesc(s_stage0 + (2 * slot) * kTile, kXPlane, 1024);
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    if (ks < zsteps) {
                        const uint64_t ao = (uint64_t)((((ks >> 2) * kOpSub) + (ks & 3) * 32) >> 4);
                        const uint64_t bo = (uint64_t)((ks * 2048) >> 4);
                        tc_mma(t_dz0, dbz + ao, dxz + bo, id_z, (ks == 0 && zfirst) ? 0 : 1);
                    }
                }
                zfirst = false;
                tc_commit(smem_u32(&C.bz_empty[db]));
                tc_commit(smem_u32(&C.empty[slot]));
                if (run_last(p, t, T1, sp.m) || seg.zl == kLmax) tc_commit(smem_u32(&C.dz_full));
            }
            tc_commit(smem_u32(&C.drain[1]));
            mbar_drain(smem_u32(&C.drain[1]), 0, p.status);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ------------------------------------------------------------ workers
        // Warps 4-11, two per TMEM lane quadrant.  Step t of the loop drains
        // D_Y of step t: thread = TMEM lane (row i) and 32 rank columns (warp half).
        const int wk = warp - 4;
        const int q = warp & 3;                  // TMEM lane quadrant of this warp
        const int cb = kWCols * (wk >> 2);       // first rank column of this warp's D_Y / D_Z share
        const int row = q * 32 + lane;           // lane of D_Y (row i) and of D_Z (row rho)
        const int et = wk * 32 + lane;           // 0 .. kWork - 1
        auto grp_wait = [&](uint32_t bar, uint32_t parity) -> bool {
            mbar_wait(bar, parity, abort_s, p.status);
            named_sync(2, kWork);
            if (et == 0) C.dec[1] = *abort_s;
            named_sync(2, kWork);
            return C.dec[1] == 0;
        };
        float a1r[kWCols], m1acc[kWCols];  // A^(1) row `row` (columns cb ..) and the M^(1) partial
        int pb = -1;
        StepId sp = step_of(p, T0);
        SegTrack seg;
        int done = 0;
        bool ok = true;
        int64_t tt = 0;
        for (int64_t t = T0; t < T1 && ok; ++t, ++tt, sp.next(p)) {
            bool run_start, seg_start;
            seg.enter(t, T0, sp.m, run_start, seg_start);
            if (run_start) {
                if (sp.b != pb) {
                    pb = sp.b;
                    const int64_t gi = (int64_t)sp.b * kBI + row;
#pragma unroll
                    for (int r = 0; r < kWCols; ++r) a1r[r] = gi < p.s1 ? p.A1f[gi * kRT + cb + r] : 0.0f;
                }
#pragma unroll
                for (int r = 0; r < kWCols; ++r) m1acc[r] = 0.0f;
            }
            const int db = (int)(tt & 1);
            const int ws = (int)(tt % kWRing);
            if (!(ok = grp_wait(smem_u32(&C.w_full[ws]), (uint32_t)((tt / kWRing) & 1)))) break;
            if (!(ok = grp_wait(smem_u32(&C.dy_full[db]), (uint32_t)((tt >> 1) & 1)))) break;
            tc_fence_after();
            const uint32_t ta = t_dy0 + db * 128 + cb + ((uint32_t)(q * 32) << 16);
#pragma unroll
            for (int j = 0; j < kWCols; j += 16) {
                uint32_t ra[16], rb[16];
                tmem_ld16x2_wait(ta + j, ta + 64 + j, ra, rb);
                float v[16];
#pragma unroll
                for (int u = 0; u < 16; u += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(&C.wring[ws][cb + j + u]);
                    const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float y = __uint_as_float(ra[u + x]) + __uint_as_float(rb[u + x]);
                        m1acc[j + u + x] = fmaf(w[x], y, m1acc[j + u + x]);
                        v[u + x] = y * a1r[j + u + x];
                    }
                }
                if (p.N >= 3) {
                    butterfly16(v, lane);
                    if ((lane & 1) == 0) C.red[q][cb + j + butterfly16_col(lane)] = v[0];
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&C.dy_empty[db]));
            mbar_arrive(smem_u32(&C.w_empty[ws]));
            if (p.N >= 3) {
                named_sync(2, kWork);
                if (et < kRT)
                    p.P_c[(((int64_t)sp.b * p.ngr + sp.g) * p.mid + sp.m) * kRT + et] =
                        C.red[0][et] + C.red[1][et] + C.red[2][et] + C.red[3][et];
                named_sync(2, kWork);
            }
            const bool rl = run_last(p, t, T1, sp.m);
            if (rl || seg.zl == kLmax) {
                const bool slot_ok = seg.zs < p.smax;
                const int64_t slot = (int64_t)blockIdx.x * p.smax + seg.zs;
                if (rl && slot_ok) {
                    float* py = p.P_Y1 + (slot * kBI + row) * kRT + cb;
#pragma unroll
                    for (int r = 0; r < kWCols; r += 4)
                        *reinterpret_cast<float4*>(py + r) =
                            make_float4(m1acc[r], m1acc[r + 1], m1acc[r + 2], m1acc[r + 3]);
                }
                if (!(ok = grp_wait(smem_u32(&C.dz_full), (uint32_t)(seg.zs & 1)))) break;
                tc_fence_after();
                // D_Z[cc][rho][n]: rho = 2r + (lo part); n < 64: x_hi column k = n, else x_lo column n - 64
                const int nc = (int)imin(kGroup, p.nch - sp.g * kGroup);
                for (int cc = 0; cc < nc; ++cc) {
                    float* pz = p.P_Z + ((slot * kGroup + cc) * kRT + (row >> 1)) * kKC + cb;
                    const uint32_t tz = t_dz0 + cc * 128 + cb + ((uint32_t)(q * 32) << 16);
#pragma unroll
                    for (int j = 0; j < kWCols; j += 16) {
                        uint32_t za[16], zb[16];
                        tmem_ld16x2_wait(tz + j, tz + 64 + j, za, zb);
                        float z[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            z[u] = __uint_as_float(za[u]) + __uint_as_float(zb[u]);
                            z[u] += __shfl_xor_sync(0xffffffffu, z[u], 1);  // hi + lo rows of column r
                        }
                        if (slot_ok && (lane & 1) == 0) {
#pragma unroll
                            for (int u = 0; u < 16; u += 4)
                                *reinterpret_cast<float4*>(pz + j + u) = make_float4(z[u], z[u + 1], z[u + 2], z[u + 3]);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&C.dz_empty));
                if (et == 0) {
                    if (slot_ok)
                        p.seg[slot] = make_int4(sp.b, sp.g, rl ? 1 : 0, 0);
                    else
                        atomicCAS(p.status, 0, CP_ERR_UNSUPPORTED);  // segment count above the host's bound
                }
                done = seg.zs + 1;
            }
        }
        // slots without a (complete) segment are marked unused
        if (et == 0)
            for (int k = done; k < p.smax; ++k) p.seg[(int64_t)blockIdx.x * p.smax + k] = make_int4(-1, -1, 0, 0);
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
// X -> bf16 planes in PlaneTiling layout (hi, lo; zero outside the tensor).
// A block handles rows (i, m) of the padded range, a thread four consecutive
// columns (8-byte stores, which stay contiguous under the 16-byte swizzle).
// FP32 arithmetic for FP32 input (x - hi is exact), FP64 only for FP64 input.
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
__global__ void split_x_kernel(const TX* __restrict__ X, __nv_bfloat16* __restrict__ planes, PlaneTiling pt) {
    const int nq = pt.nch * 16;  // quads per padded row
    const int64_t nrows = pt.rows_padded() * pt.mid;
    for (int64_t rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
        const int64_t i = rr / pt.mid, m = rr - (rr / pt.mid) * pt.mid;
        const TX* xr = X + (i * pt.mid + m) * pt.sN;
        const bool row_ok = i < pt.s1;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int64_t k = 4 * (int64_t)q;
            __nv_bfloat16 hi[4], lo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split1<TX>(row_ok && k + u < pt.sN ? xr[k + u] : (TX)0, hi[u], lo[u]);
            uint2 vh, vl;
            vh.x = (uint32_t)__bfloat16_as_ushort(hi[0]) | ((uint32_t)__bfloat16_as_ushort(hi[1]) << 16);
            vh.y = (uint32_t)__bfloat16_as_ushort(hi[2]) | ((uint32_t)__bfloat16_as_ushort(hi[3]) << 16);
            vl.x = (uint32_t)__bfloat16_as_ushort(lo[0]) | ((uint32_t)__bfloat16_as_ushort(lo[1]) << 16);
            vl.y = (uint32_t)__bfloat16_as_ushort(lo[2]) | ((uint32_t)__bfloat16_as_ushort(lo[3]) << 16);
            *reinterpret_cast<uint2*>(planes + pt.elem(i, m, k, 0)) = vh;
            *reinterpret_cast<uint2*>(planes + pt.elem(i, m, k, 1)) = vl;
        }
    }
}

// One launch prepares a rank tile r0 .. r0 + 63.  blockIdx.y selects the part:
// 0 = B_Y planes [128][pitch] (rows 0..63 hi of a^(N)[:, r0 + r]^T, rows
// 64..127 lo), 1 = FP32 rows of A^(1) [s1][64], 2 = w_m for every slice
// [mid][64] (the product over the middle modes in FP64, rounded once); all
// zero padded in r.
__global__ void prep_kernel(Shape s, Ptrs<const double> A, int r0, int64_t pitch, __nv_bfloat16* __restrict__ BY,
                            float* __restrict__ A1f, float* __restrict__ W) {
    const int R = s.R, N = s.N;
    const int part = blockIdx.y;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (part == 0) {
        const double* AN = A.p[N - 1];
        const int64_t total = (int64_t)kRT * pitch, sN = s.dims[N - 1];
        for (int64_t e = e0; e < total; e += stride) {
            const int r = (int)(e / pitch);
            const int64_t k = e % pitch;
            const double a = (k < sN && r0 + r < R) ? AN[k * R + r0 + r] : 0.0;
            const __nv_bfloat16 hi = __double2bfloat16(a);
            BY[e] = hi;
            BY[total + e] = __double2bfloat16(a - (double)__bfloat162float(hi));
        }
    } else if (part == 1) {
        const int64_t total = s.dims[0] * kRT;
        for (int64_t e = e0; e < total; e += stride) {
            const int64_t i = e / kRT;
            const int r = (int)(e % kRT);
            A1f[e] = (r0 + r < R) ? (float)A.p[0][i * R + r0 + r] : 0.0f;
        }
    } else {
        const int64_t total = s.mid * kRT;
        for (int64_t e = e0; e < total; e += stride) {
            int64_t m = e / kRT;
            const int r = (int)(e % kRT);
            double w = r0 + r < R ? 1.0 : 0.0;
            for (int q = N - 2; q >= 1 && r0 + r < R; --q) {  // the last middle mode varies fastest in m
                const int64_t iq = m % s.dims[q];
                m /= s.dims[q];
                w *= A.p[q][iq * R + r0 + r];
            }
            W[e] = (float)w;
        }
    }
}

// B_Z of every (i-block b, slice m) of the rank tile: rows 2r and 2r + 1 hold
// the bf16 hi and lo parts of a^(1)_{ir} w_m[r] (FP32 product) for the 128 rows i
// of the block (K = i, two 64-column sub-tiles), in the 128-byte-swizzled
// K-major byte image the GEMM-Z MMAs read; rows i >= s_1 are zero.  A block
// stages the rows of A^(1) of its i-block transposed in shared memory
// (coalesced loads once) and writes the tiles of kBzSlices consecutive slices
// m; thread = one column pair (i, i + 1) of 16 ranks (4-byte stores that
// cover whole 128-byte rows per warp).
constexpr int kBzSlices = 4;
__global__ void __launch_bounds__(256) bz_prep_kernel(const float* __restrict__ A1f, const float* __restrict__ W,
                                                      int64_t s1, int64_t mid, int nib, unsigned char* __restrict__ BZ) {
    __shared__ __align__(16) float a1t[kRT][kBI];  // a1t[r][i] = a^(1)_{b*128+i, r}
    const int et = threadIdx.x;
    const int64_t mchunks = (mid + kBzSlices - 1) / kBzSlices;
    const int64_t b = blockIdx.x / mchunks, mc = blockIdx.x - b * mchunks;
    for (int e = et; e < kBI * kRT; e += 256) {
        const int i = e / kRT, r = e - i * kRT;
        const int64_t gi = b * kBI + i;
        a1t[r][i] = gi < s1 ? A1f[gi * kRT + r] : 0.0f;
    }
    __syncthreads();
    const int i0 = 2 * (et & 63), rq = 16 * (et >> 6), ii = i0 & 63;
    for (int64_t m = mc * kBzSlices; m < mid && m < (mc + 1) * kBzSlices; ++m) {
        unsigned char* out = BZ + (b * mid + m) * kBZBytes + (i0 >> 6) * kOpSub;
#pragma unroll 4
        for (int r = rq; r < rq + 16; ++r) {
            const float w = __ldg(W + m * kRT + r);
            const float2 a = *reinterpret_cast<const float2*>(&a1t[r][i0]);
            const float p0 = a.x * w, p1 = a.y * w;
            const __nv_bfloat162 hi = __floats2bfloat162_rn(p0, p1);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(p0 - __low2float(hi), p1 - __high2float(hi));
            const int rh = 2 * r, rl = 2 * r + 1;
            *reinterpret_cast<__nv_bfloat162*>(out + rh * 128 + ((((ii >> 3) ^ (rh & 7)) & 7) << 4) + (ii & 7) * 2) = hi;
            *reinterpret_cast<__nv_bfloat162*>(out + rl * 128 + ((((ii >> 3) ^ (rl & 7)) & 7) << 4) + (ii & 7) * 2) = lo;
        }
    }
}

// Reduce the partials into the FP64 outputs in a fixed order, columns r0 .. r0+Rt-1.
// grid.y = mode.  Mode 1: block = 8 rows i of one i-block x 32 threads (two
// columns each).  Mode N: block = 64 columns k of one chunk for one rank, four
// threads per output, each summing an interleaved quarter of the slots, the
// quarters then added in a fixed order.  Both list the slots of their i-block
// (chunk's group) in increasing order, kFinList at a time (the slot records
// are staged in shared memory by all threads, then compacted by one warp), and
// sum the listed partials with sixteen independent loads in flight.  Middle modes: block = 8
// rows x 32 threads, summing the per-step column sums c_m times the other
// middle factors.
constexpr int kFinRows = 8;
constexpr int kFinList = 1024;
__device__ __forceinline__ int fin_list(const Params& p, int e0, int e1, int which, int key, int* list, int4* stage) {
    __shared__ int cnt_s;
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) stage[e - e0] = p.seg[e];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int cnt = 0;
        for (int e = e0; e < e1; e += 32) {
            const int ee = e + lane;
            bool hit = false;
            if (ee < e1) {
                const int4 sg = stage[ee - e0];
                hit = sg.x >= 0 && (which == 0 ? (sg.x == key && sg.z != 0) : sg.y == key);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (hit) list[cnt + __popc(mask & ((1u << lane) - 1u))] = ee;
            cnt += __popc(mask);
        }
        if (lane == 0) cnt_s = cnt;
    }
    __syncthreads();
    return cnt_s;
}

__global__ void __launch_bounds__(256) finalize_kernel(Params p, Ptrs<double> M, Ptrs<const double> A, int R, int r0,
                                                       int Rt, int nslots, unsigned mode_mask) {
    __shared__ int list[kFinList];
    __shared__ int4 stage[kFinList];
    const int N = p.N;
    const int n = blockIdx.y;
    if (!(mode_mask & (1u << n))) return;
    if (n == N - 1) {
        // block = one rank r of one chunk c; thread = column k of the chunk and one
        // of four interleaved quarters of the slot list; the quarters are added in
        // a fixed order
        __shared__ double qsum[4][kKC];
        const int c = blockIdx.x >> 6, r = blockIdx.x & 63;
        if (c >= p.nch || r >= Rt) return;  // uniform over the block (ranks past the tile's own: nothing to write)
        const int kk = threadIdx.x & 63, qt = threadIdx.x >> 6;
        const int64_t k = (int64_t)c * kKC + kk;
        const int g = c / kGroup, cc = c % kGroup;
        const float* src = p.P_Z + ((int64_t)cc * kRT + r) * kKC + kk;
        const int64_t sstride = (int64_t)kGroup * kRT * kKC;  // floats per slot
        double acc = 0.0;
        for (int e0 = 0; e0 < nslots; e0 += kFinList) {
            const int cnt = fin_list(p, e0, min(nslots, e0 + kFinList), 1, g, list, stage);
            for (int j = qt; j < cnt; j += 4 * 16) {
                float v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = j + 4 * u < cnt ? src[(int64_t)list[j + 4 * u] * sstride] : 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u) acc += v[u];
            }
            __syncthreads();
        }
        qsum[qt][kk] = acc;
        __syncthreads();
        if (qt == 0 && k < p.sN && r < Rt)
            M.p[n][k * R + r0 + r] = (qsum[0][kk] + qsum[1][kk]) + (qsum[2][kk] + qsum[3][kk]);
        return;
    }
    const int64_t sn = n == 0 ? p.s1 : p.middim[n];
    const int64_t i0 = (int64_t)blockIdx.x * kFinRows;
    if (i0 >= sn) return;  // uniform over the block
    const int64_t i = i0 + (threadIdx.x >> 5);
    const int c0 = 2 * (threadIdx.x & 31);
    double acc0 = 0.0, acc1 = 0.0;
    if (n == 0) {
        const int b = (int)(i0 / kBI);  // 8 divides 128: the block's rows share an i-block
        for (int e0 = 0; e0 < nslots; e0 += kFinList) {
            const int cnt = fin_list(p, e0, min(nslots, e0 + kFinList), 0, b, list, stage);
            if (i < sn) {
                const float* src = p.P_Y1 + (i % kBI) * kRT + c0;
                for (int j = 0; j < cnt; j += 16) {
                    float2 v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        v[u] = j + u < cnt ? *reinterpret_cast<const float2*>(src + (int64_t)list[j + u] * kBI * kRT)
                                           : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        acc0 += v[u].x;
                        acc1 += v[u].y;
                    }
                }
            }
            __syncthreads();
        }
    } else {
        if (i >= sn) return;
        // middle mode n: sum over the slices m whose index in mode n is i of
        // (sum over the (b, g) partials of c_m) * (product of the other middle factors)
        const int64_t sub = p.mid / sn;
        const int nbg = p.nib * p.ngr;
        for (int64_t t = 0; t < sub; ++t) {
            int64_t rem = t, m = 0, mult = 1;
            double lo0 = 1.0, lo1 = 1.0;
            for (int q = N - 2; q >= 1; --q) {
                const int64_t dq = p.middim[q];
                int64_t iq;
                if (q == n) {
                    iq = i;
                } else {
                    iq = rem % dq;
                    rem /= dq;
                    if (c0 < Rt) lo0 *= A.p[q][iq * R + r0 + c0];
                    if (c0 + 1 < Rt) lo1 *= A.p[q][iq * R + r0 + c0 + 1];
                }
                m += iq * mult;
                mult *= dq;
            }
            const float* src = p.P_c + m * kRT + c0;
            double cs0 = 0.0, cs1 = 0.0;
            for (int j = 0; j < nbg; j += 8) {
                float2 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = j + u < nbg ? *reinterpret_cast<const float2*>(src + (int64_t)(j + u) * p.mid * kRT)
                                       : make_float2(0.0f, 0.0f);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    cs0 += v[u].x;
                    cs1 += v[u].y;
                }
            }
            acc0 += cs0 * lo0;
            acc1 += cs1 * lo1;
        }
    }
    if (i >= sn) return;
    if (c0 < Rt) M.p[n][i * R + r0 + c0] = acc0;
    if (c0 + 1 < Rt) M.p[n][i * R + r0 + c0 + 1] = acc1;
}

// ------------------------------------------------------------ host side
static EncodeTiledFn encode_fn() { return tc_encode_fn(); }



}  // namespace tc

using namespace tc;

size_t split_cache_bytes(const cp_desc* d) { return (size_t)PlaneTiling::of(make_shape(d)).total() * sizeof(__nv_bfloat16); }

int tc_launch_count(const SplitCache& c, const cp_desc* d, const Shape& s) {
    const bool hit = c.planes && c.key_ptr != nullptr && c.key_version == d->x_version && c.key_total == s.total &&
                     c.key_dtype == (int)d->x_dtype;
    const int tiles = (s.R + kRT - 1) / kRT;
    return (hit ? 0 : 1) + tiles * 4;  // per rank tile: prep, B_Z prep, main, finalize
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


// Launch geometry: grid = min(SMs, steps); CTA g takes steps
// [g T / G, (g + 1) T / G), at most ceil(T / G) of them.  Segments start at
// the range start, at every run start (m = 0) and after kLmax steps of a run,
// so a CTA has at most floor(per / kLmax) + ceil(per / mid) + 2 of them.
struct TcGeom {
    int nib, nch, ngr, grid, smax;
    int64_t steps;
};
static TcGeom tc_geom(const Shape& s, int sms) {
    TcGeom g;
    const int64_t mid = s.mid;
    g.nib = (int)((s.dims[0] + kBI - 1) / kBI);
    g.nch = (int)((s.dims[s.N - 1] + kKC - 1) / kKC);
    g.ngr = (g.nch + kGroup - 1) / kGroup;
    g.steps = (int64_t)g.nib * g.ngr * mid;
    g.grid = (int)imin(sms, g.steps);
    const int64_t per = (g.steps + g.grid - 1) / g.grid;
    g.smax = (int)(per / kLmax + (per + mid - 1) / mid + 2);
    return g;
}

// Device workspace tc_main allocates for one shape (its operand planes,
// partial sums and segment records; the rank tiles reuse it), for
// cp_workspace_size.  Same formulas as tc_main.
size_t tc_workspace_bytes(const Shape& s, int sms) {
    const TcGeom g = tc_geom(s, sms);
    const int64_t pitch = (int64_t)g.nch * kKC;
    const size_t nslots = (size_t)g.grid * g.smax;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    return al((size_t)2 * kRT * pitch * sizeof(__nv_bfloat16)) + al((size_t)s.dims[0] * kRT * sizeof(float)) +
           al((size_t)s.mid * kRT * sizeof(float)) + al(nslots * kBI * kRT * sizeof(float)) +
           al(nslots * kGroup * kRT * kKC * sizeof(float)) +
           al((size_t)g.nib * g.ngr * s.mid * kRT * sizeof(float)) + al(nslots * sizeof(int4)) +
           al((size_t)g.nib * s.mid * kBZBytes);
}

// bf16 planes of X, cached by pointer / size / version.
static cp_status tc_split_x(SplitCache& c, const cp_desc* d, const Shape& s, const void* X, int sms,
                            cudaStream_t st) {
    const PlaneTiling pt = PlaneTiling::of(s);
    const size_t pbytes = (size_t)pt.total() * sizeof(__nv_bfloat16);
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
    const int blocks = sms * 16;
    if (d->x_dtype == CP_F32)
        split_x_kernel<float><<<blocks, 128, 0, st>>>((const float*)X, (__nv_bfloat16*)c.planes, pt);
    else
        split_x_kernel<double><<<blocks, 128, 0, st>>>((const double*)X, (__nv_bfloat16*)c.planes, pt);
    c.key_ptr = X;
    c.key_version = d->x_version;
    c.key_total = s.total;
    c.key_dtype = (int)d->x_dtype;
    return CP_OK;
}

// MTTKRP on bf16 planes (PlaneTiling layout) that are already in device memory.
static cp_status tc_main(SplitCache& c, const void* planes, const Shape& s, Ptrs<const double> A, Ptrs<double> M,
                         unsigned mode_mask, int* status, cudaStream_t st) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return CP_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int N = s.N, R = s.R;
    const int64_t s1 = s.dims[0], sN = s.dims[N - 1], mid = s.mid;
    const TcGeom g = tc_geom(s, sms);
    const int64_t pitch = (int64_t)g.nch * kKC;  // row pitch of the B_Y planes
    const int nslots = g.grid * g.smax;
    Params p{};
    p.N = N;
    p.planes = (const unsigned char*)planes;
    p.pt = PlaneTiling::of(s);
    p.s1 = s1;
    p.mid = mid;
    p.sN = sN;
    p.nib = g.nib;
    p.nch = g.nch;
    p.ngr = g.ngr;
    p.steps = g.steps;
    p.smax = g.smax;
    for (int q = 1; q + 1 < N; ++q) p.middim[q] = s.dims[q];
    // ---- workspace: operand planes and partials
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t by_b = al((size_t)2 * kRT * pitch * sizeof(__nv_bfloat16));
    const size_t a1_b = al((size_t)s1 * kRT * sizeof(float));
    const size_t w_b = al((size_t)mid * kRT * sizeof(float));
    const size_t py_b = al((size_t)nslots * kBI * kRT * sizeof(float));
    const size_t pz_b = al((size_t)nslots * kGroup * kRT * kKC * sizeof(float));
    const size_t pc_b = al((size_t)g.nib * g.ngr * mid * kRT * sizeof(float));
    const size_t sg_b = al((size_t)nslots * sizeof(int4));
    const size_t bz_b = al((size_t)g.nib * mid * kBZBytes);
    if (ensure_buf(c.fac, c.fac_bytes, by_b + a1_b + w_b + py_b + pz_b + pc_b + sg_b + bz_b) != CP_OK)
        return CP_ERR_NOMEM;
    unsigned char* wb = (unsigned char*)c.fac;
    __nv_bfloat16* BY = (__nv_bfloat16*)wb;
    p.A1f = (const float*)(wb += by_b);
    p.W = (const float*)(wb += a1_b);
    p.P_Y1 = (float*)(wb += w_b);
    p.P_Z = (float*)(wb += py_b);
    p.P_c = (float*)(wb += pz_b);
    p.seg = (int4*)(wb += pc_b);
    unsigned char* BZ = (wb += sg_b);
    p.BZ = BZ;
    p.status = status;
    // ---- tensor map of the B_Y planes (rows of s_N elements; the pitch padding reads as zero)
    CUtensorMap tmBY;
    {
        cuuint64_t dims[2] = {(cuuint64_t)sN, 128};
        cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
        cuuint32_t box[2] = {(cuuint32_t)kKC, 128};
        cuuint32_t es[2] = {1, 1};
        if (enc(&tmBY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, BY, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, kL2Promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
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
    int64_t rows = s1;
    for (int q = 1; q + 1 < N; ++q) rows = std::max<int64_t>(rows, s.dims[q]);
    const int64_t fx = std::max<int64_t>((rows + kFinRows - 1) / kFinRows, (int64_t)g.nch * kRT);
    const dim3 fgrid((unsigned)fx, (unsigned)N);
    for (int r0 = 0; r0 < R; r0 += kRT) {
        const int Rt = std::min(kRT, R - r0);
        p.R = Rt;
        prep_kernel<<<dim3(sms, 3), 256, 0, st>>>(s, A, r0, pitch, BY, (float*)p.A1f, (float*)p.W);
        bz_prep_kernel<<<(unsigned)((int64_t)g.nib * ((mid + kBzSlices - 1) / kBzSlices)), 256, 0, st>>>(
            p.A1f, p.W, s1, mid, g.nib, BZ);
        mttkrp_tc_kernel<<<g.grid, kThreads, kDynSmem, st>>>(tmBY, p);
        if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
        finalize_kernel<<<fgrid, 256, 0, st>>>(p, M, A, R, r0, Rt, nslots, mode_mask);
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

