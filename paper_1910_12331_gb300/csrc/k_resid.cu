// k_resid.cu -- the residual tensor E = X - [[A^(1), ..., A^(N)]] in
// extended precision, written as bf16 high/low planes for the tensor-core
// MTTKRP, with sum E^2 and sum X^2 accumulated in double-float.
//
// Why: the gradient of f (Eq. (2.3)) is G^(n) = A^(n) Gamma^(n) - X_(n) P^(n)
// = -E_(n) P^(n), because [[A]]_(n) P^(n) = A^(n) (P^(n)T P^(n)) = A^(n) Gamma^(n).
// Near the optimum E is small, so the MTTKRP of E in bf16x3 (relative error
// ~1e-5 of |E| |P|) gives a gradient accurate to ~1e-5 * r relative to |M|,
// where the direct form A Gamma - M cancels to the ~1e-5 error of M itself.
// The reconstruction needs far more than FP32's 2^-24, and GB300 runs FP64 at
// 1/64 of its FP32 rate, so it is evaluated on the FP32 pipes:
//  * every factor entry is a double-float pair (hi + lo);
//  * the leading products hi*hi are summed into an accumulator that starts at
//    a power of two sigma >= 4 B, where B bounds sum_r |hi*hi| over the tile.
//    Every partial sum then stays in [3 sigma / 4, 5 sigma / 4], so the part
//    z = t - acc that a fused multiply-add t = fma(a, b, acc) added is exact
//    (Sterbenz), and fma(a, b, -z) is the part it dropped, itself rounded by
//    at most 2^-48 sigma (fixed-offset error-free summation: Dekker's
//    FastTwoSum against a constant offset, as in Rump, Ogita and Oishi 2008);
//  * the dropped parts and the cross products hi*lo + lo*hi go to an FP32
//    low accumulator.
// That is six FP32 instructions per rank term and element, with an error of
// order 2^-48 sigma plus 2^-24 of the low accumulator (about 1e-11 of |X|
// for Gaussian factors), incoherent from entry to entry.
#include <cuda_bf16.h>

#include "kernels.hpp"
#include "tc.hpp"

namespace cpgn {

namespace {
constexpr int TI = 64, TK = 64, RC = 32, NT = 128;

__device__ __forceinline__ float2 split_df(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

// (hi, lo) product of two double-float numbers (lo*lo dropped), normalised
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}

}  // namespace

// Error-free sum s + e = a + b (Knuth two-sum)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}
// acc (hi, lo) += x * x in double-float
__device__ __forceinline__ void df_sq_acc(float& h, float& l, float x) {
    const float p = x * x;
    const float pe = fmaf(x, x, -p);
    float s, e;
    two_sum_f(h, p, s, e);
    h = s;
    l += e + pe;
}

// Smallest power of two >= v, for finite v > 0 (0 for v == 0).
__device__ __forceinline__ float pow2_ceil(float v) {
    return __uint_as_float((__float_as_uint(v) + 0x007fffffu) & 0xff800000u);
}

// Asynchronous copy of one TX from global to shared memory (cp.async, sm_80+).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// X tile row pitch in shared memory (one pad element against bank conflicts)
constexpr int kXPitch = TK + 1;
template <typename TX>
constexpr size_t resid_dyn_smem() {
    return (size_t)TI * kXPitch * sizeof(TX);
}

// Block tile 64 (i) x 64 (k) outputs, 128 threads, each an 8 x 4 register tile
// (rows 8*ti + u, columns tk + 16 c).  amax1[ib][r] / amaxN[kb][r] hold the
// largest |hi| of column r of A^(1) / A^(N) over the 64-row block ib / kb.
// The X tile streams into shared memory (cp.async) while the block computes;
// the block's outputs are 64 consecutive rows of one PlaneTiling tile, i.e.
// one contiguous run per plane, staged in shared memory in the tile's swizzled
// byte order and written with 16-byte stores.
template <typename TX>
__global__ void __launch_bounds__(NT) resid_split_kernel(Shape s, const TX* __restrict__ X,
                                                        const float2* __restrict__ Adf,
                                                        const float* __restrict__ amax1,
                                                        const float* __restrict__ amaxN,
                                                        __nv_bfloat16* __restrict__ planes, PlaneTiling pt,
                                                        double* __restrict__ E64, DevStats* stats) {
    __shared__ __align__(16) float2 As[RC][TI];
    __shared__ __align__(16) float2 Bs[RC][TK];
    __shared__ float2 ws[RC];
    __shared__ double red[32];
    __shared__ float s_sigma;
    extern __shared__ __align__(16) unsigned char xs_raw[];
    TX* Xs = reinterpret_cast<TX*>(xs_raw);  // [TI][kXPitch]
    const int64_t m = blockIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * TI, k0 = (int64_t)blockIdx.z * TK;
    const int R = s.R, N = s.N;
    const int64_t s1 = s.dims[0], sN = s.dims[N - 1], mid = s.mid;
    // X tile: coalesced rows of 64 elements, zero outside the tensor
    for (int e = threadIdx.x; e < TI * TK; e += NT) {
        const int ii = e / TK, kk = e % TK;
        const int64_t i = i0 + ii, k = k0 + kk;
        if (i < s1 && k < sN)
            cp_async_elem<sizeof(TX)>(&Xs[ii * kXPitch + kk], &X[(i * mid + m) * sN + k]);
        else
            Xs[ii * kXPitch + kk] = (TX)0;
    }
    int64_t idx[kMaxN];
    {
        int64_t t = m;
        for (int q = N - 2; q >= 1; --q) {
            idx[q] = t % s.dims[q];
            t /= s.dims[q];
        }
    }
    if (threadIdx.x < 32) {
        // B = sum_r max_i |a_ir| |w_r| max_k |b_kr| >= every partial sum of hi*hi in the tile
        float bound = 0.0f;
        for (int r = threadIdx.x; r < R; r += 32) {
            float w = 1.0f;
            for (int q = 1; q + 1 < N; ++q) w *= fabsf(Adf[(s.roff[q] + idx[q]) * R + r].x);
            bound = fmaf(amax1[blockIdx.y * R + r] * w, amaxN[blockIdx.z * R + r], bound);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(0xffffffffu, bound, o);
        // 4.5 B covers the bound's own FP32 rounding; the floor keeps sigma normal
        if (threadIdx.x == 0) s_sigma = pow2_ceil(fmaxf(4.5f * bound, 0x1p-100f));
    }
    const int ti = threadIdx.x >> 4, tk = threadIdx.x & 15;
    __syncthreads();
    const float sigma = s_sigma;
    float sh[8][4], sl[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            sh[u][c] = sigma;
            sl[u][c] = 0.0f;
        }
    for (int r0 = 0; r0 < R; r0 += RC) {
        if (threadIdx.x < RC) {
            float2 w = make_float2(0.f, 0.f);
            if (r0 + (int)threadIdx.x < R) {
                w = make_float2(1.f, 0.f);
                for (int q = 1; q + 1 < N; ++q) w = df_mul(w, Adf[(s.roff[q] + idx[q]) * R + r0 + threadIdx.x]);
            }
            ws[threadIdx.x] = w;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < RC * TI; t += NT) {
            const int rr = t / TI, ii = t % TI;
            const int64_t i = i0 + ii;
            const int r = r0 + rr;
            As[rr][ii] = (i < s1 && r < R) ? Adf[i * R + r] : make_float2(0.f, 0.f);
        }
        for (int t = threadIdx.x; t < RC * TK; t += NT) {
            const int rr = t / TK, kk = t % TK;
            const int64_t k = k0 + kk;
            const int r = r0 + rr;
            Bs[rr][kk] = (k < sN && r < R) ? df_mul(ws[rr], Adf[(s.roff[N - 1] + k) * R + r]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int rn = R - r0 < RC ? R - r0 : RC;
#pragma unroll 2
        for (int rr = 0; rr < rn; ++rr) {
            float2 a[8], b[4];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = As[rr][ti * 8 + u];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[rr][tk + 16 * c];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float t = fmaf(a[u].x, b[c].x, sh[u][c]);
                    const float z = t - sh[u][c];  // exact: t and sh within a factor 5/3
                    float l = fmaf(a[u].x, b[c].y, sl[u][c]);
                    l = fmaf(a[u].y, b[c].x, l);
                    sl[u][c] = l + fmaf(a[u].x, b[c].x, -z);
                    sh[u][c] = t;
                }
        }
        if (r0 + RC >= R) cp_async_wait_all();
        __syncthreads();
    }
    // As is free: it stages the two bf16 planes of the block's 64 rows,
    // [plane][row][64] in the tile's swizzled order (2 x 8 KB)
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(&As[0][0]);
    float nh = 0.f, nl = 0.f, dh = 0.f, dl = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int ii = ti * 8 + u;
        const int64_t i = i0 + ii;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int kk = tk + 16 * c;
            const int64_t k = k0 + kk;
            float e = 0.0f;
            if (k < sN && i < s1) {
                const float rh = sh[u][c] - sigma;  // exact (Sterbenz)
                const TX x = Xs[ii * kXPitch + kk];
                if constexpr (sizeof(TX) == 4) {
                    // x - rh is exact when the reconstruction is close (Sterbenz)
                    e = (x - rh) - sl[u][c];
                    df_sq_acc(dh, dl, x);
                } else {
                    e = (float)((x - (double)rh) - (double)sl[u][c]);
                    const float xh = (float)x;
                    df_sq_acc(dh, dl, xh);
                }
                if (E64) E64[(i * mid + m) * sN + k] = ((double)x - (double)rh) - (double)sl[u][c];
                df_sq_acc(nh, nl, e);
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(e);
            const __nv_bfloat16 lo = __float2bfloat16_rn(e - __bfloat162float(hi));
            // row ii of the tile has (i0 + ii) mod 8 == ii mod 8 (i0 is a multiple of 64)
            const int col = (((kk >> 3) ^ (ii & 7)) << 3) | (kk & 7);
            stage[ii * 64 + col] = hi;
            stage[TI * 64 + ii * 64 + col] = lo;
        }
    }
    __syncthreads();
    // rows i0 .. i0 + nrow - 1 exist in the tile (every row and column of a tile
    // is written, zero outside the tensor)
    const int b = (int)(i0 >> 7), r0t = (int)(i0 & 127);
    const int nrow = min(TI, pt.rows(b) - r0t);
    if (planes && nrow > 0) {
        const int64_t base = pt.tile(b, (int)(k0 >> 6), m);
        const int chunks = nrow * 8;  // 16-byte pieces per plane
        for (int q = threadIdx.x; q < 2 * chunks; q += NT) {
            const int plane = q >= chunks, piece = q - plane * chunks;
            const int4 v = reinterpret_cast<const int4*>(stage + plane * TI * 64)[piece];
            __nv_bfloat16* dst = planes + base + ((int64_t)plane * pt.rows(b) + r0t) * 64;
            reinterpret_cast<int4*>(dst)[piece] = v;
        }
    }
    // per-thread double-float partials, combined in FP64 across the block
    double num = block_sum((double)nh + (double)nl, red);
    double den = block_sum((double)dh + (double)dl, red);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->eres_num, num);
        atomicAdd(&stats->eres_den, den);
    }
}

// packed double-float copy of every factor: Adf[row][r] = (hi, lo) of A^(n)[i][r];
// for the first and last mode also the block maxima amax[row / 64][r] of |hi|
// (non-negative floats order like their bit patterns, so an integer atomicMax)
__global__ void factors_df_kernel(Shape s, Ptrs<const double> A, float2* Adf, float* amax1, float* amaxN) {
    const int n = blockIdx.y, R = s.R;
    const int64_t len = s.dims[n] * R;
    float* amax = n == 0 ? amax1 : (n == s.N - 1 ? amaxN : nullptr);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = split_df(A.p[n][e]);
        Adf[s.roff[n] * R + e] = v;
        if (amax) {
            const int64_t row = e / R;
            const int r = (int)(e - row * R);
            atomicMax(reinterpret_cast<int*>(&amax[(row / TI) * R + r]), __float_as_int(fabsf(v.x)));
        }
    }
}

namespace {
// row blocks of the first mode's tiles (covering the padded rows) and of the last mode's
int64_t blocks1(const Shape& s) { return (PlaneTiling::of(s).rows_padded() + TI - 1) / TI; }
int64_t blocksN(const Shape& s) { return (int64_t)PlaneTiling::of(s).nch * 64 / TK; }
}  // namespace

size_t resid_scratch_bytes(const Shape& s) {
    return (size_t)s.roff[s.N] * s.R * sizeof(float2) + (size_t)(blocks1(s) + blocksN(s)) * s.R * sizeof(float);
}

void launch_resid_split(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, void* planes,
                        double* E64, void* scratch, DevStats* stats, cudaStream_t st) {
    float2* Adf = (float2*)scratch;
    float* amax1 = (float*)(Adf + (size_t)s.roff[s.N] * s.R);
    float* amaxN = amax1 + blocks1(s) * s.R;
    cudaMemsetAsync(amax1, 0, (size_t)(blocks1(s) + blocksN(s)) * s.R * sizeof(float), st);
    factors_df_kernel<<<dim3(32, s.N), 256, 0, st>>>(s, A, Adf, amax1, amaxN);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(resid_split_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resid_dyn_smem<float>());
        cudaFuncSetAttribute(resid_split_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resid_dyn_smem<double>());
        if (dev < 64) attr_set[dev] = true;
    }
    const PlaneTiling pt = PlaneTiling::of(s);
    dim3 grid((unsigned)s.mid, (unsigned)blocks1(s), (unsigned)blocksN(s));
    if (xdt == CP_F32)
        resid_split_kernel<float><<<grid, NT, resid_dyn_smem<float>(), st>>>(s, (const float*)X, Adf, amax1, amaxN,
                                                                              (__nv_bfloat16*)planes, pt, E64, stats);
    else
        resid_split_kernel<double><<<grid, NT, resid_dyn_smem<double>(), st>>>(
            s, (const double*)X, Adf, amax1, amaxN, (__nv_bfloat16*)planes, pt, E64, stats);
}

}  // namespace cpgn
