// k_resid.cu -- the residual tensor E = X - [[A^(1), ..., A^(N)]] in
// double-float arithmetic, written as bf16 high/low planes for the
// tensor-core MTTKRP, with sum E^2 and sum X^2 accumulated in FP64.
//
// Why: the gradient of f (Eq. (2.3)) is G^(n) = A^(n) Gamma^(n) - X_(n) P^(n)
// = -E_(n) P^(n), because [[A]]_(n) P^(n) = A^(n) (P^(n)T P^(n)) = A^(n) Gamma^(n).
// Near the optimum E is small, so the MTTKRP of E in bf16x3 (relative error
// ~1e-5 of |E| |P|) gives a gradient accurate to ~1e-5 * r relative to |M|,
// where the direct form A Gamma - M cancels to the ~1e-5 error of M itself.
// The reconstruction needs ~1e-10 relative accuracy, which FP32 cannot give;
// it is evaluated as a double-float (hi + lo FP32 pair) dot product over the
// rank with error-free products (two-product through fmaf, Dekker 1971) and
// error-free sums (two-sum, Knuth), about 2^-44 relative, on the FP32 pipes,
// which GB300 runs at 64x its FP64 rate.
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

// acc += a * b in double-float (a, b, acc as (hi, lo)); the lo*lo term is dropped.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float2 a, float2 b) {
    const float p = a.x * b.x;
    float pe = fmaf(a.x, b.x, -p);
    pe = fmaf(a.x, b.y, pe);
    pe = fmaf(a.y, b.x, pe);
    const float t = sh + p;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sh = t;
    sl += err + pe;
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

// Block tile 64 (i) x 64 (k) outputs, 128 threads, each an 8 x 4 register tile
// (rows 8*ti + u, columns tk + 16 c).
template <typename TX>
__global__ void __launch_bounds__(NT) resid_split_kernel(Shape s, const TX* __restrict__ X,
                                                        const float2* __restrict__ Adf,
                                                        __nv_bfloat16* __restrict__ planes, PlaneTiling pt,
                                                        DevStats* stats) {
    __shared__ float2 As[RC][TI];
    __shared__ float2 Bs[RC][TK];
    __shared__ float2 ws[RC];
    __shared__ double red[32];
    const int64_t m = blockIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * TI, k0 = (int64_t)blockIdx.z * TK;
    const int R = s.R, N = s.N;
    const int64_t s1 = s.dims[0], sN = s.dims[N - 1], mid = s.mid;
    int64_t idx[kMaxN];
    {
        int64_t t = m;
        for (int q = N - 2; q >= 1; --q) {
            idx[q] = t % s.dims[q];
            t /= s.dims[q];
        }
    }
    const int ti = threadIdx.x >> 4, tk = threadIdx.x & 15;
    float sh[8][4], sl[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) sh[u][c] = sl[u][c] = 0.0f;
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
                for (int c = 0; c < 4; ++c) df_mac(sh[u][c], sl[u][c], a[u], b[c]);
        }
        __syncthreads();
    }
    float nh = 0.f, nl = 0.f, dh = 0.f, dl = 0.f;
    // every row and column of every tile is written (zero outside the tensor)
    const int64_t iw = pt.rows_padded(), kw = (int64_t)pt.nch * 64;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + ti * 8 + u;
        if (i >= iw) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t k = k0 + tk + 16 * c;
            if (k >= kw) continue;
            float e = 0.0f;
            if (k < sN && i < s1) {
                const TX x = X[(i * mid + m) * sN + k];
                if constexpr (sizeof(TX) == 4) {
                    // x - sh is exact when the reconstruction is close (Sterbenz)
                    e = (x - sh[u][c]) - sl[u][c];
                    df_sq_acc(dh, dl, x);
                } else {
                    e = (float)((x - (double)sh[u][c]) - (double)sl[u][c]);
                    const float xh = (float)x;
                    df_sq_acc(dh, dl, xh);
                }
                df_sq_acc(nh, nl, e);
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(e);
            const __nv_bfloat16 lo = __float2bfloat16_rn(e - __bfloat162float(hi));
            planes[pt.elem(i, m, k, 0)] = hi;
            planes[pt.elem(i, m, k, 1)] = lo;
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

// packed double-float copy of every factor: Adf[row][r] = (hi, lo) of A^(n)[i][r]
__global__ void factors_df_kernel(Shape s, Ptrs<const double> A, float2* Adf) {
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        Adf[s.roff[n] * s.R + e] = split_df(A.p[n][e]);
}

void launch_resid_split(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, void* planes,
                        void* Adf_scratch, DevStats* stats, cudaStream_t st) {
    float2* Adf = (float2*)Adf_scratch;
    factors_df_kernel<<<dim3(32, s.N), 256, 0, st>>>(s, A, Adf);
    const PlaneTiling pt = PlaneTiling::of(s);
    dim3 grid((unsigned)s.mid, (unsigned)((pt.rows_padded() + TI - 1) / TI), (unsigned)((pt.nch * 64 + TK - 1) / TK));
    if (xdt == CP_F32)
        resid_split_kernel<float><<<grid, NT, 0, st>>>(s, (const float*)X, Adf, (__nv_bfloat16*)planes, pt, stats);
    else
        resid_split_kernel<double><<<grid, NT, 0, st>>>(s, (const double*)X, Adf, (__nv_bfloat16*)planes, pt, stats);
}

}  // namespace cpgn
