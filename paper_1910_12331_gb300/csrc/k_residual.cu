// k_residual.cu -- direct relative residual r = ||X - [[A]]||_F / ||X||_F
// (Section 5's relative residual; fitness is 1 - r).
//
// The reconstruction is formed tile by tile and never stored:
//   X~(i, m, k) = sum_r a^(1)_{ir} w_m[r] a^(N)_{kr},  w_m[r] = prod_{middle q} a^(q)_{i_q(m) r},
// in FP64, and both sum (x - x~)^2 and sum x^2 are accumulated in FP64.  The
// Gram-matrix expansion ||X||^2 - 2<M,A> + ||X~||^2 is not used: it cancels
// catastrophically below r ~ 1e-8.
#include "kernels.hpp"

namespace cpgn {

namespace {
constexpr int TI = 32, TK = 32, RC = 32, NT = 256;
}

template <typename TX>
__global__ void __launch_bounds__(NT) residual_kernel(Shape s, const TX* __restrict__ X, Ptrs<const double> A,
                                                     DevStats* stats) {
    __shared__ double Ai[TI][RC + 1];
    __shared__ double Ak[TK][RC + 1];
    __shared__ double red[32];
    const int64_t m = blockIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * TI, k0 = (int64_t)blockIdx.z * TK;
    const int R = s.R, N = s.N;
    const int64_t s1 = s.dims[0], sL = s.dims[N - 1], mid = s.mid;
    int64_t idx[kMaxN];
    {
        int64_t t = m;
        for (int q = N - 2; q >= 1; --q) { idx[q] = t % s.dims[q]; t /= s.dims[q]; }
    }
    // each thread: 4 elements (rows ti + 8u, column tk)
    const int tk = threadIdx.x & 31, ti = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int rc = 0; rc < R; rc += RC) {
        for (int t = threadIdx.x; t < TI * RC; t += NT) {
            const int ii = t / RC, c = t % RC;
            const int64_t i = i0 + ii;
            const int r = rc + c;
            Ai[ii][c] = (i < s1 && r < R) ? A.p[0][i * R + r] : 0.0;
        }
        for (int t = threadIdx.x; t < TK * RC; t += NT) {
            const int kk = t / RC, c = t % RC;
            const int64_t k = k0 + kk;
            const int r = rc + c;
            double v = 0.0;
            if (k < sL && r < R) {
                v = A.p[N - 1][k * R + r];
                for (int q = 1; q + 1 < N; ++q) v *= A.p[q][idx[q] * R + r];
            }
            Ak[kk][c] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < RC; ++c) {
            const double b = Ak[tk][c];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += Ai[ti + 8 * u][c] * b;
        }
        __syncthreads();
    }
    double num = 0.0, den = 0.0;
    const int64_t k = k0 + tk;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ti + 8 * u;
        if (i < s1 && k < sL) {
            const double x = (double)X[(i * mid + m) * sL + k];
            const double d = x - acc[u];
            num += d * d;
            den += x * x;
        }
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->res_num, num);
        atomicAdd(&stats->res_den, den);
    }
}

void launch_residual_f64(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, DevStats* stats,
                         cudaStream_t st) {
    dim3 grid((unsigned)s.mid, (unsigned)((s.dims[0] + TI - 1) / TI), (unsigned)((s.dims[s.N - 1] + TK - 1) / TK));
    if (xdt == CP_F32)
        residual_kernel<float><<<grid, NT, 0, st>>>(s, (const float*)X, A, stats);
    else
        residual_kernel<double><<<grid, NT, 0, st>>>(s, (const double*)X, A, stats);
}

}  // namespace cpgn
