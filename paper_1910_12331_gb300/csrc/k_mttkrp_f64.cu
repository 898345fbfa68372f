// k_mttkrp_f64.cu -- all-mode MTTKRP in FP64 on the SIMT pipes (the plain path).
//
// M^(n) = X_(n) P^(n) (Section 2.2) as a dimension tree over the slices of X.
// X is viewed as s_1 x mid x s_N, mid = prod of the middle mode sizes.  For a
// slice m (a multi-index of the middle modes) let w_m[r] = prod_q a^(q)_{i_q(m) r}
// over the middle modes.  The two first-level contractions of the tree are
//   Y_m = X(:, m, :) A^(N)      (s_1 x R)   -> "Y kernel"
//   Z_m = X(:, m, :)^T A^(1)    (s_N x R)   -> "Z kernel"
// and the leaves follow from them:
//   M^(1)   += w_m * Y_m                         (Y kernel epilogue)
//   M^(q)_{i_q(m)} += c_m * prod_{q' != q} a^(q')_{i_q'(m)},  c_m = colsum(A^(1) * Y_m)
//   M^(N)   += w_m * Z_m                         (Z kernel epilogue)
// Work: 2 prod(s) R multiply-adds for the two first-level contractions.
// GB300's FP64 rate (about 1/64 of FP32) makes this path DFMA-bound; it is
// the honest FP64 comparator of the tensor-core path.  Cross-slice sums use
// FP64 atomics on the (L2-resident) outputs.
#include "kernels.hpp"

namespace cpgn {

namespace {
constexpr int BI = 32;  // output rows per block
constexpr int KC = 32;  // contraction chunk
constexpr int RT = 64;  // rank columns per block
constexpr int NT = 256; // threads: 32 rows x 8 column groups, 8 columns each

// Middle multi-index of slice m, C order over modes 1..N-2.
__device__ __forceinline__ void middle_index(const Shape& s, int64_t m, int64_t* idx) {
    for (int q = s.N - 2; q >= 1; --q) {
        idx[q] = m % s.dims[q];
        m /= s.dims[q];
    }
}

template <typename TX>
__device__ __forceinline__ double ldx(const TX* X, int64_t e) { return (double)X[e]; }
}  // namespace

template <typename TX>
__global__ void __launch_bounds__(NT) mttkrp_y_kernel(Shape s, const TX* __restrict__ X, Ptrs<const double> A,
                                                     Ptrs<double> M, unsigned mask) {
    __shared__ double Xs[BI][KC + 1];
    __shared__ double As[KC][RT];
    __shared__ double ws[RT];
    __shared__ double Ps[BI][RT + 1];
    const int64_t m = blockIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * BI;
    const int r0 = blockIdx.z * RT;
    const int R = s.R, N = s.N;
    const int64_t s1 = s.dims[0], sL = s.dims[N - 1], mid = s.mid;
    int64_t idx[kMaxN];
    middle_index(s, m, idx);
    for (int c = threadIdx.x; c < RT; c += NT) {
        double w = 1.0;
        if (r0 + c < R)
            for (int q = 1; q + 1 < N; ++q) w *= A.p[q][idx[q] * R + r0 + c];
        ws[c] = w;
    }
    const int ti = threadIdx.x >> 3, tj = threadIdx.x & 7;
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    const double* AL = A.p[N - 1];
    for (int64_t k0 = 0; k0 < sL; k0 += KC) {
        for (int t = threadIdx.x; t < BI * KC; t += NT) {
            const int ii = t / KC, kk = t % KC;
            const int64_t i = i0 + ii, k = k0 + kk;
            Xs[ii][kk] = (i < s1 && k < sL) ? ldx(X, (i * mid + m) * sL + k) : 0.0;
        }
        for (int t = threadIdx.x; t < KC * RT; t += NT) {
            const int kk = t / RT, c = t % RT;
            const int64_t k = k0 + kk;
            As[kk][c] = (k < sL && r0 + c < R) ? AL[k * R + r0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            const double x = Xs[ti][kk];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += x * As[kk][tj + 8 * j];
        }
        __syncthreads();
    }
    const int64_t i = i0 + ti;
    if ((mask & 1u) && i < s1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = r0 + tj + 8 * j;
            if (r < R) atomicAdd(&M.p[0][i * R + r], ws[tj + 8 * j] * acc[j]);
        }
    }
    const unsigned mid_mask = mask & ~1u & ~(1u << (N - 1));
    if (mid_mask) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = r0 + tj + 8 * j;
            Ps[ti][tj + 8 * j] = (i < s1 && r < R) ? A.p[0][i * R + r] * acc[j] : 0.0;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < RT; c += NT) {
            const int r = r0 + c;
            if (r >= R) continue;
            double cm = 0.0;
            for (int ii = 0; ii < BI; ++ii) cm += Ps[ii][c];
            for (int q = 1; q + 1 < N; ++q) {
                if (!(mid_mask & (1u << q))) continue;
                double lo = 1.0;
                for (int q2 = 1; q2 + 1 < N; ++q2)
                    if (q2 != q) lo *= A.p[q2][idx[q2] * R + r];
                atomicAdd(&M.p[q][idx[q] * R + r], cm * lo);
            }
        }
    }
}

template <typename TX>
__global__ void __launch_bounds__(NT) mttkrp_z_kernel(Shape s, const TX* __restrict__ X, Ptrs<const double> A,
                                                     Ptrs<double> M) {
    __shared__ double Xs[KC][BI + 1];
    __shared__ double As[KC][RT];
    __shared__ double ws[RT];
    const int64_t m = blockIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * BI;
    const int r0 = blockIdx.z * RT;
    const int R = s.R, N = s.N;
    const int64_t s1 = s.dims[0], sL = s.dims[N - 1], mid = s.mid;
    int64_t idx[kMaxN];
    middle_index(s, m, idx);
    for (int c = threadIdx.x; c < RT; c += NT) {
        double w = 1.0;
        if (r0 + c < R)
            for (int q = 1; q + 1 < N; ++q) w *= A.p[q][idx[q] * R + r0 + c];
        ws[c] = w;
    }
    const int tk = threadIdx.x >> 3, tj = threadIdx.x & 7;
    double acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0;
    const double* A0 = A.p[0];
    for (int64_t i0 = 0; i0 < s1; i0 += KC) {
        for (int t = threadIdx.x; t < KC * BI; t += NT) {
            const int ii = t / BI, kk = t % BI;
            const int64_t i = i0 + ii, k = k0 + kk;
            Xs[ii][kk] = (i < s1 && k < sL) ? ldx(X, (i * mid + m) * sL + k) : 0.0;
        }
        for (int t = threadIdx.x; t < KC * RT; t += NT) {
            const int ii = t / RT, c = t % RT;
            const int64_t i = i0 + ii;
            As[ii][c] = (i < s1 && r0 + c < R) ? A0[i * R + r0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < KC; ++ii) {
            const double x = Xs[ii][tk];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += x * As[ii][tj + 8 * j];
        }
        __syncthreads();
    }
    const int64_t k = k0 + tk;
    if (k < sL) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = r0 + tj + 8 * j;
            if (r < R) atomicAdd(&M.p[N - 1][k * R + r], ws[tj + 8 * j] * acc[j]);
        }
    }
}

void launch_mttkrp_f64(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, Ptrs<double> M,
                       unsigned mode_mask, cudaStream_t st) {
    const int N = s.N;
    const unsigned last = 1u << (N - 1);
    const unsigned ymask = mode_mask & ~last;
    const unsigned rt = (unsigned)((s.R + RT - 1) / RT);
    if (ymask) {
        dim3 grid((unsigned)s.mid, (unsigned)((s.dims[0] + BI - 1) / BI), rt);
        if (xdt == CP_F32)
            mttkrp_y_kernel<float><<<grid, NT, 0, st>>>(s, (const float*)X, A, M, ymask);
        else
            mttkrp_y_kernel<double><<<grid, NT, 0, st>>>(s, (const double*)X, A, M, ymask);
    }
    if (mode_mask & last) {
        dim3 grid((unsigned)s.mid, (unsigned)((s.dims[N - 1] + BI - 1) / BI), rt);
        if (xdt == CP_F32)
            mttkrp_z_kernel<float><<<grid, NT, 0, st>>>(s, (const float*)X, A, M);
        else
            mttkrp_z_kernel<double><<<grid, NT, 0, st>>>(s, (const double*)X, A, M);
    }
}

}  // namespace cpgn
