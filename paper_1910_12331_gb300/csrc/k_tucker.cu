// k_tucker.cu -- truncated higher-order SVD (Tucker compression) ahead of the
// CP decomposition, for ranks below the tensor's sides (Section 1; Section
// 3.5's complexity comparison assumes it): U_n = an orthonormal basis of the
// dominant r_n-dimensional eigenspace of X_(n) X_(n)^T, and the core
// G = X x_1 U_1^T x_2 ... x_N U_N^T.  CP on G (r_1 x ... x r_N) then gives
// factors B_n, and A_n = U_n B_n is a CP model of X whose error is the
// compression error plus the core's CP error.
//
//   Gram      S_n = X_(n) X_(n)^T in FP64 (X read once per mode): 32 x 32 tiles
//             of S above the diagonal, the contraction index split into slabs,
//             slab partials reduced in a fixed order.
//   Subspace  orthogonal iteration on S_n from V = S_n Omega (Omega a fixed
//             +-1 Walsh pattern): W = S V, stop when ||W - V (V^T W)||_F <=
//             1e-12 ||W||_F, else V = orthonormal basis of W by Cholesky QR
//             applied twice (V^T V = L L^T, V <- V L^-T); FP64.
//   Core      successive mode products in FP64, one output entry per thread.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "kernels.hpp"

namespace cpgn {
namespace {

constexpr int kGT = 32;  // Gram tile

// part[slab][j][j'] for the tiles (ti <= tj) of S_n: sum over the slab's range
// of the contraction index kappa = (l, c) of x[l, j, c] x[l, j', c].
template <typename TX>
__global__ void __launch_bounds__(256) unfold_gram_kernel(const TX* __restrict__ X, int64_t L, int64_t sn, int64_t Rr,
                                                          int ntile, int slabs, double* part) {
    __shared__ double xa[kGT][kGT + 1], xb[kGT][kGT + 1];
    const int pair = blockIdx.x, slab = blockIdx.y;
    // pair -> (ti, tj), ti <= tj, row-major over the upper triangle
    int ti = 0, rem = pair;
    while (rem >= ntile - ti) {
        rem -= ntile - ti;
        ++ti;
    }
    const int tj = ti + rem;
    const int64_t K = L * Rr;
    const int64_t k0 = K * slab / slabs, k1 = K * (slab + 1) / slabs;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t kc = k0; kc < k1; kc += kGT) {
        for (int e = threadIdx.x; e < kGT * kGT; e += 256) {
            // consecutive threads on consecutive addresses: along c, or along j when Rr = 1
            const int rr = Rr == 1 ? e % kGT : e / kGT, cc = Rr == 1 ? e / kGT : e % kGT;
            const int64_t kap = kc + cc;
            double va = 0.0, vb = 0.0;
            if (kap < k1) {
                const int64_t l = kap / Rr, c = kap - l * Rr;
                const int64_t ja = (int64_t)ti * kGT + rr, jb = (int64_t)tj * kGT + rr;
                if (ja < sn) va = (double)X[(l * sn + ja) * Rr + c];
                if (jb < sn) vb = (double)X[(l * sn + jb) * Rr + c];
            }
            xa[rr][cc] = va;
            xb[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int cc = 0; cc < kGT; ++cc) {
            const double a0 = xa[ty * 2][cc], a1 = xa[ty * 2 + 1][cc];
            const double b0 = xb[tx * 2][cc], b1 = xb[tx * 2 + 1][cc];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int64_t j = (int64_t)ti * kGT + ty * 2 + u, jj = (int64_t)tj * kGT + tx * 2 + v;
            if (j < sn && jj < sn) part[((int64_t)slab * sn + j) * sn + jj] = acc[u][v];
        }
}

// S[j][j'] = sum over the slabs (in order) of the partial of the upper-triangle
// tile that holds (min, max) -- both halves of S from the same sums.
__global__ void gram_reduce_kernel(const double* part, int64_t sn, int slabs, double* S) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sn * sn) return;
    int64_t j = e / sn, jj = e - j * sn;
    if (j / kGT > jj / kGT) {  // a tile below the diagonal: read the transposed one
        const int64_t t = j;
        j = jj;
        jj = t;
    }
    double acc = 0.0;
    for (int k = 0; k < slabs; ++k) acc += part[((int64_t)k * sn + j) * sn + jj];
    S[e] = acc;
}

// C (m x n) = op(A) B with op(A) = A (m x k, row-major) or A^T (A k x m).
__global__ void small_mm_kernel(const double* A, const double* B, double* C, int m, int n, int k, int transA) {
    __shared__ double as[16][17], bs[16][17];
    const int row = blockIdx.y * 16 + threadIdx.y, col = blockIdx.x * 16 + threadIdx.x;
    double acc = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
        const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
        double a = 0.0;
        if (row < m && ka < k) a = transA ? A[(int64_t)ka * m + row] : A[(int64_t)row * k + ka];
        as[threadIdx.y][threadIdx.x] = a;
        bs[threadIdx.y][threadIdx.x] = (kb < k && col < n) ? B[(int64_t)kb * n + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; ++u) acc = fma(as[threadIdx.y][u], bs[u][threadIdx.x], acc);
        __syncthreads();
    }
    if (row < m && col < n) C[(int64_t)row * n + col] = acc;
}

// Omega[j][a] = (-1)^popcount(j & a), the Walsh functions: a fixed starting
// block with orthogonal (for s a power of two) +-1 columns.
__global__ void walsh_kernel(double* O, int s, int r) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s * r) return;
    const int j = e / r, a = e % r;
    O[e] = (__popc((unsigned)(j & a)) & 1) ? -1.0 : 1.0;
}

// In place: G (r x r, SPD) = L L^T, L lower triangular (upper part zeroed);
// one block.  *bad = 1 if a pivot is not positive.
__global__ void cholesky_kernel(double* G, int r, int* bad) {
    for (int k = 0; k < r; ++k) {
        __syncthreads();
        const double d = G[(int64_t)k * r + k];
        if (!(d > 0.0)) {
            if (threadIdx.x == 0) *bad = 1;
            return;
        }
        const double l = sqrt(d);
        __syncthreads();
        for (int i = k + threadIdx.x; i < r; i += blockDim.x) G[(int64_t)i * r + k] = i == k ? l : G[(int64_t)i * r + k] / l;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)(r - k - 1) * (r - k - 1); e += blockDim.x) {
            const int i = k + 1 + (int)(e / (r - k - 1)), j = k + 1 + (int)(e % (r - k - 1));
            if (j <= i) G[(int64_t)i * r + j] -= G[(int64_t)i * r + k] * G[(int64_t)j * r + k];
        }
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x)
        if (e % r > e / r) G[e] = 0.0;
}

// V (s x r) <- V L^-T: row v solves x L^T = v by forward substitution.
__global__ void trsm_rows_kernel(double* V, const double* Lm, int s, int r) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= s) return;
    double* v = V + (int64_t)row * r;
    for (int k = 0; k < r; ++k) {
        double acc = v[k];
        for (int m = 0; m < k; ++m) acc -= v[m] * Lm[(int64_t)k * r + m];
        v[k] = acc / Lm[(int64_t)k * r + k];
    }
}

// out[0] = ||W - V M||_F^2, out[1] = ||W||_F^2 (one block, fixed order).
__global__ void subspace_residual_kernel(const double* W, const double* V, const double* M, int s, int r,
                                         double* out) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int64_t e = threadIdx.x; e < (int64_t)s * r; e += blockDim.x) {
        const int64_t j = e / r;
        const int c = (int)(e - j * r);
        double vm = 0.0;
        for (int m = 0; m < r; ++m) vm = fma(V[j * r + m], M[(int64_t)m * r + c], vm);
        const double d = W[e] - vm;
        a = fma(d, d, a);
        b = fma(W[e], W[e], b);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        out[0] = sa;
        out[1] = sb;
    }
}

// Y[(l, a, c)] = sum_j U[j][a] T[(l, j, c)]  (U: sn x r row-major).
template <typename TIN>
__global__ void mode_product_kernel(const TIN* __restrict__ T, const double* __restrict__ U, double* __restrict__ Y,
                                    int64_t L, int64_t sn, int64_t Rr, int r) {
    const int64_t total = L * r * Rr;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e % Rr, la = e / Rr;
        const int a = (int)(la % r);
        const int64_t l = la / r;
        const TIN* t = T + l * sn * Rr + c;
        double acc = 0.0;
        for (int64_t j = 0; j < sn; ++j) acc = fma(U[j * r + a], (double)t[j * Rr], acc);
        Y[e] = acc;
    }
}

// A (s x R) = U (s x r) B (r x R).
__global__ void expand_kernel(const double* U, const double* B, double* A, int64_t s, int r, int R) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s * R) return;
    const int64_t i = e / R;
    const int c = (int)(e - i * R);
    double acc = 0.0;
    for (int m = 0; m < r; ++m) acc = fma(U[i * r + m], B[(int64_t)m * R + c], acc);
    A[e] = acc;
}

}  // namespace

size_t hosvd_scratch_doubles(const Shape& s, const int* ranks, int slabs) {
    int64_t smax = 0, rmax = 0, inter = 0;
    for (int n = 0; n < s.N; ++n) {
        smax = std::max<int64_t>(smax, s.dims[n]);
        rmax = std::max<int64_t>(rmax, ranks[n]);
    }
    // the intermediate tensors of the successive products (the first is the largest)
    int64_t cur = s.total;
    for (int n = 0; n < s.N; ++n) {
        cur = cur / s.dims[n] * ranks[n];
        inter = std::max(inter, cur);
    }
    return (size_t)slabs * smax * smax + smax * smax + 3 * smax * rmax + 2 * rmax * rmax + 2 * inter + 16;
}

cp_status launch_hosvd(const Shape& s, cp_dtype xdt, const void* X, const int* ranks, double* const* U, double* core,
                       int* iters, double* scratch, int slabs, double* hbuf, cudaStream_t st) {
    int64_t smax = 0, rmax = 0;
    for (int n = 0; n < s.N; ++n) {
        smax = std::max<int64_t>(smax, s.dims[n]);
        rmax = std::max<int64_t>(rmax, ranks[n]);
    }
    double* part = scratch;
    double* S = part + (size_t)slabs * smax * smax;
    double* V = S + smax * smax;
    double* W = V + smax * rmax;
    double* O = W + smax * rmax;
    double* G = O + smax * rmax;
    double* M = G + rmax * rmax;
    double* T0 = M + rmax * rmax;
    int64_t inter = 0, cur = s.total;
    for (int n = 0; n < s.N; ++n) {
        cur = cur / s.dims[n] * ranks[n];
        inter = std::max(inter, cur);
    }
    double* T1 = T0 + inter;
    double* res = T1 + inter;
    int* dflag = (int*)(res + 4);  // set by the Cholesky factorisation on a non-positive pivot
    for (int n = 0; n < s.N; ++n) {
        const int64_t sn = s.dims[n];
        const int r = ranks[n];
        int64_t L = 1, Rr = 1;
        for (int m = 0; m < n; ++m) L *= s.dims[m];
        for (int m = n + 1; m < s.N; ++m) Rr *= s.dims[m];
        // ---- Gram of the unfolding
        const int ntile = (int)((sn + kGT - 1) / kGT);
        const dim3 gg((unsigned)(ntile * (ntile + 1) / 2), (unsigned)slabs);
        if (xdt == CP_F32)
            unfold_gram_kernel<float><<<gg, 256, 0, st>>>((const float*)X, L, sn, Rr, ntile, slabs, part);
        else
            unfold_gram_kernel<double><<<gg, 256, 0, st>>>((const double*)X, L, sn, Rr, ntile, slabs, part);
        gram_reduce_kernel<<<(unsigned)((sn * sn + 255) / 256), 256, 0, st>>>(part, sn, slabs, S);
        // ---- orthogonal iteration
        const dim3 b16(16, 16);
        auto mm = [&](const double* A, const double* B, double* C, int m, int nn, int k, int ta) {
            small_mm_kernel<<<dim3((nn + 15) / 16, (m + 15) / 16), b16, 0, st>>>(A, B, C, m, nn, k, ta);
        };
        auto orth = [&](double* Vm) -> cp_status {  // Vm <- orthonormal basis of its columns (Cholesky QR, twice)
            for (int pass = 0; pass < 2; ++pass) {
                mm(Vm, Vm, G, r, r, (int)sn, 1);
                cholesky_kernel<<<1, 256, 0, st>>>(G, r, dflag);
                trsm_rows_kernel<<<(unsigned)((sn + 127) / 128), 128, 0, st>>>(Vm, G, (int)sn, r);
            }
            return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ERR_CUDA;
        };
        walsh_kernel<<<(unsigned)((sn * r + 255) / 256), 256, 0, st>>>(O, (int)sn, r);
        mm(S, O, V, (int)sn, r, (int)sn, 0);
        if (cudaMemsetAsync(dflag, 0, sizeof(int), st) != cudaSuccess) return CP_ERR_CUDA;
        cp_status rc = orth(V);
        if (rc != CP_OK) return rc;
        int it = 0;
        for (; it < 300; ++it) {
            mm(S, V, W, (int)sn, r, (int)sn, 0);       // W = S V
            mm(V, W, M, r, r, (int)sn, 1);             // M = V^T W
            subspace_residual_kernel<<<1, 256, 0, st>>>(W, V, M, (int)sn, r, res);
            if (cudaMemcpyAsync(hbuf, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(hbuf + 2, dflag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return CP_ERR_CUDA;
            int bad = 0;
            memcpy(&bad, hbuf + 2, sizeof(int));
            if (bad) return CP_ERR_NOT_SPD;  // the block lost rank: r above the rank of X_(n)
            if (!(hbuf[0] > 1e-24 * hbuf[1])) break;  // ||W - V M|| <= 1e-12 ||W||
            if (cudaMemcpyAsync(V, W, sizeof(double) * sn * r, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return CP_ERR_CUDA;
            if ((rc = orth(V)) != CP_OK) return rc;
        }
        if (iters) iters[n] = it;
        if (cudaMemcpyAsync(U[n], V, sizeof(double) * sn * r, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return CP_ERR_CUDA;
    }
    // ---- core: successive mode products, FP64
    int64_t dims[kMaxN];
    for (int n = 0; n < s.N; ++n) dims[n] = s.dims[n];
    const void* src = X;
    bool src_x = true;
    for (int n = 0; n < s.N; ++n) {
        int64_t L = 1, Rr = 1;
        for (int m = 0; m < n; ++m) L *= dims[m];
        for (int m = n + 1; m < s.N; ++m) Rr *= dims[m];
        double* dst = n == s.N - 1 ? core : (n % 2 == 0 ? T0 : T1);
        const int64_t total = L * ranks[n] * Rr;
        const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 65535);
        if (src_x && xdt == CP_F32)
            mode_product_kernel<float><<<grid, 256, 0, st>>>((const float*)src, U[n], dst, L, dims[n], Rr, ranks[n]);
        else
            mode_product_kernel<double><<<grid, 256, 0, st>>>((const double*)src, U[n], dst, L, dims[n], Rr,
                                                              ranks[n]);
        dims[n] = ranks[n];
        src = dst;
        src_x = false;
    }
    return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ERR_CUDA;
}

void launch_tucker_expand(int64_t s, int r, int R, const double* U, const double* B, double* A, cudaStream_t st) {
    expand_kernel<<<(unsigned)((s * R + 255) / 256), 256, 0, st>>>(U, B, A, s, r, R);
}

}  // namespace cpgn
