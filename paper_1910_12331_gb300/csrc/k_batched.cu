// k_batched.cu -- many small independent order-3 CP-GN problems in one
// persistent launch.
//
// Each CTA takes problems from a global counter and runs Algorithm 1 on one of
// them at a time, entirely in its shared memory: Gram matrices and the Gamma
// set (Eq. (2.2)), the three MTTKRPs (Eq. (2.1)), the gradient of Eq. (2.3),
// the varying lambda of Section 3.2, the block-Jacobi preconditioner
// (Gamma^(n,n) + lambda I)^{-1} of Section 3.3 (Gauss-Jordan in FP64), and the
// CG solve of Algorithm 2 with the implicit matvec of Eq. (3.4) (reassociated
// through Y^(p) = A^(p)^T W^(p)); CTA-local barriers only, no grid barrier.
// Vectors, factors and Gram products are FP32 in shared memory; dot products,
// norms, alpha, beta and the factor master copy are FP64 (per-thread FP32
// partials, summed as error-free FP32 pairs within each warp, then in FP64
// across the warps by one warp).  The stop test is the direct
// relative residual ||X - [[A]]||_F / ||X||_F with FP32 reconstruction and
// compensated FP32 partial sums, which resolves the target r <= 1e-6 of these
// problems.
//
// Shared memory per problem (floats): 6 (s_1 + s_2 + s_3) R for A, W, R, Z, V,
// Q; 21 R^2 for the Grams, the Gamma set, the inverses, Y and T; plus R^2 + R
// doubles for the elimination and the reduction scratch.  The launch sizes it
// for the largest problem of the batch.
#include <math.h>

#include <algorithm>
#include <vector>

#include "kernels.hpp"

namespace cpgn {
namespace {

// Threads per CTA: a template parameter BT (128, 256 or 384), chosen per plan by
// the autotuner, or set by cp_batch_plan_configure (default 256).
constexpr size_t kBatchSmemMax = 220 * 1024;

struct BProb {
    int s[3];
    int R;
    const float* X;
    double* A[3];
    double lam, lam_lo, lam_hi, mu;
    int reg, lam_fixed;        // damping lam diag(J^T J) (1) or lam I (0); constant lambda
    double armijo_c, armijo_beta;
    int armijo_max, pad;
};

struct BRes {
    int status, iters, cg_iters, converged, breakdowns, backtracks;
    double rel_residual, lam;
};

struct BArgs {
    const BProb* probs;
    BRes* res;
    int nprob;
    int* counter;
    const int* order;  // the order in which the CTAs take the problems
    double eps_cg;
    int cg_max;
    int max_iters;
    double target;
};

// Sums over the CTA of up to four FP32 values per thread: error-free FP32 pairs within each warp
// (Knuth's two-sum; the FP32 units, not GB300's slow FP64 pipe, do the thread-level work), then
// FP64 across the warps in warp 0 alone (the shuffle levels that would only add zeros skipped),
// which also forms the scalars the step needs from the sums: fin(r, lane) runs on every lane of
// warp 0, lanes 0..3 holding the full sums, and lane 0's r comes back to every thread through
// red[64..].  All threads call.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}
// sqrt(r[0]) + sqrt(r[1]) + sqrt(r[2]), the three roots taken at once by lanes 0, 1 and 2 (a warp
// instruction costs the FP64 pipe the same for one lane as for all); called by a whole warp.
__device__ __forceinline__ double sqrt3_sum(const double (&r)[8], int l) {
    const double sq = sqrt(l == 0 ? r[0] : (l == 1 ? r[1] : r[2]));
    return (__shfl_sync(0xffffffffu, sq, 0) + __shfl_sync(0xffffffffu, sq, 1)) + __shfl_sync(0xffffffffu, sq, 2);
}

template <int BT, int K, typename Fin>
__device__ __forceinline__ void bsum_k(const float (&v)[K], double* red, double (&out)[8], Fin fin) {
    constexpr int NW = BT / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    float h[K], lo[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        h[q] = v[q];
        lo[q] = 0.f;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float oh = __shfl_xor_sync(0xffffffffu, h[q], o), ol = __shfl_xor_sync(0xffffffffu, lo[q], o);
            float t, e;
            two_sum_f(h[q], oh, t, e);
            h[q] = t;
            lo[q] += ol + e;
        }
    }
    __syncthreads();  // red may still be read from the previous reduction
    if (l == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) red[q * NW + w] = (double)h[q] + (double)lo[q];
    }
    __syncthreads();
    if (w == 0) {
        constexpr int P = NW <= 4 ? 4 : (NW <= 8 ? 8 : (NW <= 16 ? 16 : 32));  // lanes >= NW hold zeros
        double t[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            t[q] = l < NW ? red[q * NW + l] : 0.0;
#pragma unroll
            for (int o = P / 2; o; o >>= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
        }
        double r[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) r[q] = q < K ? t[q] : 0.0;
        fin(r, l);
        if (l == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) red[64 + q] = r[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = red[64 + q];
}

struct Smem {
    int s[3], roff[3], S, R;
    float *A, *W, *Rv, *Z, *V, *Q;  // S x R each (rows of mode n start at roff[n])
    float *Sg, *Gm, *Pi, *Yb, *Tb;  // 3 R^2, 9 R^2, 3 R^2, 3 R^2, 3 R^2
    double *gj, *red;               // R^2 + R, 96
};

// v[n] for a run-time n by selects, so that the arrays of Smem stay in registers
__device__ __forceinline__ int pick3(const int (&v)[3], int n) { return n == 0 ? v[0] : (n == 1 ? v[1] : v[2]); }

__device__ __forceinline__ void carve(Smem& m, unsigned char* base, const BProb& pb) {
    m.R = pb.R;
    m.roff[0] = 0;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        m.s[n] = pb.s[n];
        if (n) m.roff[n] = m.roff[n - 1] + pb.s[n - 1];
    }
    m.S = m.roff[2] + pb.s[2];
    const int SR = m.S * m.R, RR = m.R * m.R;
    double* d = reinterpret_cast<double*>(base);
    m.red = d;
    m.gj = d + 96;
    float* f = reinterpret_cast<float*>(m.gj + RR + m.R);
    m.A = f;
    m.W = f + SR;
    m.Rv = f + 2 * SR;
    m.Z = f + 3 * SR;
    m.V = f + 4 * SR;
    m.Q = f + 5 * SR;
    m.Sg = f + 6 * SR;
    m.Gm = m.Sg + 3 * RR;
    m.Pi = m.Gm + 9 * RR;
    m.Yb = m.Pi + 3 * RR;
    m.Tb = m.Yb + 3 * RR;
}

// S^(n) = A^(n)^T A^(n), then Gamma^(n,p) = S^(q) (q the third mode) and Gamma^(n,n) = S^(a) * S^(b).
template <int BT>
__device__ __forceinline__ void gram_gamma(const Smem& m) {
    const int R = m.R, RR = R * R;
    for (int e = threadIdx.x; e < 3 * RR; e += BT) {
        const int n = e / RR, r = (e % RR) / R, z = e % R;
        const float* a = m.A + pick3(m.roff, n) * R;
        float acc = 0.f;
#pragma unroll 4
        for (int i = 0; i < pick3(m.s, n); ++i) acc = fmaf(a[i * R + r], a[i * R + z], acc);
        m.Sg[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * RR; e += BT) {
        const int np = e / RR, q = e % RR, n = np / 3, p = np % 3;
        float g;
        if (n == p)
            g = m.Sg[((n + 1) % 3) * RR + q] * m.Sg[((n + 2) % 3) * RR + q];
        else
            g = m.Sg[(3 - n - p) * RR + q];
        m.Gm[e] = g;
    }
    __syncthreads();
}

// ---- The three MTTKRPs and the residual with the lanes of a warp over k, the contiguous index
// of X: rows x[i, j, :] are read coalesced, and the loads of successive rows do not depend on each
// other, so several are in flight per warp (X is read from global memory, where a warp that waits
// for one load at a time is bound by the memory latency).  Accumulators over the ranks live in
// registers, MR >= R of them (a template bucket: 8, 16, 24 or 32).

// Mode 1 (mode = 0) or mode 2 (mode = 1), one warp per pair of output rows q, q + 1:
//   M1[q][r] = sum_k a3[k][r] sum_j x[q, j, k] a2[j][r],  M2[q][r] = sum_k a3[k][r] sum_i x[i, q, k] a1[i][r];
// the inner sums per lane (its k; each factor value loaded serves both rows), then a3[k][r] times
// them summed over the lanes by shuffles; lane r keeps the sum for rank r.
template <int BT, int MR>
__device__ __forceinline__ void mttkrp_m12(const Smem& m, const float* __restrict__ X, float* out, int mode) {
    const int R = m.R, s1 = m.s[0], s2 = m.s[1], s3 = m.s[2];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const float *a1 = m.A, *a2 = m.A + m.roff[1] * R, *a3t = out + m.roff[2] * R;  // a3t[r][k] = a3[k][r]
    const int nrow = mode == 0 ? s1 : s2, nin = mode == 0 ? s2 : s1;
    const float* fac = mode == 0 ? a2 : a1;
    const int64_t step = mode == 0 ? (int64_t)s3 : (int64_t)s2 * s3;  // X distance of successive summed rows
    const int64_t qstep = mode == 0 ? (int64_t)s2 * s3 : (int64_t)s3;  // X distance of successive output rows
    for (int q = 2 * w; q < nrow; q += 2 * (BT / 32)) {
        const bool two = q + 1 < nrow;
        const float* xq = X + q * qstep;
        const float* xq1 = two ? xq + qstep : xq;
        float mine0 = 0.f, mine1 = 0.f;
        for (int k0 = 0; k0 < s3; k0 += 32) {
            const int k = k0 + l;
            const bool kon = k < s3;
            float t0[MR], t1[MR];
#pragma unroll
            for (int r = 0; r < MR; ++r) t0[r] = t1[r] = 0.f;
#pragma unroll (BT > 256 ? 4 : 8)
            for (int pp = 0; pp < nin; ++pp) {
                const float x0 = kon ? __ldg(xq + pp * step + k) : 0.f;
                const float x1 = kon ? __ldg(xq1 + pp * step + k) : 0.f;
                const float* fr = fac + pp * R;
#pragma unroll
                for (int r = 0; r < MR; ++r)
                    if (r < R) {
                        const float f = fr[r];
                        t0[r] = fmaf(x0, f, t0[r]);
                        t1[r] = fmaf(x1, f, t1[r]);
                    }
            }
            const int kc = kon ? k : 0;
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                if (r < R) {
                    const float c = a3t[r * s3 + kc];
                    float v0 = kon ? t0[r] * c : 0.f, v1 = kon ? t1[r] * c : 0.f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                    }
                    if (l == r) {
                        mine0 += v0;
                        mine1 += v1;
                    }
                }
            }
        }
        if (l < R) {
            out[(pick3(m.roff, mode) + q) * R + l] = mine0;
            if (two) out[(pick3(m.roff, mode) + q + 1) * R + l] = mine1;
        }
    }
}

// Mode 3: M3[k][r] = sum_i a1[i][r] sum_j x[i, j, k] a2[j][r], lane = k, two rows i at a time (each
// factor value loaded serves both); the rows i split over up to four groups of warps whose partials
// (in W .. V, free at this point of the iteration) are added in a fixed order.
template <int BT, int MR>
__device__ __forceinline__ void mttkrp_m3(const Smem& m, const float* __restrict__ X, float* out) {
    const int R = m.R, s1 = m.s[0], s2 = m.s[1], s3 = m.s[2];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const float *a1 = m.A, *a2 = m.A + m.roff[1] * R;
    const int nkb = (s3 + 31) / 32;
    const int ig_n = max(1, min(4, (BT / 32) / nkb));
    const int64_t istep = (int64_t)s2 * s3;
    for (int task = w; task < nkb * ig_n; task += BT / 32) {
        const int kb = task % nkb, ig = task / nkb;
        const int k = kb * 32 + l;
        const bool kon = k < s3;
        const int i0 = (int)((int64_t)s1 * ig / ig_n), i1 = (int)((int64_t)s1 * (ig + 1) / ig_n);
        float acc[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) acc[r] = 0.f;
        for (int i = i0; i < i1; i += 2) {
            const bool two = i + 1 < i1;
            const float* xi = X + i * istep + (kon ? k : 0);
            const float* xi1 = two ? xi + istep : xi;
            float t0[MR], t1[MR];
#pragma unroll
            for (int r = 0; r < MR; ++r) t0[r] = t1[r] = 0.f;
#pragma unroll (BT > 256 ? 4 : 8)
            for (int j = 0; j < s2; ++j) {
                const float x0 = kon ? __ldg(xi + (int64_t)j * s3) : 0.f;
                const float x1 = kon ? __ldg(xi1 + (int64_t)j * s3) : 0.f;
                const float* fr = a2 + j * R;
#pragma unroll
                for (int r = 0; r < MR; ++r)
                    if (r < R) {
                        const float f = fr[r];
                        t0[r] = fmaf(x0, f, t0[r]);
                        t1[r] = fmaf(x1, f, t1[r]);
                    }
            }
            const float* fa = a1 + i * R;
            const float* fb = a1 + (two ? i + 1 : i) * R;
#pragma unroll
            for (int r = 0; r < MR; ++r)
                if (r < R) {
                    acc[r] = fmaf(fa[r], t0[r], acc[r]);
                    if (two) acc[r] = fmaf(fb[r], t1[r], acc[r]);
                }
        }
        float* part = m.W + (size_t)ig * s3 * R;
        if (kon) {
#pragma unroll
            for (int r = 0; r < MR; ++r)
                if (r < R) part[k * R + r] = acc[r];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s3 * R; e += BT) {
        float v = 0.f;
        for (int g = 0; g < ig_n; ++g) v += m.W[(size_t)g * s3 * R + e];
        out[m.roff[2] * R + e] = v;
    }
}

// M^(n) for all modes into out (S x R).
template <int BT, int MR>
__device__ __forceinline__ void mttkrp3_r(const Smem& m, const float* __restrict__ X, float* out) {
    {  // a3 transposed (R x s3) for modes 1 and 2, in the rows of mode 3 of out, which mode 3 writes last
        const int R = m.R, s3 = m.s[2];
        float* a3t = out + m.roff[2] * R;
        for (int e = threadIdx.x; e < s3 * R; e += BT) {
            const int k = e / R, r = e - k * R;
            a3t[r * s3 + k] = m.A[m.roff[2] * R + e];
        }
        __syncthreads();
    }
    mttkrp_m12<BT, MR>(m, X, out, 0);
    mttkrp_m12<BT, MR>(m, X, out, 1);
    mttkrp_m3<BT, MR>(m, X, out);
    __syncthreads();
}

template <int BT>
__device__ __forceinline__ void mttkrp3(const Smem& m, const float* __restrict__ X, float* out) {
    if (m.R <= 8)
        mttkrp3_r<BT, 8>(m, X, out);
    else if (m.R <= 16)
        mttkrp3_r<BT, 16>(m, X, out);
    else if (m.R <= 24)
        mttkrp3_r<BT, 24>(m, X, out);
    else
        mttkrp3_r<BT, 32>(m, X, out);
}

// ||X - [[A]]||_F^2: a warp per row (i, j), lanes over k; compensated FP32 partials, then the block
// sum.  A lane's values of x in a row (up to eight) are loaded while the previous row is
// reconstructed, and the products a1[i][r] a2[j][r] of the row are formed once, in registers.
template <int BT, int MR>
__device__ __forceinline__ double resid2_r(const Smem& m, const float* __restrict__ X) {
    const int R = m.R, s1 = m.s[0], s2 = m.s[1], s3 = m.s[2];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const float *a1 = m.A, *a2 = m.A + m.roff[1] * R;
    // a3 transposed (R x s3) into the mode-3 rows of Q, free where the residual is taken: the lanes
    // (successive k) then read successive words, free of the bank conflicts of a3[k][r]
    float* a3t = m.Q + m.roff[2] * R;
    for (int e = threadIdx.x; e < s3 * R; e += BT) {
        const int k = e / R, r = e - k * R;
        a3t[r * s3 + k] = m.A[m.roff[2] * R + e];
    }
    __syncthreads();
    float sum = 0.f, comp = 0.f;
    // the next row's values of x are loaded while this row is reconstructed
    float xn[8];
    auto load = [&](int ij) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            xn[u] = ij < s1 * s2 && l + 32 * u < s3 ? __ldg(X + (int64_t)ij * s3 + l + 32 * u) : 0.f;
    };
    load(w);
    for (int ij = w; ij < s1 * s2; ij += (BT / 32)) {
        const int i = ij / s2, j = ij % s2;
        float xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = xn[u];
        load(ij + (BT / 32));
        float wr[MR];
#pragma unroll
        for (int r = 0; r < MR; ++r) wr[r] = r < R ? a1[i * R + r] * a2[j * R + r] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = l + 32 * u;
            if (k < s3) {
                float rec = 0.f;
#pragma unroll
                for (int r = 0; r < MR; ++r)
                    if (r < R) rec = fmaf(wr[r], a3t[r * s3 + k], rec);
                const float e = xv[u] - rec;
                const float y = fmaf(e, e, -comp);  // Kahan
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            }
        }
    }
    const float v[2] = {sum, -comp};
    double o[8];
    bsum_k<BT, 2>(v, m.red, o, [](double (&r)[8], int) { r[0] += r[1]; });
    return o[0];
}

template <int BT>
__device__ __forceinline__ double resid2(const Smem& m, const float* __restrict__ X) {
    if (m.R <= 8) return resid2_r<BT, 8>(m, X);
    if (m.R <= 16) return resid2_r<BT, 16>(m, X);
    if (m.R <= 24) return resid2_r<BT, 24>(m, X);
    return resid2_r<BT, 32>(m, X);
}

// Row products of the CG in register tiles: a thread forms 4 rows (of one mode) x 2 columns
// (z and z + ch, ch = ceil(R/2)) of the S x R result, so that each value it loads from shared
// memory serves 2 or 4 multiply-adds.  Every output element keeps its own accumulation chain.
struct RowTile {
    int n, row0, nr, z0, z1;  // mode, first row, rows in the tile (1..4), columns (z1 = z0 if none)
    bool z1on;
};
__device__ __forceinline__ int tiles_of(const Smem& m) {
    const int ch = (m.R + 1) >> 1;
    return (((m.s[0] + 3) >> 2) + ((m.s[1] + 3) >> 2) + ((m.s[2] + 3) >> 2)) * ch;
}
__device__ __forceinline__ RowTile tile_at(const Smem& m, int t) {
    const int ch = (m.R + 1) >> 1;
    const int t0 = ((m.s[0] + 3) >> 2) * ch, t1 = t0 + ((m.s[1] + 3) >> 2) * ch;
    RowTile o;
    o.n = t >= t1 ? 2 : (t >= t0 ? 1 : 0);
    const int tl = t - (o.n == 2 ? t1 : (o.n == 1 ? t0 : 0));
    const int rt = tl / ch, ct = tl - rt * ch;
    o.row0 = pick3(m.roff, o.n) + 4 * rt;
    o.nr = min(4, pick3(m.s, o.n) - 4 * rt);
    o.z0 = ct;
    o.z1on = ct + ch < m.R;
    o.z1 = o.z1on ? ct + ch : ct;
    return o;
}

// out = in P_inv^(n) per mode (rows of mode n times the symmetric R x R block); per element two
// chains, even and odd r.
template <int BT>
__device__ __forceinline__ void apply_pinv(const Smem& m, const float* in, float* out) {
    const int R = m.R, nt = tiles_of(m);
    for (int t = threadIdx.x; t < nt; t += BT) {
        const RowTile tl = tile_at(m, t);
        const float* P = m.Pi + tl.n * R * R;
        const float* x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = in + (tl.row0 + min(k, tl.nr - 1)) * R;
        float e0[4][2], e1[4][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) e0[k][0] = e0[k][1] = e1[k][0] = e1[k][1] = 0.f;
        int r = 0;
        for (; r + 1 < R; r += 2) {
            const float pa0 = P[r * R + tl.z0], pa1 = P[r * R + tl.z1];
            const float pb0 = P[(r + 1) * R + tl.z0], pb1 = P[(r + 1) * R + tl.z1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float xa = x[k][r], xb = x[k][r + 1];
                e0[k][0] = fmaf(xa, pa0, e0[k][0]);
                e0[k][1] = fmaf(xa, pa1, e0[k][1]);
                e1[k][0] = fmaf(xb, pb0, e1[k][0]);
                e1[k][1] = fmaf(xb, pb1, e1[k][1]);
            }
        }
        if (r < R) {
            const float pa0 = P[r * R + tl.z0], pa1 = P[r * R + tl.z1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                e0[k][0] = fmaf(x[k][r], pa0, e0[k][0]);
                e0[k][1] = fmaf(x[k][r], pa1, e0[k][1]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < tl.nr) {
                out[(tl.row0 + k) * R + tl.z0] = e0[k][0] + e1[k][0];
                if (tl.z1on) out[(tl.row0 + k) * R + tl.z1] = e0[k][1] + e1[k][1];
            }
    }
    __syncthreads();
}

// Q = (J^T J + lam D) W via Y^(p) = A^(p)^T W^(p), T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p),
// Q^(n) = lam W^(n) D^(n) + W^(n) Gamma^(n,n) + A^(n) T^(n)^T, D^(n) = I or diag(Gamma^(n,n)).
// Y and T are kept transposed (Yb[p][r][z] = Y^(p)[z][r], Tb[n][r][z] = T^(n)[z][r]; the blocks
// Gamma^(n,p) are symmetric), so that the tiled Q reads A^(n) T^(n)^T's right factor by rows.
template <int BT>
__device__ __forceinline__ void matvec(const Smem& m, float lam, bool diag) {
    const int R = m.R, RR = R * R;
    {  // a thread forms Yb[p][r][z] for r in {r0, r0 + ch}, z in {z0, z0 + ch}, ch = ceil(R/2)
        const int ch = (R + 1) >> 1, cc = ch * ch;
        for (int t = threadIdx.x; t < 3 * cc; t += BT) {
            const int p = t / cc, tr = t - p * cc, rr = tr / ch, zz = tr - rr * ch;
            const bool r1on = rr + ch < R, z1on = zz + ch < R;
            const int r0 = rr, r1 = r1on ? rr + ch : rr, z0 = zz, z1 = z1on ? zz + ch : zz;
            const float* a = m.A + pick3(m.roff, p) * R;
            const float* w = m.W + pick3(m.roff, p) * R;
            float c0[4], c1[4];  // (r0,z0) (r0,z1) (r1,z0) (r1,z1); two chains each (even and odd i)
#pragma unroll
            for (int u = 0; u < 4; ++u) c0[u] = c1[u] = 0.f;
            const int sp = pick3(m.s, p);
            int i = 0;
            for (; i + 1 < sp; i += 2) {
                const float az0 = a[i * R + z0], az1 = a[i * R + z1], w0 = w[i * R + r0], w1 = w[i * R + r1];
                const float bz0 = a[(i + 1) * R + z0], bz1 = a[(i + 1) * R + z1];
                const float v0 = w[(i + 1) * R + r0], v1 = w[(i + 1) * R + r1];
                c0[0] = fmaf(az0, w0, c0[0]);
                c0[1] = fmaf(az1, w0, c0[1]);
                c0[2] = fmaf(az0, w1, c0[2]);
                c0[3] = fmaf(az1, w1, c0[3]);
                c1[0] = fmaf(bz0, v0, c1[0]);
                c1[1] = fmaf(bz1, v0, c1[1]);
                c1[2] = fmaf(bz0, v1, c1[2]);
                c1[3] = fmaf(bz1, v1, c1[3]);
            }
            if (i < sp) {
                const float az0 = a[i * R + z0], az1 = a[i * R + z1], w0 = w[i * R + r0], w1 = w[i * R + r1];
                c0[0] = fmaf(az0, w0, c0[0]);
                c0[1] = fmaf(az1, w0, c0[1]);
                c0[2] = fmaf(az0, w1, c0[2]);
                c0[3] = fmaf(az1, w1, c0[3]);
            }
            float* y = m.Yb + p * RR;
            y[r0 * R + z0] = c0[0] + c1[0];
            if (z1on) y[r0 * R + z1] = c0[1] + c1[1];
            if (r1on) y[r1 * R + z0] = c0[2] + c1[2];
            if (r1on && z1on) y[r1 * R + z1] = c0[3] + c1[3];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * RR; e += BT) {
        const int n = e / RR, q = e % RR;
        float t = 0.f;
        for (int p = 0; p < 3; ++p)
            if (p != n) t = fmaf(m.Gm[(n * 3 + p) * RR + q], m.Yb[p * RR + q], t);
        m.Tb[e] = t;
    }
    __syncthreads();
    const int nt = tiles_of(m);
    for (int t = threadIdx.x; t < nt; t += BT) {
        const RowTile tl = tile_at(m, t);
        const float* G = m.Gm + (tl.n * 3 + tl.n) * RR;
        const float* T = m.Tb + tl.n * RR;
        const float* w[4];
        const float* a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int row = tl.row0 + min(k, tl.nr - 1);
            w[k] = m.W + row * R;
            a[k] = m.A + row * R;
        }
        const float d0 = diag ? lam * G[tl.z0 * R + tl.z0] : lam, d1 = diag ? lam * G[tl.z1 * R + tl.z1] : lam;
        float c1[4][2], c2[4][2];  // W Gamma + lam D W and A T^T: two chains per element
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c1[k][0] = d0 * w[k][tl.z0];
            c1[k][1] = d1 * w[k][tl.z1];
            c2[k][0] = c2[k][1] = 0.f;
        }
#pragma unroll 2
        for (int r = 0; r < R; ++r) {
            const float g0 = G[r * R + tl.z0], g1 = G[r * R + tl.z1];
            const float t0 = T[r * R + tl.z0], t1 = T[r * R + tl.z1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float wv = w[k][r], av = a[k][r];
                c1[k][0] = fmaf(wv, g0, c1[k][0]);
                c1[k][1] = fmaf(wv, g1, c1[k][1]);
                c2[k][0] = fmaf(av, t0, c2[k][0]);
                c2[k][1] = fmaf(av, t1, c2[k][1]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < tl.nr) {
                m.Q[(tl.row0 + k) * R + tl.z0] = c1[k][0] + c2[k][0];
                if (tl.z1on) m.Q[(tl.row0 + k) * R + tl.z1] = c1[k][1] + c2[k][1];
            }
    }
    __syncthreads();
}

// P_inv^(n) = (Gamma^(n,n) + lam D^(n))^{-1}, D^(n) = I or diag(Gamma^(n,n)), Gauss-Jordan in
// FP64 (pivots = squared Cholesky diagonals); returns false if a pivot is not positive.
template <int BT>
__device__ __forceinline__ bool precond(const Smem& m, double lam, bool diag) {
    const int R = m.R, RR = R * R;
    __shared__ int bad;
    __shared__ double inv_s;
    if (threadIdx.x == 0) bad = 0;
    for (int n = 0; n < 3; ++n) {
        const float* G = m.Gm + (n * 3 + n) * RR;
        double* B = m.gj;
        double* f = m.gj + RR;
        for (int e = threadIdx.x; e < RR; e += BT)
            B[e] = (double)G[e] + ((e / R) == (e % R) ? lam * (diag ? (double)G[e] : 1.0) : 0.0);
        __syncthreads();
        for (int j = 0; j < R; ++j) {
            if (threadIdx.x == 0) {
                double p = B[j * R + j];
                if (!(p > 0.0)) {
                    bad = 1;
                    p = 1.0;
                }
                inv_s = 1.0 / p;
            }
            for (int i = threadIdx.x; i < R; i += BT) f[i] = B[i * R + j];
            __syncthreads();
            const double inv = inv_s;
            for (int k = threadIdx.x; k < R; k += BT) B[j * R + k] = k == j ? inv : B[j * R + k] * inv;
            __syncthreads();
            for (int e = threadIdx.x; e < RR; e += BT) {
                const int i = e / R, k = e % R;
                if (i != j) B[e] = k == j ? -f[i] * inv : B[e] - f[i] * B[j * R + k];
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < RR; e += BT) m.Pi[n * RR + e] = (float)B[e];
        __syncthreads();
    }
    return bad == 0;
}

template <int BT>
__global__ void __launch_bounds__(BT, 1) batched_gn_kernel(BArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int prob_s;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) prob_s = atomicAdd(args.counter, 1);
        __syncthreads();
        if (prob_s >= args.nprob) break;
        const int pi = args.order[prob_s];
        const BProb pb = args.probs[pi];
        Smem m;
        carve(m, smem, pb);
        const int R = m.R, SR = m.S * R;
        const float* __restrict__ X = pb.X;
        // FP32 working copy of the factors (the FP64 master stays in global memory)
        for (int e = threadIdx.x; e < SR; e += BT) {
            const int row = e / R, r = e % R;
            const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
            m.A[e] = (float)pb.A[n][(row - pick3(m.roff, n)) * R + r];
        }
        // ||X||^2
        float xs = 0.f;
        const int64_t tot = (int64_t)m.s[0] * m.s[1] * m.s[2];
        for (int64_t e = threadIdx.x; e < tot; e += BT) {
            const float x = __ldg(X + e);
            xs = fmaf(x, x, xs);
        }
        double nx2;
        {
            const float v[1] = {xs};
            double o[8];
            bsum_k<BT, 1>(v, m.red, o, [](double (&)[8], int) {});
            nx2 = o[0];
        }
        double lam = pb.lam;
        const bool diag = pb.reg == CP_REG_DIAG;
        int dir = 0, status = CP_OK, it = 0, cg_total = 0, converged = 0, breakdowns = 0, backtracks = 0;
        double rel = -1.0;
        for (;; ++it) {
            __syncthreads();
            gram_gamma<BT>(m);
            const double r2 = fmax(resid2<BT>(m, X), 0.0);  // ||X - [[A]]||^2 at the entry point
            rel = sqrt(r2 / nx2);
            if (rel <= args.target) {
                converged = 1;
                break;
            }
            if (it >= args.max_iters) break;
            if (it > 0 && !pb.lam_fixed) {  // varying lambda (Section 3.2), thresholds inclusive
                if (dir == 0) {
                    if (lam / pb.mu < pb.lam_lo) {
                        dir = 1;
                        lam *= pb.mu;
                    } else {
                        lam /= pb.mu;
                    }
                } else {
                    if (lam * pb.mu > pb.lam_hi) {
                        dir = 0;
                        lam /= pb.mu;
                    } else {
                        lam *= pb.mu;
                    }
                }
            }
            // R = -G = M - A Gamma^(n,n)
            mttkrp3<BT>(m, X, m.Q);
            float g0 = 0.f, g1 = 0.f, g2 = 0.f;  // per-mode sums (scalars: no local memory)
            for (int e = threadIdx.x; e < SR; e += BT) {
                const int row = e / R, z = e % R;
                const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
                const float* G = m.Gm + (n * 3 + n) * R * R;
                const float* a = m.A + row * R;
                float acc = m.Q[e];
#pragma unroll 4
                for (int r = 0; r < R; ++r) acc = fmaf(-a[r], G[r * R + z], acc);
                m.Rv[e] = acc;
                m.V[e] = 0.f;
                const float sq = acc * acc;
                if (n == 0) g0 += sq;
                else if (n == 1) g1 += sq;
                else g2 += sq;
            }
            double gsum;
            {
                const float v[3] = {g0, g1, g2};
                double o[8];
                bsum_k<BT, 3>(v, m.red, o, [](double (&r)[8], int l) { r[3] = sqrt3_sum(r, l); });
                gsum = o[3];
            }
            if (!(gsum == gsum) || isinf(gsum)) {
                status = CP_ERR_NONFINITE;
                break;
            }
            if (!precond<BT>(m, lam, diag)) {
                status = CP_ERR_NOT_SPD;
                break;
            }
            apply_pinv<BT>(m, m.Rv, m.Z);
            float rzp = 0.f;
            for (int e = threadIdx.x; e < SR; e += BT) {
                m.W[e] = m.Z[e];
                rzp = fmaf(m.Rv[e], m.Z[e], rzp);
            }
            double rz;
            {
                const float v[1] = {rzp};
                double o[8];
                bsum_k<BT, 1>(v, m.red, o, [](double (&)[8], int) {});
                rz = o[0];
            }
            double rnorm = gsum;
            double arz = 0.0;  // sum_k alpha_k <R_k, Z_k> = <-G, V> (PCG from V = 0)
            int k = 0;
            for (; k < args.cg_max && rnorm > args.eps_cg * gsum; ++k) {
                matvec<BT>(m, (float)lam, diag);
                float wqp = 0.f;
                for (int e = threadIdx.x; e < SR; e += BT) wqp = fmaf(m.W[e], m.Q[e], wqp);
                double o[8];
                {
                    const float v[1] = {wqp};
                    bsum_k<BT, 1>(v, m.red, o, [rz](double (&r)[8], int) { r[1] = r[0] > 0.0 ? rz / r[0] : 0.0; });
                }
                const double wq = o[0];
                if (!(wq > 0.0)) {  // FP32 curvature lost: end CG with the update found so far
                    ++breakdowns;
                    break;
                }
                const float alpha = (float)o[1];
                arz += (double)alpha * rz;
                for (int e = threadIdx.x; e < SR; e += BT) {
                    m.V[e] = fmaf(alpha, m.W[e], m.V[e]);
                    m.Rv[e] = fmaf(-alpha, m.Q[e], m.Rv[e]);
                }
                __syncthreads();
                apply_pinv<BT>(m, m.Rv, m.Z);
                float rzn = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f;
                for (int e = threadIdx.x; e < SR; e += BT) {
                    const int row = e / R;
                    const float rv = m.Rv[e];
                    rzn = fmaf(rv, m.Z[e], rzn);
                    if (row >= m.roff[2]) q2 = fmaf(rv, rv, q2);
                    else if (row >= m.roff[1]) q1 = fmaf(rv, rv, q1);
                    else q0 = fmaf(rv, rv, q0);
                }
                {
                    const float v[4] = {q0, q1, q2, rzn};
                    bsum_k<BT, 4>(v, m.red, o, [rz](double (&r)[8], int l) {
                        r[4] = sqrt3_sum(r, l);
                        r[5] = r[3] / rz;
                    });
                }
                const double rzd = o[3];
                rnorm = o[4];
                const float beta = (float)o[5];
                rz = rzd;
                for (int e = threadIdx.x; e < SR; e += BT) m.W[e] = fmaf(beta, m.W[e], m.Z[e]);
                __syncthreads();
            }
            cg_total += k;
            if (status != CP_OK) break;
            // Step-size control by Armijo's condition (Section 5): the first t in 1, beta,
            // beta^2, ... with f(A + t V) <= f(A) + c t <G, V>, f = 1/2 ||X - [[A]]||^2 (the
            // residual of the stop test), <G, V> from the CG recurrences; none: no update.
            double step = 1.0;
            if (pb.armijo_c > 0.0) {
                // relaxed by the accuracy of the FP32 evaluation of f (2 R 2^-24 ||X||^2), below
                // which a trial cannot be told from the entry point
                const double f0 = 0.5 * r2, slope = -arz, tol_f = 2.0 * R * 0x1p-24 * nx2;
                double t = 1.0;
                step = 0.0;
                for (int kk = 0; kk <= pb.armijo_max; ++kk, t *= pb.armijo_beta) {
                    for (int e = threadIdx.x; e < SR; e += BT) {
                        const int row = e / R, r = e % R;
                        const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
                        m.A[e] = (float)(pb.A[n][(row - pick3(m.roff, n)) * R + r] + t * (double)m.V[e]);
                    }
                    __syncthreads();
                    if (0.5 * fmax(resid2<BT>(m, X), 0.0) <= f0 + pb.armijo_c * t * slope + tol_f) {
                        step = t;
                        break;
                    }
                    ++backtracks;
                }
            }
            // A += t V (FP64 master, FP32 copy)
            for (int e = threadIdx.x; e < SR; e += BT) {
                const int row = e / R, r = e % R;
                const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
                double* a = pb.A[n] + (row - pick3(m.roff, n)) * R + r;
                const double v = *a + step * (double)m.V[e];
                *a = v;
                m.A[e] = (float)v;
            }
        }
        if (threadIdx.x == 0) {
            BRes out;
            out.status = status;
            out.iters = it;
            out.cg_iters = cg_total;
            out.converged = converged;
            out.breakdowns = breakdowns;
            out.backtracks = backtracks;
            out.rel_residual = rel;
            out.lam = lam;
            args.res[pi] = out;
        }
    }
}

size_t smem_bytes(int S, int R) {
    return (size_t)(96 + R * R + R) * sizeof(double) + (size_t)(6 * S * R + 21 * R * R) * sizeof(float);
}

}  // namespace
}  // namespace cpgn

namespace cpgn {

// A prepared batch: device copies of the problem descriptors, the results and
// the work counter, and the launch shape.  Launching it enqueues a counter reset
// and one kernel launch on the caller's stream, nothing else, so a launch can be
// captured into a CUDA graph and replayed.
struct BatchPlan {
    int device = 0, nprob = 0, threads = 256, grid = 0;
    size_t smem = 0;
    BProb* dp = nullptr;
    BRes* dr = nullptr;
    int* dc = nullptr;
    int* dorder = nullptr;  // [2][nprob]: the given order, then largest work first
    int order = 0;          // which of the two the launches use
    std::vector<BProb> hp;
    double eps_cg = 0.0, target = 0.0;
    int cg_max = 0, max_iters = 0;
};

namespace {

constexpr int kVariants[3] = {128, 256, 384};

cudaError_t set_attr(int threads, size_t smem) {
    switch (threads) {
        case 128: return cudaFuncSetAttribute(batched_gn_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 256: return cudaFuncSetAttribute(batched_gn_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        default: return cudaFuncSetAttribute(batched_gn_kernel<384>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
}
cudaError_t occupancy(int threads, size_t smem, int* per_sm) {
    switch (threads) {
        case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batched_gn_kernel<128>, 128, smem);
        case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batched_gn_kernel<256>, 256, smem);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batched_gn_kernel<384>, 384, smem);
    }
}
void launch(int threads, int grid, size_t smem, cudaStream_t st, const BArgs& a) {
    switch (threads) {
        case 128: batched_gn_kernel<128><<<grid, 128, smem, st>>>(a); break;
        case 256: batched_gn_kernel<256><<<grid, 256, smem, st>>>(a); break;
        default: batched_gn_kernel<384><<<grid, 384, smem, st>>>(a); break;
    }
}
// grid of a variant: every problem its own CTA, at most what fits resident
int grid_of(int device, int threads, size_t smem, int nprob) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (set_attr(threads, smem) != cudaSuccess || occupancy(threads, smem, &per_sm) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    return std::min(nprob, sms * per_sm);
}

}  // namespace

cp_status batch_plan_create(int device, cudaStream_t stream, int nprob, const cp_batch_problem* problems,
                            double eps_cg, int cg_max_iter, int max_iters, double target_residual, int autotune,
                            BatchPlan** out) {
    size_t need = 0;
    std::vector<BProb> hp(nprob);
    for (int i = 0; i < nprob; ++i) {
        const cp_batch_problem& q = problems[i];
        if (!q.X || !q.A[0] || !q.A[1] || !q.A[2] || q.rank < 1 || q.rank > CP_BATCH_MAX_RANK || !(q.mu > 1.0) ||
            !(q.lam >= 0.0) || !(q.lam_lo >= 0.0) || !(q.lam_hi >= q.lam_lo))
            return CP_ERR_ARG;
        if ((q.reg != CP_REG_IDENTITY && q.reg != CP_REG_DIAG) || !(q.armijo_c >= 0.0 && q.armijo_c < 1.0) ||
            (q.armijo_c > 0.0 && (!(q.armijo_beta > 0.0 && q.armijo_beta < 1.0) || q.armijo_max < 0)))
            return CP_ERR_ARG;
        int S = 0;
        for (int n = 0; n < 3; ++n) {
            if (q.dims[n] < 1 || q.dims[n] > CP_BATCH_MAX_SIDE) return CP_ERR_ARG;
            hp[i].s[n] = (int)q.dims[n];
            hp[i].A[n] = q.A[n];
            S += (int)q.dims[n];
        }
        hp[i].R = q.rank;
        hp[i].X = q.X;
        hp[i].lam = q.lam;
        hp[i].lam_lo = q.lam_lo;
        hp[i].lam_hi = q.lam_hi;
        hp[i].mu = q.mu;
        hp[i].reg = q.reg;
        hp[i].lam_fixed = q.lam_fixed ? 1 : 0;
        hp[i].armijo_c = q.armijo_c;
        hp[i].armijo_beta = q.armijo_beta;
        hp[i].armijo_max = q.armijo_max;
        hp[i].pad = 0;
        need = std::max(need, smem_bytes(S, q.rank));
    }
    if (need > kBatchSmemMax) return CP_ERR_UNSUPPORTED;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    BatchPlan* pl = new BatchPlan();
    pl->device = device;
    pl->nprob = nprob;
    pl->smem = need;
    pl->eps_cg = eps_cg;
    pl->cg_max = cg_max_iter;
    pl->max_iters = max_iters;
    pl->target = target_residual;
    pl->hp = hp;
    auto fail = [&](cp_status st) {
        cudaGetLastError();
        if (pl->dp) cudaFree(pl->dp);
        if (pl->dr) cudaFree(pl->dr);
        if (pl->dc) cudaFree(pl->dc);
        if (pl->dorder) cudaFree(pl->dorder);
        delete pl;
        return st;
    };
    // the two problem orders: as given, and largest work s_1 s_2 s_3 R first (ties by index)
    std::vector<int> orders(2 * (size_t)nprob);
    for (int i = 0; i < nprob; ++i) orders[i] = orders[nprob + i] = i;
    auto work = [&](int i) { return (double)hp[i].s[0] * hp[i].s[1] * hp[i].s[2] * hp[i].R; };
    std::stable_sort(orders.begin() + nprob, orders.end(), [&](int a, int b) { return work(a) > work(b); });
    if (cudaMalloc(&pl->dp, sizeof(BProb) * nprob) != cudaSuccess || cudaMalloc(&pl->dr, sizeof(BRes) * nprob) != cudaSuccess ||
        cudaMalloc(&pl->dc, sizeof(int)) != cudaSuccess || cudaMalloc(&pl->dorder, sizeof(int) * 2 * nprob) != cudaSuccess)
        return fail(CP_ERR_NOMEM);
    if (cudaMemcpyAsync(pl->dp, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(pl->dorder, orders.data(), sizeof(int) * 2 * nprob, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
        return fail(CP_ERR_CUDA);
    pl->threads = 256;
    pl->grid = grid_of(device, 256, need, nprob);
    if (autotune) {
        // Autotuner: time each block size and each problem order on a scratch copy of
        // (at most 64 of) the problems' factors -- the caller's factors are not
        // touched -- and keep the fastest.  The sample is the first 64 problems of
        // the largest-work order when the batch is larger (it sets the tail).
        const int nt = std::min(nprob, 64);
        std::vector<BProb> tp(nt);
        std::vector<int> src(nt), torders(2 * (size_t)nt);
        for (int i = 0; i < nt; ++i) src[i] = nprob > nt ? orders[nprob + i] : i;
        for (int i = 0; i < nt; ++i) tp[i] = hp[src[i]];
        for (int i = 0; i < nt; ++i) torders[i] = torders[nt + i] = i;
        std::stable_sort(torders.begin() + nt, torders.end(), [&](int a, int b) { return work(src[a]) > work(src[b]); });
        size_t words = 0;
        for (const BProb& b : tp) words += (size_t)(b.s[0] + b.s[1] + b.s[2]) * b.R;
        double* scratch = nullptr;
        BProb* dtp = nullptr;
        BRes* dtr = nullptr;
        int* dtc = nullptr;
        int* dto = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaMalloc(&scratch, words * sizeof(double)) == cudaSuccess &&
                  cudaMalloc(&dtp, sizeof(BProb) * nt) == cudaSuccess && cudaMalloc(&dtr, sizeof(BRes) * nt) == cudaSuccess &&
                  cudaMalloc(&dtc, sizeof(int)) == cudaSuccess && cudaMalloc(&dto, sizeof(int) * 2 * nt) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess &&
                  cudaEventCreate(&e1) == cudaSuccess;
        if (ok) {
            size_t off = 0;
            for (BProb& b : tp)
                for (int n = 0; n < 3; ++n) {
                    double* dst = scratch + off;
                    off += (size_t)b.s[n] * b.R;
                    b.A[n] = dst;
                }
            ok = cudaMemcpyAsync(dtp, tp.data(), sizeof(BProb) * nt, cudaMemcpyHostToDevice, stream) == cudaSuccess &&
                 cudaMemcpyAsync(dto, torders.data(), sizeof(int) * 2 * nt, cudaMemcpyHostToDevice, stream) ==
                     cudaSuccess;
        }
        float best = 0.f;
        for (int v = 0; ok && v < 6; ++v) {
            const int th = kVariants[v >> 1], ord = v & 1;
            const int g = grid_of(device, th, need, nt);
            if (g < 1) continue;
            for (int rep = 0; ok && rep < 2; ++rep) {  // the first run of a variant includes its module load
                for (int i = 0; i < nt && ok; ++i)
                    for (int n = 0; n < 3; ++n)
                        ok = ok && cudaMemcpyAsync(tp[i].A[n], hp[src[i]].A[n],
                                                   (size_t)tp[i].s[n] * tp[i].R * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, stream) == cudaSuccess;
                ok = ok && cudaMemsetAsync(dtc, 0, sizeof(int), stream) == cudaSuccess;
                ok = ok && cudaEventRecord(e0, stream) == cudaSuccess;
                launch(th, g, need, stream,
                       BArgs{dtp, dtr, nt, dtc, dto + (size_t)ord * nt, eps_cg, cg_max_iter, max_iters, target_residual});
                ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, stream) == cudaSuccess &&
                     cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0.f;
                if (ok && rep == 1 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best == 0.f || ms < best)) {
                    best = ms;
                    pl->threads = th;
                    pl->order = ord;
                    pl->grid = grid_of(device, th, need, nprob);
                }
            }
        }
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (scratch) cudaFree(scratch);
        if (dtp) cudaFree(dtp);
        if (dtr) cudaFree(dtr);
        if (dtc) cudaFree(dtc);
        if (dto) cudaFree(dto);
        if (!ok) return fail(CP_ERR_CUDA);
    }
    if (pl->grid < 1) return fail(CP_ERR_UNSUPPORTED);
    if (cudaStreamSynchronize(stream) != cudaSuccess) return fail(CP_ERR_CUDA);
    *out = pl;
    return CP_OK;
}

cp_status batch_plan_launch(BatchPlan* pl, cudaStream_t stream) {
    if (cudaMemsetAsync(pl->dc, 0, sizeof(int), stream) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    launch(pl->threads, pl->grid, pl->smem, stream,
           BArgs{pl->dp, pl->dr, pl->nprob, pl->dc, pl->dorder + (size_t)pl->order * pl->nprob, pl->eps_cg, pl->cg_max,
                 pl->max_iters, pl->target});
    if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
    return CP_OK;
}

cp_status batch_plan_results(BatchPlan* pl, cudaStream_t stream, cp_batch_result* results) {
    std::vector<BRes> hr(pl->nprob);
    if (cudaMemcpyAsync(hr.data(), pl->dr, sizeof(BRes) * pl->nprob, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    for (int i = 0; i < pl->nprob; ++i) {
        results[i].status = hr[i].status;
        results[i].iters = hr[i].iters;
        results[i].cg_iters_total = hr[i].cg_iters;
        results[i].converged = hr[i].converged;
        results[i].cg_breakdowns = hr[i].breakdowns;
        results[i].rel_residual = hr[i].rel_residual;
        results[i].lam = hr[i].lam;
        results[i].ls_backtracks = hr[i].backtracks;
    }
    return CP_OK;
}

int batch_plan_threads(const BatchPlan* pl) { return pl->threads; }

cp_status batch_plan_configure(BatchPlan* pl, int threads, int order) {
    if ((threads != 128 && threads != 256 && threads != 384) || (order != 0 && order != 1)) return CP_ERR_ARG;
    if (cudaSetDevice(pl->device) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    const int g = grid_of(pl->device, threads, pl->smem, pl->nprob);
    if (g < 1) return CP_ERR_UNSUPPORTED;
    pl->threads = threads;
    pl->order = order;
    pl->grid = g;
    return CP_OK;
}
int batch_plan_order(const BatchPlan* pl) { return pl->order; }

void batch_plan_destroy(BatchPlan* pl) {
    if (!pl) return;
    cudaSetDevice(pl->device);
    if (pl->dp) cudaFree(pl->dp);
    if (pl->dr) cudaFree(pl->dr);
    if (pl->dc) cudaFree(pl->dc);
    if (pl->dorder) cudaFree(pl->dorder);
    cudaGetLastError();
    delete pl;
}

cp_status run_batched(int device, cudaStream_t stream, int nprob, const cp_batch_problem* problems, double eps_cg,
                      int cg_max_iter, int max_iters, double target_residual, cp_batch_result* results) {
    BatchPlan* pl = nullptr;
    cp_status st = batch_plan_create(device, stream, nprob, problems, eps_cg, cg_max_iter, max_iters,
                                     target_residual, 0, &pl);
    if (st != CP_OK) return st;
    st = batch_plan_launch(pl, stream);
    if (st == CP_OK) st = batch_plan_results(pl, stream, results);
    batch_plan_destroy(pl);
    return st;
}

}  // namespace cpgn
