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
// partials of a few products, then an FP64 tree).  The stop test is the direct
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

// Threads per CTA: a template parameter (128, 256 or 384), chosen per plan by
// the autotuner (or 256).  BW = warps per CTA.
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

// Sum over the CTA of one double per thread (all threads call; result in every thread).
template <int BT>
__device__ __forceinline__ double bsum(double v, double* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = l < (BT / 32) ? red[l] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Three sums at once (all threads call).
template <int BT>
__device__ __forceinline__ void bsum3(double& a, double& b, double& c, double* red) {
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        red[w] = a;
        red[(BT / 32) + w] = b;
        red[2 * (BT / 32) + w] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
    for (int k = 0; k < (BT / 32); ++k) {
        a += red[k];
        b += red[(BT / 32) + k];
        c += red[2 * (BT / 32) + k];
    }
}

struct Smem {
    int s[3], roff[3], S, R;
    float *A, *W, *Rv, *Z, *V, *Q;  // S x R each (rows of mode n start at roff[n])
    float *Sg, *Gm, *Pi, *Yb, *Tb;  // 3 R^2, 9 R^2, 3 R^2, 3 R^2, 3 R^2
    double *gj, *red;               // R^2 + R, 96
};

__device__ __forceinline__ void carve(Smem& m, unsigned char* base, const BProb& pb) {
    m.R = pb.R;
    m.roff[0] = 0;
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
        const float* a = m.A + m.roff[n] * R;
        float acc = 0.f;
        for (int i = 0; i < m.s[n]; ++i) acc = fmaf(a[i * R + r], a[i * R + z], acc);
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

// sum_k x[k] a[k][r] with four independent partial sums
__device__ __forceinline__ float dot_k(const float* __restrict__ x, const float* a, int R, int r, int n) {
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    int k = 0;
    for (; k + 3 < n; k += 4) {
        t0 = fmaf(__ldg(x + k), a[k * R + r], t0);
        t1 = fmaf(__ldg(x + k + 1), a[(k + 1) * R + r], t1);
        t2 = fmaf(__ldg(x + k + 2), a[(k + 2) * R + r], t2);
        t3 = fmaf(__ldg(x + k + 3), a[(k + 3) * R + r], t3);
    }
    for (; k < n; ++k) t0 = fmaf(__ldg(x + k), a[k * R + r], t0);
    return (t0 + t1) + (t2 + t3);
}

// M^(n) for all modes into out (S x R): warps own rows of mode n, lanes own rank columns.
template <int BT>
__device__ __forceinline__ void mttkrp3(const Smem& m, const float* __restrict__ X, float* out) {
    const int R = m.R, s1 = m.s[0], s2 = m.s[1], s3 = m.s[2];
    const int w = threadIdx.x >> 5, r = threadIdx.x & 31;
    const bool on = r < R;
    const int rr = on ? r : 0;
    const float *a1 = m.A, *a2 = m.A + m.roff[1] * R, *a3 = m.A + m.roff[2] * R;
    // mode 1: M[i][r] = sum_j a2[j][r] sum_k X[i,j,k] a3[k][r]
    for (int i = w; i < s1; i += (BT / 32)) {
        float acc = 0.f;
        for (int j = 0; j < s2; ++j) {
            const float* x = X + ((int64_t)i * s2 + j) * s3;
            acc = fmaf(dot_k(x, a3, R, rr, s3), a2[j * R + rr], acc);
        }
        if (on) out[i * R + r] = acc;
    }
    // mode 2: M[j][r] = sum_i a1[i][r] sum_k X[i,j,k] a3[k][r]
    for (int j = w; j < s2; j += (BT / 32)) {
        float acc = 0.f;
        for (int i = 0; i < s1; ++i) {
            const float* x = X + ((int64_t)i * s2 + j) * s3;
            acc = fmaf(dot_k(x, a3, R, rr, s3), a1[i * R + rr], acc);
        }
        if (on) out[(m.roff[1] + j) * R + r] = acc;
    }
    // mode 3: M[k][r] = sum_i a1[i][r] sum_j X[i,j,k] a2[j][r]
    for (int k = w; k < s3; k += (BT / 32)) {
        float acc = 0.f;
        for (int i = 0; i < s1; ++i) {
            const float* x = X + (int64_t)i * s2 * s3 + k;
            float t = 0.f;
            for (int j = 0; j < s2; ++j) t = fmaf(__ldg(x + (int64_t)j * s3), a2[j * R + rr], t);
            acc = fmaf(t, a1[i * R + rr], acc);
        }
        if (on) out[(m.roff[2] + k) * R + r] = acc;
    }
    __syncthreads();
}

// ||X - [[A]]||_F^2: a warp per row (i, j), lanes over k; compensated FP32 partials, FP64 across threads.
template <int BT>
__device__ __forceinline__ double resid2(const Smem& m, const float* __restrict__ X) {
    const int R = m.R, s1 = m.s[0], s2 = m.s[1], s3 = m.s[2];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const float *a1 = m.A, *a2 = m.A + m.roff[1] * R, *a3 = m.A + m.roff[2] * R;
    float sum = 0.f, comp = 0.f;
    for (int ij = w; ij < s1 * s2; ij += (BT / 32)) {
        const int i = ij / s2, j = ij % s2;
        const float* x = X + (int64_t)ij * s3;
        for (int k = l; k < s3; k += 32) {
            float rec = 0.f;
            for (int r = 0; r < R; ++r) rec = fmaf(a1[i * R + r] * a2[j * R + r], a3[k * R + r], rec);
            const float e = __ldg(x + k) - rec;
            const float y = fmaf(e, e, -comp);  // Kahan
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
    }
    return bsum<BT>((double)sum - (double)comp, m.red);
}

// out = in P_inv^(n) per mode (rows of mode n times the symmetric R x R block)
template <int BT>
__device__ __forceinline__ void apply_pinv(const Smem& m, const float* in, float* out) {
    const int R = m.R, SR = m.S * R;
    for (int e = threadIdx.x; e < SR; e += BT) {
        const int row = e / R, z = e % R;
        const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
        const float* P = m.Pi + n * R * R;
        const float* x = in + row * R;
        float acc = 0.f;
        for (int r = 0; r < R; ++r) acc = fmaf(x[r], P[r * R + z], acc);
        out[e] = acc;
    }
    __syncthreads();
}

// Q = (J^T J + lam D) W via Y^(p) = A^(p)^T W^(p), T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p),
// Q^(n) = lam W^(n) D^(n) + W^(n) Gamma^(n,n) + A^(n) T^(n)^T, D^(n) = I or diag(Gamma^(n,n)).
template <int BT>
__device__ __forceinline__ void matvec(const Smem& m, float lam, bool diag) {
    const int R = m.R, RR = R * R, SR = m.S * R;
    for (int e = threadIdx.x; e < 3 * RR; e += BT) {
        const int p = e / RR, r = (e % RR) / R, z = e % R;
        const float* a = m.A + m.roff[p] * R;
        const float* w = m.W + m.roff[p] * R;
        float acc = 0.f;
        for (int i = 0; i < m.s[p]; ++i) acc = fmaf(a[i * R + r], w[i * R + z], acc);
        m.Yb[e] = acc;
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
    for (int e = threadIdx.x; e < SR; e += BT) {
        const int row = e / R, z = e % R;
        const int n = row >= m.roff[2] ? 2 : (row >= m.roff[1] ? 1 : 0);
        const float* G = m.Gm + (n * 3 + n) * RR;
        const float* T = m.Tb + n * RR;
        const float* w = m.W + row * R;
        const float* a = m.A + row * R;
        float acc = (diag ? lam * G[z * R + z] : lam) * w[z];
        for (int r = 0; r < R; ++r) {
            acc = fmaf(w[r], G[r * R + z], acc);
            acc = fmaf(a[r], T[z * R + r], acc);
        }
        m.Q[e] = acc;
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
            m.A[e] = (float)pb.A[n][(row - m.roff[n]) * R + r];
        }
        // ||X||^2
        float xs = 0.f;
        const int64_t tot = (int64_t)m.s[0] * m.s[1] * m.s[2];
        for (int64_t e = threadIdx.x; e < tot; e += BT) {
            const float x = __ldg(X + e);
            xs = fmaf(x, x, xs);
        }
        const double nx2 = bsum<BT>((double)xs, m.red);
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
                for (int r = 0; r < R; ++r) acc = fmaf(-a[r], G[r * R + z], acc);
                m.Rv[e] = acc;
                m.V[e] = 0.f;
                const float sq = acc * acc;
                if (n == 0) g0 += sq;
                else if (n == 1) g1 += sq;
                else g2 += sq;
            }
            double ga = g0, gb = g1, gc = g2;
            bsum3<BT>(ga, gb, gc, m.red);
            const double gsum = sqrt(ga) + sqrt(gb) + sqrt(gc);
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
            double rz = bsum<BT>((double)rzp, m.red);
            double rnorm = gsum;
            double arz = 0.0;  // sum_k alpha_k <R_k, Z_k> = <-G, V> (PCG from V = 0)
            int k = 0;
            for (; k < args.cg_max && rnorm > args.eps_cg * gsum; ++k) {
                matvec<BT>(m, (float)lam, diag);
                float wqp = 0.f;
                for (int e = threadIdx.x; e < SR; e += BT) wqp = fmaf(m.W[e], m.Q[e], wqp);
                const double wq = bsum<BT>((double)wqp, m.red);
                if (!(wq > 0.0)) {  // FP32 curvature lost: end CG with the update found so far
                    ++breakdowns;
                    break;
                }
                const float alpha = (float)(rz / wq);
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
                double ra = q0, rb = q1, rzd = rzn;
                bsum3<BT>(ra, rb, rzd, m.red);
                const double rc = bsum<BT>((double)q2, m.red);
                rnorm = sqrt(ra) + sqrt(rb) + sqrt(rc);
                const float beta = (float)(rzd / rz);
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
                        m.A[e] = (float)(pb.A[n][(row - m.roff[n]) * R + r] + t * (double)m.V[e]);
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
                double* a = pb.A[n] + (row - m.roff[n]) * R + r;
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
