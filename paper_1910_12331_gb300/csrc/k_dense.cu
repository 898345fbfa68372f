// k_dense.cu -- the small dense steps of a GN iteration: Gram matrices and the
// Gamma set (Eq. (2.2), Eq. (3.3)), the gradient (Algorithm 1), the
// block-Jacobi preconditioner (Section 3.3), factor packing and the update
// A += V.  All FP64 unless a float copy is requested.
#include <algorithm>

#include "kernels.hpp"

namespace cpgn {

Shape make_shape(const cp_desc* d) {
    Shape s{};
    s.N = d->order;
    s.R = d->rank;
    s.roff[0] = 0;
    s.total = 1;
    for (int n = 0; n < s.N; ++n) {
        s.dims[n] = d->dims[n];
        s.roff[n + 1] = s.roff[n] + d->dims[n];
        s.total *= d->dims[n];
    }
    s.mid = 1;
    for (int n = 1; n + 1 < s.N; ++n) s.mid *= d->dims[n];
    return s;
}

// ------------------------------------------------------------------ Gram
// Block (mode n, row chunk c, 32x32 output tile): partial S^(n) over 16 rows.
constexpr int kGramRows = 16;
constexpr int kGramTile = 32;

int gram_chunks(const Shape& s) {
    int64_t mx = 1;
    for (int n = 0; n < s.N; ++n) mx = std::max<int64_t>(mx, s.dims[n]);
    return (int)((mx + kGramRows - 1) / kGramRows);
}

__global__ void gram_partial_kernel(Shape s, Ptrs<const double> A, double* part, int chunks) {
    const int n = blockIdx.z / chunks, c = blockIdx.z % chunks;
    const int R = s.R;
    const int r0 = blockIdx.y * kGramTile, z0 = blockIdx.x * kGramTile;
    __shared__ double Ar[kGramRows][kGramTile + 1];
    __shared__ double Az[kGramRows][kGramTile + 1];
    const int64_t i0 = (int64_t)c * kGramRows;
    const double* An = A.p[n];
    for (int t = threadIdx.x; t < kGramRows * kGramTile; t += blockDim.x) {
        const int ii = t / kGramTile, jj = t % kGramTile;
        const int64_t i = i0 + ii;
        const bool rowok = i < s.dims[n];
        Ar[ii][jj] = (rowok && r0 + jj < R) ? An[i * R + r0 + jj] : 0.0;
        Az[ii][jj] = (rowok && z0 + jj < R) ? An[i * R + z0 + jj] : 0.0;
    }
    __syncthreads();
    double* P = part + ((int64_t)n * chunks + c) * R * R;
    for (int t = threadIdx.x; t < kGramTile * kGramTile; t += blockDim.x) {
        const int rr = t / kGramTile, zz = t % kGramTile;
        double acc = 0.0;
#pragma unroll
        for (int ii = 0; ii < kGramRows; ++ii) acc += Ar[ii][rr] * Az[ii][zz];
        if (r0 + rr < R && z0 + zz < R) P[(r0 + rr) * R + z0 + zz] = acc;
    }
}

void launch_gram_partial(const Shape& s, Ptrs<const double> A, double* part, int chunks, cudaStream_t st) {
    const int tiles = (s.R + kGramTile - 1) / kGramTile;
    dim3 grid(tiles, tiles, s.N * chunks);
    gram_partial_kernel<<<grid, 256, 0, st>>>(s, A, part, chunks);
}

// S^(n) = sum over the chunks that exist for mode n; Gamma^(n,p) = prod_{m != n,p} S^(m).
// The chunk partials are loaded eight at a time before they are added.
__global__ void gamma_kernel(Shape s, const double* part, int chunks, double* S, double* Gam, float* GamF) {
    const int RR = s.R * s.R;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= RR) return;
    double Sq[kMaxN];
    for (int m = 0; m < s.N; ++m) {
        // mode m's chunks (chunks == 1: part holds the finished Gram matrices)
        const int64_t cmode = (s.dims[m] + kGramRows - 1) / kGramRows;
        const int cm = cmode < chunks ? (int)cmode : chunks;
        const double* pm = part + (int64_t)m * chunks * RR + q;
        double acc = 0.0;
        int c = 0;
        for (; c + 8 <= cm; c += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = pm[(int64_t)(c + u) * RR];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += v[u];
        }
        for (; c < cm; ++c) acc += pm[(int64_t)c * RR];
        Sq[m] = acc;
        S[(int64_t)m * RR + q] = acc;
    }
    for (int n = 0; n < s.N; ++n)
        for (int p = 0; p < s.N; ++p) {
            double prod = 1.0;
            for (int m = 0; m < s.N; ++m)
                if (m != n && m != p) prod *= Sq[m];
            const int64_t o = ((int64_t)n * s.N + p) * RR + q;
            Gam[o] = prod;
            if (GamF) GamF[o] = (float)prod;
        }
}

void launch_gamma(const Shape& s, const double* part, int chunks, double* S, double* Gam, float* GamF,
                  cudaStream_t st) {
    const int RR = s.R * s.R;
    gamma_kernel<<<(RR + 255) / 256, 256, 0, st>>>(s, part, chunks, S, Gam, GamF);
}

// ------------------------------------------------------ diagonal damping
// Damping by lam diag(J^T J) (Section 3.2): the diagonal of the block (n,n) of
// J^T J is Gamma^(n,n)_{rr} at every row of column r, so the damped system is
// the undamped one with each Gamma^(n,n)_{rr} replaced by
// Gamma^(n,n)_{rr} + lam Gamma^(n,n)_{rr}.  Rewrites those N R entries of the
// FP64 Gamma and of its FP32 copy (which may be null); the preconditioner and
// the CG matvec then run with lam = 0.  One thread per (n, r).
__global__ void damp_diag_kernel(Shape s, double* Gam, float* GamF, double lam) {
    const int R = s.R;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= s.N * R) return;
    const int n = t / R, r = t - n * R;
    const int64_t e = ((int64_t)n * s.N + n) * R * R + (int64_t)r * R + r;
    const double g = Gam[e];
    const double v = g + lam * g;
    Gam[e] = v;
    if (GamF) GamF[e] = (float)v;
}

void launch_damp_diag(const Shape& s, double* Gam, float* GamF, double lam, cudaStream_t st) {
    const int nr = s.N * s.R;
    damp_diag_kernel<<<(nr + 127) / 128, 128, 0, st>>>(s, Gam, GamF, lam);
}

// -------------------------------------------------------------- gradient
// One thread per (row, column) of the packed gradient.  Each block writes its
// partial ||G||^2 and ||M||^2 to part[n][block]; grad_norms_kernel adds them in
// a fixed order (no atomics), so the norms, and every decision that depends on
// them (CG tolerance, stop test), are the same from run to run.
__global__ void gradient_kernel(Shape s, Ptrs<const double> A, const double* Gam, const double* M, double* G,
                                double* part, bool resid) {
    __shared__ double red[32];
    const int R = s.R;
    const int n = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t len = s.dims[n] * R;
    double g2 = 0.0, m2 = 0.0;
    if (e < len) {
        const int64_t i = e / R;
        const int r = (int)(e % R);
        const double* Gnn = Gam + ((int64_t)n * s.N + n) * R * R;
        const double* a = A.p[n] + i * R;
        double acc = 0.0;
        // Gamma^(n,n) is symmetric bit for bit (its Grams sum the same products in the same
        // order for (r, z) and (z, r)): read column r, contiguous across the warp's threads
        for (int z = 0; z < R; ++z) acc += a[z] * Gnn[(int64_t)z * R + r];
        const double mv = M[s.roff[n] * R + e];
        // resid: mv = (E_(n) P^(n))_{ir}, G = -mv, M = A Gamma - G
        const double g = resid ? -mv : acc - mv;
        const double mfull = resid ? acc + mv : mv;
        G[s.roff[n] * R + e] = g;
        g2 = g * g;
        m2 = mfull * mfull;
    }
    g2 = block_sum(g2, red);
    m2 = block_sum(m2, red);
    if (threadIdx.x == 0) {
        double* o = part + 2 * ((int64_t)n * gridDim.x + blockIdx.x);
        o[0] = g2;
        o[1] = m2;
    }
}

// warp n: stats->gnorm2[n], mnorm2[n] = fixed-order sums of the nb block partials of mode n
__global__ void grad_norms_kernel(int N, int nb, const double* part, DevStats* stats) {
    const int n = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (n >= N) return;
    double g2 = 0.0, m2 = 0.0;
    for (int b = lane; b < nb; b += 32) {
        g2 += part[2 * ((int64_t)n * nb + b)];
        m2 += part[2 * ((int64_t)n * nb + b) + 1];
    }
    g2 = warp_sum(g2);
    m2 = warp_sum(m2);
    if (lane == 0) {
        stats->gnorm2[n] = g2;
        stats->mnorm2[n] = m2;
        if (!isfinite(g2) || !isfinite(m2)) set_status(&stats->status, CP_ERR_NONFINITE);
    }
}

static int gradient_blocks(const Shape& s) {
    int64_t mx = 0;
    for (int n = 0; n < s.N; ++n) mx = std::max<int64_t>(mx, s.dims[n] * s.R);
    return (int)((mx + 255) / 256);
}

size_t gradient_part_doubles(const Shape& s) { return (size_t)2 * s.N * gradient_blocks(s); }

void launch_gradient(const Shape& s, Ptrs<const double> A, const double* Gam, const double* M, double* G,
                     double* part, DevStats* stats, cudaStream_t st, bool resid) {
    const int nb = gradient_blocks(s);
    gradient_kernel<<<dim3((unsigned)nb, s.N), 256, 0, st>>>(s, A, Gam, M, G, part, resid);
    grad_norms_kernel<<<1, 32 * s.N, 0, st>>>(s.N, nb, part, stats);
}

// -------------------------------------------------------- preconditioner
// P_inv^(n) = (Gamma^(n,n) + lam I)^{-1} (Algorithm 2, first loop; Section
// 3.3), one block per mode, in shared memory when it fits (else a global
// workspace): in-place Gauss-Jordan inversion without pivoting, which is
// stable for symmetric positive definite matrices.  Its pivots are the Schur
// complement diagonals, i.e. the squares of the Cholesky diagonals, so the
// positivity test of every pivot is the Cholesky SPD test.
// A non-positive pivot raises CP_ERR_NOT_SPD.  The inverse is written in FP64
// (Pinv) and, for the mixed path, rounded to FP32 (PinvF).
constexpr int kPrecondThreads = 512;

__global__ void __launch_bounds__(kPrecondThreads) precond_kernel(Shape s, const double* Gam, double lam, double* Pinv,
                                                                  float* PinvF, double* scratch, DevStats* stats) {
    using T = double;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_bad;
    __shared__ T s_inv;
    const int R = s.R, n = blockIdx.x;
    const bool in_smem = scratch == nullptr;
    T* B = in_smem ? reinterpret_cast<T*>(smem_raw) : scratch + (int64_t)n * (R * R + 2 * R);
    T* f = B + R * R;  // column j of the previous step
    const double* Gnn = Gam + ((int64_t)n * s.N + n) * R * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_bad = 0;
    for (int i = warp; i < R; i += nw)
        for (int k = lane; k < R; k += 32) B[i * R + k] = (T)(Gnn[i * R + k] + (i == k ? lam : 0.0));
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        if (threadIdx.x == 0) {
            T p = B[j * R + j];
            if (!(p > 0.0)) {
                s_bad = 1;
                p = 1.0;
            }
            s_inv = (T)1 / p;
        }
        for (int i = threadIdx.x; i < R; i += blockDim.x) f[i] = B[i * R + j];
        __syncthreads();
        const T inv = s_inv;
        // pivot row: B[j][k] /= p (k != j), B[j][j] = 1/p
        for (int k = threadIdx.x; k < R; k += blockDim.x) B[j * R + k] = k == j ? inv : B[j * R + k] * inv;
        __syncthreads();
        // other rows: B[i][k] -= f_i B[j][k] (k != j), B[i][j] = -f_i / p
        for (int i = warp; i < R; i += nw) {
            if (i == j) continue;
            const T fi = f[i];
            for (int k = lane; k < R; k += 32)
                B[i * R + k] = k == j ? -fi * inv : B[i * R + k] - fi * B[j * R + k];
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) set_status(&stats->status, CP_ERR_NOT_SPD);
        return;
    }
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
        if (Pinv) Pinv[(int64_t)n * R * R + q] = (double)B[q];
        if (PinvF) PinvF[(int64_t)n * R * R + q] = (float)B[q];
    }
}

// The same elimination in double-float (hi + lo FP32 pairs, about 2^-44
// relative: error-free products by fmaf, Dekker; error-free sums, Knuth) for
// the mixed path, whose CG runs in FP32: GB300 runs FP32 at 64 times its FP64
// rate, and the elimination's R^3 updates per mode dominate the FP64 version.
// The pivot reciprocal (double-float Newton step) and its SPD test are formed
// by one thread, without FP64 instructions.
__device__ __forceinline__ float2 df_mul2(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}
__device__ __forceinline__ float2 df_sub2(float2 a, float2 b) {  // a - b
    const float s = a.x - b.x;
    const float z = s - a.x;
    const float e = (a.x - (s - z)) + (-b.x - z);
    const float l = e + (a.y - b.y);
    const float h = s + l;
    return make_float2(h, l - (h - s));
}

__global__ void __launch_bounds__(kPrecondThreads) precond_df_kernel(Shape s, const double* Gam, double lam,
                                                                     double* Pinv, float* PinvF, float2* scratch,
                                                                     DevStats* stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_bad;
    const int R = s.R, n = blockIdx.x;
    // B (R x R), then f (column j before step j) and prow (pivot row j scaled by 1/p)
    float2* B = scratch ? scratch + (int64_t)n * (R * R + 2 * R) : reinterpret_cast<float2*>(smem_raw);
    float2* f = B + R * R;
    float2* prow = f + R;
    const double* Gnn = Gam + ((int64_t)n * s.N + n) * R * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_bad = 0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const double v = Gnn[e] + ((e / R) == (e % R) ? lam : 0.0);
        const float h = (float)v;
        B[e] = make_float2(h, (float)(v - (double)h));
    }
    __syncthreads();
    // two block barriers per pivot: (1) snapshot column j and the scaled pivot row,
    // (2) update every row from the snapshots
    for (int j = 0; j < R; ++j) {
        // 1/p in double-float, formed by every thread: FP32 reciprocal, then one Newton
        // step with an error-free residual r = 1 - p h (no FP64 instruction)
        float2 pv = B[j * R + j];
        if (!(pv.x > 0.f)) {
            if (threadIdx.x == 0) s_bad = 1;
            pv = make_float2(1.f, 0.f);
        }
        const float hr = 1.0f / pv.x;
        const float2 ph = df_mul2(pv, make_float2(hr, 0.f));
        const float rr = (1.0f - ph.x) - ph.y;
        const float cr = hr * rr;
        const float ih = hr + cr;
        const float2 inv = make_float2(ih, cr - (ih - hr));
        for (int i = threadIdx.x; i < R; i += blockDim.x) {
            f[i] = B[i * R + j];
            prow[i] = i == j ? inv : df_mul2(B[j * R + i], inv);
        }
        __syncthreads();
        // rows i != j: B[i][k] -= f_i B'[j][k] (k != j), B[i][j] = -f_i / p; row j: B'[j][k]
        for (int i = warp; i < R; i += nw) {
            const float2 fi = f[i];
            for (int k = lane; k < R; k += 32) {
                const float2 pk = prow[k];
                if (i == j) {
                    B[j * R + k] = pk;
                } else {
                    const float2 t = df_mul2(fi, pk);
                    B[i * R + k] = k == j ? make_float2(-t.x, -t.y) : df_sub2(B[i * R + k], t);
                }
            }
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) set_status(&stats->status, CP_ERR_NOT_SPD);
        return;
    }
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
        const float2 v = B[q];
        if (Pinv) Pinv[(int64_t)n * R * R + q] = (double)v.x + (double)v.y;
        if (PinvF) PinvF[(int64_t)n * R * R + q] = v.x + v.y;
    }
}

void launch_precond(const Shape& s, const double* Gam, double lam, double* Pinv, float* PinvF, double* scratch,
                    DevStats* stats, cudaStream_t st, bool fp32) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(precond_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(precond_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (dev < 64) attr_set[dev] = true;
    }
    // The blocks Gamma^(n,n) + lam I of a collinear problem at small lam are
    // too ill-conditioned for an FP32 elimination: FP64 for the plain path,
    // double-float for the mixed path (whose FP32 CG gets the inverse rounded once).
    // shared memory (or the global scratch when it does not fit): R x R + 2 R eight-byte words
    // (the FP64 kernel uses R x R + R of them)
    const size_t bytes = precond_smem_bytes(s.R);
    if (fp32) {
        if (bytes)
            precond_df_kernel<<<s.N, kPrecondThreads, bytes, st>>>(s, Gam, lam, Pinv, PinvF, nullptr, stats);
        else
            precond_df_kernel<<<s.N, kPrecondThreads, 0, st>>>(s, Gam, lam, Pinv, PinvF, (float2*)scratch, stats);
        return;
    }
    float* pf = nullptr;
    if (bytes)
        precond_kernel<<<s.N, kPrecondThreads, bytes, st>>>(s, Gam, lam, Pinv, pf, nullptr, stats);
    else
        precond_kernel<<<s.N, kPrecondThreads, 0, st>>>(s, Gam, lam, Pinv, pf, scratch, stats);
}

size_t precond_smem_bytes(int R) {
    const size_t bytes = ((size_t)R * R + 2 * (size_t)R) * sizeof(double);
    return bytes <= 200 * 1024 ? bytes : 0;
}

size_t precond_scratch_doubles(const Shape& s) { return (size_t)s.N * ((size_t)s.R * s.R + 2 * (size_t)s.R); }

// ------------------------------------------------------- pack / update
template <typename T>
__global__ void pack_kernel(Shape s, Ptrs<const double> A, T* Ap) {
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        Ap[s.roff[n] * s.R + e] = (T)A.p[n][e];
}

template <typename T>
void launch_pack(const Shape& s, Ptrs<const double> A, T* Ap, cudaStream_t st) {
    dim3 grid(64, s.N);
    pack_kernel<T><<<grid, 256, 0, st>>>(s, A, Ap);
}
template void launch_pack<double>(const Shape&, Ptrs<const double>, double*, cudaStream_t);
template void launch_pack<float>(const Shape&, Ptrs<const double>, float*, cudaStream_t);

template <typename T>
__global__ void update_kernel(Shape s, Ptrs<double> A, const T* V, double t, DevStats* stats) {
    __shared__ double red[32];
    // a step that failed on the device (non-SPD, non-finite, breakdown, timeout) leaves A unchanged
    const int st = ldcg(&stats->status);
    if (st != CP_OK && st != CP_WARN_CG_MAXIT) return;
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R;
    double v2 = 0.0, a2 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = t * (double)V[s.roff[n] * s.R + e];
        const double a = A.p[n][e] + v;
        A.p[n][e] = a;
        v2 += v * v;
        a2 += a * a;
    }
    v2 = block_sum(v2, red);
    a2 = block_sum(a2, red);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->vnorm2[n], v2);
        atomicAdd(&stats->anorm2[n], a2);
    }
}

template <typename T>
void launch_update(const Shape& s, Ptrs<double> A, const T* V, DevStats* stats, cudaStream_t st, double t) {
    dim3 grid(32, s.N);
    update_kernel<T><<<grid, 256, 0, st>>>(s, A, V, t, stats);
}
template void launch_update<double>(const Shape&, Ptrs<double>, const double*, DevStats*, cudaStream_t, double);
template void launch_update<float>(const Shape&, Ptrs<double>, const float*, DevStats*, cudaStream_t, double);

// ------------------------------------------------------ Armijo line search
// Trial factors At = A + t V (packed FP64; A in the caller's per-mode pointers).
template <typename T>
__global__ void trial_factors_kernel(Shape s, Ptrs<const double> A, const T* V, double t, double* At) {
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R, off = s.roff[n] * s.R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        At[off + e] = A.p[n][e] + t * (double)V[off + e];
}
template <typename T>
void launch_trial_factors(const Shape& s, Ptrs<const double> A, const T* V, double t, double* At, cudaStream_t st) {
    trial_factors_kernel<T><<<dim3(32, s.N), 256, 0, st>>>(s, A, V, t, At);
}
template void launch_trial_factors<double>(const Shape&, Ptrs<const double>, const double*, double, double*,
                                           cudaStream_t);
template void launch_trial_factors<float>(const Shape&, Ptrs<const double>, const float*, double, double*,
                                          cudaStream_t);

// <G, V> over the packed vectors, in a fixed order: kDotBlocks block partials
// (each a fixed stride of the vector, a fixed tree inside the block), then one
// block sums the partials in order into *out.
constexpr int kDotBlocks = 64;
template <typename T>
__global__ void dot_partial_kernel(int64_t len, const double* G, const T* V, double* part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        acc = fma(G[e], (double)V[e], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
__global__ void dot_finish_kernel(const double* part, int n, double* out) {
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += part[k];
        *out = acc;
    }
}
template <typename T>
void launch_dot_gv(int64_t len, const double* G, const T* V, double* part, double* out, cudaStream_t st) {
    dot_partial_kernel<T><<<kDotBlocks, 256, 0, st>>>(len, G, V, part);
    dot_finish_kernel<<<1, 32, 0, st>>>(part, kDotBlocks, out);
}
template void launch_dot_gv<double>(int64_t, const double*, const double*, double*, double*, cudaStream_t);
template void launch_dot_gv<float>(int64_t, const double*, const float*, double*, double*, cudaStream_t);

__global__ void als_solve_kernel(int64_t rows, int R, const double* Mn, const double* P, double* An) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * R) return;
    const int64_t i = e / R;
    const int r = (int)(e % R);
    double acc = 0.0;
    for (int z = 0; z < R; ++z) acc += Mn[i * R + z] * P[(int64_t)z * R + r];
    An[e] = acc;
}

void launch_als_solve(const Shape& s, int n, const double* Mn, const double* Pinv_n, double* An, cudaStream_t st) {
    const int64_t len = s.dims[n] * s.R;
    als_solve_kernel<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(s.dims[n], s.R, Mn, Pinv_n, An);
}

__global__ void unpack_kernel(Shape s, const double* packed, Ptrs<double> out) {
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        out.p[n][e] = packed[s.roff[n] * s.R + e];
}

void launch_unpack(const Shape& s, const double* packed, Ptrs<double> out, cudaStream_t st) {
    dim3 grid(64, s.N);
    unpack_kernel<<<grid, 256, 0, st>>>(s, packed, out);
}

}  // namespace cpgn
