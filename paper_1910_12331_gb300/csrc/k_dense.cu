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
__global__ void gamma_kernel(Shape s, const double* part, int chunks, double* S, double* Gam, float* GamF) {
    const int RR = s.R * s.R;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= RR) return;
    double Sq[kMaxN];
    for (int m = 0; m < s.N; ++m) {
        const int cm = (int)((s.dims[m] + kGramRows - 1) / kGramRows);
        double acc = 0.0;
        for (int c = 0; c < cm; ++c) acc += part[((int64_t)m * chunks + c) * RR + q];
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

// -------------------------------------------------------------- gradient
// One thread per (row, column) of the packed gradient.
__global__ void gradient_kernel(Shape s, Ptrs<const double> A, const double* Gam, const double* M, double* G,
                                DevStats* stats, bool resid) {
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
        for (int z = 0; z < R; ++z) acc += a[z] * Gnn[(int64_t)r * R + z];  // Gamma symmetric
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
        atomicAdd(&stats->gnorm2[n], g2);
        atomicAdd(&stats->mnorm2[n], m2);
        if (!isfinite(g2) || !isfinite(m2)) set_status(&stats->status, CP_ERR_NONFINITE);
    }
}

void launch_gradient(const Shape& s, Ptrs<const double> A, const double* Gam, const double* M, double* G,
                     DevStats* stats, cudaStream_t st, bool resid) {
    int64_t mx = 0;
    for (int n = 0; n < s.N; ++n) mx = std::max<int64_t>(mx, s.dims[n] * s.R);
    dim3 grid((unsigned)((mx + 255) / 256), s.N);
    gradient_kernel<<<grid, 256, 0, st>>>(s, A, Gam, M, G, stats, resid);
}

// -------------------------------------------------------- preconditioner
// One block per mode: B = Gamma^(n,n) + lam I in a dense R x R scratch (shared
// memory when it fits, else a global workspace), right-looking Cholesky
// B = L L^T with a positivity check of every pivot, then the explicit inverse
// by forward (L Y = I) and back (L^T P = Y) substitution, one column per thread.
__global__ void precond_kernel(Shape s, const double* Gam, double lam, double* Pinv, float* PinvF,
                               double* scratch, DevStats* stats) {
    extern __shared__ double smem[];
    __shared__ int s_bad;
    const int R = s.R, n = blockIdx.x;
    const bool in_smem = scratch == nullptr;
    double* L = in_smem ? smem : scratch + (int64_t)n * 2 * R * R;
    double* Y = L + (int64_t)R * R;
    const double* Gnn = Gam + ((int64_t)n * s.N + n) * R * R;
    double* P = Pinv + (int64_t)n * R * R;
    if (threadIdx.x == 0) s_bad = 0;
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
        const int i = q / R, j = q % R;
        L[q] = Gnn[q] + (i == j ? lam : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        if (threadIdx.x == 0) {
            const double d = L[j * R + j];
            if (!(d > 0.0)) s_bad = 1;
            L[j * R + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double ljj = L[j * R + j];
        for (int i = j + 1 + threadIdx.x; i < R; i += blockDim.x) L[i * R + j] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle
        const int m = R - j - 1;
        for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
            const int i = j + 1 + q / m, k = j + 1 + q % m;
            if (k <= i) L[i * R + k] -= L[i * R + j] * L[k * R + j];
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) set_status(&stats->status, CP_ERR_NOT_SPD);
        return;
    }
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        for (int i = 0; i < R; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[i * R + k] * Y[k * R + c];
            Y[i * R + c] = v / L[i * R + i];
        }
        for (int i = R - 1; i >= 0; --i) {
            double v = Y[i * R + c];
            for (int k = i + 1; k < R; ++k) v -= L[k * R + i] * P[k * R + c];
            P[i * R + c] = v / L[i * R + i];
        }
    }
    __syncthreads();
    if (PinvF)
        for (int q = threadIdx.x; q < R * R; q += blockDim.x) PinvF[(int64_t)n * R * R + q] = (float)P[q];
}

void launch_precond(const Shape& s, const double* Gam, double lam, double* Pinv, float* PinvF, double* scratch,
                    DevStats* stats, cudaStream_t st) {
    const size_t bytes = precond_smem_bytes(s.R);
    if (bytes > 0) {
        cudaFuncSetAttribute(precond_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        precond_kernel<<<s.N, 256, bytes, st>>>(s, Gam, lam, Pinv, PinvF, nullptr, stats);
    } else {
        precond_kernel<<<s.N, 256, 0, st>>>(s, Gam, lam, Pinv, PinvF, scratch, stats);
    }
}

size_t precond_smem_bytes(int R) {
    const size_t bytes = (size_t)2 * R * R * sizeof(double);
    return bytes <= 200 * 1024 ? bytes : 0;
}

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
__global__ void update_kernel(Shape s, Ptrs<double> A, const T* V, DevStats* stats) {
    __shared__ double red[32];
    const int n = blockIdx.y;
    const int64_t len = s.dims[n] * s.R;
    double v2 = 0.0, a2 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)V[s.roff[n] * s.R + e];
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
void launch_update(const Shape& s, Ptrs<double> A, const T* V, DevStats* stats, cudaStream_t st) {
    dim3 grid(32, s.N);
    update_kernel<T><<<grid, 256, 0, st>>>(s, A, V, stats);
}
template void launch_update<double>(const Shape&, Ptrs<double>, const double*, DevStats*, cudaStream_t);
template void launch_update<float>(const Shape&, Ptrs<double>, const float*, DevStats*, cudaStream_t);

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
