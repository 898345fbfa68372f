// k_pcg.cu -- CP-CG (Algorithm 2) as one persistent, cooperatively launched
// kernel, and the plain FP64 implicit matvec.
//
// The implicit matvec of Eq. (3.4) is evaluated in the order that gives the
// O(N^2 s R^2) cost stated after it:
//   Y^(p) = A^(p)^T W^(p)                                   (R x R)
//   T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p)                (R x R, Hadamard)
//   Q^(n) = lam W^(n) + W^(n) Gamma^(n,n) + A^(n) T^(n)^T   (s_n x R)
// (Gamma^(n,p) is symmetric, so sum_{l,z} a^(n)_{kz} a^(p)_{lr} Gamma_{rz} w_{lz}
//  = sum_z a^(n)_{kz} (Gamma^(n,p) * Y^(p))_{rz}.)
//
// Persistent layout: every block owns a contiguous range of rows of ONE mode
// and keeps its rows of A, V, R, Z, W, Q in shared memory for the whole
// solve.  Only R x R partials and scalar partials cross blocks, through global
// memory and bounded-spin grid barriers (4 per CG iteration).  Scalar
// reductions (dot products, norms) are FP64 and are summed by every block in
// the same fixed order, so every block takes the same alpha, beta and stop
// decision.  Vectors are FP64 (plain path) or FP32 (mixed path).
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "kernels.hpp"

namespace cpgn {

namespace {
constexpr int kThreads = 256;

// a * b + c with one rounding, in the precision of T (no promotion to double)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
struct Smem {
    T* G;   // Gamma^(n,n), R x R (or a global pointer)
    T* P;   // P_inv^(n),  R x R (or a global pointer)
    T* Tt;  // T^(n) transposed, R x R (or a global pointer)
    T* A;   // own rows of A^(n)
    T* V; T* Rv; T* Z; T* W; T* Q;
    double* red;
};

// sum_{c in [c0, c1)} v[c], computed by warp 0 with lane-strided loads and a
// shuffle tree (a fixed order, identical in every block) and broadcast to the
// whole block through shared memory.
__device__ __forceinline__ double block_gather_sum(const double* v, int c0, int c1, double* bcast) {
    if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int c = c0 + (int)threadIdx.x; c < c1; c += 32) acc += __ldcg(&v[c]);
        acc = warp_sum(acc);
        if (threadIdx.x == 0) *bcast = acc;
    }
    __syncthreads();
    const double r = *bcast;
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ double dsum_rows(const T* x, const T* y, int len, double* red) {
    double acc = 0.0;
    for (int e = threadIdx.x; e < len; e += blockDim.x) acc += (double)x[e] * (double)y[e];
    return block_sum(acc, red);
}

// out[k][r] = sum_z in[k][z] * M[z][r] for the block's rows (M symmetric or given as M[z][r]).
template <typename T>
__device__ __forceinline__ void rows_times(const T* in, const T* M, T* out, int rows, int R) {
    for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
        const int k = e / R, r = e % R;
        const T* a = in + k * R;
        T acc = 0;
#pragma unroll 4
        for (int z = 0; z < R; ++z) acc = fmadd(a[z], M[z * R + r], acc);
        out[e] = acc;
    }
}

// Ypart[r][z] = sum over own rows k of A[k][r] W[k][z]
template <typename T>
__device__ __forceinline__ void y_partial(const T* A, const T* W, T* Yp, int rows, int R) {
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
        const int r = q / R, z = q % R;
        T acc = 0;
#pragma unroll 4
        for (int k = 0; k < rows; ++k) acc = fmadd(A[k * R + r], W[k * R + z], acc);
        Yp[q] = acc;
    }
}
}  // namespace

template <typename T>
__global__ void __launch_bounds__(kThreads) pcg_kernel(PcgArgs<T> a, int stage_mats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Shape& s = a.s;
    const int R = s.R, RR = R * R, N = s.N;
    const int b = blockIdx.x;
    int n = 0;
    while (n + 1 < N && b >= a.mode_blk0[n + 1]) ++n;
    const int j = b - a.mode_blk0[n];
    const int64_t row0 = (int64_t)j * a.rpb[n];
    const int64_t left = s.dims[n] - row0;
    const int rows = (int)(left < a.rpb[n] ? left : a.rpb[n]);
    const int len = rows * R;
    const int64_t goff = (s.roff[n] + row0) * R;  // packed element offset of the block's rows

    Smem<T> sm;
    {
        sm.red = reinterpret_cast<double*>(smem_raw);
        T* p = reinterpret_cast<T*>(smem_raw + 64 * sizeof(double));
        if (stage_mats) {
            sm.G = p; p += RR;
            sm.P = p; p += RR;
            sm.Tt = p; p += RR;
        } else {
            sm.G = const_cast<T*>(a.GamT) + ((int64_t)n * N + n) * RR;
            sm.P = const_cast<T*>(a.PinvT) + (int64_t)n * RR;
            sm.Tt = a.Tm + (int64_t)n * RR;
        }
        const int rl = a.rpb[n] * R;
        sm.A = p; p += rl;
        sm.V = p; p += rl;
        sm.Rv = p; p += rl;
        sm.Z = p; p += rl;
        sm.W = p; p += rl;
        sm.Q = p;
    }
    double* const part_rz = a.part;
    double* const part_rn = a.part + a.nblocks;
    double* const part_wq = a.part + 2 * a.nblocks;
    int* const status = &a.stats->status;
    const unsigned nb = (unsigned)a.nblocks;
    const long long lim = a.spin_limit;

    // ---- set-up: stage constant matrices and own rows
    if (stage_mats) {
        for (int q = threadIdx.x; q < RR; q += blockDim.x) {
            sm.G[q] = a.GamT[((int64_t)n * N + n) * RR + q];
            sm.P[q] = a.PinvT[(int64_t)n * RR + q];
        }
    }
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        sm.A[e] = a.Ap[goff + e];
        sm.Rv[e] = (T)(-a.G[goff + e]);
        sm.V[e] = (T)0;
    }
    double gsum = 0.0, msum = 0.0;
    for (int m = 0; m < N; ++m) {
        gsum += sqrt(ldcg(&a.stats->gnorm2[m]));
        msum += sqrt(ldcg(&a.stats->mnorm2[m]));
    }
    const double tol = a.eps_cg * gsum;
    // Algorithm 1's loop test, evaluated on the device: a stationary point gets no update.
    const bool stationary = a.stop_ratio > 0.0 && gsum <= a.stop_ratio * msum;
    __syncthreads();
    rows_times(sm.Rv, sm.P, sm.Z, rows, R);
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += blockDim.x) sm.W[e] = sm.Z[e];
    double rz_p = dsum_rows(sm.Rv, sm.Z, len, sm.red);
    double rn_p = dsum_rows(sm.Rv, sm.Rv, len, sm.red);
    if (threadIdx.x == 0) { part_rz[b] = rz_p; part_rn[b] = rn_p; }
    y_partial(sm.A, sm.W, a.Ypart + (int64_t)b * RR, rows, R);

    int it = 0;
    double rsum = 0.0, rz = 0.0;
    bool ok = grid_sync(a.bar, status, nb, lim);
    double* const bcast = sm.red + 40;
    auto reduce_r = [&](double& rz_out, double& rsum_out) {
        rz_out = block_gather_sum(part_rz, 0, (int)nb, bcast);
        double tot = 0.0;
        for (int m = 0; m < N; ++m) tot += sqrt(block_gather_sum(part_rn, a.mode_blk0[m], a.mode_blk0[m + 1], bcast));
        rsum_out = tot;
    };
    if (ok) reduce_r(rz, rsum);
    if (stationary) {
        ok = false;
        if (b == 0 && threadIdx.x == 0) a.stats->stopped = 1;
    }
    while (ok) {
        if (!(rsum > tol)) break;
        if (!isfinite(rsum) || !isfinite(rz)) { set_status(status, CP_ERR_NONFINITE); break; }
        if (it >= a.maxit) { set_status(status, CP_WARN_CG_MAXIT); break; }
        // ---- T phase: T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p), stored transposed.
        // One warp per entry q: the lanes split the per-block partials of every
        // Y^(p)_q, a shuffle reduction completes them, lane n forms T^(n)_q.
        {
            const int lane = threadIdx.x & 31;
            const int64_t gw = ((int64_t)b * blockDim.x + threadIdx.x) >> 5;
            const int64_t nw = ((int64_t)nb * blockDim.x) >> 5;
            for (int64_t q = gw; q < RR; q += nw) {
                T y[kMaxN];
#pragma unroll
                for (int p = 0; p < kMaxN; ++p) {
                    if (p >= N) break;
                    T acc = 0;
                    for (int c = a.mode_blk0[p] + lane; c < a.mode_blk0[p + 1]; c += 32)
                        acc += ldcg(&a.Ypart[(int64_t)c * RR + q]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    y[p] = acc;
                }
                if (lane < N) {
                    const int nn = lane;
                    T t = 0;
#pragma unroll
                    for (int p = 0; p < kMaxN; ++p) {
                        if (p >= N) break;
                        if (p != nn) t = fmadd(a.GamT[((int64_t)nn * N + p) * RR + q], y[p], t);
                    }
                    const int r = (int)(q / R), z = (int)(q % R);
                    a.Tm[(int64_t)nn * RR + z * R + r] = t;
                }
            }
        }
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        // ---- Q phase: Q = lam W + W Gamma^(n,n) + A T^(n)^T
        if (stage_mats)
            for (int q = threadIdx.x; q < RR; q += blockDim.x) sm.Tt[q] = ldcg(&a.Tm[(int64_t)n * RR + q]);
        __syncthreads();
        const T lam = (T)a.lam;
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int k = e / R, r = e % R;
            const T* w = sm.W + k * R;
            const T* ar = sm.A + k * R;
            T acc = lam * w[r];
            if (stage_mats) {
#pragma unroll 4
                for (int z = 0; z < R; ++z) {
                    acc = fmadd(w[z], sm.G[z * R + r], acc);
                    acc = fmadd(ar[z], sm.Tt[z * R + r], acc);
                }
            } else {
                for (int z = 0; z < R; ++z) {
                    acc = fmadd(w[z], sm.G[z * R + r], acc);
                    acc = fmadd(ar[z], ldcg(&sm.Tt[z * R + r]), acc);
                }
            }
            sm.Q[e] = acc;
        }
        __syncthreads();
        const double wq_p = dsum_rows(sm.W, sm.Q, len, sm.red);
        if (threadIdx.x == 0) part_wq[b] = wq_p;
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        const double wq = block_gather_sum(part_wq, 0, (int)nb, bcast);
        if (!isfinite(wq)) { set_status(status, CP_ERR_NONFINITE); break; }
        if (!(wq > 0.0)) { set_status(status, CP_ERR_BREAKDOWN); break; }
        const double alpha = rz / wq;
        const T al = (T)alpha;
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            sm.V[e] = fmadd(al, sm.W[e], sm.V[e]);
            sm.Rv[e] = fmadd(-al, sm.Q[e], sm.Rv[e]);
        }
        __syncthreads();
        rows_times(sm.Rv, sm.P, sm.Z, rows, R);
        __syncthreads();
        rz_p = dsum_rows(sm.Rv, sm.Z, len, sm.red);
        rn_p = dsum_rows(sm.Rv, sm.Rv, len, sm.red);
        if (threadIdx.x == 0) { part_rz[b] = rz_p; part_rn[b] = rn_p; }
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        double rz_new;
        reduce_r(rz_new, rsum);
        ++it;
        if (!(rsum > tol)) break;
        if (it >= a.maxit) { set_status(status, CP_WARN_CG_MAXIT); break; }
        const double beta = rz_new / rz;
        rz = rz_new;
        const T be = (T)beta;
        for (int e = threadIdx.x; e < len; e += blockDim.x) sm.W[e] = fmadd(be, sm.W[e], sm.Z[e]);
        __syncthreads();
        y_partial(sm.A, sm.W, a.Ypart + (int64_t)b * RR, rows, R);
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += blockDim.x) a.V[goff + e] = sm.V[e];
    if (b == 0 && threadIdx.x == 0) {
        a.stats->cg_iters = it;
        a.stats->cg_rnorm = rsum;
    }
}

template <typename T>
static size_t pcg_smem_bytes(int R, int rpb_max, bool stage) {
    return (size_t)((stage ? 3 : 0) * R * R + 6 * rpb_max * R) * sizeof(T) + 64 * sizeof(double);
}

template <typename T>
cp_status launch_pcg(PcgArgs<T>& a, int max_blocks, cudaStream_t st) {
    const Shape& s = a.s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t rows_total = s.roff[s.N];
    // FP64 vectors: the work is DFMA-bound, spread it over every SM.  FP32
    // vectors: the iteration is latency-bound, so use fewer, fatter blocks
    // (about 32 rows each) to shorten the barriers and reductions.
    int want = max_blocks > 0 ? max_blocks
                              : (sizeof(T) == 8 ? sms : (int)std::min<int64_t>(sms, (rows_total + 31) / 32));
    if (const char* env = getenv(sizeof(T) == 8 ? "CPGN_PCG_BLOCKS_F64" : "CPGN_PCG_BLOCKS_F32")) want = atoi(env);
    int target = std::max(s.N, std::min<int>(want, (int)std::min<int64_t>(rows_total, 4096)));
    // choose the blocks per mode so that the smem of the largest block fits
    const size_t budget = 200 * 1024;
    for (int attempt = 0; attempt < 64; ++attempt) {
        int total = 0, rpb_max = 1;
        for (int n = 0; n < s.N; ++n) {
            int nbn = (int)std::max<int64_t>(1, (int64_t)((double)target * s.dims[n] / rows_total));
            nbn = (int)std::min<int64_t>(nbn, s.dims[n]);
            const int rpb = (int)((s.dims[n] + nbn - 1) / nbn);
            nbn = (int)((s.dims[n] + rpb - 1) / rpb);
            a.rpb[n] = rpb;
            a.mode_blk0[n] = total;
            total += nbn;
            rpb_max = std::max(rpb_max, rpb);
        }
        a.mode_blk0[s.N] = total;
        a.nblocks = total;
        bool stage = pcg_smem_bytes<T>(s.R, rpb_max, true) <= budget;
        size_t bytes = pcg_smem_bytes<T>(s.R, rpb_max, stage);
        if (bytes > budget) {  // rows do not fit: more blocks
            target = target * 2;
            continue;
        }
        cudaFuncSetAttribute(pcg_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<T>, kThreads, bytes);
        if (per_sm < 1) return CP_ERR_UNSUPPORTED;
        if (total > per_sm * sms) {
            if (target <= s.N) return CP_ERR_UNSUPPORTED;
            target = std::max(s.N, per_sm * sms - s.N);
            continue;
        }
        int stage_i = stage ? 1 : 0;
        void* args[] = {(void*)&a, (void*)&stage_i};
        cudaError_t e = cudaLaunchCooperativeKernel((void*)pcg_kernel<T>, dim3(total), dim3(kThreads), args, bytes, st);
        return e == cudaSuccess ? CP_OK : CP_ERR_CUDA;
    }
    return CP_ERR_UNSUPPORTED;
}
template cp_status launch_pcg<double>(PcgArgs<double>&, int, cudaStream_t);
template cp_status launch_pcg<float>(PcgArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------ plain matvec
// Y[p][r][z] = sum_l A^(p)[l][r] W^(p)[l][z]; one thread per entry.
__global__ void matvec_y_kernel(Shape s, Ptrs<const double> A, Ptrs<const double> W, double* Y) {
    const int R = s.R, RR = R * R;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s.N * RR) return;
    const int p = (int)(e / RR), q = (int)(e % RR), r = q / R, z = q % R;
    const double* a = A.p[p];
    const double* w = W.p[p];
    double acc = 0.0;
    for (int64_t l = 0; l < s.dims[p]; ++l) acc += a[l * R + r] * w[l * R + z];
    Y[e] = acc;
}

// Q^(n)[k][r] = lam w_kr + sum_z w_kz Gamma^(n,n)_zr + sum_{p != n} sum_z a_kz Gamma^(n,p)_rz Y^(p)_rz
__global__ void matvec_q_kernel(Shape s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W,
                                double lam, const double* Y, Ptrs<double> Q) {
    const int R = s.R, RR = R * R, N = s.N;
    const int n = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s.dims[n] * R) return;
    const int64_t k = e / R;
    const int r = (int)(e % R);
    const double* w = W.p[n] + k * R;
    const double* a = A.p[n] + k * R;
    const double* Gnn = Gam + ((int64_t)n * N + n) * RR;
    double acc = lam * w[r];
    for (int z = 0; z < R; ++z) acc += Gnn[r * R + z] * w[z];
    for (int p = 0; p < N; ++p) {
        if (p == n) continue;
        const double* Gnp = Gam + ((int64_t)n * N + p) * RR;
        const double* Yp = Y + (int64_t)p * RR;
        for (int z = 0; z < R; ++z) acc += a[z] * Gnp[r * R + z] * Yp[r * R + z];
    }
    Q.p[n][e] = acc;
}

void launch_matvec_f64(const Shape& s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W, double lam,
                       Ptrs<double> Q, double* Y, cudaStream_t st) {
    const int64_t ny = (int64_t)s.N * s.R * s.R;
    matvec_y_kernel<<<(unsigned)((ny + 255) / 256), 256, 0, st>>>(s, A, W, Y);
    int64_t mx = 0;
    for (int n = 0; n < s.N; ++n) mx = std::max<int64_t>(mx, s.dims[n] * s.R);
    dim3 grid((unsigned)((mx + 255) / 256), s.N);
    matvec_q_kernel<<<grid, 256, 0, st>>>(s, A, Gam, W, lam, Y, Q);
}

}  // namespace cpgn
