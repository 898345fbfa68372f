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
// solve (for ranks whose R x R matrices do not fit there, in a global
// region of its own, with its mode's matrices in global memory too).  Only the R x R products A^(p)T W^(p) (accumulated with atomic adds
// into a double-buffered global accumulator) and scalar partials cross
// blocks, with 3 bounded-spin grid barriers per CG iteration.  Scalar
// reductions (dot products, norms) are FP64 and are summed by every block in
// the same fixed order, so every block takes the same alpha, beta and stop
// decision.  Vectors are FP64 (plain path) or FP32 (mixed path).
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "kernels.hpp"

namespace cpgn {

namespace {
constexpr int kThreads = 512;

// a * b + c with one rounding, in the precision of T (no promotion to double)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Up to 8 partials per lane are loaded before any is consumed, so one L2
// round trip serves a whole gather (at most 256 blocks).
constexpr int kGatherPerLane = 8;
// Entries of T^(n) per thread whose loads go out together (FP32: R x R <= 8 x 512
// in one round; FP64, twice the registers per value: four).
template <typename T>
constexpr int kTQ = sizeof(T) == 4 ? 8 : 4;

// Error-free sum s + e = a + b (Knuth two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}
// (h, l) += (xh, xl) in double-float
__device__ __forceinline__ void df_add(float& h, float& l, float xh, float xl) {
    float s, e;
    two_sum(h, xh, s, e);
    h = s;
    l += xl + e;
}

// Block partials of the CG dot products, one 8-byte slot per block: FP64 for
// FP64 vectors, a double-float (hi, lo) pair of FP32 values for FP32 vectors,
// so that the cross-block sums of the FP32 path run on the FP32 pipes (on
// GB300 a chain of FP64 additions costs more than the sums are worth).
template <typename T>
struct Slot;
template <>
struct Slot<double> {
    static __device__ __forceinline__ void put(double* p, double h, double l) { *p = h + l; }
    static __device__ __forceinline__ float as_float(const double* v, int c) { return (float)__ldcg(&v[c]); }
    // sum of v[c] over lane's c in [lane, nb) step 32, fixed order; then over the warp
    static __device__ __forceinline__ double warp_total(const double* v, int nb, int lane, int c0, int c1) {
        double x[kGatherPerLane];
#pragma unroll
        for (int u = 0; u < kGatherPerLane; ++u) {
            const int c = lane + 32 * u;
            x[u] = (c < nb && c >= c0 && c < c1) ? __ldcg(&v[c]) : 0.0;
        }
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < kGatherPerLane; ++u) acc += x[u];
        return warp_sum(acc);
    }
};
template <>
struct Slot<float> {
    static __device__ __forceinline__ float as_float(const double* v, int c) {
        const float2 x = __ldcg(reinterpret_cast<const float2*>(v) + c);
        return x.x + x.y;
    }
    static __device__ __forceinline__ void put(double* p, double h, double l) {
        const float fh = (float)(h + l);
        *reinterpret_cast<float2*>(p) = make_float2(fh, (float)((h - (double)fh) + l));
    }
    static __device__ __forceinline__ double warp_total(const double* v, int nb, int lane, int c0, int c1) {
        float2 x[kGatherPerLane];
#pragma unroll
        for (int u = 0; u < kGatherPerLane; ++u) {
            const int c = lane + 32 * u;
            x[u] = (c < nb && c >= c0 && c < c1) ? __ldcg(reinterpret_cast<const float2*>(v) + c) : make_float2(0.f, 0.f);
        }
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int u = 0; u < kGatherPerLane; ++u) df_add(h, l, x[u].x, x[u].y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
            df_add(h, l, oh, ol);
        }
        return (double)h + (double)l;
    }
};

// s = sum of the block partials v[0..nb) (warp 0, fixed order) and q = numer / s,
// both broadcast to the block.  One lane divides: a division in every thread
// would load GB300's slow FP64 pipe with hundreds of divisions per block.
template <typename T>
__device__ __forceinline__ double gather_sum(const double* v, int nb, double* bcast, double numer, double& q) {
    if (threadIdx.x < 32) {
        const double acc = Slot<T>::warp_total(v, nb, (int)threadIdx.x, 0, nb);
        if (threadIdx.x == 0) {
            bcast[0] = acc;
            bcast[1] = numer / acc;
        }
    }
    __syncthreads();
    const double r = bcast[0];
    q = bcast[1];
    __syncthreads();
    return r;
}

// One pass over the <R,Z> and |R|^2 partials: rz = sum of all rz partials,
// rsum = sum over modes of sqrt(sum of that mode's |R|^2 partials), and
// ratio = rz / rz_old (beta), formed by one lane.  The per-mode norms only
// feed the CG stop test: FP32 square roots.
template <typename T>
__device__ __forceinline__ void gather_rz_rn(const double* rzp, const double* rnp, int nb, const int* mode_blk0, int N,
                                             double* bcast, double rz_old, double& rz, double& rsum, double& ratio) {
    if (threadIdx.x < 32) {
        const int lane = (int)threadIdx.x;
        // the |R|^2 partials are loaded once, with the rz partials in flight
        float xn[kGatherPerLane];
#pragma unroll
        for (int u = 0; u < kGatherPerLane; ++u) {
            const int c = lane + 32 * u;
            xn[u] = c < nb ? Slot<T>::as_float(rnp, c) : 0.f;
        }
        const double az = Slot<T>::warp_total(rzp, nb, lane, 0, nb);
        float tot = 0.f;
        for (int m = 0; m < N; ++m) {
            float am = 0.f;
#pragma unroll
            for (int u = 0; u < kGatherPerLane; ++u) {
                const int c = lane + 32 * u;
                if (c >= mode_blk0[m] && c < mode_blk0[m + 1]) am += xn[u];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) am += __shfl_xor_sync(0xffffffffu, am, o);
            tot += sqrtf(fmaxf(am, 0.f));
        }
        if (lane == 0) {
            bcast[0] = az;
            bcast[1] = (double)tot;
            bcast[2] = rz_old != 0.0 ? az / rz_old : 0.0;
        }
    }
    __syncthreads();
    rz = bcast[0];
    rsum = bcast[1];
    ratio = bcast[2];
    __syncthreads();
}

// ---- block-wide dot products of the block's rows.  FP32 vectors: each thread
// forms its products and partial sum error-free in double-float (two-product
// by fmaf, two-sum), the warps reduce (hi, lo) pairs with the same error-free
// steps on the FP32 pipes, and one warp adds the per-warp results in FP64.
// (GB300's FP64 pipe runs at 1/64 of FP32: a reduction in FP64 by every
// thread would cost more than the whole row computation.)  FP64 vectors:
// plain FP64 products and sums, the cross-warp step again in one warp.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add_prod(float x, float y) {
        const float p = x * y;
        const float pe = fmaf(x, y, -p);
        float s, e;
        two_sum(h, p, s, e);
        h = s;
        l += e + pe;
    }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, o);
            const float ol = __shfl_xor_sync(0xffffffffu, l, o);
            float s, e;
            two_sum(h, oh, s, e);
            h = s;
            l += ol + e;
        }
    }
    __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
template <>
struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add_prod(double x, double y) { v = fma(x, y, v); }
    __device__ __forceinline__ void warp_reduce() { v = warp_sum(v); }
    __device__ __forceinline__ double value() const { return v; }
};

// (sum x*y, sum u*w) over the block's rows, as (hi, lo) pairs valid in thread 0.
// red: at least 2 * (blockDim.x / 32) + 2 doubles.
template <typename T>
__device__ __forceinline__ void dot2_rows(const T* x, const T* y, const T* u, const T* w, int len, double* red,
                                          double& r0h, double& r0l, double& r1h, double& r1l) {
    DotAcc<T> a, c;
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        a.add_prod(x[e], y[e]);
        if (u) c.add_prod(u[e], w[e]);
    }
    a.warp_reduce();
    if (u) c.warp_reduce();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if constexpr (sizeof(T) == 4) {
        float2* r2 = reinterpret_cast<float2*>(red);
        if (lane == 0) {
            r2[warp] = make_float2(a.h, a.l);
            r2[32 + warp] = u ? make_float2(c.h, c.l) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (warp == 0) {
            float2 p = lane < nw ? r2[lane] : make_float2(0.f, 0.f), q = lane < nw ? r2[32 + lane] : make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ph = __shfl_xor_sync(0xffffffffu, p.x, o), pl = __shfl_xor_sync(0xffffffffu, p.y, o);
                const float qh = __shfl_xor_sync(0xffffffffu, q.x, o), ql = __shfl_xor_sync(0xffffffffu, q.y, o);
                df_add(p.x, p.y, ph, pl);
                df_add(q.x, q.y, qh, ql);
            }
            r0h = p.x;
            r0l = p.y;
            r1h = q.x;
            r1l = q.y;
        }
    } else {
        if (lane == 0) {
            red[warp] = a.value();
            red[32 + warp] = u ? c.value() : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            double s0 = lane < nw ? red[lane] : 0.0, s1 = lane < nw ? red[32 + lane] : 0.0;
            r0h = warp_sum(s0);
            r1h = warp_sum(s1);
            r0l = r1l = 0.0;
        }
    }
    __syncthreads();
}


}  // namespace

// ---- register-tiled row products on shared memory (row stride Rp = R rounded up to 4)
template <typename T>
struct V4;
template <>
struct V4<float> {
    float v[4];
    __device__ __forceinline__ void load(const float* p) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <>
struct V4<double> {
    double v[4];
    __device__ __forceinline__ void load(const double* p) {
        const double2 t0 = *reinterpret_cast<const double2*>(p);
        const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
        v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    }
};

// Tile shapes of the row products.  FP32: 2 x 4 register tiles (fewer
// shared-memory loads per FMA: 1 x 4 tiles, or a tile's sum split over two
// lanes, give more threads work but measured 1.3-1.6x slower).  FP64 is
// DFMA-bound: one output per thread spreads the work over all four
// sub-partitions of the SM.
template <typename T>
struct Tile;
template <>
struct Tile<float> {
    static constexpr int TR = 2, TC = 4;   // rows_mm
    static constexpr int YR = 2, YC = 4;   // y_tiles
};
template <>
struct Tile<double> {
    static constexpr int TR = 1, TC = 1;
    static constexpr int YR = 1, YC = 1;
};

template <typename T, int TC>
__device__ __forceinline__ void load_cols(const T* p, T* v) {
    if constexpr (TC == 4) {
        V4<T> t;
        t.load(p);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = t.v[u];
    } else {
#pragma unroll
        for (int u = 0; u < TC; ++u) v[u] = p[u];
    }
}

// out[k][c] = lam * X[k][c] + sum_z X[k][z] M1[z][c] + sum_z Y[k][z] M2[z][c]   (M2 may be null)
// for k < rows, c < Rp; each thread computes a TR x TC tile.
template <typename T>
__device__ __forceinline__ void rows_mm(const T* X, const T* M1, const T* Yr, const T* M2, T lam, T* out, int rows,
                                        int R, int Rp) {
    constexpr int TR = Tile<T>::TR, TC = Tile<T>::TC;
    const int tc_n = Rp / TC, tr_n = (rows + TR - 1) / TR;
    for (int t = threadIdx.x; t < tr_n * tc_n; t += blockDim.x) {
        const int tr = t / tc_n, tc = t - tr * tc_n;
        const int k0 = TR * tr, c0 = TC * tc;
        const T* xr[TR];
        const T* yr[TR];
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const int k = k0 + i < rows ? k0 + i : k0;
            xr[i] = X + k * Rp;
            yr[i] = M2 ? Yr + k * Rp : nullptr;
        }
        T acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int u = 0; u < TC; ++u) acc[i][u] = lam * xr[i][c0 + u];
#pragma unroll 2
        for (int z = 0; z < R; ++z) {
            T m[TC];
            load_cols<T, TC>(M1 + z * Rp + c0, m);
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                const T a = xr[i][z];
#pragma unroll
                for (int u = 0; u < TC; ++u) acc[i][u] = fmadd(a, m[u], acc[i][u]);
            }
        }
        if (M2) {
#pragma unroll 2
            for (int z = 0; z < R; ++z) {
                T m[TC];
                load_cols<T, TC>(M2 + z * Rp + c0, m);
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const T a = yr[i][z];
#pragma unroll
                    for (int u = 0; u < TC; ++u) acc[i][u] = fmadd(a, m[u], acc[i][u]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
            if (k0 + i < rows)
#pragma unroll
                for (int u = 0; u < TC; ++u) out[(k0 + i) * Rp + c0 + u] = acc[i][u];
    }
}

// Yp[r][c] = sum_k A[k][r] W[k][c] over the block's rows (TR x TC tiles),
// Yp row stride R.
template <typename T>
__device__ __forceinline__ void y_tiles(const T* A, const T* W, T* Yacc, int rows, int R, int Rp) {
    constexpr int TR = Tile<T>::YR, TC = Tile<T>::YC;
    const int tc_n = Rp / TC, tr_n = (R + TR - 1) / TR;
    for (int t = threadIdx.x; t < tr_n * tc_n; t += blockDim.x) {
        const int tr = t / tc_n, tc = t - tr * tc_n;
        const int r0 = TR * tr, c0 = TC * tc;
        T acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int u = 0; u < TC; ++u) acc[i][u] = 0;
#pragma unroll 2
        for (int k = 0; k < rows; ++k) {
            T w[TC];
            load_cols<T, TC>(W + k * Rp + c0, w);
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                const T a = A[k * Rp + r0 + i];  // r0 + i <= Rp - 1: the padding column is zero
#pragma unroll
                for (int u = 0; u < TC; ++u) acc[i][u] = fmadd(a, w[u], acc[i][u]);
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int u = 0; u < TC; ++u) {
                const int r = r0 + i, c = c0 + u;
                if (r < R && c < R) Yacc[r * R + c] = acc[i][u];
            }
    }
}

// Persistent CP-CG.  Per iteration, three grid barriers:
//   (B1) Y^(p)(W) complete: T^(n), Q rows, partial <W,Q>;
//   (B2) alpha, V/R update, Z = R P_inv, partial <R,Z>, |R^(n)|^2 and A^T Z;
//   (B3) the scalar gather (beta, stop test) and, beside it, Y^(p)(W) =
//        sum_blocks A^T Z (fixed order, split over all blocks) + beta Y^(p)(W);
//        W = Z + beta W.
// Every cross-block sum runs in a fixed order, so a solve is reproducible.
// Shared memory holds the block's Gamma^(n,p) (all p), P_inv^(n), T^(n) and
// its rows of A, V, R, Z, W, Q, every matrix with row stride Rp (zero padded).
template <typename T, bool spill>
__global__ void __launch_bounds__(kThreads, 1) pcg_kernel(PcgArgs<T> a, int stage_mats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Shape& s = a.s;
    const int R = s.R, RR = R * R, N = s.N;
    const int Rp = (R + 3) & ~3, RRp = R * Rp;
    const int b = blockIdx.x;
    int n = 0;
    while (n + 1 < N && b >= a.mode_blk0[n + 1]) ++n;
    const int j = b - a.mode_blk0[n];
    const int64_t row0 = (int64_t)j * a.rpb[n];
    const int64_t left = s.dims[n] - row0;
    const int rows = (int)(left < a.rpb[n] ? left : a.rpb[n]);
    const int lenp = rows * Rp;
    const int64_t goff = (s.roff[n] + row0) * R;  // packed element offset of the block's rows
    (void)stage_mats;

    double* red = reinterpret_cast<double*>(smem_raw);
    double* bcast = red + 72;
    T* Gx;  // Gamma^(n,p), p = 0..N-1
    T* Pm;  // P_inv^(n)
    T* p;
    if constexpr (spill) {  // the mode's matrices, then the block's own region (T^(n), rows)
        Gx = a.spill + (size_t)n * (N + 1) * RRp;
        Pm = Gx + (size_t)N * RRp;
        p = a.spill + (size_t)N * (N + 1) * RRp + (size_t)b * a.spill_stride;
    } else {
        p = reinterpret_cast<T*>(smem_raw + 80 * sizeof(double));
        Gx = p; p += (size_t)N * RRp;
        Pm = p; p += RRp;
    }
    T* Tt = p; p += RRp;               // T^(n) transposed
    const T* Gm = Gx + (size_t)n * RRp;
    const int rl = a.rpb[n] * Rp;
    T* sA = p; p += rl;
    T* sV = p; p += rl;
    T* sR = p; p += rl;
    T* sZ = p; p += rl;
    T* sW = p; p += rl;
    T* sQ = p;

    double* const part_rz = a.part;
    double* const part_rn = a.part + a.nblocks;
    double* const part_wq = a.part + 2 * a.nblocks;
    int* const status = &a.stats->status;
    const unsigned nb = (unsigned)a.nblocks;
    const long long lim = a.spin_limit;

    // ---- set-up: stage the constant matrices and the block's rows, zero padded
    // (in global memory the mode's blocks share the staging of its matrices)
    const int q0 = spill ? j * blockDim.x + threadIdx.x : threadIdx.x;
    const int qstep = spill ? (a.mode_blk0[n + 1] - a.mode_blk0[n]) * blockDim.x : blockDim.x;
    for (int q = q0; q < N * RRp; q += qstep) {
        const int pp = q / RRp, e = q - pp * RRp, z = e / Rp, c = e - z * Rp;
        Gx[q] = c < R ? a.GamT[((size_t)n * N + pp) * RR + z * R + c] : (T)0;
    }
    for (int e = q0; e < RRp; e += qstep) {
        const int z = e / Rp, c = e - z * Rp;
        Pm[e] = c < R ? a.PinvT[(size_t)n * RR + z * R + c] : (T)0;
    }
    for (int e = threadIdx.x; e < RRp; e += blockDim.x) Tt[e] = (T)0;
    for (int e = threadIdx.x; e < lenp; e += blockDim.x) {
        const int k = e / Rp, c = e - k * Rp;
        const bool in = c < R;
        sA[e] = in ? a.Ap[goff + k * R + c] : (T)0;
        sR[e] = in ? (T)(-a.G[goff + k * R + c]) : (T)0;
        sV[e] = (T)0;
    }
    double gsum = 0.0, msum = 0.0;
    for (int m = 0; m < N; ++m) {
        gsum += sqrt(ldcg(&a.stats->gnorm2[m]));
        msum += sqrt(ldcg(&a.stats->mnorm2[m]));
    }
    const double tol = a.eps_cg * gsum;
    // Algorithm 1's loop test, evaluated on the device: a stationary point gets no update.
    const bool stationary = a.stop_ratio > 0.0 && gsum <= a.stop_ratio * msum;
    bool ok = true;
    if constexpr (spill) ok = grid_sync(a.bar, status, nb, lim);  // the mode's matrices are complete
    __syncthreads();
    double rz_h = 0.0, rz_l = 0.0, rn_h = 0.0, rn_l = 0.0;
    if (ok) {
        rows_mm<T>(sR, Pm, nullptr, nullptr, (T)0, sZ, rows, R, Rp);
        __syncthreads();
        for (int e = threadIdx.x; e < lenp; e += blockDim.x) sW[e] = sZ[e];
        dot2_rows(sR, sZ, sR, sR, lenp, red, rz_h, rz_l, rn_h, rn_l);
        if (threadIdx.x == 0) {
            Slot<T>::put(part_rz + b, rz_h, rz_l);
            Slot<T>::put(part_rn + b, rn_h, rn_l);
        }
        y_tiles(sA, sZ, a.Zpart + (size_t)b * RR, rows, R, Rp);
    }

    int it = 0;
    double rsum = 0.0, rz = 0.0, beta = 0.0;
    ok = ok && grid_sync(a.bar, status, nb, lim);
    double ratio = 0.0;
    // After the set-up and after every third barrier: Y^(p)(W) = Y^(p)(Z) + beta Y^(p)(W_old) (Y is
    // linear in W and W = Z + beta W_old), Y^(p)(Z) the sum over the blocks of mode p of their A^T Z in a
    // fixed order, spread over warps 1.. of all blocks, while warp 0 of every block gathers the scalar
    // partials (rz = <R,Z>, the per-mode |R|, beta = rz / rz_old): both read only what the barrier
    // completed, so their L2 round trips overlap; a thread's first entry waits for beta in registers.
    const size_t ny = (size_t)N * RR;
    auto sum_partials = [&](size_t e) -> T {
        const int pp = (int)(e / RR), q = (int)(e - (size_t)pp * RR);
        const int c0 = a.mode_blk0[pp], c1 = a.mode_blk0[pp + 1];
        T acc = (T)0;
        int c = c0;
        constexpr int kIn = sizeof(T) == 4 ? 32 : 16;  // partials in flight per round
        for (; c + kIn <= c1; c += kIn) {
            T v[kIn];
#pragma unroll
            for (int u = 0; u < kIn; ++u) v[u] = ldcg(&a.Zpart[(size_t)(c + u) * RR + q]);
#pragma unroll
            for (int u = 0; u < kIn; ++u) acc += v[u];
        }
        if (c < c1) {
            T v[kIn];
#pragma unroll
            for (int u = 0; u < kIn; ++u) v[u] = c + u < c1 ? ldcg(&a.Zpart[(size_t)(c + u) * RR + q]) : (T)0;
#pragma unroll
            for (int u = 0; u < kIn; ++u) acc += v[u];
        }
        return acc;
    };
    auto gather = [&](double rz_old, bool first, double& rz_out, double& rsum_out) {
        const size_t nw = blockDim.x - 32, estep = (size_t)nb * nw;
        const size_t e0 = (size_t)b * nw + (threadIdx.x - 32);
        const bool have0 = threadIdx.x >= 32 && e0 < ny;
        T acc0 = (T)0, y0 = (T)0;
        if (have0) {
            if (!first) y0 = a.Yfull[e0];
            acc0 = sum_partials(e0);
        }
        gather_rz_rn<T>(part_rz, part_rn, (int)nb, a.mode_blk0, N, bcast, rz_old, rz_out, rsum_out, ratio);
        const T be = first ? (T)0 : (T)ratio;
        if (have0) {
            a.Yfull[e0] = fmadd(be, y0, acc0);
            // (at the first gather Y^(p)(W_old) does not exist yet: the buffer holds whatever an
            // earlier call left there, so it is not read)
            for (size_t e = e0 + estep; e < ny; e += estep)
                a.Yfull[e] = first ? sum_partials(e) : fmadd(be, a.Yfull[e], sum_partials(e));
        }
    };
    if (ok) gather(0.0, true, rz, rsum);
    if (stationary) {
        ok = false;
        if (b == 0 && threadIdx.x == 0) a.stats->stopped = 1;
    }
    while (ok) {
        if (!(rsum > tol)) break;
        if (!isfinite(rsum) || !isfinite(rz)) { set_status(status, CP_ERR_NONFINITE); break; }
        if (it >= a.maxit) { set_status(status, CP_WARN_CG_MAXIT); break; }
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        // ---- T^(n) = sum_{p != n} Gamma^(n,p) * Y^(p)(W), stored transposed (Tt[z][r] = T[r][z]);
        // every thread issues its loads of Y (up to kTQ entries, the modes but n) before using them
        {
            for (int q0 = threadIdx.x; q0 < RR; q0 += kTQ<T> * blockDim.x) {
                T y[kTQ<T>][kMaxN];
#pragma unroll
                for (int u = 0; u < kTQ<T>; ++u) {
                    const int q = q0 + u * blockDim.x;
#pragma unroll
                    for (int pp = 0; pp < kMaxN; ++pp)
                        y[u][pp] = (pp < N && pp != n && q < RR) ? ldcg(&a.Yfull[(size_t)pp * RR + q]) : (T)0;
                }
#pragma unroll
                for (int u = 0; u < kTQ<T>; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q >= RR) break;
                    const int r = q / R, z = q - r * R;
                    T t = 0;
#pragma unroll
                    for (int pp = 0; pp < kMaxN; ++pp)
                        if (pp < N && pp != n) t = fmadd(Gx[(size_t)pp * RRp + r * Rp + z], y[u][pp], t);
                    Tt[z * Rp + r] = t;
                }
            }
        }
        __syncthreads();
        // ---- Q = lam W + W Gamma^(n,n) + A T^(n)^T, partial <W,Q>
        rows_mm<T>(sW, Gm, sA, Tt, (T)a.lam, sQ, rows, R, Rp);
        __syncthreads();
        double wq_h, wq_l, unused_h, unused_l;
        dot2_rows<T>(sW, sQ, nullptr, nullptr, lenp, red, wq_h, wq_l, unused_h, unused_l);
        if (threadIdx.x == 0) Slot<T>::put(part_wq + b, wq_h, wq_l);
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        double alpha;
        const double wq = gather_sum<T>(part_wq, (int)nb, bcast, rz, alpha);
        if (!isfinite(wq)) { set_status(status, CP_ERR_NONFINITE); break; }
        if (!(wq > 0.0)) { set_status(status, CP_ERR_BREAKDOWN); break; }
        const T al = (T)alpha;
        for (int e = threadIdx.x; e < lenp; e += blockDim.x) {
            sV[e] = fmadd(al, sW[e], sV[e]);
            sR[e] = fmadd(-al, sQ[e], sR[e]);
        }
        __syncthreads();
        rows_mm<T>(sR, Pm, nullptr, nullptr, (T)0, sZ, rows, R, Rp);
        __syncthreads();
        dot2_rows(sR, sZ, sR, sR, lenp, red, rz_h, rz_l, rn_h, rn_l);
        if (threadIdx.x == 0) {
            Slot<T>::put(part_rz + b, rz_h, rz_l);
            Slot<T>::put(part_rn + b, rn_h, rn_l);
        }
        y_tiles(sA, sZ, a.Zpart + (size_t)b * RR, rows, R, Rp);
        if (!(ok = grid_sync(a.bar, status, nb, lim))) break;
        double rz_new;
        gather(rz, false, rz_new, rsum);
        ++it;
        if (!(rsum > tol)) break;
        if (it >= a.maxit) { set_status(status, CP_WARN_CG_MAXIT); break; }
        beta = ratio;  // rz_new / rz, formed by one lane
        rz = rz_new;
        const T be = (T)beta;
        for (int e = threadIdx.x; e < lenp; e += blockDim.x) sW[e] = fmadd(be, sW[e], sZ[e]);
        __syncthreads();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < lenp; e += blockDim.x) {
        const int k = e / Rp, c = e - k * Rp;
        if (c < R) a.V[goff + k * R + c] = sV[e];
    }
    if (b == 0 && threadIdx.x == 0) {
        a.stats->cg_iters = it;
        a.stats->cg_rnorm = rsum;
    }
}

template <typename T>
static size_t pcg_smem_bytes(int N, int R, int rpb_max, bool /*stage*/) {
    const size_t Rp = (size_t)((R + 3) & ~3);
    return ((size_t)(N + 2) * R * Rp + 6 * (size_t)rpb_max * Rp) * sizeof(T) + 80 * sizeof(double);
}

// Launch geometry of the persistent CG kernel for one shape (cached: the
// attribute and occupancy queries cost tens of microseconds of host time).
struct PcgGeom {
    int N = -1, R = -1, T = 0, want = 0, sms = 0, dev = -1;
    int64_t dims[kMaxN] = {};
    int nblocks = 0, mode_blk0[kMaxN + 1] = {}, rpb[kMaxN] = {};
    size_t bytes = 0;
    bool spill = false;          // matrices and rows in global memory
    int64_t spill_stride = 0;    // elements per block region
    size_t spill_elems = 0;      // elements of the whole global region
    cp_status status = CP_OK;
};

template <typename T>
static PcgGeom pcg_geometry(const Shape& s, int want, int sms) {
    PcgGeom g;
    g.N = s.N;
    g.R = s.R;
    g.T = (int)sizeof(T);
    g.want = want;
    g.sms = sms;
    for (int n = 0; n < s.N; ++n) g.dims[n] = s.dims[n];
    const int64_t rows_total = s.roff[s.N];
    const size_t budget = 200 * 1024;
    const int64_t Rp = (s.R + 3) & ~3;
    // Large R: the N + 2 R x R matrices alone exceed shared memory.  They and the
    // row blocks then live in global memory (L2), one block per SM, few rows each.
    g.spill = (size_t)(s.N + 2) * s.R * Rp * sizeof(T) + 80 * sizeof(double) > budget;
    if (g.spill) want = std::max(want, sms);
    int target = std::max(s.N, std::min<int>(want, (int)std::min<int64_t>(rows_total, 4096)));
    cudaFuncSetAttribute(pcg_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget);
    for (int attempt = 0; attempt < 64; ++attempt) {
        int total = 0, rpb_max = 1;
        for (int n = 0; n < s.N; ++n) {
            int nbn = (int)std::max<int64_t>(1, (int64_t)((double)target * s.dims[n] / rows_total));
            nbn = (int)std::min<int64_t>(nbn, s.dims[n]);
            const int rpb = (int)((s.dims[n] + nbn - 1) / nbn);
            nbn = (int)((s.dims[n] + rpb - 1) / rpb);
            g.rpb[n] = rpb;
            g.mode_blk0[n] = total;
            total += nbn;
            rpb_max = std::max(rpb_max, rpb);
        }
        g.mode_blk0[s.N] = total;
        g.nblocks = total;
        g.bytes = g.spill ? 80 * sizeof(double) : pcg_smem_bytes<T>(s.N, s.R, rpb_max, true);
        g.spill_stride = g.spill ? (int64_t)s.R * Rp + 6 * (int64_t)rpb_max * Rp : 0;
        g.spill_elems = g.spill ? (size_t)s.N * (s.N + 1) * s.R * Rp + (size_t)total * g.spill_stride : 0;
        if (g.bytes > budget) {  // rows do not fit: more blocks
            target = target * 2;
            continue;
        }
        if (total > 32 * kGatherPerLane) {  // the scalar gathers cover at most 256 blocks
            target = 32 * kGatherPerLane - s.N;
            continue;
        }
        int per_sm = 0;
        if (g.spill)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<T, true>, kThreads, g.bytes);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<T, false>, kThreads, g.bytes);
        if (per_sm < 1) {
            g.status = CP_ERR_UNSUPPORTED;
            return g;
        }
        if (total > per_sm * sms) {
            if (target <= s.N) {
                g.status = CP_ERR_UNSUPPORTED;
                return g;
            }
            target = std::max(s.N, per_sm * sms - s.N);
            continue;
        }
        g.status = CP_OK;
        return g;
    }
    g.status = CP_ERR_UNSUPPORTED;
    return g;
}

template <typename T>
static const PcgGeom& geometry_for(const Shape& s, int max_blocks) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t rows_total = s.roff[s.N];
    // FP64 vectors: the work is DFMA-bound, spread it over every SM.  FP32
    // vectors: the iteration is latency-bound; about 16 rows per block (measured
    // at 400^3, R = 50: 19.1 us per iteration at 75-150 blocks, 20.7 us at 36).
    int want = max_blocks > 0 ? max_blocks
                              : (sizeof(T) == 8 ? sms : (int)std::min<int64_t>(sms, (rows_total + 15) / 16));
    static thread_local PcgGeom cache[2];
    PcgGeom& g = cache[sizeof(T) == 8];
    bool hit = g.N == s.N && g.R == s.R && g.want == want && g.sms == sms && g.dev == dev;
    for (int n = 0; hit && n < s.N; ++n) hit = g.dims[n] == s.dims[n];
    if (!hit) {
        g = pcg_geometry<T>(s, want, sms);
        g.want = want;
        g.dev = dev;
    }
    return g;
}

template <typename T>
cp_status pcg_plan(const Shape& s, int max_blocks, int* nblocks, size_t* spill_elems) {
    const PcgGeom& g = geometry_for<T>(s, max_blocks);
    if (g.status != CP_OK) return g.status;
    *nblocks = g.nblocks;
    *spill_elems = g.spill_elems;
    return CP_OK;
}
template cp_status pcg_plan<double>(const Shape&, int, int*, size_t*);
template cp_status pcg_plan<float>(const Shape&, int, int*, size_t*);

template <typename T>
cp_status launch_pcg(PcgArgs<T>& a, int max_blocks, cudaStream_t st) {
    const Shape& s = a.s;
    const PcgGeom& g = geometry_for<T>(s, max_blocks);
    if (g.status != CP_OK) return g.status;
    if (g.spill && !a.spill) return CP_ERR_ARG;  // the caller did not provide the global region
    if (!g.spill) a.spill = nullptr;
    a.spill_stride = g.spill_stride;
    a.nblocks = g.nblocks;
    for (int n = 0; n <= s.N; ++n) a.mode_blk0[n] = g.mode_blk0[n];
    for (int n = 0; n < s.N; ++n) a.rpb[n] = g.rpb[n];
    int stage_i = 1;
    void* args[] = {(void*)&a, (void*)&stage_i};
    void* fn = g.spill ? (void*)pcg_kernel<T, true> : (void*)pcg_kernel<T, false>;
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(g.nblocks), dim3(kThreads), args, g.bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    return CP_OK;
}
template cp_status launch_pcg<double>(PcgArgs<double>&, int, cudaStream_t);
template cp_status launch_pcg<float>(PcgArgs<float>&, int, cudaStream_t);

// ------------------------------------------------------------ plain matvec
// The implicit matvec as three plain kernels, in FP64 or (T = float) in the
// FP32 arithmetic of the mixed CG: A, W and Gamma rounded to FP32 once, every
// product and sum in FP32.
// Y[p][r][z] = sum_l A^(p)[l][r] W^(p)[l][z]; one thread per entry.
template <typename T>
__global__ void matvec_y_kernel(Shape s, Ptrs<const double> A, Ptrs<const double> W, T* Y) {
    const int R = s.R, RR = R * R;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)s.N * RR) return;
    const int p = (int)(e / RR), q = (int)(e % RR), r = q / R, z = q % R;
    const double* a = A.p[p];
    const double* w = W.p[p];
    T acc = 0;
    for (int64_t l = 0; l < s.dims[p]; ++l) acc = fmadd((T)a[l * R + r], (T)w[l * R + z], acc);
    Y[e] = acc;
}

// Q^(n)[k][r] = lam w_kr + sum_z w_kz Gamma^(n,n)_zr + sum_{p != n} sum_z a_kz Gamma^(n,p)_rz Y^(p)_rz.
// diag = true: damping by lam diag(J^T J) instead, folded into the diagonal of
// Gamma^(n,n) as (1 + lam) Gamma^(n,n)_rr (rounded once, as in the CG kernel).
template <typename T>
__global__ void matvec_q_kernel(Shape s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W,
                                double lam, bool diag, const T* Y, Ptrs<double> Q) {
    const int R = s.R, RR = R * R, N = s.N;
    const int n = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s.dims[n] * R) return;
    const int64_t k = e / R;
    const int r = (int)(e % R);
    const double* w = W.p[n] + k * R;
    const double* a = A.p[n] + k * R;
    const double* Gnn = Gam + ((int64_t)n * N + n) * RR;
    T acc = diag ? (T)0 : (T)lam * (T)w[r];
    for (int z = 0; z < R; ++z) {
        const T g = (diag && z == r) ? (T)(Gnn[r * R + r] * (1.0 + lam)) : (T)Gnn[r * R + z];
        acc = fmadd(g, (T)w[z], acc);
    }
    for (int p = 0; p < N; ++p) {
        if (p == n) continue;
        const double* Gnp = Gam + ((int64_t)n * N + p) * RR;
        const T* Yp = Y + (int64_t)p * RR;
        for (int z = 0; z < R; ++z) acc = fmadd((T)a[z], (T)Gnp[r * R + z] * Yp[r * R + z], acc);
    }
    Q.p[n][e] = (double)acc;
}

cudaError_t preload_matvec_f64() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, matvec_y_kernel<double>);
    return e != cudaSuccess ? e : cudaFuncGetAttributes(&fa, matvec_q_kernel<double>);
}

template <typename T>
void launch_matvec(const Shape& s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W, double lam,
                   bool diag, Ptrs<double> Q, T* Y, cudaStream_t st) {
    const int64_t ny = (int64_t)s.N * s.R * s.R;
    matvec_y_kernel<T><<<(unsigned)((ny + 255) / 256), 256, 0, st>>>(s, A, W, Y);
    int64_t mx = 0;
    for (int n = 0; n < s.N; ++n) mx = std::max<int64_t>(mx, s.dims[n] * s.R);
    dim3 grid((unsigned)((mx + 255) / 256), s.N);
    matvec_q_kernel<T><<<grid, 256, 0, st>>>(s, A, Gam, W, lam, diag, Y, Q);
}
template void launch_matvec<double>(const Shape&, Ptrs<const double>, const double*, Ptrs<const double>, double,
                                    bool, Ptrs<double>, double*, cudaStream_t);
template void launch_matvec<float>(const Shape&, Ptrs<const double>, const double*, Ptrs<const double>, double,
                                   bool, Ptrs<double>, float*, cudaStream_t);

void launch_matvec_f64(const Shape& s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W, double lam,
                       Ptrs<double> Q, double* Y, cudaStream_t st) {
    launch_matvec<double>(s, A, Gam, W, lam, false, Q, Y, st);
}

}  // namespace cpgn
