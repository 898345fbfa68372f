// abi.cu -- the C ABI of include/cpgn.h: argument checks, handle-owned
// workspace, and the orchestration of the kernels of one GN step
// (Algorithm 1), one ALS sweep, the MTTKRP, the matvec and the residual.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cpgn.h"
#include "kernels.hpp"
#include "tc.hpp"

using namespace cpgn;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

constexpr long long kDefaultSpin = 1LL << 24;  // polls (with 64 ns sleeps: about a second or more)

// Host code behind some entry points uses standard containers; no exception
// may leave the C ABI: an allocation failure becomes CP_ERR_NOMEM.
template <typename F>
cp_status no_throw(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return CP_ERR_NOMEM;
    } catch (...) {
        return CP_ERR_CUDA;
    }
}

}  // namespace

struct cp_handle_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevBuf gram_part, S, Gam, GamF, Pinv, PinvF, precond_scratch, grad_part;
    DevBuf Mp, Gp, Ap, vec, Ypart, Tm, pcg_part, bar, stats, Y, resid_planes, Adf, Atrial, stats2, tucker, pcg_spill;
    DevStats* h_stats = nullptr;  // pinned
    DevStats* h_stats2 = nullptr; // pinned: line-search trials
    double* h_tk = nullptr;       // pinned: HoSVD convergence checks
    SplitCache split;             // bf16 planes of X (tensor-core path)
    // step timing: start, gradient phase end, CG start, step end, gradient phase start
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t side = nullptr;  // the preconditioner beside the gradient phase
    cudaEvent_t fork = nullptr, gam = nullptr, join = nullptr;
    int launches = 0;             // kernels launched by the current call
    int cg_blocks = 0;            // blocks of the last persistent CG launch
};

static cp_status ensure_events(cp_handle h) {
    for (auto& e : h->ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return CP_ERR_CUDA;
        }
    if ((!h->side && cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) ||
        (!h->fork && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) ||
        (!h->gam && cudaEventCreateWithFlags(&h->gam, cudaEventDisableTiming) != cudaSuccess) ||
        (!h->join && cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    return CP_OK;
}

static cp_status grow(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return CP_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_NOMEM;
    }
    b.bytes = bytes;
    return CP_OK;
}

#define CP_TRY(x)                           \
    do {                                    \
        cp_status _s = (x);                 \
        if (_s != CP_OK) return _s;         \
    } while (0)

#define CUDA_TRY(x)                                  \
    do {                                             \
        if ((x) != cudaSuccess) {                    \
            cudaGetLastError();                      \
            return CP_ERR_CUDA;                      \
        }                                            \
    } while (0)

static cp_status check_desc(const cp_desc* d) {
    if (!d) return CP_ERR_ARG;
    if (d->order < 2 || d->order > CP_MAX_ORDER) return CP_ERR_ARG;
    if (d->rank < 1 || d->rank > CP_MAX_RANK) return CP_ERR_ARG;
    if (d->x_dtype != CP_F32 && d->x_dtype != CP_F64) return CP_ERR_ARG;
    double total = 1.0;
    for (int n = 0; n < d->order; ++n) {
        if (d->dims[n] < 1 || d->dims[n] > (1LL << 31)) return CP_ERR_ARG;
        total *= (double)d->dims[n];
    }
    if (total > 9.0e15) return CP_ERR_ARG;
    int64_t mid = 1;
    for (int n = 1; n + 1 < d->order; ++n) mid *= d->dims[n];
    if (mid > 0x7fffffffLL) return CP_ERR_UNSUPPORTED;  // grid.x limit of the slice kernels
    return CP_OK;
}

static cp_status check_ptrs(const void* const* P, int n) {
    if (!P) return CP_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!P[i]) return CP_ERR_ARG;
    return CP_OK;
}

// no output pointer may coincide with an input pointer
static bool aliased(const void* const* out, int nout, const void* const* in, int nin, const void* X) {
    for (int i = 0; i < nout; ++i) {
        if (out[i] == X) return true;
        for (int j = 0; j < nin; ++j)
            if (out[i] == in[j]) return true;
        for (int j = 0; j < i; ++j)
            if (out[i] == out[j]) return true;
    }
    return false;
}

template <typename T>
static Ptrs<T> ptrs_of(T* const* p, int N) {
    Ptrs<T> r{};
    for (int n = 0; n < N; ++n) r.p[n] = p[n];
    return r;
}

template <typename T>
static Ptrs<T> packed_ptrs(T* base, const Shape& s) {
    Ptrs<T> r{};
    for (int n = 0; n < s.N; ++n) r.p[n] = base + s.roff[n] * s.R;
    return r;
}

static Ptrs<const double> as_const(Ptrs<double> p) {
    Ptrs<const double> r{};
    for (int n = 0; n < kMaxN; ++n) r.p[n] = p.p[n];
    return r;
}

static cp_status ensure_common(cp_handle h, const Shape& s) {
    const size_t RR = (size_t)s.R * s.R;
    const size_t rows = (size_t)s.roff[s.N];
    CP_TRY(grow(h->gram_part, (size_t)s.N * gram_chunks(s) * RR * sizeof(double)));
    CP_TRY(grow(h->grad_part, gradient_part_doubles(s) * sizeof(double)));
    CP_TRY(grow(h->S, s.N * RR * sizeof(double)));
    CP_TRY(grow(h->Gam, (size_t)s.N * s.N * RR * sizeof(double)));
    CP_TRY(grow(h->GamF, (size_t)s.N * s.N * RR * sizeof(float)));
    CP_TRY(grow(h->Pinv, s.N * RR * sizeof(double)));
    CP_TRY(grow(h->PinvF, s.N * RR * sizeof(float)));
    if (precond_smem_bytes(s.R) == 0) CP_TRY(grow(h->precond_scratch, precond_scratch_doubles(s) * sizeof(double)));
    CP_TRY(grow(h->Mp, rows * s.R * sizeof(double)));
    CP_TRY(grow(h->Gp, rows * s.R * sizeof(double)));
    CP_TRY(grow(h->stats, sizeof(DevStats)));
    if (!h->h_stats) CUDA_TRY(cudaMallocHost((void**)&h->h_stats, sizeof(DevStats)));
    return CP_OK;
}

static cp_status sync_stats(cp_handle h) {
    CUDA_TRY(cudaMemcpyAsync(h->h_stats, h->stats.p, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return CP_OK;
}

// M (caller or packed pointers) = all-mode MTTKRP of X at `prec`.
static cp_status mttkrp_into(cp_handle h, const cp_desc* d, const Shape& s, const void* X, Ptrs<const double> A,
                             Ptrs<double> M, cp_precision prec, int reserve_sms = 0) {
    for (int n = 0; n < s.N; ++n)
        CUDA_TRY(cudaMemsetAsync(M.p[n], 0, (size_t)s.dims[n] * s.R * sizeof(double), h->stream));
    if (prec == CP_PREC_FP64) {
        launch_mttkrp_f64(s, d->x_dtype, X, A, M, (1u << s.N) - 1u, h->stream);
        h->launches += 2;
    } else if (prec == CP_PREC_BF16X3) {
        h->launches += tc_launch_count(h->split, d, s);
        CP_TRY(grow(h->stats, sizeof(DevStats)));
        CP_TRY(tc_mttkrp_all(h->split, d, s, X, A, M, &((DevStats*)h->stats.p)->status, h->stream));
    } else if (prec == CP_PREC_RESIDUAL) {
        // MTTKRP of the residual tensor E = X - [[A]] (extended precision), as bf16 planes
        CP_TRY(grow(h->stats, sizeof(DevStats)));
        CP_TRY(grow(h->resid_planes, (size_t)PlaneTiling::of(s).total() * 2));
        DevStats* ds = (DevStats*)h->stats.p;
        if (resid_tc_supported(s)) {  // reconstruction on the tensor cores (R <= 64)
            CP_TRY(grow(h->Adf, resid_tc_scratch_bytes(s)));
            h->launches += launch_resid_split_tc(s, d->x_dtype, X, A, h->resid_planes.p, nullptr, h->Adf.p, ds,
                                                 &ds->status, h->stream, reserve_sms);
        } else {
            CP_TRY(grow(h->Adf, resid_scratch_bytes(s)));
            launch_resid_split(s, d->x_dtype, X, A, h->resid_planes.p, nullptr, h->Adf.p, ds, h->stream);
            h->launches += 2;
        }
        CP_TRY(tc_mttkrp_planes(h->split, h->resid_planes.p, s, A, M, &ds->status, h->stream));
        h->launches += (s.R + 63) / 64 * 4;
    } else {
        return CP_ERR_ARG;
    }
    CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

// S, Gamma (FP64) and the float copy of Gamma.
static cp_status gram_gamma(cp_handle h, const Shape& s, Ptrs<const double> A, cudaStream_t st) {
    const int chunks = gram_chunks(s);
    launch_gram_partial(s, A, (double*)h->gram_part.p, chunks, st);
    launch_gamma(s, (const double*)h->gram_part.p, chunks, (double*)h->S.p, (double*)h->Gam.p, (float*)h->GamF.p, st);
    CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

extern "C" {

const char* cp_status_string(cp_status s) {
    switch (s) {
        case CP_OK: return "CP_OK";
        case CP_ERR_ARG: return "CP_ERR_ARG";
        case CP_ERR_CUDA: return "CP_ERR_CUDA";
        case CP_ERR_NOMEM: return "CP_ERR_NOMEM";
        case CP_ERR_UNSUPPORTED: return "CP_ERR_UNSUPPORTED";
        case CP_ERR_NOT_SPD: return "CP_ERR_NOT_SPD";
        case CP_ERR_NONFINITE: return "CP_ERR_NONFINITE";
        case CP_ERR_BREAKDOWN: return "CP_ERR_BREAKDOWN";
        case CP_ERR_TIMEOUT: return "CP_ERR_TIMEOUT";
        case CP_WARN_CG_MAXIT: return "CP_WARN_CG_MAXIT";
    }
    return "CP_UNKNOWN_STATUS";
}

cp_status cp_create(cp_handle* out, int device) {
    if (!out) return CP_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    if (device < 0 || device >= count) return CP_ERR_ARG;
    cp_handle h = new (std::nothrow) cp_handle_s();
    if (!h) return CP_ERR_NOMEM;
    h->device = device;
    *out = h;
    return CP_OK;
}

cp_status cp_destroy(cp_handle h) {
    if (!h) return CP_ERR_ARG;
    {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        DevBuf* bufs[] = {&h->gram_part, &h->grad_part, &h->S, &h->Gam, &h->GamF, &h->Pinv, &h->PinvF, &h->precond_scratch,
                          &h->Mp, &h->Gp, &h->Ap, &h->vec, &h->Ypart, &h->Tm, &h->pcg_part, &h->bar,
                          &h->stats, &h->Y, &h->resid_planes, &h->Adf, &h->Atrial, &h->stats2, &h->tucker, &h->pcg_spill};
        for (DevBuf* b : bufs)
            if (b->p) cudaFree(b->p);
        if (h->h_stats) cudaFreeHost(h->h_stats);
        if (h->h_stats2) cudaFreeHost(h->h_stats2);
        if (h->h_tk) cudaFreeHost(h->h_tk);
        for (auto& e : h->ev)
            if (e) cudaEventDestroy(e);
        if (h->side) {
            cudaStreamSynchronize(h->side);
            cudaStreamDestroy(h->side);
        }
        if (h->fork) cudaEventDestroy(h->fork);
        if (h->gam) cudaEventDestroy(h->gam);
        if (h->join) cudaEventDestroy(h->join);
        split_cache_free(h->split);
        cudaGetLastError();
    }
    delete h;
    return CP_OK;
}

cp_status cp_set_stream(cp_handle h, void* stream) {
    if (!h) return CP_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return CP_OK;
}

cp_status cp_workspace_size(cp_handle h, const cp_desc* d, cp_precision prec, size_t* bytes, size_t* split_bytes) {
    if (!h || !bytes) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    if (prec != CP_PREC_FP64 && prec != CP_PREC_BF16X3 && prec != CP_PREC_RESIDUAL) return CP_ERR_ARG;
    const Shape s = make_shape(d);
    const size_t RR = (size_t)s.R * s.R, rows = (size_t)s.roff[s.N];
    size_t b = 0;
    b += (size_t)s.N * gram_chunks(s) * RR * 8 + s.N * RR * 8 + (size_t)s.N * s.N * RR * 12 + s.N * RR * 12;
    b += rows * s.R * 8 * 2;                    // M, G
    b += rows * s.R * 8 * 7;                    // packed A and CG vectors (FP64 worst case)
    b += (size_t)4096 * RR * 8 + s.N * RR * 8;  // partial A^T W per block, T
    {  // large R: the CG kernel's matrices and row blocks in global memory (FP64 worst case)
        const size_t Rp = (size_t)((s.R + 3) & ~3);
        if ((size_t)(s.N + 2) * s.R * Rp * 8 + 640 > 200 * 1024)
            b += ((size_t)s.N * (s.N + 1) * s.R * Rp + 256 * (size_t)s.R * Rp + 6 * (rows + 256 * s.N) * Rp) * 8;
    }
    if (prec != CP_PREC_FP64) {                 // tensor-core MTTKRP: partial sums and operand planes
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
            cudaGetLastError();
            return CP_ERR_CUDA;
        }
        b += tc_workspace_bytes(s, sms);
    }
    if (prec == CP_PREC_RESIDUAL)  // bf16 planes of E and the reconstruction's scratch
        b += (size_t)PlaneTiling::of(s).total() * 2 +
             (resid_tc_supported(s) ? resid_tc_scratch_bytes(s) : resid_scratch_bytes(s));
    *bytes = b;
    if (split_bytes) *split_bytes = prec == CP_PREC_BF16X3 ? split_cache_bytes(d) : 0;
    return CP_OK;
}

cp_status cp_mttkrp_all(cp_handle h, const cp_desc* d, const void* X, const double* const* A, double* const* M,
                        cp_precision prec) {
    if (!h || !X) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    CP_TRY(check_ptrs((const void* const*)M, d->order));
    if (aliased((const void* const*)M, d->order, (const void* const*)A, d->order, X)) return CP_ERR_ARG;
    if (prec != CP_PREC_FP64 && prec != CP_PREC_BF16X3) return CP_ERR_ARG;  // RESIDUAL is gradient-only
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    return mttkrp_into(h, d, s, X, ptrs_of(A, s.N), ptrs_of(M, s.N), prec);
}

cp_status cp_gradient(cp_handle h, const cp_desc* d, const void* X, const double* const* A, double* const* G,
                      cp_precision prec, double* gnorm, double* mnorm) {
    if (!h || !X) return CP_ERR_ARG;
    if (prec != CP_PREC_FP64 && prec != CP_PREC_BF16X3 && prec != CP_PREC_RESIDUAL) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    CP_TRY(check_ptrs((const void* const*)G, d->order));
    if (aliased((const void* const*)G, d->order, (const void* const*)A, d->order, X)) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(ensure_common(h, s));
    const Ptrs<const double> Ap = ptrs_of(A, s.N);
    CUDA_TRY(cudaMemsetAsync(h->stats.p, 0, sizeof(DevStats), h->stream));
    CP_TRY(mttkrp_into(h, d, s, X, Ap, packed_ptrs((double*)h->Mp.p, s), prec));
    CP_TRY(gram_gamma(h, s, Ap, h->stream));
    launch_gradient(s, Ap, (const double*)h->Gam.p, (const double*)h->Mp.p, (double*)h->Gp.p,
                    (double*)h->grad_part.p, (DevStats*)h->stats.p, h->stream, prec == CP_PREC_RESIDUAL);
    launch_unpack(s, (const double*)h->Gp.p, ptrs_of(G, s.N), h->stream);
    CUDA_TRY(cudaGetLastError());
    CP_TRY(sync_stats(h));
    for (int n = 0; n < s.N; ++n) {
        if (gnorm) gnorm[n] = sqrt(h->h_stats->gnorm2[n]);
        if (mnorm) mnorm[n] = sqrt(h->h_stats->mnorm2[n]);
    }
    return h->h_stats->status ? (cp_status)h->h_stats->status : CP_OK;
}

cp_status cp_gn_matvec(cp_handle h, const cp_desc* d, const double* const* A, const double* grams,
                       const double* const* W, double lambda, int reg, double* const* Q, cp_precision prec) {
    if (!h) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    CP_TRY(check_ptrs((const void* const*)W, d->order));
    CP_TRY(check_ptrs((const void* const*)Q, d->order));
    if (aliased((const void* const*)Q, d->order, (const void* const*)A, d->order, grams)) return CP_ERR_ARG;
    if (aliased((const void* const*)Q, d->order, (const void* const*)W, d->order, nullptr)) return CP_ERR_ARG;
    if (!(lambda >= 0.0) || !isfinite(lambda)) return CP_ERR_ARG;
    if (reg != CP_REG_IDENTITY && reg != CP_REG_DIAG) return CP_ERR_ARG;
    if (prec != CP_PREC_FP64 && prec != CP_PREC_BF16X3 && prec != CP_PREC_RESIDUAL) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(ensure_common(h, s));
    CP_TRY(grow(h->Y, (size_t)s.N * s.R * s.R * sizeof(double)));
    const Ptrs<const double> Ap = ptrs_of(A, s.N);
    if (grams) {  // the caller's Gram matrices: Gamma from them directly
        launch_gamma(s, grams, 1, (double*)h->S.p, (double*)h->Gam.p, nullptr, h->stream);
        CUDA_TRY(cudaGetLastError());
    } else {
        CP_TRY(gram_gamma(h, s, Ap, h->stream));
    }
    const bool diag = reg == CP_REG_DIAG;
    if (prec == CP_PREC_FP64)
        launch_matvec<double>(s, Ap, (const double*)h->Gam.p, ptrs_of(W, s.N), lambda, diag, ptrs_of(Q, s.N),
                              (double*)h->Y.p, h->stream);
    else
        launch_matvec<float>(s, Ap, (const double*)h->Gam.p, ptrs_of(W, s.N), lambda, diag, ptrs_of(Q, s.N),
                             (float*)h->Y.p, h->stream);
    CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

}  // extern "C"

static void lambda_advance(cp_gn_params* p) {
    if (p->lam_fixed) return;
    if (p->lam_dir == 0) {
        const double t = p->lam / p->mu;
        if (t < p->lam_lo) {
            p->lam_dir = 1;
            p->lam = p->lam * p->mu;
        } else {
            p->lam = t;
        }
    } else {
        const double t = p->lam * p->mu;
        if (t > p->lam_hi) {
            p->lam_dir = 0;
            p->lam = p->lam / p->mu;
        } else {
            p->lam = t;
        }
    }
}

template <typename T>
static cp_status gn_pcg(cp_handle h, const Shape& s, Ptrs<const double> Acaller, const cp_gn_params* p) {
    const size_t RR = (size_t)s.R * s.R, len = (size_t)s.roff[s.N] * s.R;
    int nblocks = 0;
    size_t spill = 0;
    CP_TRY(pcg_plan<T>(s, 0, &nblocks, &spill));
    CP_TRY(grow(h->Ap, len * sizeof(T)));
    CP_TRY(grow(h->vec, len * sizeof(T)));
    CP_TRY(grow(h->Ypart, (size_t)nblocks * RR * sizeof(T)));  // per-block A^T Z
    CP_TRY(grow(h->Tm, s.N * RR * sizeof(T)));                   // Y^(p), reduced
    if (spill) CP_TRY(grow(h->pcg_spill, spill * sizeof(T)));    // large R: matrices and rows in global memory
    CP_TRY(grow(h->pcg_part, 3 * 4096 * sizeof(double)));
    CP_TRY(grow(h->bar, sizeof(GridBarrier)));
    launch_pack<T>(s, Acaller, (T*)h->Ap.p, h->stream);
    CUDA_TRY(cudaEventRecord(h->ev[2], h->stream));
    PcgArgs<T> a{};
    a.s = s;
    a.Ap = (const T*)h->Ap.p;
    if (sizeof(T) == 4) {
        a.GamT = (const T*)h->GamF.p;
        a.PinvT = (const T*)h->PinvF.p;
    } else {
        a.GamT = (const T*)h->Gam.p;
        a.PinvT = (const T*)h->Pinv.p;
    }
    a.G = (const double*)h->Gp.p;
    a.V = (T*)h->vec.p;
    a.Zpart = (T*)h->Ypart.p;
    a.Yfull = (T*)h->Tm.p;
    a.part = (double*)h->pcg_part.p;
    a.spill = spill ? (T*)h->pcg_spill.p : nullptr;
    a.bar = (GridBarrier*)h->bar.p;
    a.stats = (DevStats*)h->stats.p;
    a.lam = p->lam;
    a.eps_cg = p->eps_cg;
    a.stop_ratio = p->stop_stationarity;
    a.maxit = p->cg_max_iter;
    a.spin_limit = p->spin_limit > 0 ? p->spin_limit : kDefaultSpin;
    CUDA_TRY(cudaMemsetAsync(h->bar.p, 0, sizeof(GridBarrier), h->stream));
    CP_TRY(launch_pcg<T>(a, 0, h->stream));
    h->cg_blocks = a.nblocks;
    return CP_OK;
}

static cp_status gn_step_impl(cp_handle h, const cp_desc* d, const void* X, double* const* A, cp_gn_params* p,
                              cp_gn_stats* st) {
    const Shape s = make_shape(d);
    CP_TRY(ensure_common(h, s));
    CP_TRY(ensure_events(h));
    h->launches = 0;
    const Ptrs<const double> Ac = ptrs_of((const double* const*)A, s.N);
    DevStats* ds = (DevStats*)h->stats.p;
    CUDA_TRY(cudaEventRecord(h->ev[0], h->stream));
    CUDA_TRY(cudaMemsetAsync(ds, 0, sizeof(DevStats), h->stream));
    // Algorithm 1: MTTKRP, Gamma^(n,p), G^(n) = A^(n) Gamma^(n,n) - M^(n).
    // With identity damping, Gamma and P_inv = (Gamma^(n,n) + lambda I)^{-1} (Algorithm 2)
    // depend on A and lambda only: they run on a second stream beside the MTTKRP, whose
    // persistent reconstruction leaves N SMs to them.  (The diagonal damping changes
    // Gamma^(n,n) after the gradient has used it, so it keeps the serial order.)
    cp_gn_params q = *p;
    const bool beside = p->reg != CP_REG_DIAG;
    if (beside) {
        CUDA_TRY(cudaEventRecord(h->fork, h->stream));
        CUDA_TRY(cudaStreamWaitEvent(h->side, h->fork, 0));
        CP_TRY(gram_gamma(h, s, Ac, h->side));
        CUDA_TRY(cudaEventRecord(h->gam, h->side));
        launch_precond(s, (const double*)h->Gam.p, q.lam, (double*)h->Pinv.p, (float*)h->PinvF.p,
                       (double*)h->precond_scratch.p, ds, h->side, p->cg_fp32 != 0);
        h->launches += 3;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(h->join, h->side));
    }
    CUDA_TRY(cudaEventRecord(h->ev[4], h->stream));
    CP_TRY(mttkrp_into(h, d, s, X, Ac, packed_ptrs((double*)h->Mp.p, s), p->prec, beside ? s.N : 0));
    CUDA_TRY(cudaEventRecord(h->ev[1], h->stream));
    if (beside) {
        CUDA_TRY(cudaStreamWaitEvent(h->stream, h->gam, 0));  // the gradient reads Gamma
    } else {
        CP_TRY(gram_gamma(h, s, Ac, h->stream));
        h->launches += 2;
    }
    launch_gradient(s, Ac, (const double*)h->Gam.p, (const double*)h->Mp.p, (double*)h->Gp.p,
                    (double*)h->grad_part.p, ds, h->stream, p->prec == CP_PREC_RESIDUAL);
    h->launches += 2;  // the gradient and its fixed-order norm reduction
    if (beside) {
        CUDA_TRY(cudaStreamWaitEvent(h->stream, h->join, 0));
    } else {
        // Damping lam diag(J^T J): fold it into the diagonals of Gamma^(n,n) (the
        // gradient above used them undamped) and solve the system with lam = 0.
        launch_damp_diag(s, (double*)h->Gam.p, (float*)h->GamF.p, p->lam, h->stream);
        h->launches += 1;
        q.lam = 0.0;
        // Algorithm 2: P_inv = (Gamma^(n,n) + lambda D)^{-1}, then CG
        launch_precond(s, (const double*)h->Gam.p, q.lam, (double*)h->Pinv.p, (float*)h->PinvF.p,
                       (double*)h->precond_scratch.p, ds, h->stream, p->cg_fp32 != 0);
        h->launches += 1;
    }
    CUDA_TRY(cudaGetLastError());
    if (p->cg_fp32)
        CP_TRY(gn_pcg<float>(h, s, Ac, &q));
    else
        CP_TRY(gn_pcg<double>(h, s, Ac, &q));
    h->launches += 2;  // pack + persistent CG
    // Step-size control by Armijo's condition (Section 5): t in 1, beta, beta^2, ...
    double t_step = 1.0, f0 = -1.0;
    int trials = 0;
    bool search = p->armijo_c > 0.0;
    if (search) {  // only after a CG solve that succeeded
        CP_TRY(sync_stats(h));
        const int cs = h->h_stats->status;
        search = (cs == CP_OK || cs == CP_WARN_CG_MAXIT) && !h->h_stats->stopped;
    }
    if (search) {
        const int64_t len = (int64_t)s.roff[s.N] * s.R;
        CP_TRY(grow(h->Atrial, (size_t)len * sizeof(double)));
        CP_TRY(grow(h->stats2, sizeof(DevStats)));
        if (!h->h_stats2) CUDA_TRY(cudaMallocHost((void**)&h->h_stats2, sizeof(DevStats)));
        DevStats* d2 = (DevStats*)h->stats2.p;
        if (p->cg_fp32)
            launch_dot_gv<float>(len, (const double*)h->Gp.p, (const float*)h->vec.p, d2->dot_part, &d2->slope,
                                 h->stream);
        else
            launch_dot_gv<double>(len, (const double*)h->Gp.p, (const double*)h->vec.p, d2->dot_part, &d2->slope,
                                  h->stream);
        CUDA_TRY(cudaMemsetAsync(&d2->res_num, 0, 2 * sizeof(double), h->stream));
        launch_residual_f64(s, d->x_dtype, X, Ac, d2, h->stream);
        h->launches += 3;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(h->h_stats2, d2, sizeof(DevStats), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        f0 = 0.5 * h->h_stats2->res_num;
        const double slope = h->h_stats2->slope;
        // relaxed by the accuracy of the FP64 evaluation of f (2 R 2^-53 ||X||^2)
        const double tol_f = 2.0 * s.R * 0x1p-53 * h->h_stats2->res_den;
        double t = 1.0;
        t_step = 0.0;
        double* At = (double*)h->Atrial.p;
        for (int k = 0; k <= p->armijo_max; ++k, t *= p->armijo_beta) {
            if (p->cg_fp32)
                launch_trial_factors<float>(s, Ac, (const float*)h->vec.p, t, At, h->stream);
            else
                launch_trial_factors<double>(s, Ac, (const double*)h->vec.p, t, At, h->stream);
            CUDA_TRY(cudaMemsetAsync(&d2->res_num, 0, 2 * sizeof(double), h->stream));
            launch_residual_f64(s, d->x_dtype, X, as_const(packed_ptrs(At, s)), d2, h->stream);
            h->launches += 2;
            ++trials;
            CUDA_TRY(cudaGetLastError());
            CUDA_TRY(cudaMemcpyAsync(&h->h_stats2->res_num, &d2->res_num, sizeof(double), cudaMemcpyDeviceToHost,
                                     h->stream));
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            if (0.5 * h->h_stats2->res_num <= f0 + p->armijo_c * t * slope + tol_f) {
                t_step = t;
                break;
            }
        }
    }
    // A^(n) += t V^(n)
    Ptrs<double> Am = ptrs_of(A, s.N);
    if (p->cg_fp32)
        launch_update<float>(s, Am, (const float*)h->vec.p, ds, h->stream, t_step);
    else
        launch_update<double>(s, Am, (const double*)h->vec.p, ds, h->stream, t_step);
    h->launches += 1;
    if (p->want_residual) {
        launch_residual_f64(s, d->x_dtype, X, as_const(Am), ds, h->stream);
        h->launches += 1;
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(h->ev[3], h->stream));
    CP_TRY(sync_stats(h));
    const DevStats& hs = *h->h_stats;
    cp_status status = (cp_status)hs.status;
    if (st) {
        memset(st, 0, sizeof(*st));
        st->status = status;
        st->cg_iters = hs.cg_iters;
        st->stopped = hs.stopped;
        for (int n = 0; n < s.N; ++n) {
            st->grad_norm_sum += sqrt(hs.gnorm2[n]);
            st->m_norm_sum += sqrt(hs.mnorm2[n]);
            st->update_norm_sum += sqrt(hs.vnorm2[n]);
            st->factor_norm_sum += sqrt(hs.anorm2[n]);
        }
        st->lam_used = p->lam;
        st->cg_rnorm = hs.cg_rnorm;
        st->rel_residual = p->want_residual ? sqrt(hs.res_num) / sqrt(hs.res_den) : -1.0;
        st->entry_residual = p->prec == CP_PREC_RESIDUAL ? sqrt(hs.eres_num) / sqrt(hs.eres_den) : -1.0;
        float t01 = 0.f, t23 = 0.f, t03 = 0.f;
        cudaEventElapsedTime(&t01, h->ev[4], h->ev[1]);
        cudaEventElapsedTime(&t23, h->ev[2], h->ev[3]);
        cudaEventElapsedTime(&t03, h->ev[0], h->ev[3]);
        cudaGetLastError();
        st->mttkrp_ms = t01;
        st->pcg_ms = t23;  // CG kernel plus the factor update
        st->step_ms = t03;
        st->kernel_launches = h->launches;
        st->cg_blocks = h->cg_blocks;
        st->step = t_step;
        st->f_entry = f0;
        st->ls_trials = trials;
    }
    if ((status == CP_OK || status == CP_WARN_CG_MAXIT) && !hs.stopped) lambda_advance(p);
    return status;
}

static cp_status check_params(const cp_gn_params* p) {
    if (!p) return CP_ERR_ARG;
    if (!(p->eps_cg >= 0.0) || p->cg_max_iter < 0) return CP_ERR_ARG;
    if (!(p->lam >= 0.0) || !isfinite(p->lam)) return CP_ERR_ARG;
    if (p->reg != CP_REG_IDENTITY && p->reg != CP_REG_DIAG) return CP_ERR_ARG;
    if (!p->lam_fixed && !(p->mu > 1.0 && p->lam_lo > 0.0 && p->lam_hi >= p->lam_lo)) return CP_ERR_ARG;
    if (p->prec != CP_PREC_FP64 && p->prec != CP_PREC_BF16X3 && p->prec != CP_PREC_RESIDUAL) return CP_ERR_ARG;
    if (!(p->armijo_c >= 0.0 && p->armijo_c < 1.0)) return CP_ERR_ARG;
    if (p->armijo_c > 0.0 && (!(p->armijo_beta > 0.0 && p->armijo_beta < 1.0) || p->armijo_max < 0)) return CP_ERR_ARG;
    return CP_OK;
}

extern "C" {

cp_status cp_gn_step(cp_handle h, const cp_desc* d, const void* X, double* const* A, cp_gn_params* p,
                     cp_gn_stats* st) {
    if (!h || !X) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    CP_TRY(check_params(p));
    if (aliased((const void* const*)A, d->order, nullptr, 0, X)) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    return gn_step_impl(h, d, X, A, p, st);
}

cp_status cp_gn_solve(cp_handle h, const cp_desc* d, const void* X, double* const* A, cp_gn_params* p,
                      const cp_solve_opts* o, cp_solve_result* res) {
    if (!h || !X || !o || !res) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    CP_TRY(check_params(p));
    if (o->max_iters < 0) return CP_ERR_ARG;
    if (aliased((const void* const*)A, d->order, nullptr, 0, X)) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    memset(res, 0, sizeof(*res));
    res->rel_residual = -1.0;
    const cp_precision base_prec = p->prec;
    const cp_precision refine_prec = o->refine_prec == CP_PREC_FP64 ? CP_PREC_FP64 : CP_PREC_RESIDUAL;
    bool refining = base_prec != CP_PREC_BF16X3;
    cp_status status = CP_OK;
    for (int it = 0; it < o->max_iters; ++it) {
        cp_gn_params q = *p;
        q.prec = refining ? (base_prec == CP_PREC_BF16X3 ? refine_prec : base_prec) : base_prec;
        // Algorithm 1's loop test on sum||G||: only trusted with an FP64-accurate gradient
        q.stop_stationarity = refining ? o->target_stationarity : 0.0;
        const bool resid_now = o->target_residual > 0.0 || (o->residual_every > 0 && (it + 1) % o->residual_every == 0);
        q.want_residual = resid_now ? 1 : 0;
        cp_gn_stats st;
        status = gn_step_impl(h, d, X, A, &q, &st);
        p->lam = q.lam;
        p->lam_dir = q.lam_dir;
        res->cg_iters_total += st.cg_iters;
        res->mttkrp_ms += st.mttkrp_ms;
        res->pcg_ms += st.pcg_ms;
        res->device_ms += st.step_ms;
        res->kernel_launches += st.kernel_launches;
        res->cg_blocks = st.cg_blocks;
        res->stationarity = st.m_norm_sum > 0 ? st.grad_norm_sum / st.m_norm_sum : 0.0;
        if (status != CP_OK && status != CP_WARN_CG_MAXIT) break;
        if (st.stopped) {  // no update was applied: the entry point met the target
            res->converged = 1;
            break;
        }
        ++res->iters;
        if (q.prec != base_prec) ++res->iters_refined;
        if (resid_now) res->rel_residual = st.rel_residual;
        if (o->target_residual > 0.0 && st.rel_residual <= o->target_residual) {
            res->converged = 1;
            break;
        }
        if (!refining && o->refine_below > 0.0 && res->stationarity <= o->refine_below) refining = true;
    }
    res->lam = p->lam;
    res->status = status;
    return status == CP_WARN_CG_MAXIT ? CP_OK : status;
}

cp_status cp_als_sweep(cp_handle h, const cp_desc* d, const void* X, double* const* A, double lambda,
                       cp_precision prec, double* rel_residual) {
    if (!h || !X) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    if (!(lambda >= 0.0) || !isfinite(lambda)) return CP_ERR_ARG;
    if (prec != CP_PREC_FP64 && prec != CP_PREC_BF16X3) return CP_ERR_ARG;
    if (aliased((const void* const*)A, d->order, nullptr, 0, X)) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(ensure_common(h, s));
    DevStats* ds = (DevStats*)h->stats.p;
    CUDA_TRY(cudaMemsetAsync(ds, 0, sizeof(DevStats), h->stream));
    const Ptrs<const double> Ac = ptrs_of((const double* const*)A, s.N);
    Ptrs<double> Mp = packed_ptrs((double*)h->Mp.p, s);
    for (int n = 0; n < s.N; ++n) {
        CP_TRY(gram_gamma(h, s, Ac, h->stream));
        CUDA_TRY(cudaMemsetAsync(Mp.p[n], 0, (size_t)s.dims[n] * s.R * sizeof(double), h->stream));
        if (prec == CP_PREC_FP64)
            launch_mttkrp_f64(s, d->x_dtype, X, Ac, Mp, 1u << n, h->stream);
        else
            CP_TRY(tc_mttkrp_mode(h->split, d, s, X, Ac, Mp, n, &ds->status, h->stream));
        launch_precond(s, (const double*)h->Gam.p, lambda, (double*)h->Pinv.p, nullptr,
                       (double*)h->precond_scratch.p, ds, h->stream);
        launch_als_solve(s, n, Mp.p[n], (const double*)h->Pinv.p + (size_t)n * s.R * s.R, A[n], h->stream);
        CUDA_TRY(cudaGetLastError());
    }
    if (rel_residual) {
        launch_residual_f64(s, d->x_dtype, X, Ac, ds, h->stream);
        CP_TRY(sync_stats(h));
        *rel_residual = sqrt(h->h_stats->res_num) / sqrt(h->h_stats->res_den);
        if (h->h_stats->status) return (cp_status)h->h_stats->status;
    }
    return CP_OK;
}

cp_status cp_residual(cp_handle h, const cp_desc* d, const void* X, const double* const* A, double* rel_residual) {
    if (!h || !X || !rel_residual) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(grow(h->stats, sizeof(DevStats)));
    if (!h->h_stats) CUDA_TRY(cudaMallocHost((void**)&h->h_stats, sizeof(DevStats)));
    CUDA_TRY(cudaMemsetAsync(h->stats.p, 0, sizeof(DevStats), h->stream));
    launch_residual_f64(s, d->x_dtype, X, ptrs_of(A, s.N), (DevStats*)h->stats.p, h->stream);
    CUDA_TRY(cudaGetLastError());
    CP_TRY(sync_stats(h));
    *rel_residual = sqrt(h->h_stats->res_num) / sqrt(h->h_stats->res_den);
    return CP_OK;
}

cp_status cp_gn_solve_batched(cp_handle h, int nprob, const cp_batch_problem* problems, double eps_cg,
                              int cg_max_iter, int max_iters, double target_residual, cp_batch_result* results) {
    if (!h || nprob < 0 || (nprob > 0 && (!problems || !results)) || cg_max_iter < 0 || max_iters < 0 ||
        !(eps_cg >= 0.0))
        return CP_ERR_ARG;
    if (nprob == 0) return CP_OK;
    DeviceGuard g(h->device);
    return no_throw([&] {
        return run_batched(h->device, h->stream, nprob, problems, eps_cg, cg_max_iter, max_iters, target_residual,
                           results);
    });
}

}  // extern "C"

struct cp_batch_plan_s {
    int device;
    int nprob;
    cpgn::BatchPlan* p;
};

extern "C" {

cp_status cp_batch_plan_create(cp_handle h, int nprob, const cp_batch_problem* problems, double eps_cg,
                               int cg_max_iter, int max_iters, double target_residual, int autotune,
                               cp_batch_plan* plan) {
    if (!h || !plan || nprob < 1 || !problems || cg_max_iter < 0 || max_iters < 0 || !(eps_cg >= 0.0))
        return CP_ERR_ARG;
    *plan = nullptr;
    DeviceGuard g(h->device);
    BatchPlan* p = nullptr;
    CP_TRY(no_throw([&] {
        return batch_plan_create(h->device, h->stream, nprob, problems, eps_cg, cg_max_iter, max_iters,
                                 target_residual, autotune, &p);
    }));
    *plan = new (std::nothrow) cp_batch_plan_s{h->device, nprob, p};
    if (!*plan) {
        batch_plan_destroy(p);
        return CP_ERR_NOMEM;
    }
    return CP_OK;
}

cp_status cp_batch_plan_launch(cp_handle h, cp_batch_plan plan) {
    if (!h || !plan || plan->device != h->device) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    return batch_plan_launch(plan->p, h->stream);
}

cp_status cp_batch_plan_results(cp_handle h, cp_batch_plan plan, cp_batch_result* results) {
    if (!h || !plan || !results || plan->device != h->device) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    return no_throw([&] { return batch_plan_results(plan->p, h->stream, results); });
}

cp_status cp_batch_plan_threads(cp_batch_plan plan, int* threads) {
    if (!plan || !threads) return CP_ERR_ARG;
    *threads = batch_plan_threads(plan->p);
    return CP_OK;
}

cp_status cp_batch_plan_configure(cp_batch_plan plan, int threads, int order) {
    if (!plan) return CP_ERR_ARG;
    DeviceGuard g(plan->device);
    return batch_plan_configure(plan->p, threads, order);
}

cp_status cp_batch_plan_order(cp_batch_plan plan, int* order) {
    if (!plan || !order) return CP_ERR_ARG;
    *order = batch_plan_order(plan->p);
    return CP_OK;
}

cp_status cp_batch_plan_destroy(cp_batch_plan plan) {
    if (!plan) return CP_ERR_ARG;
    {
        DeviceGuard g(plan->device);  // the caller's current device is restored
        batch_plan_destroy(plan->p);
    }
    delete plan;
    return CP_OK;
}

cp_status cp_residual_sums(cp_handle h, const cp_desc* d, const void* X, const double* const* A, double* sq_err,
                           double* sq_x) {
    if (!h || !X) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(grow(h->stats, sizeof(DevStats)));
    if (!h->h_stats) CUDA_TRY(cudaMallocHost((void**)&h->h_stats, sizeof(DevStats)));
    CUDA_TRY(cudaMemsetAsync(h->stats.p, 0, sizeof(DevStats), h->stream));
    launch_residual_f64(s, d->x_dtype, X, ptrs_of(A, s.N), (DevStats*)h->stats.p, h->stream);
    CUDA_TRY(cudaGetLastError());
    CP_TRY(sync_stats(h));
    if (sq_err) *sq_err = h->h_stats->res_num;
    if (sq_x) *sq_x = h->h_stats->res_den;
    return CP_OK;
}

cp_status cp_hosvd(cp_handle h, const cp_desc* d, const void* X, const int* ranks, double* const* U, double* core,
                   int* iters) {
    if (!h || !X || !ranks || !core) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)U, d->order));
    for (int n = 0; n < d->order; ++n)
        if (ranks[n] < 1 || ranks[n] > d->dims[n] || ranks[n] > CP_MAX_RANK) return CP_ERR_ARG;
    if (aliased((const void* const*)U, d->order, nullptr, 0, X) || core == X) return CP_ERR_ARG;
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int64_t smax = 1;
    for (int n = 0; n < s.N; ++n) smax = std::max<int64_t>(smax, s.dims[n]);
    const int64_t tiles = (smax + 31) / 32;
    const int slabs = (int)std::max<int64_t>(1, std::min<int64_t>(64, (2 * sms + tiles * (tiles + 1) / 2 - 1) /
                                                                          (tiles * (tiles + 1) / 2)));
    CP_TRY(grow(h->tucker, hosvd_scratch_doubles(s, ranks, slabs) * sizeof(double)));
    if (!h->h_tk) CUDA_TRY(cudaMallocHost((void**)&h->h_tk, 4 * sizeof(double)));
    return launch_hosvd(s, d->x_dtype, X, ranks, U, core, iters, (double*)h->tucker.p, slabs, h->h_tk, h->stream);
}

cp_status cp_tucker_expand(cp_handle h, int order, const int64_t* dims, const int* ranks, int R,
                           const double* const* U, const double* const* B, double* const* A) {
    if (!h || !dims || !ranks || order < 1 || order > CP_MAX_ORDER || R < 1 || R > CP_MAX_RANK) return CP_ERR_ARG;
    CP_TRY(check_ptrs((const void* const*)U, order));
    CP_TRY(check_ptrs((const void* const*)B, order));
    CP_TRY(check_ptrs((const void* const*)A, order));
    for (int n = 0; n < order; ++n)
        if (dims[n] < 1 || ranks[n] < 1 || ranks[n] > dims[n]) return CP_ERR_ARG;
    if (aliased((const void* const*)A, order, (const void* const*)U, order, nullptr) ||
        aliased((const void* const*)A, order, (const void* const*)B, order, nullptr))
        return CP_ERR_ARG;
    DeviceGuard g(h->device);
    for (int n = 0; n < order; ++n) launch_tucker_expand(dims[n], ranks[n], R, U[n], B[n], A[n], h->stream);
    CUDA_TRY(cudaGetLastError());
    return CP_OK;
}

cp_status cp_residual_tensor(cp_handle h, const cp_desc* d, const void* X, const double* const* A, double* E,
                             double* sq_err, double* sq_x) {
    if (!h || !X) return CP_ERR_ARG;
    CP_TRY(check_desc(d));
    CP_TRY(check_ptrs((const void* const*)A, d->order));
    if (E) {
        const void* out[1] = {E};
        if (aliased(out, 1, (const void* const*)A, d->order, X)) return CP_ERR_ARG;
    }
    DeviceGuard g(h->device);
    const Shape s = make_shape(d);
    CP_TRY(grow(h->stats, sizeof(DevStats)));
    if (!h->h_stats) CUDA_TRY(cudaMallocHost((void**)&h->h_stats, sizeof(DevStats)));
    DevStats* ds = (DevStats*)h->stats.p;
    CUDA_TRY(cudaMemsetAsync(ds, 0, sizeof(DevStats), h->stream));
    if (resid_tc_supported(s)) {
        CP_TRY(grow(h->Adf, resid_tc_scratch_bytes(s)));
        launch_resid_split_tc(s, d->x_dtype, X, ptrs_of(A, s.N), nullptr, E, h->Adf.p, ds, &ds->status, h->stream);
    } else {
        CP_TRY(grow(h->Adf, resid_scratch_bytes(s)));
        launch_resid_split(s, d->x_dtype, X, ptrs_of(A, s.N), nullptr, E, h->Adf.p, ds, h->stream);
    }
    CUDA_TRY(cudaGetLastError());
    CP_TRY(sync_stats(h));
    if (sq_err) *sq_err = h->h_stats->eres_num;
    if (sq_x) *sq_x = h->h_stats->eres_den;
    return h->h_stats->status ? (cp_status)h->h_stats->status : CP_OK;
}

}  // extern "C"
