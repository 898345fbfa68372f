// k_noalloc.cu -- the implicit Gauss-Newton matvec for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed,
// pre-reserved device-memory budget, code inside an allocator or
// memory-pool callback, and long-running serving loops that must not
// allocate after start-up.  cp_gn_matvec needs a handle whose workspace
// grows with cudaMalloc; this variant keeps its scratch (the Gram matrices,
// the Gamma set and Y^(p) = A^(p)^T W^(p)) in one file-scope device array of
// fixed size instead, so a call allocates nothing.
//
// The array is part of the library's device image: every GPU on which the
// library's module is loaded holds it (CP_NOALLOC_SCRATCH_BYTES) until the
// process exits.  Host code cannot use its name as a device address, so the
// first call on each device (with that device current) asks the runtime for
// the array's address there (cudaGetSymbolAddress) and caches it together
// with the identity of the current CUDA context; a later call in another
// context (after cudaDeviceReset, or once the primary context was released
// and created again) looks the address up afresh instead of reusing a stale
// one.  That first call also makes the runtime load the modules of every
// kernel the call launches (through cudaFuncGetAttributes), which commits
// their device memory, this array included: make the first call on a device
// before any region in which nothing may be allocated, and before any
// stream capture.  Every call overwrites all of the scratch it reads
// (nothing accumulates from an earlier call), and all calls share the one
// array: calls that overlap on the GPU (two streams, two host threads) race
// and must be serialised by the caller.
#include <math.h>

#include <mutex>

#include "kernels.hpp"

namespace cpgn {
namespace {

constexpr int kMaxOrder = CP_NOALLOC_MAX_ORDER;
constexpr int kMaxRank = CP_NOALLOC_MAX_RANK;
constexpr int kMaxDevices = 64;
// S (N R^2) + Y (N R^2) + Gamma (N^2 R^2) at the largest supported N and R
constexpr size_t kScratchDoubles = (size_t)(2 * kMaxOrder + kMaxOrder * kMaxOrder) * kMaxRank * kMaxRank;
static_assert(kScratchDoubles * sizeof(double) == CP_NOALLOC_SCRATCH_BYTES, "scratch size mismatch");

}  // namespace

static __device__ __align__(256) double g_matvec_scratch[kScratchDoubles];

namespace {

// Identity of the current CUDA context (its unique id where the driver
// offers cuCtxGetId, else its handle); 0 if none can be had.
unsigned long long current_context_id() {
    typedef int (*GetCurrentFn)(void**);
    typedef int (*GetIdFn)(void*, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetIdFn)f;
        cudaGetLastError();
    });
    void* ctx = nullptr;
    if (!get_current || get_current(&ctx) != 0 || !ctx) return 0;
    unsigned long long id = 0;
    if (get_id && get_id(ctx, &id) == 0) return id + 1;
    return (unsigned long long)(uintptr_t)ctx;
}

struct ScratchAddr {
    unsigned long long ctx = 0;  // context the address belongs to (0: none cached)
    double* p = nullptr;
};
std::mutex g_addr_mu;
ScratchAddr g_addr[kMaxDevices];

__global__ void gram_direct_kernel(Shape s, Ptrs<const double> A, double* S);
__global__ void gamma_direct_kernel(Shape s, const double* S, double* Gam);

// Device address of the scratch array in the current device's current
// context, looked up once per (device, context).  The lookup also loads the
// modules of every kernel a call launches.
cp_status scratch_on(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return CP_ERR_UNSUPPORTED;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_addr_mu);
    ScratchAddr& c = g_addr[dev];
    if (!c.p || ctx == 0 || c.ctx != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_matvec_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CP_ERR_CUDA;
        }
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, gram_direct_kernel) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, gamma_direct_kernel) != cudaSuccess || preload_matvec_f64() != cudaSuccess) {
            cudaGetLastError();
            return CP_ERR_CUDA;
        }
        c.p = static_cast<double*>(p);
        c.ctx = current_context_id();  // the lookup created the context if there was none
    }
    *out = c.p;
    return CP_OK;
}

// S^(n)_{rz} = sum_i a^(n)_{ir} a^(n)_{iz}: one thread per entry, all rows.
__global__ void gram_direct_kernel(Shape s, Ptrs<const double> A, double* S) {
    const int R = s.R, RR = R * R;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= s.N * RR) return;
    const int n = e / RR, q = e % RR, r = q / R, z = q % R;
    const double* a = A.p[n];
    double acc = 0.0;
    for (int64_t i = 0; i < s.dims[n]; ++i) acc += a[i * R + r] * a[i * R + z];
    S[e] = acc;
}

// Gamma^(n,p)_{rz} = prod_{m != n,p} S^(m)_{rz}
__global__ void gamma_direct_kernel(Shape s, const double* S, double* Gam) {
    const int R = s.R, RR = R * R, N = s.N;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= RR) return;
    for (int n = 0; n < N; ++n)
        for (int p = 0; p < N; ++p) {
            double prod = 1.0;
            for (int m = 0; m < N; ++m)
                if (m != n && m != p) prod *= S[(int64_t)m * RR + q];
            Gam[((int64_t)n * N + p) * RR + q] = prod;
        }
}

bool any_null(const void* const* P, int n) {
    if (!P) return true;
    for (int i = 0; i < n; ++i)
        if (!P[i]) return true;
    return false;
}

}  // namespace
}  // namespace cpgn

using namespace cpgn;

extern "C" cp_status cp_gn_matvec_noalloc(const cp_desc* d, const double* const* A, const double* const* W,
                                          double lambda, double* const* Q, void* stream) {
    if (!d || d->order < 2 || d->rank < 1) return CP_ERR_ARG;
    if (d->order > kMaxOrder || d->rank > kMaxRank) return CP_ERR_UNSUPPORTED;  // beyond the static scratch
    for (int n = 0; n < d->order; ++n)
        if (d->dims[n] < 1 || d->dims[n] > (1LL << 31)) return CP_ERR_ARG;
    if (any_null((const void* const*)A, d->order) || any_null((const void* const*)W, d->order) ||
        any_null((const void* const*)Q, d->order))
        return CP_ERR_ARG;
    for (int i = 0; i < d->order; ++i)
        for (int j = 0; j < d->order; ++j)
            if ((const void*)Q[i] == (const void*)A[j] || (const void*)Q[i] == (const void*)W[j] ||
                (i != j && Q[i] == Q[j]))
                return CP_ERR_ARG;
    if (!(lambda >= 0.0) || !isfinite(lambda)) return CP_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_CUDA;
    }
    double* scratch = nullptr;
    cp_status st = CP_OK;
    try {  // the lookup's mutex may throw; nothing may leave the C ABI
        st = scratch_on(dev, &scratch);
    } catch (...) {
        return CP_ERR_CUDA;
    }
    if (st != CP_OK) return st;
    const Shape s = make_shape(d);
    const size_t RR = (size_t)s.R * s.R;
    double* S = scratch;
    double* Y = S + s.N * RR;
    double* Gam = Y + s.N * RR;
    cudaStream_t cs = (cudaStream_t)stream;
    Ptrs<const double> Ap{}, Wp{};
    Ptrs<double> Qp{};
    for (int n = 0; n < s.N; ++n) {
        Ap.p[n] = A[n];
        Wp.p[n] = W[n];
        Qp.p[n] = Q[n];
    }
    const int ns = (int)(s.N * RR);
    gram_direct_kernel<<<(ns + 255) / 256, 256, 0, cs>>>(s, Ap, S);
    gamma_direct_kernel<<<(int)((RR + 255) / 256), 256, 0, cs>>>(s, S, Gam);
    launch_matvec_f64(s, Ap, Gam, Wp, lambda, Qp, Y, cs);
    if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
    return CP_OK;
}
