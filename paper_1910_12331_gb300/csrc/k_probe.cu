// k_probe.cu -- two measurement probes that give the rooflines of the
// latency-bound and FP64-bound kernels their denominators:
//   cp_probe_grid_barrier: the round trip of the grid barrier the persistent
//     CG kernel uses (same code, same co-resident launch), per barrier;
//   cp_probe_fp64_fma: the FP64 fused multiply-add rate of the GPU (the
//     ceiling of the plain FP64 path, whose kernels are DFMA-bound).
#include "kernels.hpp"

namespace cpgn {
namespace {

// `iters` grid barriers back to back, nothing else between them.
__global__ void barrier_probe_kernel(GridBarrier* bar, int* status, int iters, long long limit) {
    for (int i = 0; i < iters; ++i)
        if (!grid_sync(bar, status, gridDim.x, limit)) return;
}

// Eight independent FMA chains per thread, `iters` steps each; the sum is
// stored so that the chains are not removed.
__global__ void fma_probe_kernel(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (double)(threadIdx.x + u) * 1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __fma_rn(x[u], a, b);
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == 12345.678) out[0] = s;  // never true for these inputs; keeps the chains live
}

struct Scratch {
    void* p = nullptr;
    ~Scratch() {
        if (p) cudaFree(p);
    }
};

}  // namespace
}  // namespace cpgn

using namespace cpgn;

extern "C" cp_status cp_probe_grid_barrier(int device, int blocks, int threads, int iters, double* us_per_barrier) {
    if (!us_per_barrier || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1)
        return CP_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_ARG;
    }
    cp_status rc = CP_OK;
    {
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_probe_kernel, threads, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        Scratch sc;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (blocks > per_sm * sms) {
            rc = CP_ERR_UNSUPPORTED;  // not co-resident: the barrier could never complete
        } else if (cudaMalloc(&sc.p, sizeof(GridBarrier) + 16) != cudaSuccess) {
            rc = CP_ERR_NOMEM;
        } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = CP_ERR_CUDA;
        } else {
            GridBarrier* bar = (GridBarrier*)sc.p;
            int* status = (int*)((char*)sc.p + sizeof(GridBarrier));
            long long limit = 1LL << 24;
            float ms[2] = {0.f, 0.f};
            const int counts[2] = {1, iters + 1};  // the difference removes the launch overhead
            for (int k = 0; k < 2 && rc == CP_OK; ++k) {
                cudaMemset(sc.p, 0, sizeof(GridBarrier) + 16);
                int it = counts[k];
                void* args[] = {(void*)&bar, (void*)&status, (void*)&it, (void*)&limit};
                cudaEventRecord(e0, 0);
                if (cudaLaunchCooperativeKernel((void*)barrier_probe_kernel, dim3(blocks), dim3(threads), args, 0, 0) !=
                    cudaSuccess)
                    rc = CP_ERR_CUDA;
                cudaEventRecord(e1, 0);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = CP_ERR_CUDA;
                cudaEventElapsedTime(&ms[k], e0, e1);
                int hs = 0;
                cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost);
                if (hs) rc = (cp_status)hs;
            }
            *us_per_barrier = (double)(ms[1] - ms[0]) * 1e3 / iters;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
    }
    cudaSetDevice(prev);
    return rc;
}

extern "C" cp_status cp_probe_fp64_fma(int device, double* tflops) {
    if (!tflops) return CP_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return CP_ERR_ARG;
    }
    cp_status rc = CP_OK;
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        Scratch sc;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaMalloc(&sc.p, 16) != cudaSuccess) {
            rc = CP_ERR_NOMEM;
        } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = CP_ERR_CUDA;
        } else {
            const int blocks = sms * 8, threads = 256, iters = 1 << 14;
            fma_probe_kernel<<<blocks, threads>>>((double*)sc.p, 256, 1.0000001, 1e-9);  // warm-up
            cudaEventRecord(e0, 0);
            fma_probe_kernel<<<blocks, threads>>>((double*)sc.p, iters, 1.0000001, 1e-9);
            cudaEventRecord(e1, 0);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = CP_ERR_CUDA;
            const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
            *tflops = rc == CP_OK && ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
    }
    cudaSetDevice(prev);
    return rc;
}
