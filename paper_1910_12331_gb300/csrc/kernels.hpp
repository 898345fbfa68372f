// kernels.hpp -- host-side launchers of the CP-GN kernels (one definition per .cu file).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace cpgn {

Shape make_shape(const cp_desc* d);

// ---- small dense kernels (k_dense.cu) ----------------------------------------
// Gram partial sums over row chunks: part[n][chunk][R][R]; returns chunk count per mode in *chunks.
int gram_chunks(const Shape& s);
void launch_gram_partial(const Shape& s, Ptrs<const double> A, double* part, int chunks, cudaStream_t st);
// S[n] = sum of partials; Gam[n][p] = prod_{m != n,p} S[m]; GamF = float copy (may be null).
void launch_gamma(const Shape& s, const double* part, int chunks, double* S, double* Gam, float* GamF,
                  cudaStream_t st);
// G^(n) = A^(n) Gam[n][n] - M^(n) (packed G, packed M); norms into stats.
// resid = true: M holds the MTTKRP of the residual tensor, G = -M and the
// reported |M^(n)| is that of A^(n) Gam[n][n] - G^(n).
// part: gradient_part_doubles(s) doubles of scratch (per-block partial norms).
void launch_gradient(const Shape& s, Ptrs<const double> A, const double* Gam, const double* M, double* G,
                     double* part, DevStats* stats, cudaStream_t st, bool resid);
size_t gradient_part_doubles(const Shape& s);
// Damping by lam diag(J^T J): Gamma^(n,n)_{rr} += lam Gamma^(n,n)_{rr} in Gam
// and GamF (may be null); the system is then solved with lam = 0.
void launch_damp_diag(const Shape& s, double* Gam, float* GamF, double lam, cudaStream_t st);
// Pinv[n] = (Gam[n][n] + lam I)^{-1} (FP64 Cholesky + inverse); PinvF float copy (may be null).
// scratch: precond_scratch_doubles(s) doubles, used only when precond_smem_bytes(R) == 0.
// fp32: the FP32 factorisation with clamped pivots (writes PinvF only).
void launch_precond(const Shape& s, const double* Gam, double lam, double* Pinv, float* PinvF, double* scratch,
                    DevStats* stats, cudaStream_t st, bool fp32 = false);
size_t precond_smem_bytes(int R);
size_t precond_scratch_doubles(const Shape& s);
// Packed copy of the factors in T.
template <typename T>
void launch_pack(const Shape& s, Ptrs<const double> A, T* Ap, cudaStream_t st);
// A^(n) += t V^(n) (V packed in T); ||t V^(n)||^2 and ||A^(n)||^2 into stats.
template <typename T>
void launch_update(const Shape& s, Ptrs<double> A, const T* V, DevStats* stats, cudaStream_t st, double t = 1.0);
// Armijo line search: trial factors At = A + t V (packed FP64), and <G, V>
// (packed, G FP64) summed in a fixed order into *out (part: 64 doubles).
template <typename T>
void launch_trial_factors(const Shape& s, Ptrs<const double> A, const T* V, double t, double* At, cudaStream_t st);
template <typename T>
void launch_dot_gv(int64_t len, const double* G, const T* V, double* part, double* out, cudaStream_t st);
// ALS mode update: A^(n) = M^(n) Pinv^(n) (M packed rows of mode n).
void launch_als_solve(const Shape& s, int n, const double* Mn, const double* Pinv_n, double* An, cudaStream_t st);
// Copy packed rows of mode n to a caller pointer set (FP64).
void launch_unpack(const Shape& s, const double* packed, Ptrs<double> out, cudaStream_t st);

// ---- FP64 SIMT MTTKRP (k_mttkrp_f64.cu) -----------------------------------------
// Accumulates (atomically) into M; M must be zeroed first.  mode_mask selects
// which modes are produced (bit n = mode n).
void launch_mttkrp_f64(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, Ptrs<double> M,
                       unsigned mode_mask, cudaStream_t st);

// ---- implicit matvec and persistent PCG (k_pcg.cu) --------------------------------
template <typename T>
struct PcgArgs {
    Shape s;
    const T* Ap;        // packed factors
    const T* GamT;      // N*N*R*R Gamma in T
    const T* PinvT;     // N*R*R preconditioner in T
    const double* G;    // packed FP64 gradient
    T* V;               // packed update (output)
    T* Zpart;           // [nblocks][R*R]: each block's A^T Z over its rows
    T* Yfull;           // [N][R*R]: Y^(p) = A^(p)T W^(p), reduced in a fixed order
    T* spill;           // large R: the matrices and row blocks in global memory (null: shared memory)
    int64_t spill_stride;  // elements of one block's region in `spill`
    double* part;       // [3][nblocks] per-block partial scalars
    GridBarrier* bar;
    DevStats* stats;
    double lam;
    double eps_cg;
    double stop_ratio;  // > 0: no CG iteration when sum||G|| <= stop_ratio sum||M||
    int maxit;
    long long spin_limit;
    int nblocks;
    // Row ownership: blocks never straddle modes.  Mode n owns blocks
    // [mode_blk0[n], mode_blk0[n+1]); its block j owns rows
    // [j * rpb[n], min(s_n, (j+1) * rpb[n])) of A^(n).
    int mode_blk0[kMaxN + 1];
    int rpb[kMaxN];
};
template <typename T>
cp_status launch_pcg(PcgArgs<T>& a, int max_blocks, cudaStream_t st);
// The CG kernel's geometry for a shape: its block count and the elements of T
// of global memory it needs when the R x R matrices do not fit in shared
// memory (0 otherwise).  Cached; launch_pcg uses the same geometry.
template <typename T>
cp_status pcg_plan(const Shape& s, int max_blocks, int* nblocks, size_t* spill_elems);
// Plain (non-persistent) matvec used by cp_gn_matvec: Q = (J^T J + lam D) W,
// D = I or (diag) diag(J^T J), in FP64 (T = double) or the mixed CG's FP32
// arithmetic (T = float).  Y: N R^2 elements of T scratch.
template <typename T>
void launch_matvec(const Shape& s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W, double lam,
                   bool diag, Ptrs<double> Q, T* Y, cudaStream_t st);
// The FP64 matvec with lam I.
void launch_matvec_f64(const Shape& s, Ptrs<const double> A, const double* Gam, Ptrs<const double> W, double lam,
                       Ptrs<double> Q, double* Y, cudaStream_t st);
// Loads the module of the plain matvec's kernels now (cudaFuncGetAttributes), not at their first launch.
cudaError_t preload_matvec_f64();

// ---- residual tensor E = X - [[A]] in extended precision (k_resid.cu): as
// bf16 planes in PlaneTiling layout (planes, may be null) and/or in FP64,
// C-contiguous like X (E64, may be null); sum E^2 and sum X^2 into stats.
// scratch: resid_scratch_bytes(s) bytes (double-float copy of the factors and
// block maxima of the first and last factor).
void launch_resid_split(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, void* planes,
                        double* E64, void* scratch, DevStats* stats, cudaStream_t st);
size_t resid_scratch_bytes(const Shape& s);
// The same residual tensor with the reconstruction on the tensor cores (R <= 64):
// error-free bf16 slice products; returns the number of kernels launched.
bool resid_tc_supported(const Shape& s);
size_t resid_tc_scratch_bytes(const Shape& s);
// reserve_sms: SMs left free for work running beside it on another stream.
int launch_resid_split_tc(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, void* planes,
                          double* E64, void* scratch, DevStats* stats, int* status, cudaStream_t st,
                          int reserve_sms = 0);

// ---- truncated HoSVD / Tucker compression (k_tucker.cu) -----------------------------
// FP64 scratch (doubles) of launch_hosvd with `slabs` contraction slabs for the Grams.
size_t hosvd_scratch_doubles(const Shape& s, const int* ranks, int slabs);
// U[n] (s_n x r_n, orthonormal columns spanning the dominant eigenspace of
// X_(n) X_(n)^T) and the core (prod r_n, C-contiguous); iters[n] (host, may be
// null) = orthogonal-iteration steps; hbuf: 4 pinned host doubles.
// Synchronises once per orthogonal-iteration step.
cp_status launch_hosvd(const Shape& s, cp_dtype xdt, const void* X, const int* ranks, double* const* U, double* core,
                       int* iters, double* scratch, int slabs, double* hbuf, cudaStream_t st);
// A (s x R) = U (s x r) B (r x R), row-major FP64.
void launch_tucker_expand(int64_t s, int r, int R, const double* U, const double* B, double* A, cudaStream_t st);

// ---- residual (k_residual.cu) ------------------------------------------------------
void launch_residual_f64(const Shape& s, cp_dtype xdt, const void* X, Ptrs<const double> A, DevStats* stats,
                         cudaStream_t st);

// ---- batched small problems (k_batched.cu) -----------------------------------------
cp_status run_batched(int device, cudaStream_t stream, int nprob, const cp_batch_problem* problems, double eps_cg,
                      int cg_max_iter, int max_iters, double target_residual, cp_batch_result* results);
struct BatchPlan;
cp_status batch_plan_create(int device, cudaStream_t stream, int nprob, const cp_batch_problem* problems,
                            double eps_cg, int cg_max_iter, int max_iters, double target_residual, int autotune,
                            BatchPlan** out);
cp_status batch_plan_launch(BatchPlan* pl, cudaStream_t stream);
cp_status batch_plan_results(BatchPlan* pl, cudaStream_t stream, cp_batch_result* results);
int batch_plan_threads(const BatchPlan* pl);
cp_status batch_plan_configure(BatchPlan* pl, int threads, int order);
int batch_plan_order(const BatchPlan* pl);
void batch_plan_destroy(BatchPlan* pl);

}  // namespace cpgn
