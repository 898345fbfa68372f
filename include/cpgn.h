/*
 * cpgn.h -- C ABI of the GB300 (sm_103a) Gauss-Newton CP decomposition library.
 *
 * Method: Singh, Ma, Yang, Solomonik, "Comparison of Accuracy and Scalability
 * of Gauss-Newton and Alternating Least Squares for CP Decomposition" (2019).
 * Section, equation and algorithm numbers below refer to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - X is a dense order-N tensor s_1 x ... x s_N, C-contiguous (mode N is the
 *    fastest index), element type cp_desc.x_dtype, in DEVICE memory.
 *  - Factor-like arguments (A, M, W, Q, G) are passed as a HOST array of N
 *    DEVICE pointers; pointer n addresses a row-major s_n x R matrix of
 *    doubles (R contiguous).
 *  - The caller owns every buffer it passes.  The library never frees or
 *    retains caller memory beyond the call.  The handle owns its device
 *    workspace (grown on demand with cudaMalloc, freed by cp_destroy) and a
 *    cache of split-precision copies of X keyed by (pointer, size, dtype,
 *    x_version).  The caller must change x_version whenever the bytes at that
 *    pointer change, including when a new tensor is allocated at the address
 *    of a freed one; otherwise a bf16x3 call reuses the old split.
 *  - Outputs must not alias inputs (CP_ERR_ARG).
 *  - All device work is enqueued on the handle's stream (cp_set_stream;
 *    default: the legacy default stream).  Calls that return host scalars or
 *    statistics synchronise that stream before returning, and say so.
 *  - Argument errors are returned before any work is enqueued.  Errors found
 *    on the device (non-SPD pivot, non-finite value, CG breakdown, barrier
 *    timeout) are returned by the synchronising call that observes them.
 *  - Supported: 2 <= N <= CP_MAX_ORDER, 1 <= R <= CP_MAX_RANK, every s_n >= 1.
 */
#ifndef CPGN_H
#define CPGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CP_MAX_ORDER 8
#define CP_MAX_RANK 1024

typedef enum {
    CP_OK = 0,
    CP_ERR_ARG = 1,          /* invalid argument (shape, pointer, aliasing, dtype) */
    CP_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    CP_ERR_NOMEM = 3,        /* workspace allocation failed */
    CP_ERR_UNSUPPORTED = 4,  /* valid, but not supported by the library on this code path */
    CP_ERR_NOT_SPD = 5,      /* Gamma^(n,n) + lambda I has a non-positive Cholesky pivot */
    CP_ERR_NONFINITE = 6,    /* a NaN/Inf appeared in a gradient or CG scalar */
    CP_ERR_BREAKDOWN = 7,    /* CG curvature <W, (J^T J + lambda I) W> <= 0 */
    CP_ERR_TIMEOUT = 8,      /* a device-side grid barrier exceeded its spin limit */
    CP_WARN_CG_MAXIT = 9     /* CG stopped at its iteration cap (result still applied) */
} cp_status;

typedef enum { CP_F32 = 0, CP_F64 = 1 } cp_dtype;

/* Arithmetic of the MTTKRP (and of the CG vectors in cp_gn_step):
 *  CP_PREC_FP64    FP64 everywhere (the plain path);
 *  CP_PREC_BF16X3  MTTKRP on tcgen05 tensor cores with each operand split into
 *                  bf16 high/low parts (hi*hi + hi*lo + lo*hi, FP32
 *                  accumulation); CG vectors and matvec in FP32.  Gram, Gamma
 *                  and the gradient stay FP64; the preconditioner inverse is
 *                  formed in double-float (relative error ~2^-44) and applied
 *                  in FP32; the CG dot products <R,Z> and <W,Q> are summed
 *                  error-free per thread and across each block as double-float
 *                  pairs of FP32 (relative error ~2^-44 of the sum of the
 *                  magnitudes of their terms), then across blocks and into
 *                  alpha and beta in FP64; the per-mode norms of R for the CG
 *                  stop test are FP32 sums (relative error ~2^-24 n, which
 *                  moves the stop by at most an iteration); the residual is
 *                  FP64. */
/*  CP_PREC_RESIDUAL (gradient only: cp_gradient, cp_gn_step, cp_gn_solve)
 *                  G^(n) = -E_(n) P^(n) with E = X - [[A]] the residual tensor
 *                  (Eq. (2.3) in residual form), split into bf16 planes and
 *                  contracted by the bf16x3 tensor-core MTTKRP;
 *                  M^(n) = A^(n) Gamma^(n,n) - G^(n).  E is reconstructed on
 *                  the tensor cores by error-free bf16 slice products for
 *                  R <= 64 (error below 2^-38.5 R sigma_i tau_k, sigma_i and
 *                  tau_k the powers of two above the row maxima of the two
 *                  product operands), else on the CUDA cores in extended FP32
 *                  arithmetic.  The same gradient as Algorithm 1's A Gamma - M,
 *                  but its error scales with |E| instead of |M|.  Used by the
 *                  mixed path (with cg_fp32 = 1) on every iteration, or after
 *                  the bf16x3 gradient stalls (cp_solve_opts.refine_below). */
typedef enum { CP_PREC_FP64 = 0, CP_PREC_BF16X3 = 1, CP_PREC_RESIDUAL = 2 } cp_precision;

typedef struct cp_handle_s* cp_handle;

typedef struct {
    int order;                     /* N */
    int rank;                      /* R */
    int64_t dims[CP_MAX_ORDER];    /* s_1 .. s_N */
    cp_dtype x_dtype;              /* element type of X */
    uint64_t x_version;            /* change whenever the bytes of X change, or a new tensor
                                      reuses X's address (split cache key) */
} cp_desc;

/* Damping of the Gauss-Newton system (Section 3.2).  CP_REG_IDENTITY solves
 * (J^T J + lam I) v = -g, the Levenberg-Marquardt form the paper uses with its
 * varying lam.  CP_REG_DIAG solves (J^T J + lam diag(J^T J)) v = -g, the
 * scale-invariant alternative the same section discusses: the diagonal of the
 * block (n,n) = Gamma^(n,n) (x) I of J^T J (Eq. (3.2)), so entry (i, r) of mode
 * n is damped by lam * Gamma^(n,n)_{rr}, in the matvec and in the
 * preconditioner (Gamma^(n,n) + lam diag(Gamma^(n,n)))^{-1}; lam is then
 * dimensionless. */
typedef enum { CP_REG_IDENTITY = 0, CP_REG_DIAG = 1 } cp_reg;

/* Parameters of one Gauss-Newton step (Algorithm 1) and its CG solve
 * (Algorithm 2).  lam / lam_dir are in/out: cp_gn_step uses lam for this
 * step and then advances it by the varying rule of Section 3.2. */
typedef struct {
    double eps_cg;        /* CG stop: sum_n ||R^(n)||_F <= eps_cg sum_n ||G^(n)||_F (paper: 1e-3) */
    int cg_max_iter;      /* CG iteration cap (>= 0) */
    double lam;           /* lambda of this step (in), of the next step (out) */
    double lam_lo;        /* lower threshold of the varying rule */
    double lam_hi;        /* upper threshold of the varying rule */
    double mu;            /* factor mu > 1 of the varying rule */
    int lam_dir;          /* 0: decreasing, 1: increasing (in/out) */
    int lam_fixed;        /* 1: keep lam constant (constant regularisation) */
    int reg;              /* cp_reg: damping lam I (0, default) or lam diag(J^T J) (1); other
                             values are CP_ERR_ARG */
    cp_precision prec;    /* MTTKRP arithmetic */
    int cg_fp32;          /* 1: CG vectors and the matvec in FP32 (dot products in double-float,
                             alpha and beta in FP64, the stop-test norms in FP32; see
                             CP_PREC_BF16X3); 0: FP64 */
    int want_residual;    /* 1: also return the direct FP64 relative residual after the update */
    double stop_stationarity; /* > 0: if sum||G||/sum||M|| <= this at the entry point, apply no
                                 update and report stats.stopped = 1 (Algorithm 1's loop test) */
    int64_t spin_limit;   /* grid-barrier spin limit in polls; 0 selects the default (~seconds) */
    /* Step-size control by Armijo's condition (Section 5, the matrix-multiplication
     * experiments): armijo_c > 0 takes the first t in 1, beta, beta^2, ..., beta^armijo_max
     * with f(A + t V) <= f(A) + armijo_c t <G, V> + 2 R 2^-53 ||X||^2 (the last term: the
     * accuracy of f = 1/2 ||X - [[A]]||_F^2 evaluated by the direct FP64 reconstruction, as
     * cp_residual), <G, V> summed in a fixed order; A += t V, or no update (t = 0) if no
     * trial meets it.  armijo_c = 0: the full step. */
    double armijo_c;      /* 0 <= c < 1 (paper: unspecified; 1e-4 is usual) */
    double armijo_beta;   /* 0 < beta < 1 when armijo_c > 0 */
    int armijo_max;       /* >= 0 reductions after the full step */
} cp_gn_params;

typedef struct {
    int status;              /* cp_status of the step */
    int cg_iters;            /* CG iterations performed */
    int stopped;             /* 1: the stationarity test held at entry; no update was applied */
    double grad_norm_sum;    /* sum_n ||G^(n)||_F at the entry point (FP64) */
    double m_norm_sum;       /* sum_n ||M^(n)||_F at the entry point */
    double update_norm_sum;  /* sum_n ||V^(n)||_F of the applied update */
    double factor_norm_sum;  /* sum_n ||A^(n)||_F after the update */
    double lam_used;         /* lambda used by this step */
    double cg_rnorm;         /* final sum_n ||R^(n)||_F of CG */
    double rel_residual;     /* ||X - [[A]]||_F / ||X||_F after the update, or -1 */
    double entry_residual;   /* residual at the entry point (CP_PREC_RESIDUAL steps), or -1 */
    double mttkrp_ms;        /* device time of the MTTKRP phase (CUDA events) */
    double pcg_ms;           /* device time of the CG kernel */
    double step_ms;          /* device time of the whole step */
    int kernel_launches;     /* kernels this step launched */
    int cg_blocks;           /* blocks of the persistent CG kernel's launch (0 if it did not run) */
    double step;             /* step length t applied (1 without the line search, 0: rejected) */
    double f_entry;          /* f = 1/2 ||X - [[A]]||_F^2 at the entry point (line search), or -1 */
    int ls_trials;           /* trial points the line search evaluated */
} cp_gn_stats;

/* Human-readable name of a status code (static storage; unknown codes give
 * "CP_UNKNOWN_STATUS").  Never fails. */
const char* cp_status_string(cp_status s);

/* Create a handle bound to CUDA device `device`.  Allocates nothing on the
 * device yet.  Errors: CP_ERR_ARG (null out-pointer, bad device), CP_ERR_CUDA. */
cp_status cp_create(cp_handle* out, int device);

/* Free the handle and all of its workspace.  Synchronises its stream. */
cp_status cp_destroy(cp_handle h);

/* Enqueue all later work of `h` on `stream` (a cudaStream_t of the handle's
 * device, owned by the caller; NULL = the legacy default stream).  Errors:
 * CP_ERR_ARG (null handle). */
cp_status cp_set_stream(cp_handle h, void* stream);

/* Bytes of handle-owned device workspace a call pattern on `desc` needs at
 * precision `prec`, an upper bound: the Gram/Gamma/gradient/CG buffers, for
 * CP_PREC_BF16X3 and CP_PREC_RESIDUAL also the tensor-core MTTKRP's partial
 * sums, and for CP_PREC_RESIDUAL the bf16 planes of E = X - [[A]] and the
 * reconstruction's scratch.  The split-X cache (CP_PREC_BF16X3 only) is
 * reported apart, by *split_bytes when non-null.  Errors: CP_ERR_ARG,
 * CP_ERR_CUDA (device query). */
cp_status cp_workspace_size(cp_handle h, const cp_desc* desc, cp_precision prec, size_t* bytes,
                            size_t* split_bytes);

/* All-mode MTTKRP, M^(n) = X_(n) P^(n) for n = 1..N, with P^(n) the Khatri-Rao
 * product of all factors but A^(n) (Section 2.2, Eq. (2.1); the
 * "main computational bottleneck").  Evaluated as a dimension tree in one
 * pass over X: for every index m of the middle modes 2..N-1, the two
 * first-level contractions Y_m = X(:,m,:) A^(N) and Z_m = X(:,m,:)^T A^(1)
 * are formed and folded into every M^(n).
 * A: host array of N device pointers (s_n x R doubles, read).
 * M: host array of N device pointers (s_n x R doubles, overwritten).
 * Asynchronous.  Errors: CP_ERR_ARG, CP_ERR_NOMEM, CP_ERR_CUDA. */
cp_status cp_mttkrp_all(cp_handle h, const cp_desc* desc, const void* X, const double* const* A,
                        double* const* M, cp_precision prec);

/* Gradient of f (Eq. (2.3)) through Algorithm 1's gradient line:
 * G^(n) = A^(n) Gamma^(n,n) - M^(n), with M from cp_mttkrp_all at `prec`;
 * at CP_PREC_RESIDUAL the same quantity in residual form, -E_(n) P^(n) with
 * E = X - [[A]].  G: host array of N device pointers (s_n x R doubles,
 * overwritten).  Also returns, in host memory, gnorm[n] = ||G^(n)||_F and
 * mnorm[n] = ||M^(n)||_F (either may be NULL).  Synchronises.  Errors:
 * CP_ERR_ARG (null or aliased pointers, bad descriptor or precision),
 * CP_ERR_NOMEM, CP_ERR_CUDA, CP_ERR_TIMEOUT (a bounded wait of a tensor-core
 * kernel expired). */
cp_status cp_gradient(cp_handle h, const cp_desc* desc, const void* X, const double* const* A,
                      double* const* G, cp_precision prec, double* gnorm, double* mnorm);

/* Implicit Gauss-Newton matvec of Algorithm 2 (Eq. (3.4)):
 * Q^(n) = lambda W^(n) + W^(n) Gamma^(n,n) + sum_{p != n} A^(n) (Gamma^(n,p) * Y^(p))^T,
 * Y^(p) = A^(p)^T W^(p), i.e. Q = (J^T J + lambda I) W with J the Jacobian of
 * Eq. (3.1); with reg = CP_REG_DIAG, Q = (J^T J + lambda diag(J^T J)) W
 * (Section 3.2's alternative damping; see cp_reg).
 * grams: NULL (the Gram matrices S^(n) = A^(n)^T A^(n) are formed from A
 * inside the call) or a DEVICE array of N row-major R x R FP64 matrices S^(n)
 * (read; Gamma^(n,p) is formed from them).
 * prec: CP_PREC_FP64 -- every product and sum in FP64; CP_PREC_BF16X3 or
 * CP_PREC_RESIDUAL -- the arithmetic of the mixed CG (cg_fp32 = 1): A, W and
 * Gamma rounded to FP32 once (Gamma formed in FP64), then Y, T^(n) and Q in
 * FP32 fused multiply-adds; Q is returned in FP64.
 * Asynchronous.  Errors: CP_ERR_ARG (null or aliased pointers, bad descriptor,
 * lambda < 0 or non-finite, unknown reg or prec), CP_ERR_NOMEM, CP_ERR_CUDA. */
cp_status cp_gn_matvec(cp_handle h, const cp_desc* desc, const double* const* A, const double* grams,
                       const double* const* W, double lambda, int reg, double* const* Q, cp_precision prec);

/* One CP-GN iteration (Algorithm 1 loop body): MTTKRP, Gram/Gamma, gradient,
 * preconditioner (Gamma^(n,n) + lambda D)^{-1} with D = I or diag(Gamma^(n,n))
 * by params->reg (Cholesky then explicit inverse, Section 3.3), CP-CG
 * (Algorithm 2, standard PCG beta) as one persistent device kernel, then
 * A^(n) += t V^(n) in place (t = 1, or chosen by Armijo's condition when
 * params->armijo_c > 0; the line search synchronises once per trial), then
 * lambda advances (unless lam_fixed).  A is
 * in/out.  Synchronises; fills *stats (host, may be NULL).  Returns the step's
 * status: CP_OK, CP_WARN_CG_MAXIT (update applied), or an error (A unchanged
 * for CP_ERR_NOT_SPD, CP_ERR_NONFINITE, CP_ERR_UNSUPPORTED; unspecified for
 * CP_ERR_BREAKDOWN, CP_ERR_TIMEOUT).
 * Ranks: the CG kernel keeps N + 2 R x R matrices (its mode's row of Gamma,
 * P_inv^(n), T^(n)) and its rows of the CG vectors in shared memory up to
 * R = 69 at N = 3 (R = 64 at N = 4) with FP64 CG vectors, R = 100 (91) with
 * FP32 ones (cg_fp32 = 1); above that it keeps them in global memory (L2),
 * one block per SM, up to CP_MAX_RANK.  The workspace then grows by about
 * N (N + 1) R^2 + nblocks (R^2 + 6 (rows per block) R) elements of the CG's
 * precision and nblocks R^2 for the partial products. */
cp_status cp_gn_step(cp_handle h, const cp_desc* desc, const void* X, double* const* A,
                     cp_gn_params* params, cp_gn_stats* stats);

/* Options of cp_gn_solve (a host loop over cp_gn_step). */
typedef struct {
    int max_iters;           /* GN iteration cap */
    double target_residual;  /* stop when the direct relative residual <= this (<= 0: unused) */
    double target_stationarity; /* stop when sum||G||/sum||M|| (FP64 gradient) <= this (<= 0: unused) */
    double refine_below;     /* BF16X3 only: switch the gradient to refine_prec once the
                                low-precision stationarity falls below this (<= 0: never) */
    cp_precision refine_prec; /* CP_PREC_FP64 (= 0) or CP_PREC_RESIDUAL (any other value) */
    int residual_every;      /* evaluate the residual every k iterations (0: only when targeted) */
} cp_solve_opts;

typedef struct {
    int status;
    int iters;               /* GN iterations performed */
    int iters_refined;       /* of which with the refined gradient */
    int cg_iters_total;
    int converged;           /* 1 if a target was met */
    double stationarity;     /* last sum||G||/sum||M|| */
    double rel_residual;     /* last residual evaluated, or -1 */
    double lam;              /* lambda after the last step */
    double mttkrp_ms;        /* summed device time of the MTTKRP phases */
    double pcg_ms;           /* summed device time of the CG kernels */
    double device_ms;        /* summed device time of all steps */
    long long kernel_launches; /* kernels launched by the solve */
    int cg_blocks;           /* blocks of the last persistent CG launch */
} cp_solve_result;

/* Run Algorithm 1 from the factors in A (in/out) until a target of `opts` is
 * met or max_iters steps have run.  params is in/out as in cp_gn_step; *result
 * (host) receives the counts, the last stationarity and residual, and summed
 * device times.  Synchronises once per GN iteration.  Returns CP_OK when the
 * loop ended without a step error, whether or not a target was met (see
 * result->converged; a step that hit the CG cap is not an error here), else
 * the failing step's status (as in cp_gn_step).  Argument errors: CP_ERR_ARG. */
cp_status cp_gn_solve(cp_handle h, const cp_desc* desc, const void* X, double* const* A,
                      cp_gn_params* params, const cp_solve_opts* opts, cp_solve_result* result);

/* One CP-ALS sweep (Section 2.2): for n = 1..N in order,
 * A^(n) <- M^(n) (Gamma^(n) + lambda I)^{-1} with M^(n) = X_(n) P^(n) formed
 * from the factors already updated in this sweep; the inverse is built from
 * the Cholesky factor.  lambda = 0 is plain ALS.  A is in/out.  prec:
 * CP_PREC_FP64 or CP_PREC_BF16X3 (the MTTKRP's arithmetic).  If rel_residual
 * is non-null, the direct FP64 residual after the sweep is written there
 * (synchronises); otherwise asynchronous.  Errors: CP_ERR_ARG, CP_ERR_NOMEM,
 * CP_ERR_CUDA, and, observed when synchronising, CP_ERR_NOT_SPD (a singular
 * Gamma^(n) + lambda I) or CP_ERR_TIMEOUT. */
cp_status cp_als_sweep(cp_handle h, const cp_desc* desc, const void* X, double* const* A, double lambda,
                       cp_precision prec, double* rel_residual);

/* Relative residual r = ||X - [[A]]||_F / ||X||_F (Section 5), with the
 * reconstruction formed element by element in FP64 and both squared sums
 * accumulated in FP64.  Writes the host scalar; synchronises.  Errors:
 * CP_ERR_ARG (null pointers, bad descriptor), CP_ERR_NOMEM, CP_ERR_CUDA. */
cp_status cp_residual(cp_handle h, const cp_desc* desc, const void* X, const double* const* A,
                      double* rel_residual);

/* The two FP64 sums behind cp_residual: *sq_err = ||X - [[A]]||_F^2 and
 * *sq_x = ||X||_F^2 (host scalars; either may be NULL).  sq_err is the CP
 * loss of Eq. (2.3) without its factor 1/2.  Synchronises.
 * Errors: CP_ERR_ARG, CP_ERR_NOMEM, CP_ERR_CUDA. */
cp_status cp_residual_sums(cp_handle h, const cp_desc* desc, const void* X, const double* const* A,
                           double* sq_err, double* sq_x);

/* The residual tensor E = X - [[A]] (the quantity whose squared norm is the
 * objective of Eq. (2.3) times 2, and whose MTTKRP is the residual form of the
 * gradient, G^(n) = -E_(n) P^(n)), element by element, written in FP64 to E:
 * a DEVICE buffer of prod_n s_n doubles, C-contiguous like X (caller-owned,
 * overwritten), or NULL for the two sums below alone.  E is formed by the reconstruction the residual-form gradient
 * uses: for R <= 64 on the tensor cores by error-free bf16 slice products
 * (error below 2^-38.5 R sigma tau per element, sigma and tau the powers of
 * two at or above max_r |a^(1)_ir w_m[r]| and max_r |a^(N)_kr|, w_m the
 * Hadamard product of the middle factors' rows), else on the CUDA cores in
 * extended FP32 arithmetic.  Also returns, in host memory, *sq_err = sum E^2
 * (of E rounded to FP32) and *sq_x = ||X||_F^2 (either may be NULL).
 * Synchronises.  Errors: CP_ERR_ARG (null X or A, E aliasing an input, bad
 * descriptor), CP_ERR_NOMEM, CP_ERR_CUDA, CP_ERR_TIMEOUT. */
cp_status cp_residual_tensor(cp_handle h, const cp_desc* desc, const void* X, const double* const* A, double* E,
                             double* sq_err, double* sq_x);

/* ---------------------------------------------------------------------------
 * Tucker compression ahead of CP for ranks below the sides (Section 1; the
 * complexity comparison of Section 3.5 assumes it).
 *
 * cp_hosvd: the truncated higher-order SVD of X with multilinear ranks
 * ranks[n] (1 <= ranks[n] <= s_n; desc->rank is not used but must be valid):
 * U[n] (host array of N DEVICE pointers, each s_n x ranks[n] row-major FP64,
 * overwritten) receives an orthonormal basis of the dominant ranks[n]-
 * dimensional eigenspace of X_(n) X_(n)^T (Gram matrix formed in FP64,
 * orthogonal iteration with Cholesky QR until ||S V - V V^T S V||_F <= 1e-12
 * ||S V||_F, at most 300 steps), and core (DEVICE, prod_n ranks[n] doubles,
 * C-contiguous, overwritten) the projection X x_1 U_1^T ... x_N U_N^T in FP64.
 * The basis is unique up to a rotation within the subspace (compare U U^T).
 * iters (host, N ints, may be NULL) receives the iteration counts.  CP of the
 * core with cp_gn_solve and cp_tucker_expand then give a CP model of X whose
 * squared error is the compression error plus the core's CP error.
 * Synchronises once per iteration step.  Errors: CP_ERR_ARG, CP_ERR_NOMEM,
 * CP_ERR_CUDA, CP_ERR_NOT_SPD (ranks[n] above the rank of X_(n)).
 *
 * cp_tucker_expand: A[n] = U[n] B[n] for n < order (U[n] dims[n] x ranks[n],
 * B[n] ranks[n] x R, A[n] dims[n] x R; host arrays of DEVICE pointers,
 * row-major FP64; A overwritten, not aliasing U or B).  Asynchronous.
 * Errors: CP_ERR_ARG, CP_ERR_CUDA. */
cp_status cp_hosvd(cp_handle h, const cp_desc* desc, const void* X, const int* ranks, double* const* U, double* core,
                   int* iters);
cp_status cp_tucker_expand(cp_handle h, int order, const int64_t* dims, const int* ranks, int R,
                           const double* const* U, const double* const* B, double* const* A);

/* ---------------------------------------------------------------------------
 * Many small independent order-3 problems (Algorithm 1 with Algorithm 2 per
 * problem) solved by one persistent kernel launch: each CTA takes problems
 * from a work counter and runs the whole Gauss-Newton iteration of one problem
 * in its shared memory (FP32 vectors, factors and Gram products; dot products
 * from per-thread FP32 partials summed error-free within each warp, then in
 * FP64 across the warps; FP64 CG scalars, preconditioner elimination and
 * factor master copy).
 * A problem stops when its direct relative residual ||X - [[A]]|| / ||X|| <=
 * target_residual (converged = 1), after max_iters GN iterations, or on an
 * error (its status).  lambda follows the varying rule of Section 3.2 from
 * lam (first iteration) with the problem's thresholds and mu. */
#define CP_BATCH_MAX_SIDE 256
#define CP_BATCH_MAX_RANK 32

typedef struct {
    int64_t dims[3];       /* s_1, s_2, s_3 (1 .. CP_BATCH_MAX_SIDE) */
    int rank;              /* R (1 .. CP_BATCH_MAX_RANK) */
    const float* X;        /* device, FP32, C-contiguous s_1 x s_2 x s_3 (caller-owned) */
    double* A[3];          /* device, FP64 row-major s_n x R, in/out (caller-owned) */
    double lam, lam_lo, lam_hi, mu;  /* regularisation of Section 3.2 */
    int reg;               /* cp_reg: damping lam I (0) or lam diag(J^T J) (1) */
    int lam_fixed;         /* 1: lambda stays lam (constant regularisation) */
    double armijo_c;       /* > 0: step-size control by Armijo's condition (as cp_gn_params, with
                              f the residual of the stop test, relaxed by its FP32 accuracy
                              2 R 2^-24 ||X||^2, and <G, V> from the CG recurrences); 0: full steps */
    double armijo_beta;    /* step reduction factor, 0 < beta < 1 when armijo_c > 0 */
    int armijo_max;        /* reductions after the full step (>= 0) */
} cp_batch_problem;

typedef struct {
    int status;            /* cp_status of this problem (CP_OK, CP_ERR_NOT_SPD, CP_ERR_NONFINITE) */
    int iters;             /* GN iterations performed */
    int cg_iters_total;
    int converged;         /* 1 if the residual target was met */
    int cg_breakdowns;     /* CG solves ended early because the FP32 curvature <W, Q W> was not
                              positive (the update found so far is applied) */
    double rel_residual;   /* last residual evaluated (FP32 reconstruction, compensated FP32
                              partials, FP64 block sum) */
    double lam;            /* lambda of the last iteration */
    int ls_backtracks;     /* step reductions the line search took in all */
} cp_batch_result;

/* Many small order-3 problems, each by Algorithm 1 with CP-CG (Algorithm 2)
 * and the varying lambda of Section 3.2, in one persistent launch (a CTA per
 * problem at a time).  problems and results are host arrays of nprob entries.  The shared memory a
 * problem needs, 8 (R^2 + R + 96) + 4 (6 (s_1 + s_2 + s_3) R + 21 R^2) bytes,
 * must not exceed 220 KB (CP_ERR_UNSUPPORTED).  Synchronises.
 * Errors: CP_ERR_ARG (null pointers, sizes out of range, mu <= 1, lam < 0,
 * lam_hi < lam_lo, unknown reg, armijo_c outside [0, 1), armijo_beta outside
 * (0, 1) or armijo_max < 0 with armijo_c > 0), CP_ERR_UNSUPPORTED,
 * CP_ERR_NOMEM, CP_ERR_CUDA; per-problem
 * device errors go to results[i].status. */
cp_status cp_gn_solve_batched(cp_handle h, int nprob, const cp_batch_problem* problems, double eps_cg,
                              int cg_max_iter, int max_iters, double target_residual, cp_batch_result* results);

/* The same batched solve as a reusable plan: cp_batch_plan_create checks the
 * problems (same rules and errors as cp_gn_solve_batched), copies their
 * descriptors to the device, allocates the results and, if `autotune` is
 * nonzero, times the kernel's block sizes (128, 256 and 384 threads), each with
 * the problems taken in the given order and largest work first (s_1 s_2 s_3 R,
 * the persistent CTAs' longest-processing-time order), on a device copy of the
 * factors of at most 64 of the problems -- the caller's factors are not
 * modified -- and keeps the fastest (otherwise 256 threads, given order).
 * Synchronises.  The plan keeps the device pointers of the problems: X and A
 * must stay allocated while the plan is used.
 *
 * cp_batch_plan_launch enqueues one solve of every problem from its current
 * factors (A in/out, as cp_gn_solve_batched) on the handle's stream: a reset of
 * the plan's work counter and one kernel launch, with no allocation and no
 * synchronisation, so it may be captured into a CUDA graph and replayed.
 * Launches of one plan must not overlap on the GPU (they share the counter
 * and the results).  cp_batch_plan_results copies the results of the last
 * completed launch to `results` (host, nprob entries); synchronises.
 * cp_batch_plan_threads returns the block size in use, cp_batch_plan_order the
 * problem order (0: as given, 1: largest work first).  cp_batch_plan_configure
 * sets both instead of the autotuner's or the default choice (threads 128, 256
 * or 384, order 0 or 1; CP_ERR_ARG otherwise, CP_ERR_UNSUPPORTED if the block
 * size cannot run with the plan's shared memory); it enqueues nothing and
 * applies to later launches.  cp_batch_plan_destroy
 * frees the plan's device memory (after its launches have finished; the
 * caller's current device is kept) and the plan.  Errors: CP_ERR_ARG,
 * CP_ERR_UNSUPPORTED, CP_ERR_NOMEM, CP_ERR_CUDA. */
typedef struct cp_batch_plan_s* cp_batch_plan;
cp_status cp_batch_plan_create(cp_handle h, int nprob, const cp_batch_problem* problems, double eps_cg,
                               int cg_max_iter, int max_iters, double target_residual, int autotune,
                               cp_batch_plan* plan);
cp_status cp_batch_plan_launch(cp_handle h, cp_batch_plan plan);
cp_status cp_batch_plan_results(cp_handle h, cp_batch_plan plan, cp_batch_result* results);
cp_status cp_batch_plan_threads(cp_batch_plan plan, int* threads);
cp_status cp_batch_plan_order(cp_batch_plan plan, int* order);
cp_status cp_batch_plan_configure(cp_batch_plan plan, int threads, int order);
cp_status cp_batch_plan_destroy(cp_batch_plan plan);

/* ---------------------------------------------------------------------------
 * Measurement probes: the denominators of the rooflines of the kernels that
 * are bound by neither HBM nor the tensor cores.
 *
 * cp_probe_grid_barrier times `iters` back-to-back grid barriers of the kind
 * the persistent CG kernel (Algorithm 2) takes three of per iteration: the
 * same barrier code, `blocks` co-resident blocks of `threads` threads launched
 * cooperatively on `device`, nothing else between the barriers.  Writes the
 * device time per barrier in microseconds (launch overhead removed by
 * differencing against a one-barrier launch).  Synchronises.  Errors:
 * CP_ERR_ARG, CP_ERR_UNSUPPORTED (the blocks cannot be co-resident),
 * CP_ERR_NOMEM, CP_ERR_CUDA, CP_ERR_TIMEOUT (a barrier's bounded wait expired).
 *
 * cp_probe_fp64_fma measures the FP64 fused multiply-add rate of `device`
 * (eight independent chains per thread, eight blocks of 256 threads per SM),
 * in TFLOP/s counting two flops per FMA: the ceiling of the plain FP64 path,
 * whose MTTKRP and CG kernels are FP64-ALU-bound.  Synchronises.  Errors:
 * CP_ERR_ARG, CP_ERR_NOMEM, CP_ERR_CUDA.
 * Both work on the legacy default stream and restore the caller's device. */
cp_status cp_probe_grid_barrier(int device, int blocks, int threads, int iters, double* us_per_barrier);
cp_status cp_probe_fp64_fma(int device, double* tflops);

/* ---------------------------------------------------------------------------
 * Matvec without device allocation.  The paper has no counterpart: this call
 * serves callers that cannot call cudaMalloc -- code running under a fixed,
 * pre-reserved device-memory budget, inside an allocator or memory-pool
 * callback, or in a serving loop that must not allocate after start-up.
 *
 * Same result as cp_gn_matvec, Q = (J^T J + lambda I) W (FP64), but with no
 * handle: the work is enqueued on `stream` (a cudaStream_t; NULL = default)
 * of the CURRENT device, and its scratch (Gram matrices, Gamma set, A^T W)
 * lives in one file-scope device array of CP_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  The call allocates
 * nothing and calls no allocating routine; the caller passes inputs and
 * outputs (host arrays of N device pointers, s_n x R doubles each).
 * The first call on a device (and the first after its CUDA context was
 * destroyed and created again, e.g. by cudaDeviceReset) looks up the array's
 * device address in the current context and loads the modules of the kernels
 * the call launches, which commits their device memory (the array included):
 * make that first call before any region in which nothing may be allocated,
 * and before any stream capture.
 * All calls share the array: calls that overlap on the GPU race, so the
 * caller must serialise them.  Each call rewrites all scratch it reads.
 * Errors: CP_ERR_ARG (null/aliased pointers, bad shape, lambda < 0),
 * CP_ERR_UNSUPPORTED (order > CP_NOALLOC_MAX_ORDER or rank >
 * CP_NOALLOC_MAX_RANK: the problem does not fit the static scratch),
 * CP_ERR_CUDA.  Asynchronous. */
#define CP_NOALLOC_MAX_ORDER 4
#define CP_NOALLOC_MAX_RANK 64
#define CP_NOALLOC_SCRATCH_BYTES ((2 * CP_NOALLOC_MAX_ORDER + CP_NOALLOC_MAX_ORDER * CP_NOALLOC_MAX_ORDER) * \
                                  CP_NOALLOC_MAX_RANK * CP_NOALLOC_MAX_RANK * 8)
cp_status cp_gn_matvec_noalloc(const cp_desc* desc, const double* const* A, const double* const* W, double lambda,
                               double* const* Q, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CPGN_H */
