/*
 * cpgn_oracle.c -- plain FP64 CPU oracle for Gauss-Newton CP decomposition
 * (Singh, Ma, Yang, Solomonik, "Comparison of Accuracy and Scalability of
 * Gauss-Newton and Alternating Least Squares for CP Decomposition", 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: it shares no code, header, table or helper with it.  Only tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  The
 * product path never calls it and never falls back to it.
 *
 * Everything is IEEE double, plain loops, no BLAS, OpenMP only over
 * independent outer indices.  Each routine cites the passage it restates.
 *
 * Layout conventions (shared with the caller through the Python wrapper):
 *   X       dense order-N tensor, C-contiguous, mode N (last) fastest.
 *   factors "packed": A^(1), ..., A^(N) stored one after the other, each
 *           row-major s_n x R.  The same packing is used for M, G, V, W, Q.
 *   S       N Gram matrices, each R x R.
 *   Gam     N*N matrices Gamma^(n,p), each R x R, at index (n*N+p).
 *
 * Parity status of each routine is recorded in its comment ("pinned by ...");
 * the pins live in the CPU test-suite.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 8

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOT_SPD = 5, ORC_ERR_BREAKDOWN = 7, ORC_WARN_CG_MAXIT = 9 };
/* damping of the CG system (Section 3.2) */
enum { ORC_REG_IDENTITY = 0, ORC_REG_DIAG = 1 };

typedef struct {
    int N;                   /* tensor order */
    int R;                   /* CP rank */
    int64_t dims[ORC_MAXN];  /* s_1 .. s_N */
} orc_desc;

/* ------------------------------------------------------------------ helpers */

static int64_t tensor_size(const orc_desc* d) {
    int64_t t = 1;
    for (int n = 0; n < d->N; ++n) t *= d->dims[n];
    return t;
}

static int64_t factor_offset(const orc_desc* d, int n) {
    int64_t off = 0;
    for (int m = 0; m < n; ++m) off += d->dims[m] * d->R;
    return off;
}

static int64_t factor_total(const orc_desc* d) { return factor_offset(d, d->N); }

/* split a linear C-order index into a multi-index */
static void unravel(const orc_desc* d, int64_t e, int64_t* idx) {
    for (int n = d->N - 1; n >= 0; --n) {
        idx[n] = e % d->dims[n];
        e /= d->dims[n];
    }
}

/* ------------------------------------------------------------- Gram, Gamma */

/* S^(n) = A^(n)^T A^(n)  (Section 2.2, the matrices S^(i) under Eq. (2.2)). */
void orc_gram(const orc_desc* d, const double* A, double* S) {
    const int R = d->R;
    for (int n = 0; n < d->N; ++n) {
        const double* An = A + factor_offset(d, n);
        double* Sn = S + (int64_t)n * R * R;
        for (int r = 0; r < R; ++r)
            for (int z = 0; z < R; ++z) {
                double acc = 0.0;
                for (int64_t i = 0; i < d->dims[n]; ++i) acc += An[i * R + r] * An[i * R + z];
                Sn[r * R + z] = acc;
            }
    }
}

/* Gamma^(n,p)_{rz} = prod_{m != n,p} S^(m)_{rz}  (Eq. (3.3)); with n = p this
 * is Gamma^(n) of Eq. (2.2).  An empty product is 1. */
void orc_gamma(const orc_desc* d, const double* S, double* Gam) {
    const int N = d->N, R = d->R;
    for (int n = 0; n < N; ++n)
        for (int p = 0; p < N; ++p) {
            double* Gnp = Gam + ((int64_t)n * N + p) * R * R;
            for (int q = 0; q < R * R; ++q) {
                double prod = 1.0;
                for (int m = 0; m < N; ++m)
                    if (m != n && m != p) prod *= S[(int64_t)m * R * R + q];
                Gnp[q] = prod;
            }
        }
}

/* ------------------------------------------------------------------ MTTKRP */

/* M^(n) = X_(n) P^(n) by its definition (Section 2.2, Eq. (2.1) for P^(n)):
 *   M^(n)_{i_n r} = sum over all other indices of x_{i_1..i_N} prod_{m!=n} a^(m)_{i_m r}.
 * Brute force over every tensor element; parallel over the output row i_n. */
void orc_mttkrp_def(const orc_desc* d, const double* X, const double* A, double* M) {
    const int N = d->N, R = d->R;
    const int64_t total = tensor_size(d);
    for (int n = 0; n < N; ++n) {
        const int64_t sn = d->dims[n];
        double* Mn = M + factor_offset(d, n);
        const int64_t sub = total / sn;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t in = 0; in < sn; ++in) {
            int64_t idx[ORC_MAXN];
            for (int r = 0; r < R; ++r) Mn[in * R + r] = 0.0;
            for (int64_t t = 0; t < sub; ++t) {
                /* t enumerates the other indices in C order; rebuild the full index */
                int64_t rem = t;
                for (int m = N - 1; m >= 0; --m) {
                    if (m == n) { idx[m] = in; continue; }
                    idx[m] = rem % d->dims[m];
                    rem /= d->dims[m];
                }
                int64_t e = 0;
                for (int m = 0; m < N; ++m) e = e * d->dims[m] + idx[m];
                const double x = X[e];
                for (int r = 0; r < R; ++r) {
                    double prod = 1.0;
                    for (int m = 0; m < N; ++m)
                        if (m != n) prod *= A[factor_offset(d, m) + idx[m] * R + r];
                    Mn[in * R + r] += x * prod;
                }
            }
        }
    }
}

/* One row M^(n)_{i, :} by the same definition; used to sample outputs of
 * large problems one by one. */
void orc_mttkrp_row(const orc_desc* d, const double* X, const double* A, int n, int64_t i, double* out) {
    const int N = d->N, R = d->R;
    const int64_t sub = tensor_size(d) / d->dims[n];
    for (int r = 0; r < R; ++r) out[r] = 0.0;
    int64_t idx[ORC_MAXN];
    for (int64_t t = 0; t < sub; ++t) {
        int64_t rem = t;
        for (int m = N - 1; m >= 0; --m) {
            if (m == n) { idx[m] = i; continue; }
            idx[m] = rem % d->dims[m];
            rem /= d->dims[m];
        }
        int64_t e = 0;
        for (int m = 0; m < N; ++m) e = e * d->dims[m] + idx[m];
        const double x = X[e];
        for (int r = 0; r < R; ++r) {
            double prod = 1.0;
            for (int m = 0; m < N; ++m)
                if (m != n) prod *= A[factor_offset(d, m) + idx[m] * R + r];
            out[r] += x * prod;
        }
    }
}

/* All-mode MTTKRP with a two-level dimension tree (Section 2.2, last
 * paragraph): the modes are split into a left group {1..h} and a right group
 * {h+1..N}, h = floor(N/2) (h = 1 for N = 2, 3).  Two bottleneck contractions
 * of X -- with the Khatri-Rao product of the right factors and with that of the
 * left factors -- give the intermediates T_L (prod_left x R) and T_R
 * (prod_right x R); every M^(n) then follows from a cheap contraction of one
 * intermediate with the remaining factors of its own group.
 * Work: 4 prod(s) R for the two bottleneck contractions. */
void orc_mttkrp_dt(const orc_desc* d, const double* X, const double* A, double* M) {
    const int N = d->N, R = d->R;
    int h = N / 2;
    if (h < 1) h = 1;
    int64_t PL = 1, PR = 1;
    for (int m = 0; m < h; ++m) PL *= d->dims[m];
    for (int m = h; m < N; ++m) PR *= d->dims[m];

    double* KL = (double*)malloc(sizeof(double) * PL * R); /* KRP of left factors  */
    double* KR = (double*)malloc(sizeof(double) * PR * R); /* KRP of right factors */
    double* TL = (double*)calloc((size_t)(PL * R), sizeof(double));
    double* TR = (double*)calloc((size_t)(PR * R), sizeof(double));

    /* Khatri-Rao rows: KL[p, r] = prod_{m<h} a^(m)_{i_m(p) r}, C order over the group */
#pragma omp parallel for
    for (int64_t p = 0; p < PL; ++p) {
        int64_t rem = p, idx[ORC_MAXN];
        for (int m = h - 1; m >= 0; --m) { idx[m] = rem % d->dims[m]; rem /= d->dims[m]; }
        for (int r = 0; r < R; ++r) {
            double prod = 1.0;
            for (int m = 0; m < h; ++m) prod *= A[factor_offset(d, m) + idx[m] * R + r];
            KL[p * R + r] = prod;
        }
    }
#pragma omp parallel for
    for (int64_t q = 0; q < PR; ++q) {
        int64_t rem = q, idx[ORC_MAXN];
        for (int m = N - 1; m >= h; --m) { idx[m] = rem % d->dims[m]; rem /= d->dims[m]; }
        for (int r = 0; r < R; ++r) {
            double prod = 1.0;
            for (int m = h; m < N; ++m) prod *= A[factor_offset(d, m) + idx[m] * R + r];
            KR[q * R + r] = prod;
        }
    }

    /* first bottleneck contraction: T_L[p, r] = sum_q X[p, q] KR[q, r] */
#pragma omp parallel for
    for (int64_t p = 0; p < PL; ++p)
        for (int64_t q = 0; q < PR; ++q) {
            const double x = X[p * PR + q];
            for (int r = 0; r < R; ++r) TL[p * R + r] += x * KR[q * R + r];
        }
    /* second bottleneck contraction: T_R[q, r] = sum_p X[p, q] KL[p, r],
     * parallel over blocks of q so that no two threads share an output row */
    const int64_t QB = 256;
#pragma omp parallel for
    for (int64_t q0 = 0; q0 < PR; q0 += QB) {
        const int64_t q1 = (q0 + QB < PR) ? q0 + QB : PR;
        for (int64_t p = 0; p < PL; ++p)
            for (int64_t q = q0; q < q1; ++q) {
                const double x = X[p * PR + q];
                for (int r = 0; r < R; ++r) TR[q * R + r] += x * KL[p * R + r];
            }
    }

    /* leaves: M^(n) for n in the left group from T_L, right group from T_R:
     * M^(n)_{i_n r} = sum over the other indices of the group of
     * T[p(idx), r] prod_{m in group, m != n} a^(m)_{i_m r} */
    for (int n = 0; n < N; ++n) {
        const int left = n < h;
        const int g0 = left ? 0 : h, g1 = left ? h : N;
        const double* T = left ? TL : TR;
        double* Mn = M + factor_offset(d, n);
        const int64_t sn = d->dims[n];
        int64_t sub = 1;
        for (int m = g0; m < g1; ++m) if (m != n) sub *= d->dims[m];
#pragma omp parallel for
        for (int64_t in = 0; in < sn; ++in) {
            int64_t idx[ORC_MAXN];
            for (int r = 0; r < R; ++r) Mn[in * R + r] = 0.0;
            for (int64_t t = 0; t < sub; ++t) {
                int64_t rem = t;
                for (int m = g1 - 1; m >= g0; --m) {
                    if (m == n) { idx[m] = in; continue; }
                    idx[m] = rem % d->dims[m];
                    rem /= d->dims[m];
                }
                int64_t p = 0;
                for (int m = g0; m < g1; ++m) p = p * d->dims[m] + idx[m];
                for (int r = 0; r < R; ++r) {
                    double prod = 1.0;
                    for (int m = g0; m < g1; ++m)
                        if (m != n) prod *= A[factor_offset(d, m) + idx[m] * R + r];
                    Mn[in * R + r] += T[p * R + r] * prod;
                }
            }
        }
    }
    free(KL); free(KR); free(TL); free(TR);
}

/* ---------------------------------------------------------------- gradient */

/* G^(n) = A^(n) Gamma^(n,n) - M^(n)  (Algorithm 1, gradient line);
 * gnorm[n] = ||G^(n)||_F.  Gradient of f in Eq. (2.3). */
void orc_gradient(const orc_desc* d, const double* A, const double* Gam, const double* M,
                  double* G, double* gnorm) {
    const int N = d->N, R = d->R;
    for (int n = 0; n < N; ++n) {
        const double* An = A + factor_offset(d, n);
        const double* Mn = M + factor_offset(d, n);
        const double* Gnn = Gam + ((int64_t)n * N + n) * R * R;
        double* Gn = G + factor_offset(d, n);
        double ss = 0.0;
        for (int64_t i = 0; i < d->dims[n]; ++i)
            for (int r = 0; r < R; ++r) {
                double acc = 0.0;
                for (int z = 0; z < R; ++z) acc += An[i * R + z] * Gnn[z * R + r];
                const double g = acc - Mn[i * R + r];
                Gn[i * R + r] = g;
                ss += g * g;
            }
        gnorm[n] = sqrt(ss);
    }
}

/* ----------------------------------------------------------- preconditioner */

/* Damping of the normal equations (Section 3.2).  reg = ORC_REG_IDENTITY:
 * J^T J + lam I.  reg = ORC_REG_DIAG: J^T J + lam diag(J^T J); the diagonal
 * of the block (n,n) = Gamma^(n,n) (x) I of Eq. (3.2) holds Gamma^(n,n)_{rr}
 * at every row of column r, so the damping of entry (i, r) of mode n is
 * lam * Gamma^(n,n)_{rr}. */
static double damping(int reg, const double* Gnn, int R, int r) {
    return reg == ORC_REG_DIAG ? Gnn[r * R + r] : 1.0;
}

/* P_inv = (Gamma^(n,n) + lam D)^{-1}  (Algorithm 2, first loop; Section 3.3),
 * D = I or diag(Gamma^(n,n)) by reg: Cholesky factorisation B = L L^T, then
 * the explicit inverse by forward and back substitution against the identity.
 * Returns ORC_ERR_NOT_SPD on a non-positive pivot. */
int orc_precond_inv(int R, const double* Gnn, double lam, int reg, double* Pinv) {
    double* L = (double*)calloc((size_t)R * R, sizeof(double));
    double* Y = (double*)calloc((size_t)R * R, sizeof(double));
    for (int j = 0; j < R; ++j) {
        double diag = Gnn[j * R + j] + lam * damping(reg, Gnn, R, j);
        for (int k = 0; k < j; ++k) diag -= L[j * R + k] * L[j * R + k];
        if (!(diag > 0.0)) { free(L); free(Y); return ORC_ERR_NOT_SPD; }
        const double ljj = sqrt(diag);
        L[j * R + j] = ljj;
        for (int i = j + 1; i < R; ++i) {
            double v = Gnn[i * R + j];
            for (int k = 0; k < j; ++k) v -= L[i * R + k] * L[j * R + k];
            L[i * R + j] = v / ljj;
        }
    }
    /* columns e_c: solve L y = e_c, then L^T x = y */
    for (int c = 0; c < R; ++c) {
        for (int i = 0; i < R; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[i * R + k] * Y[k * R + c];
            Y[i * R + c] = v / L[i * R + i];
        }
        for (int i = R - 1; i >= 0; --i) {
            double v = Y[i * R + c];
            for (int k = i + 1; k < R; ++k) v -= L[k * R + i] * Pinv[k * R + c];
            Pinv[i * R + c] = v / L[i * R + i];
        }
    }
    free(L); free(Y);
    return ORC_OK;
}

/* ------------------------------------------------------------------ matvec */

/* Q^(n) = lam D W^(n) + sum_p MatVec(A^(n), A^(p), Gamma^(n,p), W^(p))
 * (Algorithm 2, matvec line; Eq. (3.4)), D the damping chosen by reg
 * (entry (k, r) of the damping term: lam * damping(reg, Gamma^(n,n), R, r) * w^(n)_{kr}):
 *   p = n : sum_z Gamma^(n,n)_{rz} w^(n)_{kz}
 *   p != n: sum_{l,z} a^(n)_{kz} a^(p)_{lr} Gamma^(n,p)_{rz} w^(p)_{lz}
 * The off-diagonal 4-index sum is evaluated in the order that gives the
 * O(N^2 s R^2) cost the paper states after Eq. (3.4): first
 * Y^(p)_{rz} = sum_l a^(p)_{lr} w^(p)_{lz}, then sum_z a^(n)_{kz} Gamma^(n,p)_{rz} Y^(p)_{rz}. */
void orc_matvec(const orc_desc* d, const double* A, const double* Gam, const double* W, double lam, int reg,
                double* Q) {
    const int N = d->N, R = d->R;
    double* Y = (double*)malloc(sizeof(double) * (size_t)N * R * R);
    for (int p = 0; p < N; ++p) {
        const double* Ap = A + factor_offset(d, p);
        const double* Wp = W + factor_offset(d, p);
        for (int r = 0; r < R; ++r)
            for (int z = 0; z < R; ++z) {
                double acc = 0.0;
                for (int64_t l = 0; l < d->dims[p]; ++l) acc += Ap[l * R + r] * Wp[l * R + z];
                Y[(int64_t)p * R * R + r * R + z] = acc;
            }
    }
    for (int n = 0; n < N; ++n) {
        const double* An = A + factor_offset(d, n);
        const double* Wn = W + factor_offset(d, n);
        double* Qn = Q + factor_offset(d, n);
        const double* Gnn = Gam + ((int64_t)n * N + n) * R * R;
        for (int64_t k = 0; k < d->dims[n]; ++k)
            for (int r = 0; r < R; ++r) {
                double acc = lam * damping(reg, Gnn, R, r) * Wn[k * R + r];
                for (int p = 0; p < N; ++p) {
                    const double* Gnp = Gam + ((int64_t)n * N + p) * R * R;
                    if (p == n) {
                        for (int z = 0; z < R; ++z) acc += Gnp[r * R + z] * Wn[k * R + z];
                    } else {
                        const double* Yp = Y + (int64_t)p * R * R;
                        for (int z = 0; z < R; ++z) acc += An[k * R + z] * Gnp[r * R + z] * Yp[r * R + z];
                    }
                }
                Qn[k * R + r] = acc;
            }
    }
    free(Y);
}

/* --------------------------------------------------------------------- PCG */

static double dot_all(int64_t len, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

static double fro_sum(const orc_desc* d, const double* U) {
    double s = 0.0;
    for (int n = 0; n < d->N; ++n) {
        const double* Un = U + factor_offset(d, n);
        double ss = 0.0;
        for (int64_t i = 0; i < d->dims[n] * d->R; ++i) ss += Un[i] * Un[i];
        s += sqrt(ss);
    }
    return s;
}

/* Z^(n) = R^(n) P_inv^(n) for every mode */
static void apply_precond(const orc_desc* d, const double* Pinv, const double* Rv, double* Z) {
    const int N = d->N, R = d->R;
    for (int n = 0; n < N; ++n) {
        const double* Pn = Pinv + (int64_t)n * R * R;
        const double* Rn = Rv + factor_offset(d, n);
        double* Zn = Z + factor_offset(d, n);
        for (int64_t i = 0; i < d->dims[n]; ++i)
            for (int r = 0; r < R; ++r) {
                double acc = 0.0;
                for (int z = 0; z < R; ++z) acc += Rn[i * R + z] * Pn[z * R + r];
                Zn[i * R + r] = acc;
            }
    }
}

/* CP-CG, Algorithm 2: block-Jacobi (Kronecker) preconditioned CG on
 * (J^T J + lam D) V = -G, D = I or diag(J^T J) by reg.
 * beta_kind = 0: standard PCG, beta = <R,Z>_new / <R,Z>_old.
 * beta_kind = 1: the ratio as printed in Algorithm 2, <R,Z>_new / <W,Q>.
 * Stop test at the loop head: sum_n ||R^(n)||_F <= eps_cg sum_n ||G^(n)||_F, or
 * maxit iterations.  Returns ORC_OK, ORC_WARN_CG_MAXIT, ORC_ERR_NOT_SPD or
 * ORC_ERR_BREAKDOWN (<W,Q> <= 0). */
int orc_pcg(const orc_desc* d, const double* A, const double* Gam, const double* G, double lam, int reg,
            double eps_cg, int maxit, int beta_kind, double* V, int* iters_out, double* rnorm_out) {
    const int N = d->N, R = d->R;
    const int64_t len = factor_total(d);
    double* Pinv = (double*)malloc(sizeof(double) * (size_t)N * R * R);
    double* Rv = (double*)malloc(sizeof(double) * len);
    double* Z = (double*)malloc(sizeof(double) * len);
    double* W = (double*)malloc(sizeof(double) * len);
    double* Q = (double*)malloc(sizeof(double) * len);
    int status = ORC_OK;
    for (int n = 0; n < N; ++n) {
        status = orc_precond_inv(R, Gam + ((int64_t)n * N + n) * R * R, lam, reg, Pinv + (int64_t)n * R * R);
        if (status != ORC_OK) goto done;
    }
    for (int64_t i = 0; i < len; ++i) { V[i] = 0.0; Rv[i] = -G[i]; }
    apply_precond(d, Pinv, Rv, Z);
    for (int64_t i = 0; i < len; ++i) W[i] = Z[i];
    double rz = dot_all(len, Rv, Z);
    const double gsum = fro_sum(d, G);
    int it = 0;
    double rsum = fro_sum(d, Rv);
    while (rsum > eps_cg * gsum) {
        if (it >= maxit) { status = ORC_WARN_CG_MAXIT; break; }
        orc_matvec(d, A, Gam, W, lam, reg, Q);
        const double wq = dot_all(len, W, Q);
        if (!(wq > 0.0)) { status = ORC_ERR_BREAKDOWN; break; }
        const double alpha = rz / wq;
        for (int64_t i = 0; i < len; ++i) { V[i] += alpha * W[i]; Rv[i] -= alpha * Q[i]; }
        apply_precond(d, Pinv, Rv, Z);
        const double rz_new = dot_all(len, Rv, Z);
        const double beta = (beta_kind == 1) ? rz_new / wq : rz_new / rz;
        for (int64_t i = 0; i < len; ++i) W[i] = Z[i] + beta * W[i];
        rz = rz_new;
        ++it;
        rsum = fro_sum(d, Rv);
    }
    *iters_out = it;
    *rnorm_out = rsum;
done:
    free(Pinv); free(Rv); free(Z); free(W); free(Q);
    return status;
}

/* ------------------------------------------------------------ lambda rule */

/* Varying regularisation (Section 3.2): lambda is divided by mu > 1 at every
 * iteration until the next value would fall below the lower threshold, then
 * multiplied by mu until the next value would exceed the upper threshold,
 * then divided again.  dir: 0 = going down, 1 = going up. */
void orc_lambda_next(double* lam, int* dir, double lo, double hi, double mu) {
    if (*dir == 0) {
        const double t = *lam / mu;
        if (t < lo) { *dir = 1; *lam = *lam * mu; }
        else *lam = t;
    } else {
        const double t = *lam * mu;
        if (t > hi) { *dir = 0; *lam = *lam / mu; }
        else *lam = t;
    }
}

/* ------------------------------------------------------------------ GN step */

static double sq_residual(const orc_desc* d, const double* X, const double* A, double* sq_x);

/* Options of one GN iteration beyond Algorithm 1's plain loop body. */
typedef struct {
    double stop_ratio;   /* > 0: Algorithm 1's loop test at the entry point (see gn_iteration) */
    int lam_fixed;       /* 1: lambda stays constant (constant regularisation, Section 5) */
    double armijo_c;     /* > 0: step-size control by Armijo's condition (Section 5) */
    double armijo_beta;  /* step reduction factor of the backtracking, 0 < beta < 1 */
    int armijo_max;      /* reductions tried after the full step */
} gn_opts;

/* One iteration of CP-GN, Algorithm 1: M^(n) for all n, Gamma^(n,p), G^(n),
 * then Algorithm 1's loop test (stop_ratio > 0: if sum_n ||G^(n)||_F <=
 * stop_ratio sum_n ||M^(n)||_F -- the scale-free reading of the test on
 * sum_n ||G^(n)||_F -- the entry point is accepted: no CG, no update,
 * *stopped = 1), else CP-CG with the current lambda, A^(n) += V^(n), and
 * lambda advances by the varying rule (the lambda of the next iteration).
 * stats as orc_gn_step. */
static int gn_iteration(const orc_desc* d, const double* X, double* A, double* lam, int* dir, double lam_lo,
                        double lam_hi, double mu, double eps_cg, int maxit, int beta_kind, int use_dt, int reg,
                        const gn_opts* o, double* stats, int* stopped) {
    const double stop_ratio = o->stop_ratio;
    const int N = d->N, R = d->R;
    const int64_t len = factor_total(d);
    double* M = (double*)malloc(sizeof(double) * len);
    double* G = (double*)malloc(sizeof(double) * len);
    double* V = (double*)calloc((size_t)len, sizeof(double));
    double* S = (double*)malloc(sizeof(double) * (size_t)N * R * R);
    double* Gam = (double*)malloc(sizeof(double) * (size_t)N * N * R * R);
    double gnorm[ORC_MAXN];
    if (use_dt) orc_mttkrp_dt(d, X, A, M); else orc_mttkrp_def(d, X, A, M);
    orc_gram(d, A, S);
    orc_gamma(d, S, Gam);
    orc_gradient(d, A, Gam, M, G, gnorm);
    double gsum = 0.0;
    for (int n = 0; n < N; ++n) gsum += gnorm[n];
    const double msum = fro_sum(d, M);
    int iters = 0;
    double rnorm = 0.0;
    const double lam_used = *lam;
    int status = ORC_OK;
    *stopped = stop_ratio > 0.0 && gsum <= stop_ratio * msum;
    double step = 1.0, f0 = -1.0;
    int trials = 0;
    if (!*stopped) {
        status = orc_pcg(d, A, Gam, G, lam_used, reg, eps_cg, maxit, beta_kind, V, &iters, &rnorm);
        if ((status == ORC_OK || status == ORC_WARN_CG_MAXIT) && o->armijo_c > 0.0) {
            /* Armijo's condition on f = 1/2 ||X - [[A]]||^2 along V: accept the first
             * t in 1, beta, beta^2, ... with f(A + t V) <= f(A) + c t <grad f, V>
             * (grad f = G, Eq. (2.3)) up to the evaluation accuracy of f; none
             * accepted: no update (t = 0). */
            double* At = (double*)malloc(sizeof(double) * len);
            double unused, xx;
            f0 = 0.5 * sq_residual(d, X, A, &xx);
            /* the condition is relaxed by the accuracy of the FP64 evaluation of f,
             * 2 R 2^-53 ||X||^2, so that steps below it are not rejected on rounding */
            const double tol_f = 2.0 * R * 0x1p-53 * xx;
            double slope = 0.0;
            for (int64_t i = 0; i < len; ++i) slope += G[i] * V[i];
            double t = 1.0;
            step = 0.0;
            for (int k = 0; k <= o->armijo_max; ++k, t *= o->armijo_beta) {
                for (int64_t i = 0; i < len; ++i) At[i] = A[i] + t * V[i];
                ++trials;
                if (0.5 * sq_residual(d, X, At, &unused) <= f0 + o->armijo_c * t * slope + tol_f) {
                    step = t;
                    break;
                }
            }
            free(At);
        }
        if (status == ORC_OK || status == ORC_WARN_CG_MAXIT) {
            for (int64_t i = 0; i < len; ++i) A[i] += step * V[i];
            if (!o->lam_fixed) orc_lambda_next(lam, dir, lam_lo, lam_hi, mu);
        }
    }
    stats[0] = gsum;
    stats[1] = fro_sum(d, V);
    stats[2] = lam_used;
    stats[3] = iters;
    stats[4] = rnorm;
    stats[5] = msum;
    stats[6] = step;
    stats[7] = f0;
    stats[8] = trials;
    free(M); free(G); free(V); free(S); free(Gam);
    return status;
}

/* One iteration of CP-GN, Algorithm 1: M^(n) for all n, Gamma^(n,p), G^(n),
 * CP-CG with the current lambda, A^(n) += V^(n); then lambda advances by the
 * varying rule (the lambda of the next iteration).
 * stats[0] = sum_n ||G^(n)||_F at the entry point, stats[1] = sum_n ||V^(n)||_F,
 * stats[2] = lambda used, stats[3] = CG iterations, stats[4] = final CG
 * residual sum, stats[5] = sum_n ||M^(n)||_F.
 * use_dt selects the dimension-tree MTTKRP (1) or the definition (0); reg the
 * damping of the CG system (ORC_REG_IDENTITY or ORC_REG_DIAG). */
int orc_gn_step(const orc_desc* d, const double* X, double* A, double* lam, int* dir, double lam_lo,
                double lam_hi, double mu, double eps_cg, int maxit, int beta_kind, int use_dt, int reg,
                double* stats) {
    int stopped = 0;
    const gn_opts o = {0.0, 0, 0.0, 0.5, 0};
    double st[9];
    const int status = gn_iteration(d, X, A, lam, dir, lam_lo, lam_hi, mu, eps_cg, maxit, beta_kind, use_dt, reg,
                                    &o, st, &stopped);
    for (int k = 0; k < 6; ++k) stats[k] = st[k];
    return status;
}

/* One iteration of Algorithm 1 with the options of Section 5's experiments:
 * a constant lambda (lam_fixed = 1) and step-size control by Armijo's
 * condition (armijo_c > 0; backtracking by armijo_beta, at most armijo_max
 * reductions).  stats[0..5] as orc_gn_step, stats[6] = the step length t
 * applied (1 without the line search; 0 when no trial met the condition),
 * stats[7] = f(A) = 1/2 ||X - [[A]]||_F^2 at the entry point (-1 without the
 * line search), stats[8] = trial points evaluated. */
int orc_gn_step_ls(const orc_desc* d, const double* X, double* A, double* lam, int* dir, double lam_lo,
                   double lam_hi, double mu, double eps_cg, int maxit, int use_dt, int reg, int lam_fixed,
                   double armijo_c, double armijo_beta, int armijo_max, double* stats) {
    int stopped = 0;
    const gn_opts o = {0.0, lam_fixed, armijo_c, armijo_beta, armijo_max};
    return gn_iteration(d, X, A, lam, dir, lam_lo, lam_hi, mu, eps_cg, maxit, 0, use_dt, reg, &o, stats, &stopped);
}

/* Algorithm 1 to a target: GN iterations from A (in/out) with lambda starting
 * at lam0 in the decreasing direction, until the entry point of an iteration
 * has sum_n ||G^(n)||_F <= target sum_n ||M^(n)||_F (converged; that
 * iteration applies no update) or max_gn updates have been applied.
 * out[0] = updates applied, out[1] = CG iterations in all, out[2] = the last
 * sum||G|| / sum||M||, out[3] = 1 if converged, out[4] = lambda after the last
 * update.  Returns the status of the last iteration (ORC_WARN_CG_MAXIT is not
 * an error here). */
int orc_gn_solve(const orc_desc* d, const double* X, double* A, double lam0, double lam_lo, double lam_hi,
                 double mu, double eps_cg, int maxit, double target, int max_gn, int use_dt, int reg,
                 double* out) {
    double lam = lam0, stats[9];
    int dir = 0, status = ORC_OK, updates = 0, cg = 0, stopped = 0;
    double ratio = 0.0;
    const gn_opts o = {target, 0, 0.0, 0.5, 0};
    while (updates < max_gn) {
        status = gn_iteration(d, X, A, &lam, &dir, lam_lo, lam_hi, mu, eps_cg, maxit, 0, use_dt, reg, &o, stats,
                              &stopped);
        ratio = stats[5] > 0.0 ? stats[0] / stats[5] : 0.0;
        if (stopped) break;
        if (status != ORC_OK && status != ORC_WARN_CG_MAXIT) break;
        cg += (int)stats[3];
        ++updates;
    }
    out[0] = updates;
    out[1] = cg;
    out[2] = ratio;
    out[3] = stopped;
    out[4] = lam;
    return status == ORC_WARN_CG_MAXIT ? ORC_OK : status;
}

/* Threads of the OpenMP loops from now on (a timing aid: 1 gives the
 * one-core figure). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ----------------------------------------------------------------- residual */

/* r = ||X - [[A]]||_F / ||X||_F (Section 5, relative residual), with the
 * reconstruction evaluated element by element from Section 2.2's CP model and
 * both squared sums accumulated with Kahan compensation. */
double orc_residual(const orc_desc* d, const double* X, const double* A) {
    double den = 0.0;
    const double num = sq_residual(d, X, A, &den);
    return sqrt(num) / sqrt(den);
}

/* ||X - [[A]]||_F^2, with *sq_x = ||X||_F^2: the reconstruction evaluated
 * element by element, both sums with Kahan compensation. */
static double sq_residual(const orc_desc* d, const double* X, const double* A, double* sq_x) {
    const int N = d->N, R = d->R;
    const int64_t total = tensor_size(d);
    double num = 0.0, den = 0.0;
#pragma omp parallel
    {
        double s_num = 0.0, c_num = 0.0, s_den = 0.0, c_den = 0.0;
        int64_t idx[ORC_MAXN];
#pragma omp for schedule(static)
        for (int64_t e = 0; e < total; ++e) {
            unravel(d, e, idx);
            double xt = 0.0;
            for (int r = 0; r < R; ++r) {
                double prod = 1.0;
                for (int m = 0; m < N; ++m) prod *= A[factor_offset(d, m) + idx[m] * R + r];
                xt += prod;
            }
            const double diff = X[e] - xt;
            double y = diff * diff - c_num, t = s_num + y;
            c_num = (t - s_num) - y; s_num = t;
            y = X[e] * X[e] - c_den; t = s_den + y;
            c_den = (t - s_den) - y; s_den = t;
        }
#pragma omp critical
        { num += s_num; den += s_den; }
    }
    *sq_x = den;
    return num;
}

/* The residual tensor E = X - [[A]] element by element (Section 2.2's CP
 * model written out: each entry of the reconstruction is the sum over r of
 * the products of the factors' entries), in FP64, C-contiguous like X. */
void orc_residual_tensor(const orc_desc* d, const double* X, const double* A, double* E) {
    const int N = d->N, R = d->R;
    const int64_t total = tensor_size(d);
#pragma omp parallel
    {
        int64_t idx[ORC_MAXN];
#pragma omp for schedule(static)
        for (int64_t e = 0; e < total; ++e) {
            unravel(d, e, idx);
            double xt = 0.0;
            for (int r = 0; r < R; ++r) {
                double prod = 1.0;
                for (int m = 0; m < N; ++m) prod *= A[factor_offset(d, m) + idx[m] * R + r];
                xt += prod;
            }
            E[e] = X[e] - xt;
        }
    }
}

/* ----------------------------------------------------------------- ALS sweep */

/* One CP-ALS sweep (Section 2.2): for n = 1..N in order, with the factors
 * already updated in this sweep, M^(n) = X_(n) P^(n) and
 * A^(n)_new (Gamma^(n) + lam I) = M^(n), solved with the inverse of the
 * R x R matrix built from its Cholesky factor (as for the preconditioner).
 * lam = 0 gives the plain normal equations. */
int orc_als_sweep(const orc_desc* d, const double* X, double* A, double lam) {
    const int N = d->N, R = d->R;
    double* S = (double*)malloc(sizeof(double) * (size_t)N * R * R);
    double* Gam = (double*)malloc(sizeof(double) * (size_t)N * N * R * R);
    double* Pinv = (double*)malloc(sizeof(double) * (size_t)R * R);
    double* Mrow = (double*)malloc(sizeof(double) * R);
    int status = ORC_OK;
    for (int n = 0; n < N && status == ORC_OK; ++n) {
        orc_gram(d, A, S);
        orc_gamma(d, S, Gam);
        /* M^(n) rows by definition; A^(n) is replaced only after all rows are formed */
        const int64_t sn = d->dims[n];
        double* Mn = (double*)malloc(sizeof(double) * sn * R);
#pragma omp parallel for
        for (int64_t i = 0; i < sn; ++i) orc_mttkrp_row(d, X, A, n, i, Mn + i * R);
        status = orc_precond_inv(R, Gam + ((int64_t)n * N + n) * R * R, lam, ORC_REG_IDENTITY, Pinv);
        if (status == ORC_OK) {
            double* An = A + factor_offset(d, n);
            for (int64_t i = 0; i < sn; ++i)
                for (int r = 0; r < R; ++r) {
                    double acc = 0.0;
                    for (int z = 0; z < R; ++z) acc += Mn[i * R + z] * Pinv[z * R + r];
                    An[i * R + r] = acc;
                }
        }
        free(Mn);
    }
    free(S); free(Gam); free(Pinv); free(Mrow);
    return status;
}

/* ----------------------------------------------------------------- Tucker / HoSVD */

/* S = X_(n) X_(n)^T (s_n x s_n), the Gram matrix of the mode-n unfolding, by
 * its definition: S[j][j'] = sum over all indices but the n-th of
 * x[.., j, ..] x[.., j', ..]. */
void orc_unfold_gram(const orc_desc* d, const double* X, int n, double* S) {
    const int N = d->N;
    int64_t L = 1, Rr = 1;
    for (int m = 0; m < n; ++m) L *= d->dims[m];
    for (int m = n + 1; m < N; ++m) Rr *= d->dims[m];
    const int64_t sn = d->dims[n];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < sn; ++j)
        for (int64_t jj = 0; jj < sn; ++jj) {
            double acc = 0.0;
            for (int64_t l = 0; l < L; ++l) {
                const double* a = X + (l * sn + j) * Rr;
                const double* b = X + (l * sn + jj) * Rr;
                for (int64_t c = 0; c < Rr; ++c) acc += a[c] * b[c];
            }
            S[j * sn + jj] = acc;
        }
}

/* Eigen-decomposition of a symmetric s x s matrix S by the cyclic Jacobi
 * method (plane rotations annihilating S[p][q] in row order, sweeps until the
 * off-diagonal mass is below 1e-30 of the total or 100 sweeps): on return
 * w holds the eigenvalues in decreasing order and column i of V (row-major
 * s x s) the unit eigenvector of w[i].  S is overwritten. */
void orc_sym_eig(int s, double* S, double* w, double* V) {
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) V[i * s + j] = i == j ? 1.0 : 0.0;
    double tot = 0.0;
    for (int i = 0; i < s * s; ++i) tot += S[i] * S[i];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < s; ++p)
            for (int q = p + 1; q < s; ++q) off += 2.0 * S[p * s + q] * S[p * s + q];
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < s; ++p)
            for (int q = p + 1; q < s; ++q) {
                const double apq = S[p * s + q];
                if (apq == 0.0) continue;
                const double app = S[p * s + p], aqq = S[q * s + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < s; ++k) {  /* columns p, q */
                    const double skp = S[k * s + p], skq = S[k * s + q];
                    S[k * s + p] = c * skp - sn * skq;
                    S[k * s + q] = sn * skp + c * skq;
                }
                for (int k = 0; k < s; ++k) {  /* rows p, q */
                    const double spk = S[p * s + k], sqk = S[q * s + k];
                    S[p * s + k] = c * spk - sn * sqk;
                    S[q * s + k] = sn * spk + c * sqk;
                }
                for (int k = 0; k < s; ++k) {
                    const double vkp = V[k * s + p], vkq = V[k * s + q];
                    V[k * s + p] = c * vkp - sn * vkq;
                    V[k * s + q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < s; ++i) w[i] = S[i * s + i];
    /* decreasing order (selection sort, columns of V moved along) */
    for (int i = 0; i < s; ++i) {
        int b = i;
        for (int j = i + 1; j < s; ++j)
            if (w[j] > w[b]) b = j;
        if (b != i) {
            const double t = w[i];
            w[i] = w[b];
            w[b] = t;
            for (int k = 0; k < s; ++k) {
                const double x = V[k * s + i];
                V[k * s + i] = V[k * s + b];
                V[k * s + b] = x;
            }
        }
    }
}

/* Y = T x_n U^T: the mode-n product of a dense tensor T (dims `dims`, order N)
 * with U^T, U an s_n x r matrix (row-major): Y has r in place of s_n,
 * Y[.., a, ..] = sum_j U[j][a] T[.., j, ..]. */
void orc_mode_product_t(int N, const int64_t* dims, const double* T, int n, int r, const double* U, double* Y) {
    int64_t L = 1, Rr = 1;
    for (int m = 0; m < n; ++m) L *= dims[m];
    for (int m = n + 1; m < N; ++m) Rr *= dims[m];
    const int64_t sn = dims[n];
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < L; ++l)
        for (int a = 0; a < r; ++a)
            for (int64_t c = 0; c < Rr; ++c) {
                double acc = 0.0;
                for (int64_t j = 0; j < sn; ++j) acc += U[j * r + a] * T[(l * sn + j) * Rr + c];
                Y[(l * r + a) * Rr + c] = acc;
            }
}
