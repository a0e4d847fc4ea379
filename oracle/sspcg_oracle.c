/*
 * FP64 CPU oracle for the symmetric stair preconditioned CG path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA library; both are fed the same inputs.
 *
 * Plain, slow, obviously correct: every step follows the paper's order and
 * notation, in double precision, with no blocking or fusion.
 *
 *   Sec. II-A, Eq. (schur) and the theta/phi/zeta block formulas:
 *     theta_k = -A_k Q_k^-1 A_k^T - B_k R_k^-1 B_k^T - Q_{k+1}^-1
 *     phi_k   =  A_k Q_k^-1
 *     S_paper = [[-Q_0^-1, phi_0^T], [phi_0, theta_0, phi_1^T], ...]
 *   The footnote of Sec. II-A negates S to make it positive definite; the
 *   oracle returns the negated (SPD) matrix S = -S_paper = C G^-1 C^T.
 *
 *   Sec. III, Eq. (stair) and Eq. (stair_inv): Psi_l keeps the off-diagonal
 *   blocks of the even (1-based) block rows, Psi_r those of the odd rows;
 *   Psi^-1 = D^-1 (2D - Psi) D^-1.
 *   Sec. III, additive stair: Phi_add^-1 = (Psi_l^-1 + Psi_r^-1) / 2.
 *   Sec. IV: Phi_sym^-1 = Psi_l^-1 + Psi_r^-1 - D^-1.
 *   Sec. II-C, Eq. (jacobi): Phi = diag(S) or Phi = block-diag(S).
 *
 *   Sec. II-A with full SPD Q_k, R_k: the same formulas with matrix inverses
 *   (oracle_build_schur_full).
 *
 *   Sec. II-B: PCG, written as the textbook algorithm the paper cites
 *   (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.1).
 *
 *   Sec. II-C, Eq. (polynomial_precon): for a splitting S = Psi - P,
 *   Phi^-1 = (I + Psi^-1 P + (Psi^-1 P)^2 + ...) Psi^-1, truncated after the
 *   degree-d term.  Psi^-1 is one of the preconditioners above (so Psi is
 *   the matrix whose inverse that preconditioner is) and P = Psi - S, so
 *   Psi^-1 P t = t - Psi^-1 S t: each term follows from the previous one
 *   with one product by S and one by Psi^-1.
 *
 * Block-tridiagonal storage used here (row-major nx*nx blocks, FP64):
 *   d[k] = M(k, k)     k = 0..N
 *   l[k] = M(k, k-1)   k = 1..N   (slot 0 unused)
 *   u[k] = M(k, k+1)   k = 0..N-1 (slot N unused)
 * i.e. three arrays of (N+1) blocks each.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_SYM_STAIR = 0, OR_ADD_STAIR = 1, OR_BLOCK_JACOBI = 2, OR_JACOBI = 3 };
enum { OR_OK = 0, OR_MAXITER = 1, OR_BREAKDOWN = 2, OR_NOT_SPD = 3, OR_NONFINITE = 4, OR_BADARG = 5 };

#define BLK(a, k, m) ((a) + (size_t)(k) * (size_t)(m) * (size_t)(m))

/* C = alpha * X * Y + beta * C, all m x m row-major. */
static void mm(int m, double alpha, const double *X, const double *Y, double beta, double *C) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int t = 0; t < m; ++t) s += X[i * m + t] * Y[t * m + j];
            C[i * m + j] = alpha * s + beta * C[i * m + j];
        }
}

static void transpose(int m, const double *X, double *XT) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) XT[j * m + i] = X[i * m + j];
}

/*
 * Sec. II-A block formulas, then the SPD negation of the footnote.
 * A: [N][nx][nx]  B: [N][nx][nu]  qd: [N+1][nx] (diag Q_k)  rd: [N][nu] (diag R_k)
 * Output d, l, u: block-tridiagonal S = C G^-1 C^T (three arrays of N+1 blocks).
 */
int oracle_build_schur(int N, int nx, int nu, const double *A, const double *B, const double *qd,
                       const double *rd, double *d, double *l, double *u) {
    if (N < 0 || nx < 1 || nu < 0) return OR_BADARG;
    const int m = nx;
    const size_t blk = (size_t)m * m;
    memset(d, 0, sizeof(double) * blk * (N + 1));
    memset(l, 0, sizeof(double) * blk * (N + 1));
    memset(u, 0, sizeof(double) * blk * (N + 1));
    /* first diagonal block of S_paper is -Q_0^-1; negated: Q_0^-1 */
    for (int i = 0; i < m; ++i) d[i * m + i] = 1.0 / qd[i];
    double *theta = (double *)malloc(sizeof(double) * blk);
    double *phi = (double *)malloc(sizeof(double) * blk);
    for (int k = 0; k < N; ++k) {
        const double *Ak = A + (size_t)k * m * m;
        const double *Bk = B + (size_t)k * m * nu;
        const double *qk = qd + (size_t)k * m;
        const double *qk1 = qd + (size_t)(k + 1) * m;
        const double *rk = rd + (size_t)k * nu;
        /* phi_k = A_k Q_k^-1 */
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) phi[i * m + j] = Ak[i * m + j] / qk[j];
        /* theta_k = -A_k Q_k^-1 A_k^T - B_k R_k^-1 B_k^T - Q_{k+1}^-1 */
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double s = 0.0;
                for (int t = 0; t < m; ++t) s += Ak[i * m + t] * Ak[j * m + t] / qk[t];
                double sb = 0.0;
                for (int t = 0; t < nu; ++t) sb += Bk[i * nu + t] * Bk[j * nu + t] / rk[t];
                theta[i * m + j] = -s - sb - (i == j ? 1.0 / qk1[i] : 0.0);
            }
        /* S_paper(k+1,k+1) = theta_k, S_paper(k+1,k) = phi_k, S_paper(k,k+1) = phi_k^T; negate */
        for (size_t e = 0; e < blk; ++e) {
            BLK(d, k + 1, m)[e] = -theta[e];
            BLK(l, k + 1, m)[e] = -phi[e];
        }
        transpose(m, BLK(l, k + 1, m), BLK(u, k, m));
    }
    free(theta);
    free(phi);
    return OR_OK;
}

/* In-place Cholesky of an SPD m x m matrix (lower factor). Returns 0 on success. */
static int cholesky(int m, double *a) {
    for (int j = 0; j < m; ++j) {
        double s = a[j * m + j];
        for (int t = 0; t < j; ++t) s -= a[j * m + t] * a[j * m + t];
        if (!(s > 0.0) || !isfinite(s)) return -1;
        const double ljj = sqrt(s);
        a[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double v = a[i * m + j];
            for (int t = 0; t < j; ++t) v -= a[i * m + t] * a[j * m + t];
            a[i * m + j] = v / ljj;
        }
        for (int i = 0; i < j; ++i) a[i * m + j] = 0.0;
    }
    return 0;
}

/* inv = M^-1 for SPD M via Cholesky: solve L L^T x = e_c column by column. */
static int spd_inverse(int m, const double *M, double *inv) {
    double *L = (double *)malloc(sizeof(double) * m * m);
    double *y = (double *)malloc(sizeof(double) * m);
    memcpy(L, M, sizeof(double) * m * m);
    int rc = cholesky(m, L);
    if (rc == 0) {
        for (int c = 0; c < m; ++c) {
            for (int i = 0; i < m; ++i) { /* forward: L y = e_c */
                double v = (i == c) ? 1.0 : 0.0;
                for (int t = 0; t < i; ++t) v -= L[i * m + t] * y[t];
                y[i] = v / L[i * m + i];
            }
            for (int i = m - 1; i >= 0; --i) { /* backward: L^T x = y */
                double v = y[i];
                for (int t = i + 1; t < m; ++t) v -= L[t * m + i] * inv[t * m + c];
                inv[i * m + c] = v / L[i * m + i];
            }
        }
    }
    free(L);
    free(y);
    return rc;
}

/*
 * Sec. II-A block formulas with full SPD cost blocks (the paper writes Q_k^-1
 * and R_k^-1 as matrices), then the SPD negation of the footnote.
 * Q: [N+1][nx][nx]  R: [N][nu][nu]; inverses by Cholesky (spd_inverse).
 *   phi_k   = A_k Q_k^-1
 *   theta_k = -A_k Q_k^-1 A_k^T - B_k R_k^-1 B_k^T - Q_{k+1}^-1
 * Returns OR_NOT_SPD when a Q_k or R_k is not positive definite.
 */
int oracle_build_schur_full(int N, int nx, int nu, const double *A, const double *B, const double *Q,
                            const double *R, double *d, double *l, double *u) {
    if (N < 0 || nx < 1 || nu < 0) return OR_BADARG;
    const int m = nx;
    const size_t blk = (size_t)m * m;
    memset(d, 0, sizeof(double) * blk * (N + 1));
    memset(l, 0, sizeof(double) * blk * (N + 1));
    memset(u, 0, sizeof(double) * blk * (N + 1));
    double *Qi = (double *)malloc(sizeof(double) * blk * (N + 1));
    double *Ri = (double *)malloc(sizeof(double) * (size_t)(nu > 0 ? nu * nu : 1) * (N > 0 ? N : 1));
    double *theta = (double *)malloc(sizeof(double) * blk), *phi = (double *)malloc(sizeof(double) * blk);
    int rc = OR_OK;
    for (int k = 0; k <= N && rc == OR_OK; ++k)
        if (spd_inverse(m, Q + (size_t)k * blk, Qi + (size_t)k * blk) != 0) rc = OR_NOT_SPD;
    for (int k = 0; k < N && nu > 0 && rc == OR_OK; ++k)
        if (spd_inverse(nu, R + (size_t)k * nu * nu, Ri + (size_t)k * nu * nu) != 0) rc = OR_NOT_SPD;
    if (rc == OR_OK) {
        /* first diagonal block of S_paper is -Q_0^-1; negated: Q_0^-1 */
        memcpy(d, Qi, sizeof(double) * blk);
        for (int k = 0; k < N; ++k) {
            const double *Ak = A + (size_t)k * m * m, *Bk = B + (size_t)k * m * nu;
            const double *Qk = Qi + (size_t)k * blk, *Qk1 = Qi + (size_t)(k + 1) * blk;
            const double *Rk = Ri + (size_t)k * nu * nu;
            /* phi_k = A_k Q_k^-1 */
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) {
                    double s = 0.0;
                    for (int t = 0; t < m; ++t) s += Ak[i * m + t] * Qk[t * m + j];
                    phi[i * m + j] = s;
                }
            /* theta_k = -phi_k A_k^T - (B_k R_k^-1) B_k^T - Q_{k+1}^-1 */
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) {
                    double s = 0.0;
                    for (int t = 0; t < m; ++t) s += phi[i * m + t] * Ak[j * m + t];
                    double sb = 0.0;
                    for (int a = 0; a < nu; ++a) {
                        double br = 0.0;
                        for (int b = 0; b < nu; ++b) br += Bk[i * nu + b] * Rk[b * nu + a];
                        sb += br * Bk[j * nu + a];
                    }
                    theta[i * m + j] = -s - sb - Qk1[i * m + j];
                }
            for (size_t e = 0; e < blk; ++e) {
                BLK(d, k + 1, m)[e] = -theta[e];
                BLK(l, k + 1, m)[e] = -phi[e];
            }
            transpose(m, BLK(l, k + 1, m), BLK(u, k, m));
        }
    }
    free(Qi); free(Ri); free(theta); free(phi);
    return rc;
}

/*
 * Eq. (stair_inv): inverse of a stair matrix, Psi^-1 = D^-1 (2D - Psi) D^-1.
 * The stair keeps the off-diagonal blocks of S in the block rows selected by
 * ``keep_odd_rows_1based`` (1 -> Psi_r, 0 -> Psi_l).  (2D - Psi) has diagonal
 * blocks D_k and off-diagonal blocks -Psi(k, j), so Psi^-1 has diagonal blocks
 * D_k^-1 and off-diagonal blocks -D_k^-1 S(k, j) D_j^-1 in the kept rows.
 */
static void stair_inverse(int N, int m, int keep_odd_rows_1based, const double *Dinv, const double *l,
                          const double *u, double *pd, double *pl, double *pu) {
    const size_t blk = (size_t)m * m;
    double *tmp = (double *)malloc(sizeof(double) * blk);
    memset(pl, 0, sizeof(double) * blk * (N + 1));
    memset(pu, 0, sizeof(double) * blk * (N + 1));
    for (int k = 0; k <= N; ++k) {
        memcpy(BLK(pd, k, m), BLK(Dinv, k, m), sizeof(double) * blk);
        const int row1 = k + 1; /* 1-based block row */
        const int kept = keep_odd_rows_1based ? (row1 % 2 == 1) : (row1 % 2 == 0);
        if (!kept) continue;
        if (k > 0) { /* -D_k^-1 S(k,k-1) D_{k-1}^-1 */
            mm(m, 1.0, BLK(Dinv, k, m), BLK(l, k, m), 0.0, tmp);
            mm(m, -1.0, tmp, BLK(Dinv, k - 1, m), 0.0, BLK(pl, k, m));
        }
        if (k < N) { /* -D_k^-1 S(k,k+1) D_{k+1}^-1 */
            mm(m, 1.0, BLK(Dinv, k, m), BLK(u, k, m), 0.0, tmp);
            mm(m, -1.0, tmp, BLK(Dinv, k + 1, m), 0.0, BLK(pu, k, m));
        }
    }
    free(tmp);
}

/*
 * Preconditioner Phi^-1 as a block-tridiagonal matrix (pd, pl, pu: N+1 blocks each).
 *   kind 0: symmetric stair  Phi_sym^-1 = Psi_l^-1 + Psi_r^-1 - D^-1   (Sec. IV)
 *   kind 1: additive stair   Phi_add^-1 = (Psi_l^-1 + Psi_r^-1) / 2    (Sec. III)
 *   kind 2: block-Jacobi     Phi^-1 = block-diag(S)^-1                 (Eq. jacobi)
 *   kind 3: Jacobi           Phi^-1 = diag(S)^-1                       (Eq. jacobi)
 * Returns OR_NOT_SPD if a diagonal block is not positive definite.
 */
int oracle_build_precond(int N, int nx, int kind, const double *d, const double *l, const double *u,
                         double *pd, double *pl, double *pu) {
    if (N < 0 || nx < 1 || kind < 0 || kind > 3) return OR_BADARG;
    const int m = nx;
    const size_t blk = (size_t)m * m, nb = (size_t)(N + 1);
    memset(pd, 0, sizeof(double) * blk * nb);
    memset(pl, 0, sizeof(double) * blk * nb);
    memset(pu, 0, sizeof(double) * blk * nb);
    if (kind == OR_JACOBI) {
        for (int k = 0; k <= N; ++k)
            for (int i = 0; i < m; ++i) {
                const double s = BLK(d, k, m)[i * m + i];
                if (!(s > 0.0)) return OR_NOT_SPD;
                BLK(pd, k, m)[i * m + i] = 1.0 / s;
            }
        return OR_OK;
    }
    double *Dinv = (double *)malloc(sizeof(double) * blk * nb);
    for (int k = 0; k <= N; ++k)
        if (spd_inverse(m, BLK(d, k, m), BLK(Dinv, k, m)) != 0) {
            free(Dinv);
            return OR_NOT_SPD;
        }
    if (kind == OR_BLOCK_JACOBI) {
        memcpy(pd, Dinv, sizeof(double) * blk * nb);
        free(Dinv);
        return OR_OK;
    }
    double *ld = (double *)malloc(sizeof(double) * blk * nb), *ll = (double *)malloc(sizeof(double) * blk * nb),
           *lu = (double *)malloc(sizeof(double) * blk * nb);
    double *rd = (double *)malloc(sizeof(double) * blk * nb), *rl = (double *)malloc(sizeof(double) * blk * nb),
           *ru = (double *)malloc(sizeof(double) * blk * nb);
    stair_inverse(N, m, 0, Dinv, l, u, ld, ll, lu); /* Psi_l^-1 */
    stair_inverse(N, m, 1, Dinv, l, u, rd, rl, ru); /* Psi_r^-1 */
    for (size_t e = 0; e < blk * nb; ++e) {
        if (kind == OR_SYM_STAIR) {
            pd[e] = ld[e] + rd[e] - Dinv[e];
            pl[e] = ll[e] + rl[e];
            pu[e] = lu[e] + ru[e];
        } else {
            pd[e] = 0.5 * (ld[e] + rd[e]);
            pl[e] = 0.5 * (ll[e] + rl[e]);
            pu[e] = 0.5 * (lu[e] + ru[e]);
        }
    }
    free(ld); free(ll); free(lu); free(rd); free(rl); free(ru); free(Dinv);
    return OR_OK;
}

/* y = M x for block-tridiagonal M (general: lower and upper blocks independent). */
static void bt_matvec(int N, int m, const double *d, const double *l, const double *u, const double *x, double *y) {
    for (int k = 0; k <= N; ++k)
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += BLK(d, k, m)[i * m + j] * x[k * m + j];
            if (k > 0)
                for (int j = 0; j < m; ++j) s += BLK(l, k, m)[i * m + j] * x[(k - 1) * m + j];
            if (k < N)
                for (int j = 0; j < m; ++j) s += BLK(u, k, m)[i * m + j] * x[(k + 1) * m + j];
            y[k * m + i] = s;
        }
}

static double dot(size_t n, const double *a, const double *b) {
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * z = sum_{j=0..degree} (Psi^-1 P)^j Psi^-1 r  (Eq. polynomial_precon), with
 * Psi^-1 = M (pd, pl, pu) and P = Psi - S.  Term by term:
 *   t_0 = Psi^-1 r,  t_j = Psi^-1 P t_{j-1} = t_{j-1} - Psi^-1 (S t_{j-1}),  z = sum_j t_j.
 * t, s and ps are scratch vectors of the same length.  degree = 0: z = M r.
 */
static void apply_poly(int N, int m, const double *d, const double *l, const double *u, const double *pd,
                       const double *pl, const double *pu, int degree, const double *r, double *z, double *t,
                       double *s, double *ps) {
    const size_t n = (size_t)(N + 1) * m;
    bt_matvec(N, m, pd, pl, pu, r, t);
    memcpy(z, t, sizeof(double) * n);
    for (int j = 1; j <= degree; ++j) {
        bt_matvec(N, m, d, l, u, t, s);     /* S t_{j-1} */
        bt_matvec(N, m, pd, pl, pu, s, ps); /* Psi^-1 S t_{j-1} */
        for (size_t i = 0; i < n; ++i) t[i] -= ps[i];
        for (size_t i = 0; i < n; ++i) z[i] += t[i];
    }
}

/* Exported for the tests: z = Phi_d^-1 r of the degree-d polynomial preconditioner. */
int oracle_apply_poly(int N, int nx, const double *d, const double *l, const double *u, const double *pd,
                      const double *pl, const double *pu, int degree, const double *r, double *z) {
    if (N < 0 || nx < 1 || degree < 0) return OR_BADARG;
    const size_t n = (size_t)(N + 1) * nx;
    double *t = (double *)malloc(sizeof(double) * n), *s = (double *)malloc(sizeof(double) * n);
    double *ps = (double *)malloc(sizeof(double) * n);
    apply_poly(N, nx, d, l, u, pd, pl, pu, degree, r, z, t, s, ps);
    free(t); free(s); free(ps);
    return OR_OK;
}

/*
 * Textbook PCG on S x = gamma with preconditioner M = Phi^-1 (both block-tridiagonal),
 * or with its degree-d polynomial (apply_poly) when degree > 0.
 * x: in = x0 (used when warm != 0, else x0 = 0), out = solution.
 * Stops before an iteration when ||r||_2 <= tol * ||gamma||_2, or after max_iter
 * iterations.  iters = number of S*p products.  relres = ||r||_2 / ||gamma||_2 of the
 * recurrence residual; true_relres = ||gamma - S x||_2 / ||gamma||_2.
 * gamma = 0 returns x = 0 and zero iterations.
 */
int oracle_pcg_poly(int N, int nx, const double *d, const double *l, const double *u, const double *pd,
                    const double *pl, const double *pu, int degree, const double *gamma, double *x, int warm,
                    double tol, int max_iter, int *iters, double *relres, double *true_relres) {
    if (N < 0 || nx < 1 || degree < 0) return OR_BADARG;
    const int m = nx;
    const size_t n = (size_t)(N + 1) * m;
    double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n), *s = (double *)malloc(sizeof(double) * n);
    double *ps = (double *)malloc(sizeof(double) * n);
    int status = OR_OK, it = 0;
    const double gnorm = sqrt(dot(n, gamma, gamma));
    if (gnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0;
        *relres = 0.0;
        if (true_relres) *true_relres = 0.0;
        free(r); free(z); free(p); free(w); free(t); free(s); free(ps);
        return OR_OK;
    }
    if (!warm) memset(x, 0, sizeof(double) * n);
    bt_matvec(N, m, d, l, u, x, w); /* r0 = gamma - S x0 */
    for (size_t i = 0; i < n; ++i) r[i] = gamma[i] - w[i];
    apply_poly(N, m, d, l, u, pd, pl, pu, degree, r, z, t, s, ps); /* z0 = Phi^-1 r0 */
    memcpy(p, z, sizeof(double) * n);
    double rz = dot(n, r, z);
    double rnorm = sqrt(dot(n, r, r));
    while (rnorm > tol * gnorm) {
        if (it >= max_iter) { status = OR_MAXITER; break; }
        bt_matvec(N, m, d, l, u, p, w); /* w = S p */
        const double pw = dot(n, p, w);
        if (!(pw > 0.0) || !isfinite(pw)) { status = isfinite(pw) ? OR_BREAKDOWN : OR_NONFINITE; break; }
        const double alpha = rz / pw;
        for (size_t i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (size_t i = 0; i < n; ++i) r[i] -= alpha * w[i];
        apply_poly(N, m, d, l, u, pd, pl, pu, degree, r, z, t, s, ps); /* z = Phi^-1 r */
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rnorm = sqrt(dot(n, r, r));
        ++it;
        if (!isfinite(rnorm)) { status = OR_NONFINITE; break; }
    }
    *iters = it;
    *relres = rnorm / gnorm;
    if (true_relres) {
        bt_matvec(N, m, d, l, u, x, w);
        for (size_t i = 0; i < n; ++i) w[i] = gamma[i] - w[i];
        *true_relres = sqrt(dot(n, w, w)) / gnorm;
    }
    free(r); free(z); free(p); free(w); free(t); free(s); free(ps);
    return status;
}

int oracle_pcg(int N, int nx, const double *d, const double *l, const double *u, const double *pd, const double *pl,
               const double *pu, const double *gamma, double *x, int warm, double tol, int max_iter, int *iters,
               double *relres, double *true_relres) {
    return oracle_pcg_poly(N, nx, d, l, u, pd, pl, pu, 0, gamma, x, warm, tol, max_iter, iters, relres,
                           true_relres);
}

/*
 * Whole path for a batch of independent problems in FP64: Schur blocks,
 * preconditioner, PCG.  Inputs are packed back to back (offsets in doubles);
 * x is packed like gamma.  OpenMP over problems when available.
 * Returns the number of threads used.
 */
int oracle_solve_batch_poly(int nprob, const int *N, const int *nx, const int *nu, const int64_t *offA,
                            const int64_t *offB, const int64_t *offq, const int64_t *offr, const int64_t *offg,
                            const double *A, const double *B, const double *qd, const double *rd,
                            const double *gamma, int kind, int degree, double tol, int max_iter_or_0, double *x,
                            int *iters, double *relres, int *status, int nthreads) {
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int p = 0; p < nprob; ++p) {
        const int n1 = N[p] + 1, m = nx[p];
        const size_t nb = (size_t)n1 * m * m;
        double *d = (double *)malloc(sizeof(double) * nb), *l = (double *)malloc(sizeof(double) * nb),
               *u = (double *)malloc(sizeof(double) * nb);
        double *pd = (double *)malloc(sizeof(double) * nb), *pl = (double *)malloc(sizeof(double) * nb),
               *pu = (double *)malloc(sizeof(double) * nb);
        int st = oracle_build_schur(N[p], m, nu[p], A + offA[p], B + offB[p], qd + offq[p], rd + offr[p], d, l, u);
        if (st == OR_OK) st = oracle_build_precond(N[p], m, kind, d, l, u, pd, pl, pu);
        if (st == OR_OK) {
            const int max_iter = max_iter_or_0 > 0 ? max_iter_or_0 : 10 * n1 * m;
            st = oracle_pcg_poly(N[p], m, d, l, u, pd, pl, pu, degree, gamma + offg[p], x + offg[p], 0, tol,
                                 max_iter, &iters[p], &relres[p], NULL);
        } else {
            iters[p] = 0;
            relres[p] = NAN;
        }
        status[p] = st;
        free(d); free(l); free(u); free(pd); free(pl); free(pu);
    }
    return used;
}

int oracle_solve_batch(int nprob, const int *N, const int *nx, const int *nu, const int64_t *offA,
                       const int64_t *offB, const int64_t *offq, const int64_t *offr, const int64_t *offg,
                       const double *A, const double *B, const double *qd, const double *rd, const double *gamma,
                       int kind, double tol, int max_iter_or_0, double *x, int *iters, double *relres,
                       int *status, int nthreads) {
    return oracle_solve_batch_poly(nprob, N, nx, nu, offA, offB, offq, offr, offg, A, B, qd, rd, gamma, kind, 0,
                                   tol, max_iter_or_0, x, iters, relres, status, nthreads);
}
