/*
 * stotree_oracle.c -- plain FP64 CPU oracle for the scenario-tree LQ solve step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library.  It shares no code,
 * header or table with the CUDA path.
 *
 * What it computes (Sampathirao, Patrinos, Bemporad, Sopasakis, "Massively
 * parallelizable proximal algorithms for large-scale stochastic optimal
 * control problems"):
 *
 *   orc_factor  -- the offline "Riccati-type recursion" of Section III-D.  The
 *                  paper defers its formulas to an earlier reference, so they
 *                  are derived here by dynamic programming on the value
 *                  functions V^i(x) = x'P^i x + 2 s^i'x + const of the
 *                  problem in eq. (nabla-f-star), with the cost of Section II-B
 *                  written without a 1/2 factor:
 *                    leaf l:    P^l = pi^l P_N
 *                    parent i:  Rbar = pi^i R + sum_j B^j' P^j B^j
 *                               M    = sum_j B^j' P^j A^j
 *                               K^i  = -Rbar^{-1} M
 *                               P^i  = pi^i Q + sum_j A^j' P^j A^j + M' K^i
 *                               gu^i = sum_j B^j' P^j c^j + pi^i r / 2
 *                               gx^i = sum_j A^j' P^j c^j + pi^i q / 2
 *   orc_solve   -- Algorithm 3 (dual gradient x(y)) and, with homogeneous=1,
 *                  Algorithm 4 (Hessian-vector products: no c, no linear cost
 *                  terms, x^0 = 0):
 *                    backward  s^l = y^l/2 + pi^l p_N/2
 *                              v^i = y_u^i/2 + sum_j B^j' s^j + gu^i
 *                              ubar^i = -Rbar^{-1} v^i
 *                              s^i = y_x^i/2 + sum_j A^j' s^j + K^i' v^i + gx^i
 *                    forward   x^0 = p,  u^i = K^i x^i + ubar^i,
 *                              x^j = A^j x^i + B^j u^i + c^j  (eq. system_dynamics_tree)
 *                  Algorithm 3 writes "<-" in its child-sum loop where the
 *                  Hessian-vector version (Algorithm 4) accumulates; the
 *                  accumulating reading is used for both.
 *
 * Layout: node-major row-major FP64.  A [Nn][nx][nx], B [Nn][nx][nu],
 * c [Nn][nx] (row 0 unused), diagonal Q, R, P_N, vectors q, r, p_N.  The dual
 * vector y has one block per node: nonleaf i -> [x-part (nx); u-part (nu)] at
 * i*(nx+nu), leaf l -> [x-part (nx)] at Np*(nx+nu) + (l-Np)*nx.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int Nn, Np, N, nx, nu;
    const int *parent;      /* [Nn] */
    const int *cbeg, *ccnt; /* [Nn] children of i: cbeg[i] .. cbeg[i]+ccnt[i]-1 */
    const int *soff;        /* [N+2] first node of each stage, soff[N+1] = Nn */
    const double *prob;     /* [Nn] */
    const double *A, *B, *c;
    const double *Q, *R, *PN; /* diagonals */
    const double *q, *r, *pN;
} orc_problem;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Plain Cholesky: Rbar = L L', L lower triangular, row-major n x n. */
static int cholesky(int n, const double *Rb, double *L) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double d = Rb[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = Rb[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve (L L') x = b by forward then backward substitution. */
static void chol_solve(int n, const double *L, const double *b, double *x) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* Offline factor (Section III-D).  Outputs, all FP64:
 *   P  [Nn][nx][nx], K [Np][nu][nx], Lc [Np][nu][nu] (Cholesky factor of Rbar),
 *   gu [Np][nu], gx [Np][nx].  Returns 0, or -(i+1) if Rbar^i is not positive definite. */
int orc_factor(const orc_problem *p, double *P, double *K, double *Lc, double *gu, double *gx) {
    const int nx = p->nx, nu = p->nu;
    const size_t nxx = (size_t)nx * nx;
    int status = 0;
    /* leaves */
    for (int l = p->Np; l < p->Nn; ++l) {
        double *Pl = P + (size_t)l * nxx;
        memset(Pl, 0, sizeof(double) * nxx);
        for (int k = 0; k < nx; ++k) Pl[k * nx + k] = p->prob[l] * p->PN[k];
    }
    for (int t = p->N - 1; t >= 0; --t) {
        const int first = p->soff[t], last = p->soff[t + 1];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = first; i < last; ++i) {
            const double pi = p->prob[i];
            double *Rb = calloc((size_t)nu * nu, sizeof(double));
            double *M = calloc((size_t)nu * nx, sizeof(double));
            double *Nxx = calloc(nxx, sizeof(double));
            double *PA = malloc(sizeof(double) * nxx);
            double *PB = malloc(sizeof(double) * (size_t)nx * nu);
            double *Pc = malloc(sizeof(double) * nx);
            double *col = malloc(sizeof(double) * nu);
            double *sol = malloc(sizeof(double) * nu);
            double *gui = gu + (size_t)i * nu, *gxi = gx + (size_t)i * nx;
            for (int a = 0; a < nu; ++a) { Rb[a * nu + a] = pi * p->R[a]; gui[a] = 0.5 * pi * p->r[a]; }
            for (int a = 0; a < nx; ++a) { Nxx[a * nx + a] = pi * p->Q[a]; gxi[a] = 0.5 * pi * p->q[a]; }
            for (int j = p->cbeg[i]; j < p->cbeg[i] + p->ccnt[i]; ++j) {
                const double *Pj = P + (size_t)j * nxx;
                const double *Aj = p->A + (size_t)j * nxx;
                const double *Bj = p->B + (size_t)j * nx * nu;
                const double *cj = p->c + (size_t)j * nx;
                /* PA = P A, PB = P B, Pc = P c */
                for (int a = 0; a < nx; ++a) {
                    for (int b = 0; b < nx; ++b) {
                        double s = 0.0;
                        for (int k = 0; k < nx; ++k) s += Pj[a * nx + k] * Aj[k * nx + b];
                        PA[a * nx + b] = s;
                    }
                    for (int b = 0; b < nu; ++b) {
                        double s = 0.0;
                        for (int k = 0; k < nx; ++k) s += Pj[a * nx + k] * Bj[k * nu + b];
                        PB[a * nu + b] = s;
                    }
                    double s = 0.0;
                    for (int k = 0; k < nx; ++k) s += Pj[a * nx + k] * cj[k];
                    Pc[a] = s;
                }
                /* Rbar += B'PB, M += B'PA, gu += B'Pc */
                for (int a = 0; a < nu; ++a) {
                    for (int b = 0; b < nu; ++b) {
                        double s = 0.0;
                        for (int k = 0; k < nx; ++k) s += Bj[k * nu + a] * PB[k * nu + b];
                        Rb[a * nu + b] += s;
                    }
                    for (int b = 0; b < nx; ++b) {
                        double s = 0.0;
                        for (int k = 0; k < nx; ++k) s += Bj[k * nu + a] * PA[k * nx + b];
                        M[a * nx + b] += s;
                    }
                    double s = 0.0;
                    for (int k = 0; k < nx; ++k) s += Bj[k * nu + a] * Pc[k];
                    gui[a] += s;
                }
                /* N += A'PA, gx += A'Pc */
                for (int a = 0; a < nx; ++a) {
                    for (int b = 0; b < nx; ++b) {
                        double s = 0.0;
                        for (int k = 0; k < nx; ++k) s += Aj[k * nx + a] * PA[k * nx + b];
                        Nxx[a * nx + b] += s;
                    }
                    double s = 0.0;
                    for (int k = 0; k < nx; ++k) s += Aj[k * nx + a] * Pc[k];
                    gxi[a] += s;
                }
            }
            double *Li = Lc + (size_t)i * nu * nu;
            double *Ki = K + (size_t)i * nu * nx;
            if (cholesky(nu, Rb, Li) != 0) {
#pragma omp critical
                status = -(i + 1);
            } else {
                /* K = -Rbar^{-1} M, one column of M at a time */
                for (int b = 0; b < nx; ++b) {
                    for (int a = 0; a < nu; ++a) col[a] = M[a * nx + b];
                    chol_solve(nu, Li, col, sol);
                    for (int a = 0; a < nu; ++a) Ki[a * nx + b] = -sol[a];
                }
                /* P^i = pi Q + sum A'PA + M'K.  The exact P^i is symmetric; the stored
                 * one is symmetrised, since the antisymmetric part of the rounding error
                 * would otherwise be propagated by the open-loop A (and grow when
                 * rho(A) > 1) from stage to stage. */
                double *Pi = P + (size_t)i * nxx;
                for (int a = 0; a < nx; ++a)
                    for (int b = 0; b < nx; ++b) {
                        double s = Nxx[a * nx + b];
                        for (int k = 0; k < nu; ++k) s += M[k * nx + a] * Ki[k * nx + b];
                        Pi[a * nx + b] = s;
                    }
                for (int a = 0; a < nx; ++a)
                    for (int b = a + 1; b < nx; ++b) {
                        double s = 0.5 * (Pi[a * nx + b] + Pi[b * nx + a]);
                        Pi[a * nx + b] = s;
                        Pi[b * nx + a] = s;
                    }
            }
            free(Rb); free(M); free(Nxx); free(PA); free(PB); free(Pc); free(col); free(sol);
        }
        if (status != 0) return status;
    }
    return status;
}

static inline size_t dual_off(const orc_problem *p, int i) {
    return i < p->Np ? (size_t)i * (p->nx + p->nu)
                     : (size_t)p->Np * (p->nx + p->nu) + (size_t)(i - p->Np) * p->nx;
}

/* Algorithm 3 (homogeneous = 0) / Algorithm 4 (homogeneous = 1).
 * y: dual-sized, unscaled.  x0: [nx] (ignored when homogeneous).
 * Outputs x [Nn][nx] (x[0] = x0 or 0), u [Np][nu].  Work: s [Nn][nx], ubar [Np][nu]. */
int orc_solve(const orc_problem *p, const double *K, const double *Lc, const double *gu,
              const double *gx, const double *y, const double *x0, int homogeneous,
              double *x, double *u, double *s, double *ubar) {
    const int nx = p->nx, nu = p->nu;
    const size_t nxx = (size_t)nx * nx;
    for (int l = p->Np; l < p->Nn; ++l) {
        const double *yl = y + dual_off(p, l);
        for (int a = 0; a < nx; ++a)
            s[(size_t)l * nx + a] = 0.5 * yl[a] + (homogeneous ? 0.0 : 0.5 * p->prob[l] * p->pN[a]);
    }
    for (int t = p->N - 1; t >= 0; --t) {
        const int first = p->soff[t], last = p->soff[t + 1];
#pragma omp parallel for schedule(static)
        for (int i = first; i < last; ++i) {
            double *v = malloc(sizeof(double) * nu);
            const double *yi = y + dual_off(p, i);
            double *si = s + (size_t)i * nx;
            for (int a = 0; a < nu; ++a) v[a] = 0.5 * yi[nx + a] + (homogeneous ? 0.0 : gu[(size_t)i * nu + a]);
            for (int a = 0; a < nx; ++a) si[a] = 0.5 * yi[a] + (homogeneous ? 0.0 : gx[(size_t)i * nx + a]);
            for (int j = p->cbeg[i]; j < p->cbeg[i] + p->ccnt[i]; ++j) {
                const double *Aj = p->A + (size_t)j * nxx;
                const double *Bj = p->B + (size_t)j * nx * nu;
                const double *sj = s + (size_t)j * nx;
                for (int a = 0; a < nu; ++a) {
                    double acc = 0.0;
                    for (int k = 0; k < nx; ++k) acc += Bj[k * nu + a] * sj[k];
                    v[a] += acc;
                }
                for (int a = 0; a < nx; ++a) {
                    double acc = 0.0;
                    for (int k = 0; k < nx; ++k) acc += Aj[k * nx + a] * sj[k];
                    si[a] += acc;
                }
            }
            double *ub = ubar + (size_t)i * nu;
            chol_solve(nu, Lc + (size_t)i * nu * nu, v, ub);
            for (int a = 0; a < nu; ++a) ub[a] = -ub[a];
            const double *Ki = K + (size_t)i * nu * nx;
            for (int a = 0; a < nx; ++a) {
                double acc = 0.0;
                for (int k = 0; k < nu; ++k) acc += Ki[k * nx + a] * v[k];
                si[a] += acc;
            }
            free(v);
        }
    }
    for (int a = 0; a < nx; ++a) x[a] = homogeneous ? 0.0 : x0[a];
    for (int t = 0; t < p->N; ++t) {
        const int first = p->soff[t], last = p->soff[t + 1];
#pragma omp parallel for schedule(static)
        for (int i = first; i < last; ++i) {
            const double *xi = x + (size_t)i * nx;
            const double *Ki = K + (size_t)i * nu * nx;
            double *ui = u + (size_t)i * nu;
            for (int a = 0; a < nu; ++a) {
                double acc = ubar[(size_t)i * nu + a];
                for (int k = 0; k < nx; ++k) acc += Ki[a * nx + k] * xi[k];
                ui[a] = acc;
            }
            for (int j = p->cbeg[i]; j < p->cbeg[i] + p->ccnt[i]; ++j) {
                const double *Aj = p->A + (size_t)j * nxx;
                const double *Bj = p->B + (size_t)j * nx * nu;
                double *xj = x + (size_t)j * nx;
                for (int a = 0; a < nx; ++a) {
                    double acc = homogeneous ? 0.0 : p->c[(size_t)j * nx + a];
                    for (int k = 0; k < nx; ++k) acc += Aj[a * nx + k] * xi[k];
                    for (int k = 0; k < nu; ++k) acc += Bj[a * nu + k] * ui[k];
                    xj[a] = acc;
                }
            }
        }
    }
    return 0;
}
