// Offline factor of the scenario-tree LQ problem, FP64 on the device.
//
// Section III-D says the matrices of Algorithm 3 "are computed once offline following a
// Riccati-type recursion" and defers the formulas to earlier work.  They follow from
// dynamic programming on V^i(x) = x'P^i x + 2 s^i'x + const with the cost of Section II-B
// (no 1/2 factor).  For each stage t = N-1 .. 0 and each parent i of the stage, over its
// children j (Gc^j = [A^j | B^j | c^j] holds the dynamics of the edge i -> j):
//   W^j  = Gc^j' P^j Gc^j                                    (one batched GEMM pair per stage)
//   Rbar = pi^i R + sum_j W^j_BB,  M = sum_j W^j_BA,  N = pi^i Q + sum_j W^j_AA
//   gu   = pi^i r / 2 + sum_j W^j_Bc,  gx = pi^i q / 2 + sum_j W^j_Ac
//   Rbar = L L' (Cholesky, positive definiteness checked),  Rinv = L^-T L^-1
//   K^i  = -Rinv M,  P^i = N + M' K^i  (symmetrised: the antisymmetric part of the
//   rounding error would otherwise be carried along by the open-loop A from stage to stage)
// with P^l = pi^l P_N at the leaves.  The solve arrays (Algorithm 3/4) are then written in
// the handle's precision: G^j = [A^j | B^j], K^i, [-Rinv^i | K^i], gu^i, gx^i, c^j.
#include "internal.h"

namespace sto {
namespace {

constexpr int kT = 32;  // GEMM tile

// C_b = alpha op(A_b) B_b + beta C_b for b = blockIdx.z; op(A) = A (M x K) or A' (A is K x M).
template <bool TA>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double *A, int lda,
                                               long long sA, const double *B, int ldb, long long sB,
                                               double beta, double *C, int ldc, long long sC) {
    const long long b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    __shared__ double As[kT][kT + 1];
    __shared__ double Bs[kT][kT + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * kT, col0 = blockIdx.x * kT;
    double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;
    for (int k0 = 0; k0 < K; k0 += kT) {
        for (int e = threadIdx.x; e < kT * kT; e += 256) {
            int i, kk;
            if (TA) {  // consecutive threads walk the row index of op(A) = column of A
                kk = e / kT;
                i = e % kT;
            } else {
                i = e / kT;
                kk = e % kT;
            }
            const int r = row0 + i, k = k0 + kk;
            double v = 0.0;
            if (r < M && k < K) v = TA ? A[(size_t)k * lda + r] : A[(size_t)r * lda + k];
            As[i][kk] = v;
            const int kb = e / kT, j = e % kT;
            const int kr = k0 + kb, c = col0 + j;
            Bs[kb][j] = (kr < K && c < N) ? B[(size_t)kr * ldb + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kT; ++kk) {
            const double a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
            const double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            acc00 = fma(a0, b0, acc00);
            acc01 = fma(a0, b1, acc01);
            acc10 = fma(a1, b0, acc10);
            acc11 = fma(a1, b1, acc11);
        }
        __syncthreads();
    }
    const double acc[2][2] = {{acc00, acc01}, {acc10, acc11}};
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const int r = row0 + ty * 2 + di, c = col0 + tx * 2 + dj;
            if (r < M && c < N) {
                double *p = C + (size_t)r * ldc + c;
                *p = beta == 0.0 ? alpha * acc[di][dj] : alpha * acc[di][dj] + beta * *p;
            }
        }
}

void dgemm(cudaStream_t st, bool ta, int M, int N, int K, double alpha, const double *A, int lda, long long sA,
           const double *B, int ldb, long long sB, double beta, double *C, int ldc, long long sC, int batch) {
    if (batch <= 0) return;
    dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT, batch);
    if (ta)
        k_dgemm<true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
    else
        k_dgemm<false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
}

// P^l = pi^l diag(P_N) for the leaves (stage N), b = l - first.
__global__ void k_leaf_P(int first, int count, int nx, const double *prob, const double *PN, double *P) {
    const long long tot = (long long)count * nx * nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / ((long long)nx * nx);
        const int rc = (int)(e - b * nx * nx);
        const int r = rc / nx, c = rc % nx;
        P[e] = (r == c) ? prob[first + b] * PN[r] : 0.0;
    }
}

// Per parent i = first + blockIdx.x: sum the children's W^j into Rbar, M, N (into Pcur), gu, gx.
template <class T>
__global__ void k_assemble(int first, int child_first, int nx, int nu, int ld64, const int *cbeg, const int *ccnt,
                           const double *prob, const double *cost64, const double *W, double *Rb, double *M,
                           double *Pcur, T *gu, T *gx) {
    const int b = blockIdx.x, i = first + b;
    const double pi = prob[i];
    const double *Q = cost64, *R = cost64 + nx, *q = cost64 + 2 * nx + nu, *r = cost64 + 3 * nx + nu;
    const int j0 = cbeg[i] - child_first, nc = ccnt[i];
    const size_t wstride = (size_t)ld64 * ld64;
    const int cc = nx + nu;  // column of c in W
    double *Rbi = Rb + (size_t)b * nu * nu, *Mi = M + (size_t)b * nu * nx, *Ni = Pcur + (size_t)b * nx * nx;
    for (int e = threadIdx.x; e < nu * nu; e += blockDim.x) {
        const int a = e / nu, c = e % nu;
        double s = (a == c) ? pi * R[a] : 0.0;
        for (int k = 0; k < nc; ++k) s += W[(j0 + k) * wstride + (size_t)(nx + a) * ld64 + nx + c];
        Rbi[e] = s;
    }
    for (int e = threadIdx.x; e < nu * nx; e += blockDim.x) {
        const int a = e / nx, c = e % nx;
        double s = 0.0;
        for (int k = 0; k < nc; ++k) s += W[(j0 + k) * wstride + (size_t)(nx + a) * ld64 + c];
        Mi[e] = s;
    }
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
        const int a = e / nx, c = e % nx;
        double s = (a == c) ? pi * Q[a] : 0.0;
        for (int k = 0; k < nc; ++k) s += W[(j0 + k) * wstride + (size_t)a * ld64 + c];
        Ni[e] = s;
    }
    for (int a = threadIdx.x; a < nu; a += blockDim.x) {
        double s = 0.5 * pi * r[a];
        for (int k = 0; k < nc; ++k) s += W[(j0 + k) * wstride + (size_t)(nx + a) * ld64 + cc];
        gu[(size_t)i * nu + a] = (T)s;
    }
    for (int a = threadIdx.x; a < nx; a += blockDim.x) {
        double s = 0.5 * pi * q[a];
        for (int k = 0; k < nc; ++k) s += W[(j0 + k) * wstride + (size_t)a * ld64 + cc];
        gx[(size_t)i * nx + a] = (T)s;
    }
}

// Per parent: Cholesky Rbar = L L' in place, Z = L^-1, Rbar <- Rinv = Z'Z; -Rinv into the first ldr
// columns of the parent's RK block (rows of ldrk).
template <class T>
__global__ void k_chol_inv(int first, int nu, int ldr, int ldrk, double *Rb, double *Zb, T *RK, int *fstatus) {
    const int b = blockIdx.x, i = first + b;
    double *A = Rb + (size_t)b * nu * nu;
    double *Z = Zb + (size_t)b * nu * nu;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nu; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * nu + j];
            if (!(d > 0.0)) {
                bad = 1;
                A[j * nu + j] = 1.0;
            } else {
                A[j * nu + j] = sqrt(d);
            }
        }
        __syncthreads();
        const double ljj = A[j * nu + j];
        for (int r = j + 1 + threadIdx.x; r < nu; r += blockDim.x) A[r * nu + j] /= ljj;
        __syncthreads();
        const int rem = nu - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int r = j + 1 + e / rem, c = j + 1 + e % rem;
            if (c <= r) A[r * nu + c] -= A[r * nu + j] * A[c * nu + j];
        }
        __syncthreads();
    }
    if (bad && threadIdx.x == 0) atomicCAS(fstatus, 0, i + 1);
    // Z = L^-1 (lower triangular), one column per thread by forward substitution
    for (int c = threadIdx.x; c < nu; c += blockDim.x) {
        for (int r = 0; r < nu; ++r) {
            if (r < c) {
                Z[r * nu + c] = 0.0;
                continue;
            }
            double s = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s -= A[r * nu + k] * Z[k * nu + c];
            Z[r * nu + c] = s / A[r * nu + r];
        }
    }
    __syncthreads();
    // Rinv = Z'Z
    for (int e = threadIdx.x; e < nu * nu; e += blockDim.x) {
        const int a = e / nu, c = e % nu;
        const int k0 = a > c ? a : c;
        double s = 0.0;
        for (int k = k0; k < nu; ++k) s += Z[k * nu + a] * Z[k * nu + c];
        A[e] = s;  // safe: this row/column of L is no longer read (Z holds the inverse)
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nu * ldr; e += blockDim.x) {
        const int a = e / ldr, c = e % ldr;
        RK[(size_t)i * nu * ldrk + (size_t)a * ldrk + c] = c < nu ? (T)(-A[a * nu + c]) : (T)0;
    }
}

// Symmetrise P^i and write K^i in the solve precision: after -Rinv in the RK block (backward
// pass) and transposed (forward pass).
template <class T>
__global__ void k_finish(int first, int nx, int nu, int ldk, int ldr, int ldrk, double *Pcur, const double *K64,
                         T *RK, T *Kt) {
    const int b = blockIdx.x, i = first + b;
    double *P = Pcur + (size_t)b * nx * nx;
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
        const int r = e / nx, c = e % nx;
        if (c > r) {
            const double s = 0.5 * (P[r * nx + c] + P[c * nx + r]);
            P[r * nx + c] = s;
            P[c * nx + r] = s;
        }
    }
    const double *Kb = K64 + (size_t)b * nu * nx;
    for (int e = threadIdx.x; e < nu * ldk; e += blockDim.x) {
        const int a = e / ldk, c = e % ldk;
        const T val = c < nx ? (T)Kb[a * nx + c] : (T)0;
        RK[(size_t)i * nu * ldrk + (size_t)a * ldrk + ldr + c] = val;
    }
    for (int e = threadIdx.x; e < nx * ldr; e += blockDim.x) {
        const int r = e / ldr, a = e % ldr;
        Kt[(size_t)i * nx * ldr + e] = a < nu ? (T)Kb[a * nx + r] : (T)0;
    }
}

// Solve arrays of the dynamics: G^j = [A^j | B^j] (padded rows), its transpose G^j' (nx+nu rows
// of ldk) and c^j, in the solve precision.
template <class T>
__global__ void k_downcast_dyn(int Nn, int nx, int nu, int ld64, int ldg, int ldk, const double *G64, T *G, T *Gt,
                               T *c) {
    const long long rows = (long long)Nn * nx;
    for (long long rr = blockIdx.x; rr < rows; rr += gridDim.x) {
        const double *src = G64 + rr * ld64;
        T *dst = G + rr * ldg;
        for (int k = threadIdx.x; k < ldg; k += blockDim.x) dst[k] = k < nx + nu ? (T)src[k] : (T)0;
        if (threadIdx.x == 0) c[rr] = (T)src[nx + nu];
    }
    const long long trows = (long long)Nn * (nx + nu);
    for (long long tr = blockIdx.x; tr < trows; tr += gridDim.x) {
        const long long j = tr / (nx + nu);
        const int col = (int)(tr - j * (nx + nu));
        T *dst = Gt + tr * ldk;
        for (int r = threadIdx.x; r < ldk; r += blockDim.x)
            dst[r] = r < nx ? (T)G64[((size_t)j * nx + r) * ld64 + col] : (T)0;
    }
}

template <class T>
sto_status factor_impl(stotree_t h, cudaStream_t st) {
    const Layout &L = h->L;
    const int nx = h->nx, nu = h->nu, ld64 = h->ld64, N = h->N;
    const int nc64 = nx + nu + 1;  // columns of Gc
    double *G64 = h->at<double>(L.G64);
    STO_CUDA(h, cudaMemsetAsync(h->ws + L.fstatus, 0, 64, st));
    {
        const int first = h->soff[N], count = h->soff[N + 1] - first;
        k_leaf_P<<<std::min(4096, (count * nx * nx + 255) / 256), 256, 0, st>>>(
            first, count, nx, h->at<double>(L.prob64), h->at<double>(L.cost64) + nx + nu, h->at<double>(L.P[N & 1]));
    }
    for (int t = N - 1; t >= 0; --t) {
        const int pf = h->soff[t], np = h->soff[t + 1] - pf;
        const int cf = h->soff[t + 1], nchild = h->soff[t + 2] - cf;
        double *Pnext = h->at<double>(L.P[(t + 1) & 1]);
        double *Pcur = h->at<double>(L.P[t & 1]);
        double *PG = h->at<double>(L.PG), *W = h->at<double>(L.W);
        const double *Gc = G64 + (size_t)cf * nx * ld64;
        // PG^j = P^j Gc^j  (nx x nc64)
        dgemm(st, false, nx, nc64, nx, 1.0, Pnext, nx, (long long)nx * nx, Gc, ld64, (long long)nx * ld64, 0.0, PG,
              ld64, (long long)nx * ld64, nchild);
        // W^j = Gc^j' PG^j  (nc64 x nc64)
        dgemm(st, true, nc64, nc64, nx, 1.0, Gc, ld64, (long long)nx * ld64, PG, ld64, (long long)nx * ld64, 0.0, W,
              ld64, (long long)ld64 * ld64, nchild);
        k_assemble<T><<<np, 256, 0, st>>>(pf, cf, nx, nu, ld64, h->at<int>(L.cbeg), h->at<int>(L.ccnt),
                                          h->at<double>(L.prob64), h->at<double>(L.cost64), W,
                                          h->at<double>(L.Rb), h->at<double>(L.M), Pcur, h->at<T>(L.gu),
                                          h->at<T>(L.gx));
        k_chol_inv<T><<<np, 256, 0, st>>>(pf, nu, h->ldr, h->ldrk, h->at<double>(L.Rb), h->at<double>(L.Zb),
                                          h->at<T>(L.RK), h->at<int>(L.fstatus));
        // K = -Rinv M  (nu x nx)
        dgemm(st, false, nu, nx, nu, -1.0, h->at<double>(L.Rb), nu, (long long)nu * nu, h->at<double>(L.M), nx,
              (long long)nu * nx, 0.0, h->at<double>(L.K64), nx, (long long)nu * nx, np);
        // P = N + M'K  (nx x nx)
        dgemm(st, true, nx, nx, nu, 1.0, h->at<double>(L.M), nx, (long long)nu * nx, h->at<double>(L.K64), nx,
              (long long)nu * nx, 1.0, Pcur, nx, (long long)nx * nx, np);
        k_finish<T><<<np, 256, 0, st>>>(pf, nx, nu, h->ldk, h->ldr, h->ldrk, Pcur, h->at<double>(L.K64),
                                        h->at<T>(L.RK), h->at<T>(L.Kt));
    }
    const long long rows = (long long)h->Nn * nx;
    k_downcast_dyn<T><<<(int)std::min<long long>(rows, 65535), 128, 0, st>>>(
        h->Nn, nx, nu, ld64, h->ldg, h->ldk, G64, h->at<T>(L.G), h->at<T>(L.Gt), h->at<T>(L.c));
    STO_CUDA(h, cudaGetLastError());
    return STO_OK;
}

}  // namespace

sto_status factor_run(stotree_t h, cudaStream_t st) {
    return h->prec == STO_FP64 ? factor_impl<double>(h, st) : factor_impl<float>(h, st);
}

}  // namespace sto
