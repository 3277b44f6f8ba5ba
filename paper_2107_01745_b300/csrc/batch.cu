// Batched solves of many MPC instances: shape groups that share the tree, the dynamics (A, B),
// the costs and the box, and instances that differ in x0 and the disturbances c.
//
// With a shared (A, B, Q, R, P_N) and probabilities uniform within a stage (every node of stage t
// has b_t children), the factor of Section III-D collapses to one matrix set per stage: with
// P^j = pi_{t+1} P~_{t+1} for every node j of stage t+1,
//   Rbar^i = pi_t R~_t,  R~_t = R + B'P~_{t+1}B,  K_t = -R~_t^-1 B'P~_{t+1}A,
//   P~_t = Q + A'P~_{t+1}A + (B'P~_{t+1}A)'K_t,  P~_N = P_N,
// and the affine terms are gamma^i = pi_{t+1} [A | B]' P~_{t+1} sum_{j in child(i)} c^j.
// A solve round (Algorithm 3/4) then processes, stage by stage, all (node, instance) columns of
// all groups at once: per column a few products with the stage's matrices, which sit in shared
// memory and are reused by every column of a tile (a batched GEMM, FP32 on the CUDA cores).
// Stages are aligned across groups by height (backward) and depth (forward), one launch per
// aligned stage; the rounds of a solve are replayed from CUDA graphs.
//
// NAMA (Algorithm 2) runs per instance with the readings of the single-instance solver
// (solvers.cu): per-instance scalars, line search, L-BFGS memory and stopping test; the
// elementwise passes cover every active instance and reduce per instance (deterministically,
// block partials summed in block order by the instance's last block).  An instance that meets
// its tolerance stops updating and its columns are skipped by the solve rounds.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"

namespace sto {
namespace {

constexpr int kTC = 64;        // columns per solve tile
constexpr int kBT = 256;       // threads per block
constexpr int kChunkE = 2048;  // elements per block of the elementwise passes
constexpr int kMaxStages = 64;
constexpr int kBMaxMem = 8;    // L-BFGS memory of the batched solver

struct GroupDev {
    int nx, nu, N, b, s, Nn, Np, Nl, nxu, m, I, inst0;
    long long elem0;            // first element of the group's first instance in a batch vector
    long long sbase, ubase;     // first [Nn][nx] / [Np][nu] scratch entry of instance 0
    int soff[kMaxStages + 2];   // first node of each stage
    float pi[kMaxStages + 1];   // node probability of each stage
    float sq[kMaxStages + 1];   // its square root
    const float *G;             // [A | B]: nx rows of nx + nu
    const float *Kt;            // K_t: [N][nu][nx]
    const float *Ri;            // R~_t^-1: [N][nu][nu]
    const float *box;           // [lo x | lo u][hi x | hi u]
    const float *W;             // [Q | R | P_N]
    const float *sqn;           // sqrt(pi) per node
};

struct InstDev {
    int group, local;
    long long elem0;            // first element of this instance in a batch vector
    long long sbase, ubase;
    int m, nblocks, block0;     // elementwise blocks of this instance
    int pad;
};

struct BatchScalars {           // per instance (the single-instance SolverScalars, trimmed)
    double lambda, phi, res_inf, tau, gamma;
    double cand[kMaxCand];
    double SY[kBMaxMem + 1][kBMaxMem + 1], YY[kBMaxMem + 1][kBMaxMem + 1];
    double coef_s[kBMaxMem + 1], coef_y[kBMaxMem + 1];
    int active, iters, ls_done, ls_zero;
    int lb_count, lb_head, lb_pending_valid, lb_new_pair;
    int nan_flag;
    unsigned counter;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ long long doff(const GroupDev &g, int i) {
    return i < g.Np ? (long long)i * g.nxu : (long long)g.Np * g.nxu + (long long)(i - g.Np) * g.nx;
}

// ---------------------------------------------------------------------------------------------
// Solve rounds.  A task is a tile of up to kTC columns of one (group, stage); column c of a stage
// with n nodes is instance c / n, node soff_t + c % n.
// ---------------------------------------------------------------------------------------------
struct Task {
    int group, stage, col0, ncols;
};

template <int NR>
struct RoundArgs {
    const GroupDev *groups;
    const InstDev *insts;
    const Task *tasks;
    const float *y[2];
    float *h[2];
    const float *gam;     // gamma in the dual layout (x-part, u-part)
    const float *c;       // disturbances [instance][Nn][nx] (scratch layout of s)
    const float *x0;      // [instance][64]
    float *s, *ubar, *xs, *us;  // scratch; second right-hand side at +stride
    long long s_stride, u_stride;
    const int *active;    // per instance (null: all active)
    int homog, scaled;
};

constexpr int kMaxXU = 96;   // nx + nu <= 96 in the batched engine (nx <= 64)
constexpr int kTP = kTC + 4; // row stride of the column tiles in shared memory (16-byte aligned)
constexpr int kCG = kTC / 4; // column groups of 4 (one per thread of a row group)
constexpr int kRG = kBT / kCG;  // row groups
constexpr int kMR = (kMaxXU + kRG - 1) / kRG;  // output rows per thread, at most

// Stage products as register-blocked FP32 GEMMs: thread (rg, cg) owns up to kMR consecutive
// output rows and four columns of a tile, so each step of the inner dimension loads one float4 of
// the tile and kMR matrix entries for 4 kMR fused multiply-adds per right-hand side.
template <int NR>
constexpr size_t bwd_smem() {  // G [nx][nxu], K [nu][nx], R~^-1 [nu][nu], S [NR][64][kTP], V [NR][32][kTP]
    return sizeof(float) * (64 * kMaxXU + 32 * 64 + 32 * 32 + NR * 64 * kTP + NR * 32 * kTP);
}
template <int NR>
constexpr size_t fwd_smem() {  // G [nx][nxu], K [nu][nx], X [NR][kMaxXU][kTP]
    return sizeof(float) * (64 * kMaxXU + 32 * 64 + NR * kMaxXU * kTP);
}

// Columns of a task: instance data and node of each column, and whether its instance is active.
struct ColInfo {
    long long elem[kTC], sb[kTC], ub[kTC];
    int node[kTC], ok[kTC];
};
template <int NR>
__device__ __forceinline__ void load_cols(const RoundArgs<NR> &a, const GroupDev &g, const Task &tk, int n_t,
                                          ColInfo &ci) {
    if (threadIdx.x < kTC) {
        const int col = threadIdx.x;
        int ok = 0;
        if (col < tk.ncols) {
            const int cc = tk.col0 + col, inst = cc / n_t;
            const InstDev &in = a.insts[g.inst0 + inst];
            ci.elem[col] = in.elem0;
            ci.sb[col] = in.sbase;
            ci.ub[col] = in.ubase;
            ci.node[col] = g.soff[tk.stage] + cc % n_t;
            ok = !a.active || a.active[g.inst0 + inst];
        }
        ci.ok[col] = ok;
    }
}

// acc[q] += sum_u w_u x[u][q] for the four weights w of a 16-byte load and four column vectors.
__device__ __forceinline__ void fma4x4(const float4 w, const float4 *x, float *acc) {
    acc[0] = fmaf(w.x, x[0].x, acc[0]);
    acc[1] = fmaf(w.x, x[0].y, acc[1]);
    acc[2] = fmaf(w.x, x[0].z, acc[2]);
    acc[3] = fmaf(w.x, x[0].w, acc[3]);
    acc[0] = fmaf(w.y, x[1].x, acc[0]);
    acc[1] = fmaf(w.y, x[1].y, acc[1]);
    acc[2] = fmaf(w.y, x[1].z, acc[2]);
    acc[3] = fmaf(w.y, x[1].w, acc[3]);
    acc[0] = fmaf(w.z, x[2].x, acc[0]);
    acc[1] = fmaf(w.z, x[2].y, acc[1]);
    acc[2] = fmaf(w.z, x[2].z, acc[2]);
    acc[3] = fmaf(w.z, x[2].w, acc[3]);
    acc[0] = fmaf(w.w, x[3].x, acc[0]);
    acc[1] = fmaf(w.w, x[3].y, acc[1]);
    acc[2] = fmaf(w.w, x[3].z, acc[2]);
    acc[3] = fmaf(w.w, x[3].w, acc[3]);
}

// e = (k * kTC + col) * R + r over [threadIdx.x, NR * kTC * R) in steps of kBT, r fastest (so that
// a warp's global accesses to a column's R consecutive reals coalesce), with the (k, col, r)
// of each step advanced from the previous one instead of divided out per element.
template <int NR, class F>
__device__ __forceinline__ void for_kcr(int R, F f) {
    const int tot = NR * kTC * R;
    int e = threadIdx.x;
    int kc = e / R, r = e - kc * R;
    const int dq = kBT / R, dr = kBT - dq * R;
    for (; e < tot; e += kBT) {
        f(kc / kTC, kc % kTC, r);
        r += dr;
        kc += dq;
        if (r >= R) {
            r -= R;
            ++kc;
        }
    }
}

// Backward: parents of stage t.  S = sum_children s, o = [A | B]' S, v = y_u/2 + o_B + gu,
// ubar = -(1/pi_t) R~^-1 v, s = y_x/2 + o_A + K_t' v + gx.
template <int NR>
__global__ void __launch_bounds__(kBT) k_bbwd(RoundArgs<NR> a, int task0) {
    const Task tk = a.tasks[task0 + blockIdx.x];
    const GroupDev &g = a.groups[tk.group];
    const int nx = g.nx, nu = g.nu, nxu = g.nxu, t = tk.stage;
    extern __shared__ __align__(16) float bsm[];
    __shared__ ColInfo ci;
    float *Gs = bsm;                 // [r][c], r < nx, c < nx + nu
    float *Ks = Gs + 64 * kMaxXU;    // K_t [a][c]
    float *Rs = Ks + 32 * 64;        // R~_t^-1 [a][b]
    float *S = Rs + 32 * 32;         // [k][r][col]; afterwards s (without y_x/2 + gx)
    float *V = S + NR * 64 * kTP;    // [k][a][col]: v; afterwards ubar
    const int n_t = g.soff[t + 1] - g.soff[t];
    const int bt = t < g.s ? g.b : 1;
    const bool leaf_children = t + 1 == g.N;
    load_cols(a, g, tk, n_t, ci);
    // a tile whose instances have all converged writes nothing: leave it (before its matrices
    // are staged; the barrier after the gather below orders their stores before any use)
    if (!__syncthreads_or(threadIdx.x < kTC ? ci.ok[threadIdx.x] : 0)) return;
    for (int e = threadIdx.x; e < nx * nxu; e += kBT) Gs[e] = g.G[e];
    for (int e = threadIdx.x; e < nu * nx; e += kBT) Ks[e] = g.Kt[(size_t)t * nu * nx + e];
    for (int e = threadIdx.x; e < nu * nu; e += kBT) Rs[e] = g.Ri[(size_t)t * nu * nu + e];
    // S[k][r][col] = sum over the children of the column's node
    for_kcr<NR>(nx, [&](int k, int col, int r) {
        float acc = 0.f;
        if (ci.ok[col]) {
            const int i = ci.node[col];
            const int j0 = g.soff[t + 1] + (i - g.soff[t]) * bt;
            for (int j = j0; j < j0 + bt; ++j) {
                if (leaf_children) {
                    const float sc = a.scaled ? g.sq[t + 1] : 1.f;
                    acc += 0.5f * sc * a.y[k][ci.elem[col] + doff(g, j) + r];
                } else {
                    acc += a.s[k * a.s_stride + ci.sb[col] + (long long)j * nx + r];
                }
            }
        }
        S[(k * 64 + r) * kTP + col] = acc;
    });
    __syncthreads();
    const int cg = threadIdx.x % kCG, rg = threadIdx.x / kCG;
    const int mr = (nxu + kRG - 1) / kRG, r0 = rg * mr;
    float acc[NR][kMR][4];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int m = 0; m < kMR; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][m][q] = 0.f;
    // o = [A | B]' S
    for (int r = 0; r < nx; ++r) {
        float4 s4[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) s4[k] = *reinterpret_cast<const float4 *>(S + (k * 64 + r) * kTP + cg * 4);
#pragma unroll
        for (int m = 0; m < kMR; ++m)
            if (m < mr && r0 + m < nxu) {
                const float gv = Gs[r * nxu + r0 + m];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    acc[k][m][0] = fmaf(gv, s4[k].x, acc[k][m][0]);
                    acc[k][m][1] = fmaf(gv, s4[k].y, acc[k][m][1]);
                    acc[k][m][2] = fmaf(gv, s4[k].z, acc[k][m][2]);
                    acc[k][m][3] = fmaf(gv, s4[k].w, acc[k][m][3]);
                }
            }
    }
    // o_B rows -> V; then v = o_B + y_u/2 + gu
#pragma unroll
    for (int m = 0; m < kMR; ++m) {
        const int c = r0 + m;
        if (m < mr && c >= nx && c < nxu)
#pragma unroll
            for (int k = 0; k < NR; ++k)
                *reinterpret_cast<float4 *>(V + (k * 32 + c - nx) * kTP + cg * 4) =
                    make_float4(acc[k][m][0], acc[k][m][1], acc[k][m][2], acc[k][m][3]);
    }
    __syncthreads();
    {
        const float sc = a.scaled ? g.sq[t] : 1.f;
        for_kcr<NR>(nu, [&](int k, int col, int aa) {
            if (ci.ok[col]) {
                const long long o = ci.elem[col] + doff(g, ci.node[col]) + nx + aa;
                V[(k * 32 + aa) * kTP + col] += 0.5f * sc * a.y[k][o] + (a.homog ? 0.f : a.gam[o]);
            }
        });
    }
    __syncthreads();
    // rows c < nx: s = o_A + K' v; rows c = nx + a: ubar = -(1/pi_t) R~^-1 v
#pragma unroll
    for (int m = 0; m < kMR; ++m)
        if (r0 + m >= nx)
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[k][m][q] = 0.f;
    for (int aa = 0; aa < nu; ++aa) {
        float4 v4[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) v4[k] = *reinterpret_cast<const float4 *>(V + (k * 32 + aa) * kTP + cg * 4);
#pragma unroll
        for (int m = 0; m < kMR; ++m) {
            const int c = r0 + m;
            if (m < mr && c < nxu) {
                const float cf = c < nx ? Ks[aa * nx + c] : Rs[(c - nx) * nu + aa];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    acc[k][m][0] = fmaf(cf, v4[k].x, acc[k][m][0]);
                    acc[k][m][1] = fmaf(cf, v4[k].y, acc[k][m][1]);
                    acc[k][m][2] = fmaf(cf, v4[k].z, acc[k][m][2]);
                    acc[k][m][3] = fmaf(cf, v4[k].w, acc[k][m][3]);
                }
            }
        }
    }
    __syncthreads();  // every thread is done with S and V
    const float ipi = 1.f / g.pi[t];
#pragma unroll
    for (int m = 0; m < kMR; ++m) {
        const int c = r0 + m;
        if (m < mr && c < nxu)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float *dst = c < nx ? S + (k * 64 + c) * kTP + cg * 4 : V + (k * 32 + c - nx) * kTP + cg * 4;
                const float f = c < nx ? 1.f : -ipi;
                *reinterpret_cast<float4 *>(dst) =
                    make_float4(f * acc[k][m][0], f * acc[k][m][1], f * acc[k][m][2], f * acc[k][m][3]);
            }
    }
    __syncthreads();
    // coalesced write-out: ubar, and s = y_x/2 + (o_A + K'v) + gx
    for_kcr<NR>(nu, [&](int k, int col, int aa) {
        if (ci.ok[col])
            a.ubar[k * a.u_stride + ci.ub[col] + (long long)ci.node[col] * nu + aa] = V[(k * 32 + aa) * kTP + col];
    });
    {
        const float sc = a.scaled ? g.sq[t] : 1.f;
        for_kcr<NR>(nx, [&](int k, int col, int r) {
            if (ci.ok[col]) {
                const int i = ci.node[col];
                const long long o = ci.elem[col] + doff(g, i) + r;
                a.s[k * a.s_stride + ci.sb[col] + (long long)i * nx + r] =
                    S[(k * 64 + r) * kTP + col] + 0.5f * sc * a.y[k][o] + (a.homog ? 0.f : a.gam[o]);
            }
        });
    }
}

// Forward: nodes of stage t.  x from the parent's pass (or x0 at the root); u = K x + ubar;
// h = S [x; u]; every child j gets x^j = A x + B u + c^j.  Leaves (t = N) only write h.
template <int NR>
__global__ void __launch_bounds__(kBT) k_bfwd(RoundArgs<NR> a, int task0) {
    const Task tk = a.tasks[task0 + blockIdx.x];
    const GroupDev &g = a.groups[tk.group];
    const int nx = g.nx, nu = g.nu, nxu = g.nxu, t = tk.stage;
    extern __shared__ __align__(16) float bsm[];
    __shared__ ColInfo ci;
    float *Gs = bsm;
    float *Ks = Gs + 64 * kMaxXU;
    float *X = Ks + 32 * 64;  // [k][row][col]: x then u per column
    const bool leaf = t == g.N;
    const int n_t = g.soff[t + 1] - g.soff[t];
    load_cols(a, g, tk, n_t, ci);
    // a tile whose instances have all converged writes nothing: leave it (before its matrices
    // are staged; the barrier after the gather below orders their stores before any use)
    if (!__syncthreads_or(threadIdx.x < kTC ? ci.ok[threadIdx.x] : 0)) return;
    for (int e = threadIdx.x; e < nx * nxu; e += kBT) Gs[e] = g.G[e];
    if (!leaf)
        for (int e = threadIdx.x; e < nu * nx; e += kBT) Ks[e] = g.Kt[(size_t)t * nu * nx + e];
    for_kcr<NR>(nx, [&](int k, int col, int r) {
        float val = 0.f;
        if (ci.ok[col]) {
            if (t == 0) {
                const int inst = (tk.col0 + col) / n_t;
                val = a.homog ? 0.f : a.x0[(long long)(g.inst0 + inst) * 64 + r];
            } else {
                val = a.xs[k * a.s_stride + ci.sb[col] + (long long)ci.node[col] * nx + r];
            }
        }
        X[(k * kMaxXU + r) * kTP + col] = val;
    });
    __syncthreads();
    const int cg = threadIdx.x % kCG, rg = threadIdx.x / kCG;
    const float sc = a.scaled ? g.sq[t] : 1.f;
    if (!leaf) {
        // u = K x (rows a of u over the row groups), then + ubar
        const int mu = (nu + kRG - 1) / kRG, a0 = rg * mu;
        constexpr int kMU = (32 + kRG - 1) / kRG;
        float u[NR][kMU][4];
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int m = 0; m < kMU; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) u[k][m][q] = 0.f;
        for (int r = 0; r < nx; ++r) {
            float4 x4[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k)
                x4[k] = *reinterpret_cast<const float4 *>(X + (k * kMaxXU + r) * kTP + cg * 4);
#pragma unroll
            for (int m = 0; m < kMU; ++m)
                if (m < mu && a0 + m < nu) {
                    const float kv = Ks[(a0 + m) * nx + r];
#pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        u[k][m][0] = fmaf(kv, x4[k].x, u[k][m][0]);
                        u[k][m][1] = fmaf(kv, x4[k].y, u[k][m][1]);
                        u[k][m][2] = fmaf(kv, x4[k].z, u[k][m][2]);
                        u[k][m][3] = fmaf(kv, x4[k].w, u[k][m][3]);
                    }
                }
        }
#pragma unroll
        for (int m = 0; m < kMU; ++m)
            if (m < mu && a0 + m < nu)
#pragma unroll
                for (int k = 0; k < NR; ++k)
                    *reinterpret_cast<float4 *>(X + (k * kMaxXU + nx + a0 + m) * kTP + cg * 4) =
                        make_float4(u[k][m][0], u[k][m][1], u[k][m][2], u[k][m][3]);
        __syncthreads();
        for_kcr<NR>(nu, [&](int k, int col, int aa) {
            if (ci.ok[col])
                X[(k * kMaxXU + nx + aa) * kTP + col] +=
                    a.ubar[k * a.u_stride + ci.ub[col] + (long long)ci.node[col] * nu + aa];
        });
        __syncthreads();
    }
    // h for the stage's nodes, primal scratch
    const int rows = leaf ? nx : nxu;
    for_kcr<NR>(rows, [&](int k, int col, int r) {
        if (ci.ok[col]) {
            const int i = ci.node[col];
            const float val = X[(k * kMaxXU + r) * kTP + col];
            a.h[k][ci.elem[col] + doff(g, i) + r] = sc * val;
            if (r < nx)
                a.xs[k * a.s_stride + ci.sb[col] + (long long)i * nx + r] = val;
            else
                a.us[k * a.u_stride + ci.ub[col] + (long long)i * nu + r - nx] = val;
        }
    });
    if (leaf) return;
    // children: x^j = [A | B][x; u] + c^j (rows r of x over the row groups)
    const int mx = (nx + kRG - 1) / kRG, x0r = rg * mx;
    constexpr int kMX = (64 + kRG - 1) / kRG;
    float acc[NR][kMX][4];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int m = 0; m < kMX; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][m][q] = 0.f;
    int qq = 0;
    if ((nxu & 3) == 0) {
        // four inputs per step: one 16-byte load of each G row, four of the column tile
        for (; qq + 4 <= nxu; qq += 4) {
            float4 x4[NR][4];
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    x4[k][u] = *reinterpret_cast<const float4 *>(X + (k * kMaxXU + qq + u) * kTP + cg * 4);
#pragma unroll
            for (int m = 0; m < kMX; ++m)
                if (m < mx && x0r + m < nx) {
                    const float4 g4 = *reinterpret_cast<const float4 *>(Gs + (x0r + m) * nxu + qq);
#pragma unroll
                    for (int k = 0; k < NR; ++k) fma4x4(g4, x4[k], acc[k][m]);
                }
        }
    }
    for (; qq < nxu; ++qq) {
        float4 x4[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) x4[k] = *reinterpret_cast<const float4 *>(X + (k * kMaxXU + qq) * kTP + cg * 4);
#pragma unroll
        for (int m = 0; m < kMX; ++m)
            if (m < mx && x0r + m < nx) {
                const float gv = Gs[(x0r + m) * nxu + qq];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    acc[k][m][0] = fmaf(gv, x4[k].x, acc[k][m][0]);
                    acc[k][m][1] = fmaf(gv, x4[k].y, acc[k][m][1]);
                    acc[k][m][2] = fmaf(gv, x4[k].z, acc[k][m][2]);
                    acc[k][m][3] = fmaf(gv, x4[k].w, acc[k][m][3]);
                }
            }
    }
    __syncthreads();  // every thread is done with X
#pragma unroll
    for (int m = 0; m < kMX; ++m)
        if (m < mx && x0r + m < nx)
#pragma unroll
            for (int k = 0; k < NR; ++k)
                *reinterpret_cast<float4 *>(X + (k * kMaxXU + x0r + m) * kTP + cg * 4) =
                    make_float4(acc[k][m][0], acc[k][m][1], acc[k][m][2], acc[k][m][3]);
    __syncthreads();
    const int bt = t < g.s ? g.b : 1;
    for_kcr<NR>(nx, [&](int k, int col, int r) {
        if (ci.ok[col]) {
            const int i = ci.node[col];
            const int j0 = g.soff[t + 1] + (i - g.soff[t]) * bt;
            const float xv = X[(k * kMaxXU + r) * kTP + col];
            for (int j = j0; j < j0 + bt; ++j) {
                const float cj = a.homog ? 0.f : a.c[ci.sb[col] + (long long)j * nx + r];
                a.xs[k * a.s_stride + ci.sb[col] + (long long)j * nx + r] = xv + cj;
            }
        }
    });
}

// gamma^i = pi_{t+1} [A | B]' P~_{t+1} sum_j c^j for every nonleaf node and instance (set-up).
__global__ void k_bgamma(const GroupDev *groups, const InstDev *insts, const Task *tasks, int task0,
                         const double *Pt /*per group [N+1][nx][nx] at ptoff*/, const long long *ptoff,
                         const float *c, float *gam) {
    const Task tk = tasks[task0 + blockIdx.x];
    const GroupDev &g = groups[tk.group];
    const int nx = g.nx, nxu = g.nxu, t = tk.stage;
    const int n_t = g.soff[t + 1] - g.soff[t];
    const int bt = t < g.s ? g.b : 1;
    const double *P = Pt + ptoff[tk.group] + (size_t)(t + 1) * nx * nx;
    constexpr int kGH = 32;  // columns per pass (FP64 tiles within the static shared-memory limit)
    __shared__ double cs[64][kGH];
    __shared__ double w[64][kGH];
    const double pnext = g.pi[t + 1];
    for (int h0 = 0; h0 < tk.ncols; h0 += kGH) {
        const int nc = min(kGH, tk.ncols - h0);
        for (int e = threadIdx.x; e < nx * kGH; e += blockDim.x) {
            const int col = e / nx, r = e % nx;
            double acc = 0.0;
            if (col < nc) {
                const int cc = tk.col0 + h0 + col, inst = cc / n_t, i = g.soff[t] + cc % n_t;
                const InstDev &in = insts[g.inst0 + inst];
                const int j0 = g.soff[t + 1] + (i - g.soff[t]) * bt;
                for (int j = j0; j < j0 + bt; ++j) acc += (double)c[in.sbase + (long long)j * nx + r];
            }
            cs[r][col] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nx * kGH; e += blockDim.x) {
            const int col = e / nx, r = e % nx;
            double acc = 0.0;
            for (int k = 0; k < nx; ++k) acc += P[r * nx + k] * cs[k][col];
            w[r][col] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nxu * kGH; e += blockDim.x) {
            const int col = e / nxu, cidx = e % nxu;
            if (col >= nc) continue;
            const int cc = tk.col0 + h0 + col, inst = cc / n_t, i = g.soff[t] + cc % n_t;
            const InstDev &in = insts[g.inst0 + inst];
            double acc = 0.0;
            for (int r = 0; r < nx; ++r) acc += (double)g.G[r * nxu + cidx] * w[r][col];
            gam[in.elem0 + doff(g, i) + cidx] = (float)(pnext * acc);
        }
        __syncthreads();
    }
}

// FP64 stage factor, one block per group (sequential over stages): P~_N = P_N,
// R~_t = R + B'P~B, K_t = -R~^-1 B'P~A, P~_t = Q + A'P~A + (B'P~A)'K_t (symmetrised).
__global__ void k_bfactor(const GroupDev *groups, const double *AB64 /*per group [nx][nx+nu]*/,
                          const long long *aboff, double *Pt, const long long *ptoff, double *scratch,
                          const long long *scoff, int *status) {
    const GroupDev &g = groups[blockIdx.x];
    const int nx = g.nx, nu = g.nu, nxu = g.nxu, N = g.N;
    const double *AB = AB64 + aboff[blockIdx.x];
    double *P = Pt + ptoff[blockIdx.x];
    double *PA = scratch + scoff[blockIdx.x];       // P~ [A | B]: nx x nxu
    double *Rb = PA + nx * nxu;                      // nu x nu
    double *Mb = Rb + nu * nu;                       // nu x nx  (B'P~A)
    double *L = Mb + nu * nx;                        // nu x nu
    double *Z = L + nu * nu;                         // nu x nu
    double *Kd = Z + nu * nu;                        // nu x nx
    // P~_N = diag(P_N)
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
        const int r = e / nx, c = e % nx;
        P[(size_t)N * nx * nx + e] = r == c ? (double)g.W[nx + nu + r] : 0.0;
    }
    __syncthreads();
    for (int t = N - 1; t >= 0; --t) {
        const double *Pn = P + (size_t)(t + 1) * nx * nx;
        double *Pc = P + (size_t)t * nx * nx;
        for (int e = threadIdx.x; e < nx * nxu; e += blockDim.x) {
            const int r = e / nxu, c = e % nxu;
            double acc = 0.0;
            for (int k = 0; k < nx; ++k) acc += Pn[r * nx + k] * AB[k * nxu + c];
            PA[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nu * nu; e += blockDim.x) {
            const int aa = e / nu, bb = e % nu;
            double acc = aa == bb ? (double)g.W[nx + aa] : 0.0;
            for (int k = 0; k < nx; ++k) acc += AB[k * nxu + nx + aa] * PA[k * nxu + nx + bb];
            Rb[e] = acc;
        }
        for (int e = threadIdx.x; e < nu * nx; e += blockDim.x) {
            const int aa = e / nx, c = e % nx;
            double acc = 0.0;
            for (int k = 0; k < nx; ++k) acc += AB[k * nxu + nx + aa] * PA[k * nxu + c];
            Mb[e] = acc;
        }
        __syncthreads();
        // Cholesky of R~ (one thread: nu <= 32) and its inverse
        if (threadIdx.x == 0) {
            for (int j = 0; j < nu; ++j) {
                double d = Rb[j * nu + j];
                for (int k = 0; k < j; ++k) d -= L[j * nu + k] * L[j * nu + k];
                if (!(d > 0.0)) {
                    atomicCAS(status, 0, blockIdx.x + 1);
                    d = 1.0;
                }
                L[j * nu + j] = sqrt(d);
                for (int i = j + 1; i < nu; ++i) {
                    double s = Rb[i * nu + j];
                    for (int k = 0; k < j; ++k) s -= L[i * nu + k] * L[j * nu + k];
                    L[i * nu + j] = s / L[j * nu + j];
                }
                for (int i = 0; i < j; ++i) L[i * nu + j] = 0.0;
            }
            for (int c = 0; c < nu; ++c)
                for (int r = 0; r < nu; ++r) {
                    if (r < c) {
                        Z[r * nu + c] = 0.0;
                        continue;
                    }
                    double s = r == c ? 1.0 : 0.0;
                    for (int k = c; k < r; ++k) s -= L[r * nu + k] * Z[k * nu + c];
                    Z[r * nu + c] = s / L[r * nu + r];
                }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nu * nu; e += blockDim.x) {  // R~^-1 = Z'Z
            const int aa = e / nu, bb = e % nu;
            double acc = 0.0;
            for (int k = (aa > bb ? aa : bb); k < nu; ++k) acc += Z[k * nu + aa] * Z[k * nu + bb];
            Rb[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nu * nx; e += blockDim.x) {  // K = -R~^-1 M
            const int aa = e / nx, c = e % nx;
            double acc = 0.0;
            for (int k = 0; k < nu; ++k) acc += Rb[aa * nu + k] * Mb[k * nx + c];
            Kd[e] = -acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {  // P~ = Q + A'P~A + M'K
            const int r = e / nx, c = e % nx;
            double acc = r == c ? (double)g.W[r] : 0.0;
            for (int k = 0; k < nx; ++k) acc += AB[k * nxu + r] * PA[k * nxu + c];
            for (int k = 0; k < nu; ++k) acc += Mb[k * nx + r] * Kd[k * nx + c];
            Pc[e] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
            const int r = e / nx, c = e % nx;
            if (c > r) {
                const double s = 0.5 * (Pc[r * nx + c] + Pc[c * nx + r]);
                Pc[r * nx + c] = s;
                Pc[c * nx + r] = s;
            }
        }
        float *Kout = const_cast<float *>(g.Kt) + (size_t)t * nu * nx;
        float *Rout = const_cast<float *>(g.Ri) + (size_t)t * nu * nu;
        for (int e = threadIdx.x; e < nu * nx; e += blockDim.x) Kout[e] = (float)Kd[e];
        for (int e = threadIdx.x; e < nu * nu; e += blockDim.x) Rout[e] = (float)Rb[e];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Elementwise passes with per-instance reductions.  Block b covers elements
// [chunk * kChunkE, ...) of instance blk_inst[b].
// ---------------------------------------------------------------------------------------------
struct ElemArgs {
    const GroupDev *groups;
    const InstDev *insts;
    const int *blk_inst;
    BatchScalars *sc;
    double *partials;     // [block][kRedSlots]
    long long vstride;    // batch vector length (padded)
    int mem;
    double tol, eps_curv;
};

struct EMeta {
    float sq, lo, hi, w;
};
__device__ __forceinline__ EMeta emeta(const GroupDev &g, int e) {
    int node, comp, kind;
    if (e < g.Np * g.nxu) {
        node = e / g.nxu;
        const int k = e - node * g.nxu;
        kind = k < g.nx ? 0 : 1;
        comp = k < g.nx ? k : k - g.nx;
    } else {
        const int e2 = e - g.Np * g.nxu;
        node = g.Np + e2 / g.nx;
        comp = e2 - (node - g.Np) * g.nx;
        kind = 2;
    }
    EMeta M;
    M.sq = g.sqn[node];
    const int bi = kind == 1 ? g.nx + comp : comp;
    const int wi = kind == 0 ? comp : (kind == 1 ? g.nx + comp : g.nx + g.nu + comp);
    if (node == 0 && kind == 0) {
        M.lo = -INFINITY;
        M.hi = INFINITY;
    } else {
        M.lo = M.sq * g.box[bi];
        M.hi = M.sq * g.box[g.nxu + bi];
    }
    M.w = g.W[wi];
    return M;
}
__device__ __forceinline__ float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }
__device__ __forceinline__ float term(float h, float w, float lam, float ilam, const EMeta &M) {
    const float z = clampf(h + w * ilam, M.lo, M.hi);
    const float dz = h - z;
    return h * (M.w * h) + dz * (w + 0.5f * lam * dz);
}

__device__ __forceinline__ float wsumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float wmaxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Per-instance reduction of NS sums and NM maxima; true in the instance's last block.  Warp
// and block levels in FP32 (the FP64 pipe is slow on this part), block partials and the sum
// over the instance's blocks in FP64.
template <int NS, int NM>
__device__ bool inst_reduce(const ElemArgs &a, int inst, float *sums, float *maxs, double *out) {
    constexpr int NV = NS + NM;
    __shared__ float red[kBT / 32][NV > 0 ? NV : 1];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NS; ++k) sums[k] = wsumf(sums[k]);
#pragma unroll
    for (int k = 0; k < NM; ++k) maxs[k] = wmaxf(maxs[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) red[warp][k] = sums[k];
#pragma unroll
        for (int k = 0; k < NM; ++k) red[warp][NS + k] = maxs[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        float acc = k < NS ? 0.f : -INFINITY;
        for (int w = 0; w < kBT / 32; ++w) acc = k < NS ? acc + red[w][k] : fmaxf(acc, red[w][k]);
        a.partials[(size_t)k * gridDim.x + blockIdx.x] = (double)acc;  // slot-major: coalesced in the tail
        __threadfence();  // only the writers of partials publish anything
    }
    __syncthreads();
    const InstDev &in = a.insts[inst];
    if (threadIdx.x == 0) last = atomicAdd(&a.sc[inst].counter, 1u) == (unsigned)in.nblocks - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int k = warp; k < NV; k += kBT / 32) {
        const double ident = k < NS ? 0.0 : -INFINITY;
        const double *src = a.partials + (size_t)k * gridDim.x + in.block0;
        double acc = ident;
        for (int b0 = lane; b0 < in.nblocks; b0 += 32 * 4) {  // four loads in flight, summed in order
            double v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = b0 + 32 * q < in.nblocks ? __ldcg(src + b0 + 32 * q) : ident;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc = k < NS ? acc + v[q] : fmax(acc, v[q]);
        }
        acc = k < NS ? wsum(acc) : wmax(acc);
        if (lane == 0) out[k] = acc;
    }
    if (threadIdx.x == 0) a.sc[inst].counter = 0u;
    __syncthreads();
    return true;
}

#define BLOCK_PROLOGUE                                                   \
    const int inst = a.blk_inst[blockIdx.x];                             \
    const InstDev &in = a.insts[inst];                                   \
    BatchScalars &S = a.sc[inst];                                        \
    if (!S.active) return;                                               \
    const GroupDev &g = a.groups[in.group];                              \
    const int chunk = blockIdx.x - in.block0;                            \
    const int e0 = chunk * kChunkE, e1 = min(in.m, e0 + kChunkE);        \
    const long long base = in.elem0;                                     \
    (void)g;

// residual, FBE, stop test; with pair = 1 the NAMA L-BFGS pair q = r_new - r_old
__global__ void __launch_bounds__(kBT) k_bpoint(ElemArgs a, const float *yb, const float *h, float *r, float *ringS,
                                                float *ringY, int pair) {
    BLOCK_PROLOGUE
    __shared__ double tot[8];
    const float lam = (float)S.lambda, ilam = 1.f / lam;
    const int p = (S.lb_head + S.lb_count) % (a.mem + 1);
    float fs = 0.f, sq = 0.f, s2 = 0.f, g2 = 0.f, mx = 0.f;
    int nan = 0;
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const EMeta M = emeta(g, e);
        const long long ge = base + e;
        const float he = h[ge], ye = yb[ge];
        const float z = clampf(he + ye * ilam, M.lo, M.hi);
        const float re = z - he;
        fs += term(he, ye, lam, ilam, M);
        const float ra = fabsf(re) / M.sq;
        if (!(ra <= 3.0e38f)) nan = 1;
        mx = fmaxf(mx, ra);
        if (pair) {
            const float ro = r[ge], q = re - ro, s = ringS[p * a.vstride + ge];
            ringY[p * a.vstride + ge] = q;
            sq += s * q;
            s2 += s * s;
            g2 += ro * ro;
        }
        r[ge] = re;
    }
    float sums[5] = {fs, sq, s2, g2, (float)nan};
    float maxs[1] = {mx};
    if (inst_reduce<5, 1>(a, inst, sums, maxs, tot) && threadIdx.x == 0) {
        S.phi = -tot[0];
        S.res_inf = tot[5];
        if (tot[4] > 0.0 || !(tot[0] == tot[0])) S.nan_flag = 1;
        if (pair && S.lb_pending_valid) {
            if (tot[1] > a.eps_curv * tot[2] * tot[3]) {
                if (S.lb_count < a.mem)
                    S.lb_count += 1;
                else
                    S.lb_head = (S.lb_head + 1) % (a.mem + 1);
                S.lb_new_pair = 1;
            }
            S.lb_pending_valid = 0;
        }
    }
}

template <int MEM>
__global__ void __launch_bounds__(kBT) k_blb_dots(ElemArgs a, const float *gv, const float *ringS, const float *ringY) {
    BLOCK_PROLOGUE
    __shared__ double tot[4 * MEM];
    const int cnt = S.lb_count, head = S.lb_head, M1 = a.mem + 1, newp = S.lb_new_pair;
    if (cnt == 0) {
        if (chunk == 0 && threadIdx.x == 0) {
            S.gamma = S.lambda;
            S.lb_new_pair = 0;
        }
        return;
    }
    const int nslot = (head + cnt - 1) % M1;
    float av[MEM], bv[MEM], cv[MEM], dv[MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) av[k] = bv[k] = cv[k] = dv[k] = 0.f;
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const long long ge = base + e;
        const float x = gv[ge];
        const float yn = newp ? ringY[nslot * a.vstride + ge] : 0.f;
#pragma unroll
        for (int k = 0; k < MEM; ++k)
            if (k < cnt) {
                const int sl = (head + k) % M1;
                const float se = ringS[sl * a.vstride + ge], qe = ringY[sl * a.vstride + ge];
                av[k] += se * x;
                bv[k] += qe * x;
                cv[k] += se * yn;
                dv[k] += qe * yn;
            }
    }
    float sums[4 * MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) {
        sums[k] = av[k];
        sums[MEM + k] = bv[k];
        sums[2 * MEM + k] = cv[k];
        sums[3 * MEM + k] = dv[k];
    }
    float maxs[1];
    if (inst_reduce<4 * MEM, 0>(a, inst, sums, maxs, tot) && threadIdx.x == 0) {
        int sl[MEM];
        for (int k = 0; k < cnt; ++k) sl[k] = (head + k) % M1;
        if (newp) {
            for (int k = 0; k < cnt; ++k) {
                S.SY[sl[k]][nslot] = tot[2 * MEM + k];
                S.YY[sl[k]][nslot] = tot[3 * MEM + k];
                S.YY[nslot][sl[k]] = tot[3 * MEM + k];
            }
            S.lb_new_pair = 0;
        }
        const double gam = S.SY[nslot][nslot] / S.YY[nslot][nslot];
        double x1[MEM], tv[MEM], top[MEM];
        for (int i = cnt - 1; i >= 0; --i) {
            double s = tot[i];
            for (int j = i + 1; j < cnt; ++j) s -= S.SY[sl[i]][sl[j]] * x1[j];
            x1[i] = s / S.SY[sl[i]][sl[i]];
        }
        for (int i = 0; i < cnt; ++i) {
            double s = S.SY[sl[i]][sl[i]] * x1[i] - gam * tot[MEM + i];
            for (int j = 0; j < cnt; ++j) s += gam * S.YY[sl[i]][sl[j]] * x1[j];
            tv[i] = s;
        }
        for (int i = 0; i < cnt; ++i) {
            double s = tv[i];
            for (int j = 0; j < i; ++j) s -= S.SY[sl[j]][sl[i]] * top[j];
            top[i] = s / S.SY[sl[i]][sl[i]];
        }
        S.gamma = gam;
        for (int i = 0; i < cnt; ++i) {
            S.coef_s[i] = top[i];
            S.coef_y[i] = -gam * x1[i];
        }
    }
}

template <int MEM>
__global__ void __launch_bounds__(kBT) k_blb_dir(ElemArgs a, const float *gv, const float *ringS, const float *ringY,
                                                 float *d) {
    BLOCK_PROLOGUE
    const int cnt = S.lb_count, head = S.lb_head, M1 = a.mem + 1;
    const float gam = (float)S.gamma;
    float cs[MEM], cy[MEM];
    int sl[MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) {
        sl[k] = (head + (k < cnt ? k : 0)) % M1;
        cs[k] = k < cnt ? (float)S.coef_s[k] : 0.f;
        cy[k] = k < cnt ? (float)S.coef_y[k] : 0.f;
    }
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const long long ge = base + e;
        float acc = gam * gv[ge];
#pragma unroll
        for (int k = 0; k < MEM; ++k)
            if (k < cnt) acc += cs[k] * ringS[sl[k] * a.vstride + ge] + cy[k] * ringY[sl[k] * a.vstride + ge];
        d[ge] = -acc;
    }
}

// NAMA line search: w = ybar - lam r + tau (d + lam r), h(w) = h - lam hr + tau (hd + lam hr).
template <int J>
__global__ void __launch_bounds__(kBT) k_bls(ElemArgs a, const float *yb, const float *h, const float *r,
                                             const float *d, const float *hr, const float *hd, int e0x, int nc,
                                             int last_group) {
    BLOCK_PROLOGUE
    __shared__ double tot[J];
    if (S.ls_done) return;
    const float lam = (float)S.lambda, ilam = 1.f / lam;
    float tau[J], acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        tau[j] = ldexpf(1.f, -(e0x + j));
        acc[j] = 0.f;
    }
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const EMeta M = emeta(g, e);
        const long long ge = base + e;
        const float y0 = yb[ge], h0 = h[ge], re = r[ge], hre = hr[ge];
        const float wa = y0 - lam * re, wb = d[ge] + lam * re, ha = h0 - lam * hre, hb = hd[ge] + lam * hre;
        const float c0 = term(h0, y0, lam, ilam, M);
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] += term(ha + tau[j] * hb, wa + tau[j] * wb, lam, ilam, M) - c0;
    }
    float sums[J];
#pragma unroll
    for (int j = 0; j < J; ++j) sums[j] = acc[j];
    float maxs[1];
    if (inst_reduce<J, 0>(a, inst, sums, maxs, tot) && threadIdx.x == 0) {
        for (int j = 0; j < nc; ++j) {
            if (-tot[j] <= 0.0) {
                S.tau = ldexp(1.0, -(e0x + j));
                S.ls_done = 1;
                return;
            }
        }
        if (last_group) {
            S.tau = 0.0;
            S.ls_done = 1;
            S.ls_zero += 1;
        }
    }
}

__global__ void __launch_bounds__(kBT) k_bfbstep(ElemArgs a, float *yb, const float *h, const float *r, const float *d,
                                                 const float *hr, const float *hd, float *ringS) {
    BLOCK_PROLOGUE
    const float lam = (float)S.lambda, ilam = 1.f / lam, tau = (float)S.tau;
    const int p = (S.lb_head + S.lb_count) % (a.mem + 1);
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const EMeta M = emeta(g, e);
        const long long ge = base + e;
        const float y0 = yb[ge], re = r[ge], hre = hr[ge];
        const float w = y0 - lam * re + tau * (d[ge] + lam * re);
        const float hw = h[ge] - lam * hre + tau * (hd[ge] + lam * hre);
        const float z = clampf(hw + w * ilam, M.lo, M.hi);
        const float yn = w + lam * (hw - z);
        ringS[p * a.vstride + ge] = yn - y0;
        yb[ge] = yn;
    }
}

// Per-instance bookkeeping.  advance = 1 after the FB step: a pair is pending, one more
// iteration, the next line search starts afresh.  advance = 0 after a residual pass: the stop
// test (||z - Hx||_inf <= tol, or a NaN) retires the instance.
__global__ void k_bstep_done(BatchScalars *sc, int ninst, double tol, int *active, int *nactive, int advance) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    BatchScalars &S = sc[i];
    if (!S.active) return;
    if (advance) {
        S.lb_pending_valid = 1;
        S.iters += 1;
        S.ls_done = 0;
        return;
    }
    if (S.res_inf <= tol || S.nan_flag) {
        S.active = 0;
        active[i] = 0;
        atomicSub(nactive, 1);
    }
}

// Outputs of every instance: y = S ybar, Hx = S^-1 h, z = S^-1 proj(h + ybar / lambda).
__global__ void k_bfinish(ElemArgs a, const float *yb, const float *h, float *y, float *hx, float *z) {
    const int inst = a.blk_inst[blockIdx.x];
    const InstDev &in = a.insts[inst];
    const GroupDev &g = a.groups[in.group];
    const float ilam = (float)(1.0 / a.sc[inst].lambda);
    const int chunk = blockIdx.x - in.block0;
    const int e0 = chunk * kChunkE, e1 = min(in.m, e0 + kChunkE);
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const EMeta M = emeta(g, e);
        const long long ge = in.elem0 + e;
        const float ye = yb[ge], he = h[ge];
        y[ge] = M.sq * ye;
        if (hx) hx[ge] = he / M.sq;
        if (z) z[ge] = clampf(he + ye * ilam, M.lo, M.hi) / M.sq;
    }
}

__global__ void k_bscale(ElemArgs a, const float *y, float *yb, int dir) {
    const int inst = a.blk_inst[blockIdx.x];
    const InstDev &in = a.insts[inst];
    const GroupDev &g = a.groups[in.group];
    const int chunk = blockIdx.x - in.block0;
    const int e0 = chunk * kChunkE, e1 = min(in.m, e0 + kChunkE);
    for (int e = e0 + threadIdx.x; e < e1; e += kBT) {
        const EMeta M = emeta(g, e);
        const long long ge = in.elem0 + e;
        yb[ge] = dir > 0 ? y[ge] / M.sq : y[ge] * M.sq;
    }
}

}  // namespace
}  // namespace sto

// =============================================================================================
// Host side
// =============================================================================================
using namespace sto;

struct stobatch_s {
    std::vector<sto_group_desc> desc;
    std::vector<GroupDev> groups;   // host copies (device pointers filled at bind)
    std::vector<InstDev> insts;
    std::vector<int> blk_inst;
    std::vector<Task> tasks;
    std::vector<int> bwd_phase, fwd_phase;  // task offsets per phase (size phases + 1)
    std::vector<int> gam_phase;
    int maxN = 0, ninst = 0, nblocks = 0;
    long long M = 0, vpad = 0, Ssz = 0, Usz = 0;  // vector length, padded stride, scratch sizes
    // layout (byte offsets)
    size_t o_groups, o_insts, o_blk, o_tasks, o_G, o_K, o_R, o_box, o_W, o_AB64, o_P64, o_scr, o_off, o_gam, o_c,
        o_x0, o_s, o_ub, o_xs, o_us, o_vec, o_ringS, o_ringY, o_part, o_sc, o_active, o_nact, o_status, o_sqn, total;
    std::vector<long long> aboff, ptoff, scoff;
    char *ws = nullptr;
    bool factored = false;
    std::string err;
    BatchScalars *hs = nullptr;
    std::map<std::tuple<const void *, const void *, const void *, const void *, const void *, int, int, int>,
             cudaGraphExec_t>
        graphs;
    template <class T>
    T *at(size_t o) const { return reinterpret_cast<T *>(ws + o); }
};

static size_t ru(size_t v, size_t a) { return (v + a - 1) / a * a; }

static sto_status bfail(stobatch_t b, cudaError_t e, const char *what) {
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return STO_ERR_CUDA;
}
#define BCUDA(b, call)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return bfail(b, _e, #call); \
    } while (0)

extern "C" {

STO_API sto_status stobatch_create(const sto_group_desc *groups, int32_t ngroups, stobatch_t *out) {
    if (!groups || ngroups < 1 || !out) return STO_ERR_INVALID_ARG;
    stobatch_t b = new stobatch_s();
    long long elem = 0, sb = 0, ub = 0;
    int inst = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
        const sto_group_desc &d = groups[gi];
        if (d.nx < 1 || d.nx > 64 || d.nu < 1 || d.nu > 32 || d.horizon < 1 || d.horizon > kMaxStages ||
            d.branching < 1 || d.branch_stages < 0 || d.branch_stages > d.horizon || d.num_instances < 1 || !d.A ||
            !d.B || !d.Q || !d.R || !d.PN || !d.xlo || !d.xhi || !d.ulo || !d.uhi) {
            delete b;
            return STO_ERR_INVALID_ARG;
        }
        b->desc.push_back(d);
        GroupDev g{};
        g.nx = d.nx;
        g.nu = d.nu;
        g.N = d.horizon;
        g.b = d.branching;
        g.s = d.branch_stages;
        g.nxu = d.nx + d.nu;
        int n = 1, node = 0;
        double pi = 1.0;
        for (int t = 0; t <= g.N; ++t) {
            g.soff[t] = node;
            g.pi[t] = (float)pi;
            g.sq[t] = (float)std::sqrt(pi);
            node += n;
            if (t < g.N) {
                const int bt = t < g.s ? g.b : 1;
                n *= bt;
                pi /= bt;
            }
            if (node > (1 << 24)) {
                delete b;
                return STO_ERR_INVALID_ARG;
            }
        }
        g.soff[g.N + 1] = node;
        g.Nn = node;
        g.Nl = g.soff[g.N + 1] - g.soff[g.N];
        g.Np = g.Nn - g.Nl;
        g.m = g.Np * g.nxu + g.Nl * g.nx;
        g.I = d.num_instances;
        g.inst0 = inst;
        g.elem0 = elem;
        g.sbase = sb;
        g.ubase = ub;
        for (int k = 0; k < g.I; ++k) {
            InstDev in{};
            in.group = gi;
            in.local = k;
            in.elem0 = elem;
            in.sbase = sb;
            in.ubase = ub;
            in.m = g.m;
            in.nblocks = (g.m + kChunkE - 1) / kChunkE;
            in.block0 = b->nblocks;
            for (int q = 0; q < in.nblocks; ++q) b->blk_inst.push_back(inst);
            b->nblocks += in.nblocks;
            b->insts.push_back(in);
            elem += g.m;
            sb += (long long)g.Nn * g.nx;
            ub += (long long)g.Np * g.nu;
            ++inst;
        }
        b->maxN = std::max(b->maxN, g.N);
        b->groups.push_back(g);
    }
    b->ninst = inst;
    b->M = elem;
    b->vpad = (long long)ru((size_t)elem, 64);
    b->Ssz = sb;
    b->Usz = ub;
    // tasks: backward phase p = stage N_g - 1 - p, forward phase p = stage p, gamma = stages 0..N-1
    auto add_tasks = [&](int gi, int t) {
        const GroupDev &g = b->groups[gi];
        const int cols = (g.soff[t + 1] - g.soff[t]) * g.I;
        for (int c0 = 0; c0 < cols; c0 += kTC) b->tasks.push_back(Task{gi, t, c0, std::min(kTC, cols - c0)});
    };
    for (int p = 0; p < b->maxN; ++p) {
        b->bwd_phase.push_back((int)b->tasks.size());
        for (int gi = 0; gi < ngroups; ++gi)
            if (b->groups[gi].N > p) add_tasks(gi, b->groups[gi].N - 1 - p);
    }
    b->bwd_phase.push_back((int)b->tasks.size());
    for (int p = 0; p <= b->maxN; ++p) {
        b->fwd_phase.push_back((int)b->tasks.size());
        for (int gi = 0; gi < ngroups; ++gi)
            if (b->groups[gi].N >= p) add_tasks(gi, p);
    }
    b->fwd_phase.push_back((int)b->tasks.size());
    // layout
    size_t tot = 0;
    auto add = [&](size_t bytes) {
        size_t o = ru(tot, 256);
        tot = o + ru(bytes, 16);
        return o;
    };
    const int G = ngroups;
    b->o_groups = add(G * sizeof(GroupDev));
    b->o_insts = add(b->ninst * sizeof(InstDev));
    b->o_blk = add(b->nblocks * 4);
    b->o_tasks = add(b->tasks.size() * sizeof(Task));
    size_t gsz = 0, ksz = 0, rsz = 0, absz = 0, psz = 0, scsz = 0;
    for (auto &g : b->groups) {
        gsz += (size_t)g.nx * g.nxu;
        ksz += (size_t)g.N * g.nu * g.nx;
        rsz += (size_t)g.N * g.nu * g.nu;
        b->aboff.push_back((long long)absz);
        absz += (size_t)g.nx * g.nxu;
        b->ptoff.push_back((long long)psz);
        psz += (size_t)(g.N + 1) * g.nx * g.nx;
        b->scoff.push_back((long long)scsz);
        scsz += (size_t)g.nx * g.nxu + 4 * g.nu * g.nu + 2 * g.nu * g.nx;
    }
    b->o_G = add(gsz * 4);
    b->o_K = add(ksz * 4);
    b->o_R = add(rsz * 4);
    b->o_box = add(G * 2 * 96 * 4);
    b->o_W = add(G * 3 * 64 * 4);
    b->o_AB64 = add(absz * 8);
    b->o_P64 = add(psz * 8);
    b->o_scr = add(scsz * 8);
    b->o_off = add(3 * G * 8);
    b->o_gam = add(b->vpad * 4);
    b->o_c = add(b->Ssz * 4);
    b->o_x0 = add((size_t)b->ninst * 64 * 4);
    b->o_s = add(2 * b->Ssz * 4);
    b->o_ub = add(2 * b->Usz * 4);
    b->o_xs = add(2 * b->Ssz * 4);
    b->o_us = add(2 * b->Usz * 4);
    b->o_vec = add(8 * b->vpad * 4);
    b->o_ringS = add((kBMaxMem + 1) * b->vpad * 4);
    b->o_ringY = add((kBMaxMem + 1) * b->vpad * 4);
    b->o_part = add((size_t)b->nblocks * kRedSlots * 8);
    b->o_sc = add(b->ninst * sizeof(BatchScalars));
    b->o_active = add(b->ninst * 4);
    b->o_nact = add(64);
    b->o_status = add(64);
    size_t nsum = 0;
    for (auto &g : b->groups) nsum += g.Nn;
    b->o_sqn = add(nsum * 4);
    b->total = ru(tot, 256);
    if (cudaMallocHost(&b->hs, b->ninst * sizeof(BatchScalars)) != cudaSuccess) b->hs = new BatchScalars[b->ninst];
    *out = b;
    return STO_OK;
}

STO_API void stobatch_destroy(stobatch_t b) {
    if (!b) return;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->hs && cudaFreeHost(b->hs) != cudaSuccess) delete[] b->hs;
    delete b;
}

STO_API sto_status stobatch_sizes(stobatch_t b, int64_t *total_dual, int32_t *num_instances, int64_t *inst_offsets,
                                  int64_t *inst_sizes) {
    if (!b) return STO_ERR_INVALID_ARG;
    if (total_dual) *total_dual = b->M;
    if (num_instances) *num_instances = b->ninst;
    for (int i = 0; i < b->ninst; ++i) {
        if (inst_offsets) inst_offsets[i] = b->insts[i].elem0;
        if (inst_sizes) inst_sizes[i] = b->insts[i].m;
    }
    return STO_OK;
}

STO_API sto_status stobatch_workspace_size(stobatch_t b, size_t *bytes) {
    if (!b || !bytes) return STO_ERR_INVALID_ARG;
    *bytes = b->total;
    return STO_OK;
}

STO_API sto_status stobatch_bind_workspace(stobatch_t b, void *dev, size_t bytes, sto_stream_t stream) {
    if (!b || !dev) return STO_ERR_INVALID_ARG;
    if (bytes < b->total) return STO_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(dev) % 256) return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    b->ws = static_cast<char *>(dev);
    BCUDA(b, cudaMemsetAsync(b->ws, 0, b->total, st));
    // device pointers of the per-group arrays and the shared data (FP32 solve copies, FP64 factor input)
    size_t goff = 0, koff = 0, roff = 0;
    std::vector<float> Gh, boxh(b->groups.size() * 2 * 96), Wh(b->groups.size() * 3 * 64), sqh;
    std::vector<double> ABh;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        GroupDev &g = b->groups[gi];
        const sto_group_desc &d = b->desc[gi];
        g.G = b->at<float>(b->o_G) + goff;
        g.Kt = b->at<float>(b->o_K) + koff;
        g.Ri = b->at<float>(b->o_R) + roff;
        g.box = b->at<float>(b->o_box) + gi * 2 * 96;
        g.W = b->at<float>(b->o_W) + gi * 3 * 64;
        g.sqn = b->at<float>(b->o_sqn) + sqh.size();
        for (int t = 0; t <= g.N; ++t)
            for (int i = g.soff[t]; i < g.soff[t + 1]; ++i) sqh.push_back(g.sq[t]);
        for (int r = 0; r < g.nx; ++r) {
            for (int c = 0; c < g.nx; ++c) {
                Gh.push_back((float)d.A[r * g.nx + c]);
                ABh.push_back(d.A[r * g.nx + c]);
            }
            for (int c = 0; c < g.nu; ++c) {
                Gh.push_back((float)d.B[r * g.nu + c]);
                ABh.push_back(d.B[r * g.nu + c]);
            }
        }
        for (int k = 0; k < g.nx; ++k) {
            boxh[gi * 192 + k] = (float)d.xlo[k];
            boxh[gi * 192 + g.nxu + k] = (float)d.xhi[k];
            Wh[gi * 192 + k] = (float)d.Q[k];
            Wh[gi * 192 + g.nx + g.nu + k] = (float)d.PN[k];
        }
        for (int k = 0; k < g.nu; ++k) {
            boxh[gi * 192 + g.nx + k] = (float)d.ulo[k];
            boxh[gi * 192 + g.nxu + g.nx + k] = (float)d.uhi[k];
            Wh[gi * 192 + g.nx + k] = (float)d.R[k];
        }
        goff += (size_t)g.nx * g.nxu;
        koff += (size_t)g.N * g.nu * g.nx;
        roff += (size_t)g.N * g.nu * g.nu;
    }
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_groups, b->groups.data(), b->groups.size() * sizeof(GroupDev),
                             cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_insts, b->insts.data(), b->insts.size() * sizeof(InstDev),
                             cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_blk, b->blk_inst.data(), b->blk_inst.size() * 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_tasks, b->tasks.data(), b->tasks.size() * sizeof(Task),
                             cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_G, Gh.data(), Gh.size() * 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_AB64, ABh.data(), ABh.size() * 8, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_box, boxh.data(), boxh.size() * 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_W, Wh.data(), Wh.size() * 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_sqn, sqh.data(), sqh.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<long long> offs;
    offs.insert(offs.end(), b->aboff.begin(), b->aboff.end());
    offs.insert(offs.end(), b->ptoff.begin(), b->ptoff.end());
    offs.insert(offs.end(), b->scoff.begin(), b->scoff.end());
    BCUDA(b, cudaMemcpyAsync(b->ws + b->o_off, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaStreamSynchronize(st));
    b->factored = false;
    return STO_OK;
}

// Per-instance data: x0 [nx] and disturbances c [Nn][nx] (row 0 unused), host FP64.
STO_API sto_status stobatch_set_instance(stobatch_t b, int32_t group, int32_t instance, const double *x0,
                                         const double *c, sto_stream_t stream) {
    if (!b || !b->ws || !x0 || !c || group < 0 || group >= (int)b->groups.size()) return STO_ERR_INVALID_ARG;
    const GroupDev &g = b->groups[group];
    if (instance < 0 || instance >= g.I) return STO_ERR_INVALID_ARG;
    const InstDev &in = b->insts[g.inst0 + instance];
    std::vector<float> xf(64, 0.f), cf((size_t)g.Nn * g.nx);
    for (int k = 0; k < g.nx; ++k) xf[k] = (float)x0[k];
    for (size_t k = 0; k < cf.size(); ++k) cf[k] = (float)c[k];
    for (int k = 0; k < g.nx; ++k) cf[k] = 0.f;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BCUDA(b, cudaMemcpyAsync(b->at<float>(b->o_x0) + (size_t)(g.inst0 + instance) * 64, xf.data(), 64 * 4,
                             cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(b->at<float>(b->o_c) + in.sbase, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaStreamSynchronize(st));
    b->factored = false;
    return STO_OK;
}

STO_API sto_status stobatch_factor(stobatch_t b, sto_stream_t stream) {
    if (!b || !b->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int G = (int)b->groups.size();
    const long long *offs = b->at<long long>(b->o_off);
    BCUDA(b, cudaMemsetAsync(b->ws + b->o_status, 0, 64, st));
    k_bfactor<<<G, 256, 0, st>>>(b->at<GroupDev>(b->o_groups), b->at<double>(b->o_AB64), offs, b->at<double>(b->o_P64),
                                 offs + G, b->at<double>(b->o_scr), offs + 2 * G, b->at<int>(b->o_status));
    // gamma for every nonleaf node (backward-phase task lists cover every (group, stage < N))
    for (size_t p = 0; p + 1 < b->bwd_phase.size(); ++p) {
        const int t0 = b->bwd_phase[p], nt = b->bwd_phase[p + 1] - t0;
        if (nt > 0)
            k_bgamma<<<nt, 256, 0, st>>>(b->at<GroupDev>(b->o_groups), b->at<InstDev>(b->o_insts),
                                        b->at<Task>(b->o_tasks), t0, b->at<double>(b->o_P64), offs + G,
                                        b->at<float>(b->o_c), b->at<float>(b->o_gam));
    }
    int flag = 0;
    BCUDA(b, cudaMemcpyAsync(&flag, b->ws + b->o_status, 4, cudaMemcpyDeviceToHost, st));
    BCUDA(b, cudaStreamSynchronize(st));
    if (flag) {
        b->err = "R + B'PB not positive definite in group " + std::to_string(flag - 1);
        return STO_ERR_NUMERICAL;
    }
    b->factored = true;
    return STO_OK;
}

}  // extern "C"

namespace {

template <int NR>
void launch_round(stobatch_t b, const RoundArgs<NR> &a, cudaStream_t st) {
    raise_smem_cap((const void *)k_bbwd<NR>, bwd_smem<NR>());
    raise_smem_cap((const void *)k_bfwd<NR>, fwd_smem<NR>());
    for (size_t p = 0; p + 1 < b->bwd_phase.size(); ++p) {
        const int t0 = b->bwd_phase[p], nt = b->bwd_phase[p + 1] - t0;
        if (nt > 0) k_bbwd<NR><<<nt, kBT, bwd_smem<NR>(), st>>>(a, t0);
    }
    for (size_t p = 0; p + 1 < b->fwd_phase.size(); ++p) {
        const int t0 = b->fwd_phase[p], nt = b->fwd_phase[p + 1] - t0;
        if (nt > 0) k_bfwd<NR><<<nt, kBT, fwd_smem<NR>(), st>>>(a, t0);
    }
}

// One solve round for nrhs (1 or 2) right-hand sides, replayed from a cached CUDA graph.
sto_status bround(stobatch_t b, const float *y0, const float *y1, float *h0, float *h1, int nrhs, bool homog,
                  bool scaled, const int *active, cudaStream_t st) {
    auto key = std::make_tuple((const void *)y0, (const void *)y1, (const void *)h0, (const void *)h1,
                               (const void *)active, nrhs, (int)homog, (int)scaled);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaStream_t cap;
        BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        BCUDA(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        auto fill = [&](auto &a) {
            a.groups = b->at<GroupDev>(b->o_groups);
            a.insts = b->at<InstDev>(b->o_insts);
            a.tasks = b->at<Task>(b->o_tasks);
            a.y[0] = y0;
            a.y[1] = y1 ? y1 : y0;
            a.h[0] = h0;
            a.h[1] = h1 ? h1 : h0;
            a.gam = b->at<float>(b->o_gam);
            a.c = b->at<float>(b->o_c);
            a.x0 = b->at<float>(b->o_x0);
            a.s = b->at<float>(b->o_s);
            a.ubar = b->at<float>(b->o_ub);
            a.xs = b->at<float>(b->o_xs);
            a.us = b->at<float>(b->o_us);
            a.s_stride = b->Ssz;
            a.u_stride = b->Usz;
            a.active = active;
            a.homog = homog ? 1 : 0;
            a.scaled = scaled ? 1 : 0;
        };
        if (nrhs == 1) {
            RoundArgs<1> a;
            fill(a);
            launch_round<1>(b, a, cap);
        } else {
            RoundArgs<2> a;
            fill(a);
            launch_round<2>(b, a, cap);
        }
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return bfail(b, e, "capture of a batched solve round");
        }
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return bfail(b, e, "cudaGraphInstantiate");
        it = b->graphs.emplace(key, exec).first;
    }
    BCUDA(b, cudaGraphLaunch(it->second, st));
    return STO_OK;
}

template <int MEM>
void blbfgs(stobatch_t b, const ElemArgs &ea, const float *gv, float *d, cudaStream_t st) {
    float *rs = b->at<float>(b->o_ringS), *ry = b->at<float>(b->o_ringY);
    k_blb_dots<MEM><<<b->nblocks, kBT, 0, st>>>(ea, gv, rs, ry);
    k_blb_dir<MEM><<<b->nblocks, kBT, 0, st>>>(ea, gv, rs, ry, d);
}

}  // namespace

extern "C" {

// Batched solve round (Algorithm 3/4) on caller vectors laid out as the batch (instances
// concatenated, each in the single-instance dual layout).
STO_API sto_status stobatch_solve_step(stobatch_t b, const void *y, void *hx, int32_t homogeneous, int32_t scaled,
                                       sto_stream_t stream) {
    if (!b || !y || !hx) return STO_ERR_INVALID_ARG;
    if (!b->factored) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    sto_status s = bround(b, static_cast<const float *>(y), nullptr, static_cast<float *>(hx), nullptr, 1,
                          homogeneous != 0, scaled != 0, nullptr, st);
    if (s != STO_OK) return s;
    BCUDA(b, cudaGetLastError());
    return STO_OK;
}

// Batched NAMA (Algorithm 2) for every instance; lambdas[g] per group (the Hessian of the dual
// does not depend on x0 or c).  y (batch layout, unscaled; zeros for a cold start) is
// overwritten by the final dual iterates, z (may be NULL) by z_lambda, h (may be NULL) by Hx.
// infos[i] (per instance) receives iterations, status and the final residual; the call returns
// STO_NOT_CONVERGED if any instance hit max_iter.  Synchronises the stream.
STO_API sto_status stobatch_nama_solve(stobatch_t b, const sto_opts *o, const double *lambdas, void *yv, void *zv,
                                       void *hv, sto_info *infos, sto_stream_t stream) {
    if (!b || !o || !lambdas || !yv) return STO_ERR_INVALID_ARG;
    if (!b->factored) return STO_ERR_NOT_READY;
    if (o->lbfgs_mem < 1 || o->lbfgs_mem > kBMaxMem || o->max_ls < 0 || o->max_ls > 30 || !(o->tol > 0))
        return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long vs = b->vpad;
    float *V = b->at<float>(b->o_vec);
    float *yb = V, *h = V + vs, *r = V + 2 * vs, *d = V + 3 * vs, *hr = V + 4 * vs, *hd = V + 5 * vs;
    BatchScalars *sc = b->at<BatchScalars>(b->o_sc);
    int *active = b->at<int>(b->o_active), *nact = b->at<int>(b->o_nact);
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    BCUDA(b, cudaEventRecord(e0, st));
    std::memset(b->hs, 0, b->ninst * sizeof(BatchScalars));
    std::vector<int> act(b->ninst, 1);
    for (int i = 0; i < b->ninst; ++i) {
        b->hs[i].lambda = lambdas[b->insts[i].group];
        b->hs[i].active = 1;
    }
    BCUDA(b, cudaMemcpyAsync(sc, b->hs, b->ninst * sizeof(BatchScalars), cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaMemcpyAsync(active, act.data(), b->ninst * 4, cudaMemcpyHostToDevice, st));
    const int ninst = b->ninst;
    BCUDA(b, cudaMemcpyAsync(nact, &ninst, 4, cudaMemcpyHostToDevice, st));
    BCUDA(b, cudaStreamSynchronize(st));
    ElemArgs ea;
    ea.groups = b->at<GroupDev>(b->o_groups);
    ea.insts = b->at<InstDev>(b->o_insts);
    ea.blk_inst = b->at<int>(b->o_blk);
    ea.sc = sc;
    ea.partials = b->at<double>(b->o_part);
    ea.vstride = vs;
    ea.mem = o->lbfgs_mem;
    ea.tol = o->tol;
    ea.eps_curv = o->eps_curv;
    float *ringS = b->at<float>(b->o_ringS), *ringY = b->at<float>(b->o_ringY);
    const int nb = b->nblocks;
    int gfirst[3], gcount[3], ng = 0;
    {
        int left = o->max_ls + 1, e = 0;
        const int sizes[3] = {4, 8, 19};
        for (int k = 0; k < 3 && left > 0; ++k) {
            const int c = left < sizes[k] ? left : sizes[k];
            gfirst[ng] = e;
            gcount[ng] = c;
            ++ng;
            e += c;
            left -= c;
        }
    }
    k_bscale<<<nb, kBT, 0, st>>>(ea, static_cast<const float *>(yv), yb, 1);
    sto_status s = bround(b, yb, nullptr, h, nullptr, 1, false, true, active, st);
    if (s != STO_OK) return s;
    k_bpoint<<<nb, kBT, 0, st>>>(ea, yb, h, r, ringS, ringY, 0);
    k_bstep_done<<<(ninst + 127) / 128, 128, 0, st>>>(sc, ninst, o->tol, active, nact, 0);
    int iters = 0, nleft = ninst;
    sto_status result = STO_OK;
    while (true) {
        BCUDA(b, cudaMemcpyAsync(&nleft, nact, 4, cudaMemcpyDeviceToHost, st));
        BCUDA(b, cudaStreamSynchronize(st));
        if (nleft == 0) break;
        if (iters >= o->max_iter) {
            result = STO_NOT_CONVERGED;
            break;
        }
        if (o->lbfgs_mem <= 5)
            blbfgs<5>(b, ea, r, d, st);
        else
            blbfgs<8>(b, ea, r, d, st);
        if ((s = bround(b, r, d, hr, hd, 2, true, true, active, st)) != STO_OK) return s;
        for (int k = 0; k < ng; ++k) {
            const int last = k == ng - 1;
            if (k == 0)
                k_bls<4><<<nb, kBT, 0, st>>>(ea, yb, h, r, d, hr, hd, gfirst[k], gcount[k], last);
            else if (k == 1)
                k_bls<8><<<nb, kBT, 0, st>>>(ea, yb, h, r, d, hr, hd, gfirst[k], gcount[k], last);
            else
                k_bls<19><<<nb, kBT, 0, st>>>(ea, yb, h, r, d, hr, hd, gfirst[k], gcount[k], last);
        }
        k_bfbstep<<<nb, kBT, 0, st>>>(ea, yb, h, r, d, hr, hd, ringS);
        k_bstep_done<<<(ninst + 127) / 128, 128, 0, st>>>(sc, ninst, o->tol, active, nact, 1);
        if ((s = bround(b, yb, nullptr, h, nullptr, 1, false, true, active, st)) != STO_OK) return s;
        k_bpoint<<<nb, kBT, 0, st>>>(ea, yb, h, r, ringS, ringY, 1);
        k_bstep_done<<<(ninst + 127) / 128, 128, 0, st>>>(sc, ninst, o->tol, active, nact, 0);
        ++iters;
        BCUDA(b, cudaGetLastError());
    }
    k_bfinish<<<nb, kBT, 0, st>>>(ea, yb, h, static_cast<float *>(yv), static_cast<float *>(hv),
                                  static_cast<float *>(zv));
    BCUDA(b, cudaEventRecord(e1, st));
    BCUDA(b, cudaMemcpyAsync(b->hs, sc, b->ninst * sizeof(BatchScalars), cudaMemcpyDeviceToHost, st));
    BCUDA(b, cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (infos)
        for (int i = 0; i < b->ninst; ++i) {
            infos[i].iters = b->hs[i].iters;
            infos[i].solve_calls = 0;
            infos[i].status = b->hs[i].nan_flag ? STO_ERR_NUMERICAL : (b->hs[i].active ? STO_NOT_CONVERGED : STO_OK);
            infos[i].ls_zero = b->hs[i].ls_zero;
            infos[i].launches = 0;
            infos[i].halvings = 0;
            infos[i].lambda = lambdas[b->insts[i].group];  // the step is per group
            infos[i].res_inf = b->hs[i].res_inf;
            infos[i].fbe = b->hs[i].phi;
            infos[i].ms = ms;
        }
    BCUDA(b, cudaGetLastError());
    return result;
}

STO_API const char *stobatch_last_error(stobatch_t b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
