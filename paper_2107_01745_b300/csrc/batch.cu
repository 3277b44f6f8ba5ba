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
    int al_d, al_s, al_u;       // widest vector (4, 2 or 1 floats) that every instance's dual blocks,
                                // state rows (s, x, c) and input rows (ubar) are aligned to
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
// Solve rounds.  A tile is up to TC (node, instance) columns of one (group, stage) and one pass;
// column c of a stage with n nodes is instance c / n, node soff_t + c % n.  A round is one
// persistent launch (one wave of CTAs) that hands the tiles out in ticket order: the backward
// tiles by height (stage N_g - 1 - p of every group g, for p = 0, 1, ...), then the forward tiles
// by depth.  Each tile raises its own done flag, and first waits (bounded) for the flags of the
// tiles that hold the columns it reads: column c of stage t has children c b_t + j at stage t + 1
// and parent floor(c / b_{t-1}) at stage t - 1 (instances stay contiguous), so backward (g, t)
// waits on the backward tiles of (g, t + 1) covering its children (the leaves' s comes from y),
// forward (g, t) on the forward tiles of (g, t - 1) covering its parents, forward (g, 0) on the
// backward tile of (g, 0) with its columns (which, transitively, covers every backward tile of
// its instances).  Those tiles hold earlier tickets and every CTA is resident, so every wait
// ends; a wait that gives up raises an error word, and the round runs to its end without that
// input.  Data other CTAs write during the round (s, ubar, x) is read through L2.
// ---------------------------------------------------------------------------------------------
struct Task {  // set-up passes (gamma): a tile of kGC columns of one (group, stage)
    int group, stage, col0, ncols;
};
constexpr int kGC = 64;

struct RTask {
    int group, stage, col0, ncols;
    int pass;       // 0 backward, 1 forward
    int dep0, ndep; // the tiles (ticket indices dep0 .. dep0 + ndep - 1) whose flags it waits on
    int pad;
};

template <int NR>
struct RoundArgs {
    const GroupDev *groups;
    const InstDev *insts;
    const RTask *tasks;
    int ntasks;
    const float *y[2];
    float *h[2];
    const float *gam;     // gamma in the dual layout (x-part, u-part)
    const float *c;       // disturbances [instance][Nn][nx] (scratch layout of s)
    const float *x0;      // [instance][64]
    float *s, *ubar, *xs;  // scratch; second right-hand side at +stride
    long long s_stride, u_stride;
    const int *active;    // per instance (null: all active)
    unsigned *ctrs;       // done flag per tile (ticket index)
    unsigned *ticket;     // next tile to hand out
    int *err;             // raised by a dependency wait that gave up
    int homog, scaled;
};

constexpr unsigned long long kBWaitNs = 1500000000ull;  // bounded waits: 1.5 s of wall time

// Tile geometry for TC columns and nx + nu <= XU (XU = 48: nx <= 32, nu <= 16; XU = 96: nx <= 64,
// nu <= 32).  Stage products are register-blocked FP32 GEMMs: thread (rg, cg) owns up to MR
// consecutive output rows and four columns of the tile.
template <int TC, int XU, int NT>
struct Cfg {
    static constexpr int NXM = XU * 2 / 3, NUM = XU / 3;
    static constexpr int TP = TC + 4;                 // row stride of the column tiles (16-byte aligned)
    static constexpr int CG = TC / 4;                 // column groups of 4
    static constexpr int RG = NT / CG;                // row groups
    static constexpr int MR = (XU + RG - 1) / RG;     // rows of [x; u] per thread
    static constexpr int MU = (NUM + RG - 1) / RG;    // rows of u per thread
    static constexpr int MX = (NXM + RG - 1) / RG;    // rows of x per thread
    static constexpr int MAT = NXM * XU + NUM * NXM + NUM * NUM;  // G, K, R~^-1
};
template <int NR, int TC, int XU, int NT>
constexpr size_t round_smem() {
    // matrices, then backward S [NR][NXM][TP], V [NR][NUM][TP], Wb [NR][XU][TP]
    // or forward X [NR][XU][TP], UB [NR][NUM][TP], CB [NR][NXM][TP]
    using C = Cfg<TC, XU, NT>;
    return sizeof(float) * (C::MAT + 2 * NR * XU * C::TP);
}

// What a tile needs of its group and stage, loaded into registers once per tile (the group record
// sits in global memory, and stores inside the tile would otherwise force its fields to be
// re-read in every loop).
struct Geo {
    int nx, nu, nxu, Np, Nn, m, s0, s1, n_t, bt, inst0;
    long long elem0, sbase, ubase;
    float sq_t, sq_t1, pi_t;
    const float *G, *Kt, *Ri;
    int al_d, al_s, al_u;
};
__device__ __forceinline__ Geo load_geo(const GroupDev &g, int t) {
    Geo q;
    q.nx = g.nx;
    q.nu = g.nu;
    q.nxu = g.nxu;
    q.Np = g.Np;
    q.Nn = g.Nn;
    q.m = g.m;
    q.s0 = g.soff[t];
    q.s1 = g.soff[t + 1];
    q.n_t = q.s1 - q.s0;
    q.bt = t < g.s ? g.b : 1;
    q.inst0 = g.inst0;
    q.elem0 = g.elem0;
    q.sbase = g.sbase;
    q.ubase = g.ubase;
    q.sq_t = g.sq[t];
    q.sq_t1 = t < g.N ? g.sq[t + 1] : 1.f;
    q.pi_t = g.pi[t];
    q.G = g.G;
    q.Kt = g.Kt;
    q.Ri = g.Ri;
    q.al_d = g.al_d;
    q.al_s = g.al_s;
    q.al_u = g.al_u;
    return q;
}
__device__ __forceinline__ long long doff(const Geo &q, int i) {
    return i < q.Np ? (long long)i * q.nxu : (long long)q.Np * q.nxu + (long long)(i - q.Np) * q.nx;
}

// Columns of a tile: instance data and node of each column, and whether its instance is active.
// A group's instances lie one after another in every batch array, so their offsets follow from
// the instance index (no per-instance record is read).
template <int TC>
struct ColInfo {
    long long elem[TC], sb[TC], ub[TC];
    int node[TC], ok[TC];
};
template <int NR, int TC>
__device__ __forceinline__ void load_cols(const RoundArgs<NR> &a, const Geo &q, const RTask &tk, ColInfo<TC> &ci) {
    if (threadIdx.x < TC) {
        const int col = threadIdx.x;
        int ok = 0;
        if (col < tk.ncols) {
            const int cc = tk.col0 + col, inst = cc / q.n_t;
            ci.elem[col] = q.elem0 + (long long)inst * q.m;
            ci.sb[col] = q.sbase + (long long)inst * q.Nn * q.nx;
            ci.ub[col] = q.ubase + (long long)inst * q.Np * q.nu;
            ci.node[col] = q.s0 + cc - inst * q.n_t;
            ok = !a.active || a.active[q.inst0 + inst];
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

// e = (k * TC + col) * R + r over [threadIdx.x, NR * TC * R) in steps of NT, r fastest (so that
// a warp's global accesses to a column's R consecutive reals coalesce), with the (k, col, r)
// of each step advanced from the previous one instead of divided out per element.
template <int NR, int TC, int NT, class F>
__device__ __forceinline__ void for_kcr(int R, F f) {
    const int tot = NR * TC * R;
    int e = threadIdx.x;
    int kc = e / R, r = e - kc * R;
    const int dq = NT / R, dr = NT - dq * R;
    for (; e < tot; e += NT) {
        f(kc / TC, kc % TC, r);
        r += dr;
        kc += dq;
        if (r >= R) {
            r -= R;
            ++kc;
        }
    }
}

// gather: v = load(k, col, r) for every (k, col, r) of for_kcr's enumeration, U elements per
// thread at a time with their loads issued together, then store(k, col, r, v).
template <int NR, int TC, int NT, int U, class L, class S>
__device__ __forceinline__ void gather_kcr(int R, L load, S store) {
    const int tot = NR * TC * R;
    int e = threadIdx.x;
    int kc = e / R, r = e - kc * R;
    const int dq = NT / R, dr = NT - dq * R;
    while (e < tot) {
        float v[U];
        int kk[U], cc[U], rr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            kk[u] = e < tot ? kc / TC : -1;
            cc[u] = kc % TC;
            rr[u] = r;
            v[u] = kk[u] >= 0 ? load(kk[u], cc[u], rr[u]) : 0.f;
            e += NT;
            r += dr;
            kc += dq;
            if (r >= R) {
                r -= R;
                ++kc;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (kk[u] >= 0) store(kk[u], cc[u], rr[u], v[u]);
    }
}

__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait until *c >= need; on expiry the error word is raised and the wait gives up.
__device__ void wait_count(const unsigned *c, unsigned need, int *err) {
    if (ld_acq(c) >= need) return;
    const unsigned long long t0 = gtimer();
    while (gtimer() - t0 < kBWaitNs) {
        for (int it = 0; it < 32; ++it) {
            if (ld_acq(c) >= need) return;
            __nanosleep(64);
        }
        if (*(volatile int *)err) return;
    }
    atomicCAS(err, 0, 1);
}

// The first warp waits for a tile's dependencies, one flag per lane at a time.
template <int NR>
__device__ __forceinline__ void wait_deps(const RoundArgs<NR> &a, const RTask &tk) {
    for (int d = threadIdx.x; d < tk.ndep; d += 32) wait_count(a.ctrs + tk.dep0 + d, 1u, a.err);
}

// Staging copies of the stage matrices: one 4-byte asynchronous global-to-shared copy per entry, so
// that a thread's copies are all in flight at once (a plain load-then-store loop waits out the
// L2 latency once per entry); cp_wait() before the barrier that publishes them.
__device__ __forceinline__ void cp4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Backward tile: parents of stage t.  S = sum_children s, o = [A | B]' S, v = y_u/2 + o_B + gu,
// ubar = -(1/pi_t) R~^-1 v, s = y_x/2 + o_A + K_t' v + gx.  Every global read of the tile (the
// children's s, or the leaves' y, and the column's y and gamma block) is issued in one gather.
template <int NR, int TC, int XU, int NT>
__device__ __forceinline__ void bwd_tile(const RoundArgs<NR> &a, const RTask &tk, float *sm, ColInfo<TC> &ci,
                                         int &staged) {
    using C = Cfg<TC, XU, NT>;
    const int t = tk.stage;
    const Geo q = load_geo(a.groups[tk.group], t);
    const int nx = q.nx, nu = q.nu, nxu = q.nxu;
    float *Gs = sm;                      // [r][c], r < nx, c < nx + nu
    float *Ks = Gs + C::NXM * XU;        // K_t [a][c]
    float *Rs = Ks + C::NUM * C::NXM;    // R~_t^-1 [a][b]
    float *S = sm + C::MAT;              // [k][r][col]; afterwards s (without y_x/2 + gx)
    float *V = S + NR * C::NXM * C::TP;  // [k][a][col]: v; afterwards ubar
    float *Wb = V + NR * C::NUM * C::TP; // [k][c][col]: y/2 (scaled) + gamma of the column's block
    const int bt = q.bt;
    const bool leaf_children = q.s1 >= q.Np;  // the children of stage t are leaves
    load_cols<NR, TC>(a, q, tk, ci);
    // a tile whose instances have all converged reads and writes nothing (the barrier after the
    // gather below orders the matrices' staging stores before any use)
    if (!__syncthreads_or(threadIdx.x < TC ? ci.ok[threadIdx.x] : 0)) return;
    const int key = 2 * (tk.group * (kMaxStages + 1) + t);
    if (staged != key) {
        for (int e = threadIdx.x; e < nx * nxu; e += NT) cp4(Gs + e, q.G + e);
        for (int e = threadIdx.x; e < nu * nx; e += NT) cp4(Ks + e, q.Kt + (size_t)t * nu * nx + e);
        for (int e = threadIdx.x; e < nu * nu; e += NT) cp4(Rs + e, q.Ri + (size_t)t * nu * nu + e);
        staged = key;
    }
    {
        const float sc = a.scaled ? q.sq_t : 1.f, scc = a.scaled ? q.sq_t1 : 1.f;
        // rows r < nx: S; rows nx + c: the block's entry c
        gather_kcr<NR, TC, NT, 4>(
            nx + nxu,
            [&](int k, int col, int r) -> float {
                if (!ci.ok[col]) return 0.f;
                const int i = ci.node[col];
                if (r < nx) {
                    const int j0 = q.s1 + (i - q.s0) * bt;
                    float acc = 0.f;
                    for (int j = j0; j < j0 + bt; ++j)
                        acc += leaf_children ? 0.5f * scc * a.y[k][ci.elem[col] + doff(q, j) + r]
                                             : __ldcg(a.s + k * a.s_stride + ci.sb[col] + (long long)j * nx + r);
                    return acc;
                }
                const long long o = ci.elem[col] + doff(q, i) + (r - nx);
                return 0.5f * sc * a.y[k][o] + (a.homog ? 0.f : a.gam[o]);
            },
            [&](int k, int col, int r, float v) {
                if (r < nx)
                    S[(k * C::NXM + r) * C::TP + col] = v;
                else
                    Wb[(k * XU + r - nx) * C::TP + col] = v;
            });
    }
    cp_wait();
    __syncthreads();
    const int cg = threadIdx.x % C::CG, rg = threadIdx.x / C::CG;
    const int mr = (nxu + C::RG - 1) / C::RG, r0 = rg * mr;
    float acc[NR][C::MR][4];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int m = 0; m < C::MR; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][m][q] = 0.f;
    // o = [A | B]' S
    for (int r = 0; r < nx; ++r) {
        float4 s4[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) s4[k] = *reinterpret_cast<const float4 *>(S + (k * C::NXM + r) * C::TP + cg * 4);
#pragma unroll
        for (int m = 0; m < C::MR; ++m)
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
    // v = o_B + y_u/2 + gu -> V
#pragma unroll
    for (int m = 0; m < C::MR; ++m) {
        const int c = r0 + m;
        if (m < mr && c >= nx && c < nxu)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const float4 w = *reinterpret_cast<const float4 *>(Wb + (k * XU + c) * C::TP + cg * 4);
                *reinterpret_cast<float4 *>(V + (k * C::NUM + c - nx) * C::TP + cg * 4) =
                    make_float4(acc[k][m][0] + w.x, acc[k][m][1] + w.y, acc[k][m][2] + w.z, acc[k][m][3] + w.w);
            }
    }
    __syncthreads();
    // rows c < nx: s = o_A + K' v; rows c = nx + a: ubar = -(1/pi_t) R~^-1 v
#pragma unroll
    for (int m = 0; m < C::MR; ++m)
        if (r0 + m >= nx)
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[k][m][q] = 0.f;
    for (int aa = 0; aa < nu; ++aa) {
        float4 v4[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) v4[k] = *reinterpret_cast<const float4 *>(V + (k * C::NUM + aa) * C::TP + cg * 4);
#pragma unroll
        for (int m = 0; m < C::MR; ++m) {
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
    // results in place: s = o_A + K'v + y_x/2 + gx over S (read only before the barrier above),
    // ubar over the u rows of Wb (consumed into V before it); this thread alone reads the Wb
    // entries it overwrites
    const float ipi = 1.f / q.pi_t;
#pragma unroll
    for (int m = 0; m < C::MR; ++m) {
        const int c = r0 + m;
        if (m < mr && c < nxu)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float4 *wp = reinterpret_cast<float4 *>(Wb + (k * XU + c) * C::TP + cg * 4);
                if (c < nx) {
                    const float4 w = *wp;
                    *reinterpret_cast<float4 *>(S + (k * C::NXM + c) * C::TP + cg * 4) =
                        make_float4(acc[k][m][0] + w.x, acc[k][m][1] + w.y, acc[k][m][2] + w.z, acc[k][m][3] + w.w);
                } else {
                    *wp = make_float4(-ipi * acc[k][m][0], -ipi * acc[k][m][1], -ipi * acc[k][m][2], -ipi * acc[k][m][3]);
                }
            }
    }
    __syncthreads();
    // coalesced write-out of ubar and s
    for_kcr<NR, TC, NT>(nxu, [&](int k, int col, int c) {
        if (!ci.ok[col]) return;
        const int i = ci.node[col];
        if (c < nx)
            a.s[k * a.s_stride + ci.sb[col] + (long long)i * nx + c] = S[(k * C::NXM + c) * C::TP + col];
        else
            a.ubar[k * a.u_stride + ci.ub[col] + (long long)i * nu + c - nx] = Wb[(k * XU + c) * C::TP + col];
    });
}

// Forward tile: nodes of stage t.  x from the parent's tile (or x0 at the root); u = K x + ubar;
// h = S [x; u]; every child j gets x^j = A x + B u + c^j.  Leaves (t = N) only write h.  Every
// global read (x, ubar, and the only child's c on non-branching stages) is one gather.
template <int NR, int TC, int XU, int NT>
__device__ __forceinline__ void fwd_tile(const RoundArgs<NR> &a, const RTask &tk, float *sm, ColInfo<TC> &ci,
                                         int &staged) {
    using C = Cfg<TC, XU, NT>;
    const int t = tk.stage;
    const Geo q = load_geo(a.groups[tk.group], t);
    const int nx = q.nx, nu = q.nu, nxu = q.nxu;
    float *Gs = sm;
    float *Ks = Gs + C::NXM * XU;
    float *X = sm + C::MAT;                 // [k][row][col]: x then u per column
    float *UB = X + NR * XU * C::TP;        // [k][a][col]: ubar
    float *CB = UB + NR * C::NUM * C::TP;   // [k][r][col]: c of the only child (one child per node)
    const bool leaf = q.s0 >= q.Np;
    const int bt = q.bt;
    const bool one_child = !leaf && bt == 1 && !a.homog;
    load_cols<NR, TC>(a, q, tk, ci);
    if (!__syncthreads_or(threadIdx.x < TC ? ci.ok[threadIdx.x] : 0)) return;
    const int key = 2 * (tk.group * (kMaxStages + 1) + t) + 1;
    if (staged != key) {
        for (int e = threadIdx.x; e < nx * nxu; e += NT) cp4(Gs + e, q.G + e);
        if (!leaf)
            for (int e = threadIdx.x; e < nu * nx; e += NT) cp4(Ks + e, q.Kt + (size_t)t * nu * nx + e);
        staged = key;
    }
    {
        // rows r < nx: x; nx <= r < nx + nu: ubar (nonleaf); nx + nu <= r: c of the only child
        const int R = leaf ? nx : (one_child ? nxu + nx : nxu);
        gather_kcr<NR, TC, NT, 4>(
            R,
            [&](int k, int col, int r) -> float {
                if (!ci.ok[col]) return 0.f;
                const int i = ci.node[col];
                if (r < nx) {
                    if (t == 0) {
                        const int inst = (tk.col0 + col) / q.n_t;
                        return a.homog ? 0.f : a.x0[(long long)(q.inst0 + inst) * 64 + r];
                    }
                    return __ldcg(a.xs + k * a.s_stride + ci.sb[col] + (long long)i * nx + r);
                }
                if (r < nxu) return __ldcg(a.ubar + k * a.u_stride + ci.ub[col] + (long long)i * nu + r - nx);
                const int j = q.s1 + (i - q.s0);
                return a.c[ci.sb[col] + (long long)j * nx + r - nxu];
            },
            [&](int k, int col, int r, float v) {
                if (r < nx)
                    X[(k * XU + r) * C::TP + col] = v;
                else if (r < nxu)
                    UB[(k * C::NUM + r - nx) * C::TP + col] = v;
                else
                    CB[(k * C::NXM + r - nxu) * C::TP + col] = v;
            });
    }
    cp_wait();
    __syncthreads();
    const int cg = threadIdx.x % C::CG, rg = threadIdx.x / C::CG;
    const float sc = a.scaled ? q.sq_t : 1.f;
    if (!leaf) {
        // u = K x + ubar (rows a of u over the row groups)
        const int mu = (nu + C::RG - 1) / C::RG, a0 = rg * mu;
        float u[NR][C::MU][4];
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int m = 0; m < C::MU; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) u[k][m][q] = 0.f;
        for (int r = 0; r < nx; ++r) {
            float4 x4[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k)
                x4[k] = *reinterpret_cast<const float4 *>(X + (k * XU + r) * C::TP + cg * 4);
#pragma unroll
            for (int m = 0; m < C::MU; ++m)
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
        for (int m = 0; m < C::MU; ++m)
            if (m < mu && a0 + m < nu)
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const float4 w = *reinterpret_cast<const float4 *>(UB + (k * C::NUM + a0 + m) * C::TP + cg * 4);
                    *reinterpret_cast<float4 *>(X + (k * XU + nx + a0 + m) * C::TP + cg * 4) =
                        make_float4(u[k][m][0] + w.x, u[k][m][1] + w.y, u[k][m][2] + w.z, u[k][m][3] + w.w);
                }
        __syncthreads();
    }
    // h for the stage's nodes
    const int rows = leaf ? nx : nxu;
    for_kcr<NR, TC, NT>(rows, [&](int k, int col, int r) {
        if (ci.ok[col]) a.h[k][ci.elem[col] + doff(q, ci.node[col]) + r] = sc * X[(k * XU + r) * C::TP + col];
    });
    if (leaf) return;
    // children: x^j = [A | B][x; u] + c^j (rows r of x over the row groups)
    const int mx = (nx + C::RG - 1) / C::RG, x0r = rg * mx;
    float acc[NR][C::MX][4];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int m = 0; m < C::MX; ++m)
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
                    x4[k][u] = *reinterpret_cast<const float4 *>(X + (k * XU + qq + u) * C::TP + cg * 4);
#pragma unroll
            for (int m = 0; m < C::MX; ++m)
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
        for (int k = 0; k < NR; ++k) x4[k] = *reinterpret_cast<const float4 *>(X + (k * XU + qq) * C::TP + cg * 4);
#pragma unroll
        for (int m = 0; m < C::MX; ++m)
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
    // the children's states over CB (this thread alone reads the CB entries it overwrites)
#pragma unroll
    for (int m = 0; m < C::MX; ++m)
        if (m < mx && x0r + m < nx)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                float4 *cp = reinterpret_cast<float4 *>(CB + (k * C::NXM + x0r + m) * C::TP + cg * 4);
                float4 v = make_float4(acc[k][m][0], acc[k][m][1], acc[k][m][2], acc[k][m][3]);
                if (one_child) {
                    const float4 w = *cp;
                    v.x += w.x;
                    v.y += w.y;
                    v.z += w.z;
                    v.w += w.w;
                }
                *cp = v;
            }
    __syncthreads();
    for_kcr<NR, TC, NT>(nx, [&](int k, int col, int r) {
        if (ci.ok[col]) {
            const int i = ci.node[col];
            const int j0 = q.s1 + (i - q.s0) * bt;
            const float xv = CB[(k * C::NXM + r) * C::TP + col];
            if (one_child || a.homog) {
                a.xs[k * a.s_stride + ci.sb[col] + (long long)j0 * nx + r] = xv;
                for (int j = j0 + 1; j < j0 + bt; ++j) a.xs[k * a.s_stride + ci.sb[col] + (long long)j * nx + r] = xv;
            } else {
                for (int j = j0; j < j0 + bt; ++j)
                    a.xs[k * a.s_stride + ci.sb[col] + (long long)j * nx + r] = xv + a.c[ci.sb[col] + (long long)j * nx + r];
            }
        }
    });
}

// One solve round as one persistent launch over the round's tiles (see above).  Thread 0 draws the
// next ticket while the CTA works on the current tile; a CTA that holds a drawn ticket is working
// on a lower one, so the holder of the lowest unfinished ticket is always working on it.
template <int NR, int TC, int XU, int NT>
__global__ void __launch_bounds__(NT) k_bround(RoundArgs<NR> a) {
    extern __shared__ __align__(16) float bsm[];
    __shared__ ColInfo<TC> ci;
    __shared__ int s_tick[2];
    int staged = -1;  // (group, stage, pass) whose matrices sit in shared memory
    if (threadIdx.x == 0) s_tick[0] = (int)atomicAdd(a.ticket, 1u);
    __syncthreads();
    for (int it = 0;; ++it) {
        const int k = s_tick[it & 1];
        if (k >= a.ntasks) return;
        const RTask tk = a.tasks[k];
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) s_tick[(it + 1) & 1] = (int)atomicAdd(a.ticket, 1u);
            wait_deps(a, tk);
        }
        __syncthreads();
        if (tk.pass == 0)
            bwd_tile<NR, TC, XU, NT>(a, tk, bsm, ci, staged);
        else
            fwd_tile<NR, TC, XU, NT>(a, tk, bsm, ci, staged);
        // every thread's stores of the tile precede thread 0's fence and count
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.ctrs + k, 1u);
        }
    }
}

// Row access of the column kernel: n (runtime, at most N) consecutive floats at p, with 16- or
// 8-byte vector accesses when al = 4 or 2 (p aligned to al floats and al dividing n); the entries
// of d beyond n are zero.  cg: read through L2 (data other CTAs write during the round).
template <int N>
__device__ __forceinline__ void row_load(float (&d)[N], const float *p, int n, int al, bool cg) {
    if (al == 4) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * q < n) v = cg ? __ldcg(reinterpret_cast<const float4 *>(p) + q) : reinterpret_cast<const float4 *>(p)[q];
            d[4 * q] = v.x;
            d[4 * q + 1] = v.y;
            d[4 * q + 2] = v.z;
            d[4 * q + 3] = v.w;
        }
    } else if (al == 2) {
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            float2 v = make_float2(0.f, 0.f);
            if (2 * q < n) v = cg ? __ldcg(reinterpret_cast<const float2 *>(p) + q) : reinterpret_cast<const float2 *>(p)[q];
            d[2 * q] = v.x;
            d[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r) d[r] = r < n ? (cg ? __ldcg(p + r) : p[r]) : 0.f;
    }
}
template <int N>
__device__ __forceinline__ void row_store(float *p, const float (&v)[N], int n, int al) {
    if (al == 4) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            if (4 * q < n) reinterpret_cast<float4 *>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if (al == 2) {
#pragma unroll
        for (int q = 0; q < N / 2; ++q)
            if (2 * q < n) reinterpret_cast<float2 *>(p)[q] = make_float2(v[2 * q], v[2 * q + 1]);
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r)
            if (r < n) p[r] = v[r];
    }
}

// Column kernel: one (node, instance) column per thread, for batches whose groups all have
// nx <= NXP and nu <= NUP (NXP, NUP compile-time).  The stage matrices sit in shared memory
// zero-padded to the compile-time widths (A columns at [0, NXP), B columns at [NXP, NXP + NUP)),
// so every product runs over registers with fixed indices; all threads read the same matrix
// entry at once (a broadcast).  A thread loads its own column's vectors, so a tile needs no
// barrier beyond the matrices' staging.  Tiles and their ticket order are those of k_bround
// with NT columns per tile.
template <int NXP, int NUP>
__device__ __forceinline__ void col_stage(const Geo &q, int t, bool leaf, float *Gp, float *Kp, float *Rp, int NT) {
    const int nx = q.nx, nu = q.nu, nxu = q.nxu;
    for (int e = threadIdx.x; e < NXP * (NXP + NUP); e += NT) {
        const int r = e / (NXP + NUP), c = e - r * (NXP + NUP);
        const int gc = c < NXP ? (c < nx ? c : -1) : (c - NXP < nu ? nx + c - NXP : -1);
        if (r < nx && gc >= 0)
            cp4(Gp + e, q.G + r * nxu + gc);
        else
            Gp[e] = 0.f;
    }
    if (!leaf) {
        for (int e = threadIdx.x; e < NUP * NXP; e += NT) {
            const int aa = e / NXP, c = e - aa * NXP;
            if (aa < nu && c < nx)
                cp4(Kp + e, q.Kt + (size_t)t * nu * nx + aa * nx + c);
            else
                Kp[e] = 0.f;
        }
        for (int e = threadIdx.x; e < NUP * NUP; e += NT) {
            const int aa = e / NUP, bb = e - aa * NUP;
            if (aa < nu && bb < nu)
                cp4(Rp + e, q.Ri + (size_t)t * nu * nu + aa * nu + bb);
            else
                Rp[e] = 0.f;
        }
    }
}

template <int NR, int NXP, int NUP>
__device__ __forceinline__ void col_bwd(const RoundArgs<NR> &a, const Geo &q, int t, int inst, int i,
                                        const float *Gp, const float *Kp, const float *Rp) {
    constexpr int NXU = NXP + NUP;
    const int nx = q.nx, nu = q.nu;
    const long long elem = q.elem0 + (long long)inst * q.m;
    const long long sb = q.sbase + (long long)inst * q.Nn * nx;
    const long long ub = q.ubase + (long long)inst * q.Np * nu;
    const bool leaf_children = q.s1 >= q.Np;
    const int j0 = q.s1 + (i - q.s0) * q.bt;
    const float sc = a.scaled ? q.sq_t : 1.f, scc = a.scaled ? q.sq_t1 : 1.f;
    const float ipi = 1.f / q.pi_t;
    const long long oi = elem + doff(q, i);
#pragma unroll 1
    for (int k = 0; k < NR; ++k) {
        // S = sum of the children's s (or the leaves' y / 2), then o = [A | B]' S
        float S[NXP];
        if (leaf_children) {
            row_load<NXP>(S, a.y[k] + elem + doff(q, j0), nx, q.al_d, false);
#pragma unroll
            for (int r = 0; r < NXP; ++r) S[r] *= 0.5f * scc;
        } else {
            row_load<NXP>(S, a.s + k * a.s_stride + sb + (long long)j0 * nx, nx, q.al_s, true);
        }
        for (int j = j0 + 1; j < j0 + q.bt; ++j) {
            float Sj[NXP];
            if (leaf_children) {
                row_load<NXP>(Sj, a.y[k] + elem + doff(q, j), nx, q.al_d, false);
#pragma unroll
                for (int r = 0; r < NXP; ++r) S[r] += 0.5f * scc * Sj[r];
            } else {
                row_load<NXP>(Sj, a.s + k * a.s_stride + sb + (long long)j * nx, nx, q.al_s, true);
#pragma unroll
                for (int r = 0; r < NXP; ++r) S[r] += Sj[r];
            }
        }
        float o[NXU];
#pragma unroll
        for (int c = 0; c < NXU; ++c) o[c] = 0.f;
#pragma unroll
        for (int r = 0; r < NXP; ++r) {
            const float sr = S[r];
#pragma unroll
            for (int c4 = 0; c4 < NXU / 4; ++c4) {
                const float4 g = *reinterpret_cast<const float4 *>(Gp + r * NXU + 4 * c4);
                o[4 * c4 + 0] = fmaf(g.x, sr, o[4 * c4 + 0]);
                o[4 * c4 + 1] = fmaf(g.y, sr, o[4 * c4 + 1]);
                o[4 * c4 + 2] = fmaf(g.z, sr, o[4 * c4 + 2]);
                o[4 * c4 + 3] = fmaf(g.w, sr, o[4 * c4 + 3]);
            }
        }
        // v = o_B + y_u/2 + gu
        const float *yi = a.y[k] + oi;
        const float *gi = a.gam + oi;
        float v[NUP], w[NUP];
        row_load<NUP>(v, yi + nx, nu, q.al_d, false);
        if (!a.homog) row_load<NUP>(w, gi + nx, nu, q.al_d, false);
#pragma unroll
        for (int aa = 0; aa < NUP; ++aa) v[aa] = o[NXP + aa] + 0.5f * sc * v[aa] + (a.homog ? 0.f : w[aa]);
        // ubar = -(1/pi) R~^-1 v
        {
            float ubv[NUP];
#pragma unroll
            for (int aa = 0; aa < NUP; ++aa) {
                float acc = 0.f;
#pragma unroll
                for (int b4 = 0; b4 < NUP / 4; ++b4) {
                    const float4 rr = *reinterpret_cast<const float4 *>(Rp + aa * NUP + 4 * b4);
                    acc = fmaf(rr.x, v[4 * b4 + 0], acc);
                    acc = fmaf(rr.y, v[4 * b4 + 1], acc);
                    acc = fmaf(rr.z, v[4 * b4 + 2], acc);
                    acc = fmaf(rr.w, v[4 * b4 + 3], acc);
                }
                ubv[aa] = -ipi * acc;
            }
            row_store<NUP>(a.ubar + k * a.u_stride + ub + (long long)i * nu, ubv, nu, q.al_u);
        }
        // s = o_A + K'v + y_x/2 + gx
#pragma unroll
        for (int aa = 0; aa < NUP; ++aa) {
            const float va = v[aa];
#pragma unroll
            for (int c4 = 0; c4 < NXP / 4; ++c4) {
                const float4 kk = *reinterpret_cast<const float4 *>(Kp + aa * NXP + 4 * c4);
                o[4 * c4 + 0] = fmaf(kk.x, va, o[4 * c4 + 0]);
                o[4 * c4 + 1] = fmaf(kk.y, va, o[4 * c4 + 1]);
                o[4 * c4 + 2] = fmaf(kk.z, va, o[4 * c4 + 2]);
                o[4 * c4 + 3] = fmaf(kk.w, va, o[4 * c4 + 3]);
            }
        }
        {
            float wx[NXP], gx[NXP];
            row_load<NXP>(wx, yi, nx, q.al_d, false);
            if (!a.homog) row_load<NXP>(gx, gi, nx, q.al_d, false);
#pragma unroll
            for (int r = 0; r < NXP; ++r) wx[r] = o[r] + 0.5f * sc * wx[r] + (a.homog ? 0.f : gx[r]);
            row_store<NXP>(a.s + k * a.s_stride + sb + (long long)i * nx, wx, nx, q.al_s);
        }
    }
}

template <int NR, int NXP, int NUP>
__device__ __forceinline__ void col_fwd(const RoundArgs<NR> &a, const Geo &q, int t, int inst, int i,
                                        const float *Gp, const float *Kp) {
    constexpr int NXU = NXP + NUP;
    const int nx = q.nx, nu = q.nu;
    const long long elem = q.elem0 + (long long)inst * q.m;
    const long long sb = q.sbase + (long long)inst * q.Nn * nx;
    const long long ub = q.ubase + (long long)inst * q.Np * nu;
    const bool leaf = q.s0 >= q.Np;
    const float sc = a.scaled ? q.sq_t : 1.f;
    const long long oi = elem + doff(q, i);
#pragma unroll 1
    for (int k = 0; k < NR; ++k) {
        float x[NXP], u[NUP];
        if (t == 0) {
            if (a.homog) {
#pragma unroll
                for (int r = 0; r < NXP; ++r) x[r] = 0.f;
            } else {
                row_load<NXP>(x, a.x0 + (long long)(q.inst0 + inst) * 64, nx, (nx & 3) == 0 ? 4 : 1, false);
            }
        } else {
            row_load<NXP>(x, a.xs + k * a.s_stride + sb + (long long)i * nx, nx, q.al_s, true);
        }
        float *hi = a.h[k] + oi;
        if (leaf) {
            float hx[NXP];
#pragma unroll
            for (int r = 0; r < NXP; ++r) hx[r] = sc * x[r];
            row_store<NXP>(hi, hx, nx, q.al_d);
            continue;
        }
        row_load<NUP>(u, a.ubar + k * a.u_stride + ub + (long long)i * nu, nu, q.al_u, true);
        // u = K x + ubar
#pragma unroll
        for (int aa = 0; aa < NUP; ++aa) {
            float acc = u[aa];
#pragma unroll
            for (int c4 = 0; c4 < NXP / 4; ++c4) {
                const float4 kk = *reinterpret_cast<const float4 *>(Kp + aa * NXP + 4 * c4);
                acc = fmaf(kk.x, x[4 * c4 + 0], acc);
                acc = fmaf(kk.y, x[4 * c4 + 1], acc);
                acc = fmaf(kk.z, x[4 * c4 + 2], acc);
                acc = fmaf(kk.w, x[4 * c4 + 3], acc);
            }
            u[aa] = aa < nu ? acc : 0.f;
        }
        {
            float hx[NXP], hu[NUP];
#pragma unroll
            for (int r = 0; r < NXP; ++r) hx[r] = sc * x[r];
#pragma unroll
            for (int aa = 0; aa < NUP; ++aa) hu[aa] = sc * u[aa];
            row_store<NXP>(hi, hx, nx, q.al_d);
            row_store<NUP>(hi + nx, hu, nu, q.al_d);
        }
        // children: x^j = [A | B][x; u] + c^j
        float xc[NXP];
#pragma unroll
        for (int r = 0; r < NXP; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < NXP / 4; ++c4) {
                const float4 g = *reinterpret_cast<const float4 *>(Gp + r * NXU + 4 * c4);
                acc = fmaf(g.x, x[4 * c4 + 0], acc);
                acc = fmaf(g.y, x[4 * c4 + 1], acc);
                acc = fmaf(g.z, x[4 * c4 + 2], acc);
                acc = fmaf(g.w, x[4 * c4 + 3], acc);
            }
#pragma unroll
            for (int a4 = 0; a4 < NUP / 4; ++a4) {
                const float4 g = *reinterpret_cast<const float4 *>(Gp + r * NXU + NXP + 4 * a4);
                acc = fmaf(g.x, u[4 * a4 + 0], acc);
                acc = fmaf(g.y, u[4 * a4 + 1], acc);
                acc = fmaf(g.z, u[4 * a4 + 2], acc);
                acc = fmaf(g.w, u[4 * a4 + 3], acc);
            }
            xc[r] = acc;
        }
        const int j0 = q.s1 + (i - q.s0) * q.bt;
        for (int j = j0; j < j0 + q.bt; ++j) {
            float xj[NXP];
            if (a.homog) {
#pragma unroll
                for (int r = 0; r < NXP; ++r) xj[r] = xc[r];
            } else {
                row_load<NXP>(xj, a.c + sb + (long long)j * nx, nx, q.al_s, false);
#pragma unroll
                for (int r = 0; r < NXP; ++r) xj[r] += xc[r];
            }
            row_store<NXP>(a.xs + k * a.s_stride + sb + (long long)j * nx, xj, nx, q.al_s);
        }
    }
}

template <int NR, int NXP, int NUP, int NT>
__global__ void __launch_bounds__(NT, 4) k_bcol(RoundArgs<NR> a) {
    __shared__ __align__(16) float Gp[NXP * (NXP + NUP)];
    __shared__ __align__(16) float Kp[NUP * NXP];
    __shared__ __align__(16) float Rp[NUP * NUP];
    __shared__ int s_tick[2];
    int staged = -1;
    if (threadIdx.x == 0) s_tick[0] = (int)atomicAdd(a.ticket, 1u);
    __syncthreads();
    for (int it = 0;; ++it) {
        const int k = s_tick[it & 1];
        if (k >= a.ntasks) return;
        const RTask tk = a.tasks[k];
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) s_tick[(it + 1) & 1] = (int)atomicAdd(a.ticket, 1u);
            wait_deps(a, tk);
        }
        const int t = tk.stage;
        const Geo q = load_geo(a.groups[tk.group], t);
        const int key = 2 * (tk.group * (kMaxStages + 1) + t) + tk.pass;
        if (staged != key) {
            __syncthreads();  // every thread is done with the previous matrices
            col_stage<NXP, NUP>(q, t, q.s0 >= q.Np, Gp, Kp, Rp, NT);
            staged = key;
        }
        cp_wait();
        __syncthreads();  // the matrices, the next ticket and the dependency wait
        const int col = threadIdx.x;
        if (col < tk.ncols) {
            const int cc = tk.col0 + col, inst = cc / q.n_t, i = q.s0 + cc - inst * q.n_t;
            if (!a.active || a.active[q.inst0 + inst]) {
                if (tk.pass == 0)
                    col_bwd<NR, NXP, NUP>(a, q, t, inst, i, Gp, Kp, Rp);
                else
                    col_fwd<NR, NXP, NUP>(a, q, t, inst, i, Gp, Kp);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.ctrs + k, 1u);
        }
    }
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

// Tile variants: 0-2 the tile kernel (k_bround) with 32 columns on 128 or 256 threads or 64 columns
// on 256 threads; 3 the column kernel (k_bcol, one column per thread, 128 columns per tile), for
// batches whose groups all have nx <= 32 and nu <= 16.
constexpr int kTileVars = 4;
constexpr int kTileCols[kTileVars] = {32, 32, 64, 128};         // columns per tile of each variant
constexpr int kTileThreads[kTileVars] = {128, 256, 256, 128};   // threads per CTA of each variant
constexpr int kColVar = 3;

struct stobatch_s {
    std::vector<sto_group_desc> desc;
    std::vector<GroupDev> groups;   // host copies (device pointers filled at bind)
    std::vector<InstDev> insts;
    std::vector<int> blk_inst;
    std::vector<Task> tasks;                // set-up (gamma) tiles
    std::vector<int> bwd_phase, fwd_phase;  // task offsets per phase (size phases + 1)
    std::vector<int> gam_phase;
    // solve rounds: tiles of kTileCols[v] columns (tile variant v) in ticket order, and the
    // number of per-(group, stage, pass) counters they wait on
    std::vector<RTask> rtasks[kTileVars];
    int nctr = 0;
    int xu = 96;                          // shape class: 48 if every group has nx <= 32, nu <= 16
    int nxp = 32, nup = 16;               // the column kernel's padded widths (when xu == 48)
    int tile_var[3] = {1, 1, 1};          // variant per right-hand-side count (set by the tuner)
    double tuned_ms[3][kTileVars] = {};   // round time of each variant, measured by the tuner
    int grid[3][kTileVars] = {};          // CTAs of one wave per (right-hand sides, variant)
    bool tuned = false;
    size_t o_rtask[kTileVars] = {}, o_ctr = 0;
    int maxN = 0, ninst = 0, nblocks = 0;
    long long M = 0, vpad = 0, Ssz = 0, Usz = 0;  // vector length, padded stride, scratch sizes
    // layout (byte offsets)
    size_t o_groups, o_insts, o_blk, o_tasks, o_G, o_K, o_R, o_box, o_W, o_AB64, o_P64, o_scr, o_off, o_gam, o_c,
        o_x0, o_s, o_ub, o_xs, o_vec, o_ringS, o_ringY, o_part, o_sc, o_active, o_nact, o_status, o_sqn, total;
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

namespace {
sto_status tune_rounds(stobatch_t b, cudaStream_t st);
}

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
    // widest vector access every instance's rows allow (the arrays start 256-byte aligned)
    auto widest = [](std::initializer_list<long long> vals) {
        for (int p : {4, 2}) {
            bool ok = true;
            for (long long v : vals) ok = ok && v % p == 0;
            if (ok) return p;
        }
        return 1;
    };
    for (auto &g : b->groups) {
        g.al_d = widest({g.nx, g.nu, (long long)g.m, g.elem0, b->vpad});
        g.al_s = widest({g.nx, g.sbase, (long long)g.Nn * g.nx, sb});
        g.al_u = widest({g.nu, g.ubase, (long long)g.Np * g.nu, ub});
    }
    // set-up tiles: backward phase p = stage N_g - 1 - p (gamma covers every nonleaf stage)
    auto add_tasks = [&](int gi, int t) {
        const GroupDev &g = b->groups[gi];
        const int cols = (g.soff[t + 1] - g.soff[t]) * g.I;
        for (int c0 = 0; c0 < cols; c0 += kGC) b->tasks.push_back(Task{gi, t, c0, std::min(kGC, cols - c0)});
    };
    // solve-round tiles in ticket order, per tile variant: backward by height, then forward by
    // depth; first[cbase[g] + pass (N_g + 1) + t] = ticket of the first tile of (g, t, pass)
    std::vector<int> cbase(ngroups);
    int nsets = 0;
    b->xu = 48;
    int maxnx = 0, maxnu = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
        cbase[gi] = nsets;
        nsets += 2 * (b->groups[gi].N + 1);
        if (b->groups[gi].nx > 32 || b->groups[gi].nu > 16) b->xu = 96;
        maxnx = std::max(maxnx, b->groups[gi].nx);
        maxnu = std::max(maxnu, b->groups[gi].nu);
    }
    b->nxp = maxnx <= 16 ? 16 : (maxnx <= 24 ? 24 : 32);
    b->nup = maxnu <= 8 ? 8 : 16;
    b->nctr = 0;
    for (int v = 0; v < kTileVars; ++v) {
        const int tc = kTileCols[v];
        std::vector<int> first(nsets, -1);
        auto bt_of = [&](const GroupDev &g, int t) { return t < g.s ? g.b : 1; };  // children per node of stage t
        // tiles of (gi, t, pass) columns [c0, c0 + ncols); dep(c0, ncols) -> the dependency range
        auto add = [&](int gi, int t, int pass, auto dep) {
            const GroupDev &g = b->groups[gi];
            const int cols = (g.soff[t + 1] - g.soff[t]) * g.I;
            first[cbase[gi] + pass * (g.N + 1) + t] = (int)b->rtasks[v].size();
            for (int c0 = 0; c0 < cols; c0 += tc) {
                const int nc = std::min(tc, cols - c0);
                int d0 = -1, nd = 0;
                dep(c0, nc, d0, nd);
                b->rtasks[v].push_back(RTask{gi, t, c0, nc, pass, d0, nd, 0});
            }
        };
        for (int p = 0; p < b->maxN; ++p)
            for (int gi = 0; gi < ngroups; ++gi) {
                const GroupDev &g = b->groups[gi];
                if (g.N <= p) continue;
                const int t = g.N - 1 - p;
                add(gi, t, 0, [&](int c0, int nc, int &d0, int &nd) {
                    if (t + 1 >= g.N) return;  // children are leaves: s from y
                    const int bt = bt_of(g, t), f = first[cbase[gi] + t + 1];
                    const int lo = c0 * bt / tc, hi = ((c0 + nc) * bt - 1) / tc;
                    d0 = f + lo;
                    nd = hi - lo + 1;
                });
            }
        for (int p = 0; p <= b->maxN; ++p)
            for (int gi = 0; gi < ngroups; ++gi) {
                const GroupDev &g = b->groups[gi];
                if (g.N < p) continue;
                add(gi, p, 1, [&](int c0, int nc, int &d0, int &nd) {
                    if (p == 0) {  // the backward tile of stage 0 with the same columns
                        d0 = first[cbase[gi] + 0] + c0 / tc;
                        nd = 1;
                        return;
                    }
                    const int bp = bt_of(g, p - 1), f = first[cbase[gi] + (g.N + 1) + p - 1];
                    const int lo = c0 / bp / tc, hi = (c0 + nc - 1) / bp / tc;
                    d0 = f + lo;
                    nd = hi - lo + 1;
                });
            }
        b->nctr = std::max(b->nctr, (int)b->rtasks[v].size());
    }
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
    for (int v = 0; v < kTileVars; ++v) b->o_rtask[v] = add(b->rtasks[v].size() * sizeof(RTask));
    b->o_ctr = add((size_t)(b->nctr + 1) * 4);  // the tiles' done flags, then the ticket
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
    for (int v = 0; v < kTileVars; ++v)
        BCUDA(b, cudaMemcpyAsync(b->ws + b->o_rtask[v], b->rtasks[v].data(), b->rtasks[v].size() * sizeof(RTask),
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
    if (!b->tuned) {  // the round's tile shape, once per batch (shapes do not change)
        const sto_status s = tune_rounds(b, st);
        if (s != STO_OK) return s;
        b->tuned = true;
    }
    return STO_OK;
}

STO_API sto_status stobatch_round_status(stobatch_t b, sto_stream_t stream) {
    if (!b) return STO_ERR_INVALID_ARG;
    if (!b->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int err = 0;
    BCUDA(b, cudaMemcpyAsync(&err, b->at<int>(b->o_nact) + 1, 4, cudaMemcpyDeviceToHost, st));
    BCUDA(b, cudaStreamSynchronize(st));
    if (!err) return STO_OK;
    BCUDA(b, cudaMemsetAsync(b->at<int>(b->o_nact) + 1, 0, 4, st));
    BCUDA(b, cudaStreamSynchronize(st));
    b->err = "a batched solve round gave up waiting for a dependency";
    return STO_ERR_TIMEOUT;
}

STO_API sto_status stobatch_set_round_variant(stobatch_t b, int32_t nrhs, int32_t variant) {
    if (!b || nrhs < 1 || nrhs > 2 || variant < 0 || variant >= kTileVars) return STO_ERR_INVALID_ARG;
    if (variant == kColVar && b->xu == 96) return STO_ERR_INVALID_ARG;
    b->tile_var[nrhs] = variant;
    return STO_OK;
}

STO_API sto_status stobatch_round_config(stobatch_t b, int32_t nrhs, int32_t *tile_cols, int32_t *cta_threads,
                                         int32_t *ctas, double *tuned_ms) {
    if (!b || nrhs < 1 || nrhs > 2) return STO_ERR_INVALID_ARG;
    const int v = b->tile_var[nrhs];
    if (tile_cols) *tile_cols = kTileCols[v];
    if (cta_threads) *cta_threads = kTileThreads[v];
    if (ctas) *ctas = b->grid[nrhs][v];
    if (tuned_ms)
        for (int k = 0; k < kTileVars; ++k) tuned_ms[k] = b->tuned_ms[nrhs][k];
    return STO_OK;
}

}  // extern "C"

namespace {

template <int NR>
RoundArgs<NR> round_args(stobatch_t b, const float *y0, const float *y1, float *h0, float *h1, bool homog,
                         bool scaled, const int *active, int var) {
    RoundArgs<NR> a;
    a.groups = b->at<GroupDev>(b->o_groups);
    a.insts = b->at<InstDev>(b->o_insts);
    a.tasks = b->at<RTask>(b->o_rtask[var]);
    a.ntasks = (int)b->rtasks[var].size();
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
    a.s_stride = b->Ssz;
    a.u_stride = b->Usz;
    a.active = active;
    a.ctrs = b->at<unsigned>(b->o_ctr);
    a.ticket = a.ctrs + b->nctr;
    a.err = b->at<int>(b->o_nact) + 1;
    a.homog = homog ? 1 : 0;
    a.scaled = scaled ? 1 : 0;
    return a;
}

// One wave of the round kernel (every CTA resident: tiles wait only on earlier tickets).
template <int NR, int TC, int XU, int NT>
int round_grid(int ntasks) {
    const size_t smem = round_smem<NR, TC, XU, NT>();
    raise_smem_cap((const void *)k_bround<NR, TC, XU, NT>, smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bround<NR, TC, XU, NT>, NT, smem) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return std::max(1, std::min(per_sm * sms, ntasks));
}

template <int NR, int TC, int XU, int NT>
void round_launch(const RoundArgs<NR> &a, int grid, cudaStream_t st) {
    k_bround<NR, TC, XU, NT><<<grid, NT, round_smem<NR, TC, XU, NT>(), st>>>(a);
}

template <int NR, int NXP, int NUP>
int col_grid(int ntasks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bcol<NR, NXP, NUP, 128>, 128, 0) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return std::max(1, std::min(per_sm * sms, ntasks));
}
template <int NR>
int col_grid_for(int nxp, int nup, int ntasks) {
    if (nup == 8) return nxp == 16 ? col_grid<NR, 16, 8>(ntasks) : (nxp == 24 ? col_grid<NR, 24, 8>(ntasks) : col_grid<NR, 32, 8>(ntasks));
    return nxp == 16 ? col_grid<NR, 16, 16>(ntasks) : (nxp == 24 ? col_grid<NR, 24, 16>(ntasks) : col_grid<NR, 32, 16>(ntasks));
}
template <int NR>
void col_launch_for(int nxp, int nup, const RoundArgs<NR> &a, int grid, cudaStream_t st) {
    if (nup == 8) {
        if (nxp == 16) k_bcol<NR, 16, 8, 128><<<grid, 128, 0, st>>>(a);
        else if (nxp == 24) k_bcol<NR, 24, 8, 128><<<grid, 128, 0, st>>>(a);
        else k_bcol<NR, 32, 8, 128><<<grid, 128, 0, st>>>(a);
    } else {
        if (nxp == 16) k_bcol<NR, 16, 16, 128><<<grid, 128, 0, st>>>(a);
        else if (nxp == 24) k_bcol<NR, 24, 16, 128><<<grid, 128, 0, st>>>(a);
        else k_bcol<NR, 32, 16, 128><<<grid, 128, 0, st>>>(a);
    }
}

// The kernel of tile variant v (kTileCols[v] columns, kTileThreads[v] threads) for the batch's
// shape class: grid of one wave, or a launch.
template <int NR, int XU>
int variant_grid(int v, int ntasks) {
    switch (v) {
        case 0: return round_grid<NR, 32, XU, 128>(ntasks);
        case 1: return round_grid<NR, 32, XU, 256>(ntasks);
        default: return round_grid<NR, 64, XU, 256>(ntasks);
    }
}
template <int NR, int XU>
void variant_launch(int v, const RoundArgs<NR> &a, int grid, cudaStream_t st) {
    switch (v) {
        case 0: round_launch<NR, 32, XU, 128>(a, grid, st); break;
        case 1: round_launch<NR, 32, XU, 256>(a, grid, st); break;
        default: round_launch<NR, 64, XU, 256>(a, grid, st); break;
    }
}

// The round's counters and ticket start at zero, then one persistent launch.
template <int NR>
sto_status launch_round(stobatch_t b, const RoundArgs<NR> &a, int var, cudaStream_t st) {
    int &grid = b->grid[NR][var];
    const bool big = b->xu == 96;
    if (var == kColVar && big) {
        b->err = "the column kernel needs nx <= 32 and nu <= 16 in every group";
        return STO_ERR_INVALID_ARG;
    }
    if (grid == 0) {
        if (var == kColVar)
            grid = col_grid_for<NR>(b->nxp, b->nup, a.ntasks);
        else
            grid = big ? variant_grid<NR, 96>(var, a.ntasks) : variant_grid<NR, 48>(var, a.ntasks);
        if (grid <= 0) {
            b->err = "batched round kernel does not fit on this device";
            return STO_ERR_CUDA;
        }
    }
    BCUDA(b, cudaMemsetAsync(a.ctrs, 0, (size_t)(b->nctr + 1) * 4, st));
    if (var == kColVar)
        col_launch_for<NR>(b->nxp, b->nup, a, grid, st);
    else if (big)
        variant_launch<NR, 96>(var, a, grid, st);
    else
        variant_launch<NR, 48>(var, a, grid, st);
    return STO_OK;
}

// One solve round for nrhs (1 or 2) right-hand sides with the tuned tile variant, replayed from
// a cached CUDA graph (the counters' reset and the persistent launch).
sto_status bround(stobatch_t b, const float *y0, const float *y1, float *h0, float *h1, int nrhs, bool homog,
                  bool scaled, const int *active, cudaStream_t st) {
    const int var = b->tile_var[nrhs];
    auto key = std::make_tuple((const void *)y0, (const void *)y1, (const void *)h0, (const void *)h1,
                               (const void *)active, nrhs * 8 + var, (int)homog, (int)scaled);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaStream_t cap;
        BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        BCUDA(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        sto_status ls;
        if (nrhs == 1)
            ls = launch_round<1>(b, round_args<1>(b, y0, y1, h0, h1, homog, scaled, active, var), var, cap);
        else
            ls = launch_round<2>(b, round_args<2>(b, y0, y1, h0, h1, homog, scaled, active, var), var, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (ls != STO_OK || e != cudaSuccess) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            return ls != STO_OK ? ls : bfail(b, e, "capture of a batched solve round");
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

// Round tuner: times a homogeneous round of every tile variant that fits the batch's shapes, for
// one and for two right-hand sides, on zeroed scratch vectors (one launch to warm up, then the
// mean of three) and keeps the fastest per right-hand-side count.
sto_status tune_rounds(stobatch_t b, cudaStream_t st) {
    const long long vs = b->vpad;
    float *V = b->at<float>(b->o_vec);
    float *y = V + 6 * vs, *h0 = V + 7 * vs, *h1 = V + 5 * vs;
    BCUDA(b, cudaMemsetAsync(y, 0, (size_t)vs * 4, st));
    cudaEvent_t e0, e1;
    BCUDA(b, cudaEventCreate(&e0));
    BCUDA(b, cudaEventCreate(&e1));
    sto_status s = STO_OK;
    for (int nr = 1; nr <= 2 && s == STO_OK; ++nr) {
        double best = 1e30;
        for (int v = 0; v < kTileVars && s == STO_OK; ++v) {
            if (v == kColVar && b->xu == 96) {
                b->tuned_ms[nr][v] = -1.0;  // not applicable to this batch's shapes
                continue;
            }
            for (int rep = 0; rep < 4 && s == STO_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, st);
                if (nr == 1)
                    s = launch_round<1>(b, round_args<1>(b, y, nullptr, h0, nullptr, true, true, nullptr, v), v, st);
                else
                    s = launch_round<2>(b, round_args<2>(b, y, y, h0, h1, true, true, nullptr, v), v, st);
            }
            if (s != STO_OK) break;
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                s = bfail(b, e, "timing a batched round");
                break;
            }
            b->tuned_ms[nr][v] = ms / 3.0;
            if (ms / 3.0 < best) {
                best = ms / 3.0;
                b->tile_var[nr] = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != STO_OK) return s;
    int err = 0;
    BCUDA(b, cudaMemcpyAsync(&err, b->at<int>(b->o_nact) + 1, 4, cudaMemcpyDeviceToHost, st));
    BCUDA(b, cudaStreamSynchronize(st));
    if (err) {
        BCUDA(b, cudaMemsetAsync(b->at<int>(b->o_nact) + 1, 0, 4, st));
        b->err = "a batched solve round gave up waiting for a dependency";
        return STO_ERR_TIMEOUT;
    }
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
    if ((reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(hx)) & 15) return STO_ERR_INVALID_ARG;
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
    int iters = 0;
    int head[2] = {ninst, 0};  // active instances, round error word
    sto_status result = STO_OK;
    while (true) {
        BCUDA(b, cudaMemcpyAsync(head, nact, 8, cudaMemcpyDeviceToHost, st));
        BCUDA(b, cudaStreamSynchronize(st));
        if (head[1]) {
            BCUDA(b, cudaMemsetAsync(nact + 1, 0, 4, st));
            BCUDA(b, cudaStreamSynchronize(st));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            b->err = "a batched solve round gave up waiting for a dependency";
            return STO_ERR_TIMEOUT;
        }
        if (head[0] == 0) break;
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
