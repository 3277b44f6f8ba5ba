// Algorithms 1 (dual MINFBE) and 2 (NAMA) on the preconditioned dual, the power-iteration
// estimate of L, and the FP64 KKT check.
//
// Every step except the solve rounds is an elementwise pass over the m dual entries with a
// deterministic two-level reduction (per-block partials, the last block to finish sums them in
// block order and takes the algorithm's decision on the device):
//   k_point   z = proj_{SY}(h + ybar/lam), r = z - h, FBE, ||S^-1 r||_inf          (Section II-D, III-A)
//   k_grad    g = r + lam S H x_lin(r) = grad FBE                                  (Section III-A)
//   k_lb_dots / k_lb_dir   L-BFGS direction d = -B g, compact form               (Alg. 1, 2: quasi-Newton direction)
//   k_ls      FBE at up to 19 step sizes tau = 2^-k in one pass                    (Alg. 1, 2: line search)
//   k_fbstep  ybar+ = T_lam(w), s = ybar+ - ybar                                   (Alg. 1, 2: forward-backward update)
//   k_gpad    GPAD step ybar+ = T_lam(w), next extrapolated point                 (Section III-F, Section IV)
//
// Readings of the text used here:
//   * T_lam(y) = y + lam (Hx(y) - z_lam(y)), the sign used by Algorithm 2's update.
//   * NAMA's extrapolation is w = y + tau d + (1 - tau)(T(y) - y) (tau = 0 is the FB step) and
//     its update y+ = T(w); MINFBE's update (printed as x^{k+1}) is y+ = T(w).
//   * "Choose the smallest tau" means the largest tau = 2^-nu, nu = 0, 1, ...; after max_ls
//     halvings tau = 0, for which the FB step always decreases the FBE.
//   * x(y + tau d) = x(y) + tau x_lin(d) with x_lin from Algorithm 4 (the printed x(d) holds
//     only without affine terms), so every trial point costs one elementwise pass.
//   * The FBE is evaluated as -[f(x) + <y, Hx - z> + lam/2 ||Hx - z||^2], equal to the
//     definition of Section III-A; with diagonal costs f(x) is a weighted sum over the
//     entries of S Hx.  The line search sums the per-entry change against the current point.
//   * Termination uses the unscaled residual ||z - Hx||_inf (Section III-B).
//   * L-BFGS: H0 = gamma I with gamma = <s,q>/<q,q> of the newest pair, lam I while empty;
//     pairs are kept when <s,q> > eps' ||s||^2 ||g||^2 (Algorithms 1, 2: the curvature test).
#include <cmath>
#include <cstring>
#include <utility>

#include "internal.h"

namespace sto {
namespace {

constexpr int kThreads = 256;

template <class T>
struct DualView {
    int m, Np, nb, nbl, leaf_base;   // dual length, nonleaf nodes, nonleaf / leaf block sizes
    float inv_nb, inv_nbl;
    int nx, nu;                      // state and input dimensions
    // the per-component table: tab_n entries per row, leaf components at leaf_off + c (the
    // selection layout: the leaves' x part shares the nonleaf rows, leaf_off = 0); root_free: the
    // root's state block is the parameter (selection layout only); has_cost: the cost weights
    // belong to the dual entries (selection layout: Hx holds x and u), else f(x) comes from the
    // primal separately
    int tab_n, leaf_off, root_free, has_cost;
    const T *sqp, *box, *Wc;  // box = [lo][hi][rho][delta][kind] rows of tab_n, Wc = [Q|R|PN][q|r|pN]

    // per element: sqrt(pi) of its node, scaled bounds sqrt(pi) lo, sqrt(pi) hi, cost weights,
    // and the kind of its nonsmooth term g with rho, delta (Section II-B)
    struct Meta {
        T sq, lo, hi, w, l, rho, delta;
        int kind;
    };

    // Scalar path (caller-facing conversions): per-entry constants read from global memory.
    __device__ __forceinline__ Meta meta(int e) const {
        int node, comp;
        bool leaf;
        if (e < leaf_base) {
            node = e / nb;
            comp = e - node * nb;
            leaf = false;
        } else {
            const int e2 = e - leaf_base;
            node = Np + e2 / nbl;
            comp = e2 - (node - Np) * nbl;
            leaf = true;
        }
        Meta M;
        M.sq = sqp[node];
        const int bi = leaf ? leaf_off + comp : comp;
        if (root_free && !leaf && node == 0 && comp < nx) {
            M.lo = -INFINITY;
            M.hi = INFINITY;
            M.kind = 0;
        } else {
            M.lo = M.sq * box[bi];
            M.hi = M.sq * box[tab_n + bi];
            M.kind = (int)box[4 * tab_n + bi];
        }
        M.rho = box[2 * tab_n + bi];
        M.delta = box[3 * tab_n + bi];
        if (has_cost) {
            const int wi = leaf ? nx + nu + comp : comp;
            M.w = Wc[wi];
            M.l = M.sq * Wc[2 * nx + nu + wi];
        } else {
            M.w = M.l = T(0);
        }
        return M;
    }
};

// Position of a dual entry in the node blocks ([x; u] per nonleaf node, [x] per leaf): found
// once per vector of entries by a float reciprocal with an exact integer fix-up, then advanced
// entry by entry, so the passes need no integer division per entry.
struct Pos {
    int node, comp;
    bool leaf;
};
__device__ __forceinline__ int div_fix(int e, int d, float inv, int &r) {
    int q = (int)((float)e * inv);
    r = e - q * d;
    while (r < 0) {
        --q;
        r += d;
    }
    while (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}
template <class T>
__device__ __forceinline__ Pos pos_of(const DualView<T> &dv, int e) {
    Pos p;
    if (e < dv.leaf_base) {
        p.node = div_fix(e, dv.nb, dv.inv_nb, p.comp);
        p.leaf = false;
    } else {
        p.node = dv.Np + div_fix(e - dv.leaf_base, dv.nbl, dv.inv_nbl, p.comp);
        p.leaf = true;
    }
    return p;
}
template <class T>
__device__ __forceinline__ void pos_next(const DualView<T> &dv, Pos &p) {
    ++p.comp;
    if (!p.leaf) {
        if (p.comp == dv.nb) {
            p.comp = 0;
            ++p.node;
            p.leaf = p.node >= dv.Np;
        }
    } else if (p.comp == dv.nbl) {
        p.comp = 0;
        ++p.node;
    }
}

// Per-component constants of the dual layout in shared memory (dynamic, 9 tab_n reals): lo, hi,
// quadratic and linear cost weights of nonleaf entries and of leaf entries, rho, delta and kind of
// the term g.  Selection layout: nonleaf [x; u] components, the leaves the x part with the
// terminal weights; general maps: the z components of nonleaf blocks, then those of leaf blocks,
// no cost weights.
template <class T>
struct CompTab {
    T *lo, *hi, *w, *l, *wl, *ll, *rh, *dl, *kd;
    __device__ void load(const DualView<T> &dv, T *sm) {
        const int n = dv.tab_n;
        lo = sm;
        hi = sm + n;
        w = sm + 2 * n;
        l = sm + 3 * n;
        wl = sm + 4 * n;
        ll = sm + 5 * n;
        rh = sm + 6 * n;
        dl = sm + 7 * n;
        kd = sm + 8 * n;
        nx_ = dv.nx;
        leaf_off_ = dv.leaf_off;
        root_free_ = dv.root_free;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            lo[c] = dv.box[c];
            hi[c] = dv.box[n + c];
            rh[c] = dv.box[2 * n + c];
            dl[c] = dv.box[3 * n + c];
            kd[c] = dv.box[4 * n + c];
            const int nxu = dv.nx + dv.nu;
            w[c] = dv.has_cost && c < nxu ? dv.Wc[c] : T(0);
            l[c] = dv.has_cost && c < nxu ? dv.Wc[2 * dv.nx + dv.nu + c] : T(0);
            wl[c] = dv.has_cost && c < dv.nx ? dv.Wc[nxu + c] : T(0);
            ll[c] = dv.has_cost && c < dv.nx ? dv.Wc[2 * dv.nx + dv.nu + nxu + c] : T(0);
        }
        __syncthreads();
    }
    // the constants of the entry at p, scaled by sq = sqrt(pi) of its node (G = false: the
    // term's kind is the box for every element and rho, delta are not read)
    template <bool G = true>
    __device__ __forceinline__ typename DualView<T>::Meta meta(const Pos &p, T sq) const {
        typename DualView<T>::Meta M;
        M.sq = sq;
        const int c = p.comp;
        const int bi = p.leaf ? leaf_off_ + c : c;
        if (root_free_ && !p.leaf && p.node == 0 && c < nx_) {  // the root state is the parameter: unboxed
            M.lo = -INFINITY;
            M.hi = INFINITY;
            M.kind = 0;
        } else {
            M.lo = sq * lo[bi];
            M.hi = sq * hi[bi];
            M.kind = G ? (int)kd[bi] : 0;
        }
        M.rho = G ? rh[bi] : T(0);
        M.delta = G ? dl[bi] : T(1);
        M.w = p.leaf ? wl[c] : w[c];
        M.l = sq * (p.leaf ? ll[c] : l[c]);
        return M;
    }
    int nx_, leaf_off_, root_free_;
};
template <class T>
size_t comp_tab_bytes(const DualView<T> &dv) {
    return (size_t)9 * dv.tab_n * sizeof(T);
}

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};
// n entries (n = VN: one 16-byte load) of v starting at e0 into x[]
template <class T>
__device__ __forceinline__ void ldv(const T *v, int e0, int n, T *x) {
    constexpr int VN = Vec16<T>::n;
    if (n == VN) {
        const typename Vec16<T>::type t = *reinterpret_cast<const typename Vec16<T>::type *>(v + e0);
        const T *tt = reinterpret_cast<const T *>(&t);
#pragma unroll
        for (int q = 0; q < VN; ++q) x[q] = tt[q];
    } else {
#pragma unroll
        for (int q = 0; q < VN; ++q) x[q] = q < n ? v[e0 + q] : T(0);
    }
}
template <class T>
__device__ __forceinline__ void stv(T *v, int e0, int n, const T *x) {
    constexpr int VN = Vec16<T>::n;
    if (n == VN) {
        typename Vec16<T>::type t;
        T *tt = reinterpret_cast<T *>(&t);
#pragma unroll
        for (int q = 0; q < VN; ++q) tt[q] = x[q];
        *reinterpret_cast<typename Vec16<T>::type *>(v + e0) = t;
    } else {
        for (int q = 0; q < n; ++q) v[e0 + q] = x[q];
    }
}
// Grid-stride loop over 16-byte vectors of entries [0, m): f(e0, n) with n = VN, and the last
// m % VN entries by one thread.  Every solver vector starts on a 256-byte boundary.
template <class T, class F>
__device__ __forceinline__ void for_vectors(int m, F f) {
    constexpr int VN = Vec16<T>::n;
    const int nvec = m / VN;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += gridDim.x * blockDim.x) f(v * VN, VN);
    if (nvec * VN < m && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) f(nvec * VN, m - nvec * VN);
}

template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// z_lambda of one element (Section II-D): argmin_z g~(z) + lam/2 (z - v)^2 for the element's
// term (Section II-B) in the scaled dual, g~(z) = g(z / s), s = sqrt(pi): kind 0 clamps to the
// scaled box; outside it by e, kind 1 moves back by at most rho / (lam s) without crossing the
// bound, kind 2 maps e to e / (1 + q) when e <= s delta (1 + q), q = rho / (lam s^2), and to
// e - rho delta / (lam s) beyond (the proximal map of the Huber function).
// G = false: every element's term is the indicator of its box (the projection only).
template <class T, bool G>
__device__ __forceinline__ T prox_el(T v, T lam, const typename DualView<T>::Meta &M) {
    if (!G || M.kind == 0) return clampv(v, M.lo, M.hi);
    T base, e, sg;
    if (v > M.hi) {
        base = M.hi;
        e = v - M.hi;
        sg = T(1);
    } else if (v < M.lo) {
        base = M.lo;
        e = M.lo - v;
        sg = T(-1);
    } else {
        return v;
    }
    const T sh = M.rho / (lam * M.sq);
    T ez;
    if (M.kind == 1) {
        ez = fmax(e - sh, T(0));
    } else {
        const T q = sh / M.sq;
        ez = e <= M.sq * M.delta * (T(1) + q) ? e / (T(1) + q) : e - sh * M.delta;
    }
    return base + sg * ez;
}

// g~(z) of one element: 0 (kind 0, z in the box), rho d (kind 1) or rho Huber_delta(d)
// (kind 2), d = unscaled distance of z / s to the box.
template <class T, bool G>
__device__ __forceinline__ T g_el(T z, const typename DualView<T>::Meta &M) {
    if (!G || M.kind == 0) return T(0);
    const T d = (fmax(M.lo - z, T(0)) + fmax(z - M.hi, T(0))) / M.sq;
    if (M.kind == 1) return M.rho * d;
    return M.rho * (d <= M.delta ? T(0.5) * d * d : M.delta * (d - T(0.5) * M.delta));
}

// Per-entry term of -FBE: W h^2 + l h + g~(z) + w (h - z) + lam/2 (h - z)^2, z = z_lambda.
template <class T, bool G>
__device__ __forceinline__ T fbe_term(T h, T w, T lam, T ilam, const typename DualView<T>::Meta &M) {
    const T z = prox_el<T, G>(h + w * ilam, lam, M);
    const T dz = h - z;
    return h * (M.w * h + M.l) + g_el<T, G>(z, M) + dz * (w + T(0.5) * lam * dz);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Two-level deterministic reduction of NS sums and NM maxima.  Returns true in the last
// block to finish, where out[0..NS+NM) holds the totals (summed in block order).  The warp and
// block levels run in the kernel's type T (the FP64 pipe is slow on this part: an FP64 shuffle
// tree per value would dominate an elementwise pass); each block's partial and the sum over
// blocks are FP64.
template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T>
__device__ __forceinline__ T warp_max_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class T, int NS, int NM>
__device__ bool reduce_last(T *sums, T *maxs, double *partials, unsigned *counter, double *out) {
    constexpr int NV = NS + NM;
    __shared__ T red[kThreads / 32][NV > 0 ? NV : 1];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NS; ++k) sums[k] = warp_sum_t(sums[k]);
#pragma unroll
    for (int k = 0; k < NM; ++k) maxs[k] = warp_max_t(maxs[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) red[warp][k] = sums[k];
#pragma unroll
        for (int k = 0; k < NM; ++k) red[warp][NS + k] = maxs[k];
    }
    __syncthreads();
    // partials are slot-major ([slot][block]) so that the last block reads them coalesced
    if (threadIdx.x < NV) {
        const int k = threadIdx.x;
        T acc = k < NS ? T(0) : T(-INFINITY);
        for (int w = 0; w < kThreads / 32; ++w) acc = k < NS ? acc + red[w][k] : fmax(acc, red[w][k]);
        partials[k * kRedBlocks + blockIdx.x] = (double)acc;
        __threadfence();  // only the writers of partials publish anything
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // warp w sums slots w, w+8, ...; lane l takes blocks l, l+32, ... (all loads issued before
    // the first add), sums them in that order, then a fixed butterfly: the result does not
    // depend on which block finished last
    constexpr int kPerLane = (kRedBlocks + 31) / 32;
    for (int k = warp; k < NV; k += kThreads / 32) {
        const double ident = k < NS ? 0.0 : -INFINITY;
        double v[kPerLane];
#pragma unroll
        for (int q = 0; q < kPerLane; ++q) {
            const int b = lane + 32 * q;
            v[q] = b < (int)gridDim.x ? __ldcg(partials + k * kRedBlocks + b) : ident;
        }
        double acc = ident;
#pragma unroll
        for (int q = 0; q < kPerLane; ++q) acc = k < NS ? acc + v[q] : fmax(acc, v[q]);
        acc = k < NS ? warp_sum_d(acc) : warp_max_d(acc);
        if (lane == 0) out[k] = acc;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------------------
// k_point: residual, FBE and stopping test at the current ybar (h = S H x(ybar)).
// pair = 1 (NAMA after a step): q = r_new - r_old -> Y[p], curvature test, commit pair.
// BT = 1 (original backtracking test): rw, hw are r and h at the point w the step was taken
// from; reduces <rw, h - hw> and ||rw||^2.  BT = 2 (simple backtracking test): ||r||^2.
// ---------------------------------------------------------------------------------------
template <class T, int BT, bool G>
__global__ void __launch_bounds__(kThreads) k_point(DualView<T> dv, const T *__restrict__ yb, const T *__restrict__ h,
                                                    T *r, T *ringS, T *ringY, long long vstride, int pair,
                                                    SolverScalars *sc, double *partials, const T *__restrict__ rw,
                                                    const T *__restrict__ hw) {
    __shared__ double tot[9];
    if (sc->stop) return;  // a look-ahead iteration after the run stopped
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(dv, reinterpret_cast<T *>(tab_raw));
    constexpr int VN = Vec16<T>::n;
    const T lam = (T)sc->lambda, ilam = T(1) / lam;
    const int p = (sc->lb_head + sc->lb_count) % (sc->mem + 1);
    const T *sv = ringS + p * vstride;
    T *qv = ringY + p * vstride;
    T fsum = 0, sq_dot = 0, s2 = 0, g2 = 0, rmax = 0, r2 = 0, bta = 0, btb = 0;
    int nan = 0;
    for_vectors<T>(dv.m, [&](int e0, int n) {
        T he[VN], ye[VN], re[VN], ro[VN], se[VN], q[VN], rwe[VN], hwe[VN];
        ldv(h, e0, n, he);
        ldv(yb, e0, n, ye);
        if (pair) {
            ldv<T>(r, e0, n, ro);
            ldv(sv, e0, n, se);
        }
        if constexpr (BT == 1) {
            ldv(rw, e0, n, rwe);
            ldv(hw, e0, n, hwe);
        }
        Pos ps = pos_of(dv, e0);
        int cur = -1;
        T sq = 1, isq = 1;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            if (k < n) {
                if (ps.node != cur) {
                    cur = ps.node;
                    sq = dv.sqp[cur];
                    isq = T(1) / sq;
                }
                const auto M = tab.template meta<G>(ps, sq);
                const T z = prox_el<T, G>(he[k] + ye[k] * ilam, lam, M);
                re[k] = z - he[k];
                fsum += fbe_term<T, G>(he[k], ye[k], lam, ilam, M);
                const T ra = fabs(re[k]) * isq;
                if (!(ra <= T(3.0e38))) nan = 1;
                rmax = fmax(rmax, ra);
                if constexpr (BT == 2) r2 += re[k] * re[k];
                if constexpr (BT == 1) {
                    bta += rwe[k] * (he[k] - hwe[k]);
                    btb += rwe[k] * rwe[k];
                }
                if (pair) {
                    q[k] = re[k] - ro[k];
                    sq_dot += se[k] * q[k];
                    s2 += se[k] * se[k];
                    g2 += ro[k] * ro[k];
                }
                pos_next(dv, ps);
            }
        }
        if (pair) stv(qv, e0, n, q);
        stv(r, e0, n, re);
    });
    constexpr int NS = BT == 0 ? 5 : (BT == 1 ? 7 : 6);
    T sums[NS];
    sums[0] = fsum;
    sums[1] = sq_dot;
    sums[2] = s2;
    sums[3] = g2;
    sums[4] = (T)nan;
    if constexpr (BT == 1) {
        sums[5] = bta;
        sums[6] = btb;
    }
    if constexpr (BT == 2) sums[5] = r2;
    T maxs[1] = {rmax};
    if (reduce_last<T, NS, 1>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        sc->phi = -(tot[0] + sc->f_pt);  // f(x) from the primal with general maps (else 0)
        sc->res_inf = tot[NS];
        if constexpr (BT == 1) {
            sc->bt_a = tot[5];
            sc->bt_b = tot[6];
        }
        if constexpr (BT == 2) sc->r2 = tot[5];
        if (tot[4] > 0.0 || !(tot[0] == tot[0])) sc->nan_flag = 1;
        if (sc->lookahead && (sc->nan_flag || sc->res_inf <= sc->tol)) sc->stop = 1;
        if (pair && sc->lb_pending_valid) {
            if (tot[1] > sc->eps_curv * tot[2] * tot[3]) {
                if (sc->lb_count < sc->mem)
                    sc->lb_count += 1;
                else
                    sc->lb_head = (sc->lb_head + 1) % (sc->mem + 1);
                sc->lb_new_pair = 1;
            }
            sc->lb_pending_valid = 0;
        }
    }
}

// MINFBE: g_new = r + lam hr = grad FBE; with a pending pair q = g_new - g_old -> Y[p];
// ||hr||^2 for the simple backtracking test.
template <class T>
__global__ void __launch_bounds__(kThreads) k_grad(int m, const T *__restrict__ r, const T *__restrict__ hr, T *g,
                                                   T *ringS, T *ringY, long long vstride, SolverScalars *sc,
                                                   double *partials) {
    __shared__ double tot[8];
    if (sc->stop) return;
    constexpr int VN = Vec16<T>::n;
    const T lam = (T)sc->lambda;
    const int pair = sc->lb_pending_valid;
    const int p = (sc->lb_head + sc->lb_count) % (sc->mem + 1);
    const T *sv = ringS + p * vstride;
    T *qv = ringY + p * vstride;
    T sq_dot = 0, s2 = 0, g2 = 0, hr2 = 0;
    for_vectors<T>(m, [&](int e0, int n) {
        T re[VN], he[VN], gn[VN], go[VN], se[VN], q[VN];
        ldv(r, e0, n, re);
        ldv(hr, e0, n, he);
        if (pair) {
            ldv<T>(g, e0, n, go);
            ldv(sv, e0, n, se);
        }
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            gn[k] = re[k] + lam * he[k];
            hr2 += he[k] * he[k];  // zero past n (ldv pads)
            if (pair && k < n) {
                q[k] = gn[k] - go[k];
                sq_dot += se[k] * q[k];
                s2 += se[k] * se[k];
                g2 += go[k] * go[k];
            }
        }
        if (pair) stv(qv, e0, n, q);
        stv(g, e0, n, gn);
    });
    T sums[4] = {sq_dot, s2, g2, hr2};
    T maxs[1];
    if (reduce_last<T, 4, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        sc->hr2 = tot[3];
        if (pair) {
            if (tot[0] > sc->eps_curv * tot[1] * tot[2]) {
                if (sc->lb_count < sc->mem)
                    sc->lb_count += 1;
                else
                    sc->lb_head = (sc->lb_head + 1) % (sc->mem + 1);
                sc->lb_new_pair = 1;
            }
            sc->lb_pending_valid = 0;
        }
    }
}

// L-BFGS, compact representation (Byrd, Nocedal, Schnabel 1994): one pass for S'g, Y'g and the
// Gram column of a newly committed pair, then the small solve in the last block.  MEM >= mem.
template <class T, int MEM>
__global__ void __launch_bounds__(kThreads, 4) k_lb_dots(int m, const T *__restrict__ g, const T *ringS,
                                                      const T *ringY, long long vstride, SolverScalars *sc,
                                                      double *partials) {
    __shared__ double tot[4 * MEM];
    if (sc->stop) return;
    const int cnt = sc->lb_count, head = sc->lb_head, M1 = sc->mem + 1, newp = sc->lb_new_pair;
    if (cnt == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->gamma = sc->lambda;
            sc->lb_new_pair = 0;
        }
        return;
    }
    const int nslot = (head + cnt - 1) % M1;
    const T *yn = ringY + nslot * vstride;
    const T *sp[MEM];
    const T *yp[MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) {
        const int sl = (head + (k < cnt ? k : 0)) % M1;
        sp[k] = ringS + sl * vstride;
        yp[k] = ringY + sl * vstride;
    }
    constexpr int VN = Vec16<T>::n;
    T a[MEM], b[MEM], c[MEM], d[MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) a[k] = b[k] = c[k] = d[k] = T(0);
    for_vectors<T>(m, [&](int e0, int n) {
        T ge[VN], ye[VN];
        ldv(g, e0, n, ge);
        if (newp)
            ldv(yn, e0, n, ye);
        else
#pragma unroll
            for (int q = 0; q < VN; ++q) ye[q] = T(0);
#pragma unroll
        for (int k = 0; k < MEM; ++k) {
            if (k < cnt) {
                T se[VN], qe[VN];
                ldv(sp[k], e0, n, se);
                ldv(yp[k], e0, n, qe);
#pragma unroll
                for (int q = 0; q < VN; ++q) {
                    a[k] += se[q] * ge[q];
                    b[k] += qe[q] * ge[q];
                    c[k] += se[q] * ye[q];
                    d[k] += qe[q] * ye[q];
                }
            }
        }
    });
    T sums[4 * MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) {
        sums[k] = a[k];
        sums[MEM + k] = b[k];
        sums[2 * MEM + k] = c[k];
        sums[3 * MEM + k] = d[k];
    }
    T maxs[1];
    if (reduce_last<T, 4 * MEM, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        int sl[MEM];
        for (int k = 0; k < cnt; ++k) sl[k] = (head + k) % M1;
        if (newp) {
            for (int k = 0; k < cnt; ++k) {
                sc->SY[sl[k]][nslot] = tot[2 * MEM + k];
                sc->YY[sl[k]][nslot] = tot[3 * MEM + k];
                sc->YY[nslot][sl[k]] = tot[3 * MEM + k];
            }
            sc->lb_new_pair = 0;
        }
        const double gamma = sc->SY[nslot][nslot] / sc->YY[nslot][nslot];
        double x1[MEM], t[MEM], top[MEM];
        // x1 = R^-1 a with R_ij = s_i'y_j (i <= j)
        for (int i = cnt - 1; i >= 0; --i) {
            double s = tot[i];
            for (int j = i + 1; j < cnt; ++j) s -= sc->SY[sl[i]][sl[j]] * x1[j];
            x1[i] = s / sc->SY[sl[i]][sl[i]];
        }
        // t = (D + gamma Y'Y) x1 - gamma b,  top = R^-T t
        for (int i = 0; i < cnt; ++i) {
            double s = sc->SY[sl[i]][sl[i]] * x1[i] - gamma * tot[MEM + i];
            for (int j = 0; j < cnt; ++j) s += gamma * sc->YY[sl[i]][sl[j]] * x1[j];
            t[i] = s;
        }
        for (int i = 0; i < cnt; ++i) {
            double s = t[i];
            for (int j = 0; j < i; ++j) s -= sc->SY[sl[j]][sl[i]] * top[j];
            top[i] = s / sc->SY[sl[i]][sl[i]];
        }
        sc->gamma = gamma;
        for (int i = 0; i < cnt; ++i) {
            sc->coef_s[i] = top[i];
            sc->coef_y[i] = -gamma * x1[i];
        }
    }
}

// d = -(gamma g + sum_i coef_s[i] s_i + sum_i coef_y[i] y_i)
template <class T, int MEM>
__global__ void __launch_bounds__(kThreads, 4) k_lb_dir(int m, const T *__restrict__ g, const T *ringS, const T *ringY,
                                                     long long vstride, const SolverScalars *sc, T *dvec) {
    if (sc->stop) return;
    const int cnt = sc->lb_count, head = sc->lb_head, M1 = sc->mem + 1;
    const T gamma = (T)sc->gamma;
    T cs[MEM], cy[MEM];
    const T *sp[MEM];
    const T *yp[MEM];
#pragma unroll
    for (int k = 0; k < MEM; ++k) {
        const int sl = (head + (k < cnt ? k : 0)) % M1;
        cs[k] = k < cnt ? (T)sc->coef_s[k] : T(0);
        cy[k] = k < cnt ? (T)sc->coef_y[k] : T(0);
        sp[k] = ringS + sl * vstride;
        yp[k] = ringY + sl * vstride;
    }
    constexpr int VN = Vec16<T>::n;
    for_vectors<T>(m, [&](int e0, int n) {
        T acc[VN];
        ldv(g, e0, n, acc);
#pragma unroll
        for (int q = 0; q < VN; ++q) acc[q] *= gamma;
#pragma unroll
        for (int k = 0; k < MEM; ++k)
            if (k < cnt) {
                T se[VN], qe[VN];
                ldv(sp[k], e0, n, se);
                ldv(yp[k], e0, n, qe);
#pragma unroll
                for (int q = 0; q < VN; ++q) acc[q] += cs[k] * se[q] + cy[k] * qe[q];
            }
#pragma unroll
        for (int q = 0; q < VN; ++q) acc[q] = -acc[q];
        stv(dvec, e0, n, acc);
    });
}

template <class T, int MEM>
void lb_direction_t(int grid, cudaStream_t st, int m, const T *g, const T *ringS, const T *ringY, long long vs,
                    SolverScalars *sc, double *part, T *d) {
    const int g1 = wave_grid((const void *)k_lb_dots<T, MEM>, kThreads, 0, grid);
    const int g2 = wave_grid((const void *)k_lb_dir<T, MEM>, kThreads, 0, grid);
    k_lb_dots<T, MEM><<<g1, kThreads, 0, st>>>(m, g, ringS, ringY, vs, sc, part);
    k_lb_dir<T, MEM><<<g2, kThreads, 0, st>>>(m, g, ringS, ringY, vs, sc, d);
}

template <class T>
void lb_direction(int mem, int grid, cudaStream_t st, int m, const T *g, const T *ringS, const T *ringY, long long vs,
                  SolverScalars *sc, double *part, T *d) {
    if (mem <= 2)
        lb_direction_t<T, 2>(grid, st, m, g, ringS, ringY, vs, sc, part, d);
    else if (mem <= 5)
        lb_direction_t<T, 5>(grid, st, m, g, ringS, ringY, vs, sc, part, d);
    else if (mem <= 8)
        lb_direction_t<T, 8>(grid, st, m, g, ringS, ringY, vs, sc, part, d);
    else
        lb_direction_t<T, 16>(grid, st, m, g, ringS, ringY, vs, sc, part, d);
}

// Line search: candidates tau_j = 2^-(e0 + j), j < nc <= J, evaluated in one pass.
// NAMA (nama = 1): w = ybar - lam r + tau (d + lam r),  h(w) = h - lam hr + tau (hd + lam hr).
// MINFBE:          w = ybar + tau d,                     h(w) = h + tau hd.
// Accept the largest tau with FBE(w) <= FBE(ybar); after the last group tau = 0.
template <class T, int J, bool G>
__global__ void __launch_bounds__(kThreads) k_ls(DualView<T> dv, const T *__restrict__ yb, const T *__restrict__ h,
                                                 const T *__restrict__ r, const T *__restrict__ dvec,
                                                 const T *__restrict__ hr, const T *__restrict__ hd, int nama, int e0,
                                                 int nc, int last_group, SolverScalars *sc, double *partials) {
    __shared__ double tot[J];
    if (sc->ls_done || sc->stop) return;
    const T lam = (T)sc->lambda, ilam = T(1) / lam;
    T tau[J];
#pragma unroll
    for (int j = 0; j < J; ++j) tau[j] = (T)ldexp(1.0, -(e0 + j));
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(dv, reinterpret_cast<T *>(tab_raw));
    constexpr int VN = Vec16<T>::n;
    T acc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = T(0);
    for_vectors<T>(dv.m, [&](int e0, int n) {
        T y0[VN], h0[VN], re[VN], dd[VN], hre[VN], hdd[VN];
        ldv(yb, e0, n, y0);
        ldv(h, e0, n, h0);
        ldv(dvec, e0, n, dd);
        ldv(hd, e0, n, hdd);
        if (nama) {
            ldv(r, e0, n, re);
            ldv(hr, e0, n, hre);
        }
        Pos ps = pos_of(dv, e0);
        int cur = -1;
        T sq = 1;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            if (k < n) {
                if (ps.node != cur) {
                    cur = ps.node;
                    sq = dv.sqp[cur];
                }
                const auto M = tab.template meta<G>(ps, sq);
                T wa, wb, ha, hb;
                if (nama) {
                    wa = y0[k] - lam * re[k];
                    wb = dd[k] + lam * re[k];
                    ha = h0[k] - lam * hre[k];
                    hb = hdd[k] + lam * hre[k];
                } else {
                    wa = y0[k];
                    wb = dd[k];
                    ha = h0[k];
                    hb = hdd[k];
                }
                const T c0 = fbe_term<T, G>(h0[k], y0[k], lam, ilam, M);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const T cj = fbe_term<T, G>(ha + tau[j] * hb, wa + tau[j] * wb, lam, ilam, M);
                    acc[j] += cj - c0;
                }
                pos_next(dv, ps);
            }
        }
    });
    T sums[J];
#pragma unroll
    for (int j = 0; j < J; ++j) sums[j] = acc[j];
    T maxs[1];
    if (reduce_last<T, J, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        // FBE(w) - FBE(ybar) = -sum_e (term(w) - term(ybar))
        for (int j = 0; j < nc; ++j) {
            // with general maps f(x(w(tau))) - f(x(ybar)) from the primal (else 0)
            const double t = ldexp(1.0, -(e0 + j));
            const double dphi = -(tot[j] + sc->f_ls[0] + t * (sc->f_ls[1] + t * sc->f_ls[2]));
            sc->cand[e0 + j] = dphi;
            if (dphi <= 0.0) {
                sc->tau = ldexp(1.0, -(e0 + j));
                sc->ls_done = 1;
                return;
            }
        }
        if (last_group) {
            sc->tau = 0.0;
            sc->ls_done = 1;
            sc->ls_zero += 1;
        }
    }
}

// ybar+ = T_lam(w(tau)) = w + lam (h(w) - z(w)); s = ybar+ - ybar -> S[p]; ybar <- ybar+.
// rw_out, hw_out (non-null with the original backtracking test): r(w) = z(w) - h(w) and h(w).
template <class T, bool G>
__global__ void __launch_bounds__(kThreads) k_fbstep(DualView<T> dv, T *yb, const T *__restrict__ h,
                                                     const T *__restrict__ r, const T *__restrict__ dvec,
                                                     const T *__restrict__ hr, const T *__restrict__ hd, int nama,
                                                     T *ringS, long long vstride, SolverScalars *sc, T *rw_out,
                                                     T *hw_out) {
    if (sc->stop) return;
    const T lam = (T)sc->lambda, ilam = T(1) / lam;
    const T tau = (T)sc->tau;
    const int p = (sc->lb_head + sc->lb_count) % (sc->mem + 1);
    T *sv = ringS + p * vstride;
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(dv, reinterpret_cast<T *>(tab_raw));
    constexpr int VN = Vec16<T>::n;
    for_vectors<T>(dv.m, [&](int e0, int n) {
        T y0[VN], h0[VN], re[VN], dd[VN], hre[VN], hdd[VN], yn[VN], sn[VN], rwv[VN], hwv[VN];
        ldv(yb, e0, n, y0);
        ldv(h, e0, n, h0);
        ldv(dvec, e0, n, dd);
        ldv(hd, e0, n, hdd);
        if (nama) {
            ldv(r, e0, n, re);
            ldv(hr, e0, n, hre);
        }
        Pos ps = pos_of(dv, e0);
        int cur = -1;
        T sq = 1;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            if (k < n) {
                if (ps.node != cur) {
                    cur = ps.node;
                    sq = dv.sqp[cur];
                }
                const auto M = tab.template meta<G>(ps, sq);
                T w, hw;
                if (nama) {
                    w = y0[k] - lam * re[k] + tau * (dd[k] + lam * re[k]);
                    hw = h0[k] - lam * hre[k] + tau * (hdd[k] + lam * hre[k]);
                } else {
                    w = y0[k] + tau * dd[k];
                    hw = h0[k] + tau * hdd[k];
                }
                const T z = prox_el<T, G>(hw + w * ilam, lam, M);
                yn[k] = w + lam * (hw - z);
                sn[k] = yn[k] - y0[k];
                rwv[k] = z - hw;
                hwv[k] = hw;
                pos_next(dv, ps);
            }
        }
        stv(sv, e0, n, sn);
        stv(yb, e0, n, yn);
        if (rw_out) {
            stv(rw_out, e0, n, rwv);
            stv(hw_out, e0, n, hwv);
        }
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->lb_pending_valid = 1;
        sc->ls_done = 0;
        sc->iters += 1;
    }
}

// GPAD, the accelerated dual projected gradient of the warm start (Section III-F) and of the
// comparison in Section IV, in the theta form of Patrinos and Bemporad (2014).  At the
// extrapolated point w with h = S H x(w): z = proj(h + w/lam), r = z - h, the step
// ybar+ = T_lam(w) = w - lam r, and the next extrapolated point
// w+ = ybar+ + beta (ybar+ - ybar), beta = theta_{k+1} (1/theta_k - 1).  The FBE at w and
// ||S^-1 r||_inf are reduced for the stopping test, which the host applies to w.
template <class T, bool G>
__global__ void __launch_bounds__(kThreads) k_gpad(DualView<T> dv, const T *__restrict__ w, const T *__restrict__ h,
                                                   T *yb, T *wn, T beta, int it, int max_iter, SolverScalars *sc,
                                                   double *partials) {
    __shared__ double tot[3];
    if (sc->status) return;  // an earlier step stopped the run: this (look-ahead) step does nothing
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(dv, reinterpret_cast<T *>(tab_raw));
    constexpr int VN = Vec16<T>::n;
    const T lam = (T)sc->lambda, ilam = T(1) / lam;
    T fsum = 0, rmax = 0;
    int nan = 0;
    for_vectors<T>(dv.m, [&](int e0, int n) {
        T we[VN], he[VN], ye[VN], yn[VN], wv[VN];
        ldv(w, e0, n, we);
        ldv(h, e0, n, he);
        ldv<T>(yb, e0, n, ye);
        Pos ps = pos_of(dv, e0);
        int cur = -1;
        T sq = 1, isq = 1;
#pragma unroll
        for (int k = 0; k < VN; ++k) {
            if (k < n) {
                if (ps.node != cur) {
                    cur = ps.node;
                    sq = dv.sqp[cur];
                    isq = T(1) / sq;
                }
                const auto M = tab.template meta<G>(ps, sq);
                const T z = prox_el<T, G>(he[k] + we[k] * ilam, lam, M);
                const T r = z - he[k];
                fsum += fbe_term<T, G>(he[k], we[k], lam, ilam, M);
                const T ra = fabs(r) * isq;
                if (!(ra <= T(3.0e38))) nan = 1;
                rmax = fmax(rmax, ra);
                yn[k] = we[k] - lam * r;
                wv[k] = yn[k] + beta * (yn[k] - ye[k]);
                pos_next(dv, ps);
            }
        }
        stv(yb, e0, n, yn);
        stv(wn, e0, n, wv);
    });
    T sums[2] = {fsum, (T)nan};
    T maxs[1] = {rmax};
    if (reduce_last<T, 2, 1>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        sc->phi = -(tot[0] + sc->f_pt);  // f(x) from the primal with general maps (else 0)
        sc->res_inf = tot[2];
        if (tot[1] > 0.0 || !(tot[0] == tot[0])) sc->nan_flag = 1;
        // stop: converged at w, NaN, or the iteration cap (the host returns w of this step)
        if (sc->nan_flag || tot[2] <= sc->tol || it >= max_iter) sc->status = 1;
    }
}

// ||v||^2 -> sc->hr2 (the simple backtracking test of NAMA, v = S H x_lin(r)).
template <class T>
__global__ void __launch_bounds__(kThreads) k_norm2(int m, const T *__restrict__ v, SolverScalars *sc,
                                                    double *partials) {
    __shared__ double tot[1];
    constexpr int VN = Vec16<T>::n;
    T acc = 0;
    for_vectors<T>(m, [&](int e0, int n) {
        T x[VN];
        ldv(v, e0, n, x);
#pragma unroll
        for (int k = 0; k < VN; ++k) acc += x[k] * x[k];
    });
    T sums[1] = {acc};
    T maxs[1];
    if (reduce_last<T, 1, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) sc->hr2 = tot[0];
}

// A halving of the step (Section III-B backtracking): the new lambda, and the L-BFGS memory
// emptied.
__global__ void k_set_lambda(SolverScalars *sc, double lam) {
    sc->lambda = lam;
    sc->lb_count = 0;
    sc->lb_head = 0;
    sc->lb_pending_valid = 0;
    sc->lb_new_pair = 0;
    sc->ls_done = 0;
}

// ybar = y / sqrt(pi) (in) and y = sqrt(pi) ybar, z = z_bar / sqrt(pi), x, u = S^-1 h (out).
template <class T>
__global__ void k_scale_in(DualView<T> dv, const T *y, T *yb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < dv.m; e += gridDim.x * blockDim.x)
        yb[e] = y[e] / dv.meta(e).sq;
}

template <class T>
__global__ void k_finish_out(DualView<T> dv, const T *yb, const T *h, const SolverScalars *sc, T *y, T *z) {
    const T lam = (T)sc->lambda, ilam = T(1) / lam;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < dv.m; e += gridDim.x * blockDim.x) {
        const auto M = dv.meta(e);
        const T ye = yb[e], he = h[e];
        y[e] = M.sq * ye;
        if (z) z[e] = prox_el<T, true>(he + ye * ilam, lam, M) / M.sq;
    }
}

// x [Nn][nx], u [Np][nu] from a primal vector in the [x; u] layout scaled by sqrt(pi) per node (sv:
// the selection layout's view): Hx itself for the selection maps, the primal output of the
// solve round for general maps.
template <class T>
__global__ void k_primal_out(DualView<T> sv, const T *p, T *x, T *u) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sv.m; e += gridDim.x * blockDim.x) {
        int node, k;
        if (e < sv.leaf_base) {
            node = e / sv.nb;
            k = e - node * sv.nb;
            const T v = p[e] / sv.sqp[node];
            if (k < sv.nx)
                x[(size_t)node * sv.nx + k] = v;
            else
                u[(size_t)node * sv.nu + (k - sv.nx)] = v;
        } else {
            const int e2 = e - sv.leaf_base;
            node = sv.Np + e2 / sv.nbl;
            k = e2 - (node - sv.Np) * sv.nbl;
            x[(size_t)node * sv.nx + k] = p[e] / sv.sqp[node];
        }
    }
}

// The cost f(x) of Section II-B for general maps, from the primal vectors of the solve rounds in
// the [x; u] layout scaled by sqrt(pi) (p = sqrt(pi) [x; u], so pi x'Qx = p'Qp, pi q'x =
// sqrt(pi) q'p), summed in FP64 over blocks:
//   k_fcost: f(p0) -> sc->f_pt (the FBE at a point adds it to the dual terms);
//   k_fquad: for the line search's affine primal p(tau) = pa + tau pb with pa = p0 - lam pr,
//   pb = pd + lam pr (NAMA) or pa = p0, pb = pd (MINFBE): f(pa) - f(p0), the linear and the
//   quadratic coefficient of f(p(tau)) in tau -> sc->f_ls[0..2].
template <class T>
__global__ void __launch_bounds__(kThreads) k_fcost(DualView<T> sv, const T *__restrict__ p0, SolverScalars *sc,
                                                    double *partials) {
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(sv, reinterpret_cast<T *>(tab_raw));
    T acc = T(0);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sv.m; e += gridDim.x * blockDim.x) {
        const Pos ps = pos_of(sv, e);
        const auto M = tab.meta(ps, sv.sqp[ps.node]);
        const T v = p0[e];
        acc += v * (M.w * v + M.l);
    }
    T sums[1] = {acc};
    T maxs[1];
    __shared__ double tot[1];
    if (reduce_last<T, 1, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) sc->f_pt = tot[0];
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_fquad(DualView<T> sv, const T *__restrict__ p0, const T *__restrict__ pr,
                                                    const T *__restrict__ pd, int nama, SolverScalars *sc,
                                                    double *partials) {
    extern __shared__ __align__(16) unsigned char tab_raw[];
    CompTab<T> tab;
    tab.load(sv, reinterpret_cast<T *>(tab_raw));
    const T lam = (T)sc->lambda;
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sv.m; e += gridDim.x * blockDim.x) {
        const Pos ps = pos_of(sv, e);
        const auto M = tab.meta(ps, sv.sqp[ps.node]);
        const T v0 = p0[e];
        const T pa = nama ? v0 - lam * pr[e] : v0;
        const T pb = nama ? pd[e] + lam * pr[e] : pd[e];
        s0 += (pa - v0) * (M.w * (pa + v0) + M.l);
        s1 += pb * (T(2) * M.w * pa + M.l);
        s2 += M.w * pb * pb;
    }
    T sums[3] = {s0, s1, s2};
    T maxs[1];
    __shared__ double tot[3];
    if (reduce_last<T, 3, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        sc->f_ls[0] = tot[0];
        sc->f_ls[1] = tot[1];
        sc->f_ls[2] = tot[2];
    }
}

// Power iteration on r -> -hr (hr = S H x_lin(S r)): L = <r, -hr> / <r, r>, r <- -hr / ||hr||.
template <class T>
__global__ void __launch_bounds__(kThreads) k_power_dots(int m, const T *r, const T *hr, SolverScalars *sc,
                                                         double *partials) {
    __shared__ double tot[3];
    T a = 0, b = 0, c = 0;
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < m; e += gridDim.x * kThreads) {
        const T re = r[e], he = hr[e];
        a += -re * he;
        b += he * he;
        c += re * re;
    }
    T sums[3] = {a, b, c};
    T maxs[1];
    if (reduce_last<T, 3, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0) {
        sc->pw_L = tot[0] / tot[2];
        sc->pw_inv_norm = tot[1] > 0.0 ? 1.0 / sqrt(tot[1]) : 0.0;
    }
}

template <class T>
__global__ void k_power_next(int m, T *r, const T *hr, const SolverScalars *sc) {
    const T s = (T)(-sc->pw_inv_norm);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) r[e] = s * hr[e];
}

template <class T>
__global__ void k_normalize(int m, T *r, SolverScalars *sc, double *partials) {
    __shared__ double tot[1];
    T a = 0;
    for (int e = blockIdx.x * kThreads + threadIdx.x; e < m; e += gridDim.x * kThreads) a += r[e] * r[e];
    T sums[1] = {a};
    T maxs[1];
    if (reduce_last<T, 1, 0>(sums, maxs, partials, &sc->red_counter, tot) && threadIdx.x == 0)
        sc->pw_inv_norm = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
}

template <class T>
__global__ void k_scale_by(int m, T *r, const SolverScalars *sc) {
    const T s = (T)sc->pw_inv_norm;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) r[e] *= s;
}

int red_grid(int64_t m) {
    const int64_t b = (m + kThreads - 1) / kThreads;
    return (int)(b < kRedBlocks ? (b > 0 ? b : 1) : kRedBlocks);
}

// The selection layout ([x; u] per nonleaf node, x per leaf) with the box and cost of the x and u
// components: the dual of the selection maps, and the primal of every problem.
template <class T>
DualView<T> make_sel_view(stotree_t h) {
    DualView<T> dv;
    dv.Np = h->Np;
    dv.nx = h->nx;
    dv.nu = h->nu;
    dv.nb = h->nx + h->nu;
    dv.nbl = h->nx;
    dv.m = (int)((int64_t)h->Np * dv.nb + (int64_t)h->Nl * dv.nbl);
    dv.leaf_base = h->Np * dv.nb;
    dv.inv_nb = 1.0f / (float)dv.nb;
    dv.inv_nbl = 1.0f / (float)dv.nbl;
    dv.tab_n = dv.nb;
    dv.leaf_off = 0;
    dv.root_free = 1;
    dv.has_cost = 1;
    dv.sqp = h->at<T>(h->L.sqp);
    dv.box = h->at<T>(h->L.box);
    dv.Wc = h->at<T>(h->L.cost);
    return dv;
}

// The dual layout: the selection layout, or the z blocks of general maps (nc per nonleaf node, ncN
// per leaf) with their box and no cost weights (f(x) then comes from the primal).
template <class T>
DualView<T> make_view(stotree_t h) {
    DualView<T> dv = make_sel_view<T>(h);
    if (!h->fg) return dv;
    dv.m = (int)h->m;
    dv.nb = h->nc;
    dv.nbl = h->ncN;
    dv.leaf_base = h->Np * h->nc;
    dv.inv_nb = 1.0f / (float)dv.nb;
    dv.inv_nbl = 1.0f / (float)dv.nbl;
    dv.tab_n = h->nc + h->ncN;
    dv.leaf_off = h->nc;
    dv.root_free = 0;
    dv.has_cost = 0;
    dv.box = h->at<T>(h->L.zbox);
    return dv;
}

size_t vstride_of(stotree_t h) { return (size_t)((h->m + 63) / 64 * 64); }

template <class T>
sto_status solver_impl(stotree_t h, int method, const sto_opts *o, const void *x0v, void *yv, void *xv, void *uv,
                       void *zv, sto_info *info, cudaStream_t st) {
    const Layout &L = h->L;
    const int m = (int)h->m;
    const long long vs = (long long)vstride_of(h);
    T *V = h->at<T>(L.vec);
    T *yb = V, *hv = V + vs, *r = V + 2 * vs, *d = V + 3 * vs, *hr = V + 4 * vs, *hd = V + 5 * vs, *g = V + 6 * vs;
    // the original backtracking test keeps ybar, h of the iterate and r, h at the step's origin w
    T *ysave = V + 7 * vs, *hsave = V + 8 * vs, *rw = V + 9 * vs, *hw = V + 10 * vs;
    const int bt = o->backtrack;
    T *rw_arg = bt == 1 ? rw : nullptr, *hw_arg = bt == 1 ? hw : nullptr;  // k_fbstep outputs
    T *ringS = h->at<T>(L.ringS), *ringY = h->at<T>(L.ringY);
    SolverScalars *sc = h->at<SolverScalars>(L.scal);
    double *part = h->at<double>(L.partials);
    const DualView<T> dv = make_view<T>(h);
    const int grid = red_grid(m);
    const bool nama = method == 0;
    const size_t tabb = comp_tab_bytes(dv);
    // general maps: the primal vectors ([x; u] layout) of x(ybar), x_lin(r), x_lin(d), and a copy of
    // the first (the original backtracking rule restores it); f(x) is evaluated from them
    const bool fg = h->fg;
    const DualView<T> sv = make_sel_view<T>(h);
    const int sgrid = red_grid(sv.m);
    const size_t stabb = comp_tab_bytes(sv);
    const long long ps = (long long)((h->msel + 63) / 64 * 64);
    T *P = fg ? h->at<T>(h->L.pvec) : nullptr;
    T *pvh = fg ? P : nullptr, *pvr = fg ? P + ps : nullptr, *pvd = fg ? P + 2 * ps : nullptr;
    T *psave = fg ? P + 3 * ps : nullptr;

    cudaEvent_t e0, e1;
    STO_CUDA(h, cudaEventCreate(&e0));
    STO_CUDA(h, cudaEventCreate(&e1));
    STO_CUDA(h, cudaEventRecord(e0, st));
    const int64_t calls0 = h->solve_calls;
    const int64_t launches0 = h->launches;

    SolverScalars *hs = h->host_scal;
    std::memset(hs, 0, sizeof(SolverScalars));
    hs->lambda = o->lambda;
    hs->tol = o->tol;
    hs->eps_curv = o->eps_curv;
    hs->mem = o->lbfgs_mem;
    hs->max_ls = o->max_ls;
    hs->method = method;
    // look-ahead needs an iteration whose kernels the host does not have to inspect: a fixed
    // step (no backtracking test between the kernels) and the selection maps
    const bool ahead = bt == 0 && !fg;
    hs->lookahead = ahead ? 1 : 0;
    STO_CUDA(h, cudaMemcpyAsync(sc, hs, sizeof(SolverScalars), cudaMemcpyHostToDevice, st));
    // the host mirror is rewritten below; make sure the upload has consumed it
    STO_CUDA(h, cudaStreamSynchronize(st));

    // line-search candidate groups: 4, 8, then the rest up to max_ls halvings
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

    auto full_solve = [&]() -> sto_status {
        const void *ys[1] = {yb};
        void *hs_[1] = {hv};
        void *po[1] = {pvh};
        return solve_round(h, ys, x0v, hs_, 1, false, true, st, nullptr, fg ? po : nullptr, &sc->stop);
    };
    auto lin_solve = [&](T *in, T *out, T *pout) -> sto_status {
        const void *ys[1] = {in};
        void *hs_[1] = {out};
        void *po[1] = {pout};
        return solve_round(h, ys, nullptr, hs_, 1, true, true, st, nullptr, fg ? po : nullptr, &sc->stop);
    };

    k_scale_in<T><<<grid, kThreads, 0, st>>>(dv, static_cast<const T *>(yv), yb);
    h->launches += 1;
    sto_status s = full_solve();
    if (s != STO_OK) return s;
    // k_point with the backtracking reductions the rule needs (with general maps, f(x) at the
    // point from its primal first)
    const bool gen = h->general;  // some element's term is not the box indicator
    auto point = [&](int pair, const T *rwp, const T *hwp) {
        if (fg) {
            k_fcost<T><<<sgrid, kThreads, stabb, st>>>(sv, pvh, sc, part);
            h->launches += 1;
        }
#define STO_POINT(BT, G) \
    k_point<T, BT, G><<<grid, kThreads, tabb, st>>>(dv, yb, hv, r, ringS, ringY, vs, pair, sc, part, rwp, hwp)
        if (bt == 1) {
            if (gen) STO_POINT(1, true); else STO_POINT(1, false);
        } else if (bt == 2) {
            if (gen) STO_POINT(2, true); else STO_POINT(2, false);
        } else {
            if (gen) STO_POINT(0, true); else STO_POINT(0, false);
        }
#undef STO_POINT
    };
    point(0, hv, hv);  // (with BT = 1 the w terms of this call are not used)
    h->launches += 1;
    if (!nama) {
        if ((s = lin_solve(r, hr, pvr)) != STO_OK) return s;
        k_grad<T><<<grid, kThreads, 0, st>>>(m, r, hr, g, ringS, ringY, vs, sc, part);
        h->launches += 1;
    }
    // Backtracking (Section III-B): halve lambda, empty the L-BFGS memory and re-evaluate the
    // residual (and for MINFBE the FBE gradient) at the current iterate, whose x(ybar) does not
    // depend on lambda.
    double lam = o->lambda;
    int halvings = 0;
    auto halve = [&]() -> sto_status {
        lam *= 0.5;
        ++halvings;
        k_set_lambda<<<1, 1, 0, st>>>(sc, lam);
        point(0, hv, hv);
        h->launches += 2;
        if (!nama) {
            const sto_status e = lin_solve(r, hr, pvr);
            if (e != STO_OK) return e;
            k_grad<T><<<grid, kThreads, 0, st>>>(m, r, hr, g, ringS, ringY, vs, sc, part);
            h->launches += 1;
        }
        return STO_OK;
    };
    auto read_head = [&]() -> sto_status {
        STO_CUDA(h, cudaMemcpyAsync(hs, sc, kScalHead, cudaMemcpyDeviceToHost, st));
        STO_CUDA(h, cudaStreamSynchronize(st));
        return STO_OK;
    };
    // lambda ||S H x_lin(r)|| > eps'' ||r||, i.e. eq. (simple-backtracking) with
    // T(y) - y = -lambda r and grad fhat(T(y)) - grad fhat(y) = lambda S H x_lin(r)
    auto simple_fails = [&]() { return lam * lam * hs->hr2 > o->bt_param * o->bt_param * hs->r2; };
    // One iteration (the FB step and the L-BFGS update around it); restart = the iteration was
    // abandoned for a step-size halving (backtracking rules), to be tried again.
    auto body = [&](bool &restart) -> sto_status {
        sto_status s;
        restart = false;
        T *gdir = nama ? r : g;
        lb_direction<T>(o->lbfgs_mem, grid, st, m, gdir, ringS, ringY, vs, sc, part, d);
        h->launches += 2 + ng + 2;  // L-BFGS pair, line-search groups, FB step, residual pass
        if (nama) {
            const void *ys[2] = {r, d};
            void *outs[2] = {hr, hd};
            void *po[2] = {pvr, pvd};
            if ((s = solve_round(h, ys, nullptr, outs, 2, true, true, st, nullptr, fg ? po : nullptr, &sc->stop)) !=
                STO_OK)
                return s;
            if (bt == 2) {  // NAMA: the test needs x_lin(r) of this round
                k_norm2<T><<<grid, kThreads, 0, st>>>(m, hr, sc, part);
                h->launches += 1;
                if ((s = read_head()) != STO_OK) return s;
                if (simple_fails()) {
                    if ((s = halve()) != STO_OK) return s;
                    { restart = true; return STO_OK; }
                }
            }
        } else {
            if ((s = lin_solve(d, hd, pvd)) != STO_OK) return s;
        }
        if (fg) {  // f along the line search's affine primal
            k_fquad<T><<<sgrid, kThreads, stabb, st>>>(sv, pvh, pvr, pvd, nama ? 1 : 0, sc, part);
            h->launches += 1;
        }
        for (int k = 0; k < ng; ++k) {
            const int last = k == ng - 1;
#define STO_LS(J, G) \
    k_ls<T, J, G><<<grid, kThreads, tabb, st>>>(dv, yb, hv, r, d, hr, hd, nama, gfirst[k], gcount[k], last, sc, part)
            if (k == 0) {
                if (gen) STO_LS(4, true); else STO_LS(4, false);
            } else if (k == 1) {
                if (gen) STO_LS(8, true); else STO_LS(8, false);
            } else {
                if (gen) STO_LS(19, true); else STO_LS(19, false);
            }
#undef STO_LS
        }
        if (bt == 1) {
            STO_CUDA(h, cudaMemcpyAsync(ysave, yb, (size_t)m * sizeof(T), cudaMemcpyDeviceToDevice, st));
            STO_CUDA(h, cudaMemcpyAsync(hsave, hv, (size_t)m * sizeof(T), cudaMemcpyDeviceToDevice, st));
            if (fg) STO_CUDA(h, cudaMemcpyAsync(psave, pvh, (size_t)sv.m * sizeof(T), cudaMemcpyDeviceToDevice, st));
        }
        if (gen)
            k_fbstep<T, true><<<grid, kThreads, tabb, st>>>(dv, yb, hv, r, d, hr, hd, nama, ringS, vs, sc, rw_arg, hw_arg);
        else
            k_fbstep<T, false><<<grid, kThreads, tabb, st>>>(dv, yb, hv, r, d, hr, hd, nama, ringS, vs, sc, rw_arg, hw_arg);
        if ((s = full_solve()) != STO_OK) return s;
        point(nama ? 1 : 0, rw, hw);
        if (bt == 1) {
            // eq. (original-backtracking) at w: for the quadratic fhat it reads
            // <r_w, h(T(w)) - h(w)> > (1 - beta) ||r_w||^2; on failure the step is rejected
            if ((s = read_head()) != STO_OK) return s;
            if (hs->nan_flag == 0 && hs->bt_a > (1.0 - o->bt_param) * hs->bt_b) {
                STO_CUDA(h, cudaMemcpyAsync(yb, ysave, (size_t)m * sizeof(T), cudaMemcpyDeviceToDevice, st));
                STO_CUDA(h, cudaMemcpyAsync(hv, hsave, (size_t)m * sizeof(T), cudaMemcpyDeviceToDevice, st));
                if (fg)
                    STO_CUDA(h, cudaMemcpyAsync(pvh, psave, (size_t)sv.m * sizeof(T), cudaMemcpyDeviceToDevice, st));
                if ((s = halve()) != STO_OK) return s;
                { restart = true; return STO_OK; }
            }
        }
        if (!nama) {
            if ((s = lin_solve(r, hr, pvr)) != STO_OK) return s;
            k_grad<T><<<grid, kThreads, 0, st>>>(m, r, hr, g, ringS, ringY, vs, sc, part);
            h->launches += 1;
        }
        STO_CUDA(h, cudaGetLastError());
        return STO_OK;
    };
    sto_status result = STO_OK;
    int iters = 0;
    if (ahead) {
        // One iteration of look-ahead: iteration k + 1 is enqueued before the host reads the
        // result of iteration k, so the GPU does not idle on the host's decision.  Once a
        // residual pass finds the run converged (or a NaN), it sets the device's stop flag and
        // the look-ahead iteration's kernels and solve rounds do nothing; its solve calls and
        // round timings are taken back below (its launches did happen and stay counted).
        SolverScalars *hb[2] = {hs, h->host_scal2};
        cudaEvent_t ev[2];
        STO_CUDA(h, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        STO_CUDA(h, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        auto head_to = [&](int k) -> sto_status {
            STO_CUDA(h, cudaMemcpyAsync(hb[k & 1], sc, kScalHead, cudaMemcpyDeviceToHost, st));
            STO_CUDA(h, cudaEventRecord(ev[k & 1], st));
            return STO_OK;
        };
        const int64_t *cnt[3] = {&h->solve_calls, &h->solve_launches, &h->solve_rhs};
        int64_t saved[3] = {0, 0, 0};
        size_t saved_ev = 0;
        bool pending = false;
        if ((s = head_to(0)) != STO_OK) return s;
        while (true) {
            pending = false;
            if (iters < o->max_iter) {
                for (int q = 0; q < 3; ++q) saved[q] = *cnt[q];
                saved_ev = h->ev_used;
                bool restart;
                if ((s = body(restart)) != STO_OK) return s;
                if ((s = head_to(iters + 1)) != STO_OK) return s;
                pending = true;
            }
            STO_CUDA(h, cudaEventSynchronize(ev[iters & 1]));
            const SolverScalars *hk = hb[iters & 1];
            if (hk->nan_flag) {
                result = STO_ERR_NUMERICAL;
                h->err = "NaN or Inf in the residual";
                break;
            }
            if (hk->res_inf <= o->tol) break;
            if (iters >= o->max_iter) {
                result = STO_NOT_CONVERGED;
                break;
            }
            ++iters;
        }
        if (pending) {  // the look-ahead iteration did nothing on the device
            h->solve_calls = saved[0];
            h->solve_launches = saved[1];
            h->solve_rhs = saved[2];
            h->ev_used = saved_ev;
        }
        STO_CUDA(h, cudaStreamSynchronize(st));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    } else {
    while (true) {
        if ((s = read_head()) != STO_OK) return s;
        if (hs->nan_flag) {
            result = STO_ERR_NUMERICAL;
            h->err = "NaN or Inf in the residual";
            break;
        }
        if (hs->res_inf <= o->tol) break;
        if (iters >= o->max_iter || halvings > o->max_halvings) {
            result = STO_NOT_CONVERGED;
            break;
        }
        if (bt == 2 && !nama && simple_fails()) {  // MINFBE: ||hr||^2 came with the FBE gradient
            if ((s = halve()) != STO_OK) return s;
            continue;
        }
        bool restart;
        if ((s = body(restart)) != STO_OK) return s;
        if (restart) continue;
        ++iters;
    }
    }
    h->launches += 1;
    k_finish_out<T><<<grid, kThreads, 0, st>>>(dv, yb, hv, sc, static_cast<T *>(yv), static_cast<T *>(zv));
    if (xv) {
        k_primal_out<T><<<sgrid, kThreads, 0, st>>>(sv, fg ? pvh : hv, static_cast<T *>(xv), static_cast<T *>(uv));
        h->launches += 1;
        // the root state is the parameter p
        STO_CUDA(h, cudaMemcpyAsync(xv, x0v, h->nx * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }
    STO_CUDA(h, cudaEventRecord(e1, st));
    STO_CUDA(h, cudaMemcpyAsync(hs, sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    {
        const sto_status es = check_round_error(h, st);
        if (es != STO_OK) result = es;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iters = iters;
        info->solve_calls = (int32_t)(h->solve_calls - calls0);
        info->status = result;
        info->ls_zero = hs->ls_zero;
        info->res_inf = hs->res_inf;
        info->fbe = hs->phi;
        info->ms = ms;
        info->launches = (int32_t)(h->launches - launches0);
        info->halvings = halvings;
        info->lambda = lam;
    }
    STO_CUDA(h, cudaGetLastError());
    return result;
}

// GPAD on the preconditioned dual.  Iteration k solves at the extrapolated point w_k
// (w_0 = ybar_0), tests ||z(w_k) - Hx(w_k)||_inf <= tol and otherwise takes the step; the
// result is the point of the last test, w_k, with x(w_k) and z(w_k).  theta_{-1} = theta_0 = 1,
// theta_{k+1} = (sqrt(theta_k^4 + 4 theta_k^2) - theta_k^2) / 2.
template <class T>
sto_status gpad_impl(stotree_t h, const sto_opts *o, const void *x0v, void *yv, void *xv, void *uv, void *zv,
                     sto_info *info, cudaStream_t st) {
    const Layout &L = h->L;
    const long long vs = (long long)vstride_of(h);
    T *V = h->at<T>(L.vec);
    T *yb = V, *hv = V + vs, *w = V + 3 * vs, *wn = V + 5 * vs;
    SolverScalars *sc = h->at<SolverScalars>(L.scal);
    double *part = h->at<double>(L.partials);
    const DualView<T> dv = make_view<T>(h);
    const int grid = red_grid(dv.m);
    const size_t tabb = comp_tab_bytes(dv);

    cudaEvent_t e0, e1;
    STO_CUDA(h, cudaEventCreate(&e0));
    STO_CUDA(h, cudaEventCreate(&e1));
    STO_CUDA(h, cudaEventRecord(e0, st));
    const int64_t launches0 = h->launches;

    SolverScalars *hs = h->host_scal;
    std::memset(hs, 0, sizeof(SolverScalars));
    hs->lambda = o->lambda;
    hs->tol = o->tol;
    hs->method = 2;
    STO_CUDA(h, cudaMemcpyAsync(sc, hs, sizeof(SolverScalars), cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaStreamSynchronize(st));

    k_scale_in<T><<<grid, kThreads, 0, st>>>(dv, static_cast<const T *>(yv), yb);
    STO_CUDA(h, cudaMemcpyAsync(w, yb, (size_t)dv.m * sizeof(T), cudaMemcpyDeviceToDevice, st));
    h->launches += 1;
    // One step of look-ahead: step k + 1 is enqueued before the host reads step k's residual,
    // so the GPU does not idle on the host's decision.  w and S H x(w) alternate between two
    // buffers; once a step stops the run (device flag), the look-ahead step leaves the
    // buffers of the stopped step alone.
    T *wb[2] = {w, wn}, *hb[2] = {hv, V + 11 * vs};
    // general maps: the primal of each buffer's solve, for f(x) and the returned x, u
    const bool fg = h->fg;
    const DualView<T> sv = make_sel_view<T>(h);
    const int sgrid = red_grid(sv.m);
    const long long ps = (long long)((h->msel + 63) / 64 * 64);
    T *pb[2] = {fg ? h->at<T>(h->L.pvec) : nullptr, fg ? h->at<T>(h->L.pvec) + ps : nullptr};
    SolverScalars *hbuf[2] = {hs, h->host_scal2};
    cudaEvent_t ev[2];
    STO_CUDA(h, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    STO_CUDA(h, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    double theta = 1.0;
    auto enqueue = [&](int k) -> sto_status {
        const double theta_next = 0.5 * (std::sqrt(theta * theta * theta * theta + 4.0 * theta * theta) - theta * theta);
        const T beta = (T)(theta_next * (1.0 / theta - 1.0));
        theta = theta_next;
        const void *ys[1] = {wb[k & 1]};
        void *hs_[1] = {hb[k & 1]};
        void *po[1] = {pb[k & 1]};
        const sto_status s = solve_round(h, ys, x0v, hs_, 1, false, true, st, nullptr, fg ? po : nullptr);
        if (s != STO_OK) return s;
        if (fg) {
            k_fcost<T><<<sgrid, kThreads, comp_tab_bytes(sv), st>>>(sv, pb[k & 1], sc, part);
            h->launches += 1;
        }
        if (h->general)
            k_gpad<T, true><<<grid, kThreads, tabb, st>>>(dv, wb[k & 1], hb[k & 1], yb, wb[(k + 1) & 1], beta, k,
                                                          o->max_iter, sc, part);
        else
            k_gpad<T, false><<<grid, kThreads, tabb, st>>>(dv, wb[k & 1], hb[k & 1], yb, wb[(k + 1) & 1], beta, k,
                                                           o->max_iter, sc, part);
        h->launches += 1;
        STO_CUDA(h, cudaGetLastError());
        STO_CUDA(h, cudaMemcpyAsync(hbuf[k & 1], sc, kScalHead, cudaMemcpyDeviceToHost, st));
        STO_CUDA(h, cudaEventRecord(ev[k & 1], st));
        return STO_OK;
    };
    sto_status result = STO_OK;
    int iters = 0;
    sto_status s = enqueue(0);
    while (s == STO_OK) {
        if (iters + 1 <= o->max_iter && (s = enqueue(iters + 1)) != STO_OK) break;
        STO_CUDA(h, cudaEventSynchronize(ev[iters & 1]));
        const SolverScalars *hk = hbuf[iters & 1];
        if (hk->nan_flag) {
            result = STO_ERR_NUMERICAL;
            h->err = "NaN or Inf in the residual";
            break;
        }
        if (hk->res_inf <= o->tol) break;
        if (iters >= o->max_iter) {
            result = STO_NOT_CONVERGED;
            break;
        }
        ++iters;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (s != STO_OK) return s;
    const double res_final = hbuf[iters & 1]->res_inf, phi_final = hbuf[iters & 1]->phi;
    w = wb[iters & 1];
    hv = hb[iters & 1];
    h->launches += 1;
    k_finish_out<T><<<grid, kThreads, 0, st>>>(dv, w, hv, sc, static_cast<T *>(yv), static_cast<T *>(zv));
    if (xv) {
        k_primal_out<T><<<sgrid, kThreads, 0, st>>>(sv, fg ? pb[iters & 1] : hv, static_cast<T *>(xv),
                                                   static_cast<T *>(uv));
        h->launches += 1;
        STO_CUDA(h, cudaMemcpyAsync(xv, x0v, h->nx * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }
    STO_CUDA(h, cudaEventRecord(e1, st));
    STO_CUDA(h, cudaMemcpyAsync(hs, sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    {
        const sto_status es = check_round_error(h, st);
        if (es != STO_OK) result = es;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iters = iters;
        info->solve_calls = iters + 1;  // the look-ahead solve is not one of the method's calls
        info->status = result;
        info->ls_zero = 0;
        info->res_inf = res_final;
        info->fbe = phi_final;
        info->ms = ms;
        info->launches = (int32_t)(h->launches - launches0);
        info->halvings = 0;
        info->lambda = o->lambda;
    }
    STO_CUDA(h, cudaGetLastError());
    return result;
}

template <class T>
sto_status lambda_impl(stotree_t h, void *r0, int iters, double safety, double *lambda, double *Lout,
                       cudaStream_t st) {
    const int m = (int)h->m;
    const long long vs = (long long)vstride_of(h);
    T *hr = h->at<T>(h->L.vec) + 4 * vs;
    T *r = static_cast<T *>(r0);
    SolverScalars *sc = h->at<SolverScalars>(h->L.scal);
    double *part = h->at<double>(h->L.partials);
    const int grid = red_grid(m);
    STO_CUDA(h, cudaMemsetAsync(sc, 0, sizeof(SolverScalars), st));
    k_normalize<T><<<grid, kThreads, 0, st>>>(m, r, sc, part);
    k_scale_by<T><<<grid, kThreads, 0, st>>>(m, r, sc);
    for (int k = 0; k < iters; ++k) {
        const void *ys[1] = {r};
        void *outs[1] = {hr};
        sto_status s = solve_round(h, ys, nullptr, outs, 1, true, true, st);
        if (s != STO_OK) return s;
        k_power_dots<T><<<grid, kThreads, 0, st>>>(m, r, hr, sc, part);
        k_power_next<T><<<grid, kThreads, 0, st>>>(m, r, hr, sc);
    }
    SolverScalars *hs = h->host_scal;
    STO_CUDA(h, cudaMemcpyAsync(hs, sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    const sto_status es = check_round_error(h, st);
    if (es != STO_OK) return es;
    if (!(hs->pw_L > 0.0)) {
        h->err = "power iteration gave a non-positive estimate";
        return STO_ERR_NUMERICAL;
    }
    *lambda = safety / hs->pw_L;
    if (Lout) *Lout = hs->pw_L;
    return STO_OK;
}

// ------------------------------- FP64 KKT check ---------------------------------------
// Costates mu^j = grad_x^j of f + <y, Hx> through the dynamics, from the leaves up:
//   leaf  mu^l = 2 pi^l P_N x^l + pi^l p_N + y^l
//   j>=1  mu^j = 2 pi^j Q x^j + pi^j q + y_x^j + sum_k A^k' mu^k
// and at every nonleaf i the input stationarity 2 pi^i R u^i + pi^i r + y_u^i + sum_j B^j' mu^j.
__device__ void atomic_max_nonneg(double *addr, double v) {
    if (!(v >= 0.0)) v = INFINITY;  // NaN counts as a failure
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class T, class TY>
__global__ void k_kkt_stage(int first, int nx, int nu, int Np, int ld64, const int *cbeg, const int *ccnt,
                            const double *prob, const double *G64, const double *cost64, const T *x, const T *u,
                            const TY *y, double *mu, double *out) {
    const int i = first + blockIdx.x;
    const int nxu = nx + nu;
    const long long oi = i < Np ? (long long)i * nxu : (long long)Np * nxu + (long long)(i - Np) * nx;
    const double pi = prob[i];
    const double *Q = cost64, *R = cost64 + nx, *PN = cost64 + nx + nu, *q = cost64 + 2 * nx + nu,
                 *r = cost64 + 3 * nx + nu, *pN = cost64 + 3 * nx + 2 * nu;
    for (int c = threadIdx.x; c < nxu; c += blockDim.x) {
        double acc = 0.0;
        if (i < Np) {
            for (int j = cbeg[i]; j < cbeg[i] + ccnt[i]; ++j) {
                const double *Gj = G64 + (size_t)j * nx * ld64;
                const double *mj = mu + (size_t)j * nx;
                for (int k = 0; k < nx; ++k) acc += Gj[(size_t)k * ld64 + c] * mj[k];
            }
        }
        if (c < nx) {
            if (i == 0) continue;
            const double xv = (double)x[(size_t)i * nx + c];
            const double loc = i < Np ? 2.0 * pi * Q[c] * xv + pi * q[c] : 2.0 * pi * PN[c] * xv + pi * pN[c];
            mu[(size_t)i * nx + c] = loc + (double)y[oi + c] + acc;
        } else if (i < Np) {
            const int a = c - nx;
            const double res = 2.0 * pi * R[a] * (double)u[(size_t)i * nu + a] + pi * r[a] + (double)y[oi + c] + acc;
            atomic_max_nonneg(out + 1, fabs(res));
        }
    }
}

// One component's Fenchel-Young gap g(h) + g*(y) - y h (>= 0, zero exactly when y is in the
// subdifferential of g at h): g the indicator of [lo, hi] (kind 0, taken as 0: feasibility is
// out[2]), rho dist (kind 1) or rho Huber_delta(dist) (kind 2); g*(y) = sigma_[lo,hi](y), plus
// y^2 / (2 rho) for kind 2 (the conjugates' domains |y| <= rho, |y| <= rho delta are not imposed
// here: outputs 3 and 4 measure y against the subdifferential).  sigma(y) - y h is formed as
// y (hi - h) or y (lo - h), so no large terms cancel.
__device__ __forceinline__ double gap_term(double hv, double ye, double lo, double hi, int kind, double rho,
                                           double dl) {
    double t = ye > 0.0 ? ye * (hi - hv) : (ye < 0.0 ? ye * (lo - hv) : 0.0);
    if (kind != 0) {
        const double d = fmax(lo - hv, 0.0) + fmax(hv - hi, 0.0);
        t += kind == 1 ? rho * d : rho * (d <= dl ? 0.5 * d * d : dl * (d - 0.5 * dl)) + ye * ye / (2.0 * rho);
    }
    return t;
}
// Sum of the gap terms of a block into partial[blockIdx.x] (fixed order inside the block; the host
// adds the blocks' partials in order).
__device__ __forceinline__ void block_gap_partial(double v, double *partial) {
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_kkt_elem(int Nn, int nx, int nu, int Np, int ld64, const int *parent,
                                                  const double *G64, const double *box64, const T *x0, const T *x,
                                                  const T *u, const T *y, double tol_act, double *out,
                                                  double *gap_part, int box_terms) {
    const int nxu = nx + nu;
    // dynamics residual per node and state component
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)(Nn - 1) * nx;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = 1 + (int)(e / nx), rr = (int)(e % nx);
        const int i = parent[j];
        const double *row = G64 + ((size_t)j * nx + rr) * ld64;
        double acc = row[nx + nu];
        for (int k = 0; k < nx; ++k) acc += row[k] * (double)(i == 0 ? x0[k] : x[(size_t)i * nx + k]);
        for (int k = 0; k < nu; ++k) acc += row[nx + k] * (double)u[(size_t)i * nu + k];
        atomic_max_nonneg(out + 0, fabs((double)x[(size_t)j * nx + rr] - acc));
    }
    if (!box_terms) return;  // general maps: k_kkt_fg_box checks z
    // box feasibility, complementarity, multiplier signs and the gap per dual entry
    const long long m = (long long)Np * nxu + (long long)(Nn - Np) * nx;
    double gap = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        int node, k, bi;
        double hv;
        if (e < (long long)Np * nxu) {
            node = (int)(e / nxu);
            k = (int)(e % nxu);
            if (k < nx) {
                hv = node == 0 ? (double)x0[k] : (double)x[(size_t)node * nx + k];
                bi = k;
            } else {
                hv = (double)u[(size_t)node * nu + (k - nx)];
                bi = k;
            }
        } else {
            const long long e2 = e - (long long)Np * nxu;
            node = Np + (int)(e2 / nx);
            k = (int)(e2 % nx);
            hv = (double)x[(size_t)node * nx + k];
            bi = k;
        }
        double lo = box64[bi], hi = box64[nxu + bi];
        const double rho = box64[2 * nxu + bi], dl = box64[3 * nxu + bi];
        int kind = (int)box64[4 * nxu + bi];
        const bool param = node == 0 && k < nx;  // the root state is the parameter: no term
        if (param) {
            lo = -INFINITY;
            hi = INFINITY;
            kind = 0;
        }
        const double ye = (double)y[e];
        if (!param) gap += gap_term(hv, ye, lo, hi, kind, rho, dl);
        if (kind == 0) {
            atomic_max_nonneg(out + 2, fmax(0.0, fmax(lo - hv, hv - hi)));
            const bool at_hi = hv >= hi - tol_act, at_lo = hv <= lo + tol_act;
            if (!at_hi && !at_lo) atomic_max_nonneg(out + 3, fabs(ye));
            double sgn = 0.0;
            if (at_hi && !at_lo) sgn = fmax(0.0, -ye);
            if (at_lo && !at_hi) sgn = fmax(0.0, ye);
            atomic_max_nonneg(out + 4, sgn);
        } else {
            // y must lie in the subdifferential [slo, shi] of g at Hx (bounds within tol_act
            // count as kinks); a single-valued subdifferential goes to out[3], a kink to out[4]
            double slo = 0.0, shi = 0.0;
            if (kind == 1) {
                if (hv > hi + tol_act) {
                    slo = shi = rho;
                } else if (hv < lo - tol_act) {
                    slo = shi = -rho;
                } else {
                    if (hv <= lo + tol_act) slo = -rho;
                    if (hv >= hi - tol_act) shi = rho;
                }
            } else {
                const double d = fmax(lo - hv, 0.0) + fmax(hv - hi, 0.0);
                const double gd = rho * fmin(d, dl);
                slo = shi = hv > hi ? gd : (hv < lo ? -gd : 0.0);
            }
            const double res = fmax(0.0, fmax(slo - ye, ye - shi));
            atomic_max_nonneg(out + (slo == shi ? 3 : 4), res);
        }
    }
    block_gap_partial(gap, gap_part);
}

// General maps: feasibility, complementarity and multiplier signs of the box on z = F x + G u
// (FN x at the leaves; the root's x is x0), z formed in FP64 from x and u.
template <class T>
__global__ void __launch_bounds__(256) k_kkt_fg_box(int Nn, int nx, int nu, int Np, int nc, int ncN,
                                                    const double *FG64, const double *zbox64, const T *x0,
                                                    const T *x, const T *u, const T *y, double tol_act, double *out,
                                                    double *gap_part) {
    const double *F = FG64, *G = FG64 + (size_t)nc * nx, *FN = G + (size_t)nc * nu;
    const int nb = nc + ncN;
    const long long m = (long long)Np * nc + (long long)(Nn - Np) * ncN;
    double gap = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        double z = 0.0;
        int bi;
        if (e < (long long)Np * nc) {
            const int i = (int)(e / nc), c = (int)(e - (long long)i * nc);
            const T *xi = i == 0 ? x0 : x + (size_t)i * nx;
            for (int k = 0; k < nx; ++k) z += F[(size_t)c * nx + k] * (double)xi[k];
            for (int a = 0; a < nu; ++a) z += G[(size_t)c * nu + a] * (double)u[(size_t)i * nu + a];
            bi = c;
        } else {
            const long long e2 = e - (long long)Np * nc;
            const int l = Np + (int)(e2 / ncN), c = (int)(e2 - (long long)(l - Np) * ncN);
            for (int k = 0; k < nx; ++k) z += FN[(size_t)c * nx + k] * (double)x[(size_t)l * nx + k];
            bi = nc + c;
        }
        const double lo = zbox64[bi], hi = zbox64[nb + bi], ye = (double)y[e];
        gap += gap_term(z, ye, lo, hi, 0, 0.0, 1.0);
        atomic_max_nonneg(out + 2, fmax(0.0, fmax(lo - z, z - hi)));
        const bool at_hi = z >= hi - tol_act, at_lo = z <= lo + tol_act;
        if (!at_hi && !at_lo) atomic_max_nonneg(out + 3, fabs(ye));
        double sgn = 0.0;
        if (at_hi && !at_lo) sgn = fmax(0.0, -ye);
        if (at_lo && !at_hi) sgn = fmax(0.0, ye);
        atomic_max_nonneg(out + 4, sgn);
    }
    block_gap_partial(gap, gap_part);
}

template <class T>
sto_status kkt_impl(stotree_t h, const void *x0, const void *x, const void *u, const void *y, double tol_act,
                    double *out, cudaStream_t st) {
    const Layout &L = h->L;
    double *mu = h->at<double>(L.kkt);
    double *dout = mu + (size_t)h->Nn * h->nx + (size_t)h->Np * h->nu;
    double *hty = dout + 64;  // general maps: H'y in FP64, laid out like [x; u]
    constexpr int kGapBlocks = 592;
    double *gap_part = h->at<double>(L.partials);  // the gap's per-block sums (the solvers' scratch)
    STO_CUDA(h, cudaMemsetAsync(dout, 0, 8 * sizeof(double), st));
    if (h->fg) {
        const sto_status s = fg_ht(h, y, hty, true, st);
        if (s != STO_OK) return s;
    }
    for (int t = h->N; t >= 0; --t) {
        const int first = h->soff[t], count = h->soff[t + 1] - first;
        if (h->fg)
            k_kkt_stage<T, double><<<count, 128, 0, st>>>(first, h->nx, h->nu, h->Np, h->ld64, h->at<int>(L.cbeg),
                                                          h->at<int>(L.ccnt), h->at<double>(L.prob64),
                                                          h->at<double>(L.G64), h->at<double>(L.cost64),
                                                          static_cast<const T *>(x), static_cast<const T *>(u), hty,
                                                          mu, dout);
        else
            k_kkt_stage<T, T><<<count, 128, 0, st>>>(first, h->nx, h->nu, h->Np, h->ld64, h->at<int>(L.cbeg),
                                                     h->at<int>(L.ccnt), h->at<double>(L.prob64), h->at<double>(L.G64),
                                                     h->at<double>(L.cost64), static_cast<const T *>(x),
                                                     static_cast<const T *>(u), static_cast<const T *>(y), mu, dout);
    }
    k_kkt_elem<T><<<kGapBlocks, 256, 0, st>>>(h->Nn, h->nx, h->nu, h->Np, h->ld64, h->at<int>(L.parent),
                                              h->at<double>(L.G64), h->at<double>(L.box64),
                                              static_cast<const T *>(x0), static_cast<const T *>(x),
                                              static_cast<const T *>(u), static_cast<const T *>(y), tol_act, dout,
                                              gap_part, h->fg ? 0 : 1);
    if (h->fg)
        k_kkt_fg_box<T><<<kGapBlocks, 256, 0, st>>>(h->Nn, h->nx, h->nu, h->Np, h->nc, h->ncN,
                                                    h->at<double>(L.FG64), h->at<double>(L.zbox64),
                                                    static_cast<const T *>(x0), static_cast<const T *>(x),
                                                    static_cast<const T *>(u), static_cast<const T *>(y), tol_act,
                                                    dout, gap_part);
    std::vector<double> parts(kGapBlocks);
    STO_CUDA(h, cudaMemcpyAsync(out, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaMemcpyAsync(parts.data(), gap_part, kGapBlocks * sizeof(double), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    STO_CUDA(h, cudaGetLastError());
    double gap = 0.0;
    for (double v : parts) gap += v;  // blocks in order
    out[5] = gap;
    return STO_OK;
}

}  // namespace

sto_status solver_run(stotree_t h, int method, const sto_opts *o, const void *x0, void *y, void *x, void *u,
                      void *z, sto_info *info, cudaStream_t st) {
    if (method == 2)
        return h->prec == STO_FP64 ? gpad_impl<double>(h, o, x0, y, x, u, z, info, st)
                                   : gpad_impl<float>(h, o, x0, y, x, u, z, info, st);
    return h->prec == STO_FP64 ? solver_impl<double>(h, method, o, x0, y, x, u, z, info, st)
                               : solver_impl<float>(h, method, o, x0, y, x, u, z, info, st);
}

sto_status lambda_run(stotree_t h, void *r0, int iters, double safety, double *lambda, double *L, cudaStream_t st) {
    return h->prec == STO_FP64 ? lambda_impl<double>(h, r0, iters, safety, lambda, L, st)
                               : lambda_impl<float>(h, r0, iters, safety, lambda, L, st);
}

sto_status kkt_run(stotree_t h, const void *x0, const void *x, const void *u, const void *y, double tol_active,
                   double *out, cudaStream_t st) {
    return h->prec == STO_FP64 ? kkt_impl<double>(h, x0, x, u, y, tol_active, out, st)
                               : kkt_impl<float>(h, x0, x, u, y, tol_active, out, st);
}

}  // namespace sto
