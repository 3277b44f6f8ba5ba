// Algorithm 3 (dual gradient x(y)) and Algorithm 4 (Hessian-vector products) on the device.
//
// With the factor of Section III-D (see factor.cu), one solve round is
//   backward, stages t = N-1 .. 0, every parent i of the stage in parallel:
//     s^l    = y^l / 2 + pi^l p_N / 2                    (leaf children, formed on the fly)
//     acc    = sum_{j in child(i)} G^j' s^j   with G^j = [A^j | B^j]  -> [A's ; B's]
//     v^i    = y_u^i / 2 + acc_B + gu^i
//     ubar^i = -Rbar^-1 v^i,     s^i = y_x^i / 2 + acc_A + K^i' v^i + gx^i
//   forward, stages t = 0 .. N:
//     x^0 = p,   x^j = G^j [x^i; u^i] + c^j,   u^j = K^j x^j + ubar^j
// and Algorithm 4 is the same with c, gu, gx, the leaf term and p set to zero.  Algorithm 3
// overwrites u^i, q^i in its child loop where Algorithm 4 accumulates; both accumulate here.
// Several right-hand sides share every matrix load (the parallel x(r), x(d) of Section III-C).
//
// Layout: G^j is nx rows of ldg reals (16-byte padded), row-major, node-major; the backward
// pass reads it in axpy form (warps over rows, lanes over 16-byte column groups) and the
// forward pass in dot form (one warp per row, shuffle reduction), both coalesced.
#include "internal.h"

namespace sto {
namespace {

template <class T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int n = 2;
};

template <class T>
__device__ __forceinline__ void v_fma(T s, const typename V16<T>::type &g, T *acc);
template <>
__device__ __forceinline__ void v_fma<float>(float s, const float4 &g, float *acc) {
    acc[0] = fmaf(s, g.x, acc[0]);
    acc[1] = fmaf(s, g.y, acc[1]);
    acc[2] = fmaf(s, g.z, acc[2]);
    acc[3] = fmaf(s, g.w, acc[3]);
}
template <>
__device__ __forceinline__ void v_fma<double>(double s, const double2 &g, double *acc) {
    acc[0] = fma(s, g.x, acc[0]);
    acc[1] = fma(s, g.y, acc[1]);
}

template <class T>
__device__ __forceinline__ T v_dot(const typename V16<T>::type &g, const T *x);
template <>
__device__ __forceinline__ float v_dot<float>(const float4 &g, const float *x) {
    return fmaf(g.x, x[0], fmaf(g.y, x[1], fmaf(g.z, x[2], g.w * x[3])));
}
template <>
__device__ __forceinline__ double v_dot<double>(const double2 &g, const double *x) {
    return fma(g.x, x[0], g.y * x[1]);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
struct SolveArgs {
    int nx, nu, ldg, ldk, ldr, Np, nxu;
    const T *G, *K, *Ri, *gu, *gx, *c, *sqp, *pN;
    const double *prob;
    const int *cbeg, *ccnt, *parent;
    const T *y[kMaxRhs];
    T *h[kMaxRhs];
    const T *x0;
    T *s, *ubar, *xs, *us;  // scratch, [kMaxRhs][Nn][nx] and [kMaxRhs][Np][nu]
    long long s_stride, u_stride;
    int homog, scaled;
};

__device__ __forceinline__ long long dual_off(int i, int Np, int nxu, int nx) {
    return i < Np ? (long long)i * nxu : (long long)Np * nxu + (long long)(i - Np) * nx;
}

constexpr int kWarps = 8;

// Backward pass over one stage: one CTA per parent node.
template <class T, int NR, int KV>
__global__ void __launch_bounds__(256) k_bwd(SolveArgs<T> a, int first) {
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int nx = a.nx, nu = a.nu, ldg = a.ldg;
    T *s_in = sm;                              // [NR][nx]
    T *part = s_in + NR * nx;                  // [kWarps][NR][ldg]
    T *accs = part + kWarps * NR * ldg;        // [NR][ldg]
    T *v = accs + NR * ldg;                    // [NR][nu]
    const int i = first + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvec = ldg / VN;
    const T sci = a.scaled ? a.sqp[i] : T(1);

    T acc[NR][KV][VN];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int q = 0; q < KV; ++q)
#pragma unroll
            for (int e = 0; e < VN; ++e) acc[k][q][e] = T(0);

    const int jb = a.cbeg[i], je = jb + a.ccnt[i];
    for (int j = jb; j < je; ++j) {
        if (j >= a.Np) {  // leaf: s^l = y^l / 2 + pi^l p_N / 2
            const long long o = dual_off(j, a.Np, a.nxu, nx);
            const T scj = a.scaled ? a.sqp[j] : T(1);
            const T cj = a.homog ? T(0) : T(0.5 * a.prob[j]);
            for (int e = threadIdx.x; e < NR * nx; e += blockDim.x) {
                const int k = e / nx, r = e - k * nx;
                s_in[e] = T(0.5) * scj * a.y[k][o + r] + cj * a.pN[r];
            }
        } else {
            for (int e = threadIdx.x; e < NR * nx; e += blockDim.x) {
                const int k = e / nx, r = e - k * nx;
                s_in[e] = a.s[k * a.s_stride + (long long)j * nx + r];
            }
        }
        __syncthreads();
        const VT *Gj = reinterpret_cast<const VT *>(a.G + (size_t)j * nx * ldg);
        for (int r = warp; r < nx; r += kWarps) {
            T sr[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) sr[k] = s_in[k * nx + r];
            const VT *row = Gj + (size_t)r * nvec;
#pragma unroll
            for (int q = 0; q < KV; ++q) {
                const int cv = lane + 32 * q;
                if (cv < nvec) {
                    const VT g = __ldg(row + cv);
#pragma unroll
                    for (int k = 0; k < NR; ++k) v_fma<T>(sr[k], g, acc[k][q]);
                }
            }
        }
        __syncthreads();
    }
    // cross-warp reduction of the column sums
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int q = 0; q < KV; ++q) {
            const int cv = lane + 32 * q;
            if (cv < nvec) {
#pragma unroll
                for (int e = 0; e < VN; ++e) part[(warp * NR + k) * ldg + cv * VN + e] = acc[k][q][e];
            }
        }
    __syncthreads();
    for (int e = threadIdx.x; e < NR * ldg; e += blockDim.x) {
        const int k = e / ldg, c = e - k * ldg;
        T sum = T(0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += part[(w * NR + k) * ldg + c];
        accs[e] = sum;
    }
    __syncthreads();
    const long long oi = (long long)i * a.nxu;
    for (int e = threadIdx.x; e < NR * nu; e += blockDim.x) {
        const int k = e / nu, c = e - k * nu;
        v[e] = T(0.5) * sci * a.y[k][oi + nx + c] + accs[k * ldg + nx + c] +
               (a.homog ? T(0) : a.gu[(size_t)i * nu + c]);
    }
    __syncthreads();
    // ubar = -Rbar^-1 v (Ri holds -Rbar^-1, symmetric) and s = y_x/2 + A's + K'v + gx
    const T *Ri = a.Ri + (size_t)i * nu * a.ldr;
    const T *Ki = a.K + (size_t)i * nu * a.ldk;
    for (int e = threadIdx.x; e < NR * (nu + nx); e += blockDim.x) {
        const int k = e / (nu + nx), c = e - k * (nu + nx);
        const T *vk = v + k * nu;
        if (c < nu) {
            T sum = T(0);
            for (int r = 0; r < nu; ++r) sum += vk[r] * Ri[(size_t)r * a.ldr + c];
            a.ubar[k * a.u_stride + (long long)i * nu + c] = sum;
        } else {
            const int cx = c - nu;
            T sum = T(0);
            for (int r = 0; r < nu; ++r) sum += vk[r] * Ki[(size_t)r * a.ldk + cx];
            a.s[k * a.s_stride + (long long)i * nx + cx] = T(0.5) * sci * a.y[k][oi + cx] + accs[k * ldg + cx] + sum +
                                                           (a.homog ? T(0) : a.gx[(size_t)i * nx + cx]);
        }
    }
}

// Forward pass over one stage: one CTA per node (the root when first == 0).
template <class T, int NR>
__global__ void __launch_bounds__(256) k_fwd(SolveArgs<T> a, int first) {
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int nx = a.nx, nu = a.nu, ldg = a.ldg, ldk = a.ldk;
    T *xu = sm;                 // [NR][ldg]
    T *xj = xu + NR * ldg;      // [NR][ldk]
    const int j = first + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T scj = a.scaled ? a.sqp[j] : T(1);
    if (j == 0) {
        for (int e = threadIdx.x; e < NR * ldk; e += blockDim.x) {
            const int k = e / ldk, r = e - k * ldk;
            xj[e] = (r < nx && !a.homog) ? a.x0[r] : T(0);
        }
        __syncthreads();
    } else {
        const int i = a.parent[j];
        for (int e = threadIdx.x; e < NR * ldg; e += blockDim.x) {
            const int k = e / ldg, c = e - k * ldg;
            T v = T(0);
            if (c < nx)
                v = a.xs[k * a.s_stride + (long long)i * nx + c];
            else if (c < nx + nu)
                v = a.us[k * a.u_stride + (long long)i * nu + (c - nx)];
            xu[e] = v;
        }
        for (int e = threadIdx.x; e < NR * ldk; e += blockDim.x) xj[e] = T(0);
        __syncthreads();
        const int nvec = ldg / VN;
        const VT *Gj = reinterpret_cast<const VT *>(a.G + (size_t)j * nx * ldg);
        for (int r = warp; r < nx; r += kWarps) {
            const VT *row = Gj + (size_t)r * nvec;
            T sum[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) sum[k] = T(0);
            for (int cv = lane; cv < nvec; cv += 32) {
                const VT g = __ldg(row + cv);
#pragma unroll
                for (int k = 0; k < NR; ++k) sum[k] += v_dot<T>(g, xu + k * ldg + cv * VN);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const T tot = warp_sum(sum[k]);
                if (lane == 0) xj[k * ldk + r] = tot + (a.homog ? T(0) : a.c[(size_t)j * nx + r]);
            }
        }
        __syncthreads();
    }
    const long long oj = dual_off(j, a.Np, a.nxu, nx);
    for (int e = threadIdx.x; e < NR * nx; e += blockDim.x) {
        const int k = e / nx, r = e - k * nx;
        const T val = xj[k * ldk + r];
        a.xs[k * a.s_stride + (long long)j * nx + r] = val;
        a.h[k][oj + r] = scj * val;
    }
    if (j < a.Np) {
        const int nvec = ldk / VN;
        const VT *Kj = reinterpret_cast<const VT *>(a.K + (size_t)j * nu * ldk);
        for (int r = warp; r < nu; r += kWarps) {
            const VT *row = Kj + (size_t)r * nvec;
            T sum[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) sum[k] = T(0);
            for (int cv = lane; cv < nvec; cv += 32) {
                const VT g = __ldg(row + cv);
#pragma unroll
                for (int k = 0; k < NR; ++k) sum[k] += v_dot<T>(g, xj + k * ldk + cv * VN);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const T tot = warp_sum(sum[k]);
                if (lane == 0) {
                    const T uval = tot + a.ubar[k * a.u_stride + (long long)j * nu + r];
                    a.us[k * a.u_stride + (long long)j * nu + r] = uval;
                    a.h[k][oj + nx + r] = scj * uval;
                }
            }
        }
    }
}

template <class T, int NR, int KV>
void launch_bwd(const SolveArgs<T> &a, int first, int count, cudaStream_t st) {
    const size_t smem = sizeof(T) * ((size_t)NR * a.nx + (size_t)kWarps * NR * a.ldg + (size_t)NR * a.ldg + (size_t)NR * a.nu);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_bwd<T, NR, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bwd<T, NR, KV><<<count, 256, smem, st>>>(a, first);
}

template <class T, int NR>
void launch_bwd_kv(const SolveArgs<T> &a, int first, int count, cudaStream_t st) {
    const int nvec = a.ldg / V16<T>::n;
    const int kv = (nvec + 31) / 32;
    switch (kv) {
        case 1: launch_bwd<T, NR, 1>(a, first, count, st); break;
        case 2: launch_bwd<T, NR, 2>(a, first, count, st); break;
        case 3: launch_bwd<T, NR, 3>(a, first, count, st); break;
        default: launch_bwd<T, NR, 4>(a, first, count, st); break;
    }
}

template <class T, int NR>
void launch_fwd(const SolveArgs<T> &a, int first, int count, cudaStream_t st) {
    const size_t smem = sizeof(T) * ((size_t)NR * a.ldg + (size_t)NR * a.ldk);
    k_fwd<T, NR><<<count, 256, smem, st>>>(a, first);
}

template <class T, int NR>
void run_round(stotree_t h, const SolveArgs<T> &a, cudaStream_t st) {
    for (int t = h->N - 1; t >= 0; --t) {
        const int first = h->soff[t], count = h->soff[t + 1] - first;
        launch_bwd_kv<T, NR>(a, first, count, st);
    }
    for (int t = 0; t <= h->N; ++t) {
        const int first = h->soff[t], count = h->soff[t + 1] - first;
        launch_fwd<T, NR>(a, first, count, st);
    }
    h->launches += 2 * h->N + 1;
}

template <class T>
sto_status solve_impl(stotree_t h, const void *const *y, const void *x0, void *const *hx, int nrhs, bool homog,
                      bool scaled, cudaStream_t st, const SolveScratch *scratch) {
    const Layout &L = h->L;
    SolveArgs<T> a;
    a.nx = h->nx;
    a.nu = h->nu;
    a.ldg = h->ldg;
    a.ldk = h->ldk;
    a.ldr = h->ldr;
    a.Np = h->Np;
    a.nxu = h->nx + h->nu;
    a.G = h->at<T>(L.G);
    a.K = h->at<T>(L.K);
    a.Ri = h->at<T>(L.Ri);
    a.gu = h->at<T>(L.gu);
    a.gx = h->at<T>(L.gx);
    a.c = h->at<T>(L.c);
    a.sqp = h->at<T>(L.sqp);
    a.pN = h->at<T>(L.cost) + (2 * h->nx + h->nu) + h->nx + h->nu;  // ell = [q | r | pN]
    a.prob = h->at<double>(L.prob64);
    a.cbeg = h->at<int>(L.cbeg);
    a.ccnt = h->at<int>(L.ccnt);
    a.parent = h->at<int>(L.parent);
    for (int k = 0; k < kMaxRhs; ++k) {
        a.y[k] = static_cast<const T *>(y[k < nrhs ? k : 0]);
        a.h[k] = static_cast<T *>(hx[k < nrhs ? k : 0]);
    }
    a.x0 = static_cast<const T *>(x0);
    if (scratch) {  // caller-supplied scratch for one right-hand side
        a.s = static_cast<T *>(scratch->s);
        a.ubar = static_cast<T *>(scratch->ubar);
        a.xs = static_cast<T *>(scratch->xs);
        a.us = static_cast<T *>(scratch->us);
    } else {
        a.s = h->at<T>(L.s);
        a.ubar = h->at<T>(L.ubar);
        a.xs = h->at<T>(L.xs);
        a.us = h->at<T>(L.us);
    }
    a.s_stride = (long long)h->Nn * h->nx;
    a.u_stride = (long long)h->Np * h->nu;
    a.homog = homog ? 1 : 0;
    a.scaled = scaled ? 1 : 0;
    cudaEvent_t ev;
    timing_begin(h, st, &ev);
    switch (nrhs) {
        case 1: run_round<T, 1>(h, a, st); break;
        case 2: run_round<T, 2>(h, a, st); break;
        case 3: run_round<T, 3>(h, a, st); break;
        default: run_round<T, 4>(h, a, st); break;
    }
    timing_end(h, st, ev, nrhs);
    h->solve_calls += nrhs;
    STO_CUDA(h, cudaGetLastError());
    return STO_OK;
}

}  // namespace

sto_status solve_round(stotree_t h, const void *const *y, const void *x0, void *const *hx, int nrhs, bool homog,
                       bool scaled, cudaStream_t st, const SolveScratch *scratch) {
    if (scratch && nrhs != 1) return STO_ERR_INVALID_ARG;
    return h->prec == STO_FP64 ? solve_impl<double>(h, y, x0, hx, nrhs, homog, scaled, st, scratch)
                               : solve_impl<float>(h, y, x0, hx, nrhs, homog, scaled, st, scratch);
}

}  // namespace sto
