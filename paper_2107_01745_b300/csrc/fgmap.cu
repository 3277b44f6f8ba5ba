// General constraint maps (Section II-C): z^i = F x^i + G u^i at every nonleaf node (the root
// included, x^0 = p) and z^l = FN x^l at every leaf, F, G, FN shared by all nodes.  Algorithm 3
// minimises f(x) + <y, Hx>, so with these maps it runs unchanged on H'y laid out like [x; u]
// (per nonleaf node [F'y^i; G'y^i], per leaf FN'y^l), and Hx follows from its [x; u] output.
// These two maps run around the solve round; both are per node, so they commute with the
// per-node scaling sqrt(pi) of the preconditioned dual (Section III-E).
#include "internal.h"

namespace sto {
namespace {

constexpr int kMapThreads = 256;

// out (the [x; u] layout, msel entries, type TO) = H'y (y: the z layout, m entries, type TI), with
// the maps in type TM, accumulated in TO.
template <class TI, class TM, class TO>
__global__ void k_fg_ht(int Np, int Nn, int nx, int nu, int nc, int ncN, const TM *FG, const TI *y, TO *out) {
    const int nxu = nx + nu;
    const TM *F = FG, *G = FG + (size_t)nc * nx, *FN = G + (size_t)nc * nu;
    const long long msel = (long long)Np * nxu + (long long)(Nn - Np) * nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < msel;
         e += (long long)gridDim.x * blockDim.x) {
        TO acc = TO(0);
        if (e < (long long)Np * nxu) {
            const int i = (int)(e / nxu), k = (int)(e - (long long)i * nxu);
            const TI *yi = y + (long long)i * nc;
            if (k < nx) {
                for (int c = 0; c < nc; ++c) acc += (TO)F[(size_t)c * nx + k] * (TO)yi[c];
            } else {
                for (int c = 0; c < nc; ++c) acc += (TO)G[(size_t)c * nu + k - nx] * (TO)yi[c];
            }
        } else {
            const long long e2 = e - (long long)Np * nxu;
            const int l = (int)(e2 / nx), k = (int)(e2 - (long long)l * nx);
            const TI *yl = y + (long long)Np * nc + (long long)l * ncN;
            for (int c = 0; c < ncN; ++c) acc += (TO)FN[(size_t)c * nx + k] * (TO)yl[c];
        }
        out[e] = acc;
    }
}

// out (the z layout, m entries) = H p, p in the [x; u] layout.
template <class T>
__global__ void k_fg_hx(int Np, int Nn, int nx, int nu, int nc, int ncN, const T *FG, const T *p, T *out) {
    const int nxu = nx + nu;
    const T *F = FG, *G = FG + (size_t)nc * nx, *FN = G + (size_t)nc * nu;
    const long long m = (long long)Np * nc + (long long)(Nn - Np) * ncN;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        T acc = T(0);
        if (e < (long long)Np * nc) {
            const int i = (int)(e / nc), c = (int)(e - (long long)i * nc);
            const T *pi = p + (long long)i * nxu;
            for (int k = 0; k < nx; ++k) acc += F[(size_t)c * nx + k] * pi[k];
            for (int a = 0; a < nu; ++a) acc += G[(size_t)c * nu + a] * pi[nx + a];
        } else {
            const long long e2 = e - (long long)Np * nc;
            const int l = (int)(e2 / ncN), c = (int)(e2 - (long long)l * ncN);
            const T *pl = p + (long long)Np * nxu + (long long)l * nx;
            for (int k = 0; k < nx; ++k) acc += FN[(size_t)c * nx + k] * pl[k];
        }
        out[e] = acc;
    }
}

int map_grid(long long n) {
    const long long b = (n + kMapThreads - 1) / kMapThreads;
    return (int)(b < 4 * 148 ? (b < 1 ? 1 : b) : 4 * 148);
}

}  // namespace

// H'y of the handle's precision (round input) or in FP64 (the optimality check).
sto_status fg_ht(stotree_t h, const void *y, void *out, bool fp64_out, cudaStream_t st) {
    const int g = map_grid(h->msel);
    if (h->prec == STO_FP64) {
        k_fg_ht<double, double, double><<<g, kMapThreads, 0, st>>>(h->Np, h->Nn, h->nx, h->nu, h->nc, h->ncN,
                                                                   h->at<double>(h->L.FG), static_cast<const double *>(y),
                                                                   static_cast<double *>(out));
    } else if (fp64_out) {
        k_fg_ht<float, double, double><<<g, kMapThreads, 0, st>>>(h->Np, h->Nn, h->nx, h->nu, h->nc, h->ncN,
                                                                  h->at<double>(h->L.FG64), static_cast<const float *>(y),
                                                                  static_cast<double *>(out));
    } else {
        k_fg_ht<float, float, float><<<g, kMapThreads, 0, st>>>(h->Np, h->Nn, h->nx, h->nu, h->nc, h->ncN,
                                                                h->at<float>(h->L.FG), static_cast<const float *>(y),
                                                                static_cast<float *>(out));
    }
    h->launches += 1;
    STO_CUDA(h, cudaGetLastError());
    return STO_OK;
}

sto_status fg_hx(stotree_t h, const void *p, void *out, cudaStream_t st) {
    const int g = map_grid(h->m);
    if (h->prec == STO_FP64)
        k_fg_hx<double><<<g, kMapThreads, 0, st>>>(h->Np, h->Nn, h->nx, h->nu, h->nc, h->ncN, h->at<double>(h->L.FG),
                                                   static_cast<const double *>(p), static_cast<double *>(out));
    else
        k_fg_hx<float><<<g, kMapThreads, 0, st>>>(h->Np, h->Nn, h->nx, h->nu, h->nc, h->ncN, h->at<float>(h->L.FG),
                                                  static_cast<const float *>(p), static_cast<float *>(out));
    h->launches += 1;
    STO_CUDA(h, cudaGetLastError());
    return STO_OK;
}

}  // namespace sto
