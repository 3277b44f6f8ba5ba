// C ABI of libstotree: handle, workspace layout and data upload.
// Problem statement: Section II of the paper (scenario tree, dynamics, costs, box).
#include <cmath>
#include <cstdio>
#include <cstring>

#include <map>
#include <tuple>
#include <mutex>

#include "internal.h"

using namespace sto;

namespace sto {

sto_status cuda_fail(stotree_t h, cudaError_t e, const char *what) {
    if (h) {
        h->err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return STO_ERR_CUDA;
}

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Work items of a solve round: maximal paths of at most kSegMax nodes along which every node
// has one child, so that a CTA keeps the recursion's vector in shared memory along the path.
// Backward: over nonleaf nodes, lowest node first; a node joins its only child's segment when
// that child is nonleaf and the segment is not full.  Segments are ordered by lowest node
// descending, so every segment's children segments come earlier (tickets are handed out in
// this order and a segment only waits on earlier ones).  Forward: over all nodes, top node
// first; a node joins its parent's segment when it is the parent's only child.  Ordered by top
// node ascending, so the parent's segment always comes earlier.
static void build_segments(stotree_t h) {
    const int Nn = h->Nn, Np = h->Np;
    std::vector<std::vector<int>> segs;
    std::vector<int> seg_of(Nn, -1);
    for (int i = Np - 1; i >= 0; --i) {
        if (h->ccnt[i] == 1 && h->cbeg[i] < Np) {
            const int c = h->cbeg[i], sc = seg_of[c];
            if ((int)segs[sc].size() < kSegMax && segs[sc].back() == c) {
                segs[sc].push_back(i);
                seg_of[i] = sc;
                continue;
            }
        }
        seg_of[i] = (int)segs.size();
        segs.push_back({i});
    }
    h->bstart.assign(1, 0);
    h->bnodes.clear();
    for (auto &s : segs) {
        for (int v : s) h->bnodes.push_back(v);
        h->bstart.push_back((int)h->bnodes.size());
    }
    segs.clear();
    std::fill(seg_of.begin(), seg_of.end(), -1);
    for (int j = 0; j < Nn; ++j) {
        const int p = h->parent[j];
        if (p >= 0 && h->ccnt[p] == 1) {
            const int sp = seg_of[p];
            if ((int)segs[sp].size() < kSegMax && segs[sp].back() == p) {
                segs[sp].push_back(j);
                seg_of[j] = sp;
                continue;
            }
        }
        seg_of[j] = (int)segs.size();
        segs.push_back({j});
    }
    h->fstart.assign(1, 0);
    h->fnodes.clear();
    for (auto &s : segs) {
        for (int v : s) h->fnodes.push_back(v);
        h->fstart.push_back((int)h->fnodes.size());
    }
}

static void compute_layout(stotree_t h) {
    Layout &L = h->L;
    size_t total = 0;
    auto add = [&](size_t bytes) {
        size_t off = round_up(total, 256);
        total = off + round_up(bytes, 16);
        return off;
    };
    const size_t Nn = h->Nn, Np = h->Np, nx = h->nx, nu = h->nu, Wd = h->max_width;
    const size_t es = h->esz;
    const size_t mpad = round_up((size_t)h->m, 64);
    L.parent = add(Nn * 4);
    L.cbeg = add(Nn * 4);
    L.ccnt = add(Nn * 4);
    L.soff = add((h->N + 2) * 4);
    L.node_stage = add(Nn * 4);
    L.prob64 = add(Nn * 8);
    L.sqp = add(Nn * es);
    L.G64 = add(Nn * nx * h->ld64 * 8);
    L.cost64 = add((4 * nx + 2 * nu) * 8);
    L.box64 = add(5 * (nx + nu) * 8);
    L.P[0] = add(Wd * nx * nx * 8);
    L.P[1] = add(Wd * nx * nx * 8);
    L.PG = add(Wd * nx * h->ld64 * 8);
    L.W = add(Wd * h->ld64 * h->ld64 * 8);
    L.Rb = add(Wd * nu * nu * 8);
    L.Zb = add(Wd * nu * nu * 8);
    L.M = add(Wd * nu * nx * 8);
    L.K64 = add(Wd * nu * nx * 8);
    L.fstatus = add(64);
    L.G = add(Nn * nx * h->ldg * es);
    L.RK = add(Np * nu * h->ldrk * es);
    L.Gt = add(Nn * (nx + nu) * h->ldk * es);
    L.Kt = add(Np * nx * h->ldr * es);
    L.gu = add(Np * nu * es);
    L.gx = add(Np * nx * es);
    L.c = add(Nn * nx * es);
    L.cost = add(2 * (2 * nx + nu) * es);
    L.box = add(5 * (nx + nu) * es);
    L.ubar = add(kMaxRhs * Np * nu * es);
    L.xs = add(kMaxRhs * Nn * nx * es);
    L.us = add(kMaxRhs * Np * nu * es);
    L.ts = add(kMaxRhs * Nn * nx * 2 * es);  // one 8-byte word per 4 bytes of a value
    L.txs = add(kMaxRhs * Nn * nx * 2 * es);
    L.tus = add(kMaxRhs * Np * nu * 2 * es);
    L.tus_end = L.tus + kMaxRhs * Np * nu * 2 * es;
    L.vec = add(kNumVec * mpad * es);
    L.ringS = add((kMaxMem + 1) * mpad * es);
    L.ringY = add((kMaxMem + 1) * mpad * es);
    L.partials = add((size_t)kRedBlocks * kRedSlots * 8);
    L.scal = add(sizeof(SolverScalars));
    L.kkt = add((Nn * nx + Np * nu) * 8 + 64 * 8 + (h->fg ? (size_t)h->msel * 8 : 0));
    L.bstart = add(h->bstart.size() * 4);
    L.bnodes = add(h->bnodes.size() * 4);
    L.fstart = add(h->fstart.size() * 4);
    L.fnodes = add(h->fnodes.size() * 4);
    L.flags = add(2 * Nn * 4);
    L.ticket = add(64);
    if (h->fg) {
        const size_t nfg = (size_t)h->nc * (nx + nu) + (size_t)h->ncN * nx;
        const size_t nzb = 5 * (size_t)(h->nc + h->ncN);
        const size_t spad = round_up((size_t)h->msel, 64);
        L.FG = add(nfg * es);
        L.FG64 = add(nfg * 8);
        L.zbox = add(nzb * es);
        L.zbox64 = add(nzb * 8);
        L.ht = add(kMaxRhs * spad * es);
        L.pv = add(kMaxRhs * spad * es);
        L.pvec = add(4 * spad * es);
        L.zcost = add(4 * (size_t)(h->nc + h->ncN + nx + nu) * es);
    }
    L.total = round_up(total, 256);
}

void timing_begin(stotree_t h, cudaStream_t st, cudaEvent_t *ev) {
    *ev = nullptr;
    if (!h->timing) return;
    if (h->ev_used + 2 > h->ev_pool.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            h->ev_pool.push_back(e);
        }
    }
    *ev = h->ev_pool[h->ev_used];
    h->ev_used += 2;
    cudaEventRecord(*ev, st);
}

void timing_end(stotree_t h, cudaStream_t st, cudaEvent_t ev0, int nrhs) {
    if (!ev0) return;
    // the end event sits right after the start event in the pool
    size_t idx = 0;
    for (; idx < h->ev_pool.size(); ++idx)
        if (h->ev_pool[idx] == ev0) break;
    cudaEventRecord(h->ev_pool[idx + 1], st);
    h->solve_launches += 1;
    h->solve_rhs += nrhs;
}

}  // namespace sto

extern "C" {

const char *stotree_status_str(sto_status s) {
    switch (s) {
        case STO_OK: return "ok";
        case STO_ERR_INVALID_ARG: return "invalid argument";
        case STO_ERR_TREE: return "invalid scenario tree";
        case STO_ERR_NOT_READY: return "workspace, data or factor missing";
        case STO_ERR_NUMERICAL: return "numerical failure";
        case STO_ERR_CUDA: return "CUDA error";
        case STO_ERR_TIMEOUT: return "bounded device wait expired";
        case STO_NOT_CONVERGED: return "iteration limit reached";
        case STO_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

const char *stotree_last_error(stotree_t h) { return h ? h->err.c_str() : ""; }

}  // extern "C"

namespace sto {

cudaError_t raise_smem_cap(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> caps;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cap = caps[{dev, func}];
    if (bytes <= cap) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
}

int wave_grid(const void *func, int threads, size_t smem, int want) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return want;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dev, func, threads, smem);
    auto it = cache.find(key);
    int full = 0;
    if (it != cache.end()) {
        full = it->second;
    } else {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return want;
        }
        full = per_sm * sms;
        cache[key] = full;
    }
    return full > 0 && full < want ? full : want;
}

// Tree conventions (Section II-A with the numbering of the boundary): root 0 with probability 1,
// parent[i] < i, stage-major order with the children of a node contiguous, positive
// probabilities that sum over the children to the parent's, leaves exactly at the last stage.
sto_status validate_tree(const int32_t *parent, const double *prob, int Nn, int horizon, std::vector<int32_t> &stage,
                         std::vector<int32_t> &ccnt, std::vector<int32_t> &cbeg) {
    stage.assign(Nn, 0);
    ccnt.assign(Nn, 0);
    cbeg.assign(Nn, 0);
    if (parent[0] != -1 || std::fabs(prob[0] - 1.0) > 1e-9) return STO_ERR_TREE;
    for (int i = 1; i < Nn; ++i) {
        int p = parent[i];
        if (p < 0 || p >= i) return STO_ERR_TREE;
        if (i >= 2 && p < parent[i - 1]) return STO_ERR_TREE;  // children contiguous, BFS order
        stage[i] = stage[p] + 1;
        if (stage[i] < stage[i - 1]) return STO_ERR_TREE;
        if (ccnt[p] == 0) cbeg[p] = i;
        ccnt[p] += 1;
        if (!(prob[i] > 0.0)) return STO_ERR_TREE;
    }
    for (int i = 0; i < Nn; ++i) {
        const bool leaf = ccnt[i] == 0;
        if (leaf != (stage[i] == horizon)) return STO_ERR_TREE;
        if (!leaf) {
            double s = 0.0;
            for (int j = cbeg[i]; j < cbeg[i] + ccnt[i]; ++j) s += prob[j];
            if (std::fabs(s - prob[i]) > 1e-9 * std::fmax(1.0, prob[i])) return STO_ERR_TREE;
        }
    }
    return STO_OK;
}

}  // namespace sto

extern "C" {

sto_status stotree_create(const sto_tree_desc *t, int32_t precision, stotree_t *out) {
    if (!t || !out || !t->parent || !t->prob) return STO_ERR_INVALID_ARG;
    if (t->nx < 1 || t->nu < 1 || t->nx > kMaxDim || t->nu > kMaxDim || t->num_nodes < 2 ||
        t->horizon < 1)
        return STO_ERR_INVALID_ARG;
    if (precision != STO_FP64 && precision != STO_FP32) return STO_ERR_INVALID_ARG;
    const int Nn = t->num_nodes;
    std::vector<int32_t> stage, ccnt, cbeg;
    if (validate_tree(t->parent, t->prob, Nn, t->horizon, stage, ccnt, cbeg) != STO_OK) return STO_ERR_TREE;
    stotree_t h = new stotree_s();
    h->Nn = Nn;
    h->N = t->horizon;
    h->nx = t->nx;
    h->nu = t->nu;
    h->prec = precision;
    h->esz = precision == STO_FP64 ? 8 : 4;
    h->parent.assign(t->parent, t->parent + Nn);
    h->prob.assign(t->prob, t->prob + Nn);
    h->stage = stage;
    h->cbeg = cbeg;
    h->ccnt = ccnt;
    h->soff.assign(h->N + 2, 0);
    for (int s = 0; s <= h->N + 1; ++s) {
        int k = 0;
        while (k < Nn && stage[k] < s) ++k;
        h->soff[s] = k;
    }
    h->soff[h->N + 1] = Nn;
    h->max_width = 0;
    for (int s = 0; s <= h->N; ++s) h->max_width = std::max(h->max_width, h->soff[s + 1] - h->soff[s]);
    h->Nl = h->soff[h->N + 1] - h->soff[h->N];
    h->Np = Nn - h->Nl;
    for (int i = 0; i < h->Np; ++i)
        if (ccnt[i] == 0) {
            delete h;
            return STO_ERR_TREE;
        }
    h->m = (int64_t)h->Np * (h->nx + h->nu) + (int64_t)h->Nl * h->nx;
    h->n = (int64_t)h->Np * h->nu + (int64_t)(Nn - 1) * h->nx;
    if (h->m >= (int64_t)1 << 31) {
        delete h;
        return STO_ERR_INVALID_ARG;
    }
    const int vec = 16 / (int)h->esz;
    h->ld64 = (int)round_up(h->nx + h->nu + 1, 2);
    h->ldg = (int)round_up(h->nx + h->nu, vec);
    h->ldk = (int)round_up(h->nx, vec);
    h->ldr = (int)round_up(h->nu, vec);
    h->ldrk = h->ldr + h->ldk;
    // register tiling of the solve kernel: padded row widths of [A | B] and [-Rbar^-1 | K]
    if (std::max(h->ldg, h->ldrk) > (precision == STO_FP64 ? 256 : 512)) {
        delete h;
        return STO_ERR_INVALID_ARG;
    }
    h->have_dyn.assign(Nn, 0);
    h->have_dyn[0] = 1;
    build_segments(h);
    compute_layout(h);
    if (cudaMallocHost(&h->host_scal, sizeof(SolverScalars)) != cudaSuccess) {
        h->host_scal = new SolverScalars();
    }
    if (cudaMallocHost(&h->host_scal2, sizeof(SolverScalars)) != cudaSuccess) {
        h->host_scal2 = new SolverScalars();
    }
    *out = h;
    return STO_OK;
}

void stotree_destroy(stotree_t h) {
    if (!h) return;
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->host_scal) {
        if (cudaFreeHost(h->host_scal) != cudaSuccess) delete h->host_scal;
    }
    if (h->host_scal2) {
        if (cudaFreeHost(h->host_scal2) != cudaSuccess) delete h->host_scal2;
    }
    delete h;
}

sto_status stotree_set_constraint_maps(stotree_t h, int32_t nc, int32_t ncN, const double *F, const double *G,
                                       const double *FN) {
    if (!h || nc < 1 || ncN < 1 || nc > kMaxDim || ncN > kMaxDim || !F || !G || !FN) return STO_ERR_INVALID_ARG;
    if (h->ws) return STO_ERR_INVALID_ARG;  // the dual length is part of the workspace layout
    const int64_t m = (int64_t)h->Np * nc + (int64_t)h->Nl * ncN;
    if (m >= (int64_t)1 << 31) return STO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < (int64_t)nc * h->nx; ++k)
        if (!std::isfinite(F[k])) return STO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < (int64_t)nc * h->nu; ++k)
        if (!std::isfinite(G[k])) return STO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < (int64_t)ncN * h->nx; ++k)
        if (!std::isfinite(FN[k])) return STO_ERR_INVALID_ARG;
    h->fg = true;
    h->nc = nc;
    h->ncN = ncN;
    h->Fm.assign(F, F + (size_t)nc * h->nx);
    h->Gm.assign(G, G + (size_t)nc * h->nu);
    h->FNm.assign(FN, FN + (size_t)ncN * h->nx);
    h->msel = (int64_t)h->Np * (h->nx + h->nu) + (int64_t)h->Nl * h->nx;  // the [x; u] layout of the round
    h->m = m;
    h->have_zbox = false;
    compute_layout(h);
    return STO_OK;
}

sto_status stotree_set_zbox(stotree_t h, const double *zlo, const double *zhi, const double *zNlo, const double *zNhi,
                            sto_stream_t stream) {
    if (!h || !zlo || !zhi || !zNlo || !zNhi) return STO_ERR_INVALID_ARG;
    if (!h->fg) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    const int n = h->nc + h->ncN;
    std::vector<double> b(5 * (size_t)n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double lo = k < h->nc ? zlo[k] : zNlo[k - h->nc], hi = k < h->nc ? zhi[k] : zNhi[k - h->nc];
        if (!(lo <= hi)) return STO_ERR_INVALID_ARG;
        b[k] = lo;
        b[n + k] = hi;
        b[3 * n + k] = 1.0;  // delta (unused: hard box)
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.zbox64, b.data(), b.size() * 8, cudaMemcpyHostToDevice, st));
    if (h->prec == STO_FP64) {
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.zbox, b.data(), b.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> bf(b.begin(), b.end());
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.zbox, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
    }
    STO_CUDA(h, cudaStreamSynchronize(st));
    h->zboxv = b;
    h->have_zbox = true;
    return STO_OK;
}

sto_status stotree_sizes(stotree_t h, int64_t *m, int64_t *n, int32_t *np, int32_t *nl) {
    if (!h) return STO_ERR_INVALID_ARG;
    if (m) *m = h->m;
    if (n) *n = h->n;
    if (np) *np = h->Np;
    if (nl) *nl = h->Nl;
    return STO_OK;
}

sto_status stotree_workspace_size(stotree_t h, size_t *bytes) {
    if (!h || !bytes) return STO_ERR_INVALID_ARG;
    *bytes = h->L.total;
    return STO_OK;
}

sto_status stotree_bind_workspace(stotree_t h, void *dev, size_t bytes, sto_stream_t stream) {
    if (!h || !dev) return STO_ERR_INVALID_ARG;
    if (bytes < h->L.total) return STO_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(dev) % 256 != 0) return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    h->ws = static_cast<char *>(dev);
    h->ws_bytes = bytes;
    const Layout &L = h->L;
    STO_CUDA(h, cudaMemsetAsync(h->ws, 0, L.total, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.parent, h->parent.data(), h->Nn * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.cbeg, h->cbeg.data(), h->Nn * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.ccnt, h->ccnt.data(), h->Nn * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.soff, h->soff.data(), (h->N + 2) * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.node_stage, h->stage.data(), h->Nn * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.prob64, h->prob.data(), h->Nn * 8, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.bstart, h->bstart.data(), h->bstart.size() * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.bnodes, h->bnodes.data(), h->bnodes.size() * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.fstart, h->fstart.data(), h->fstart.size() * 4, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(h->ws + L.fnodes, h->fnodes.data(), h->fnodes.size() * 4, cudaMemcpyHostToDevice, st));
    h->epoch = 0;          // flags and ticket counter start at zero (memset above)
    h->ticket_base = 0;
    if (h->prec == STO_FP64) {
        std::vector<double> sq(h->Nn);
        for (int i = 0; i < h->Nn; ++i) sq[i] = std::sqrt(h->prob[i]);
        STO_CUDA(h, cudaMemcpyAsync(h->ws + L.sqp, sq.data(), h->Nn * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> sq(h->Nn);
        for (int i = 0; i < h->Nn; ++i) sq[i] = (float)std::sqrt(h->prob[i]);
        STO_CUDA(h, cudaMemcpyAsync(h->ws + L.sqp, sq.data(), h->Nn * 4, cudaMemcpyHostToDevice, st));
    }
    if (h->fg) {
        std::vector<double> fg64(h->Fm);
        fg64.insert(fg64.end(), h->Gm.begin(), h->Gm.end());
        fg64.insert(fg64.end(), h->FNm.begin(), h->FNm.end());
        STO_CUDA(h, cudaMemcpyAsync(h->ws + L.FG64, fg64.data(), fg64.size() * 8, cudaMemcpyHostToDevice, st));
        if (h->prec == STO_FP64) {
            STO_CUDA(h, cudaMemcpyAsync(h->ws + L.FG, fg64.data(), fg64.size() * 8, cudaMemcpyHostToDevice, st));
        } else {
            std::vector<float> f32(fg64.begin(), fg64.end());
            STO_CUDA(h, cudaMemcpyAsync(h->ws + L.FG, f32.data(), f32.size() * 4, cudaMemcpyHostToDevice, st));
        }
        h->have_zbox = false;
    }
    STO_CUDA(h, cudaStreamSynchronize(st));
    std::fill(h->have_dyn.begin() + 1, h->have_dyn.end(), 0);
    h->have_cost = h->have_box = h->factored = false;
    return STO_OK;
}

sto_status stotree_set_dynamics(stotree_t h, int32_t first, int32_t count, const double *A,
                                const double *B, const double *c, sto_stream_t stream) {
    if (!h || !c || (A == nullptr) != (B == nullptr) || first < 0 || count < 1 || first + count > h->Nn)
        return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    if (!A)  // the disturbances only: the nodes keep their matrices
        for (int i = first; i < first + count; ++i)
            if (!h->have_dyn[i]) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t nx = h->nx, nu = h->nu, ld = h->ld64;
    double *dst = h->at<double>(h->L.G64) + (size_t)first * nx * ld;
    if (A) {
        STO_CUDA(h, cudaMemcpy2DAsync(dst, ld * 8, A, nx * 8, nx * 8, (size_t)count * nx, cudaMemcpyHostToDevice, st));
        STO_CUDA(h, cudaMemcpy2DAsync(dst + nx, ld * 8, B, nu * 8, nu * 8, (size_t)count * nx, cudaMemcpyHostToDevice,
                                      st));
    }
    STO_CUDA(h, cudaMemcpy2DAsync(dst + nx + nu, ld * 8, c, 8, 8, (size_t)count * nx, cudaMemcpyHostToDevice, st));
    STO_CUDA(h, cudaStreamSynchronize(st));  // host arrays may be released on return
    for (int i = first; i < first + count; ++i) h->have_dyn[i] = 1;
    h->factored = false;
    return STO_OK;
}

sto_status stotree_set_costs(stotree_t h, const double *Q, const double *R, const double *PN,
                             const double *q, const double *r, const double *pN, sto_stream_t stream) {
    if (!h || !Q || !R || !PN) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    const int nx = h->nx, nu = h->nu;
    for (int k = 0; k < nu; ++k)
        if (!(R[k] > 0.0)) return STO_ERR_INVALID_ARG;
    for (int k = 0; k < nx; ++k)
        if (!(Q[k] >= 0.0) || !(PN[k] >= 0.0)) return STO_ERR_INVALID_ARG;
    // cost64 = [Q nx][R nu][PN nx][q nx][r nu][pN nx]
    std::vector<double> c64(4 * nx + 2 * nu, 0.0);
    std::memcpy(&c64[0], Q, nx * 8);
    std::memcpy(&c64[nx], R, nu * 8);
    std::memcpy(&c64[nx + nu], PN, nx * 8);
    if (q) std::memcpy(&c64[2 * nx + nu], q, nx * 8);
    if (r) std::memcpy(&c64[3 * nx + nu], r, nu * 8);
    if (pN) std::memcpy(&c64[3 * nx + 2 * nu], pN, nx * 8);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.cost64, c64.data(), c64.size() * 8, cudaMemcpyHostToDevice, st));
    // real copy: [W: Q | R | PN][ell: q | r | pN]
    if (h->prec == STO_FP64) {
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.cost, c64.data(), c64.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> cf(c64.begin(), c64.end());
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.cost, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice, st));
    }
    STO_CUDA(h, cudaStreamSynchronize(st));
    h->have_cost = true;
    h->factored = false;
    return STO_OK;
}

// Upload [lo | hi | rho | delta | kind] (each nx + nu, x part then u part) in FP64 and in the
// handle's precision.
static sto_status upload_g(stotree_t h, cudaStream_t st) {
    const int n = h->nx + h->nu;
    if (h->pen.size() != (size_t)3 * n) {  // default: every component a hard box
        h->pen.assign((size_t)3 * n, 0.0);
        for (int k = 0; k < n; ++k) h->pen[n + k] = 1.0;
    }
    std::vector<double> b(5 * (size_t)n);
    std::copy(h->boxv.begin(), h->boxv.end(), b.begin());
    std::copy(h->pen.begin(), h->pen.end(), b.begin() + 2 * n);
    STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.box64, b.data(), b.size() * 8, cudaMemcpyHostToDevice, st));
    if (h->prec == STO_FP64) {
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.box, b.data(), b.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> bf(b.begin(), b.end());
        STO_CUDA(h, cudaMemcpyAsync(h->ws + h->L.box, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
    }
    STO_CUDA(h, cudaStreamSynchronize(st));
    return STO_OK;
}

sto_status stotree_set_box(stotree_t h, const double *xlo, const double *xhi, const double *ulo,
                           const double *uhi, sto_stream_t stream) {
    if (!h || !xlo || !xhi || !ulo || !uhi) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    const int nx = h->nx, nu = h->nu;
    // [lo: x | u][hi: x | u]
    std::vector<double> b(2 * (nx + nu));
    for (int k = 0; k < nx; ++k) {
        if (!(xlo[k] <= xhi[k])) return STO_ERR_INVALID_ARG;
        b[k] = xlo[k];
        b[nx + nu + k] = xhi[k];
    }
    for (int k = 0; k < nu; ++k) {
        if (!(ulo[k] <= uhi[k])) return STO_ERR_INVALID_ARG;
        b[nx + k] = ulo[k];
        b[2 * nx + nu + k] = uhi[k];
    }
    h->boxv = b;
    const sto_status s = upload_g(h, reinterpret_cast<cudaStream_t>(stream));
    if (s != STO_OK) return s;
    h->have_box = true;
    return STO_OK;
}

sto_status stotree_set_penalty(stotree_t h, const int32_t *kind, const double *rho, const double *delta,
                               sto_stream_t stream) {
    if (!h) return STO_ERR_INVALID_ARG;
    if (h->fg && kind) return STO_ERR_INVALID_ARG;  // soft terms are per component of [x; u]
    const int n = h->nx + h->nu;
    std::vector<double> pen(3 * (size_t)n, 0.0);
    for (int k = 0; k < n; ++k) {
        const int kd = kind ? kind[k] : 0;
        const double r = rho ? rho[k] : 0.0, d = delta ? delta[k] : 1.0;
        if (kd < 0 || kd > 2) return STO_ERR_INVALID_ARG;
        if (kd >= 1 && !(r > 0.0 && r < INFINITY)) return STO_ERR_INVALID_ARG;
        if (kd == 2 && !(d > 0.0 && d < INFINITY)) return STO_ERR_INVALID_ARG;
        pen[k] = kd >= 1 ? r : 0.0;
        pen[n + k] = kd == 2 ? d : 1.0;
        pen[2 * n + k] = kd;
    }
    h->pen = pen;
    h->general = false;
    for (int k = 0; k < n; ++k) h->general = h->general || pen[2 * n + k] != 0.0;
    if (!h->have_box) return STO_OK;  // uploaded with the box
    if (!h->ws) return STO_ERR_NOT_READY;
    return upload_g(h, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_factor(stotree_t h, int32_t sync, sto_stream_t stream) {
    if (!h) return STO_ERR_INVALID_ARG;
    if (!h->ws || !h->have_cost) return STO_ERR_NOT_READY;
    for (int i = 1; i < h->Nn; ++i)
        if (!h->have_dyn[i]) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    sto_status s = factor_run(h, st);
    if (s != STO_OK) return s;
    s = prepare_round(h);
    if (s != STO_OK) return s;
    h->factored = true;
    if (sync) {
        int flag = 0;
        STO_CUDA(h, cudaMemcpyAsync(&flag, h->ws + h->L.fstatus, 4, cudaMemcpyDeviceToHost, st));
        STO_CUDA(h, cudaStreamSynchronize(st));
        if (flag != 0) {
            h->factored = false;
            h->err = "Rbar not positive definite at node " + std::to_string(flag - 1);
            return STO_ERR_NUMERICAL;
        }
    }
    return STO_OK;
}

sto_status stotree_solve_step(stotree_t h, const void *y, const void *x0, void *hx, int32_t nrhs,
                              int32_t homogeneous, int32_t scaled, sto_stream_t stream) {
    if (!h || !y || !hx || nrhs < 1 || nrhs > kMaxRhs) return STO_ERR_INVALID_ARG;
    if (!homogeneous && !x0) return STO_ERR_INVALID_ARG;
    if (!h->factored) return STO_ERR_NOT_READY;
    const void *ys[kMaxRhs];
    void *hs[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) {
        ys[k] = static_cast<const char *>(y) + (size_t)k * h->m * h->esz;
        hs[k] = static_cast<char *>(hx) + (size_t)k * h->m * h->esz;
    }
    return solve_round(h, ys, x0, hs, nrhs, homogeneous != 0, scaled != 0,
                       reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_set_wait_limit(stotree_t h, double seconds) {
    if (!h || !(seconds >= 0.0 && seconds <= 60.0)) return STO_ERR_INVALID_ARG;
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return STO_OK;
}

sto_status stotree_round_status(stotree_t h, sto_stream_t stream) {
    if (!h) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    return check_round_error(h, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_last_primal(stotree_t h, void *x, void *u, sto_stream_t stream) {
    if (!h || !x || !u) return STO_ERR_INVALID_ARG;
    if (!h->factored) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    STO_CUDA(h, cudaMemcpyAsync(x, h->ws + h->L.xs, (size_t)h->Nn * h->nx * h->esz, cudaMemcpyDeviceToDevice, st));
    STO_CUDA(h, cudaMemcpyAsync(u, h->ws + h->L.us, (size_t)h->Np * h->nu * h->esz, cudaMemcpyDeviceToDevice, st));
    return STO_OK;
}

sto_status stotree_estimate_lambda(stotree_t h, void *r0, int32_t iters, double safety, double *lambda,
                                   double *L, sto_stream_t stream) {
    if (!h || !r0 || iters < 1 || !(safety > 0.0) || !lambda) return STO_ERR_INVALID_ARG;
    if (!h->factored) return STO_ERR_NOT_READY;
    return lambda_run(h, r0, iters, safety, lambda, L, reinterpret_cast<cudaStream_t>(stream));
}

static sto_status check_opts(const sto_opts *o) {
    if (!o) return STO_ERR_INVALID_ARG;
    if (!(o->lambda > 0.0) || !(o->tol > 0.0) || o->lbfgs_mem < 1 || o->lbfgs_mem > kMaxMem ||
        o->max_iter < 0 || o->max_ls < 0 || o->max_ls > 30 || !(o->eps_curv >= 0.0))
        return STO_ERR_INVALID_ARG;
    if (o->backtrack < 0 || o->backtrack > 2 || o->max_halvings < 0) return STO_ERR_INVALID_ARG;
    if (o->backtrack == 1 && !(o->bt_param >= 0.0 && o->bt_param < 1.0)) return STO_ERR_INVALID_ARG;
    if (o->backtrack == 2 && !(o->bt_param > 0.0 && o->bt_param < 0.5)) return STO_ERR_INVALID_ARG;
    return STO_OK;
}

sto_status stotree_nama_solve(stotree_t h, const sto_opts *o, const void *x0, void *y, void *x, void *u,
                              void *z, sto_info *info, sto_stream_t stream) {
    if (!h || !x0 || !y) return STO_ERR_INVALID_ARG;
    sto_status s = check_opts(o);
    if (s != STO_OK) return s;
    if (!h->factored || !(h->fg ? h->have_zbox : h->have_box)) return STO_ERR_NOT_READY;
    return solver_run(h, 0, o, x0, y, x, u, z, info, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_minfbe_solve(stotree_t h, const sto_opts *o, const void *x0, void *y, void *x, void *u,
                                void *z, sto_info *info, sto_stream_t stream) {
    if (!h || !x0 || !y) return STO_ERR_INVALID_ARG;
    sto_status s = check_opts(o);
    if (s != STO_OK) return s;
    if (!h->factored || !(h->fg ? h->have_zbox : h->have_box)) return STO_ERR_NOT_READY;
    return solver_run(h, 1, o, x0, y, x, u, z, info, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_gpad_solve(stotree_t h, const sto_opts *o, const void *x0, void *y, void *x, void *u,
                              void *z, sto_info *info, sto_stream_t stream) {
    if (!h || !x0 || !y) return STO_ERR_INVALID_ARG;
    sto_status s = check_opts(o);
    if (s != STO_OK) return s;
    if (!h->factored || !(h->fg ? h->have_zbox : h->have_box)) return STO_ERR_NOT_READY;
    return solver_run(h, 2, o, x0, y, x, u, z, info, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_kkt_check(stotree_t h, const void *x0, const void *x, const void *u, const void *y,
                             double tol_active, double *out, sto_stream_t stream) {
    if (!h || !x0 || !x || !u || !y || !out) return STO_ERR_INVALID_ARG;
    if (!h->ws || !h->have_cost || !(h->fg ? h->have_zbox : h->have_box)) return STO_ERR_NOT_READY;
    return kkt_run(h, x0, x, u, y, tol_active, out, reinterpret_cast<cudaStream_t>(stream));
}

sto_status stotree_set_timing(stotree_t h, int32_t enable) {
    if (!h) return STO_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return STO_OK;
}

sto_status stotree_get_timing(stotree_t h, double *ms, int64_t *launches, int64_t *rhs) {
    if (!h) return STO_ERR_INVALID_ARG;
    double total = h->solve_ms;
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float t = 0.f;
        STO_CUDA(h, cudaEventSynchronize(h->ev_pool[k + 1]));
        STO_CUDA(h, cudaEventElapsedTime(&t, h->ev_pool[k], h->ev_pool[k + 1]));
        total += t;
    }
    h->solve_ms = 0.0;
    h->ev_used = 0;
    if (ms) *ms = total;
    if (launches) *launches = h->solve_launches;
    if (rhs) *rhs = h->solve_rhs;
    h->solve_launches = 0;
    h->solve_rhs = 0;
    return STO_OK;
}

sto_status stotree_solve_bytes(stotree_t h, double *matrix_bytes, double *vector_bytes_per_rhs) {
    if (!h) return STO_ERR_INVALID_ARG;
    const double es = (double)h->esz, nx = h->nx, nu = h->nu, Nn = h->Nn, Np = h->Np;
    // backward and forward each read A^j, B^j of every non-root node; K^i twice, Rbar^-1 once
    if (matrix_bytes) *matrix_bytes = es * (2.0 * (nx * nx + nx * nu) * (Nn - 1) + (2.0 * nu * nx + nu * nu) * Np);
    // y in, Hx out, s and ubar written and read, x and u written and read
    if (vector_bytes_per_rhs)
        *vector_bytes_per_rhs = es * (2.0 * (double)h->m + 2.0 * nu * Np + 2.0 * nx * Nn);
    return STO_OK;
}

}  // extern "C"
