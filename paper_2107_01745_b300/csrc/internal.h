// Internal declarations of libstotree (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "stotree.h"

namespace sto {

constexpr int kMaxMem = 16;          // L-BFGS memory limit (ring has kMaxMem + 1 slots)
constexpr int kMaxRhs = 4;           // right-hand sides per solve round
constexpr int kMaxDim = 1024;        // nx, nu limit
constexpr int kRedBlocks = 592;      // blocks of the reduction kernels (4 per SM on 148 SMs)
constexpr int kRedSlots = 80;        // doubles per block in the partials buffer
constexpr int kMaxCand = 32;         // line-search candidates

// Device-resident state of one MINFBE / NAMA run: every decision of the algorithms is
// taken by device code and read by the host only for the stopping test.
struct SolverScalars {
    // header: the host reads only these first kScalHead bytes per iteration
    double lambda, tol, eps_curv;
    int mem, max_ls, method, nan_flag;
    double phi;       // FBE at the current iterate
    double res_inf;   // ||z - Hx||_inf (unscaled) at the current iterate
    double tau;       // accepted line-search step
    int ls_done, ls_zero, iters, status;
    // step-size backtracking tests (Section III-B): <r_w, Hx(T(w)) - Hx(w)> and ||r_w||^2 of the
    // last forward-backward step, ||r||^2 at the current iterate, ||S H x_lin(r)||^2 there
    double bt_a, bt_b, r2, hr2;
    double cand[kMaxCand];
    // L-BFGS ring of mem+1 slots (slot order = oldest .. newest starting at head)
    int lb_count, lb_head, lb_pending_valid, lb_new_pair;
    double SY[kMaxMem + 1][kMaxMem + 1];   // s_a' y_b by slot
    double YY[kMaxMem + 1][kMaxMem + 1];   // y_a' y_b by slot
    double gamma;                          // H0 = gamma I
    double coef_s[kMaxMem + 1];            // direction d = -(gamma g + sum coef_s[a] s_a + sum coef_y[a] y_a)
    double coef_y[kMaxMem + 1];
    // curvature test pieces of the pending pair
    double sq_dot, s_norm2, g_norm2_prev, g_norm2;
    // power iteration
    double pw_L, pw_inv_norm;
    // general constraint maps: f(x) at the point (k_fcost) and the line search's f(pa) - f(p0),
    // linear and quadratic coefficients in tau (k_fquad); zero for the selection maps
    double f_pt, f_ls[3];
    // reduction bookkeeping
    unsigned int red_counter;
    unsigned int pad2;
    // look-ahead (an iteration is enqueued before the host reads the previous one's result):
    // with `lookahead` set, the residual pass sets `stop` once the run has converged or met a
    // NaN, and every kernel of a later iteration (solve rounds included) then does nothing
    int lookahead, stop;
};
constexpr size_t kScalHead = 112;

struct Layout {
    size_t total = 0;
    // tree
    size_t parent, cbeg, ccnt, soff, node_stage;
    size_t prob64;               // double [Nn]
    size_t sqp;                  // real [Nn] sqrt(pi)
    // FP64 problem data
    size_t G64;                  // double [Nn][nx][ld64] = [A | B | c]
    size_t cost64;               // double [3nx + 3nu... ] Q R PN q r pN
    size_t box64;                // double [5(nx+nu)]: lo, hi, rho, delta, kind
    // factor scratch (FP64)
    size_t P[2], PG, W, Rb, Zb, M, K64;
    size_t fstatus;              // int
    // solve arrays (real)
    size_t G, RK, gu, gx, c;     // RK = [-Rbar^-1 | K] per nonleaf node (nu rows of ldrk)
    size_t Gt, Kt;               // forward pass: [A | B]' per node (nx+nu rows of ldk), K' (nx rows of ldr)
    size_t cost, box;            // real copies: W (Q|R|PN), ell (q|r|pN), lo/hi/rho/delta/kind (x|u)
    // solve scratch: ubar, x, u (real); tagged s, x, u (64-bit words, sizeof(real) / 4 per
    // value; [ts, tus_end) is one range)
    size_t ubar, xs, us;
    size_t ts, txs, tus, tus_end;
    // solver
    size_t vec;                  // kNumVec vectors of m reals
    size_t ringS, ringY;         // (kMaxMem+1) vectors of m reals each
    size_t partials;             // double [kRedBlocks][kRedSlots]
    size_t scal;                 // SolverScalars
    size_t kkt;                  // double scratch for the KKT check
    // solve-round work items (path segments) and their dependency flags
    size_t bstart, bnodes, fstart, fnodes;  // int: segment offsets and node lists
    size_t flags;                // unsigned [2][Nn]: backward / forward completion epochs
    size_t ticket;               // unsigned long long: work-item counter
    // general constraint maps z = F x + G u (FN x at the leaves)
    size_t FG, FG64;             // real / double: F [nc][nx], G [nc][nu], FN [ncN][nx]
    size_t zbox, zbox64;         // real / double: [lo | hi | rho | delta | kind] rows of nc + ncN
    size_t ht, pv;               // real [kMaxRhs][msel]: H'y into and the primal out of a round
    size_t pvec;                 // real [4][msel]: the solvers' primal vectors
    size_t zcost;                // real zeros: the (absent) cost weights of the z entries
};

constexpr int kSegMax = 4;       // nodes per path segment (work item) of a solve round

constexpr int kNumVec = 12;      // ybar, h, r, d, hr, hd, g, tmp0, tmp1, tmp2, tmp3, tmp4

}  // namespace sto

struct stotree_s {
    int Nn = 0, Np = 0, Nl = 0, N = 0, nx = 0, nu = 0;
    int prec = STO_FP32;
    int64_t m = 0, n = 0;
    std::vector<int32_t> parent, cbeg, ccnt, soff, stage;
    std::vector<double> prob;
    int max_width = 0;
    int ld64 = 0;     // G64 row length (nx + nu + 1 rounded to 2)
    int ldg = 0;      // solve G row length (nx + nu rounded to 16 bytes)
    int ldk = 0;      // K row length (nx rounded)
    int ldr = 0;      // -Rbar^-1 columns in RK (nu rounded)
    int ldrk = 0;     // RK row length (ldr + ldk)
    size_t esz = 4;   // sizeof(real)
    sto::Layout L;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<uint8_t> have_dyn;   // per node
    bool have_cost = false, have_box = false, factored = false;
    // host copies of the nonsmooth term g (Section II-B): box [lo | hi] and per component
    // [rho | delta | kind] (kind 0 = indicator of the box, 1 = rho dist, 2 = rho Huber(dist))
    std::vector<double> boxv, pen;
    bool general = false;   // some component's kind is not 0
    // general constraint maps (Section II-C): z^i = F x^i + G u^i at nonleaf nodes, FN x^l at
    // leaves; the dual then has nc entries per nonleaf node and ncN per leaf (m), the solve round
    // keeps its [x; u] layout (msel entries)
    bool fg = false;
    int nc = 0, ncN = 0;
    int64_t msel = 0;
    std::vector<double> Fm, Gm, FNm, zboxv;
    bool have_zbox = false;
    std::string err;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double solve_ms = 0.0;
    int64_t solve_launches = 0, solve_rhs = 0;
    int64_t solve_calls = 0;
    int64_t launches = 0;   // kernels launched through this handle
    // solve-round work items: backward segments (lowest node first, ordered by lowest node
    // descending) and forward segments (top node first, ordered by top node ascending)
    std::vector<int32_t> bstart, bnodes, fstart, fnodes;
    unsigned epoch = 0;                 // last epoch written to the flags
    unsigned long long ticket_base = 0;  // value of the ticket counter before the next round
    int grid_ctas[5] = {0, 0, 0, 0, 0};  // CTAs of the persistent solve kernel, per nrhs
    unsigned long long wait_ns = 1500000000ull;  // limit of each dependency wait in a solve round
    // pinned host mirror of the device scalars
    sto::SolverScalars *host_scal = nullptr;
    sto::SolverScalars *host_scal2 = nullptr;  // second header buffer (GPAD look-ahead)

    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
};

namespace sto {

sto_status cuda_fail(stotree_t h, cudaError_t e, const char *what);
// Raise (never lower) a kernel's dynamic shared-memory cap on the current device.  A cap that a
// later, smaller launch lowered would sit below the size recorded in an earlier captured graph.
cudaError_t raise_smem_cap(const void *func, size_t bytes);
// Blocks that one wave of `func` holds on this device (occupancy x SMs), capped at `want`:
// a grid-stride pass launched with more blocks than one wave leaves a partial second wave.
int wave_grid(const void *func, int threads, size_t smem, int want);
sto_status validate_tree(const int32_t *parent, const double *prob, int Nn, int horizon, std::vector<int32_t> &stage,
                         std::vector<int32_t> &ccnt, std::vector<int32_t> &cbeg);
#define STO_CUDA(h, call)                                       \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return sto::cuda_fail(h, _e, #call); \
    } while (0)

// factor.cu
sto_status factor_run(stotree_t h, cudaStream_t st);

// solve.cu: one round of Algorithm 3/4 on nrhs vectors (real pointers in the workspace
// or caller memory).  scaled: input is ybar and output S Hx.  With `scratch`, the round
// (one right-hand side) keeps its intermediate vectors there instead of in the workspace.
struct SolveScratch {
    void *ubar;                // real [Np][nu]
    void *ts, *txs, *tus;      // tagged words, sizeof(real) / 4 per value: [Nn][nx], [Nn][nx], [Np][nu]
    void *flags;               // unsigned [2][Nn] (cleared by the round)
    void *ticket;              // unsigned long long (cleared by the round)
    unsigned epoch;            // the round's epoch: never used before with these tagged words
};
// With general maps the round computes H'y, runs Algorithm 3/4 in the [x; u] layout into the
// primal vectors pout[k] (the workspace's when pout is null; msel reals, scaled like hx) and
// writes hx = H p.
sto_status solve_round(stotree_t h, const void *const *y, const void *x0, void *const *hx, int nrhs,
                       bool homogeneous, bool scaled, cudaStream_t st, const SolveScratch *scratch = nullptr,
                       void *const *pout = nullptr, const int *stop = nullptr);

// Grid and shared-memory caps of the one-right-hand-side round, set up ahead of its first launch
// (called when the factor is computed, so that later rounds do no host-side set-up work).
sto_status prepare_round(stotree_t h);

sto_status check_round_error(stotree_t h, cudaStream_t st);

// fgmap.cu: H'y into the [x; u] layout (handle precision, or FP64 for the optimality check) and
// Hx = H p from the [x; u] layout, for general constraint maps.
sto_status fg_ht(stotree_t h, const void *y, void *out, bool fp64_out, cudaStream_t st);
sto_status fg_hx(stotree_t h, const void *p, void *out, cudaStream_t st);

sto_status solver_run(stotree_t h, int method, const sto_opts *o, const void *x0, void *y, void *x,
                      void *u, void *z, sto_info *info, cudaStream_t st);
sto_status lambda_run(stotree_t h, void *r0, int iters, double safety, double *lambda, double *L,
                      cudaStream_t st);
sto_status kkt_run(stotree_t h, const void *x0, const void *x, const void *u, const void *y,
                   double tol_active, double *out, cudaStream_t st);

void timing_begin(stotree_t h, cudaStream_t st, cudaEvent_t *ev);
void timing_end(stotree_t h, cudaStream_t st, cudaEvent_t ev0, int nrhs);

}  // namespace sto
