/*
 * stotree.h -- C ABI of the B300 scenario-tree solver library (libstotree.so).
 *
 * The library computes, on one NVIDIA B300 (sm_103a), the data-parallel hot path of
 * dual MINFBE and NAMA for scenario-based stochastic optimal control, after
 * Sampathirao, Patrinos, Bemporad and Sopasakis, "Massively parallelizable proximal
 * algorithms for large-scale stochastic optimal control problems":
 *   - the offline factor of the tree LQ problem (Section III-D),
 *   - the dual-gradient solve x(y) (Algorithm 3) and Hessian-vector products
 *     (Algorithm 4), for one or several right-hand sides,
 *   - Algorithm 1 (dual MINFBE with L-BFGS) and Algorithm 2 (NAMA) around them,
 *   - an FP64 KKT-residual check of a returned primal-dual pair.
 *
 * Problem (Section II): scenario tree with nodes 0..Nn-1 numbered stage by stage,
 * root 0, children of a node contiguous, every leaf at stage N; node probabilities
 * pi^i.  Dynamics x^j = A^j x^i + B^j u^i + c^j for j in child(i) (eq.
 * system_dynamics_tree).  Cost sum over nonleaf i of pi^i (x'Qx + u'Ru + q'x + r'u)
 * plus sum over leaves l of pi^l (x'P_N x + p_N'x), with diagonal Q, R, P_N shared by
 * all nodes (no 1/2 factor, as in Section II-B).  Constraints: box on the block
 * z^i = [x^i; u^i] of every nonleaf node and on z^l = x^l of every leaf; the root
 * state is the parameter p = x0 and is not boxed.
 *
 * Vector layouts.  A dual-sized vector (y, Hx, z; length m = Np(nx+nu) + Nl nx) has
 * one block per node: nonleaf i at offset i(nx+nu) holding [x-part (nx); u-part (nu)],
 * leaf l at offset Np(nx+nu) + (l-Np)nx holding [x-part (nx)].  With general constraint
 * maps (stotree_set_constraint_maps) the blocks hold z^i = F x^i + G u^i (nc entries) and
 * z^l = FN x^l (ncN).  Primal outputs are x [Nn][nx] (x[0] = x0) and u [Np][nu].
 *
 * Precision: a handle is created either FP64 (every device array and vector of the
 * solve path in double) or FP32 (solve step, prox and L-BFGS in float; the factor
 * always runs in FP64 and is rounded to FP32 once).  "real" below is double or
 * float accordingly; scalars crossing the ABI are double.
 *
 * Memory.  The library never allocates device memory: the caller asks for the
 * workspace size, allocates it (e.g. as a torch tensor) and binds it.  All vector
 * arguments of the solve calls are device pointers owned by the caller, 16-byte
 * aligned.  Host arrays passed to the set-up calls are copied before return.
 *
 * Streams and errors.  Every call taking a cudaStream_t enqueues its work on that
 * stream; the *_solve calls and stotree_estimate_lambda synchronise the stream
 * before returning (their results are host scalars).  Errors are returned, never
 * trapped; a CUDA error is reported as STO_ERR_CUDA and the message is kept for
 * stotree_last_error().  Calls on one handle must not overlap in time: the handle's
 * workspace holds the intermediate state of every call.
 */
#ifndef STOTREE_H
#define STOTREE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STO_API __attribute__((visibility("default")))
#else
#define STO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sto_stream_t; /* = cudaStream_t; NULL is the legacy default stream */
typedef struct stotree_s *stotree_t;

typedef enum {
    STO_OK = 0,
    STO_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad option value */
    STO_ERR_TREE = 2,          /* numbering or probabilities violate the tree conventions */
    STO_ERR_NOT_READY = 3,     /* workspace not bound, data missing or not factored */
    STO_ERR_NUMERICAL = 4,     /* Rbar not positive definite, or NaN/Inf met in a solve */
    STO_ERR_CUDA = 5,          /* a CUDA runtime call failed (see stotree_last_error) */
    STO_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    STO_NOT_CONVERGED = 7,     /* max_iter reached; the last iterate is still returned */
    STO_ERR_WORKSPACE = 8      /* workspace smaller than stotree_workspace_size() */
} sto_status;

typedef enum { STO_FP64 = 0, STO_FP32 = 1 } sto_precision;

/* Tree (Section II-A).  parent[0] = -1, parent[i] < i, stage(parent[i]) = stage(i) - 1,
 * nodes sorted by stage, children of each node contiguous, all leaves at stage horizon;
 * prob[0] = 1, prob > 0, sum over child(i) of prob = prob[i] (relative tolerance 1e-9).
 * Host pointers, copied. */
typedef struct {
    int32_t num_nodes, horizon, nx, nu;
    const int32_t *parent;
    const double *prob;
} sto_tree_desc;

/* Options of Algorithms 1 and 2 (stotree_nama_solve, stotree_minfbe_solve), of GPAD
 * (stotree_gpad_solve: lambda, tol, max_iter) and of the batched NAMA (stobatch_nama_solve: no
 * backtracking, the step comes per group). */
typedef struct {
    double lambda;      /* step, in (0, 1/L) (Algorithm 1 input); see stotree_estimate_lambda */
    double tol;         /* stop when ||z - Hx||_inf <= tol (unscaled residual, Section III-B) */
    double eps_curv;    /* epsilon' of the L-BFGS curvature test (Li-Fukushima) */
    int32_t lbfgs_mem;  /* L-BFGS memory, 1..16 */
    int32_t max_iter;   /* iteration cap; STO_NOT_CONVERGED when hit */
    int32_t max_ls;     /* line-search halvings tau = 2^0 .. 2^-max_ls (<= 30), then tau = 0 */
    int32_t backtrack;  /* step-size backtracking when L is unknown (Section III-B), Algorithms 1
                           and 2 only: 0 = fixed lambda; 1 = eq. (original-backtracking): after
                           the forward-backward step from the accepted line-search point w,
                           lambda is halved if fhat(T(w)) > fhat(w) - lambda <grad fhat(w), R(w)>
                           + (1 - beta) lambda/2 ||R(w)||^2 (for this quadratic fhat: if
                           <R(w), Hx(T(w)) - Hx(w)> > (1 - beta) ||R(w)||^2), and the iteration is
                           repeated from the current iterate; 2 = eq. (simple-backtracking): at
                           the current iterate y, lambda is halved while lambda ||grad fhat(T(y))
                           - grad fhat(y)|| > eps'' ||T(y) - y|| (= lambda ||H x_lin(R)|| >
                           eps'' ||R||).  Every halving empties the L-BFGS memory. */
    double bt_param;    /* beta in [0, 1) for backtrack = 1, eps'' in (0, 1/2) for backtrack = 2 */
    int32_t max_halvings; /* cap on halvings (>= 0); STO_NOT_CONVERGED beyond it */
    int32_t pad_;
} sto_opts;

typedef struct {
    int32_t iters;        /* iterations k performed */
    int32_t solve_calls;  /* right-hand sides pushed through Algorithm 3/4 ("oracle calls") */
    int32_t status;       /* sto_status of the solve */
    int32_t ls_zero;      /* iterations whose line search fell back to tau = 0 */
    int32_t launches;     /* CUDA kernels launched by the call */
    int32_t halvings;     /* step-size halvings of the backtracking (sto_opts.backtrack) */
    double res_inf;       /* ||z - Hx||_inf at the returned iterate */
    double fbe;           /* phi_lambda at the returned iterate (scaled dual) */
    double ms;            /* wall time of the call on the stream, milliseconds */
    double lambda;        /* the step at return (opts->lambda unless backtracking halved it) */
} sto_info;

/* Validate the tree and create a handle.  No device work.  The tree is the scenario tree of
 * Section II-A: every node's probability is the sum of its children's, and the probabilities
 * of each stage add up to one.
 * Errors: STO_ERR_INVALID_ARG (null pointer, nx < 1, nu < 1, m >= 2^31, or a padded row width
 * above the solve kernel's register tiling: max(pad(nx + nu), pad(nx) + pad(nu)) > 512 for FP32
 * or > 256 for FP64, pad = round up to 16 bytes), STO_ERR_TREE. */
STO_API sto_status stotree_create(const sto_tree_desc *tree, int32_t precision, stotree_t *out);

/* General constraint maps (Section II-C) instead of the selection of [x; u]: z^i = F x^i + G u^i at
 * every nonleaf node (the root included, with x^0 = x0) and z^l = FN x^l at every leaf, the same
 * F [nc][nx], G [nc][nu], FN [ncN][nx] (host FP64, row-major, copied) at every node.  The dual
 * then has one block of nc entries per nonleaf node and of ncN per leaf (m = Np nc + Nl ncN, the
 * same block order as the selection layout); y, Hx, z and every dual-sized argument below use
 * that layout, and the box is the one of stotree_set_zbox (stotree_set_box is not used).  Call it
 * after stotree_create and before stotree_workspace_size / stotree_bind_workspace (it changes m
 * and the workspace).  A solve round then computes H'y, runs Algorithm 3/4 in the [x; u] layout
 * and forms Hx = H [x; u]; the solvers take f(x) of the FBE from the primal of each round.  Not
 * with soft terms (stotree_set_penalty) or the no-allocation solve step.
 * Errors: STO_ERR_INVALID_ARG (sizes < 1 or > 1024, m >= 2^31, non-finite entries, workspace
 * already bound). */
STO_API sto_status stotree_set_constraint_maps(stotree_t h, int32_t nc, int32_t ncN, const double *F, const double *G,
                                               const double *FN);

/* The box zlo <= z <= zhi [nc] of the nonleaf blocks and zNlo <= z <= zNhi [ncN] of the leaf blocks
 * (general maps; +-INFINITY allowed; host FP64).  Synchronises.  Errors: STO_ERR_INVALID_ARG
 * (no general maps, lo > hi), STO_ERR_NOT_READY (no workspace). */
STO_API sto_status stotree_set_zbox(stotree_t h, const double *zlo, const double *zhi, const double *zNlo,
                                    const double *zNhi, sto_stream_t stream);

/* Release the handle (host memory only; the workspace belongs to the caller). */
STO_API void stotree_destroy(stotree_t h);

/* Problem sizes: m (dual length), n (primal length Np nu + (Nn-1) nx), Np, Nl. */
STO_API sto_status stotree_sizes(stotree_t h, int64_t *m, int64_t *n, int32_t *num_nonleaf, int32_t *num_leaves);

/* Device workspace needed for every call of this handle, in bytes (256-byte aligned
 * sections; the caller passes a 256-byte aligned base). */
STO_API sto_status stotree_workspace_size(stotree_t h, size_t *bytes);

/* Bind caller-owned device memory of at least stotree_workspace_size() bytes and
 * upload the tree arrays on the stream.  Errors: STO_ERR_WORKSPACE, STO_ERR_INVALID_ARG. */
STO_API sto_status stotree_bind_workspace(stotree_t h, void *dev_ptr, size_t bytes, sto_stream_t stream);

/* Upload the dynamics of nodes [first, first+count) (eq. system_dynamics_tree): host
 * FP64 A [count][nx][nx], B [count][nx][nu], c [count][nx], row-major, where entry k
 * belongs to node first+k.  Node 0's data is ignored.  May be called in chunks.  A and B may
 * both be NULL to replace only the disturbances c of nodes that already have their matrices
 * (a new scenario draw of the same system; STO_ERR_NOT_READY otherwise).  Invalidates the
 * factor. */
STO_API sto_status stotree_set_dynamics(stotree_t h, int32_t first, int32_t count, const double *A,
                                const double *B, const double *c, sto_stream_t stream);

/* Upload the shared costs (Section II-B): diagonals Q [nx], R [nu] (> 0), P_N [nx] (>= 0)
 * and linear terms q [nx], r [nu], p_N [nx] (NULL = zero).  Host FP64.  Invalidates the factor. */
STO_API sto_status stotree_set_costs(stotree_t h, const double *Q, const double *R, const double *PN,
                             const double *q, const double *r, const double *pN, sto_stream_t stream);

/* Upload the shared box (Section II-B, indicator of Y): xlo <= x <= xhi on every non-root
 * node's state, ulo <= u <= uhi on every nonleaf input.  +-INFINITY allowed.  Host FP64. */
STO_API sto_status stotree_set_box(stotree_t h, const double *xlo, const double *xhi, const double *ulo,
                           const double *uhi, sto_stream_t stream);

/* The nonsmooth term g of Section II-B beyond the indicator of the box, per component of
 * [x; u] (host arrays of nx + nu; the leaf terms use the x part; the root state has none):
 *   kind[k] = 0: indicator of [lo_k, hi_k] (hard constraint, the default);
 *   kind[k] = 1: rho[k] * dist(z_k, [lo_k, hi_k]) (soft constraint, "distance-to-set";
 *                lo_k = hi_k = c gives rho |z_k - c|, the l1 norm);
 *   kind[k] = 2: rho[k] * Huber_delta[k](dist(z_k, [lo_k, hi_k])), Huber(d) = d^2/2 for
 *                d <= delta, delta (d - delta/2) beyond (lo_k = hi_k = c: the Huber loss).
 * Their proximal maps are element-wise (Section III-D), so Algorithms 1 and 2 and GPAD use
 * them unchanged; the bounds come from stotree_set_box (+-INFINITY allowed).  kind = NULL
 * restores all-hard.  Needs rho > 0 for kinds 1 and 2, delta > 0 for kind 2 (finite), else
 * STO_ERR_INVALID_ARG.  Does not invalidate the factor.  Synchronises when the box is set. */
STO_API sto_status stotree_set_penalty(stotree_t h, const int32_t *kind, const double *rho, const double *delta,
                               sto_stream_t stream);

/* Offline factor (Section III-D, Riccati-type recursion), FP64 on the device, then the
 * solve arrays in the handle's precision.  Enqueued on the stream; the positive
 * definiteness check of Rbar is reported by the next synchronising call, or here when
 * sync != 0.  Errors: STO_ERR_NOT_READY, STO_ERR_NUMERICAL (sync only). */
STO_API sto_status stotree_factor(stotree_t h, int32_t sync, sto_stream_t stream);

/* One solve round of Algorithm 3 (homogeneous = 0) or Algorithm 4 (homogeneous = 1) for
 * nrhs right-hand sides (1..4) sharing one pass over the factor arrays (the parallel
 * x(r), x(d) evaluation of Section III-C).
 *   y    device real [nrhs][m]: dual vectors.  scaled = 0: unscaled y; scaled = 1: the
 *        preconditioned ybar of Section III-E, i.e. y = sqrt(pi) ybar per node block.
 *   x0   device real [nx], the root state p (ignored when homogeneous).
 *   hx   device real [nrhs][m]: Hx(y) laid out like y; with scaled = 1 the output is
 *        sqrt(pi) Hx per block.  The root block holds [x0; u^0] ([0; u^0] if homogeneous).
 * Asynchronous; a dependency wait that gives up is reported by stotree_round_status.
 * Errors: STO_ERR_INVALID_ARG, STO_ERR_NOT_READY. */
STO_API sto_status stotree_solve_step(stotree_t h, const void *y, const void *x0, void *hx, int32_t nrhs,
                              int32_t homogeneous, int32_t scaled, sto_stream_t stream);

/* stotree_solve_step for one right-hand side without any allocation (the paper has no
 * counterpart).  For callers that cannot call cudaMalloc, or any allocator, while they run a
 * solve: e.g. a controller whose device-memory plan is frozen after start-up.  The handle must
 * be set up and factored beforehand (stotree_factor also sets up this call's launch, so even
 * the handle's first solve needs no host-side set-up); a call then touches only y, hx, the
 * factor arrays in the bound workspace and a fixed 32 MiB scratch array compiled into the
 * library, which every GPU that loads the library holds until the process exits.  Solve-step
 * timing (stotree_set_timing) does not cover this call.
 *   y, x0, hx, homogeneous, scaled: as stotree_solve_step with nrhs = 1.
 * Limit: with esz = sizeof(real) and a256(v) = v rounded up to a multiple of 256, the call
 * needs a256(Np nu esz) + 2 a256(2 Nn nx esz) + a256(2 Np nu esz) + a256(8 Nn) + 256 bytes of
 * scratch (ubar; s, x and u as tagged words, 8 bytes per 4 bytes of a value; the round's
 * dependency flags and its work counter), at most 33554432 (32 MiB); larger problems get
 * STO_ERR_INVALID_ARG and a message in stotree_last_error.  The first call on a
 * device looks the array's address up (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other handles) race and give wrong results.  The
 * primal trajectory stays in the array, so stotree_last_primal keeps reporting the last
 * round of stotree_solve_step.  A dependency wait that gives up is reported by
 * stotree_round_status.
 * Asynchronous.  Errors: STO_ERR_INVALID_ARG, STO_ERR_NOT_READY, STO_ERR_CUDA. */
STO_API sto_status stotree_solve_step_noalloc(stotree_t h, const void *y, const void *x0, void *hx,
                                              int32_t homogeneous, int32_t scaled, sto_stream_t stream);

/* Limit of each dependency wait inside a solve round (a node waiting for the round's work on
 * its children in the backward pass, or on its parent in the forward pass), in seconds, from 0
 * to 60; default 1.5.  Waits that give up let the round finish without them (its output is then
 * wrong) and are reported as STO_ERR_TIMEOUT by the next synchronising call or by
 * stotree_round_status.  0 gives up at the first check that finds the dependency unfinished.
 * Copy waits inside the round keep their fixed 1.5 s limit.  Host only. */
STO_API sto_status stotree_set_wait_limit(stotree_t h, double seconds);

/* Status of the solve rounds enqueued since the last synchronising call (stotree_solve_step,
 * stotree_solve_step_noalloc): synchronises the stream and returns STO_ERR_TIMEOUT if a bounded
 * wait inside one of them gave up (the results of those rounds are wrong), else STO_OK.  On
 * STO_ERR_TIMEOUT the round state (dependency flags, work counter, error word) is reset, so the
 * next round runs normally.  The *_solve calls and stotree_estimate_lambda check this themselves.
 * Errors: STO_ERR_INVALID_ARG, STO_ERR_NOT_READY, STO_ERR_CUDA, STO_ERR_TIMEOUT. */
STO_API sto_status stotree_round_status(stotree_t h, sto_stream_t stream);

/* Primal trajectory of the last solve round's first right-hand side: x [Nn][nx],
 * u [Np][nu] (device real).  Asynchronous. */
STO_API sto_status stotree_last_primal(stotree_t h, void *x, void *u, sto_stream_t stream);

/* Estimate L = ||grad^2 fhat|| of the preconditioned dual by `iters` power iterations on
 * r -> -sqrt(pi) H x_lin(sqrt(pi) r) (Algorithm 4) from the caller's start vector r0
 * (device real [m], overwritten), and return lambda = safety / L.  Synchronises. */
STO_API sto_status stotree_estimate_lambda(stotree_t h, void *r0, int32_t iters, double safety,
                                   double *lambda, double *L, sto_stream_t stream);

/* Algorithm 2 (NAMA) on the preconditioned dual, from y (device real [m], unscaled; zeros
 * for a cold start).  On return: y = the final dual iterate (unscaled), x [Nn][nx],
 * u [Np][nu] = x(y), z [m] = z_lambda(y) (unscaled); any of x, u, z may be NULL.
 * x0 is the device root state.  Synchronises the stream; fills info.
 * Errors: STO_ERR_INVALID_ARG, STO_ERR_NOT_READY, STO_ERR_NUMERICAL, STO_NOT_CONVERGED. */
STO_API sto_status stotree_nama_solve(stotree_t h, const sto_opts *opts, const void *x0, void *y, void *x,
                              void *u, void *z, sto_info *info, sto_stream_t stream);

/* Algorithm 1 (dual MINFBE with L-BFGS directions); arguments as stotree_nama_solve. */
STO_API sto_status stotree_minfbe_solve(stotree_t h, const sto_opts *opts, const void *x0, void *y, void *x,
                                void *u, void *z, sto_info *info, sto_stream_t stream);

/* GPAD, the accelerated dual projected gradient (Section III-F, where a few of its steps warm
 * start Algorithms 1 and 2, and Section IV, where it is the comparison method), on the
 * preconditioned dual with the theta sequence of Patrinos and Bemporad (2014):
 * w_k = ybar_k + theta_k (1/theta_{k-1} - 1)(ybar_k - ybar_{k-1}), w_0 = ybar_0,
 * ybar_{k+1} = T_lambda(w_k), theta_{-1} = theta_0 = 1,
 * theta_{k+1} = (sqrt(theta_k^4 + 4 theta_k^2) - theta_k^2) / 2.
 * Each iteration is one solve round at w_k and one elementwise pass.  The stopping test
 * ||z - Hx||_inf <= tol (unscaled) is applied at w_k; on return y = w_k (unscaled) and
 * x, u, z are x(w_k), z_lambda(w_k), with info->iters = the number of steps taken before it
 * (max_iter = 5 gives the five-step warm start: six solve rounds).  opts->lbfgs_mem, max_ls
 * and eps_curv are not used but must be valid.  Arguments, synchronisation and errors as
 * stotree_nama_solve. */
STO_API sto_status stotree_gpad_solve(stotree_t h, const sto_opts *opts, const void *x0, void *y, void *x,
                              void *u, void *z, sto_info *info, sto_stream_t stream);

/* FP64 optimality check of a primal-dual pair (x, u, y), all device real, against the FP64
 * problem data (conditions listed under Algorithm 1):
 *   out[0] = max |x^j - A^j x^i - B^j u^i - c^j|              (dynamics, x^0 = x0)
 *   out[1] = max |stationarity of f(x) + <y, Hx> in (x, u)|   (-H'y in the subdifferential of f)
 *   out[2] = max over box violation of Hx                      (primal feasibility, hard terms)
 *   out[3] = max |y_k| over components strictly inside the box by more than tol_active;
 *            for soft terms (stotree_set_penalty) the distance of y_k to the gradient of
 *            g_k at Hx where g_k is differentiable there
 *   out[4] = max of -y_k at upper bounds / +y_k at lower bounds (sign of the multipliers);
 *            for soft terms the distance of y_k to the subdifferential at a kink
 *   out[5] = sum over the components of g_k(h_k) + g_k*(y_k) - y_k h_k, h = Hx (the
 *            Fenchel-Young gap: >= 0, zero exactly at y in the subdifferential; with x = x(y) it is
 *            the duality gap of the primal and dual objectives of Section II-D).  For the box,
 *            g_k = 0 and g_k*(y) = hi y (y > 0) or lo y (y < 0); the soft terms add rho dist or
 *            rho Huber(dist), and y^2 / (2 rho) for Huber, without imposing the conjugates'
 *            domains (out[3], out[4] measure those).  Summed in FP64 in a fixed order.
 * Synchronises.  out is host double[6]. */
STO_API sto_status stotree_kkt_check(stotree_t h, const void *x0, const void *x, const void *u, const void *y,
                             double tol_active, double *out, sto_stream_t stream);

/* Per-launch timing of the solve-step kernels with CUDA events on the launching stream:
 * enable (1) / disable (0); read the accumulated device milliseconds and launch count. */
STO_API sto_status stotree_set_timing(stotree_t h, int32_t enable);
STO_API sto_status stotree_get_timing(stotree_t h, double *solve_ms, int64_t *solve_launches,
                              int64_t *solve_rhs);

/* Bytes of matrix data one solve round reads (algorithmic, independent of nrhs) and of
 * vector data per right-hand side, for roofline accounting. */
STO_API sto_status stotree_solve_bytes(stotree_t h, double *matrix_bytes, double *vector_bytes_per_rhs);

STO_API const char *stotree_status_str(sto_status s);
STO_API const char *stotree_last_error(stotree_t h);

/* ---------------------------------------------------------------------------------------------
 * Batched instances.  Many MPC problems solved together: shape groups that share the tree, the
 * dynamics (A, B), the diagonal costs and the box, and instances that differ in the root state
 * x0 and the disturbances c^j.  The group's tree has `branching` children per node for the first
 * `branch_stages` stages and one child after that, so node probabilities are uniform within a
 * stage and the factor of Section III-D reduces to one matrix set per stage (R~_t, K_t); a solve
 * round (Algorithm 3/4) processes every (node, instance) column of a stage of every group
 * together, and NAMA (Algorithm 2) runs per instance with the readings of stotree_nama_solve.
 * Limits: nx <= 64, nu <= 32, horizon <= 64, zero linear cost terms, FP32 solve path.
 * Batch vectors hold the instances one after another (groups in order, instances in order),
 * each in the single-instance dual layout.
 * ------------------------------------------------------------------------------------------- */
typedef struct stobatch_s *stobatch_t;

typedef struct {
    int32_t horizon, branching, branch_stages, nx, nu, num_instances;
    const double *A, *B;             /* [nx][nx], [nx][nu], shared by the group; host, copied */
    const double *Q, *R, *PN;        /* diagonals */
    const double *xlo, *xhi, *ulo, *uhi;
} sto_group_desc;

/* Create a batch from ngroups group descriptions.  Errors: STO_ERR_INVALID_ARG (limits above). */
STO_API sto_status stobatch_create(const sto_group_desc *groups, int32_t ngroups, stobatch_t *out);
STO_API void stobatch_destroy(stobatch_t b);

/* Total batch vector length, number of instances, and per-instance offset / length (arrays of
 * num_instances entries, may be NULL). */
STO_API sto_status stobatch_sizes(stobatch_t b, int64_t *total_dual, int32_t *num_instances, int64_t *inst_offsets,
                                  int64_t *inst_sizes);
STO_API sto_status stobatch_workspace_size(stobatch_t b, size_t *bytes);
STO_API sto_status stobatch_bind_workspace(stobatch_t b, void *dev_ptr, size_t bytes, sto_stream_t stream);

/* Instance data: x0 [nx] and disturbances c [Nn][nx] of the group's tree (row 0 unused; the
 * parameter p and the c^j of eq. system_dynamics_tree), host FP64.  Invalidates the factor. */
STO_API sto_status stobatch_set_instance(stobatch_t b, int32_t group, int32_t instance, const double *x0,
                                         const double *c, sto_stream_t stream);

/* FP64 stage factor of every group (the recursion of Section III-D, one matrix set per stage)
 * and the affine terms of every instance.  Synchronises;
 * STO_ERR_NUMERICAL if some R + B'PB is not positive definite. */
STO_API sto_status stobatch_factor(stobatch_t b, sto_stream_t stream);

/* One batched solve round (Algorithm 3 / 4, one right-hand side per instance): y, hx device
 * float batch vectors, 16-byte aligned (else STO_ERR_INVALID_ARG); scaled as in stotree_solve_step.  The round is one persistent launch that
 * hands out tiles of (node, instance) columns of one (group, stage) in dependency order; each
 * tile waits, bounded, for the tiles of the stage it reads.  Asynchronous; a wait that gives up
 * is reported by stobatch_round_status (or by the next stobatch_nama_solve). */
STO_API sto_status stobatch_solve_step(stobatch_t b, const void *y, void *hx, int32_t homogeneous, int32_t scaled,
                                       sto_stream_t stream);

/* NAMA (Algorithm 2) for every instance (opts.lbfgs_mem <= 8).  lambdas [ngroups] host.  y (device float batch
 * vector, unscaled; zeros for a cold start) receives the final duals, z and hx (may be NULL) the
 * z_lambda and Hx of each instance's final iterate; infos [num_instances] (may be NULL).  An
 * instance stops at its own tolerance; the call returns STO_NOT_CONVERGED if some instance hit
 * max_iter.  Synchronises the stream. */
STO_API sto_status stobatch_nama_solve(stobatch_t b, const sto_opts *opts, const double *lambdas, void *y, void *z,
                                       void *hx, sto_info *infos, sto_stream_t stream);
/* Status of the batched rounds enqueued since the last synchronising call: synchronises and
 * returns STO_ERR_TIMEOUT if a dependency wait inside one of them gave up (their results are
 * wrong; the error word is cleared), else STO_OK.  Errors: STO_ERR_INVALID_ARG, STO_ERR_NOT_READY,
 * STO_ERR_CUDA, STO_ERR_TIMEOUT. */
STO_API sto_status stobatch_round_status(stobatch_t b, sto_stream_t stream);

/* The round configuration chosen by the batch's tuner, which stobatch_factor runs once per batch
 * (the paper has no counterpart).  It times one round of each candidate -- the tile kernel with 32
 * columns on 128-thread CTAs, 32 columns on 256-thread CTAs and 64 columns on 256-thread CTAs
 * (each thread a block of rows and columns of the stage products), and the column kernel with
 * one column per thread on 128-thread CTAs (only when every group has nx <= 32 and nu <= 16) --
 * and keeps the fastest, separately for one and two right-hand sides.  For nrhs = 1 or 2: the
 * chosen tile width in columns, the threads per CTA, the CTAs of the persistent launch (0 before
 * a round of that variant was set up) and the measured round time of each candidate in the order
 * above (host double[4], may be NULL; -1 for a candidate that does not apply), in milliseconds.
 * Host only. */
STO_API sto_status stobatch_round_config(stobatch_t b, int32_t nrhs, int32_t *tile_cols, int32_t *cta_threads,
                                         int32_t *ctas, double *tuned_ms);

/* Override the tuner's choice for rounds with nrhs = 1 or 2 right-hand sides: variant 0..3 in the
 * order of stobatch_round_config's candidates.  Every variant computes the same round.  Errors:
 * STO_ERR_INVALID_ARG (bad nrhs or variant, or the column kernel for a batch with nx > 32 or
 * nu > 16).  Host only. */
STO_API sto_status stobatch_set_round_variant(stobatch_t b, int32_t nrhs, int32_t variant);
STO_API const char *stobatch_last_error(stobatch_t b);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start: a per-node perceptron that predicts the scaled dual ybar^i = y^i/sqrt(pi^i)
 * (Section III-E) of every node of a tree from the node's data, trained with Adam on the duals
 * that the batched solver returns.  The paper's own warm start is a few accelerated dual
 * gradient steps (Section III-F); this predictor replaces them for families of problems that
 * share a tree and its dynamics.
 *
 * Network: d_in = 4 nx + 1 inputs [x0, t/N, c^i, c^anc(i), c^anc(anc(i))] (missing ancestors and
 * the root's c are zeros) -> hidden -> hidden -> d_out = nx + nu, GELU (tanh form) on the hidden
 * layers.  Products run on the tensor cores in BF16 with FP32 accumulation; weights are kept in
 * FP32 for Adam and copied to BF16 after each step; hidden activations and output gradients are
 * stored in BF16.  Loss: mean over the valid outputs (nx + nu at nonleaf nodes, nx at leaves) of
 * the squared difference to ybar.
 *
 * Parameter vector order (FP32, host): W1 [hidden][d_in], b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], W3 [d_out][hidden], b3 [d_out].
 * ------------------------------------------------------------------------------------------- */
typedef struct stowarm_s *stowarm_t;

typedef struct {
    int32_t num_nodes, horizon, nx, nu;  /* tree and sizes, rules as in sto_tree_desc (nx + nu <= 256) */
    const int32_t *parent;               /* host [num_nodes] */
    const double *prob;                  /* host [num_nodes] */
    int32_t hidden;                      /* 128 or 256 */
    int32_t batch;                       /* rows per training step: a multiple of 256, at most 65536 */
    uint64_t seed;                       /* weight initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) */
} sto_warm_desc;

/* STO_ERR_INVALID_ARG / STO_ERR_TREE on bad sizes or tree. */
STO_API sto_status stowarm_create(const sto_warm_desc *desc, stowarm_t *out);
STO_API void stowarm_destroy(stowarm_t h);
STO_API sto_status stowarm_dims(stowarm_t h, int32_t *d_in, int32_t *d_out, int64_t *num_params);
STO_API sto_status stowarm_workspace_size(stowarm_t h, size_t *bytes);
/* Device workspace (>= workspace_size bytes, 1024-byte aligned, caller-owned); initialises the
 * weights and the Adam state.  Synchronises. */
STO_API sto_status stowarm_bind_workspace(stowarm_t h, void *dev_ptr, size_t bytes, sto_stream_t stream);
/* Host FP32 parameter vector in the order above; set_params also resets the Adam state.
 * Both synchronise. */
STO_API sto_status stowarm_set_params(stowarm_t h, const float *params, sto_stream_t stream);
STO_API sto_status stowarm_get_params(stowarm_t h, float *params, sto_stream_t stream);
/* Inference on caller features: X device [rows][d_in] FP32 -> Y device [rows][d_out] FP32;
 * rows <= batch.  Asynchronous. */
STO_API sto_status stowarm_forward(stowarm_t h, const float *X, int32_t rows, float *Y, sto_stream_t stream);
/* Loss and gradient (device [num_params] FP32; loss: device scalar, may be NULL) of one batch
 * of caller rows: X [rows][d_in], targets T [rows][d_out], nvalid [rows] (outputs beyond
 * nvalid[r] are ignored).  Asynchronous. */
STO_API sto_status stowarm_gradients(stowarm_t h, const float *X, const float *T, const int32_t *nvalid,
                                     int32_t rows, float *grad, float *loss, sto_stream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on one batch of caller rows.  Asynchronous. */
STO_API sto_status stowarm_train_batch(stowarm_t h, const float *X, const float *T, const int32_t *nvalid,
                                       int32_t rows, float lr, sto_stream_t stream);
/* Training set: num_draws problems on the tree, device FP32 x0 [D][nx], c [D][num_nodes][nx]
 * (row 0 unused) and, for training, their duals y [D][m] (unscaled, the dual layout of the
 * single-instance API; may be NULL for prediction only).  The arrays stay caller-owned and
 * must outlive their use. */
STO_API sto_status stowarm_set_draws(stowarm_t h, int32_t num_draws, const float *x0, const float *c,
                                     const float *y);
/* `steps` Adam steps on batches of (draw, node) samples, each epoch visiting the samples in
 * the order of a seeded affine permutation of the sample index (the remainder of an epoch
 * that does not fill a batch is skipped).  loss_hist: device [steps] or NULL.  Replays one
 * CUDA graph per step; asynchronous. */
STO_API sto_status stowarm_train(stowarm_t h, int32_t steps, float lr, uint64_t shuffle_seed, float *loss_hist,
                                 sto_stream_t stream);
/* Predicted duals of draws [draw0, draw0 + num_draws): y_out device [num_draws][m], unscaled
 * (sqrt(pi^i) times the predicted ybar^i).  Asynchronous. */
STO_API sto_status stowarm_predict(stowarm_t h, int32_t draw0, int32_t num_draws, float *y_out,
                                   sto_stream_t stream);
/* The tensor-core product used above, on its own: C [M][N] (FP32, row stride ldc) = A B' with
 * A [M][K] and B [N][K] BF16, row strides lda, ldb (elements, multiples of 8), device pointers
 * aligned to 16 bytes.  Asynchronous. */
STO_API sto_status stowarm_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc,
                                     int32_t M, int32_t N, int32_t K, sto_stream_t stream);
STO_API const char *stowarm_last_error(stowarm_t h);

#ifdef __cplusplus
}
#endif

#endif /* STOTREE_H */
