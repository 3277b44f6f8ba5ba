// Algorithm 3 (dual gradient x(y)) and Algorithm 4 (Hessian-vector products) on the device:
// one persistent kernel per solve round.
//
// With the factor of Section III-D (see factor.cu), one solve round is
//   backward, children before parents:
//     s^l    = y^l / 2 + pi^l p_N / 2                    (leaf children, formed on the fly)
//     acc    = sum_{j in child(i)} G^j' s^j   with G^j = [A^j | B^j]  -> [A's ; B's]
//     v^i    = y_u^i / 2 + acc_B + gu^i
//     ubar^i = -Rbar^-1 v^i,     s^i = y_x^i / 2 + acc_A + K^i' v^i + gx^i
//   forward, parents before children:
//     x^0 = p,   x^j = G^j [x^i; u^i] + c^j,   u^j = K^j x^j + ubar^j
// and Algorithm 4 is the same with c, gu, gx, the leaf term and p set to zero.  Algorithm 3
// overwrites u^i, q^i in its child loop where Algorithm 4 accumulates; both accumulate here.
// Several right-hand sides share every matrix load (the parallel x(r), x(d) of Section III-C).
//
// Scheduling.  "For k = N-1..0, in parallel over nodes(k)" needs a grid-wide barrier per
// stage; instead the round is a dataflow over work items, each a path segment of up to
// kSegMax nodes (api.cu: build_segments).  A ticket counter hands the items out in an order in
// which every item depends only on earlier ones; an item waits (bounded) for the vectors of the
// segments it depends on, so a CTA holding a ticket never waits on a later one and all CTAs are
// resident (grid = occupancy): no deadlock.  Inside a segment the recursion's vector stays in
// shared memory; between segments it travels as tagged words (below).
//
// Data movement.  The node matrices are independent of the solve, so one producer warp per
// CTA streams the matrices of its items with cp.async.bulk (TMA bulk copies) into a ring of
// shared-memory slots, running ahead of the four consumer warps by up to the ring depth; the
// consumers read the slots in axpy form (warps over rows, lanes over 16-byte column groups,
// one cross-warp reduction per matrix; the forward pass reads transposed copies G^j', K^j' so
// that it has the same form) and release them through mbarriers.  Every wait is bounded: on expiry the kernel raises an error flag, stops waiting
// and runs to its end, and the host reports STO_ERR_TIMEOUT.
#include <cstdint>

#include "internal.h"

namespace sto {
namespace {

constexpr int kCW = 4;               // consumer warps
constexpr int kCtasPerSm = 3;        // resident CTAs per SM (shared memory and registers allow 3)
constexpr int kThreadsT = (kCW + 1) * 32;
constexpr int kSlots = 4;            // ring depth
constexpr int kChunk = 15360;        // bytes per ring slot (three CTAs fit in an SM's shared memory)
constexpr unsigned long long kWaitNs = 1500000000ull;  // bounded waits: 1.5 s of wall time

enum : int { KIND_END = 0, KIND_BG = 1, KIND_BP = 2, KIND_FG = 4, KIND_FK = 5 };
enum : int {
    F_FIRST = 1,        // first chunk of this (kind, node) run
    F_LAST = 2,         // last chunk of this run
    F_FIRST_CHILD = 4,  // backward G: first child of the parent
    F_INSEG = 8,        // the child (backward) / parent (forward) is the previous node of the segment
    F_END_NODE = 16,    // last chunk of the node's step
    F_END_ITEM = 32,    // last chunk of the work item (segment)
    F_ROOT = 64,        // forward root step
    F_PUB_X = 128       // forward: the node's x is published (tagged) as soon as it is known
};

struct Meta {
    int kind, node, aux, row0, nrows, flags, pad0, pad1;
};

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
__device__ __forceinline__ T v_dot(const typename V16<T>::type &g, const typename V16<T>::type &x);
template <>
__device__ __forceinline__ float v_dot<float>(const float4 &g, const float4 &x) {
    return fmaf(g.x, x.x, fmaf(g.y, x.y, fmaf(g.z, x.z, g.w * x.w)));
}
template <>
__device__ __forceinline__ double v_dot<double>(const double2 &g, const double2 &x) {
    return fma(g.x, x.x, g.y * x.y);
}

// Explicit shared-space loads (the ring and the small vectors live in shared memory; the
// pointers reach the consumer as generic pointers).
template <class T>
__device__ __forceinline__ typename V16<T>::type lds_vec(unsigned addr);
template <>
__device__ __forceinline__ float4 lds_vec<float>(unsigned addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
template <>
__device__ __forceinline__ double2 lds_vec<double>(unsigned addr) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr));
    return v;
}
template <class T>
__device__ __forceinline__ T lds_one(unsigned addr);
template <>
__device__ __forceinline__ float lds_one<float>(unsigned addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
template <>
__device__ __forceinline__ double lds_one<double>(unsigned addr) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(addr));
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- PTX: mbarrier, bulk copy, flags ------------------------------------------------------
__device__ __forceinline__ unsigned sm_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(sm_addr(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(sm_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for a phase; on expiry the error flag is raised and the wait gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, int *err) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        for (int it = 0; it < 64; ++it)
            if (mbar_try(b, parity)) return true;
        if (now_ns() - t0 > kWaitNs) break;
    }
    atomicExch(err, 2);
    return false;
}
// The node matrices are streamed once per round and do not fit in L2, so their bulk copies carry
// an evict-first L2 policy: they then displace the solver's vectors (read by the elementwise
// passes between rounds) as little as possible.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            sm_addr(dst)),
        "l"(src), "r"(bytes), "r"(sm_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait until *f == epoch, for at most `limit` ns (the handle's dependency-wait limit;
// 0 gives up at the first check that finds the flag unset).  Gives up without a new error when
// the error flag is already raised; the first cause recorded is kept.
__device__ __forceinline__ void wait_flag(const unsigned *f, unsigned epoch, int *err, unsigned long long limit) {
    if (ld_acquire(f) == epoch) return;
    const unsigned long long t0 = now_ns();
    while (now_ns() - t0 < limit) {
        for (int it = 0; it < 32; ++it) {
            if (ld_acquire(f) == epoch) return;
            __nanosleep(32);
        }
        if (*(volatile int *)err) return;
    }
    atomicCAS(err, 0, 1);
}
// Tagged hand-off of a vector between work items (a segment's last s in the backward pass, its
// last [x; u] in the forward pass).  Each 32 bits of a value travel as one 64-bit word
// {bits, epoch}, written with a relaxed store by the thread that computed the value and polled
// by the thread that needs it: a word carrying the round's epoch is that value (a 64-bit
// aligned access is single-copy atomic), so the writer needs no release fence and the reader no
// flag and no second load.  On the paper-scale tree the binary top stages form the round's
// serial path, and this hand-off is the largest part of each of their steps.
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Bounded poll of one tagged word, with the limits and the error reporting of wait_flag.
__device__ __forceinline__ unsigned poll_word(const unsigned long long *w, unsigned epoch, int *err,
                                              unsigned long long limit) {
    unsigned long long v = ld_relaxed_u64(w);
    if ((unsigned)(v >> 32) == epoch) return (unsigned)v;
    const unsigned long long t0 = now_ns();
    while (now_ns() - t0 < limit) {
        for (int it = 0; it < 32; ++it) {
            v = ld_relaxed_u64(w);
            if ((unsigned)(v >> 32) == epoch) return (unsigned)v;
            __nanosleep(32);
        }
        if (*(volatile int *)err) return (unsigned)v;
    }
    atomicCAS(err, 0, 1);
    return (unsigned)v;
}
template <class T>
struct Tagged;
template <>
struct Tagged<float> {
    static constexpr int W = 1;  // words per value
    __device__ static void put(unsigned long long *w, float v, unsigned epoch) {
        st_relaxed_u64(w, ((unsigned long long)epoch << 32) | __float_as_uint(v));
    }
    __device__ static float get(const unsigned long long *w, unsigned epoch, int *err, unsigned long long limit) {
        return __uint_as_float(poll_word(w, epoch, err, limit));
    }
};
template <>
struct Tagged<double> {
    static constexpr int W = 2;
    __device__ static void put(unsigned long long *w, double v, unsigned epoch) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        st_relaxed_u64(w, ((unsigned long long)epoch << 32) | (b & 0xffffffffull));
        st_relaxed_u64(w + 1, ((unsigned long long)epoch << 32) | (b >> 32));
    }
    __device__ static double get(const unsigned long long *w, unsigned epoch, int *err, unsigned long long limit) {
        const unsigned lo = poll_word(w, epoch, err, limit);
        const unsigned hi = poll_word(w + 1, epoch, err, limit);
        return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
    }
};

// Asynchronous element copies global -> shared (the small per-node vectors); the issuing thread
// waits for its own copies with cp_async_wait, a named barrier then publishes them.
template <int B>
__device__ __forceinline__ void cp_async_elem(void *dst, const void *src);
template <>
__device__ __forceinline__ void cp_async_elem<4>(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sm_addr(dst)), "l"(src) : "memory");
}
template <>
__device__ __forceinline__ void cp_async_elem<8>(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sm_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory"); }

template <class T>
struct TreeArgs {
    int nx, nu, ldg, ldk, ldr, ldrk, lda, Np, Nn, nxu;  // lda = max(ldg, ldrk): accumulator row width
    int Tb, Tf;
    const int *bstart, *bnodes, *fstart, *fnodes;
    const int *cbeg, *ccnt, *parent;
    const T *G, *RK, *Gt, *Kt, *gu, *gx, *c, *sqp, *pN;
    const double *prob;
    const T *y[kMaxRhs];
    T *h[kMaxRhs];
    const T *x0;
    T *ubar, *xs, *us;      // scratch, [kMaxRhs][Np][nu], [kMaxRhs][Nn][nx], [kMaxRhs][Np][nu] (xs, us may be null)
    unsigned long long *ts, *txs, *tus;  // tagged s, x, u of the segments' last nodes (Tagged<T>::W words per value)
    long long s_stride, u_stride;
    unsigned *flags;        // [2][Nn]: flags[0] = the root's backward step is done
    unsigned long long *ticket;
    int *err;
    unsigned long long wait_ns;  // limit of each dependency wait
    int homog, scaled;
    int rpcG, rpcRK, rpcGt, rpcKt;  // rows per ring slot
    const int *stop;                // a solver's stop flag (null: always run)
};

__device__ __forceinline__ long long dual_off(int i, int Np, int nxu, int nx) {
    return i < Np ? (long long)i * nxu : (long long)Np * nxu + (long long)(i - Np) * nx;
}

// ---- producer ----------------------------------------------------------------------------
template <class T>
struct Producer {
    const TreeArgs<T> &a;
    unsigned char *ring;
    Meta *meta;
    uint64_t *full, *empty;
    unsigned long long n = 0;

    uint64_t pol;  // L2 policy of the matrix copies

    __device__ Producer(const TreeArgs<T> &a_, unsigned char *r, Meta *m, uint64_t *f, uint64_t *e)
        : a(a_), ring(r), meta(m), full(f), empty(e), pol(evict_first_policy()) {}

    // false when a slot never came free (the error flag is then raised): stop issuing copies
    __device__ bool slot_acquire(int &slot) {
        slot = (int)(n % kSlots);
        const unsigned long long round = n / kSlots;
        if (round > 0) return mbar_wait(&empty[slot], (unsigned)((round - 1) & 1), a.err);
        return true;
    }
    bool dead = false;
    __device__ void emit(int kind, int node, int aux, int row0, int nrows, int flags, const T *src, int ld) {
        int slot;
        if (dead || !slot_acquire(slot)) {
            dead = true;
            return;
        }
        Meta md;
        md.kind = kind;
        md.node = node;
        md.aux = aux;
        md.row0 = row0;
        md.nrows = nrows;
        md.flags = flags;
        md.pad0 = md.pad1 = 0;
        meta[slot] = md;
        const unsigned bytes = (unsigned)(nrows * ld * sizeof(T));
        mbar_expect_tx(&full[slot], bytes);
        bulk_load(ring + (size_t)slot * kChunk, src + (size_t)row0 * ld, bytes, &full[slot], pol);
        ++n;
    }
    __device__ void emit_end() {
        int slot;
        if (dead || !slot_acquire(slot)) return;
        Meta md = {KIND_END, -1, -1, 0, 0, 0, 0, 0};
        meta[slot] = md;
        mbar_arrive(&full[slot]);
        ++n;
    }
    // the chunks of one matrix: rows [0, rows) in runs of rpc rows
    __device__ void matrix(int kind, int node, int aux, const T *base, int rows, int ld, int rpc, int flags_first,
                           int flags_last) {
        for (int r0 = 0; r0 < rows; r0 += rpc) {
            const int nr = min(rpc, rows - r0);
            int f = 0;
            if (r0 == 0) f |= F_FIRST | flags_first;
            if (r0 + nr == rows) f |= F_LAST | flags_last;
            emit(kind, node, aux, r0, nr, f, base);
        }
    }
    __device__ void emit(int kind, int node, int aux, int row0, int nrows, int flags, const T *base) {
        const int ld = kind == KIND_BG ? a.ldg : (kind == KIND_BP ? a.ldrk : (kind == KIND_FG ? a.ldk : a.ldr));
        emit(kind, node, aux, row0, nrows, flags, base, ld);
    }

    // phase 0: the backward items [0, Tb); phase 1: the forward items [Tb, Tb + Tf)
    __device__ void run(unsigned long long tbase, int phase) {
        const int nx = a.nx, nu = a.nu;
        const int total = phase == 0 ? a.Tb : a.Tf;
        if (a.stop && *(volatile const int *)a.stop) {
            // a look-ahead round of a solver that has stopped: no work, but the tickets of the
            // launch are drawn all the same (the host's count of the ticket counter stays right)
            if (blockIdx.x == 0) atomicAdd(a.ticket, (unsigned long long)(total + gridDim.x));
            emit_end();
            return;
        }
        for (;;) {
            if (dead) return;
            const unsigned long long tk = atomicAdd(a.ticket, 1ull) - tbase;
            if (tk >= (unsigned long long)total) break;
            const int item = (int)tk + (phase == 0 ? 0 : a.Tb);
            if (item < a.Tb) {
                const int b0 = a.bstart[item], b1 = a.bstart[item + 1];
                for (int k = b0; k < b1; ++k) {
                    const int i = a.bnodes[k];
                    const bool last_node = k == b1 - 1;
                    const int jb = k == b0 ? a.cbeg[i] : a.bnodes[k - 1];
                    const int je = k == b0 ? a.cbeg[i] + a.ccnt[i] : jb + 1;
                    for (int j = jb; j < je; ++j) {
                        int ff = (j == jb ? F_FIRST_CHILD : 0) | (k > b0 ? F_INSEG : 0);
                        matrix(KIND_BG, j, i, a.G + (size_t)j * nx * a.ldg, nx, a.ldg, a.rpcG, ff, 0);
                    }
                    matrix(KIND_BP, i, -1, a.RK + (size_t)i * nu * a.ldrk, nu, a.ldrk, a.rpcRK, 0,
                           F_END_NODE | (last_node ? F_END_ITEM : 0));
                }
            } else {
                const int it = item - a.Tb;
                const int f0 = a.fstart[it], f1 = a.fstart[it + 1];
                for (int k = f0; k < f1; ++k) {
                    const int j = a.fnodes[k];
                    const bool last_node = k == f1 - 1;
                    const int endf = F_END_NODE | (last_node ? F_END_ITEM : 0);
                    const bool nonleaf = j < a.Np;
                    // a segment's last nonleaf node hands x^j to its children before its K step
                    const int pubx = nonleaf && last_node ? F_PUB_X : 0;
                    if (j != 0)
                        matrix(KIND_FG, j, -1, a.Gt + (size_t)j * (nx + nu) * a.ldk, nx + nu, a.ldk, a.rpcGt,
                               k > f0 ? F_INSEG : 0, nonleaf ? pubx : endf);
                    if (nonleaf)
                        matrix(KIND_FK, j, -1, a.Kt + (size_t)j * nx * a.ldr, nx, a.ldr, a.rpcKt,
                               j == 0 ? F_ROOT | pubx : 0, endf);
                }
            }
        }
        emit_end();
    }
};

// ---- consumers ---------------------------------------------------------------------------
template <class T, int NR, int KV, int PH>
struct Consumer {
    using VT = typename V16<T>::type;
    static constexpr int VN = V16<T>::n;
    const TreeArgs<T> &a;
    unsigned char *ring;
    const Meta *meta;
    uint64_t *full, *empty;
    unsigned epoch;
    int warp, lane, tid;
    int *abort_flag;  // shared
    // shared vectors
    T *s_in, *s_out, *part, *accs, *v, *xu, *xj, *uj;
    T *pre;  // per-node vectors copied ahead of use (backward: y block, gu, gx; forward: c, ubar)

    // cp.async of n reals from src to pre + off, one element per thread and step
    __device__ void prefetch(int off, const T *src, int n) {
        for (int e = tid; e < n; e += kCW * 32) cp_async_elem<sizeof(T)>(pre + off + e, src + e);
    }
    T acc[NR][KV][VN];

    __device__ void zero_acc() {
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int q = 0; q < KV; ++q)
#pragma unroll
                for (int e = 0; e < VN; ++e) acc[k][q][e] = T(0);
    }
    // part[warp] <- acc over the first `width` columns; cbar; dst[k][c] = sum_w part[w][k][c]
    __device__ void reduce_acc(int width, T *dst, int dst_stride) {
        const int nvec = width / VN;
#pragma unroll
        for (int k = 0; k < NR; ++k)
#pragma unroll
            for (int q = 0; q < KV; ++q) {
                const int cv = lane + 32 * q;
                if (cv < nvec)
                    *reinterpret_cast<VT *>(part + ((size_t)warp * NR + k) * a.lda + cv * VN) =
                        *reinterpret_cast<const VT *>(acc[k][q]);
            }
        cbar();
        for (int e = tid; e < NR * width; e += kCW * 32) {
            const int k = e / width, c = e - k * width;
            T sum = T(0);
#pragma unroll
            for (int w = 0; w < kCW; ++w) sum += part[((size_t)w * NR + k) * a.lda + c];
            dst[k * dst_stride + c] = sum;
        }
        cbar();
    }
    // acc[k] += coef[k][row0 + r] * M[r][:] over the rows of the slot; RU rows per step so that
    // their shared-memory loads are in flight together
    __device__ void axpy_rows(const T *M, int ld, int nrows, const T *coef, int cstride, int row0) {
        const int nvec = ld / VN;
        constexpr int RU = KV <= 1 ? 4 : 2;  // rows in flight per warp (register budget of 3 CTAs/SM)
        const unsigned m_addr = sm_addr(M), c_addr = sm_addr(coef);
        for (int rb = warp; rb < nrows; rb += kCW * RU) {
            T cr[RU][NR];
            VT g[RU][KV];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int r = rb + u * kCW;
                const bool ok = r < nrows;
#pragma unroll
                for (int k = 0; k < NR; ++k)
                    cr[u][k] = ok ? lds_one<T>(c_addr + (unsigned)((k * cstride + row0 + r) * sizeof(T))) : T(0);
                const unsigned row = m_addr + (unsigned)((ok ? r : 0) * ld * sizeof(T));
#pragma unroll
                for (int q = 0; q < KV; ++q) {
                    const int cv = lane + 32 * q;
                    if (cv < nvec) g[u][q] = lds_vec<T>(row + (unsigned)(cv * 16));
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u)
#pragma unroll
                for (int q = 0; q < KV; ++q) {
                    const int cv = lane + 32 * q;
                    if (cv < nvec)
#pragma unroll
                        for (int k = 0; k < NR; ++k) v_fma<T>(cr[u][k], g[u][q], acc[k][q]);
                }
        }
    }
    __device__ void run() {
        const int nx = a.nx, nu = a.nu;
        unsigned long long n = 0;
        int upend = -1;  // forward: parent whose u^i this node's [x; u] still waits for
        zero_acc();
        for (;;) {
            const int slot = (int)(n % kSlots);
            // a copy that never lands leaves nothing sensible to do: every consumer warp leaves
            // the loop together (the decision is shared before anyone can reach a named barrier)
            if (!mbar_wait(&full[slot], (unsigned)((n / kSlots) & 1), a.err)) *abort_flag = 1;
            cbar();
            if (*(volatile int *)abort_flag) break;
            const Meta md = meta[slot];
            if (md.kind == KIND_END) break;
            const T *M = reinterpret_cast<const T *>(ring + (size_t)slot * kChunk);
            const int f = md.flags;
            if constexpr (PH == 0) {
            if (md.kind == KIND_BG) {
                // child md.node of parent md.aux: s of the child into s_in
                if (f & F_FIRST) {
                    const int j = md.node;
                    cbar();  // every warp is done with the previous s_in
                    if (f & F_FIRST_CHILD) {
                        zero_acc();
                        // node md.aux's y block [NR][nx+nu], gu, gx: consumed after its G chunks
                        const int i = md.aux;
                        for (int k = 0; k < NR; ++k) prefetch(k * a.nxu, a.y[k] + (long long)i * a.nxu, a.nxu);
                        if (!a.homog) {
                            prefetch(NR * a.nxu, a.gu + (size_t)i * nu, nu);
                            prefetch(NR * a.nxu + nu, a.gx + (size_t)i * nx, nx);
                        }
                        cp_async_commit();
                    }
                    if (f & F_INSEG) {
                        for (int e = tid; e < NR * nx; e += kCW * 32) s_in[e] = s_out[e];
                    } else if (j >= a.Np) {
                        const long long o = dual_off(j, a.Np, a.nxu, nx);
                        const T scj = a.scaled ? a.sqp[j] : T(1);
                        const T cj = a.homog ? T(0) : T(0.5 * a.prob[j]);
                        for (int e = tid; e < NR * nx; e += kCW * 32) {
                            const int k = e / nx, r = e - k * nx;
                            s_in[e] = T(0.5) * scj * a.y[k][o + r] + cj * a.pN[r];
                        }
                    } else {
                        for (int e = tid; e < NR * nx; e += kCW * 32) {
                            const int k = e / nx, r = e - k * nx;
                            s_in[e] = Tagged<T>::get(a.ts + (k * a.s_stride + (long long)j * nx + r) * Tagged<T>::W,
                                                     epoch, a.err, a.wait_ns);
                        }
                    }
                    cbar();
                }
                axpy_rows(M, a.ldg, md.nrows, s_in, nx, md.row0);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            } else if (md.kind == KIND_BP) {
                // parent step over RK^i = [-Rbar^-1 | K^i]: [ubar ; K'v] = RK' v (Rbar symmetric)
                const int i = md.node;
                if (f & F_FIRST) {
                    // all children done: accs = sum over warps, v = y_u/2 + acc_B + gu
                    cp_async_wait();
                    reduce_acc(a.ldg, accs, a.lda);
                    const T sci = a.scaled ? a.sqp[i] : T(1);
                    for (int e = tid; e < NR * nu; e += kCW * 32) {
                        const int k = e / nu, cc = e - k * nu;
                        v[e] = T(0.5) * sci * pre[k * a.nxu + nx + cc] + accs[k * a.lda + nx + cc] +
                               (a.homog ? T(0) : pre[NR * a.nxu + cc]);
                    }
                    zero_acc();
                    cbar();
                }
                axpy_rows(M, a.ldrk, md.nrows, v, nu, md.row0);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (f & F_LAST) {
                    // ubar = -Rbar^-1 v;  s^i = y_x/2 + acc_A + K'v + gx
                    reduce_acc(a.ldrk, xu, a.lda);  // xu is free during the backward pass
                    const T sci = a.scaled ? a.sqp[i] : T(1);
                    for (int e = tid; e < NR * nu; e += kCW * 32) {
                        const int k = e / nu, cc = e - k * nu;
                        a.ubar[k * a.u_stride + (long long)i * nu + cc] = xu[k * a.lda + cc];
                    }
                    for (int e = tid; e < NR * nx; e += kCW * 32) {
                        const int k = e / nx, cc = e - k * nx;
                        const T val = T(0.5) * sci * pre[k * a.nxu + cc] + accs[k * a.lda + cc] +
                                      xu[k * a.lda + a.ldr + cc] + (a.homog ? T(0) : pre[NR * a.nxu + nu + cc]);
                        s_out[e] = val;
                        if (f & F_END_ITEM)
                            Tagged<T>::put(a.ts + (k * a.s_stride + (long long)i * nx + cc) * Tagged<T>::W, val, epoch);
                    }
                    zero_acc();
                    cbar();
                    // the forward launch's root step starts from this flag; the named barrier above
                    // orders every consumer's stores before thread 0's release store (release is
                    // cumulative), so no separate fence is needed
                    if (i == 0 && tid == 0) st_release(a.flags, epoch);
                }
            }
            } else {
            if (md.kind == KIND_FG) {
                // x^j = G^j [x^i; u^i] + c^j, axpy form over the rows of G^j' (one row per input)
                const int j = md.node;
                if (f & F_FIRST) {
                    cbar();  // every warp is done with the previous xu / xj and pre
                    if (f & F_INSEG) {
                        // parent = previous node of the segment: [x; u] from xj, uj
                        for (int e = tid; e < NR * a.ldg; e += kCW * 32) {
                            const int k = e / a.ldg, cc = e - k * a.ldg;
                            xu[e] = cc < nx ? xj[k * a.ldk + cc] : (cc < nx + nu ? uj[k * a.ldr + cc - nx] : T(0));
                        }
                    } else {
                        // the parent's x^i now; its u^i (published after the parent's K step)
                        // only before the first chunk that reaches the u rows of G^j'
                        const int i = a.parent[j];
                        for (int e = tid; e < NR * a.ldg; e += kCW * 32) {
                            const int k = e / a.ldg, cc = e - k * a.ldg;
                            if (cc < nx)
                                xu[e] = Tagged<T>::get(a.txs + (k * a.s_stride + (long long)i * nx + cc) * Tagged<T>::W,
                                                       epoch, a.err, a.wait_ns);
                            else if (cc >= nx + nu)
                                xu[e] = T(0);
                        }
                        upend = i;
                    }
                    // c^j and ubar^j, consumed at the end of the node's G and K runs (ubar^j was
                    // written by the backward launch, which ended before this one started)
                    if (!a.homog) prefetch(0, a.c + (size_t)j * nx, nx);
                    if (j < a.Np)
                        for (int k = 0; k < NR; ++k)
                            prefetch(nx + k * nu, a.ubar + k * a.u_stride + (long long)j * nu, nu);
                    cp_async_commit();
                    cbar();
                }
                if (upend >= 0 && md.row0 + md.nrows > nx) {
                    for (int e = tid; e < NR * nu; e += kCW * 32) {
                        const int k = e / nu, cc = e - k * nu;
                        xu[k * a.ldg + nx + cc] =
                            Tagged<T>::get(a.tus + (k * a.u_stride + (long long)upend * nu + cc) * Tagged<T>::W, epoch,
                                           a.err, a.wait_ns);
                    }
                    upend = -1;
                    cbar();
                }
                axpy_rows(M, a.ldk, md.nrows, xu, a.ldg, md.row0);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (f & F_LAST) {
                    cp_async_wait();
                    reduce_acc(a.ldk, xj, a.ldk);  // the padding columns of G' are zero
                    if (!a.homog)
                        for (int e = tid; e < NR * nx; e += kCW * 32) {
                            const int k = e / nx, r = e - k * nx;
                            xj[k * a.ldk + r] += pre[r];
                        }
                    zero_acc();
                    cbar();
                    if (f & F_PUB_X)
                        for (int e = tid; e < NR * nx; e += kCW * 32) {
                            const int k = e / nx, r = e - k * nx;
                            Tagged<T>::put(a.txs + (k * a.s_stride + (long long)j * nx + r) * Tagged<T>::W,
                                           xj[k * a.ldk + r], epoch);
                        }
                }
                if (f & F_END_NODE) {  // leaf: no K step
                    const long long oj = dual_off(j, a.Np, a.nxu, nx);
                    const T scj = a.scaled ? a.sqp[j] : T(1);
                    for (int e = tid; e < NR * nx; e += kCW * 32) {
                        const int k = e / nx, r = e - k * nx;
                        const T val = xj[k * a.ldk + r];
                        a.h[k][oj + r] = scj * val;
                        if (a.xs) a.xs[k * a.s_stride + (long long)j * nx + r] = val;
                    }
                }
            } else if (md.kind == KIND_FK) {
                // u^j = K^j x^j + ubar^j, axpy form over the rows of K^j'
                const int j = md.node;
                if ((f & F_FIRST) && (f & F_ROOT)) {
                    if (tid == 0) wait_flag(a.flags + 0, epoch, a.err, a.wait_ns);  // backward pass finished
                    cbar();
                    for (int k = 0; k < NR; ++k) prefetch(nx + k * nu, a.ubar + k * a.u_stride, nu);
                    cp_async_commit();
                    for (int e = tid; e < NR * a.ldk; e += kCW * 32) {
                        const int r = e % a.ldk;
                        xj[e] = (r < nx && !a.homog) ? a.x0[r] : T(0);
                    }
                    cbar();
                    if (f & F_PUB_X)
                        for (int e = tid; e < NR * nx; e += kCW * 32) {
                            const int k = e / nx, r = e - k * nx;
                            Tagged<T>::put(a.txs + (k * a.s_stride + r) * Tagged<T>::W, xj[k * a.ldk + r], epoch);
                        }
                }
                axpy_rows(M, a.ldr, md.nrows, xj, a.ldk, md.row0);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (f & F_LAST) {
                    cp_async_wait();
                    reduce_acc(a.ldr, uj, a.ldr);
                    for (int e = tid; e < NR * nu; e += kCW * 32) {
                        const int k = e / nu, r = e - k * nu;
                        uj[k * a.ldr + r] += pre[nx + e];
                    }
                    zero_acc();
                    cbar();
                    const long long oj = dual_off(j, a.Np, a.nxu, nx);
                    const T scj = a.scaled ? a.sqp[j] : T(1);
                    for (int e = tid; e < NR * (nx + nu); e += kCW * 32) {
                        const int k = e / (nx + nu), r = e - k * (nx + nu);
                        const T val = r < nx ? xj[k * a.ldk + r] : uj[k * a.ldr + r - nx];
                        a.h[k][oj + r] = scj * val;
                        if (r < nx) {  // x^j was handed on after the G step
                            if (a.xs) a.xs[k * a.s_stride + (long long)j * nx + r] = val;
                        } else {
                            const long long o = k * a.u_stride + (long long)j * nu + r - nx;
                            if (a.us) a.us[o] = val;
                            if (f & F_END_ITEM) Tagged<T>::put(a.tus + o * Tagged<T>::W, val, epoch);
                        }
                    }
                    cbar();
                }
            }
            }
            ++n;
        }
    }
};

template <class T, int NR, int KV, int PH>
__global__ void __launch_bounds__(kThreadsT, kCtasPerSm) k_tree(TreeArgs<T> a, unsigned epoch, unsigned long long tbase) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int abort_flag;
    unsigned char *ring = smem;
    Meta *meta = reinterpret_cast<Meta *>(smem + kSlots * kChunk);
    uint64_t *full = reinterpret_cast<uint64_t *>(meta + kSlots);
    uint64_t *empty = full + kSlots;
    T *vec = reinterpret_cast<T *>(empty + kSlots);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == kCW) {
        if (lane == 0) {
            Producer<T> p(a, ring, meta, full, empty);
            p.run(tbase, PH);
        }
        return;
    }
    Consumer<T, NR, KV, PH> c{a, ring, meta, full, empty, epoch, warp, lane, (int)threadIdx.x, &abort_flag};
    const int nx = a.nx, nu = a.nu;
    // shared vectors (offsets multiple of 16 bytes: every width is padded to a 16-byte multiple)
    T *p = vec;
    c.s_in = p;
    p += NR * a.ldk;
    c.s_out = p;
    p += NR * a.ldk;
    c.part = p;
    p += kCW * NR * a.lda;
    c.accs = p;
    p += NR * a.lda;
    c.v = p;
    p += NR * a.ldr;
    c.xu = p;
    p += NR * a.lda;
    c.xj = p;
    p += NR * a.ldk;
    c.uj = p;
    p += NR * a.ldr;
    c.pre = p;
    (void)nx;
    (void)nu;
    c.run();
}

size_t tree_smem(int NR, int lda, int ldg, int ldk, int ldr, size_t esz) {
    // s_in, s_out, xj: NR ldk; part: kCW NR lda; accs, xu: NR lda; v, uj: NR ldr;
    // pre: NR (nx + nu) + nx + nu <= (NR + 1) ldg
    const size_t vec = (size_t)NR * (3 * ldk + (kCW + 2) * lda + 2 * ldr) + (size_t)(NR + 1) * ldg;
    return (size_t)kSlots * kChunk + kSlots * sizeof(Meta) + 2 * kSlots * sizeof(uint64_t) + vec * esz;
}

template <class T, int NR, int KV, int PH>
void launch_tree(stotree_t h, const TreeArgs<T> &a, unsigned epoch, unsigned long long tbase, int grid,
                 cudaStream_t st) {
    const size_t smem = tree_smem(NR, a.lda, a.ldg, a.ldk, a.ldr, sizeof(T));
    raise_smem_cap((const void *)k_tree<T, NR, KV, PH>, smem);
    k_tree<T, NR, KV, PH><<<grid, kThreadsT, smem, st>>>(a, epoch, tbase);
}

// One round: the backward launch, then the forward launch (each with a consumer loop for its own
// item kinds); the forward items of the same epoch start after the whole backward pass.
template <class T, int NR>
void launch_tree_kv(stotree_t h, const TreeArgs<T> &a, unsigned epoch, unsigned long long tbase, int grid,
                    cudaStream_t st) {
    const int kv = (a.lda / V16<T>::n + 31) / 32;
    const unsigned long long tb1 = tbase + (unsigned long long)(a.Tb + grid);  // phase 1's first ticket
    switch (kv) {
        case 1: launch_tree<T, NR, 1, 0>(h, a, epoch, tbase, grid, st); launch_tree<T, NR, 1, 1>(h, a, epoch, tb1, grid, st); break;
        case 2: launch_tree<T, NR, 2, 0>(h, a, epoch, tbase, grid, st); launch_tree<T, NR, 2, 1>(h, a, epoch, tb1, grid, st); break;
        case 3: launch_tree<T, NR, 3, 0>(h, a, epoch, tbase, grid, st); launch_tree<T, NR, 3, 1>(h, a, epoch, tb1, grid, st); break;
        default: launch_tree<T, NR, 4, 0>(h, a, epoch, tbase, grid, st); launch_tree<T, NR, 4, 1>(h, a, epoch, tb1, grid, st); break;
    }
}

// Raise the shared-memory caps of both passes' kernels and return the occupancy of one CTA.
template <class T, int NR, int KV>
cudaError_t tree_caps(size_t smem, int *per_sm) {
    raise_smem_cap((const void *)k_tree<T, NR, KV, 0>, smem);
    raise_smem_cap((const void *)k_tree<T, NR, KV, 1>, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_tree<T, NR, KV, 0>, kThreadsT, smem);
}

// CTAs of the persistent kernel: every CTA must be resident at once (items wait on earlier ones).
template <class T, int NR>
int tree_grid(const TreeArgs<T> &a) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = tree_smem(NR, a.lda, a.ldg, a.ldk, a.ldr, sizeof(T));
    const int kv = (a.lda / V16<T>::n + 31) / 32;
    cudaError_t e;
    switch (kv) {
        case 1: e = tree_caps<T, NR, 1>(smem, &per_sm); break;
        case 2: e = tree_caps<T, NR, 2>(smem, &per_sm); break;
        case 3: e = tree_caps<T, NR, 3>(smem, &per_sm); break;
        default: e = tree_caps<T, NR, 4>(smem, &per_sm); break;
    }
    if (e != cudaSuccess || per_sm < 1) return 0;
    return sms * (per_sm < kCtasPerSm ? per_sm : kCtasPerSm);
}

// Row widths and item counts of a round (the part of TreeArgs the grid and caps depend on).
template <class T>
void tree_dims(stotree_t h, TreeArgs<T> &a) {
    a.nx = h->nx;
    a.nu = h->nu;
    a.ldg = h->ldg;
    a.ldk = h->ldk;
    a.ldr = h->ldr;
    a.ldrk = h->ldrk;
    a.lda = h->ldrk > h->ldg ? h->ldrk : h->ldg;
}

template <class T>
sto_status prepare_impl(stotree_t h) {
    TreeArgs<T> a;
    tree_dims(h, a);
    if (h->grid_ctas[1] <= 0) h->grid_ctas[1] = tree_grid<T, 1>(a);
    if (h->grid_ctas[1] <= 0) {
        h->err = "solve kernel does not fit on this device";
        return STO_ERR_CUDA;
    }
    return STO_OK;
}

template <class T>
sto_status solve_impl(stotree_t h, const void *const *y, const void *x0, void *const *hx, int nrhs, bool homog,
                      bool scaled, cudaStream_t st, const SolveScratch *scratch, const int *stop) {
    const Layout &L = h->L;
    TreeArgs<T> a;
    tree_dims(h, a);
    a.Np = h->Np;
    a.Nn = h->Nn;
    a.nxu = h->nx + h->nu;
    a.Tb = (int)h->bstart.size() - 1;
    a.Tf = (int)h->fstart.size() - 1;
    a.bstart = h->at<int>(L.bstart);
    a.bnodes = h->at<int>(L.bnodes);
    a.fstart = h->at<int>(L.fstart);
    a.fnodes = h->at<int>(L.fnodes);
    a.cbeg = h->at<int>(L.cbeg);
    a.ccnt = h->at<int>(L.ccnt);
    a.parent = h->at<int>(L.parent);
    a.G = h->at<T>(L.G);
    a.Gt = h->at<T>(L.Gt);
    a.Kt = h->at<T>(L.Kt);
    a.RK = h->at<T>(L.RK);
    a.gu = h->at<T>(L.gu);
    a.gx = h->at<T>(L.gx);
    a.c = h->at<T>(L.c);
    a.sqp = h->at<T>(L.sqp);
    a.pN = h->at<T>(L.cost) + (2 * h->nx + h->nu) + h->nx + h->nu;  // ell = [q | r | pN]
    a.prob = h->at<double>(L.prob64);
    for (int k = 0; k < kMaxRhs; ++k) {
        a.y[k] = static_cast<const T *>(y[k < nrhs ? k : 0]);
        a.h[k] = static_cast<T *>(hx[k < nrhs ? k : 0]);
    }
    a.x0 = static_cast<const T *>(x0);
    a.s_stride = (long long)h->Nn * h->nx;
    a.u_stride = (long long)h->Np * h->nu;
    a.homog = homog ? 1 : 0;
    a.scaled = scaled ? 1 : 0;
    a.rpcG = kChunk / (h->ldg * (int)sizeof(T));
    a.rpcRK = kChunk / (h->ldrk * (int)sizeof(T));
    a.rpcGt = kChunk / (h->ldk * (int)sizeof(T));
    a.rpcKt = kChunk / (h->ldr * (int)sizeof(T));
    a.err = h->at<int>(L.fstatus) + 8;
    a.wait_ns = h->wait_ns;
    a.stop = stop;
    unsigned epoch;
    unsigned long long tbase;
    int &grid = h->grid_ctas[nrhs];
    if (grid <= 0) {
        switch (nrhs) {
            case 1: grid = tree_grid<T, 1>(a); break;
            case 2: grid = tree_grid<T, 2>(a); break;
            case 3: grid = tree_grid<T, 3>(a); break;
            default: grid = tree_grid<T, 4>(a); break;
        }
        if (grid <= 0) {
            h->err = "solve kernel does not fit on this device";
            return STO_ERR_CUDA;
        }
    }
    if (scratch) {  // caller scratch for one right-hand side: its flags and counter are cleared first
        a.ubar = static_cast<T *>(scratch->ubar);
        a.xs = a.us = nullptr;  // the trajectory is not kept
        a.ts = static_cast<unsigned long long *>(scratch->ts);
        a.txs = static_cast<unsigned long long *>(scratch->txs);
        a.tus = static_cast<unsigned long long *>(scratch->tus);
        a.flags = static_cast<unsigned *>(scratch->flags);
        a.ticket = static_cast<unsigned long long *>(scratch->ticket);
        STO_CUDA(h, cudaMemsetAsync(scratch->flags, 0, (size_t)2 * h->Nn * sizeof(unsigned), st));
        STO_CUDA(h, cudaMemsetAsync(scratch->ticket, 0, sizeof(unsigned long long), st));
        epoch = scratch->epoch;  // unique per call on the device: stale tagged words never match
        tbase = 0;
    } else {
        a.ubar = h->at<T>(L.ubar);
        a.xs = h->at<T>(L.xs);
        a.us = h->at<T>(L.us);
        a.ts = h->at<unsigned long long>(L.ts);
        a.txs = h->at<unsigned long long>(L.txs);
        a.tus = h->at<unsigned long long>(L.tus);
        a.flags = h->at<unsigned>(L.flags);
        a.ticket = h->at<unsigned long long>(L.ticket);
        if (h->epoch == 0xffffffffu) {  // epochs wrapped: start the flags and tagged words over
            STO_CUDA(h, cudaMemsetAsync(a.flags, 0, (size_t)2 * h->Nn * sizeof(unsigned), st));
            STO_CUDA(h, cudaMemsetAsync(h->ws + L.ts, 0, L.tus_end - L.ts, st));
            h->epoch = 0;
        }
        epoch = ++h->epoch;
        tbase = h->ticket_base;
        // every CTA's producer draws one ticket past the last item
        h->ticket_base += (unsigned long long)(a.Tb + a.Tf + 2 * grid);
    }
    // the scratch (no-allocation) path is never timed: timing may create events
    cudaEvent_t ev = nullptr;
    if (!scratch) timing_begin(h, st, &ev);
    switch (nrhs) {
        case 1: launch_tree_kv<T, 1>(h, a, epoch, tbase, grid, st); break;
        case 2: launch_tree_kv<T, 2>(h, a, epoch, tbase, grid, st); break;
        case 3: launch_tree_kv<T, 3>(h, a, epoch, tbase, grid, st); break;
        default: launch_tree_kv<T, 4>(h, a, epoch, tbase, grid, st); break;
    }
    timing_end(h, st, ev, nrhs);
    h->launches += 2;
    h->solve_calls += nrhs;
    STO_CUDA(h, cudaGetLastError());
    return STO_OK;
}

}  // namespace

sto_status prepare_round(stotree_t h) {
    return h->prec == STO_FP64 ? prepare_impl<double>(h) : prepare_impl<float>(h);
}

sto_status solve_round(stotree_t h, const void *const *y, const void *x0, void *const *hx, int nrhs, bool homog,
                       bool scaled, cudaStream_t st, const SolveScratch *scratch, void *const *pout, const int *stop) {
    if (scratch && nrhs != 1) return STO_ERR_INVALID_ARG;
    if (!h->fg)
        return h->prec == STO_FP64 ? solve_impl<double>(h, y, x0, hx, nrhs, homog, scaled, st, scratch, stop)
                                   : solve_impl<float>(h, y, x0, hx, nrhs, homog, scaled, st, scratch, stop);
    // general maps: H'y -> the round in the [x; u] layout -> Hx = H p
    if (scratch) {
        h->err = "the no-allocation solve step takes the selection maps only";
        return STO_ERR_INVALID_ARG;
    }
    const size_t spad = (size_t)((h->msel + 63) / 64 * 64) * h->esz;
    const void *ys[kMaxRhs];
    void *ps[kMaxRhs];
    for (int k = 0; k < nrhs; ++k) {
        void *ht = h->ws + h->L.ht + k * spad;
        const sto_status s = fg_ht(h, y[k], ht, false, st);
        if (s != STO_OK) return s;
        ys[k] = ht;
        ps[k] = pout ? pout[k] : h->ws + h->L.pv + k * spad;
    }
    const sto_status s = h->prec == STO_FP64 ? solve_impl<double>(h, ys, x0, ps, nrhs, homog, scaled, st, nullptr, stop)
                                             : solve_impl<float>(h, ys, x0, ps, nrhs, homog, scaled, st, nullptr, stop);
    if (s != STO_OK) return s;
    for (int k = 0; k < nrhs; ++k) {
        const sto_status e = fg_hx(h, ps[k], hx[k], st);
        if (e != STO_OK) return e;
    }
    return STO_OK;
}

}  // namespace sto

namespace sto {

// After a synchronising call: report a bounded device wait that expired (STO_ERR_TIMEOUT) and
// reset the round state it may have left inconsistent (flags, ticket counter, error flag).
sto_status check_round_error(stotree_t h, cudaStream_t st) {
    int err = 0;
    int *dev_err = h->at<int>(h->L.fstatus) + 8;
    STO_CUDA(h, cudaMemcpyAsync(&err, dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    if (err == 0) return STO_OK;
    STO_CUDA(h, cudaMemsetAsync(h->ws + h->L.flags, 0, (size_t)2 * h->Nn * sizeof(unsigned), st));
    STO_CUDA(h, cudaMemsetAsync(h->ws + h->L.ticket, 0, 64, st));
    STO_CUDA(h, cudaMemsetAsync(dev_err, 0, sizeof(int), st));
    STO_CUDA(h, cudaStreamSynchronize(st));
    h->ticket_base = 0;  // the epoch keeps counting: tagged words of the failed round never match again
    h->err = err == 1 ? "a solve round gave up waiting for a dependency" : "a solve round gave up waiting for a copy";
    return STO_ERR_TIMEOUT;
}

}  // namespace sto
