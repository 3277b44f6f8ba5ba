// Learned warm start: a per-node perceptron that predicts the scaled dual ybar^i of every node
// of a scenario tree (the variable the solvers iterate on, Section III-E), trained with Adam on
// solved draws.  The paper warm-starts from a few accelerated dual gradient steps (Section
// III-F); this predictor stands in for them when many problems share a tree and its dynamics.
//
// Every product runs on the 5th-generation tensor cores: C[128 x BN] tiles of A B' with A and B
// K-major BF16, staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a shared-memory ring
// guarded by mbarriers, multiplied by tcgen05.mma (kind::f16, FP32 accumulators in tensor memory)
// issued by one thread, and read back with tcgen05.ld by four epilogue warps that fuse bias,
// GELU, its derivative, the loss gradient and the BF16 transposed copies the next products
// need.  Weight gradients split the batch dimension over CTAs and are summed, in a fixed order,
// by the Adam kernel, so a training step is deterministic.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "internal.h"

struct stowarm_s;

namespace sto {
namespace {

constexpr int kBM = 128;     // rows of an output tile (one TMEM lane per row)
constexpr int kBK = 64;      // K per stage: one 128-byte swizzle atom of BF16
constexpr int kStages = 4;   // shared-memory ring depth
constexpr int kThreads = 256; // 8 warps: 2 per TMEM lane quarter in the epilogue
constexpr int kMaxBN = 64;   // column tile of the network's products (more CTAs for the epilogues)
constexpr int kSplitK = 256; // batch rows per CTA in the weight-gradient products
constexpr unsigned long long kMmaWaitNs = 1000000000ull;  // bounded waits: 1 s
constexpr float kGeluC = 0.7978845608028654f;            // sqrt(2/pi)
constexpr float kGeluA = 0.044715f;

// ------------------------------------------------------------------------------------------
// PTX wrappers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t *b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for a phase.  On expiry the CTA's abort flag and the caller's error word are set;
// later waits of the CTA return at once.
__device__ __forceinline__ bool mb_wait(uint64_t *b, unsigned parity, volatile int *abort_flag, int *err) {
    if (mb_try(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int it = 0; it < 32; ++it)
            if (mb_try(b, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kMmaWaitNs) break;
    }
    *abort_flag = 1;
    if (err) atomicExch(err, STO_ERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Shared-memory matrix descriptor of a K-major tile written by TMA with the 128-byte swizzle:
// rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), leading byte offset
// unused for this layout, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sw128_desc(const void *tile) {
    const uint64_t a = smem_u32(tile);
    return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives row (warp quarter * 32
// + t), columns col .. col + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float z) {
    return 0.5f * z * (1.f + tanhf(kGeluC * (z + kGeluA * z * z * z)));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
    const float th = tanhf(kGeluC * (z + kGeluA * z * z * z));
    return 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * kGeluC * (1.f + 3.f * kGeluA * z * z);
}

// ------------------------------------------------------------------------------------------
// The product kernel.  Grid: x = row tiles of 128, y = column tiles of BN, z = K splits of
// nk stages each.  Warp 0 lane 0 loads, warp 1 (all lanes) owns tensor memory and its lane 0
// issues the MMAs; all four warps run the epilogue on their 32 rows.
// ------------------------------------------------------------------------------------------
enum Epi { EPI_F32 = 0, EPI_GELU = 1, EPI_OUT = 2, EPI_DGELU = 3, EPI_PART = 4, EPI_PRED = 5 };

struct EpiArgs {
    int M, N;                     // valid rows / columns (EPI_F32)
    const float *bias;            // [N] (GELU, OUT, PRED)
    float *C;                     // FP32 output: EPI_F32 [M][ldc]; EPI_PART [split][.][ldc]; GELU: Z (or null); OUT: Y
    long long ldc, split_stride;
    __nv_bfloat16 *A;             // BF16 row-major copy (GELU: activation, OUT: dY, DGELU: dZ), may be null
    long long lda;
    __nv_bfloat16 *AT;            // BF16 transposed copy [col][ldat] (GELU: may be null)
    long long ldat;
    const float *Zin;             // DGELU: pre-activation, row-major [row][ldzin]
    long long ldzin;
    const float *T;               // OUT: targets [row][ldt]
    long long ldt;
    const int *nvalid;            // OUT / PRED: valid outputs per row
    const int *count;             // OUT: number of valid outputs in the batch
    float *loss_part;             // OUT: per (CTA, warp) sum of squared errors
    const long long *row_off;     // PRED: first dual entry of the row's node (or -1)
    const float *row_sq;          // PRED: sqrt(pi) of the row's node
    float *yout;                  // PRED: unscaled dual output
    int *err;
};

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int BN, int nk,
           unsigned tmem_cols, EpiArgs ep) {
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ float sbias[256];
    extern __shared__ uint8_t dsm_raw[];
    uint8_t *dsm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, ks0 = blockIdx.z * nk;
    const unsigned a_bytes = kBM * 128, b_bytes = (unsigned)BN * 128;
    const int nst = nk < kStages ? nk : kStages;
    uint8_t *sA = dsm;
    uint8_t *sB = dsm + nst * a_bytes;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], 1);
        }
        mb_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, tmem_cols);
    if (EPI == EPI_GELU || EPI == EPI_OUT || EPI == EPI_PRED)
        for (int i = threadIdx.x; i < BN; i += kThreads) sbias[i] = ep.bias[n0 + i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_slot;

    if (warp == 0 && lane == 0) {
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % nst, use = ks / nst;
            if (use > 0 && !mb_wait(&empty[s], (use - 1) & 1, &abort_flag, ep.err)) break;
            mb_expect_tx(&full[s], a_bytes + b_bytes);
            tma_load_2d(sA + s * a_bytes, &tmA, (ks0 + ks) * kBK, m0, &full[s]);
            tma_load_2d(sB + s * b_bytes, &tmB, (ks0 + ks) * kBK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(BN);
        for (int ks = 0; ks < nk; ++ks) {
            const int s = ks % nst, use = ks / nst;
            if (!mb_wait(&full[s], use & 1, &abort_flag, ep.err)) break;
            tc_fence_after();
            const uint64_t da = sw128_desc(sA + s * a_bytes), db = sw128_desc(sB + s * b_bytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)  // K = 16 per MMA: 32 bytes along the swizzled row
                mma_bf16(tbase, da + 2 * kk, db + 2 * kk, idesc, (ks | kk) != 0);
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = mb_wait(&done, 0, &abort_flag, ep.err);
    tc_fence_after();
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the (w / 4)-th half of the columns
    const int quarter = warp & 3, half = warp >> 2;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
    const int hc = (BN + 31) / 32 * 16;
    const int c_begin = half * hc, c_end = min(BN, (half + 1) * hc);
    float sq_err = 0.f;
    if (ok) {
        for (int c0 = c_begin; c0 < c_end; c0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            const int nb = n0 + c0;
            if (EPI == EPI_F32) {
                if (row < ep.M)
                    for (int j = 0; j < 16; ++j)
                        if (nb + j < ep.N) ep.C[(long long)row * ep.ldc + nb + j] = v[j];
            } else if (EPI == EPI_PART) {
                float *dst = ep.C + (long long)blockIdx.z * ep.split_stride + (long long)row * ep.ldc + nb;
#pragma unroll
                for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else if (EPI == EPI_GELU) {
                // Z and the transposed copy feed only the backward pass: null when predicting
                __align__(16) __nv_bfloat16 a[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float zz = v[j] + sbias[c0 + j];
                    v[j] = zz;
                    a[j] = __float2bfloat16_rn(gelu_f(zz));
                }
                if (ep.C) {
                    float *z = ep.C + (long long)row * ep.ldc + nb;
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4 *>(z + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
                uint4 *ad = reinterpret_cast<uint4 *>(ep.A + (long long)row * ep.lda + nb);
                ad[0] = reinterpret_cast<uint4 *>(a)[0];
                ad[1] = reinterpret_cast<uint4 *>(a)[1];
                if (ep.AT)
#pragma unroll
                    for (int j = 0; j < 16; ++j) ep.AT[(long long)(nb + j) * ep.ldat + row] = a[j];
            } else if (EPI == EPI_DGELU) {
                const float *z = ep.Zin + (long long)row * ep.ldzin + nb;
                __align__(16) __nv_bfloat16 d[16];
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const float4 zz = *reinterpret_cast<const float4 *>(z + j);
                    d[j] = __float2bfloat16_rn(v[j] * gelu_grad_f(zz.x));
                    d[j + 1] = __float2bfloat16_rn(v[j + 1] * gelu_grad_f(zz.y));
                    d[j + 2] = __float2bfloat16_rn(v[j + 2] * gelu_grad_f(zz.z));
                    d[j + 3] = __float2bfloat16_rn(v[j + 3] * gelu_grad_f(zz.w));
                }
                if (ep.A) {
                    uint4 *ad = reinterpret_cast<uint4 *>(ep.A + (long long)row * ep.lda + nb);
                    ad[0] = reinterpret_cast<uint4 *>(d)[0];
                    ad[1] = reinterpret_cast<uint4 *>(d)[1];
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) ep.AT[(long long)(nb + j) * ep.ldat + row] = d[j];
            } else if (EPI == EPI_OUT) {
                const int nv = ep.nvalid[row];
                const float scale = 2.f / (float)max(1, *ep.count);
                float *y = ep.C + (long long)row * ep.ldc + nb;
                __align__(16) __nv_bfloat16 d[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float yy = v[j] + sbias[c0 + j];
                    y[j] = yy;
                    const float diff = nb + j < nv ? yy - ep.T[(long long)row * ep.ldt + nb + j] : 0.f;
                    sq_err += diff * diff;
                    d[j] = __float2bfloat16_rn(scale * diff);
                }
                uint4 *ad = reinterpret_cast<uint4 *>(ep.A + (long long)row * ep.lda + nb);
                ad[0] = reinterpret_cast<uint4 *>(d)[0];
                ad[1] = reinterpret_cast<uint4 *>(d)[1];
#pragma unroll
                for (int j = 0; j < 16; ++j) ep.AT[(long long)(nb + j) * ep.ldat + row] = d[j];
            } else if (EPI == EPI_PRED) {
                const int nv = ep.nvalid[row];
                const long long off = ep.row_off[row];
                if (off >= 0) {
                    const float sq = ep.row_sq[row];
                    for (int j = 0; j < 16; ++j)
                        if (nb + j < nv) ep.yout[off + nb + j] = sq * (v[j] + sbias[c0 + j]);
                }
            }
        }
    }
    if (EPI == EPI_OUT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq_err += __shfl_xor_sync(0xffffffffu, sq_err, o);
        if (lane == 0) ep.loss_part[(blockIdx.x * gridDim.y + blockIdx.y) * 8 + warp] = sq_err;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_free(tbase, tmem_cols);
}

size_t umma_smem(int BN, int nk) {
    const int nst = nk < kStages ? nk : kStages;
    return (size_t)nst * (kBM * 128 + (size_t)BN * 128) + 1024;
}
unsigned tmem_cols_for(int BN) {
    unsigned c = 32;
    while ((int)c < BN) c <<= 1;
    return c;
}

// ------------------------------------------------------------------------------------------
// Tensor maps
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// BF16 matrix [rows][k_extent] with row stride ld (elements), boxes of 64 x box_rows; elements
// outside the extents read as zero.
bool make_map(CUtensorMap *m, const void *base, long long k_extent, long long rows, long long ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 8) || box_rows < 8 || box_rows > 256) return false;
    cuuint64_t dims[2] = {(cuuint64_t)k_extent, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Gemm {
    CUtensorMap a, b;
    int BN, nk;
    dim3 grid;
};

template <int EPI>
cudaError_t run_gemm(const Gemm &g, const EpiArgs &ep, cudaStream_t st) {
    cudaError_t e = raise_smem_cap((const void *)k_umma<EPI>, umma_smem(g.BN, g.nk));
    if (e != cudaSuccess) return e;
    const size_t sm = umma_smem(g.BN, g.nk);
    k_umma<EPI><<<g.grid, kThreads, sm, st>>>(g.a, g.b, g.BN, g.nk, tmem_cols_for(g.BN), ep);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Warm-start network state and the non-GEMM kernels
// ------------------------------------------------------------------------------------------
struct NodeInfo {
    int parent, stage, nvalid;
    int grand;        // parent's parent when both are below the root, else -1 (feature gather)
    long long doff;   // first dual entry of the node
    float sq;         // sqrt(pi)
    float pad2;
};

struct NetDev {
    int d_in, d_out, H, D0, DO, B, S;   // padded widths D0 (inputs), DO (outputs); S weight-gradient splits
    int nx, nu, Nn, horizon;
    long long m;
    float *W;          // FP32 master, padded: W1 [H][D0] | b1 [H] | W2 [H][H] | b2 [H] | W3 [DO][H] | b3 [DO]
    float *mom, *vel;  // Adam moments, same layout
    __nv_bfloat16 *W1b, *W2b, *W3b, *W2bT, *W3bT;
    __nv_bfloat16 *X, *XT;
    float *T;
    int *nvalid, *count, *tstep;
    double *adam_pow;  // beta1^t, beta2^t after t steps
    long long *row_off;
    float *row_sq;
    float *Z1, *Z2, *Y;
    __nv_bfloat16 *A1, *A1T, *A2, *A2T, *dY, *dYT, *dZ2, *dZ2T, *dZ1T;
    float *P1, *P2, *P3;   // weight-gradient partials [S][H][D0], [S][H][H], [S][H][DO]
    float *gbias;          // [DO | H | H]: bias gradients of layers 3, 2, 1
    float *loss_part;      // [B/128 * 8]: per (row tile, warp) of the output product
    const NodeInfo *nodes;
    long long *perm;       // per epoch: multiplier, offset
    int *err;
};

__host__ __device__ inline long long w1_off(const NetDev &) { return 0; }
__host__ __device__ inline long long b1_off(const NetDev &n) { return (long long)n.H * n.D0; }
__host__ __device__ inline long long w2_off(const NetDev &n) { return b1_off(n) + n.H; }
__host__ __device__ inline long long b2_off(const NetDev &n) { return w2_off(n) + (long long)n.H * n.H; }
__host__ __device__ inline long long w3_off(const NetDev &n) { return b2_off(n) + n.H; }
__host__ __device__ inline long long b3_off(const NetDev &n) { return w3_off(n) + (long long)n.DO * n.H; }
__host__ __device__ inline long long nparam_padded(const NetDev &n) { return b3_off(n) + n.DO; }

// Batch rows of (draw, node) samples: features, target and valid count; one warp per row, 16
// rows per block, the transposed copy (training only) staged in shared memory so both copies
// are written in contiguous runs.  mode 0: training sample from the permutation of the current
// epoch; mode 1: sample index base + b (prediction).  Past the end of the samples a row is
// zeros, nvalid 0.
constexpr int kGatherRows = 16;
__global__ void __launch_bounds__(256) k_gather(NetDev n, const float *x0, const float *c, const float *y,
                                                long long num_samples, long long base, long long steps_per_epoch,
                                                int t0, int mode, int draw0) {
    __shared__ __nv_bfloat16 tile[256][kGatherRows + 2];
    __shared__ int cnt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b0 = blockIdx.x * kGatherRows;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const long long st = mode == 0 ? (long long)(*n.tstep - t0) : 0;
    for (int rr = warp; rr < kGatherRows; rr += blockDim.x / 32) {
        const int b = b0 + rr;
        long long j = -1;
        if (mode == 0) {
            const long long e = st / steps_per_epoch, k = (st % steps_per_epoch) * n.B + b;
            j = (long long)(((unsigned long long)n.perm[2 * e] * (unsigned long long)k +
                             (unsigned long long)n.perm[2 * e + 1]) %
                            (unsigned long long)num_samples);
        } else if (base + b < num_samples) {
            j = base + b;
        }
        int nv = 0;
        long long off = -1;
        float sq = 1.f;
        if (j >= 0) {
            const long long d = j / n.Nn;
            const int i = (int)(j % n.Nn);
            const NodeInfo ni = n.nodes[i];
            nv = ni.nvalid;
            sq = ni.sq;
            off = (d - (mode == 1 ? draw0 : 0)) * n.m + ni.doff;
            const int anc1 = i > 0 ? ni.parent : -1;
            const int anc2 = ni.grand;  // stored, so no dependent load of the parent's record
            // features: x0 | t/N | c^i | c^anc | c^anc^2 (zeros for the root and missing ancestors)
            for (int f = lane; f < n.D0; f += 32) {
                float v = 0.f;
                if (f < n.nx) {
                    v = x0[d * n.nx + f];
                } else if (f == n.nx) {
                    v = (float)ni.stage / (float)n.horizon;
                } else if (f < n.d_in) {
                    const int a = (f - n.nx - 1) / n.nx, r = (f - n.nx - 1) % n.nx;
                    const int node = a == 0 ? i : (a == 1 ? anc1 : anc2);
                    if (node > 0) v = c[(d * n.Nn + node) * n.nx + r];
                }
                const __nv_bfloat16 bv = __float2bfloat16_rn(v);
                n.X[(long long)b * n.D0 + f] = bv;
                if (mode == 0) tile[f][rr] = bv;
            }
            if (y)
                for (int k = lane; k < n.DO; k += 32)
                    n.T[(long long)b * n.DO + k] = k < nv ? y[d * n.m + ni.doff + k] / ni.sq : 0.f;
        } else {
            for (int f = lane; f < n.D0; f += 32) {
                n.X[(long long)b * n.D0 + f] = __float2bfloat16_rn(0.f);
                if (mode == 0) tile[f][rr] = __float2bfloat16_rn(0.f);
            }
            for (int k = lane; k < n.DO; k += 32) n.T[(long long)b * n.DO + k] = 0.f;
        }
        if (lane == 0) {
            n.nvalid[b] = nv;
            n.row_off[b] = off;
            n.row_sq[b] = sq;
            atomicAdd(&cnt, nv);
        }
    }
    __syncthreads();
    // the transposed copy feeds only the first layer's weight gradient: training batches only
    if (mode == 0)
        for (int e = threadIdx.x; e < n.D0 * kGatherRows; e += blockDim.x) {
            const int f = e / kGatherRows, rr = e % kGatherRows;
            n.XT[(long long)f * n.B + b0 + rr] = tile[f][rr];
        }
    if (threadIdx.x == 0) atomicAdd(n.count, cnt);   // integer sums: order-independent
}

// Caller rows (FP32) into the padded BF16 batch.
__global__ void k_load_rows(NetDev n, const float *X, const float *T, const int *nvalid, int rows) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    if (b < n.B) {
        const bool in = b < rows;
        for (int f = 0; f < n.D0; ++f) {
            const __nv_bfloat16 v = __float2bfloat16_rn(in && f < n.d_in ? X[(long long)b * n.d_in + f] : 0.f);
            n.X[(long long)b * n.D0 + f] = v;
            n.XT[(long long)f * n.B + b] = v;
        }
        int nv = 0;
        if (in) nv = nvalid ? min(max(nvalid[b], 0), n.d_out) : n.d_out;
        for (int k = 0; k < n.DO; ++k)
            n.T[(long long)b * n.DO + k] = (T && in && k < n.d_out) ? T[(long long)b * n.d_out + k] : 0.f;
        n.nvalid[b] = nv;
        n.row_off[b] = in ? (long long)b * n.d_out : -1;
        n.row_sq[b] = 1.f;
        atomicAdd(&cnt, nv);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(n.count, cnt);
}

// Bias gradients: row sums (over the batch) of dY', dZ2', dZ1', one warp per row, fixed order.
__global__ void k_bias_grad(NetDev n) {
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int total = n.DO + 2 * n.H;
    if (r >= total) return;
    const __nv_bfloat16 *src = r < n.DO ? n.dYT + (long long)r * n.B
                                        : (r < n.DO + n.H ? n.dZ2T + (long long)(r - n.DO) * n.B
                                                          : n.dZ1T + (long long)(r - n.DO - n.H) * n.B);
    const uint4 *src4 = reinterpret_cast<const uint4 *>(src);   // B is a multiple of 256
    float s = 0.f;
#pragma unroll 8
    for (int q = lane; q < n.B / 8; q += 32) {
        const uint4 u = src4[q];
        const __nv_bfloat16 *hv = reinterpret_cast<const __nv_bfloat16 *>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) s += __bfloat162float(hv[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) n.gbias[r] = s;
}

// Gradient of padded parameter p: split partials summed in split order.
__device__ __forceinline__ float param_grad(const NetDev &n, long long p) {
    float g = 0.f;
    if (p < b1_off(n)) {
        const long long o = p / n.D0, i = p % n.D0;
        if (i < n.d_in)
            #pragma unroll 8
            for (int s = 0; s < n.S; ++s) g += n.P1[((long long)s * n.H + o) * n.D0 + i];
    } else if (p < w2_off(n)) {
        g = n.gbias[n.DO + n.H + (p - b1_off(n))];
    } else if (p < b2_off(n)) {
        const long long q = p - w2_off(n), o = q / n.H, i = q % n.H;
#pragma unroll 8
        for (int s = 0; s < n.S; ++s) g += n.P2[((long long)s * n.H + o) * n.H + i];
    } else if (p < w3_off(n)) {
        g = n.gbias[n.DO + (p - b2_off(n))];
    } else if (p < b3_off(n)) {
        const long long q = p - w3_off(n), o = q / n.H, i = q % n.H;
        if (o < n.d_out)
            for (int s = 0; s < n.S; ++s) g += n.P3[((long long)s * n.H + i) * n.DO + o];
    } else {
        const long long o = p - b3_off(n);
        if (o < n.d_out) g = n.gbias[o];
    }
    return g;
}

__device__ __forceinline__ void write_bf16_copies(const NetDev &n, long long p, float w) {
    const __nv_bfloat16 v = __float2bfloat16_rn(w);
    if (p < b1_off(n)) {
        n.W1b[p] = v;
    } else if (p >= w2_off(n) && p < b2_off(n)) {
        const long long q = p - w2_off(n), o = q / n.H, i = q % n.H;
        n.W2b[q] = v;
        n.W2bT[i * n.H + o] = v;
    } else if (p >= w3_off(n) && p < b3_off(n)) {
        const long long q = p - w3_off(n), o = q / n.H, i = q % n.H;
        n.W3b[q] = v;
        n.W3bT[i * n.DO + o] = v;
    }
}

// mode 0: gradient out (unpadded order, grad may be null), loss out; mode 1: Adam step.
__global__ void __launch_bounds__(256) k_adam(NetDev n, int mode, float lr, float *grad, float *loss,
                                              float *loss_hist, int t0) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = *n.tstep;
    if (blockIdx.x == 0 && (loss || loss_hist)) {
        // the loss partials (one per warp of the output-layer product) summed by the first block
        // in a fixed order: strided per thread, a shuffle tree per warp, the warps in order
        __shared__ float red[8];
        float s = 0.f;
        for (int k = threadIdx.x; k < (n.B / kBM) * 8; k += 256) s += n.loss_part[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.f;
            for (int w = 0; w < 8; ++w) tot += red[w];
            const float l = tot / (float)max(1, *n.count);
            if (loss) *loss = l;
            if (loss_hist) loss_hist[t - t0] = l;
        }
    }
    if (p >= nparam_padded(n)) return;
    const float g = param_grad(n, p);
    if (mode == 0) {
        if (!grad) return;
        // unpadded order: W1 [H][d_in] | b1 | W2 | b2 | W3 [d_out][H] | b3
        long long q = -1;
        if (p < b1_off(n)) {
            const long long o = p / n.D0, i = p % n.D0;
            if (i < n.d_in) q = o * n.d_in + i;
        } else if (p < w3_off(n)) {
            q = (long long)n.H * n.d_in + (p - b1_off(n));
        } else if (p < b3_off(n)) {
            const long long r = p - w3_off(n), o = r / n.H;
            if (o < n.d_out) q = (long long)n.H * n.d_in + 2LL * n.H + (long long)n.H * n.H + r;
        } else {
            const long long o = p - b3_off(n);
            if (o < n.d_out) q = (long long)n.H * n.d_in + 2LL * n.H + (long long)n.H * n.H + (long long)n.d_out * n.H + o;
        }
        if (q >= 0) grad[q] = g;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * n.mom[p] + (1.f - b1) * g;
    const float v = b2 * n.vel[p] + (1.f - b2) * g * g;
    n.mom[p] = m;
    n.vel[p] = v;
    // bias corrections 1 - beta^(t+1) from the running powers (no per-thread pow)
    const float c1 = (float)(1.0 - n.adam_pow[0] * 0.9), c2 = (float)(1.0 - n.adam_pow[1] * 0.999);
    const float w = n.W[p] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    n.W[p] = w;
    write_bf16_copies(n, p, w);
}

__global__ void k_refresh_bf16(NetDev n) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nparam_padded(n)) write_bf16_copies(n, p, n.W[p]);
}

__global__ void k_tick(NetDev n) {
    *n.tstep += 1;
    *n.count = 0;
    n.adam_pow[0] *= 0.9;
    n.adam_pow[1] *= 0.999;
}
__global__ void k_reset_step(NetDev n) {
    *n.tstep = 0;
    n.adam_pow[0] = 1.0;
    n.adam_pow[1] = 1.0;
}
__global__ void k_zero_count(NetDev n) { *n.count = 0; }

}  // namespace
}  // namespace sto

using namespace sto;

struct stowarm_s {
    int Nn = 0, horizon = 0, nx = 0, nu = 0, H = 0, B = 0;
    uint64_t seed = 0;
    long long m = 0;
    std::vector<NodeInfo> nodes;
    NetDev n{};
    uint8_t *ws = nullptr;
    size_t total = 0;
    std::vector<std::pair<size_t *, size_t>> layout;
    size_t o_W, o_mom, o_vel, o_W1b, o_W2b, o_W3b, o_W2bT, o_W3bT, o_X, o_XT, o_T, o_nv, o_cnt, o_t, o_roff, o_rsq,
        o_pow, o_Z1, o_Z2, o_Y, o_A1, o_A1T, o_A2, o_A2T, o_dY, o_dYT, o_dZ2, o_dZ2T, o_dZ1T, o_P1, o_P2, o_P3, o_gb, o_lp,
        o_nodes, o_perm, o_err;
    int max_epochs = 4096;
    Gemm g_l1, g_l2, g_l3, g_da2, g_da1, g_dw3, g_dw2, g_dw1;
    int draws = 0;
    const float *x0 = nullptr, *c = nullptr, *y = nullptr;
    long long tstep_host = 0;
    std::string err;
    // the backward pass's side branches (weight-gradient products) run on three streams of
    // their own, forked from and joined back into the caller's stream by events
    cudaStream_t side[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork[3] = {nullptr, nullptr, nullptr}, join[3] = {nullptr, nullptr, nullptr};
    ~stowarm_s() {
        for (int k = 0; k < 3; ++k) {
            if (side[k]) cudaStreamDestroy(side[k]);
            if (fork[k]) cudaEventDestroy(fork[k]);
            if (join[k]) cudaEventDestroy(join[k]);
        }
    }
};

namespace {

sto_status wfail(stowarm_t h, cudaError_t e, const char *what) {
    if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
    return STO_ERR_CUDA;
}
#define WCUDA(h, call)                                    \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return wfail(h, _e, #call); \
    } while (0)

long long rup(long long v, long long a) { return (v + a - 1) / a * a; }

void compute_layout(stowarm_t h) {
    NetDev &n = h->n;
    size_t off = 0;
    auto take = [&](size_t &o, size_t bytes) {
        o = off;
        off += (bytes + 1023) / 1024 * 1024;
    };
    const size_t P = (size_t)nparam_padded(n);
    const size_t B = n.B, H = n.H, D0 = n.D0, DO = n.DO, S = n.S;
    take(h->o_W, P * 4);
    take(h->o_mom, P * 4);
    take(h->o_vel, P * 4);
    take(h->o_W1b, H * D0 * 2);
    take(h->o_W2b, H * H * 2);
    take(h->o_W3b, DO * H * 2);
    take(h->o_W2bT, H * H * 2);
    take(h->o_W3bT, H * DO * 2);
    take(h->o_X, B * D0 * 2);
    take(h->o_XT, D0 * B * 2);
    take(h->o_T, B * DO * 4);
    take(h->o_nv, B * 4);
    take(h->o_cnt, 4);
    take(h->o_t, 4);
    take(h->o_pow, 16);
    take(h->o_roff, B * 8);
    take(h->o_rsq, B * 4);
    take(h->o_Z1, B * H * 4);
    take(h->o_Z2, B * H * 4);
    take(h->o_Y, B * DO * 4);
    take(h->o_A1, B * H * 2);
    take(h->o_A1T, H * B * 2);
    take(h->o_A2, B * H * 2);
    take(h->o_A2T, H * B * 2);
    take(h->o_dY, B * DO * 2);
    take(h->o_dYT, DO * B * 2);
    take(h->o_dZ2, B * H * 2);
    take(h->o_dZ2T, H * B * 2);
    take(h->o_dZ1T, H * B * 2);
    take(h->o_P1, S * H * D0 * 4);
    take(h->o_P2, S * H * H * 4);
    take(h->o_P3, S * H * DO * 4);
    take(h->o_gb, (DO + 2 * H) * 4);
    take(h->o_lp, (B / kBM) * 8 * 4);
    take(h->o_nodes, h->nodes.size() * sizeof(NodeInfo));
    take(h->o_perm, (size_t)h->max_epochs * 2 * 8);
    take(h->o_err, 4);
    h->total = off;
}

template <typename T>
T *at(stowarm_t h, size_t o) {
    return reinterpret_cast<T *>(h->ws + o);
}

bool setup_gemms(stowarm_t h) {
    NetDev &n = h->n;
    const int B = n.B, H = n.H, D0 = n.D0, DO = n.DO;
    bool ok = true;
    auto fwd = [&](Gemm &g, const void *A, int K, const void *W, int N) {
        g.BN = N < kMaxBN ? N : kMaxBN;
        ok = ok && make_map(&g.a, A, K, B, K, kBM) && make_map(&g.b, W, K, N, K, g.BN);
        g.nk = (K + kBK - 1) / kBK;
        g.grid = dim3(B / kBM, (N + g.BN - 1) / g.BN, 1);
    };
    fwd(h->g_l1, n.X, D0, n.W1b, H);
    fwd(h->g_l2, n.A1, H, n.W2b, H);
    fwd(h->g_l3, n.A2, H, n.W3b, DO);
    fwd(h->g_da2, n.dY, DO, n.W3bT, H);
    fwd(h->g_da1, n.dZ2, H, n.W2bT, H);
    auto wgrad = [&](Gemm &g, const void *AT, const void *BT, int N) {
        g.BN = N < kMaxBN ? N : kMaxBN;
        ok = ok && make_map(&g.a, AT, B, H, B, kBM) && make_map(&g.b, BT, B, N, B, g.BN);
        g.nk = kSplitK / kBK;
        g.grid = dim3(H / kBM, (N + g.BN - 1) / g.BN, n.S);
    };
    wgrad(h->g_dw3, n.A2T, n.dYT, DO);
    wgrad(h->g_dw2, n.dZ2T, n.A1T, H);
    wgrad(h->g_dw1, n.dZ1T, n.XT, D0);
    return ok;
}

EpiArgs epi0(stowarm_t h) {
    EpiArgs e;
    std::memset(&e, 0, sizeof(e));
    e.err = h->n.err;
    return e;
}

// Forward products; train: also the loss gradient and the backward products.
sto_status run_net(stowarm_t h, bool train, bool predict, float *yout, cudaStream_t st) {
    NetDev &n = h->n;
    EpiArgs e = epi0(h);
    // a prediction keeps only the BF16 activations the next layer reads
    e.bias = n.W + b1_off(n);
    e.C = predict ? nullptr : n.Z1;
    e.ldc = n.H;
    e.A = n.A1;
    e.lda = n.H;
    e.AT = predict ? nullptr : n.A1T;
    e.ldat = n.B;
    WCUDA(h, run_gemm<EPI_GELU>(h->g_l1, e, st));
    e.bias = n.W + b2_off(n);
    e.C = predict ? nullptr : n.Z2;
    e.A = n.A2;
    e.AT = predict ? nullptr : n.A2T;
    WCUDA(h, run_gemm<EPI_GELU>(h->g_l2, e, st));
    e = epi0(h);
    e.bias = n.W + b3_off(n);
    e.nvalid = n.nvalid;
    if (predict) {
        e.row_off = n.row_off;
        e.row_sq = n.row_sq;
        e.yout = yout;
        WCUDA(h, run_gemm<EPI_PRED>(h->g_l3, e, st));
        return STO_OK;
    }
    e.C = n.Y;
    e.ldc = n.DO;
    e.T = n.T;
    e.ldt = n.DO;
    e.count = n.count;
    e.loss_part = n.loss_part;
    e.A = n.dY;
    e.lda = n.DO;
    e.AT = n.dYT;
    e.ldat = n.B;
    WCUDA(h, run_gemm<EPI_OUT>(h->g_l3, e, st));
    if (!train) return STO_OK;
    // Backward.  The data products dZ2 -> dZ1 are the chain; each weight-gradient product only
    // needs the transposed copies of one layer, so it runs on a side stream as soon as they are
    // written (dW3 beside dZ2, dW2 beside dZ1, dW1 beside the bias gradients) and joins the
    // caller's stream before the optimiser step.  Each writes its own split-K partials, so the
    // step is the same as when they run one after another.
    for (int k = 0; k < 3; ++k) {
        if (!h->side[k]) WCUDA(h, cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking));
        if (!h->fork[k]) WCUDA(h, cudaEventCreateWithFlags(&h->fork[k], cudaEventDisableTiming));
        if (!h->join[k]) WCUDA(h, cudaEventCreateWithFlags(&h->join[k], cudaEventDisableTiming));
    }
    // dW3 = dY' A2 (dY' and A2' written by the output layer's epilogue)
    WCUDA(h, cudaEventRecord(h->fork[0], st));
    WCUDA(h, cudaStreamWaitEvent(h->side[0], h->fork[0], 0));
    EpiArgs w = epi0(h);
    w.C = n.P3;
    w.ldc = n.DO;
    w.split_stride = (long long)n.H * n.DO;
    WCUDA(h, run_gemm<EPI_PART>(h->g_dw3, w, h->side[0]));
    WCUDA(h, cudaEventRecord(h->join[0], h->side[0]));
    e = epi0(h);
    e.Zin = n.Z2;
    e.ldzin = n.H;
    e.A = n.dZ2;
    e.lda = n.H;
    e.AT = n.dZ2T;
    e.ldat = n.B;
    WCUDA(h, run_gemm<EPI_DGELU>(h->g_da2, e, st));
    // dW2 = dZ2' A1
    WCUDA(h, cudaEventRecord(h->fork[1], st));
    WCUDA(h, cudaStreamWaitEvent(h->side[1], h->fork[1], 0));
    w = epi0(h);
    w.C = n.P2;
    w.ldc = n.H;
    w.split_stride = (long long)n.H * n.H;
    WCUDA(h, run_gemm<EPI_PART>(h->g_dw2, w, h->side[1]));
    WCUDA(h, cudaEventRecord(h->join[1], h->side[1]));
    e.Zin = n.Z1;
    e.A = nullptr;
    e.AT = n.dZ1T;
    WCUDA(h, run_gemm<EPI_DGELU>(h->g_da1, e, st));
    // dW1 = dZ1' X
    WCUDA(h, cudaEventRecord(h->fork[2], st));
    WCUDA(h, cudaStreamWaitEvent(h->side[2], h->fork[2], 0));
    w = epi0(h);
    w.C = n.P1;
    w.ldc = n.D0;
    w.split_stride = (long long)n.H * n.D0;
    WCUDA(h, run_gemm<EPI_PART>(h->g_dw1, w, h->side[2]));
    WCUDA(h, cudaEventRecord(h->join[2], h->side[2]));
    const int rows = n.DO + 2 * n.H;
    k_bias_grad<<<(rows + 7) / 8, 256, 0, st>>>(n);
    WCUDA(h, cudaGetLastError());
    for (int k = 0; k < 3; ++k) WCUDA(h, cudaStreamWaitEvent(st, h->join[k], 0));
    return STO_OK;
}

sto_status check_err(stowarm_t h, cudaStream_t st) {
    int e = 0;
    WCUDA(h, cudaMemcpyAsync(&e, h->n.err, 4, cudaMemcpyDeviceToHost, st));
    WCUDA(h, cudaStreamSynchronize(st));
    if (e) {
        h->err = "a bounded wait in the tensor-core product expired";
        return STO_ERR_TIMEOUT;
    }
    return STO_OK;
}

int adam_blocks(const NetDev &n) { return (int)((nparam_padded(n) + 255) / 256); }

}  // namespace

extern "C" {

STO_API sto_status stowarm_create(const sto_warm_desc *d, stowarm_t *out) {
    if (!d || !out || !d->parent || !d->prob) return STO_ERR_INVALID_ARG;
    if (d->nx < 1 || d->nu < 1 || d->nx + d->nu > 256 || 4 * d->nx + 1 > 256 || d->num_nodes < 2 || d->horizon < 1)
        return STO_ERR_INVALID_ARG;
    if (d->hidden != 128 && d->hidden != 256) return STO_ERR_INVALID_ARG;  // whole 128-row tiles of W'
    if (d->batch < 256 || d->batch > 65536 || d->batch % kSplitK) return STO_ERR_INVALID_ARG;
    std::vector<int32_t> stage, ccnt, cbeg;
    if (validate_tree(d->parent, d->prob, d->num_nodes, d->horizon, stage, ccnt, cbeg) != STO_OK) return STO_ERR_TREE;
    stowarm_t h = new stowarm_s();
    h->Nn = d->num_nodes;
    h->horizon = d->horizon;
    h->nx = d->nx;
    h->nu = d->nu;
    h->H = d->hidden;
    h->B = d->batch;
    h->seed = d->seed;
    h->nodes.resize(h->Nn);
    long long off = 0;
    for (int i = 0; i < h->Nn; ++i) {
        NodeInfo &ni = h->nodes[i];
        ni.parent = d->parent[i];
        ni.stage = stage[i];
        ni.nvalid = ccnt[i] > 0 ? d->nx + d->nu : d->nx;
        const int par = d->parent[i];
        ni.grand = (i > 0 && par > 0) ? d->parent[par] : -1;
        ni.doff = off;
        ni.sq = (float)std::sqrt(d->prob[i]);
        ni.pad2 = 0.f;
        off += ni.nvalid;
    }
    h->m = off;
    NetDev &n = h->n;
    n.d_in = 4 * d->nx + 1;
    n.d_out = d->nx + d->nu;
    n.H = d->hidden;
    n.D0 = (int)rup(n.d_in, 16);
    n.DO = (int)rup(n.d_out, 16);
    n.B = d->batch;
    n.S = d->batch / kSplitK;
    n.nx = d->nx;
    n.nu = d->nu;
    n.Nn = d->num_nodes;
    n.horizon = d->horizon;
    n.m = h->m;
    compute_layout(h);
    *out = h;
    return STO_OK;
}

STO_API void stowarm_destroy(stowarm_t h) { delete h; }

STO_API sto_status stowarm_dims(stowarm_t h, int32_t *d_in, int32_t *d_out, int64_t *num_params) {
    if (!h) return STO_ERR_INVALID_ARG;
    const NetDev &n = h->n;
    if (d_in) *d_in = n.d_in;
    if (d_out) *d_out = n.d_out;
    if (num_params)
        *num_params = (int64_t)n.H * n.d_in + n.H + (int64_t)n.H * n.H + n.H + (int64_t)n.d_out * n.H + n.d_out;
    return STO_OK;
}

STO_API sto_status stowarm_workspace_size(stowarm_t h, size_t *bytes) {
    if (!h || !bytes) return STO_ERR_INVALID_ARG;
    *bytes = h->total;
    return STO_OK;
}

STO_API sto_status stowarm_set_params(stowarm_t h, const float *params, sto_stream_t stream);

STO_API sto_status stowarm_bind_workspace(stowarm_t h, void *dev_ptr, size_t bytes, sto_stream_t stream) {
    if (!h || !dev_ptr) return STO_ERR_INVALID_ARG;
    if (bytes < h->total) return STO_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 1023) return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    h->ws = static_cast<uint8_t *>(dev_ptr);
    NetDev &n = h->n;
    n.W = at<float>(h, h->o_W);
    n.mom = at<float>(h, h->o_mom);
    n.vel = at<float>(h, h->o_vel);
    n.W1b = at<__nv_bfloat16>(h, h->o_W1b);
    n.W2b = at<__nv_bfloat16>(h, h->o_W2b);
    n.W3b = at<__nv_bfloat16>(h, h->o_W3b);
    n.W2bT = at<__nv_bfloat16>(h, h->o_W2bT);
    n.W3bT = at<__nv_bfloat16>(h, h->o_W3bT);
    n.X = at<__nv_bfloat16>(h, h->o_X);
    n.XT = at<__nv_bfloat16>(h, h->o_XT);
    n.T = at<float>(h, h->o_T);
    n.nvalid = at<int>(h, h->o_nv);
    n.count = at<int>(h, h->o_cnt);
    n.tstep = at<int>(h, h->o_t);
    n.adam_pow = at<double>(h, h->o_pow);
    n.row_off = at<long long>(h, h->o_roff);
    n.row_sq = at<float>(h, h->o_rsq);
    n.Z1 = at<float>(h, h->o_Z1);
    n.Z2 = at<float>(h, h->o_Z2);
    n.Y = at<float>(h, h->o_Y);
    n.A1 = at<__nv_bfloat16>(h, h->o_A1);
    n.A1T = at<__nv_bfloat16>(h, h->o_A1T);
    n.A2 = at<__nv_bfloat16>(h, h->o_A2);
    n.A2T = at<__nv_bfloat16>(h, h->o_A2T);
    n.dY = at<__nv_bfloat16>(h, h->o_dY);
    n.dYT = at<__nv_bfloat16>(h, h->o_dYT);
    n.dZ2 = at<__nv_bfloat16>(h, h->o_dZ2);
    n.dZ2T = at<__nv_bfloat16>(h, h->o_dZ2T);
    n.dZ1T = at<__nv_bfloat16>(h, h->o_dZ1T);
    n.P1 = at<float>(h, h->o_P1);
    n.P2 = at<float>(h, h->o_P2);
    n.P3 = at<float>(h, h->o_P3);
    n.gbias = at<float>(h, h->o_gb);
    n.loss_part = at<float>(h, h->o_lp);
    n.nodes = at<NodeInfo>(h, h->o_nodes);
    n.perm = at<long long>(h, h->o_perm);
    n.err = at<int>(h, h->o_err);
    WCUDA(h, cudaMemsetAsync(h->ws, 0, h->total, st));
    WCUDA(h, cudaMemcpyAsync(h->ws + h->o_nodes, h->nodes.data(), h->nodes.size() * sizeof(NodeInfo),
                             cudaMemcpyHostToDevice, st));
    if (!setup_gemms(h)) {
        h->err = "tensor map encoding failed";
        return STO_ERR_CUDA;
    }
    // seeded initial weights, U(-1/sqrt(fan_in), 1/sqrt(fan_in)), in the unpadded order
    int32_t din, dout;
    int64_t np;
    stowarm_dims(h, &din, &dout, &np);
    std::vector<float> p((size_t)np);
    std::mt19937_64 rng(h->seed);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    size_t k = 0;
    auto fill = [&](long long count, int fan_in) {
        const double s = 1.0 / std::sqrt((double)fan_in);
        for (long long i = 0; i < count; ++i) p[k++] = (float)(s * u(rng));
    };
    fill((long long)n.H * din, din);
    fill(n.H, din);
    fill((long long)n.H * n.H, n.H);
    fill(n.H, n.H);
    fill((long long)dout * n.H, n.H);
    fill(dout, n.H);
    return stowarm_set_params(h, p.data(), stream);
}

STO_API sto_status stowarm_set_params(stowarm_t h, const float *params, sto_stream_t stream) {
    if (!h || !params) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const NetDev &n = h->n;
    std::vector<float> pad((size_t)nparam_padded(n), 0.f);
    size_t k = 0;
    for (int o = 0; o < n.H; ++o)
        for (int i = 0; i < n.d_in; ++i) pad[(size_t)(w1_off(n) + (long long)o * n.D0 + i)] = params[k++];
    for (int o = 0; o < n.H; ++o) pad[(size_t)(b1_off(n) + o)] = params[k++];
    for (long long q = 0; q < (long long)n.H * n.H; ++q) pad[(size_t)(w2_off(n) + q)] = params[k++];
    for (int o = 0; o < n.H; ++o) pad[(size_t)(b2_off(n) + o)] = params[k++];
    for (int o = 0; o < n.d_out; ++o)
        for (int i = 0; i < n.H; ++i) pad[(size_t)(w3_off(n) + (long long)o * n.H + i)] = params[k++];
    for (int o = 0; o < n.d_out; ++o) pad[(size_t)(b3_off(n) + o)] = params[k++];
    const size_t bytes = pad.size() * 4;
    WCUDA(h, cudaMemcpyAsync(n.W, pad.data(), bytes, cudaMemcpyHostToDevice, st));
    WCUDA(h, cudaMemsetAsync(n.mom, 0, bytes, st));
    WCUDA(h, cudaMemsetAsync(n.vel, 0, bytes, st));
    k_reset_step<<<1, 1, 0, st>>>(n);
    h->tstep_host = 0;
    k_refresh_bf16<<<adam_blocks(n), 256, 0, st>>>(n);
    WCUDA(h, cudaGetLastError());
    WCUDA(h, cudaStreamSynchronize(st));
    return STO_OK;
}

STO_API sto_status stowarm_get_params(stowarm_t h, float *params, sto_stream_t stream) {
    if (!h || !params) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const NetDev &n = h->n;
    std::vector<float> pad((size_t)nparam_padded(n));
    WCUDA(h, cudaMemcpyAsync(pad.data(), n.W, pad.size() * 4, cudaMemcpyDeviceToHost, st));
    WCUDA(h, cudaStreamSynchronize(st));
    size_t k = 0;
    for (int o = 0; o < n.H; ++o)
        for (int i = 0; i < n.d_in; ++i) params[k++] = pad[(size_t)(w1_off(n) + (long long)o * n.D0 + i)];
    for (int o = 0; o < n.H; ++o) params[k++] = pad[(size_t)(b1_off(n) + o)];
    for (long long q = 0; q < (long long)n.H * n.H; ++q) params[k++] = pad[(size_t)(w2_off(n) + q)];
    for (int o = 0; o < n.H; ++o) params[k++] = pad[(size_t)(b2_off(n) + o)];
    for (int o = 0; o < n.d_out; ++o)
        for (int i = 0; i < n.H; ++i) params[k++] = pad[(size_t)(w3_off(n) + (long long)o * n.H + i)];
    for (int o = 0; o < n.d_out; ++o) params[k++] = pad[(size_t)(b3_off(n) + o)];
    return STO_OK;
}

STO_API sto_status stowarm_forward(stowarm_t h, const float *X, int32_t rows, float *Y, sto_stream_t stream) {
    if (!h || !X || !Y || rows < 0 || rows > h->B) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NetDev &n = h->n;
    k_zero_count<<<1, 1, 0, st>>>(n);
    k_load_rows<<<(n.B + 255) / 256, 256, 0, st>>>(n, X, nullptr, nullptr, rows);
    WCUDA(h, cudaGetLastError());
    return run_net(h, false, true, Y, st);
}

STO_API sto_status stowarm_gradients(stowarm_t h, const float *X, const float *T, const int32_t *nvalid, int32_t rows,
                                     float *grad, float *loss, sto_stream_t stream) {
    if (!h || !X || !T || rows < 0 || rows > h->B) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NetDev &n = h->n;
    k_zero_count<<<1, 1, 0, st>>>(n);
    k_load_rows<<<(n.B + 255) / 256, 256, 0, st>>>(n, X, T, nvalid, rows);
    WCUDA(h, cudaGetLastError());
    sto_status s = run_net(h, true, false, nullptr, st);
    if (s != STO_OK) return s;
    k_adam<<<adam_blocks(n), 256, 0, st>>>(n, 0, 0.f, grad, loss, nullptr, 0);
    WCUDA(h, cudaGetLastError());
    return check_err(h, st);
}

STO_API sto_status stowarm_train_batch(stowarm_t h, const float *X, const float *T, const int32_t *nvalid,
                                       int32_t rows, float lr, sto_stream_t stream) {
    if (!h || !X || !T || rows < 0 || rows > h->B || !(lr > 0.f)) return STO_ERR_INVALID_ARG;
    if (!h->ws) return STO_ERR_NOT_READY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NetDev &n = h->n;
    k_zero_count<<<1, 1, 0, st>>>(n);
    k_load_rows<<<(n.B + 255) / 256, 256, 0, st>>>(n, X, T, nvalid, rows);
    WCUDA(h, cudaGetLastError());
    sto_status s = run_net(h, true, false, nullptr, st);
    if (s != STO_OK) return s;
    k_adam<<<adam_blocks(n), 256, 0, st>>>(n, 1, lr, nullptr, nullptr, nullptr, 0);
    k_tick<<<1, 1, 0, st>>>(n);
    WCUDA(h, cudaGetLastError());
    h->tstep_host += 1;
    return STO_OK;
}

STO_API sto_status stowarm_set_draws(stowarm_t h, int32_t num_draws, const float *x0, const float *c, const float *y) {
    if (!h || num_draws < 1 || !x0 || !c) return STO_ERR_INVALID_ARG;
    h->draws = num_draws;
    h->x0 = x0;
    h->c = c;
    h->y = y;
    return STO_OK;
}

STO_API sto_status stowarm_train(stowarm_t h, int32_t steps, float lr, uint64_t shuffle_seed, float *loss_hist,
                                 sto_stream_t stream) {
    if (!h || steps < 0 || !(lr > 0.f)) return STO_ERR_INVALID_ARG;
    if (!h->ws || !h->draws || !h->y) return STO_ERR_NOT_READY;
    if (steps == 0) return STO_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NetDev &n = h->n;
    const long long S = (long long)h->draws * h->Nn;
    const long long spe = S / n.B;
    if (spe < 1) return STO_ERR_INVALID_ARG;
    const long long epochs = (steps + spe - 1) / spe;
    if (epochs > h->max_epochs) return STO_ERR_INVALID_ARG;
    // per epoch an affine permutation k -> (a k + b) mod S with gcd(a, S) = 1
    std::mt19937_64 rng(shuffle_seed);
    std::vector<long long> perm(2 * epochs);
    for (long long e = 0; e < epochs; ++e) {
        long long a;
        do {
            a = (long long)(rng() % (unsigned long long)S);
        } while (a < 1 || std::gcd(a, S) != 1);
        perm[2 * e] = a;
        perm[2 * e + 1] = (long long)(rng() % (unsigned long long)S);
    }
    WCUDA(h, cudaMemcpyAsync(n.perm, perm.data(), perm.size() * 8, cudaMemcpyHostToDevice, st));
    k_zero_count<<<1, 1, 0, st>>>(n);
    const int t0 = (int)h->tstep_host;
    // one training step captured once, replayed `steps` times
    cudaStream_t cap;
    WCUDA(h, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    WCUDA(h, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    k_gather<<<n.B / kGatherRows, 256, 0, cap>>>(n, h->x0, h->c, h->y, S, 0, spe, t0, 0, 0);
    sto_status s = run_net(h, true, false, nullptr, cap);
    k_adam<<<adam_blocks(n), 256, 0, cap>>>(n, 1, lr, nullptr, nullptr, loss_hist, t0);
    k_tick<<<1, 1, 0, cap>>>(n);
    cudaGraph_t graph;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (s != STO_OK) return s;
    if (e != cudaSuccess) return wfail(h, e, "capture of a training step");
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return wfail(h, e, "cudaGraphInstantiate");
    for (int k = 0; k < steps; ++k) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) break;
    }
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return wfail(h, e, "cudaGraphLaunch");
    h->tstep_host += steps;
    return check_err(h, st);
}

STO_API sto_status stowarm_predict(stowarm_t h, int32_t draw0, int32_t num_draws, float *y_out, sto_stream_t stream) {
    if (!h || draw0 < 0 || num_draws < 1 || !y_out) return STO_ERR_INVALID_ARG;
    if (!h->ws || !h->draws) return STO_ERR_NOT_READY;
    if (draw0 + num_draws > h->draws) return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    NetDev &n = h->n;
    const long long first = (long long)draw0 * h->Nn, last = (long long)(draw0 + num_draws) * h->Nn;
    for (long long base = first; base < last; base += n.B) {
        k_zero_count<<<1, 1, 0, st>>>(n);
        k_gather<<<n.B / kGatherRows, 256, 0, st>>>(n, h->x0, h->c, nullptr, last, base, 1, 0, 1, draw0);
        WCUDA(h, cudaGetLastError());
        sto_status s = run_net(h, false, true, y_out, st);
        if (s != STO_OK) return s;
    }
    return STO_OK;
}

STO_API sto_status stowarm_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc,
                                     int32_t M, int32_t N, int32_t K, sto_stream_t stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N) return STO_ERR_INVALID_ARG;
    if ((lda % 8) || (ldb % 8) || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return STO_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Gemm g;
    g.BN = N >= 256 ? 256 : (int)rup(N, 16);
    g.nk = (K + kBK - 1) / kBK;
    g.grid = dim3((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + g.BN - 1) / g.BN), 1);
    if (!make_map(&g.a, A, K, M, lda, kBM) || !make_map(&g.b, B, K, N, ldb, g.BN)) return STO_ERR_CUDA;
    EpiArgs e;
    std::memset(&e, 0, sizeof(e));
    e.M = M;
    e.N = N;
    e.C = C;
    e.ldc = ldc;
    if (run_gemm<EPI_F32>(g, e, st) != cudaSuccess) return STO_ERR_CUDA;
    return STO_OK;
}

STO_API const char *stowarm_last_error(stowarm_t h) { return h ? h->err.c_str() : ""; }

}  // extern "C"
