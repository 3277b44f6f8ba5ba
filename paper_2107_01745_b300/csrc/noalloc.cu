// stotree_solve_step_noalloc: the solve step (Algorithm 3/4, one right-hand side) with its
// per-call scratch in a fixed array compiled into the library instead of the caller's workspace.
//
// Who needs it: callers that cannot call cudaMalloc -- or any allocator -- when they run a
// solve, for example a controller whose device-memory plan is frozen after start-up, or code
// driven by a host framework that forbids allocation while it is issuing work.  Their handle
// is set up (workspace bound, data uploaded, factor computed) once; each call of this entry
// point then touches only the caller's y and Hx buffers, the factor arrays already in the
// workspace, and this file's static array.
//
// The array (kScratchBytes) lives on every GPU that loads the library until the process exits.
// Host code cannot use its name as a device address: the address is looked up once per
// device, with that device current, by cudaGetSymbolAddress, and passed to the kernels.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
unsigned g_epoch[kMaxDevices] = {};  // last epoch of a call on each device (the array starts zeroed)

// Device address of g_scratch on the current device (looked up on first use per device).
cudaError_t scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" STO_API sto_status stotree_solve_step_noalloc(stotree_t h, const void *y, const void *x0, void *hx,
                                                         int32_t homogeneous, int32_t scaled, sto_stream_t stream) {
    if (!h || !y || !hx) return STO_ERR_INVALID_ARG;
    if (!homogeneous && !x0) return STO_ERR_INVALID_ARG;
    // ubar [Np][nu] of one right-hand side; the tagged words (8 bytes per 4 bytes of a value) of
    // s [Nn][nx], x [Nn][nx] and u [Np][nu]; the round's dependency flags [2][Nn] and its
    // work-item counter
    const size_t bu = align256((size_t)h->Np * h->nu * h->esz);
    const size_t tx = align256((size_t)h->Nn * h->nx * 2 * h->esz);
    const size_t tu = align256((size_t)h->Np * h->nu * 2 * h->esz);
    const size_t bf = align256((size_t)2 * h->Nn * sizeof(unsigned));
    const size_t need = bu + 2 * tx + tu + bf + 256;
    if (need > kScratchBytes) {
        h->err = "stotree_solve_step_noalloc: the problem needs " + std::to_string(need) +
                 " bytes of scratch, more than the fixed " + std::to_string(kScratchBytes) + " bytes";
        return STO_ERR_INVALID_ARG;
    }
    if (!h->factored) return STO_ERR_NOT_READY;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return sto::cuda_fail(h, e, "cudaGetSymbolAddress(g_scratch)");
    char *b = static_cast<char *>(base);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // Every entry of ubar is written before it is read within one round.  A tagged word is read
    // only once it carries the round's epoch, and every call on a device gets an epoch of its
    // own, so words left by earlier calls (of any handle) never match; when the epochs wrap,
    // the tagged words are cleared.  The flags and the counter start at zero: the round clears
    // them (cudaMemsetAsync on the caller's stream, no allocation).
    unsigned epoch;
    {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return sto::cuda_fail(h, e, "cudaGetDevice");
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_epoch[dev] == 0xffffffffu) {
            e = cudaMemsetAsync(b + bu, 0, 2 * tx + tu, st);
            if (e != cudaSuccess) return sto::cuda_fail(h, e, "cudaMemsetAsync(tagged words)");
            g_epoch[dev] = 0;
        }
        epoch = ++g_epoch[dev];
    }
    sto::SolveScratch sc{b, b + bu, b + bu + tx, b + bu + 2 * tx, b + bu + 2 * tx + tu, b + bu + 2 * tx + tu + bf, epoch};
    const void *ys[1] = {y};
    void *hs[1] = {hx};
    return sto::solve_round(h, ys, x0, hs, 1, homogeneous != 0, scaled != 0, st, &sc);
}
