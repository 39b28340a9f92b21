// lbm_tau1_reduce_noalloc: the FP64 state reduction for callers that cannot
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: code that
// works from a fixed device arena it manages itself, or inside a framework
// whose allocator must account for every byte of device memory, and code
// that cannot afford the device-wide synchronisation that cudaMalloc and
// cudaFree may cause. This entry point runs the same two-pass reduction as
// lbm_tau1_reduce, on arrays the caller owns, with its per-block partial sums
// kept in a fixed-size static device array instead of handle memory.
//
// The array lives in every GPU that loads this library, from load until the
// process exits: LBM_TAU1_NOALLOC_MAX_BLOCKS rows of 8 doubles (64 KiB).
// Every call on a device shares it. Pass 1 overwrites each row that pass 2
// reads, so stale contents from an earlier call are never used and nothing
// needs clearing. Two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array and may return wrong
// sums.
#include <cstdio>
#include <mutex>

#include "kernels.h"
#include "lbm_tau1.h"

using namespace lbm;

namespace {

// Per-block partial sums of pass 1 (RED_FIELDS doubles per block).
static __device__ __align__(256) double g_noalloc_partials[LBM_TAU1_NOALLOC_MAX_BLOCKS * 8];

static_assert(RED_FIELDS == 8, "partial rows hold RED_FIELDS doubles");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of g_noalloc_partials, per device

thread_local char g_msg[256];

lbm_status noalloc_fail(lbm_status st, const char* what, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess)
        snprintf(g_msg, sizeof(g_msg), "reduce_noalloc: %s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    else
        snprintf(g_msg, sizeof(g_msg), "reduce_noalloc: %s", what);
    return st;
}

// Looks up, once per device and with that device current, the device address
// of the scratch array. In host code the name g_noalloc_partials is only a
// host-side stand-in, never a device address. The cached address belongs to
// the device's primary context: it does not survive cudaDeviceReset (the
// module, and with it the array, is loaded anew), so a process that resets a
// device must not call this entry point on that device afterwards.
lbm_status scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return noalloc_fail(LBM_ECUDA, "cudaGetSymbolAddress", e);
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_tau1_noalloc_last_error(void) { return g_msg; }

lbm_status lbm_tau1_reduce_noalloc(int32_t storage, int64_t n, const void* drho, const void* ux, const void* uy,
                                   const void* uz, const float* inv_scale, const uint8_t* solid, const double* g,
                                   double* out, void* cuda_stream)
{
    g_msg[0] = '\0';
    if (storage < LBM_F64 || storage > LBM_BF16S) return noalloc_fail(LBM_EINVAL, "bad storage");
    if (n < 1) return noalloc_fail(LBM_EINVAL, "n must be >= 1");
    if (n > LBM_TAU1_NOALLOC_MAX_NODES) return noalloc_fail(LBM_EINVAL, "n exceeds LBM_TAU1_NOALLOC_MAX_NODES");
    if (!drho || !ux || !uy || !uz || !solid || !g || !out) return noalloc_fail(LBM_EINVAL, "NULL argument");
    // reduce_blocks() never asks for more than LBM_TAU1_NOALLOC_MAX_BLOCKS rows
    // (it caps the block count); the check guards the array against a change there
    const int blocks = reduce_blocks(n);
    if (blocks > LBM_TAU1_NOALLOC_MAX_BLOCKS)
        return noalloc_fail(LBM_EINVAL, "n needs more partial rows than the static scratch holds");
    void* partials = nullptr;
    if (lbm_status st = scratch_address(&partials)) return st;
    const float one[4] = {1.f, 1.f, 1.f, 1.f};
    const void* fields[4] = {drho, ux, uy, uz};
    cudaError_t e = launch_reduce(storage, false, n, fields, inv_scale ? inv_scale : one, solid, g,
                                  static_cast<double*>(partials), out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, "kernel launch", e);
    return LBM_OK;
}

}  // extern "C"
