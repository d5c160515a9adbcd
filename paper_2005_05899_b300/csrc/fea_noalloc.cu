// Allocation-free RK stage entry point.
//
// Callers that run under a fixed device-memory budget (a pre-reserved pool,
// an embedding that forbids further cudaMalloc/cudaFree once set up) cannot
// let the library allocate per call.  fea_rk_stage_noalloc keeps its
// per-call scratch -- the intermediate FP64 right-hand side and the FP32
// packed copy of the stage velocity and pressure -- in one file-scope device
// array of fixed size.  The array belongs to this file's device module, which
// CUDA loads lazily; fea_create looks up its address on the context's
// device, so the module is loaded and the array reserved at set-up, and held
// until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "fea_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)FEA_NOALLOC_MAX_NODES * (3 * sizeof(double) + sizeof(float4));

// Shared by every call on a device: the last call's contents stay here.
static __device__ __align__(256) unsigned char g_stage_scratch[kScratchBytes];

// Device address of g_stage_scratch per device ordinal.  In host code the
// symbol itself is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
void *g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

}  // namespace

cudaError_t fea::noalloc_scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[device]) {
        int prev = 0;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stage_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        g_scratch_dev[device] = p;
    }
    *out = g_scratch_dev[device];
    return cudaSuccess;
}

extern "C" fea_status fea_rk_stage_noalloc(fea_ctx *ctx, int32_t mesh, int32_t stage, double dt, fea_prec prec,
                                           fea_closure closure, double nu, double c_vreman, const double *un,
                                           const double *uk, const double *p, double *uk_out, void *stream) {
    if (!ctx) return FEA_EINVAL;
    const int device = fea::context_device(ctx);
    if (device < 0 || device >= kMaxDevices) return fea::context_fail(ctx, FEA_EINVAL, "device ordinal out of range");
    void *base = nullptr;
    cudaError_t e = fea::noalloc_scratch_address(device, &base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fea::context_fail(ctx, FEA_ECUDA, cudaGetErrorString(e));
    }
    double *rhs = static_cast<double *>(base);
    float4 *up = reinterpret_cast<float4 *>(static_cast<unsigned char *>(base) +
                                            (size_t)FEA_NOALLOC_MAX_NODES * 3 * sizeof(double));
    return fea::stage_with_scratch(ctx, mesh, stage, dt, prec, closure, nu, c_vreman, un, uk, p, uk_out, rhs, up,
                                   FEA_NOALLOC_MAX_NODES, (cudaStream_t)stream);
}
