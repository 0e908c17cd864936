// lbm_step_noalloc_f32: one two-pass FP32 step that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being captured
// on a stream that forbids new allocations, applications that hand all device memory to
// their own pool or arena up front, or embedded hosts whose allocator must not be entered
// from the solver.  For them this entry point takes the populations in and out as caller
// memory and keeps its only scratch buffer -- the pseudopotential field read by the
// collide pass -- in a file-scope device array of fixed size.  Every device that loads the
// library holds that array (LBM_NOALLOC_MAX_NODES floats) until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "k_twopass.cuh"

namespace lbm {
lbm_status kparams_for(const lbm_params *p, int64_t pitch, KParams *out);
lbm_status set_global_error(lbm_status s, const std::string &msg);
}  // namespace lbm

using namespace lbm;

// psi scratch of the allocation-free step, shared by every call on a device.
static __device__ __align__(256) float g_noalloc_psi[LBM_NOALLOC_MAX_NODES];

// Device address of g_noalloc_psi (host code cannot use the symbol's name as a device
// address), looked up with the device current and cached per device together with the ID
// of the context it belongs to: a reset device (cudaDeviceReset) or another context made
// current gets a new ID, and the next call looks the address up again in that context.
struct NoallocSlot {
    unsigned long long ctx_id;
    float *addr;
};
static std::mutex g_noalloc_mutex;
static NoallocSlot g_noalloc_slot[256];

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// ID of the calling thread's current context (0: none is current); driver entry points are
// fetched through the runtime, so the library needs no link to the driver library.
static lbm_status current_context_id(unsigned long long *id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess || !a || !b || qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess)
            return set_global_error(LBM_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
        get_current = reinterpret_cast<PfnCtxGetCurrent>(a);
        get_id = reinterpret_cast<PfnCtxGetId>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return set_global_error(LBM_ECUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return set_global_error(LBM_ECUDA, "cuCtxGetId failed");
    return LBM_OK;
}

static lbm_status noalloc_scratch(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_global_error(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return set_global_error(LBM_ENOTSUP, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long ctx = 0;
    lbm_status s = current_context_id(&ctx);
    if (s != LBM_OK) return s;
    NoallocSlot &slot = g_noalloc_slot[dev];
    if (ctx == 0 || ctx != slot.ctx_id || !slot.addr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_psi);
        if (e != cudaSuccess)
            return set_global_error(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        // the look-up made the device's primary context current if none was
        if ((s = current_context_id(&ctx)) != LBM_OK) return s;
        slot.ctx_id = ctx;
        slot.addr = static_cast<float *>(ptr);
    }
    *out = slot.addr;
    return LBM_OK;
}

extern "C" lbm_status lbm_step_noalloc_f32(const lbm_params *p, const float *src, float *dst, int64_t pitch,
                                           void *cuda_stream)
{
    if (!p || !src || !dst) return set_global_error(LBM_EINVAL, "null argument");
    if (src == dst) return set_global_error(LBM_EINVAL, "src and dst must be different buffers");
    if (p->struct_size != (int32_t)sizeof(lbm_params))
        return set_global_error(LBM_EINVAL, "lbm_params.struct_size does not match this library");
    if (p->precision != LBM_F32) return set_global_error(LBM_ENOTSUP, "lbm_step_noalloc_f32 needs precision LBM_F32");
    if (p->force_mode == LBM_FORCE_FIELD)
        return set_global_error(LBM_ENOTSUP, "lbm_step_noalloc_f32 takes no force field (use CONST or BUOYANT)");
    if (p->nx < 1 || p->ny < 1) return set_global_error(LBM_EINVAL, "nx and ny must be >= 1");
    if ((int64_t)p->nx * p->ny > (int64_t)LBM_NOALLOC_MAX_NODES)
        return set_global_error(LBM_EINVAL, "lattice larger than LBM_NOALLOC_MAX_NODES (" +
                                                std::to_string((long long)LBM_NOALLOC_MAX_NODES) + " nodes)");
    if (p->ny > 65535) return set_global_error(LBM_EINVAL, "ny must be <= 65535 (one grid row of blocks per lattice row)");
    if (pitch < p->nx) return set_global_error(LBM_EINVAL, "pitch must be >= nx");
    KParams kp{};
    lbm_status s = kparams_for(p, pitch, &kp);
    if (s != LBM_OK) return s;
    float *psi = nullptr;
    if ((s = noalloc_scratch(&psi)) != LBM_OK) return s;
    kp.src = src;
    kp.dst = dst;
    kp.psi = psi;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = TwoPass<float>::psi_pass(kp, st);
    if (e == cudaSuccess) e = TwoPass<float>::collide_pass(kp, st);
    if (e != cudaSuccess) return set_global_error(LBM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}
