// ctx_id.h -- identity of the calling thread's current CUDA context, for host-side
// caches of per-context objects (device symbol addresses, memory pools) that must be
// looked up again after cudaDeviceReset, when the device's context is created afresh.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

namespace lbmace {

// cuCtxGetId of the current context: unique for the life of the process, so a context
// created after cudaDeviceReset gets a new one. The two driver functions come through
// the runtime, so the library does not link the driver library itself. False when no
// context is current or the driver lacks the functions.
inline bool current_ctx_id(unsigned long long* id)
{
    using CtxGetCurrentFn = CUresult (*)(CUcontext*);
    using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
    });
    if (!get_cur || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

} // namespace lbmace
