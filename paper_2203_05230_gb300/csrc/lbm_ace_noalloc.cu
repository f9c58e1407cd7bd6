// lbm_ace_noalloc.cu -- lbm_ace_mass_noalloc: the global-mass reduction for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already
// handed out by its own pool or caching allocator (a stray allocation would fail or
// fragment that budget), or a time-critical loop that cannot afford the implicit
// device synchronisation that cudaMalloc/cudaFree may bring. They still need the
// compensated global mass of a population field they hold in their own buffers.
//
// This variant of the mass reduction keeps its per-CTA partial sums in a fixed,
// file-scope array of static device memory instead of a buffer allocated per context.
// The array (LBM_ACE_NOALLOC_MAX_PARTIALS doubles, 32 KiB) exists on every GPU that
// loads the library, for as long as the library stays loaded. The entry point calls
// no cudaMalloc, cudaFree or other allocating routine.
#include "lbm_ace.h"
#include "ctx_id.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch: one partial sum per chunk of LBM_ACE_NOALLOC_CHUNK values.
static __device__ __align__(256) double g_mass_partials[LBM_ACE_NOALLOC_MAX_PARTIALS];

__device__ __forceinline__ void neumaier_add(double& s, double& c, double v)
{
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

// CTA b sums values [b * CHUNK, min((b + 1) * CHUNK, n)): each thread a fixed strided
// subset with compensation, then a fixed tree over the CTA. Writes partials[b].
template <typename T>
__global__ void __launch_bounds__(kThreads)
mass_chunks(const T* __restrict__ v, long long n, double* __restrict__ partials)
{
    __shared__ double sh[kThreads];
    const long long lo = (long long)blockIdx.x * LBM_ACE_NOALLOC_CHUNK;
    long long hi = lo + LBM_ACE_NOALLOC_CHUNK;
    if (hi > n) hi = n;
    double s = 0.0, c = 0.0;
    for (long long k = lo + threadIdx.x; k < hi; k += kThreads) neumaier_add(s, c, (double)v[k]);
    sh[threadIdx.x] = s + c;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// One warp: compensated sum of the first n partials in a fixed order into *out.
__global__ void mass_partials_final(const double* __restrict__ partials, int n, double* __restrict__ out)
{
    const int lane = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int k = lane; k < n; k += 32) neumaier_add(s, c, partials[k]);
    double S = 0.0, C = 0.0;
    for (int j = 0; j < 32; ++j) {
        neumaier_add(S, C, __shfl_sync(0xffffffffu, s, j));
        neumaier_add(S, C, __shfl_sync(0xffffffffu, c, j));
    }
    if (lane == 0) *out = S + C;
}

// Device address of the scratch array for the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up
// (cudaGetSymbolAddress, with the device current) at the first call on a device and
// again whenever that device's context has changed since (after cudaDeviceReset the
// module is loaded afresh and the array may sit elsewhere).
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};

cudaError_t scratch_for(int dev, double** out)
{
    unsigned long long id = 0;
    if (!lbmace::current_ctx_id(&id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev] || g_ctx[dev] != id) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_mass_partials);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<double*>(p);
        g_ctx[dev] = id;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

// True when p is memory the current device `dev` can address as device memory:
// device allocations of that device, or managed memory. Host memory (pageable or
// pinned) and other devices' allocations are refused before any launch. A range is
// checked at its first and last byte, which catches a count that runs past the end
// of an allocation into unmapped or host memory.
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError(); // the query's own error; nothing else was pending
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

} // namespace

extern "C" int lbm_ace_mass_noalloc(const void* values, int precision, long long count, double* out,
                                    void* stream)
{
    if (!out) return LBM_ACE_EINVAL;
    if (count < 0 || count > LBM_ACE_NOALLOC_MAX_COUNT) return LBM_ACE_EINVAL;
    if (count > 0 && !values) return LBM_ACE_EINVAL;
    if (precision != LBM_ACE_F64 && precision != LBM_ACE_F32) return LBM_ACE_EINVAL;
    // an error left by an earlier call of the caller's stays theirs: no launch, and it
    // is neither reported as this call's own nor cleared
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ACE_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ACE_ECUDA;
    const size_t bytes = (size_t)count * (precision == LBM_ACE_F64 ? sizeof(double) : sizeof(float));
    if (!on_device(out, dev) || !on_device(reinterpret_cast<const char*>(out) + sizeof(double) - 1, dev))
        return LBM_ACE_EINVAL;
    if (count > 0 && (!on_device(values, dev) || !on_device(static_cast<const char*>(values) + bytes - 1, dev)))
        return LBM_ACE_EINVAL;
    double* partials = nullptr;
    if (scratch_for(dev, &partials) != cudaSuccess) return LBM_ACE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int chunks = (int)((count + LBM_ACE_NOALLOC_CHUNK - 1) / LBM_ACE_NOALLOC_CHUNK);
    if (chunks > 0) {
        if (precision == LBM_ACE_F64)
            mass_chunks<double><<<chunks, kThreads, 0, s>>>(static_cast<const double*>(values), count, partials);
        else
            mass_chunks<float><<<chunks, kThreads, 0, s>>>(static_cast<const float*>(values), count, partials);
        if (cudaPeekAtLastError() != cudaSuccess) return LBM_ACE_ECUDA;
    }
    mass_partials_final<<<1, 32, 0, s>>>(partials, chunks, out);
    return cudaPeekAtLastError() == cudaSuccess ? LBM_ACE_OK : LBM_ACE_ECUDA;
}
