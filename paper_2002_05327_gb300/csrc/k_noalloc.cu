// Subdomain solve without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a solve:
// code running where cudaMalloc is off limits or too slow (inside a custom
// allocator's callback, a real-time loop with a fixed memory budget, or a
// host that pre-reserves all device memory for itself).  For them,
// helm_subdomain_solve_noalloc works entirely inside memory that exists
// already: the caller's input and output buffers, the context's factors, and
// one file-scope scratch array below, which every GPU that loads this library
// holds from load until exit.
//
// The scratch holds the task descriptor (first 256 bytes) and the subdomain
// window buffer in the working precision.  Host code may not use the array's
// name as a device address (in host code it names a host-side stand-in), so
// the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and caches it.  That
// first call therefore does set-up work; make it before any stream capture.
// Every call reuses the same scratch and leaves its contents behind; each
// call overwrites everything it reads, so nothing needs clearing, but two
// calls whose GPU work overlaps (on different streams or contexts of the same
// device) race on the scratch.
#include <mutex>

#include "helm_internal.h"

namespace helm {

// 64 MiB: e.g. 123 complex128 right-hand sides (or 247 complex64) on a
// 184 x 184 window.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr size_t kNoAllocTaskBytes = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t noalloc_capacity_bytes() { return kNoAllocScratchBytes - kNoAllocTaskBytes; }

namespace {
std::mutex g_mu;
void* g_addr[128] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device and cached; after cudaDeviceReset the cached address is stale, so a
// process that resets a device must not call this entry point again).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}
}  // namespace

__global__ void noalloc_write_task(Task* dst, Task t) { *dst = t; }

template <typename T>
__global__ void noalloc_pack(const cplx<double>* __restrict__ src, cplx<T>* dst, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = ccast<T>(src[i]);
}

template <typename T>
__global__ void noalloc_unpack(const cplx<T>* __restrict__ src, cplx<double>* dst, int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = ccast<double>(src[i]);
}

template <typename T>
static cudaError_t run(const NoAllocArgs& a, void* scratch) {
    Task* task = static_cast<Task*>(scratch);
    cplx<T>* wb = reinterpret_cast<cplx<T>*>(static_cast<unsigned char*>(scratch) + kNoAllocTaskBytes);
    const int64_t count = (int64_t)a.nrhs * a.win_elems;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    noalloc_write_task<<<1, 1, 0, a.stream>>>(task, Task{0, a.sub, 0, 0, 0});
    noalloc_pack<T><<<blocks, 256, 0, a.stream>>>(a.R, wb, count);
    a.solve(a.ctx, task, a.nrhs, wb, a.win_elems);  // the context's own kernel choice, in place
    noalloc_unpack<T><<<blocks, 256, 0, a.stream>>>(wb, a.U, count);
    return cudaGetLastError();
}

cudaError_t noalloc_subdomain_solve(const NoAllocArgs& a) {
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return e;
    return a.f64 ? run<double>(a, scratch) : run<float>(a, scratch);
}

}  // namespace helm
