// Element energies, sensitivities and compliance without any device
// allocation by the library.
//
// Every other entry point works on a context whose buffers to3d_create
// allocates with cudaMalloc.  Some callers cannot allow that: programs that
// hand all device memory to their own pool or arena up front (a cudaMalloc
// from the library would sit outside that budget and may fail once the pool
// has reserved the device), and latency-critical loops that must never enter
// the driver's allocator (cudaMalloc and cudaFree can synchronise the device
// and take an unbounded time).  For them to3d_sensitivity_noalloc computes
// what to3d_sensitivity computes from caller-owned device buffers, and keeps
// the only scratch it needs -- the per-block partial sums of the grid-wide
// compliance reduction, its arrival counter and the result slot -- in one
// fixed array that lives in this library's device image.
#include <mutex>

#include "internal.cuh"

namespace to3d {

// Largest grid the scratch serves: one partial sum per block of 256 elements.
constexpr int kNoAllocMaxBlocks = 32768;
constexpr long long kNoAllocMaxElements = (long long)kNoAllocMaxBlocks * kElementThreads;
constexpr size_t kNoAllocPartialBytes = sizeof(double) * kNoAllocMaxBlocks;
constexpr size_t kNoAllocScratchBytes = kNoAllocPartialBytes + 256;   // + counter, result

// 256 KiB + 256 B, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device (it stays
// valid while the device's primary context lives; a device reset in the same
// process makes it stale, which the header documents).  In host
// code the symbol g_noalloc_scratch is only a host-side stand-in: handing it
// to a kernel would fault (or, where the GPU can reach host memory, silently
// use the wrong memory), so the real address comes from
// cudaGetSymbolAddress with that device current.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {};

static cudaError_t noalloc_scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace to3d

using namespace to3d;

extern "C" to3d_status to3d_sensitivity_noalloc(int32_t nelx, int32_t nely, int32_t nelz,
                                                double penal, double E0, double Emin, double nu,
                                                const double* x, const double* u, double* ce,
                                                double* dc, double* compliance, void* stream) {
    if (nelx < 1 || nely < 1 || nelz < 1 || !x || !u || !ce || !dc || !compliance)
        return TO3D_EINVAL;
    const long long nel = (long long)nelx * nely * nelz;
    if (nel > kNoAllocMaxElements) return TO3D_EINVAL;   // beyond the fixed scratch
    if (!(penal >= 1) || !(E0 > 0) || !(Emin > 0) || !(nu > -1) || !(nu < 0.5)) return TO3D_EINVAL;
    KE64 ke;
    if (!unit_ke(nu, &ke)) return TO3D_EINVAL;
    Grid g;
    g.nelx = nelx; g.nely = nely; g.nelz = nelz;
    g.nx = nelx + 1; g.ny = nely + 1; g.nz = nelz + 1;
    g.nel = nel;
    g.nnode = (long long)g.nx * g.ny * g.nz;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TO3D_ECUDA;
    unsigned char* scratch = nullptr;
    if (noalloc_scratch_address(dev, &scratch) != cudaSuccess) return TO3D_ECUDA;
    Reducer red;
    red.partials = (double*)scratch;
    red.counter = (unsigned int*)(scratch + kNoAllocPartialBytes);
    double* result = (double*)(scratch + kNoAllocPartialBytes + 128);

    const cudaStream_t s = (cudaStream_t)stream;
    // The array keeps whatever the previous call left; the arrival counter of
    // the reduction must start at zero.
    if (cudaMemsetAsync(red.counter, 0, sizeof(unsigned int), s) != cudaSuccess) return TO3D_ECUDA;
    launch_sensitivity_raw(ke, g, s, x, u, penal, E0, Emin, ce, dc, red, result);
    if (cudaGetLastError() != cudaSuccess) return TO3D_ECUDA;
    if (cudaMemcpyAsync(compliance, result, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TO3D_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TO3D_ECUDA;
    return TO3D_OK;
}
