// rfps_noalloc.cu -- rfps_fps_noalloc: single-cloud RadiusFPS whose scratch
// memory is a fixed array compiled into the library, so the call itself
// allocates nothing.
//
// Who needs it: code that must not call cudaMalloc or any allocating routine
// on its own path -- for example a real-time loop that cannot tolerate the
// implicit device synchronisation and unbounded latency of an allocation, a
// plug-in running inside a host application whose allocator owns all device
// memory, or code that runs while the device heap is reserved for someone
// else.  Such a caller passes only its input and output buffers.
//
// The scratch array is a file-scope __device__ array of kNoAllocScratchBytes
// (64 MiB).  Every GPU that loads the library holds it until the process
// exits, and every call on that GPU shares it: the array keeps the last
// call's contents, and two calls whose work overlaps on the GPU race on it.
// Everything the kernels need to start at zero (status word, counters, work
// queue, bounding-box accumulators) is reset by the first kernel of each
// call, so no clearing is needed between calls.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so every call looks the address up with
// cudaGetSymbolAddress, with the calling device current, and checks the return
// code.  The lookup is not cached: after cudaDeviceReset, or in another CUDA
// context on the same device, the module can be loaded at another address,
// and a cached pointer would then address memory the array no longer occupies.
// Once the module is loaded on a device the lookup allocates nothing; the first
// call on each device may load it, so that first call should come before any
// stream capture.
//
// Device-side errors (a non-finite coordinate, a cluster exchange wait that
// gave up, a cloud too large for one CTA's index) are written to the status
// word at the start of the array; rfps_noalloc_status_read returns it.
#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the current device's scratch array, looked up on every call.
cudaError_t noalloc_scratch(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace rfps

using namespace rfps;

extern "C" rfps_status rfps_fps_noalloc(const float* points, int64_t n, int64_t m, int64_t start, int64_t* out_idx,
                                        const rfps_opts* opts, void* stream)
{
    if (!points || !out_idx || n < 1 || n >= (int64_t(1) << 31) || m < 1 || m > n || start < 0 || start >= n)
        return RFPS_EINVAL;
    // same option rules as rfps_fps (rfps_fps_workspace_size returns 0 for invalid options)
    const size_t need = rfps_fps_workspace_size(n, opts);
    if (need == 0) return RFPS_EINVAL;
    if (need > kNoAllocScratchBytes) return RFPS_ENOMEM;   // beyond the fixed scratch: rejected
    void* ws = nullptr;
    if (noalloc_scratch(&ws) != cudaSuccess) return RFPS_ECUDA;
    // the same launches as rfps_fps, on the fixed scratch instead of a caller workspace
    return rfps_fps(points, n, m, start, out_idx, opts, ws, kNoAllocScratchBytes, stream);
}

extern "C" rfps_status rfps_noalloc_status_read(void* stream)
{
    void* ws = nullptr;
    if (noalloc_scratch(&ws) != cudaSuccess) return RFPS_ECUDA;
    // the status word opens the workspace header; copied into a host local, then the stream is synchronised
    uint32_t status = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&status, ws, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RFPS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RFPS_ECUDA;
    return static_cast<rfps_status>(status);
}
