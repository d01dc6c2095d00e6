// rfps_probe.cu -- on-chip bandwidth probes: the denominators of the sampling
// kernel's on-chip roofline.  Its working set (records, resident points, the
// exchange slots) lives in shared memory and L2, not DRAM, so the HBM copy
// bandwidth alone says little about how close it runs to a bandwidth limit.
//
//   kind 0  every SM streams a device buffer with L2-only loads
//           (ld.global.cg), `reps` passes: the L2 read bandwidth of the whole
//           GPU for a buffer that fits in L2.
//   kind 1  every resident CTA reads its own 48 KiB shared-memory array
//           `reps` times with 16-byte loads, each warp reading 512 contiguous
//           bytes (no bank conflicts): the shared-memory read bandwidth.
//
// The shared-memory loads are ld.volatile, and every L2 pass starts at another
// vector (the grid-stride walk rotated by the pass number), so that the
// assembler can neither hoist a pass out of its loop nor merge two of them
// (plain loads of unchanged addresses with no store in between may be).  Every
// warp XORs the 32-bit words it read into
// `sink`, so nothing is dead, and after an odd number of passes the sink holds
// the XOR of every word read once: the caller can check that all of it was read.
// Kind 1 fills vector i of CTA b with (i, 3i, 5i, b * 2654435761 + i), mod 2^32.
#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {

constexpr int kProbeThreads = 512;
constexpr int kSmemVec = 3072;   // 48 KiB of 16-byte vectors per CTA

__device__ __forceinline__ uint4 ld_cg_v4(const uint4* p)
{
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ void fold_into(unsigned long long* sink, uint32_t acc)
{
    acc = __reduce_xor_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31u) == 0) atomicXor(sink, static_cast<unsigned long long>(acc));
}

// kind 0: grid-stride passes over n4 16-byte vectors, four loads in flight per thread
__global__ void __launch_bounds__(kProbeThreads) k_probe_l2(const uint4* buf, int64_t n4, int reps,
                                                            unsigned long long* sink)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kProbeThreads;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kProbeThreads + threadIdx.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r) {
        // this pass's walk: the threads' start vectors rotated by r, so each vector is still read once
        const int64_t i0 = (t0 + r) % stride;
        int64_t i = i0;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const uint4 a = ld_cg_v4(buf + i);
            const uint4 b = ld_cg_v4(buf + i + stride);
            const uint4 c = ld_cg_v4(buf + i + 2 * stride);
            const uint4 d = ld_cg_v4(buf + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^
                   (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n4; i += stride) {
            const uint4 a = ld_cg_v4(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    fold_into(sink, acc);
}

// kind 1: each CTA fills its array once, then reads all of it `reps` times
__global__ void __launch_bounds__(kProbeThreads) k_probe_smem(int reps, unsigned long long* sink)
{
    __shared__ uint4 s[kSmemVec];
    for (int i = threadIdx.x; i < kSmemVec; i += kProbeThreads)   // content the caller can recompute
        s[i] = make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(i) * 3u, static_cast<uint32_t>(i) * 5u,
                          blockIdx.x * 2654435761u + static_cast<uint32_t>(i));
    __syncthreads();
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(s)) + 16u * threadIdx.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < kSmemVec / kProbeThreads; ++k) {
            const uint4 v = ld_shared_v4(base + 16u * static_cast<uint32_t>(k * kProbeThreads));
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    fold_into(sink, acc);
}

}  // namespace

cudaError_t launch_bw_probe(int kind, const void* buf, int64_t bytes, int reps, unsigned long long* sink,
                            cudaStream_t st, int64_t* moved, int* sms_out)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (kind == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_l2, kProbeThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t n4 = bytes / 16;
        k_probe_l2<<<per_sm * sms, kProbeThreads, 0, st>>>(static_cast<const uint4*>(buf), n4, reps, sink);
        if (moved) *moved = n4 * 16 * reps;
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_smem, kProbeThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        k_probe_smem<<<per_sm * sms, kProbeThreads, 0, st>>>(reps, sink);
        if (moved) *moved = static_cast<int64_t>(per_sm) * sms * kSmemVec * 16 * reps;
    }
    if (sms_out) *sms_out = sms;
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rfps
