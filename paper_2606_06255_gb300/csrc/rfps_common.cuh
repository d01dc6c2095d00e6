// rfps_common.cuh -- device arithmetic shared by the sampling kernels.
//
// Every floating-point step below uses the explicitly rounded intrinsics
// (__fsub_rn, __fmul_rn, __fadd_rn, __fsqrt_rn) so that nvcc can neither
// contract a multiply and an add into an FMA nor reassociate: the squared
// distance is exactly (dx*dx + dy*dy) + dz*dz in FP32 round-to-nearest, the
// canonical arithmetic of the library (reading of Sec. 3.1: "same
// floating-point precision").  The library is built without --use_fast_math
// and without flush-to-zero.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rfps {

constexpr uint32_t kStatusOk = 0;
constexpr uint32_t kStatusInval = 1;
constexpr uint32_t kStatusNonFinite = 2;
constexpr uint32_t kStatusTimeout = 5;
constexpr uint32_t kStatusUnsupported = 6;
constexpr uint32_t kStatusBounds = 7;      // bounds-checked builds only

// Canonical FP32 squared distance between p and s.
__device__ __forceinline__ float sq_dist(float px, float py, float pz, float sx, float sy, float sz)
{
    const float dx = __fsub_rn(px, sx);
    const float dy = __fsub_rn(py, sy);
    const float dz = __fsub_rn(pz, sz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Argmax key of a point: (bits of its squared distance) << 32 | ~index.
// Stored distances are >= +0 (never -0: a difference of equal floats is +0
// and squares are non-negative), so the IEEE bit pattern orders like the
// value, +inf included.  The low word ~index makes the larger key the one
// with the smaller index on equal distances: max over keys is the argmax
// with the smallest-original-index tie rule of Sec. 3.1, and the same
// max-of-keys over a voxel is its Dist_v (Eq. preprocess_distv) together
// with the index that attains it (the tie-exact two-level selection of
// Eq. global_equivalent_selection).
__device__ __forceinline__ unsigned long long make_key(float d2, uint32_t index)
{
    return (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) | static_cast<unsigned long long>(~index);
}
__device__ __forceinline__ float key_d2(unsigned long long key) { return __uint_as_float(static_cast<uint32_t>(key >> 32)); }
__device__ __forceinline__ uint32_t key_index(unsigned long long key) { return ~static_cast<uint32_t>(key); }

// Spherical-voxel radius pruning (Sec. 3.4.2: Eq. spherical_voxel_bound and
// radius_pruning_condition) in FP32, decided without a square root per test.
//
// The paper prunes record k when LB = max(0, |s - c| - r) >= Dist_v, i.e.
// when |s - c| >= r + sqrt(Dist_v).  Each record keeps a threshold T, computed
// once whenever its Dist_v key changes, and a test is one canonical FP32 squared
// distance and one compare: prune iff fl d2(s, c) >= T.
//
// Safety (u = 2^-24; r >= |p - c| for every member p, exact reals, from the
// build; every rounding of T is upward, so T >= (r + rho)^2 (1 + 2^-20)):
//   rho = sqrt(dv) (1 + 2^-20) (rounded up), so (1 - 5u) rho^2 >= dv (1 + 26u).
//   fl d2(s, c) <= (1 + u)^5 |s - c|^2 + 3 * 2^-150; with T >= 2^-100 the
//   test gives |s - c|^2 >= (r + rho)^2, so |s - p| >= |s - c| - |p - c|
//   >= rho for every member p, and fl d2(p, s) >= (1 - 5u) rho^2 - 3 * 2^-150
//   >= dv >= stored d2(p) when dv >= 2^-100: the strict update cannot fire.
//   (An overflowed fl d2(s, c) = +inf only happens for |s - c|^2 above
//   FLT_MAX / (1 + u)^5 >= T, so pruning on it is also safe.)
// dv = 0: nothing can decrease, T = 0 always prunes.  dv tiny (< 2^-100) or
// +inf, or T not finite: T = NaN, which never prunes.
__device__ __forceinline__ float prune_threshold(float r, unsigned long long key)
{
    const float nan = __int_as_float(0x7fc00000);
    const float dv = key_d2(key);
    if (dv == 0.0f) return 0.0f;
    if (!(dv >= 0x1p-100f) || !(dv <= 3.4028234e38f)) return nan;
    const float rho = __fmul_ru(__fsqrt_ru(dv), 0x1.00001p0f);   // 1 + 2^-20
    const float s = __fadd_ru(r, rho);
    float t = __fmul_ru(__fmul_ru(s, s), 0x1.00001p0f);
    t = fmaxf(t, 0x1p-100f);
    return t <= 3.4028234e38f ? t : nan;
}

// The per-iteration test: record (centre, threshold) = ct.
__device__ __forceinline__ bool prune_by_threshold(float4 ct, float sx, float sy, float sz)
{
    return sq_dist(sx, sy, sz, ct.x, ct.y, ct.z) >= ct.w;
}

// Coordinate-wise point skip (Sec. 3.4.3, Eq. point_skip_condition) in the
// squared domain: skip iff fl(da*da) >= stored d2 for some axis, with the
// same rounded terms that make up d2.  Adding non-negative floats under
// round-to-nearest never decreases, so d2 >= fl(da*da) >= stored d2 and the
// strict update could not fire: the skip is exact, not just conservative.
__device__ __forceinline__ bool skip_point(float xx, float yy, float zz, float d2old)
{
    return xx >= d2old || yy >= d2old || zz >= d2old;
}

// ---------------------------------------------------------------------------
// Warp helpers
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    uint32_t hi = static_cast<uint32_t>(v >> 32);
    const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
    uint32_t lo = (hi == mhi) ? static_cast<uint32_t>(v) : 0u;
    const uint32_t mlo = __reduce_max_sync(0xffffffffu, lo);
    return (static_cast<unsigned long long>(mhi) << 32) | mlo;
}

// Lane holding the warp-wide maximum key (keys are unique per point; for
// equal keys the lowest lane).
__device__ __forceinline__ int warp_argmax_lane(unsigned long long v, unsigned long long* vmax)
{
    const unsigned long long m = warp_max_u64(v);
    *vmax = m;
    const uint32_t b = __ballot_sync(0xffffffffu, v == m);
    return __ffs(b) - 1;
}

// ---------------------------------------------------------------------------
// Thread-block cluster helpers (sm_90+ PTX).
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Full cluster barrier: release my prior shared::cluster writes, acquire the others'.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of `p` (my shared memory) in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t map_shared(const void* p, uint32_t rank)
{
    const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
    return remote;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster_u64(uint32_t addr, unsigned long long v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_f32x4(uint32_t addr, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

// Order-preserving float <-> uint encoding for atomic min/max of floats.
__device__ __forceinline__ uint32_t float_to_ordered(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

}  // namespace rfps

namespace rfps {

// ---------------------------------------------------------------------------
// One-way DSMEM exchange with transaction-counting mbarriers (sm_90+ PTX).
// A consumer CTA arms its barrier for the bytes it expects (one arrival plus
// expect_tx); producers write with st.async, each store completing its byte
// count on the consumer's barrier; the consumer waits for the phase.  No
// cluster-wide barrier and no release fence is needed per round.
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init_cluster()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned long long* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void st_async_u64(uint32_t raddr, unsigned long long v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(raddr), "l"(v),
                 "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f32x4(uint32_t raddr, float4 v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
                 : "memory");
}
// Bounded wait for a barrier phase; false if it gave up (the caller records
// RFPS_ETIMEOUT and winds down).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait_cluster(bar, parity)) return true;
    return false;
}

}  // namespace rfps
