// rfps_plain.cu -- plain O(N * M) GPU FPS (Alg. 1), the comparison baseline.
// Same arithmetic and tie rule as the RadiusFPS path; no voxel index.
//
//   variant 0  one CTA per cloud streams the whole cloud from global memory
//              every iteration (the classic FPS kernel design);
//   variant 1  one thread-block cluster per cloud; each CTA holds a
//              contiguous slice of the cloud as float4 (x, y, z, d2) in shared
//              memory when it fits (else streams it), argmax via warp shuffles,
//              shared memory and a DSMEM push + one barrier.cluster;
//   variant 2  one cloud on the whole GPU: one CTA per SM, each slice in
//              shared memory, a software grid barrier per iteration with a
//              bounded wait (cooperative launch: all CTAs are co-resident).
#include <cfloat>

#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {

struct PlainArgs {
    WsHeader* hdr;
    const CloudDev* clouds;
    const uint32_t* order;
    int64_t n_clouds;
    const float* pts;
    float* d2buf;                  // per point (global), variants 0 and streaming 1/2
    unsigned long long* gkey;      // variant 2: [2][grid] slot keys
    float4* gxyz;                  // variant 2: [2][grid] slot coordinates
    int64_t* out;
    uint32_t cap;                  // points per CTA held in shared memory
};

// Update one point and fold its key into the lane's best.
__device__ __forceinline__ void visit_point(float x, float y, float z, float& d2, bool first, float sx, float sy,
                                            float sz, uint32_t idx, unsigned long long& lk, float& bx, float& by,
                                            float& bz, bool& changed)
{
    float cur = first ? __int_as_float(0x7f800000) : d2;
    const float nd = sq_dist(x, y, z, sx, sy, sz);
    changed = first;
    if (nd < cur) {
        cur = nd;
        changed = true;
    }
    d2 = cur;
    const unsigned long long k = make_key(cur, idx);
    if (k > lk) {
        lk = k;
        bx = x; by = y; bz = z;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_plain_classic(const PlainArgs a)
{
    constexpr int NW = NT / 32;
    __shared__ unsigned long long s_key[2][NW];
    __shared__ float4 s_xyz[2][NW];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (a.hdr->status != 0) return;
    for (int64_t item = blockIdx.x; item < a.n_clouds; item += gridDim.x) {
        const CloudDev c = a.clouds[a.order[item]];
        if (!c.valid) continue;
        const float* p = a.pts + 3 * c.pt_off;
        float* D = a.d2buf + c.pt_off;
        const uint32_t n = static_cast<uint32_t>(c.n);
        float sx = p[3 * c.start], sy = p[3 * c.start + 1], sz = p[3 * c.start + 2];
        if (t == 0) a.out[c.out_off] = c.start;
        for (int64_t j = 1; j < c.m; ++j) {
            const bool first = j == 1;
            const int par = static_cast<int>(j & 1);
            unsigned long long lk = 0ull;
            float bx = 0.f, by = 0.f, bz = 0.f;
            for (uint32_t i = t; i < n; i += NT) {
                float d2 = first ? 0.f : D[i];
                bool changed;
                visit_point(p[3 * i], p[3 * i + 1], p[3 * i + 2], d2, first, sx, sy, sz, i, lk, bx, by, bz, changed);
                if (changed) D[i] = d2;
            }
            unsigned long long wk;
            const int wl = warp_argmax_lane(lk, &wk);
            const float wx = __shfl_sync(0xffffffffu, bx, wl);
            const float wy = __shfl_sync(0xffffffffu, by, wl);
            const float wz = __shfl_sync(0xffffffffu, bz, wl);
            if (lane == 0) {
                s_key[par][w] = wk;
                s_xyz[par][w] = make_float4(wx, wy, wz, 0.f);
            }
            __syncthreads();
            const unsigned long long k = lane < NW ? s_key[par][lane] : 0ull;
            unsigned long long best;
            const int bl = warp_argmax_lane(k, &best);
            const float4 xyz = s_xyz[par][bl];
            sx = xyz.x; sy = xyz.y; sz = xyz.z;
            if (t == 0) a.out[c.out_off + j] = key_index(best);
        }
        __syncthreads();
    }
}

// Variant 1: one cluster per cloud; CTA r owns rows [lo_r, hi_r).
template <int NT, bool SMEM>
__global__ void __launch_bounds__(NT, 1) k_plain_cluster(const PlainArgs a)
{
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_pts = reinterpret_cast<float4*>(smem);
    __shared__ unsigned long long s_key[2][NW];
    __shared__ float4 s_xyz[2][NW];
    __shared__ unsigned long long s_ckey[2][16];
    __shared__ float4 s_cxyz[2][16];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t rank = cluster_ctarank(), C = cluster_nctarank();
    if (a.hdr->status != 0) return;
    cluster_sync();
    for (int64_t item = cluster_id_x(); item < a.n_clouds; item += cluster_count_x()) {
        const CloudDev c = a.clouds[a.order[item]];
        if (!c.valid) continue;
        const float* p = a.pts + 3 * c.pt_off;
        float* D = a.d2buf + c.pt_off;
        const uint32_t n = static_cast<uint32_t>(c.n);
        const uint32_t per = (n + C - 1) / C;
        const uint32_t lo = min(n, rank * per), hi = min(n, lo + per);
        const uint32_t cnt = hi - lo;
        if (SMEM) {
            for (uint32_t i = t; i < cnt; i += NT)
                s_pts[i] = make_float4(p[3 * (lo + i)], p[3 * (lo + i) + 1], p[3 * (lo + i) + 2], 0.f);
        }
        float sx = p[3 * c.start], sy = p[3 * c.start + 1], sz = p[3 * c.start + 2];
        if (rank == 0 && t == 0) a.out[c.out_off] = c.start;
        __syncthreads();
        for (int64_t j = 1; j < c.m; ++j) {
            const bool first = j == 1;
            const int par = static_cast<int>(j & 1);
            unsigned long long lk = 0ull;
            float bx = 0.f, by = 0.f, bz = 0.f;
            for (uint32_t i = t; i < cnt; i += NT) {
                bool changed;
                if (SMEM) {
                    float4 q = s_pts[i];
                    visit_point(q.x, q.y, q.z, q.w, first, sx, sy, sz, lo + i, lk, bx, by, bz, changed);
                    if (changed) s_pts[i].w = q.w;
                } else {
                    const uint32_t g = lo + i;
                    float d2 = first ? 0.f : D[g];
                    visit_point(p[3 * g], p[3 * g + 1], p[3 * g + 2], d2, first, sx, sy, sz, g, lk, bx, by, bz,
                                changed);
                    if (changed) D[g] = d2;
                }
            }
            unsigned long long wk;
            const int wl = warp_argmax_lane(lk, &wk);
            const float wx = __shfl_sync(0xffffffffu, bx, wl);
            const float wy = __shfl_sync(0xffffffffu, by, wl);
            const float wz = __shfl_sync(0xffffffffu, bz, wl);
            if (lane == 0) {
                s_key[par][w] = wk;
                s_xyz[par][w] = make_float4(wx, wy, wz, 0.f);
            }
            __syncthreads();
            const unsigned long long k = lane < NW ? s_key[par][lane] : 0ull;
            unsigned long long cbest;
            const int bl = warp_argmax_lane(k, &cbest);
            const float4 cxyz = s_xyz[par][bl];
            if (w == 0 && lane < static_cast<int>(C)) {
                st_cluster_u64(map_shared(&s_ckey[par][rank], lane), cbest);
                st_cluster_f32x4(map_shared(&s_cxyz[par][rank], lane), cxyz);
            }
            cluster_sync();
            const unsigned long long kk = lane < static_cast<int>(C) ? s_ckey[par][lane] : 0ull;
            unsigned long long gbest;
            const int gl = warp_argmax_lane(kk, &gbest);
            const float4 xyz = s_cxyz[par][gl];
            sx = xyz.x; sy = xyz.y; sz = xyz.z;
            if (rank == 0 && t == 0) a.out[c.out_off + j] = key_index(gbest);
        }
        cluster_sync();
    }
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Variant 2: the whole GPU on cloud 0; CTA b owns rows [lo_b, hi_b).
// Grid barrier: each CTA publishes its best in slot [parity][b], fences,
// increments the arrival counter, and waits until gridDim.x * j arrivals are
// visible.  The wait is bounded; on timeout the CTA records RFPS_ETIMEOUT and
// stops (every other CTA then times out in turn) -- the kernel always ends.
template <int NT, bool SMEM>
__global__ void __launch_bounds__(NT, 1) k_plain_grid(const PlainArgs a, uint32_t spin_limit)
{
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_pts = reinterpret_cast<float4*>(smem);
    __shared__ unsigned long long s_key[2][NW];
    __shared__ float4 s_xyz[2][NW];
    __shared__ uint32_t s_abort;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t G = gridDim.x, cta = blockIdx.x;
    if (a.hdr->status != 0) return;
    const CloudDev c = a.clouds[0];
    if (!c.valid) return;
    const float* p = a.pts + 3 * c.pt_off;
    float* D = a.d2buf + c.pt_off;
    const uint32_t n = static_cast<uint32_t>(c.n);
    const uint32_t per = (n + G - 1) / G;
    const uint32_t lo = min(n, cta * per), hi = min(n, lo + per);
    const uint32_t cnt = hi - lo;
    if (SMEM) {
        for (uint32_t i = t; i < cnt; i += NT)
            s_pts[i] = make_float4(p[3 * (lo + i)], p[3 * (lo + i) + 1], p[3 * (lo + i) + 2], 0.f);
    }
    if (t == 0) s_abort = 0;
    float sx = p[3 * c.start], sy = p[3 * c.start + 1], sz = p[3 * c.start + 2];
    if (cta == 0 && t == 0) a.out[c.out_off] = c.start;
    __syncthreads();
    for (int64_t j = 1; j < c.m; ++j) {
        const bool first = j == 1;
        const int par = static_cast<int>(j & 1);
        unsigned long long lk = 0ull;
        float bx = 0.f, by = 0.f, bz = 0.f;
        for (uint32_t i = t; i < cnt; i += NT) {
            bool changed;
            if (SMEM) {
                float4 q = s_pts[i];
                visit_point(q.x, q.y, q.z, q.w, first, sx, sy, sz, lo + i, lk, bx, by, bz, changed);
                if (changed) s_pts[i].w = q.w;
            } else {
                const uint32_t g = lo + i;
                float d2 = first ? 0.f : D[g];
                visit_point(p[3 * g], p[3 * g + 1], p[3 * g + 2], d2, first, sx, sy, sz, g, lk, bx, by, bz, changed);
                if (changed) D[g] = d2;
            }
        }
        unsigned long long wk;
        const int wl = warp_argmax_lane(lk, &wk);
        const float wx = __shfl_sync(0xffffffffu, bx, wl);
        const float wy = __shfl_sync(0xffffffffu, by, wl);
        const float wz = __shfl_sync(0xffffffffu, bz, wl);
        if (lane == 0) {
            s_key[par][w] = wk;
            s_xyz[par][w] = make_float4(wx, wy, wz, 0.f);
        }
        __syncthreads();
        if (w == 0) {
            const unsigned long long k = lane < NW ? s_key[par][lane] : 0ull;
            unsigned long long cbest;
            const int bl = warp_argmax_lane(k, &cbest);
            if (lane == 0) {
                __stcg(&a.gkey[par * G + cta], cbest);
                __stcg(&a.gxyz[par * G + cta], s_xyz[par][bl]);
                __threadfence();
                atomicAdd(&a.hdr->grid_arrive, 1u);
                const uint32_t target = static_cast<uint32_t>(j) * G;
                uint32_t spins = 0;
                while (ld_acquire_gpu(&a.hdr->grid_arrive) < target) {
                    if (++spins > spin_limit) {
                        atomicCAS(&a.hdr->status, 0u, kStatusTimeout);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
        // every warp reduces the G slots (L1-bypassing loads)
        unsigned long long kk = 0ull;
        uint32_t kb = 0;
        for (uint32_t q = lane; q < G; q += 32) {
            const unsigned long long v = __ldcg(&a.gkey[par * G + q]);
            if (v > kk) {
                kk = v;
                kb = q;
            }
        }
        unsigned long long gbest;
        const int gl = warp_argmax_lane(kk, &gbest);
        kb = __shfl_sync(0xffffffffu, kb, gl);
        const float4 xyz = __ldcg(&a.gxyz[par * G + kb]);
        sx = xyz.x; sy = xyz.y; sz = xyz.z;
        if (cta == 0 && t == 0) a.out[c.out_off + j] = key_index(gbest);
    }
}

template <int NT>
cudaError_t launch_cluster_variant(const PlainArgs& a, int64_t max_n, int64_t n_clouds, cudaStream_t st)
{
    // cluster size: enough CTAs that a slice fits in shared memory, up to 16
    int C = 1;
    while (C < 16 && (max_n + C - 1) / C > a.cap) C *= 2;
    const bool smem = (max_n + C - 1) / C <= a.cap;
    const size_t dyn = smem ? static_cast<size_t>((max_n + C - 1) / C) * 16 : 0;
    auto kern = smem ? k_plain_cluster<NT, true> : k_plain_cluster<NT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cfg.gridDim = dim3(C);
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorInvalidConfiguration;
    const int groups = static_cast<int>(n_clouds < max_clusters ? n_clouds : max_clusters);
    cfg.gridDim = dim3(C * groups);
    e = cudaLaunchKernelEx(&cfg, kern, a);
    note_launches(1);
    return e;
}

}  // namespace

cudaError_t launch_plain(char* ws, const WsLayout& L, const float* points, int64_t* out, int variant,
                         int64_t n_clouds, int64_t max_n, cudaStream_t st)
{
    PlainArgs a;
    a.hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    a.clouds = reinterpret_cast<const CloudDev*>(ws + L.clouds);
    a.order = reinterpret_cast<const uint32_t*>(ws + L.order);
    a.n_clouds = n_clouds;
    a.pts = points;
    a.d2buf = reinterpret_cast<float*>(ws + L.keys0);
    a.gkey = reinterpret_cast<unsigned long long*>(ws + L.hist);
    a.gxyz = reinterpret_cast<float4*>(ws + L.rec_best);
    a.out = out;
    a.cap = static_cast<uint32_t>((200 * 1024) / 16);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (variant == 0) {
        const int64_t g = n_clouds < 4 * sms ? n_clouds : 4 * sms;
        k_plain_classic<1024><<<static_cast<unsigned>(g), 1024, 0, st>>>(a);
        note_launches(1);
        return cudaGetLastError();
    }
    if (variant == 1) return launch_cluster_variant<1024>(a, max_n, n_clouds, st);
    // variant 2: single cloud over every SM
    constexpr int NT = 1024;
    int G = sms;
    const bool smem = (max_n + G - 1) / G <= a.cap;
    const size_t dyn = smem ? static_cast<size_t>((max_n + G - 1) / G) * 16 : 0;
    auto kern = smem ? k_plain_grid<NT, true> : k_plain_grid<NT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint32_t spin_limit = 1u << 24;
    void* params[] = {&a, &spin_limit};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(G), dim3(NT), params, dyn, st);
    note_launches(1);
    return e;
}

}  // namespace rfps
