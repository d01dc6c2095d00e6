// rfps_sample.cu -- the persistent RadiusFPS sampling kernel (Sec. 3.3-3.4;
// the GPU roles of Fusion Kernels 1 and 2 of Sec. 4.2-4.3, fused into one
// launch for the whole loop).
//
// One thread-block cluster of C CTAs samples one cloud at a time and takes
// the next cloud from a device work queue (largest first).  The cloud's
// voxel records are dealt round-robin to the C CTAs (record k -> CTA k mod
// C), so the few records that a new sample touches, which are spatial
// neighbours with consecutive ids, land on different CTAs.  Each CTA keeps
// its records (sphere, Dist_v key, best point, point range) in shared memory
// (any that do not fit stay in global memory and are read there), and the
// points in the sorted float4 (x, y, z, d2) layout in global memory / L2.
//
// Iteration j (update with s_{j-1}, then select s_j):
//   every warp takes a strided set of its CTA's records (adjacent records go
//   to different warps); each lane tests one record with the FP-safe radius
//   pruning bound (prune_record); the warp then walks the unpruned records of
//   its lanes one by one: lanes stride over the record's points with the
//   point skip, the exact update and the new record key (the Dist_v sync,
//   Eq. point_skip_distv_sync);
//   the max key over all records -- pruned records keep their key -- is
//   reduced warp -> CTA (shared memory, one __syncthreads) -> cluster (each
//   CTA pushes its best (key, x, y, z) into every CTA's shared memory, one
//   barrier.cluster); every thread then knows s_j and its coordinates.
// Iteration 1 is the initial update of Sec. 3.3: every record is visited and
// the stored distances are treated as +inf, so a reused index needs no reset.
// There is no per-iteration kernel launch and no global-memory round trip for
// the selection.
#include <cfloat>

#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {

struct SampleArgs {
    WsHeader* hdr;
    const CloudDev* clouds;
    const uint32_t* order;
    int64_t n_clouds;
    const float* pts;          // caller's AoS points
    float4* pts4;              // sorted (x, y, z, d2)
    const uint32_t* porig;     // sorted position -> point row
    const float4* rec_sph;
    const uint2* rec_rng;
    unsigned long long* rec_key;
    float4* rec_best;
    int64_t* out;
    uint32_t cap;              // records per CTA held in shared memory
    int prune, skip;
};

constexpr int kMaxCluster = 16;

template <int NT, bool CLUSTER, bool COUNTERS>
__global__ void __launch_bounds__(NT, 1) k_sample(const SampleArgs a)
{
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_sph = reinterpret_cast<float4*>(smem);
    float4* s_best = s_sph + a.cap;
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(s_best + a.cap);
    uint2* s_rng = reinterpret_cast<uint2*>(s_key + a.cap);
    __shared__ unsigned long long s_wkey[2][NW];
    __shared__ uint32_t s_wrec[2][NW];
    __shared__ unsigned long long s_ckey[2][kMaxCluster];
    __shared__ float4 s_cxyz[2][kMaxCluster];
    __shared__ uint32_t s_item;

    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t C = CLUSTER ? cluster_nctarank() : 1u;
    if (a.hdr->status != 0) return;   // same value in every CTA: uniform exit
    if (CLUSTER) cluster_sync();       // every CTA of the cluster is running before any DSMEM store

    uint64_t c_tests = 0, c_pruned = 0, c_visit = 0, c_skip = 0, c_upd = 0, c_iter = 0;

    for (;;) {
        if (rank == 0 && t == 0) {
            const uint32_t item = atomicAdd(&a.hdr->work, 1u);
            if (CLUSTER) {
                for (uint32_t r = 0; r < C; ++r)
                    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(map_shared(&s_item, r)), "r"(item)
                                 : "memory");
            } else {
                s_item = item;
            }
        }
        if (CLUSTER) cluster_sync(); else __syncthreads();
        const uint32_t item = s_item;
        if (item >= a.n_clouds) break;
        const CloudDev c = a.clouds[a.order[item]];
        if (c.valid) {
            const uint32_t K = c.rec_end - c.rec_off;
            const uint32_t nloc = K > rank ? (K - rank + C - 1) / C : 0u;
            const uint32_t nsm = nloc < a.cap ? nloc : a.cap;
            const uint32_t gbase = c.rec_off + rank;
            for (uint32_t l = t; l < nsm; l += NT) {
                const uint32_t k = gbase + l * C;
                s_sph[l] = a.rec_sph[k];
                s_rng[l] = a.rec_rng[k];
                s_key[l] = a.rec_key[k];
                s_best[l] = a.rec_best[k];
            }
            const int64_t g0 = c.pt_off + c.start;
            float sx = a.pts[3 * g0 + 0], sy = a.pts[3 * g0 + 1], sz = a.pts[3 * g0 + 2];
            if (rank == 0 && t == 0) a.out[c.out_off] = c.start;
            __syncthreads();

            for (int64_t j = 1; j < c.m; ++j) {
                const bool first = (j == 1);
                const int par = static_cast<int>(j & 1);
                unsigned long long tk = 0ull;
                uint32_t tr = 0xffffffffu;
                for (uint32_t base = 0; base < nloc; base += NT) {
                    const uint32_t l = base + static_cast<uint32_t>(lane * NW + w);
                    const bool valid = l < nloc;
                    bool visit = false;
                    if (valid) {
                        const bool in_smem = l < nsm;
                        const float4 sph = in_smem ? s_sph[l] : a.rec_sph[gbase + l * C];
                        const unsigned long long key = in_smem ? s_key[l] : a.rec_key[gbase + l * C];
                        visit = first || !a.prune || !prune_record(sph, key, sx, sy, sz);
                        if (!visit && key > tk) {
                            tk = key;
                            tr = l;
                        }
                        if (COUNTERS) {
                            c_tests += first ? 0 : 1;
                            c_pruned += visit ? 0 : 1;
                        }
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, visit);
                    while (mask) {
                        const int src = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const uint32_t lr = __shfl_sync(0xffffffffu, l, src);
                        const bool in_smem = lr < nsm;
                        const uint2 rng = in_smem ? s_rng[lr] : a.rec_rng[gbase + lr * C];
                        unsigned long long lk = 0ull;
                        float bx = 0.f, by = 0.f, bz = 0.f;
                        for (uint32_t q = lane; q < rng.y; q += 32) {
                            const uint32_t pos = rng.x + q;
                            const float4 p = a.pts4[pos];
                            const uint32_t g = a.porig[pos];
                            float d2 = first ? __int_as_float(0x7f800000) : p.w;
                            const float dx = __fsub_rn(p.x, sx);
                            const float dy = __fsub_rn(p.y, sy);
                            const float dz = __fsub_rn(p.z, sz);
                            const float xx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy), zz = __fmul_rn(dz, dz);
                            if (a.skip && skip_point(xx, yy, zz, d2)) {
                                if (COUNTERS) ++c_skip;
                                if (first) a.pts4[pos].w = d2;
                            } else {
                                const float nd = __fadd_rn(__fadd_rn(xx, yy), zz);
                                if (nd < d2) {
                                    d2 = nd;
                                    if (COUNTERS) ++c_upd;
                                    a.pts4[pos].w = d2;
                                } else if (first) {
                                    a.pts4[pos].w = d2;
                                }
                            }
                            if (COUNTERS) ++c_visit;
                            const unsigned long long k = make_key(d2, g);
                            if (k > lk) {
                                lk = k;
                                bx = p.x; by = p.y; bz = p.z;
                            }
                        }
                        unsigned long long rk;
                        const int wl = warp_argmax_lane(lk, &rk);
                        const float wx = __shfl_sync(0xffffffffu, bx, wl);
                        const float wy = __shfl_sync(0xffffffffu, by, wl);
                        const float wz = __shfl_sync(0xffffffffu, bz, wl);
                        if (lane == 0) {
                            if (in_smem) {
                                s_key[lr] = rk;
                                s_best[lr] = make_float4(wx, wy, wz, 0.f);
                            } else {
                                a.rec_key[gbase + lr * C] = rk;
                                a.rec_best[gbase + lr * C] = make_float4(wx, wy, wz, 0.f);
                            }
                        }
                        if (lane == src && rk > tk) {
                            tk = rk;
                            tr = lr;
                        }
                    }
                }
                // warp -> CTA
                unsigned long long wk;
                const int wl = warp_argmax_lane(tk, &wk);
                const uint32_t wr = __shfl_sync(0xffffffffu, tr, wl);
                if (lane == 0) {
                    s_wkey[par][w] = wk;
                    s_wrec[par][w] = wr;
                }
                __syncthreads();
                unsigned long long ck = lane < NW ? s_wkey[par][lane] : 0ull;
                uint32_t cr = lane < NW ? s_wrec[par][lane] : 0xffffffffu;
                unsigned long long cbest;
                const int cl = warp_argmax_lane(ck, &cbest);
                cr = __shfl_sync(0xffffffffu, cr, cl);
                float4 cxyz = make_float4(0.f, 0.f, 0.f, 0.f);
                if (cbest != 0ull) cxyz = cr < nsm ? s_best[cr] : a.rec_best[gbase + cr * C];
                unsigned long long gbest = cbest;
                if (CLUSTER) {
                    // CTA -> cluster: push (key, xyz) into slot `rank` of every CTA
                    if (w == 0 && lane < static_cast<int>(C)) {
                        st_cluster_u64(map_shared(&s_ckey[par][rank], lane), cbest);
                        st_cluster_f32x4(map_shared(&s_cxyz[par][rank], lane), cxyz);
                    }
                    cluster_sync();
                    const unsigned long long kk = lane < static_cast<int>(C) ? s_ckey[par][lane] : 0ull;
                    const int gl = warp_argmax_lane(kk, &gbest);
                    cxyz = s_cxyz[par][gl];
                }
                sx = cxyz.x;
                sy = cxyz.y;
                sz = cxyz.z;
                if (rank == 0 && t == 0)
                    a.out[c.out_off + j] = static_cast<int64_t>(key_index(gbest)) - c.pt_off;
                if (COUNTERS) ++c_iter;
            }
        }
        if (CLUSTER) cluster_sync(); else __syncthreads();
    }
    if (COUNTERS) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[0]), c_tests);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[1]), c_pruned);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[2]), c_visit);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[3]), c_skip);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[4]), c_upd);
        if (t == 0 && rank == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[5]), c_iter);
    }
}

template <int NT, bool CLUSTER, bool COUNTERS>
cudaError_t launch_one(const SampleArgs& args, int C, int64_t n_clouds, cudaStream_t st)
{
    auto kern = k_sample<NT, CLUSTER, COUNTERS>;
    const size_t dyn = static_cast<size_t>(args.cap) * 48;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    int n_groups = 0;
    if (CLUSTER) {
        if (C > 8) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(C);
        int max_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (max_clusters < 1) return cudaErrorInvalidConfiguration;
        n_groups = static_cast<int>(n_clouds < max_clusters ? n_clouds : max_clusters);
        cfg.gridDim = dim3(C * n_groups);
    } else {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int64_t cap = static_cast<int64_t>(per_sm) * sms;
        n_groups = static_cast<int>(n_clouds < cap ? n_clouds : cap);
        cfg.gridDim = dim3(n_groups);
    }
    e = cudaLaunchKernelEx(&cfg, kern, args);
    note_launches(1);
    return e;
}

template <bool CLUSTER, bool COUNTERS>
cudaError_t launch_nt(const SampleArgs& args, int NT, int C, int64_t n_clouds, cudaStream_t st)
{
    switch (NT) {
    case 256: return launch_one<256, CLUSTER, COUNTERS>(args, C, n_clouds, st);
    case 512: return launch_one<512, CLUSTER, COUNTERS>(args, C, n_clouds, st);
    default: return launch_one<1024, CLUSTER, COUNTERS>(args, C, n_clouds, st);
    }
}

}  // namespace

cudaError_t launch_sample(char* ws, const WsLayout& L, const float* points, int64_t* out, const rfps_opts& o,
                          int64_t n_clouds, int64_t max_n, cudaStream_t st)
{
    (void)max_n;
    SampleArgs a;
    a.hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    a.clouds = reinterpret_cast<const CloudDev*>(ws + L.clouds);
    a.order = reinterpret_cast<const uint32_t*>(ws + L.order);
    a.n_clouds = n_clouds;
    a.pts = points;
    a.pts4 = reinterpret_cast<float4*>(ws + L.pts4);
    a.porig = reinterpret_cast<const uint32_t*>(ws + L.porig);
    a.rec_sph = reinterpret_cast<const float4*>(ws + L.rec_sph);
    a.rec_rng = reinterpret_cast<const uint2*>(ws + L.rec_rng);
    a.rec_key = reinterpret_cast<unsigned long long*>(ws + L.rec_key);
    a.rec_best = reinterpret_cast<float4*>(ws + L.rec_best);
    a.out = out;
    a.prune = o.prune;
    a.skip = o.skip;
    // shared memory: as many records as fit beside the static slots
    const size_t budget = 200 * 1024;
    a.cap = static_cast<uint32_t>(budget / 48);
    const int C = o.cluster;
    const bool cl = C > 1;
    if (o.counters) {
        return cl ? launch_nt<true, true>(a, o.threads, C, n_clouds, st)
                  : launch_nt<false, true>(a, o.threads, C, n_clouds, st);
    }
    return cl ? launch_nt<true, false>(a, o.threads, C, n_clouds, st)
              : launch_nt<false, false>(a, o.threads, C, n_clouds, st);
}

}  // namespace rfps
