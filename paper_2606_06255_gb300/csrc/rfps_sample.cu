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
//   every lane owns a fixed strided set of its CTA's records (adjacent
//   records go to different warps) and tests them with the FP-safe radius
//   pruning threshold (prune_threshold / prune_by_threshold: one squared
//   distance and one compare per record, no square root); the warp then
//   walks the unpruned records of its lanes one by one: lanes load the
//   record's points with several loads in flight, apply the point skip, the
//   exact update and form the new record key (the Dist_v sync, Eq.
//   point_skip_distv_sync), and the record's threshold is recomputed;
//   each lane caches the max key over the records it owns (keys only
//   decrease, so it rescans only when the record holding its max changed);
//   the max is reduced warp -> CTA (shared memory, one __syncthreads) ->
//   cluster (each CTA pushes its best (key, x, y, z) into every CTA's shared
//   memory, one barrier.cluster); every thread then knows s_j.
// Iteration 1 is the initial update of Sec. 3.3: every record is visited and
// the stored distances are treated as +inf, so a reused index needs no reset.
// There is no per-iteration kernel launch and no global-memory round trip for
// the selection.
//
// Runner-up shortcut (records in shared memory, on a cluster or one CTA).  With
// the exchange (or, on one CTA, the warps' shared slots), every CTA also learns
// r, the best candidate among the other warps, and each
// warp sends, in the spare fourth coordinate, a bound on every key of its
// records other than its own candidate (records also keep their second point
// key for this).  Let s be the selected sample.  If d2(r) > 0, r beats the
// winning warp's bound, and the canonical squared distance from r to s is not
// below d2(r), then the update with s leaves r's key unchanged, lowers every
// other key or keeps it, and sets s's own distance to 0; r is therefore
// Alg. 1's next argmax, exactly, ties included.  Every thread evaluates the
// same FP32 test on the same exchanged values, so the cluster agrees without
// another exchange, and the next round applies s and r together (one visit per
// record, the two updates in order).  On room- and LiDAR-like clouds the test
// holds in about 97 % of the rounds, so a round selects about two samples.  The
// second sample of a round is never the cloud's last, so a kept index still
// ends with one pending sample.  The register-record kernel for small clouds
// applies the same rule over the warps of its one CTA (a thread's record is its
// points, its second key the second largest of their keys), and the
// hierarchical path over super-records: a record in global memory keeps its
// second-key bound in rec_best.w (its radius is rec_sph.w), and a super-record
// keeps a bound on its keys but the max, refreshed with it.
#include <cfloat>

#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {

struct SampleArgs {
    WsHeader* hdr;
    CloudDev* clouds;
    const uint32_t* order;
    int64_t n_clouds;
    const float* pts;          // caller's AoS points
    float4* pts4;              // sorted (x, y, z, d2)
    const uint32_t* porig;     // sorted position -> point row
    const float4* rec_sph;     // centre, covering radius (read-only after the build)
    const uint2* rec_rng;      // first sorted position, count
    unsigned long long* rec_key;   // Dist_v key
    float4* rec_best;          // best point xyz, radius in .w (records kept in global memory)
    float* rec_thr;            // prune threshold (records kept in global memory)
    int64_t* out;
    size_t smem_bytes;         // dynamic shared memory per CTA
    int prune, skip;
    int resident;              // 1: keep records' points in shared memory while they fit
    int save_state;            // 1: write the sampling state back at the end (resumable index)
    // Failure-path test (counting kernels only): in exchange round `lost_iter` no warp sends its
    // candidate, and each exchange wait gives up after `spin_limit` polls.  lost_iter 0: none.
    int64_t lost_iter;
    uint32_t spin_limit;
#ifdef RFPS_CHECKED
    uint32_t n_total;          // points of all clouds (the length of pts4 / porig)
#endif
};

constexpr int kMaxCluster = 16;

// Bounds-checked test builds (-DRFPS_CHECKED): an index taken from data (a record's range, a list
// entry, the record that owns a candidate) that falls outside its array records RFPS_EBOUNDS in the
// status word and the access is skipped.  Every checked index is warp-uniform, so a failed check
// leaves warp-collective code converged.  Release builds compile the checks away.
#ifdef RFPS_CHECKED
#define RFPS_IN(cond) in_bounds((cond), a.hdr)
__device__ __forceinline__ bool in_bounds(bool ok, WsHeader* hdr)
{
    if (!ok) atomicCAS(&hdr->status, 0u, kStatusBounds);
    return ok;
}
#else
#define RFPS_IN(cond) true
#endif
constexpr uint32_t kResident = 0x80000000u;   // rng.x flag: the record's points are in shared memory
constexpr uint32_t kSpinLimit = 1u << 22;   // try_wait rounds before a wait gives up

// Shared-memory record state of one CTA (fast path): ct = (centre, prune
// threshold), best = (best point, covering radius), key = Dist_v key, rng =
// point range; local record l is global record gbase + l * C.
//
// When a lane holds more than two records (the loop that reads them from shared memory every
// iteration), the four arrays are stored warp-major: the record of slot s = l mod NT (lane
// s / NW of warp s mod NW) sits at pp(l), where the records of one warp are consecutive, so the
// lanes of a warp reading their own records touch consecutive addresses instead of addresses
// NW * 16 bytes apart in the same banks.  The last, partial block of NT records is packed the
// same way.  The register-held paths keep the plain order (at(l) = l): they read the arrays
// rarely and the index arithmetic would lengthen their critical path (both measured).
template <int NT>
struct RecView {
    static constexpr uint32_t NW = NT / 32;
    float4* ct;
    float4* best;
    unsigned long long* key;
    unsigned long long* key2;   // second-largest point key of the record (a bound until first visited)
    uint2* rng;
    uint32_t gbase, C, nloc;
    bool perm;
    const SampleArgs* a;
    __device__ __forceinline__ uint32_t g(uint32_t l) const { return gbase + l * C; }
    __device__ __forceinline__ uint32_t pp(uint32_t l) const
    {
        const uint32_t s = l % NT, base = l - s, w = s % NW, ln = s / NW;
        const uint32_t rem = min(static_cast<uint32_t>(NT), nloc - base);
        const uint32_t q = rem / NW, r = rem % NW;
        return base + w * q + min(w, r) + ln;
    }
    __device__ __forceinline__ uint32_t at(uint32_t l) const { return perm ? pp(l) : l; }
};

struct Cnt {
    uint64_t tests = 0, pruned = 0, visit = 0, skip = 0, upd = 0, iter = 0, rounds = 0;
    uint64_t pviol = 0, sviol = 0;   // shadow checks: see shadow_pruned and the skip branch below
};

// Counting runs only: the points of a record the bound pruned are checked
// against the new sample s anyway.  A distance that would strictly decrease
// means the prune bound was not safe for that record (must never happen).
__device__ uint64_t shadow_pruned(const float4* pts, uint32_t off, uint32_t cnt, float sx, float sy, float sz)
{
    uint64_t v = 0;
    for (uint32_t q = 0; q < cnt; ++q) {
        const float4 p = pts[off + q];
        if (sq_dist(p.x, p.y, p.z, sx, sy, sz) < p.w) ++v;
    }
    return v;
}

// The update of one point against sample s (Sec. 3.4.3 point skip, strict decrease of d2).
// `skipped` is cleared when the skip does not apply; `write` is set when d2 decreased.
template <bool COUNTERS>
__device__ __forceinline__ void update_point(const float4& p, float sx, float sy, float sz, int skip, float& d2,
                                             bool& write, bool& skipped, Cnt& k)
{
    const float dx = __fsub_rn(p.x, sx);
    const float dy = __fsub_rn(p.y, sy);
    const float dz = __fsub_rn(p.z, sz);
    const float xx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy), zz = __fmul_rn(dz, dz);
    if (skip && skip_point(xx, yy, zz, d2)) {
        if (COUNTERS && __fadd_rn(__fadd_rn(xx, yy), zz) < d2) ++k.sviol;   // the skip was not exact
    } else {
        skipped = false;
        const float nd = __fadd_rn(__fadd_rn(xx, yy), zz);
        if (nd < d2) {
            d2 = nd;
            write = true;
        }
    }
}

// Work counters of one visited point: skipped when every sample of the round skipped it, updated
// when its distance decreased (the visit counts the point once, however many samples it applies).
__device__ __forceinline__ void count_point(Cnt& k, bool skipped, bool updated)
{
    ++k.visit;
    if (skipped) ++k.skip;
    if (updated) ++k.upd;
}

// One warp updates the points [off, off + cnt) of a record against s, and then against t when
// `two` (a round that applies two samples), with the point skip, the strict update and the d2
// write-back.  Returns the lane's max key over its points, with that point in (bx, by, bz), and
// the lane's second-largest key in lk2.  `pts` / `orig` are either the CTA's shared-memory copy or
// the workspace arrays.  PPL loads are in flight per lane.
template <int PPL, bool COUNTERS>
__device__ __forceinline__ unsigned long long visit_points(float4* pts, const uint32_t* orig, uint32_t off,
                                                           uint32_t cnt, bool first, int skip, float sx, float sy,
                                                           float sz, int lane, float& bx, float& by, float& bz,
                                                           Cnt& k, bool two, float tx, float ty, float tz,
                                                           unsigned long long& lk2)
{
    unsigned long long lk = 0ull;
    lk2 = 0ull;
    for (uint32_t q0 = 0; q0 < cnt; q0 += 32u * PPL) {
        float4 p[PPL];
        uint32_t gi[PPL];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const uint32_t q = q0 + u * 32 + lane;
            if (q < cnt) {
                p[u] = pts[off + q];
                gi[u] = orig[off + q];
            }
        }
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const uint32_t q = q0 + u * 32 + lane;
            if (q < cnt) {
                float d2 = first ? __int_as_float(0x7f800000) : p[u].w;
                const float d0 = d2;
                bool write = first, skipped = true;
                update_point<COUNTERS>(p[u], sx, sy, sz, skip, d2, write, skipped, k);
                if (two) update_point<COUNTERS>(p[u], tx, ty, tz, skip, d2, write, skipped, k);
                if (write) pts[off + q].w = d2;
                if (COUNTERS) count_point(k, skipped, d2 < d0);
                const unsigned long long kk = make_key(d2, gi[u]);
                if (kk > lk) {
                    lk2 = lk;
                    lk = kk;
                    bx = p[u].x; by = p[u].y; bz = p[u].z;
                } else if (kk > lk2) {
                    lk2 = kk;
                }
            }
        }
    }
    return lk;
}

// The same update for a record held in shared memory, one point per lane per
// pass.  With 16 warps per CTA the other warps hide the shared-memory latency and
// the unrolled, predicated slots above only lengthen the critical warp; with 8
// warps the unrolled form is faster (both measured), so 512-thread CTAs use this.
template <bool COUNTERS>
__device__ __forceinline__ unsigned long long visit_points_smem(float4* pts, const uint32_t* orig, uint32_t off,
                                                                uint32_t cnt, bool first, int skip, float sx,
                                                                float sy, float sz, int lane, float& bx, float& by,
                                                                float& bz, Cnt& k, bool two, float tx, float ty,
                                                                float tz, unsigned long long& lk2)
{
    unsigned long long lk = 0ull;
    lk2 = 0ull;
#pragma unroll 1
    for (uint32_t q = lane; q < cnt; q += 32) {
        const float4 p = pts[off + q];
        float d2 = first ? __int_as_float(0x7f800000) : p.w;
        const float d0 = d2;
        bool write = first, skipped = true;
        update_point<COUNTERS>(p, sx, sy, sz, skip, d2, write, skipped, k);
        if (two) update_point<COUNTERS>(p, tx, ty, tz, skip, d2, write, skipped, k);
        if (write) pts[off + q].w = d2;
        if (COUNTERS) count_point(k, skipped, d2 < d0);
        const unsigned long long kk = make_key(d2, orig[off + q]);
        if (kk > lk) {
            lk2 = lk;
            lk = kk;
            bx = p.x; by = p.y; bz = p.z;
        } else if (kk > lk2) {
            lk2 = kk;
        }
    }
    return lk;
}

template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* s_scr, uint32_t* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_scr[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < NW ? s_scr[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < NW) s_scr[lane] = x;
    }
    __syncthreads();
    const uint32_t before = w > 0 ? s_scr[w - 1] : 0u;
    *total = s_scr[NW - 1];
    __syncthreads();
    return before + inc - v;
}

template <int V>
struct IntC {
    static constexpr int value = V;
};

template <int NT, bool CLUSTER, bool COUNTERS>
__global__ void __launch_bounds__(NT, 1) k_sample(const SampleArgs a)
{
    constexpr int NW = NT / 32;
    constexpr int PPL = 4;                      // point loads in flight per lane
    constexpr int NSLOT = CLUSTER ? kMaxCluster * NW : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_wkey[2][NW];
    __shared__ float4 s_wxyz[2][NW];
    __shared__ unsigned long long s_ckey[2][NSLOT];
    __shared__ float4 s_cxyz[2][NSLOT];
    __shared__ uint32_t s_scr[NW + 1];
    __shared__ uint32_t s_item, s_wlc[2], s_rlc[2], s_rlcut[2], s_abort;
    __shared__ unsigned long long s_mbar[2];

    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t C = CLUSTER ? cluster_nctarank() : 1u;
    if (t == 0) {
        s_abort = 0;
        if (CLUSTER) {
            mbar_init(&s_mbar[0], 1);
            mbar_init(&s_mbar[1], 1);
            fence_mbar_init_cluster();
        }
    }
    if (CLUSTER) cluster_sync();       // barriers initialised, every CTA running before any DSMEM store
    else __syncthreads();
    // this lane's destination (CTA `lane` of the cluster) for both exchange buffers: slot
    // [rank][warp] of the keys and coordinates, and that CTA's barrier
    uint32_t rkey0 = 0, rkey1 = 0, rxyz0 = 0, rxyz1 = 0, rbar0 = 0, rbar1 = 0;
    if (CLUSTER && lane < static_cast<int>(C)) {
        rkey0 = map_shared(&s_ckey[0][rank * NW + w], lane);
        rkey1 = map_shared(&s_ckey[1][rank * NW + w], lane);
        rxyz0 = map_shared(&s_cxyz[0][rank * NW + w], lane);
        rxyz1 = map_shared(&s_cxyz[1][rank * NW + w], lane);
        rbar0 = map_shared(&s_mbar[0], lane);
        rbar1 = map_shared(&s_mbar[1], lane);
    }
    uint32_t it = 0;                   // exchange rounds so far (same count in every CTA of the cluster)
    const float nan = __int_as_float(0x7fc00000);
    const uint32_t my = static_cast<uint32_t>(lane * NW + w);   // my slot inside each batch of NT records
    Cnt cn;

    for (;;) {
        if (rank == 0 && t == 0) {
            // an error recorded anywhere in the launch (before it or by another group) ends this
            // group: one decision, taken by rank 0 and sent to every CTA of the cluster
            uint32_t item = atomicAdd(&a.hdr->work, 1u);
            if (*static_cast<volatile uint32_t*>(&a.hdr->status) != 0u) item = 0xffffffffu;
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
        const uint32_t cloud = a.order[item];
        const CloudDev c = a.clouds[cloud];
        if (c.valid) {
            const bool resume = c.resume != 0;
            const uint32_t K = c.rec_end - c.rec_off;
            const uint32_t nloc = K > rank ? (K - rank + C - 1) / C : 0u;
            const uint32_t gbase = c.rec_off + rank;
            // Fast path: every record of this CTA in shared memory (60 bytes each),
            // then as many points as fit (20 bytes each).
            const bool fast = static_cast<size_t>(nloc) * 60 + 16 <= a.smem_bytes && nloc <= 32u * NT;
            const int nb = static_cast<int>((nloc + NT - 1) / NT);   // records per lane (fast path)
            RecView<NT> v;
            v.a = &a;
            v.C = C;
            v.gbase = gbase;
            v.nloc = nloc;
            v.perm = fast && !(NT <= 256 && nb <= 2);   // the iteration loop of MODE 3 below
            float4* s_pts = nullptr;
            uint32_t* s_orig = nullptr;
            uint32_t* s_soff = nullptr;
            bool resident = false;
#ifdef RFPS_CHECKED
            uint32_t pcap = 0;   // points the CTA's shared memory holds (fast path)
#endif
            // hierarchical path (records in global memory, super-records in shared memory)
            float4* s_sct = nullptr;             // super centre, prune threshold
            float4* s_sxyz = nullptr;            // best point of the super, radius in .w
            unsigned long long* s_skey = nullptr;
            uint32_t* s_slist = nullptr;         // unpruned super-records of this iteration
            float* s_sk2 = nullptr;              // per super-record: bound on its keys but the max (d2)
            float* s_rk2 = nullptr;              // per record-list entry: the visit's second-key bound
            uint2* s_sent = nullptr;             // per super-record: its range in the record list
            // record list (unpruned records of this iteration): local record, point range, and
            // the new key and best point its visit produced
            uint32_t* s_rlist = nullptr;
            uint2* s_rrng = nullptr;
            unsigned long long* s_rkey = nullptr;
            float4* s_rxyz = nullptr;
            uint32_t G = 0, W = 0;
            if (fast) {
                v.ct = reinterpret_cast<float4*>(smem);
                v.best = v.ct + nloc;
                v.key = reinterpret_cast<unsigned long long*>(v.best + nloc);
                v.key2 = v.key + nloc;
                v.rng = reinterpret_cast<uint2*>(v.key2 + nloc);
                s_soff = reinterpret_cast<uint32_t*>(v.rng + nloc);
                const size_t poff = (static_cast<size_t>(nloc) * 60 + 15) & ~static_cast<size_t>(15);
                s_pts = reinterpret_cast<float4*>(smem + poff);
                const uint32_t P = static_cast<uint32_t>((a.smem_bytes - poff) / 20);
#ifdef RFPS_CHECKED
                pcap = P;
#endif
                s_orig = reinterpret_cast<uint32_t*>(s_pts + P);
                uint32_t mine = 0;
                for (uint32_t l = t; l < nloc; l += NT) {
                    const uint32_t k = v.g(l);
                    const float4 sph = a.rec_sph[k];
                    const uint2 rg = a.rec_rng[k];
                    if (resume) {   // saved state: threshold, best point (radius in .w), key
                        v.ct[v.at(l)] = make_float4(sph.x, sph.y, sph.z, a.rec_thr[k]);
                        const float4 rb = a.rec_best[k];
                        v.best[v.at(l)] = make_float4(rb.x, rb.y, rb.z, sph.w);
                        v.key[v.at(l)] = a.rec_key[k];
                        v.key2[v.at(l)] = a.rec_key[k];   // a bound until the record's next visit
                    } else {
                        v.ct[v.at(l)] = make_float4(sph.x, sph.y, sph.z, nan);
                        v.best[v.at(l)] = make_float4(0.f, 0.f, 0.f, sph.w);
                        v.key[v.at(l)] = 0ull;
                        v.key2[v.at(l)] = 0ull;   // every record is visited in the first iteration
                    }
                    v.rng[v.at(l)] = rg;
                    mine += rg.y;
                }
                (void)mine;
                __syncthreads();   // every record's range is in shared memory before the chunked scan reads it
                if (a.resident && P > 0) {
                    // Records are made resident in order while their points fit: shared-memory
                    // offsets from a block scan of the counts (contiguous chunks per thread); a
                    // resident record's rng.x becomes kResident | offset in the CTA's point array.
                    const uint32_t per = (nloc + NT - 1) / NT;
                    const uint32_t l0 = min(nloc, t * per), l1 = min(nloc, l0 + per);
                    uint32_t sum = 0;
                    for (uint32_t l = l0; l < l1; ++l) sum += v.rng[v.at(l)].y;
                    uint32_t total;
                    uint32_t off = block_exclusive_sum<NT>(sum, s_scr, &total);
                    for (uint32_t l = l0; l < l1; ++l) {
                        const uint32_t cnt = v.rng[v.at(l)].y;
                        s_soff[l] = (off + cnt <= P) ? off : 0xffffffffu;   // shared-memory offset, or not resident
                        off += cnt;
                    }
                    __syncthreads();
                    for (uint32_t l = w; l < nloc; l += NW) {
                        const uint2 rg = v.rng[v.at(l)];
                        const uint32_t so = s_soff[l];
                        if (so == 0xffffffffu) continue;
                        for (uint32_t q = lane; q < rg.y; q += 32) {
                            s_pts[so + q] = a.pts4[rg.x + q];
                            s_orig[so + q] = a.porig[rg.x + q];
                        }
                    }
                    __syncthreads();
                    for (uint32_t l = t; l < nloc; l += NT)
                        if (s_soff[l] != 0xffffffffu) v.rng[v.at(l)].x = kResident | s_soff[l];
                    resident = true;
                }
            } else {
                // Hierarchical path: every record stays in global memory; each group of 32
                // consecutive local records is a super-record with a sphere covering all its
                // records' spheres, the max of their Dist_v keys and the coordinates of the point
                // that attains it, kept in shared memory.  Pruning tests super-records first.
                G = (nloc + 31) / 32;
                if (static_cast<size_t>(G) * 56 + 16 > a.smem_bytes) {
                    // more records than one CTA can index (beyond ~140k per CTA): larger clusters
                    // or records are needed; record the error and skip the cloud uniformly
                    if (t == 0) atomicCAS(&a.hdr->status, 0u, kStatusUnsupported);
                    G = 0;
                }
                // 56 bytes per super-record (16-byte arrays first), then 40 per record-list entry
                s_sct = reinterpret_cast<float4*>(smem);
                s_sxyz = s_sct + G;
                s_skey = reinterpret_cast<unsigned long long*>(s_sxyz + G);
                s_sent = reinterpret_cast<uint2*>(s_skey + G);
                s_slist = reinterpret_cast<uint32_t*>(s_sent + G);
                s_sk2 = reinterpret_cast<float*>(s_slist + G);
                const size_t used = (static_cast<size_t>(G) * 56 + 15) & ~static_cast<size_t>(15);
                const size_t room = a.smem_bytes > used ? (a.smem_bytes - used) / 40 : 0;
                W = static_cast<uint32_t>(room < nloc ? room : nloc);
                s_rxyz = reinterpret_cast<float4*>(smem + used);
                s_rkey = reinterpret_cast<unsigned long long*>(s_rxyz + W);
                s_rrng = reinterpret_cast<uint2*>(s_rkey + W);
                s_rlist = reinterpret_cast<uint32_t*>(s_rrng + W);
                s_rk2 = reinterpret_cast<float*>(s_rlist + W);
                // records in global memory keep, in rec_best.w, a bound on the squared distances of their
                // points but the best one (the runner-up shortcut's second key); on a resume it is reset
                // to the record's max, a safe bound until the record's next visit
                for (uint32_t l = t; l < nloc; l += NT) {
                    const uint32_t k = v.g(l);
                    if (!resume) {
                        a.rec_thr[k] = nan;
                        a.rec_key[k] = 0ull;
                        a.rec_best[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        float4 rb = a.rec_best[k];
                        rb.w = key_d2(a.rec_key[k]);
                        a.rec_best[k] = rb;
                    }
                }
                __syncthreads();
                for (uint32_t g = w; g < G; g += NW) {
                    const uint32_t l = g * 32 + lane;
                    const bool valid = l < nloc;
                    float4 sph = make_float4(0.f, 0.f, 0.f, 0.f);
                    unsigned long long kk = 0ull;
                    if (valid) {
                        sph = a.rec_sph[v.g(l)];
                        if (resume) kk = a.rec_key[v.g(l)];
                    }
                    // bounding box of the member spheres (rounded outwards), its centre
                    float lo[3], hi[3], cs[3];
                    const float cc[3] = {sph.x, sph.y, sph.z};
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        lo[ax] = valid ? __fsub_rd(cc[ax], sph.w) : 3.4028234e38f;
                        hi[ax] = valid ? __fadd_ru(cc[ax], sph.w) : -3.4028234e38f;
                        for (int o = 16; o > 0; o >>= 1) {
                            lo[ax] = fminf(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], o));
                            hi[ax] = fmaxf(hi[ax], __shfl_xor_sync(0xffffffffu, hi[ax], o));
                        }
                        cs[ax] = __fmul_rn(__fadd_rn(lo[ax], hi[ax]), 0.5f);
                    }
                    // radius: max over members of |c_m - c_s| + r_m, every step rounded up
                    float e = 0.f;
                    if (valid) {
                        const float d2 = sq_dist(cc[0], cc[1], cc[2], cs[0], cs[1], cs[2]);
                        const float dist = __fsqrt_ru(__fadd_ru(__fmul_ru(d2, 0x1.00004p0f), 0x1p-120f));
                        e = __fadd_ru(dist, sph.w);
                    }
                    for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
                    const float srad = fmaxf(__fmul_ru(e, 0x1.00001p0f), 0x1p-50f);
                    unsigned long long gk;
                    const int gl = warp_argmax_lane(kk, &gk);
                    float4 bxyz = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (resume && lane == gl && valid) bxyz = a.rec_best[v.g(l)];
                    bxyz.x = __shfl_sync(0xffffffffu, bxyz.x, gl);
                    bxyz.y = __shfl_sync(0xffffffffu, bxyz.y, gl);
                    bxyz.z = __shfl_sync(0xffffffffu, bxyz.z, gl);
                    if (lane == 0) {
                        s_sct[g] = make_float4(cs[0], cs[1], cs[2], resume ? prune_threshold(srad, gk) : nan);
                        s_sxyz[g] = make_float4(bxyz.x, bxyz.y, bxyz.z, srad);
                        s_skey[g] = gk;
                        s_sk2[g] = key_d2(gk);   // safe until the super-record is refreshed
                    }
                }
            }
            // the sample whose update comes first: the start point, or the saved last sample
            const int64_t g0 = c.pt_off + c.start;
            float sx = resume ? c.last[0] : a.pts[3 * g0 + 0];
            float sy = resume ? c.last[1] : a.pts[3 * g0 + 1];
            float sz = resume ? c.last[2] : a.pts[3 * g0 + 2];
            if (t == 0) {
                s_wlc[0] = 0;   // every CTA's own list counters (hierarchical path)
                s_wlc[1] = 0;
                s_rlc[0] = 0;
                s_rlc[1] = 0;
                s_rlcut[0] = W;
                s_rlcut[1] = W;
            }
            if (rank == 0 && t == 0 && !resume) a.out[c.out_off] = c.start;
            // a second sample applied in the same round (the runner-up shortcut, below)
            bool two = false;
            float tx = 0.f, ty = 0.f, tz = 0.f;
            // this lane's cached max over the records it owns (my, my + NT, ...), and a bound on
            // every other key of them (the second-largest of their key and key2 values)
            unsigned long long lkey = 0ull, lkey2 = 0ull;
            uint32_t lrec = 0xffffffffu;
            bool dirty = true;
            __syncthreads();

            // The iteration loop, compiled once per path so that each is scheduled on its own:
            // MODE 0 hierarchical; 1 and 2 fast with this lane's one or two records' centres and
            // thresholds held in registers (nloc <= NT, <= 2 NT; 128- and 256-thread CTAs, whose
            // register budget has room for it); 3 fast with any number per lane.
            auto iterate = [&](auto mode) {
                constexpr int MODE = decltype(mode)::value;
                constexpr bool FAST = MODE != 0;
                constexpr int NREG = MODE == 1 || MODE == 2 ? MODE : 0;
                // position of record l in the shared-memory arrays (warp-major in MODE 3)
                auto Q = [&](uint32_t l) -> uint32_t {
                    if constexpr (MODE == 3) return v.pp(l);
                    else return l;
                };
                float4 ct0 = make_float4(0.f, 0.f, 0.f, 0.f), ct1 = ct0;
                // counting runs: the shadow check of a pruned record held by this CTA
                auto shadow_record = [&](uint32_t l) -> uint64_t {
                    const uint2 rg = v.rng[Q(l)];
                    float4* base = (resident && (rg.x & kResident)) ? s_pts : a.pts4;
                    const uint32_t off = (resident && (rg.x & kResident)) ? (rg.x & ~kResident) : rg.x;
                    return shadow_pruned(base, off, rg.y, sx, sy, sz) + (two ? shadow_pruned(base, off, rg.y, tx, ty, tz) : 0);
                };
                if constexpr (NREG > 0) {
                    if (my < nloc) ct0 = v.ct[Q(my)];
                    if (NREG == 2 && my + NT < nloc) ct1 = v.ct[Q(my + NT)];
                }
                int64_t rnd = 0;   // rounds so far (a round selects one or two samples)
                for (int64_t j = 1; j < c.m; ++rnd) {
                    const bool first = (j == 1) && !resume;   // the initial update of Sec. 3.3
                    const int par = static_cast<int>(rnd & 1);
                    unsigned long long pk;   // this lane's partial max (key, record) for the selection
                    unsigned long long pk2;  // a bound on this lane's other keys
                    uint32_t prec;
                    uint32_t vis = 0;        // my records visited now (bit b: record b * NT + my)
                    // a visited record's bookkeeping waits until the warp's candidate is pushed
                    uint32_t dl = 0xffffffffu;
                    unsigned long long dk = 0ull, dk2 = 0ull;
                    float dx = 0.f, dy = 0.f, dz = 0.f;
                    bool ppt = false;        // this lane's candidate is a point of a record visited now
                    float px = 0.f, py = 0.f, pz = 0.f;
                    auto finish_record = [&](uint32_t l, unsigned long long lk, unsigned long long lk2, float bx,
                                             float by, float bz) {
                        unsigned long long rk;
                        const int rl = warp_argmax_lane(lk, &rk);
                        const unsigned long long rk2 = warp_max_u64(lane == rl ? lk2 : lk);   // second point key
                        const float wx = __shfl_sync(0xffffffffu, bx, rl);
                        const float wy = __shfl_sync(0xffffffffu, by, rl);
                        const float wz = __shfl_sync(0xffffffffu, bz, rl);
                        if (lane == 0) {
                            const float r = v.best[Q(l)].w;
                            v.key[Q(l)] = rk;
                            v.key2[Q(l)] = rk2;
                            v.best[Q(l)] = make_float4(wx, wy, wz, r);
                            v.ct[Q(l)].w = prune_threshold(r, rk);
                        }
                    };
                    if constexpr (FAST) {
                        // ---- prune test of my records (bit b of um: record b * NT + my is kept)
                        uint32_t um = 0;
                        if constexpr (NREG > 0) {
                            const bool h0 = my < nloc, h1 = NREG == 2 && my + NT < nloc;
                            const bool k0 = h0 && (first || !a.prune || !prune_by_threshold(ct0, sx, sy, sz) ||
                                                   (two && !prune_by_threshold(ct0, tx, ty, tz)));
                            const bool k1 = h1 && (first || !a.prune || !prune_by_threshold(ct1, sx, sy, sz) ||
                                                   (two && !prune_by_threshold(ct1, tx, ty, tz)));
                            um = (k0 ? 1u : 0u) | (k1 ? 2u : 0u);
                            if (COUNTERS && !first) {
                                cn.tests += (h0 ? 1 : 0) + (h1 ? 1 : 0);
                                cn.pruned += (h0 && !k0 ? 1 : 0) + (h1 && !k1 ? 1 : 0);
                                if (h0 && !k0) cn.pviol += shadow_record(my);
                                if (h1 && !k1) cn.pviol += shadow_record(my + NT);
                            }
                        } else {
                            for (int b = 0; b < nb; ++b) {
                                const uint32_t l = static_cast<uint32_t>(b) * NT + my;
                                if (l < nloc) {
                                    const float4 ctl = v.ct[Q(l)];
                                    const bool keep = first || !a.prune || !prune_by_threshold(ctl, sx, sy, sz) ||
                                                      (two && !prune_by_threshold(ctl, tx, ty, tz));
                                    um |= keep ? (1u << b) : 0u;
                                    if (COUNTERS && !first) {
                                        ++cn.tests;
                                        cn.pruned += keep ? 0 : 1;
                                        if (!keep) cn.pviol += shadow_record(l);
                                    }
                                }
                            }
                        }
                        // ---- partial max over my records that are not revisited this iteration
                        const bool lrec_visited = lrec != 0xffffffffu && ((um >> (lrec / NT)) & 1u);
                        if (dirty || lrec_visited) {
                            lkey = 0ull;
                            lkey2 = 0ull;
                            lrec = 0xffffffffu;
                            for (int b = 0; b < (NREG > 0 ? NREG : nb); ++b) {
                                const uint32_t l = static_cast<uint32_t>(b) * NT + my;
                                if (l < nloc && !((um >> b) & 1u)) {
                                    const unsigned long long kk = v.key[Q(l)];
                                    if (kk > lkey) {
                                        lkey2 = max(lkey, v.key2[Q(l)]);
                                        lkey = kk;
                                        lrec = l;
                                    } else {
                                        lkey2 = max(lkey2, kk);
                                    }
                                }
                            }
                        }
                        dirty = um != 0;
                        vis = um;
                        pk = lkey;
                        pk2 = lkey2;
                        prec = lrec;
                        // ---- one warp per unpruned record: every warp visits the records its own lanes
                        // hold (record l belongs to slot l mod NT, and consecutive records, which are
                        // neighbours in Morton order, fall to different warps).  Record state is then
                        // touched by one warp only, so the record work needs no CTA barrier: the selection
                        // below is the iteration's only wait.
                        uint32_t rem = um;
                        for (;;) {
                            const uint32_t ball = __ballot_sync(0xffffffffu, rem != 0u);
                            if (!ball) break;
                            const int src = __ffs(ball) - 1;
                            const uint32_t mm = __shfl_sync(0xffffffffu, rem, src);
                            const uint32_t l = static_cast<uint32_t>(__ffs(mm) - 1) * NT + static_cast<uint32_t>(src * NW + w);
                            if (lane == src) rem &= rem - 1u;
                            if (!RFPS_IN(l < nloc)) continue;
                            const uint2 rg = v.rng[Q(l)];
                            float bx = 0.f, by = 0.f, bz = 0.f;
                            unsigned long long lk2 = 0ull;
                            const bool in_smem = resident && (rg.x & kResident);
#ifdef RFPS_CHECKED
                            if (!RFPS_IN(in_smem ? (rg.x & ~kResident) + rg.y <= pcap
                                                 : static_cast<uint64_t>(rg.x) + rg.y <= a.n_total))
                                continue;
#endif
                            const unsigned long long lk =
                                !in_smem ? visit_points<PPL, COUNTERS>(a.pts4, a.porig, rg.x, rg.y, first, a.skip, sx,
                                                                       sy, sz, lane, bx, by, bz, cn, two, tx, ty, tz, lk2)
                                : NT >= 512 ? visit_points_smem<COUNTERS>(s_pts, s_orig, rg.x & ~kResident, rg.y,
                                                                          first, a.skip, sx, sy, sz, lane, bx, by, bz, cn,
                                                                          two, tx, ty, tz, lk2)
                                            : visit_points<PPL, COUNTERS>(s_pts, s_orig, rg.x & ~kResident, rg.y, first,
                                                                          a.skip, sx, sy, sz, lane, bx, by, bz, cn, two,
                                                                          tx, ty, tz, lk2);
                            if constexpr (CLUSTER) {
                                // the candidate may now be a visited point (its coordinates are in
                                // registers); the record's own update waits until the candidate is
                                // pushed, overlapping the exchange (one record pending at most)
                                if (lk > pk) {
                                    pk2 = max(pk, lk2);
                                    pk = lk;
                                    ppt = true;
                                    px = bx;
                                    py = by;
                                    pz = bz;
                                } else {
                                    pk2 = max(pk2, lk);
                                }
                                if (dl != 0xffffffffu) finish_record(dl, dk, dk2, dx, dy, dz);
                                dl = l;
                                dk = lk;
                                dk2 = lk2;
                                dx = bx;
                                dy = by;
                                dz = bz;
                            } else {
                                // one CTA: a CTA barrier follows the selection and nothing would overlap
                                // the update, so it is done here and merged into lane 0's candidate
                                unsigned long long rk;
                                const int rl = warp_argmax_lane(lk, &rk);
                                const unsigned long long rk2 = warp_max_u64(lane == rl ? lk2 : lk);
                                const float wx = __shfl_sync(0xffffffffu, bx, rl);
                                const float wy = __shfl_sync(0xffffffffu, by, rl);
                                const float wz = __shfl_sync(0xffffffffu, bz, rl);
                                if (lane == 0) {
                                    const float r = v.best[Q(l)].w;
                                    v.key[Q(l)] = rk;
                                    v.key2[Q(l)] = rk2;
                                    v.best[Q(l)] = make_float4(wx, wy, wz, r);
                                    v.ct[Q(l)].w = prune_threshold(r, rk);
                                    if (rk > pk) {
                                        pk2 = max(pk, rk2);
                                        pk = rk;
                                        prec = l;
                                    } else {
                                        pk2 = max(pk2, rk);
                                    }
                                }
                            }
                        }
                    } else {
                        // one warp updates record l (global memory; point range rg, covering radius r):
                        // its points' distances, then its key, best point and prune threshold in global
                        // memory.  The new key and best point are returned to every lane.
                        auto visit_global = [&](uint32_t l, uint2 rg, float r, unsigned long long& rk, float& rk2d,
                                                float& wx, float& wy, float& wz) {
                            rk = 0ull;
                            rk2d = 0.f;
                            wx = wy = wz = 0.f;
                            if (!RFPS_IN(l < nloc)) return;
                            const uint32_t k = v.g(l);
#ifdef RFPS_CHECKED
                            if (!RFPS_IN(static_cast<uint64_t>(rg.x) + rg.y <= a.n_total)) return;
#endif
                            float bx = 0.f, by = 0.f, bz = 0.f;
                            unsigned long long lk2;
                            const unsigned long long lk = visit_points<PPL, COUNTERS>(
                                a.pts4, a.porig, rg.x, rg.y, first, a.skip, sx, sy, sz, lane, bx, by, bz, cn, two, tx,
                                ty, tz, lk2);
                            const int wl = warp_argmax_lane(lk, &rk);
                            rk2d = key_d2(warp_max_u64(lane == wl ? lk2 : lk));
                            wx = __shfl_sync(0xffffffffu, bx, wl);
                            wy = __shfl_sync(0xffffffffu, by, wl);
                            wz = __shfl_sync(0xffffffffu, bz, wl);
                            if (lane == 0) {
                                a.rec_key[k] = rk;
                                a.rec_best[k] = make_float4(wx, wy, wz, rk2d);
                                a.rec_thr[k] = prune_threshold(r, rk);
                            }
                        };
                        // ---- A1: prune test of my super-records; unpruned ones to the super list
                        for (uint32_t g0s = 0; g0s < G; g0s += 32u * NT) {
                            uint32_t su = 0;
                            for (int b = 0; b < 32; ++b) {
                                const uint32_t g = g0s + static_cast<uint32_t>(b) * NT + my;
                                if (g >= G) break;
                                const bool keep = first || !a.prune || !prune_by_threshold(s_sct[g], sx, sy, sz) ||
                                                  (two && !prune_by_threshold(s_sct[g], tx, ty, tz));
                                su |= keep ? (1u << b) : 0u;
                                if (COUNTERS && !first) {
                                    ++cn.tests;
                                    cn.pruned += keep ? 0 : 1;
                                    if (!keep) {   // every record of the pruned super-record
                                        for (uint32_t l = g * 32; l < min(nloc, g * 32 + 32); ++l) {
                                            const uint2 rg = a.rec_rng[v.g(l)];
                                            cn.pviol += shadow_pruned(a.pts4, rg.x, rg.y, sx, sy, sz) +
                                                        (two ? shadow_pruned(a.pts4, rg.x, rg.y, tx, ty, tz) : 0);
                                        }
                                    }
                                }
                            }
                            const uint32_t nkeep = __popc(su);
                            uint32_t incl = nkeep;
    #pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += u;
                            }
                            const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
                            if (wtot) {
                                uint32_t base = 0;
                                if (lane == 31) base = atomicAdd(&s_wlc[par], wtot);
                                base = __shfl_sync(0xffffffffu, base, 31);
                                uint32_t pos = base + incl - nkeep;
                                for (uint32_t mm = su; mm; mm &= mm - 1)
                                    s_slist[pos++] = g0s + static_cast<uint32_t>(__ffs(mm) - 1) * NT + my;
                            }
                        }
                        __syncthreads();
                        if (CLUSTER && s_abort) break;   // uniform: read after the barrier
                        if (t == 0) {
                            s_wlc[par ^ 1] = 0;
                            s_rlc[par ^ 1] = 0;
                            s_rlcut[par ^ 1] = W;
                        }
                        const uint32_t nsl = s_wlc[par];
                        // ---- A2: records of the unpruned super-records (one per lane).  Each record's
                        // sphere, threshold, point range, key and best point come in one round of
                        // loads; unpruned records go to the record list with their range and radius (or
                        // are visited in place when the list is full).  The max key over the others,
                        // which this iteration leaves unchanged, and its point go into the super-record's
                        // key and best point (read by nothing before the refresh in C rewrites them).
                        for (uint32_t i = w; i < nsl; i += NW) {
                            const uint32_t g = s_slist[i];
                            if (!RFPS_IN(g < G)) continue;
                            const uint32_t l = g * 32 + lane;
                            bool keep = false;
                            uint2 rg = make_uint2(0u, 0u);
                            unsigned long long kk = 0ull;
                            float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            float rad = 0.f;
                            if (l < nloc) {
                                const uint32_t k = v.g(l);
                                const float4 sp = a.rec_sph[k];
                                const float thr = a.rec_thr[k];
                                rg = a.rec_rng[k];
                                kk = a.rec_key[k];
                                b4 = a.rec_best[k];
                                rad = sp.w;
                                const float4 ctr = make_float4(sp.x, sp.y, sp.z, thr);
                                keep = first || !a.prune || !prune_by_threshold(ctr, sx, sy, sz) ||
                                       (two && !prune_by_threshold(ctr, tx, ty, tz));
                                if (COUNTERS && !first) {
                                    ++cn.tests;
                                    cn.pruned += keep ? 0 : 1;
                                    if (!keep && a.prune)
                                        cn.pviol += shadow_pruned(a.pts4, rg.x, rg.y, sx, sy, sz) +
                                                    (two ? shadow_pruned(a.pts4, rg.x, rg.y, tx, ty, tz) : 0);
                                }
                            }
                            unsigned long long pmk;
                            const int pl = warp_argmax_lane(keep ? 0ull : kk, &pmk);
                            // bound on the unchanged records' keys but pmk: the others' maxima and pmk's
                            // record's second key
                            float sk2d = fmaxf(key_d2(warp_max_u64(keep || lane == pl ? 0ull : kk)),
                                               pmk != 0ull ? __shfl_sync(0xffffffffu, b4.w, pl) : 0.f);
                            float px4 = __shfl_sync(0xffffffffu, b4.x, pl);
                            float py4 = __shfl_sync(0xffffffffu, b4.y, pl);
                            float pz4 = __shfl_sync(0xffffffffu, b4.z, pl);
                            uint32_t mask = __ballot_sync(0xffffffffu, keep);
                            uint2 ent = make_uint2(0u, 0u);
                            if (mask) {
                                uint32_t base = 0;
                                if (lane == 0) base = atomicAdd(&s_rlc[par], static_cast<uint32_t>(__popc(mask)));
                                base = __shfl_sync(0xffffffffu, base, 0);
                                if (base + __popc(mask) <= W) {
                                    if (keep) {
                                        const uint32_t e = base + __popc(mask & ((1u << lane) - 1u));
                                        s_rlist[e] = l;
                                        s_rrng[e] = rg;
                                        s_rxyz[e] = make_float4(0.f, 0.f, 0.f, rad);
                                    }
                                    ent = make_uint2(base, static_cast<uint32_t>(__popc(mask)));
                                } else {
                                    // list full: later appends fail too, so the list holds [0, first failed base)
                                    if (lane == 0) atomicMin(&s_rlcut[par], base);
                                    while (mask) {
                                        const int src = __ffs(mask) - 1;
                                        mask &= mask - 1;
                                        const uint2 rs = make_uint2(__shfl_sync(0xffffffffu, rg.x, src),
                                                                    __shfl_sync(0xffffffffu, rg.y, src));
                                        const float rr = __shfl_sync(0xffffffffu, rad, src);
                                        unsigned long long rk;
                                        float rk2d, wx, wy, wz;
                                        visit_global(g * 32 + static_cast<uint32_t>(src), rs, rr, rk, rk2d, wx, wy, wz);
                                        if (rk > pmk) {
                                            sk2d = fmaxf(sk2d, fmaxf(key_d2(pmk), rk2d));
                                            pmk = rk;
                                            px4 = wx;
                                            py4 = wy;
                                            pz4 = wz;
                                        } else {
                                            sk2d = fmaxf(sk2d, key_d2(rk));
                                        }
                                    }
                                }
                            }
                            if (lane == 0) {
                                s_skey[g] = pmk;
                                s_sk2[g] = sk2d;
                                s_sxyz[g] = make_float4(px4, py4, pz4, s_sxyz[g].w);
                                s_sent[g] = ent;
                            }
                        }
                        __syncthreads();
                        // ---- B: one warp per listed record; its new key and best point also go to the list
                        const uint32_t nrl = min(min(s_rlc[par], s_rlcut[par]), W);
                        for (uint32_t e = w; e < nrl; e += NW) {
                            const float r = s_rxyz[e].w;
                            unsigned long long rk;
                            float rk2d, wx, wy, wz;
                            visit_global(s_rlist[e], s_rrng[e], r, rk, rk2d, wx, wy, wz);
                            if (lane == 0) {
                                s_rkey[e] = rk;
                                s_rk2[e] = rk2d;
                                s_rxyz[e] = make_float4(wx, wy, wz, r);
                            }
                        }
                        __syncthreads();
                        // ---- C: refresh the unpruned super-records: max of the records left unchanged (A2)
                        // and of the ones visited (B), from shared memory
                        for (uint32_t i = w; i < nsl; i += NW) {
                            const uint32_t g = s_slist[i];
                            if (!RFPS_IN(g < G)) continue;
                            const uint2 ent = s_sent[g];
                            if (!RFPS_IN(ent.x + ent.y <= W)) continue;
                            unsigned long long kk = 0ull;
                            float k2d = 0.f;
                            if (static_cast<uint32_t>(lane) < ent.y) {
                                kk = s_rkey[ent.x + lane];
                                k2d = s_rk2[ent.x + lane];
                            }
                            unsigned long long gk;
                            const int gl = warp_argmax_lane(kk, &gk);
                            // the visited records' other keys: the second-largest max and the winner's
                            // second key
                            const float vk2d = fmaxf(key_d2(warp_max_u64(lane == gl ? 0ull : kk)),
                                                     __shfl_sync(0xffffffffu, k2d, gl));
                            if (lane == 0) {
                                const unsigned long long pmk = s_skey[g];   // unchanged records (A2)
                                float4 bx = s_sxyz[g];
                                const float srad = bx.w;
                                float sk2d = s_sk2[g];                        // their other keys (A2)
                                if (gk > pmk) {
                                    bx = s_rxyz[ent.x + gl];
                                    sk2d = fmaxf(fmaxf(sk2d, key_d2(pmk)), vk2d);
                                } else {
                                    sk2d = fmaxf(sk2d, key_d2(gk));
                                    gk = pmk;
                                }
                                s_skey[g] = gk;
                                s_sk2[g] = sk2d;
                                s_sxyz[g] = make_float4(bx.x, bx.y, bx.z, srad);
                                s_sct[g].w = prune_threshold(srad, gk);
                            }
                        }
                        __syncthreads();
                        // ---- D: my super-records' max, and a bound on every other key of them (the
                        // second-largest max, and the winner's bound, as the largest key of that distance)
                        pk = 0ull;
                        pk2 = 0ull;
                        prec = 0xffffffffu;
                        for (uint32_t g = my; g < G; g += NT) {
                            const unsigned long long kk = s_skey[g];
                            if (kk > pk) {
                                pk2 = pk;
                                pk = kk;
                                prec = g;
                            } else if (kk > pk2) {
                                pk2 = kk;
                            }
                        }
                        if (prec != 0xffffffffu) pk2 = max(pk2, make_key(s_sk2[prec], 0u));
                    }
                    // ---- selection: warp -> CTA -> cluster
                    __syncwarp();
                    // 128-thread clusters: each lane loads its own candidate's coordinates (a visited
                    // point's are in registers already) while the warp reduces, and the winner's arrive
                    // by shuffle, one shuffle and a dependent shared load shorter than fetching the
                    // winning record's best point after the reduction.  With 8 or 16 warps per CTA the
                    // extra loads cost more than that (measured), so larger CTAs keep the fetch.
                    constexpr bool OWN_XYZ = FAST && CLUSTER && NT == 128;
                    float ox = 0.f, oy = 0.f, oz = 0.f;
                    if constexpr (OWN_XYZ) {
                        ox = px;
                        oy = py;
                        oz = pz;
                        if (!ppt && prec != 0xffffffffu && RFPS_IN(prec < nloc)) {
                            const float4 b4 = v.best[Q(prec)];
                            ox = b4.x;
                            oy = b4.y;
                            oz = b4.z;
                        }
                    }
                    unsigned long long wk;
                    const int wl = warp_argmax_lane(pk, &wk);
                    // every key of this warp's records other than its candidate is at most wb (the
                    // runner-up shortcut below needs it; the hierarchical path gives no bound)
                    float wbd = __int_as_float(0x7f800000);
                    wbd = key_d2(warp_max_u64(lane == wl ? pk2 : pk));
                    const uint32_t wr = OWN_XYZ ? 0u : __shfl_sync(0xffffffffu, prec, wl);
                    bool wpt = false;                 // the warp's candidate coordinates are in vxyz
                    float4 vxyz = make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (OWN_XYZ) {
                        wpt = true;
                        vxyz.x = __shfl_sync(0xffffffffu, ox, wl);
                        vxyz.y = __shfl_sync(0xffffffffu, oy, wl);
                        vxyz.z = __shfl_sync(0xffffffffu, oz, wl);
                    } else if constexpr (FAST && CLUSTER) {
                        wpt = __shfl_sync(0xffffffffu, ppt, wl);   // the candidate is a point visited now
                        if (wpt) {
                            vxyz.x = __shfl_sync(0xffffffffu, px, wl);
                            vxyz.y = __shfl_sync(0xffffffffu, py, wl);
                            vxyz.z = __shfl_sync(0xffffffffu, pz, wl);
                        }
                    }
                    float4 cxyz = make_float4(0.f, 0.f, 0.f, 0.f);
                    unsigned long long gbest;
                    bool nsc = false;                 // the next round applies two samples
                    unsigned long long nk2 = 0ull;
                    float ntx = 0.f, nty = 0.f, ntz = 0.f;
                    if (!CLUSTER) {
                        // each warp publishes its candidate's key and coordinates (the record's owner
                        // may rewrite its best point in the next iteration, before a slower warp reads it)
                        if (lane == 0) {
                            s_wkey[par][w] = wk;
                            float4 b4 = wk != 0ull && RFPS_IN(wr < (FAST ? nloc : G))
                                            ? (FAST ? v.best[Q(wr)] : s_sxyz[wr]) : make_float4(0.f, 0.f, 0.f, 0.f);
                            b4.w = wbd;   // this warp's bound on its other keys
                            s_wxyz[par][w] = b4;
                        }
                        if constexpr (NREG > 0) {   // thresholds rewritten by this iteration's visits
                            if (vis & 1u) ct0.w = v.ct[Q(my)].w;
                            if (NREG == 2 && (vis & 2u)) ct1.w = v.ct[Q(my + NT)].w;
                        }
                        __syncthreads();
                        const unsigned long long ck = lane < NW ? s_wkey[par][lane] : 0ull;
                        const int cl = warp_argmax_lane(ck, &gbest);
                        cxyz = s_wxyz[par][cl];
                        {   // the runner-up shortcut over the CTA's warps
                            unsigned long long rk2;
                            const int cl2 = warp_argmax_lane(lane == cl ? 0ull : ck, &rk2);
                            const float4 r4 = s_wxyz[par][cl2];
                            const float rd = key_d2(rk2);
                            nsc = j + 2 < c.m && rk2 != 0ull && rd > 0.f && rd > cxyz.w &&
                                  sq_dist(r4.x, r4.y, r4.z, cxyz.x, cxyz.y, cxyz.z) >= rd;
                            nk2 = rk2;
                            ntx = r4.x;
                            nty = r4.y;
                            ntz = r4.z;
                        }
                    } else {
                        // Every warp pushes its best (key, xyz) by st.async into slot [rank][warp] of every
                        // CTA; each CTA's barrier for this round expects C * NW * 24 bytes.  (Reducing in the
                        // CTA first and pushing one candidate per CTA has a lower isolated floor at 16 CTAs
                        // but adds a CTA barrier after the record work, and measured slower in the kernel.)
                        const uint32_t buf = it & 1u, ph = (it >> 1) & 1u;
                        ++it;
                        const uint32_t nslot = C * NW;
                        if (t == 0) mbar_arrive_expect_tx(&s_mbar[buf], 24u * nslot);
                        float4 wxyz = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (wpt) wxyz = vxyz;
                        else if (wk != 0ull && lane < static_cast<int>(C) && RFPS_IN(wr < (FAST ? nloc : G)))
                            wxyz = FAST ? v.best[Q(wr)] : s_sxyz[wr];
                        wxyz.w = wbd;
                        // (counting kernels: a lost round sends nothing, so its waits run out)
                        if (lane < static_cast<int>(C) && !(COUNTERS && j == a.lost_iter)) {
                            const uint32_t rb = buf ? rbar1 : rbar0;
                            st_async_u64(buf ? rkey1 : rkey0, wk, rb);
                            st_async_f32x4(buf ? rxyz1 : rxyz0, wxyz, rb);
                        }
                        if constexpr (FAST) {   // the last visited record's update overlaps the exchange
                            if (dl != 0xffffffffu) finish_record(dl, dk, dk2, dx, dy, dz);
                            __syncwarp();
                            if constexpr (NREG > 0) {   // thresholds rewritten by this iteration's visits
                                if (vis & 1u) ct0.w = v.ct[Q(my)].w;
                                if (NREG == 2 && (vis & 2u)) ct1.w = v.ct[Q(my + NT)].w;
                            }
                        }
                        if (!__all_sync(0xffffffffu,
                                        mbar_wait_bounded(&s_mbar[buf], ph, COUNTERS ? a.spin_limit : kSpinLimit))) {
                            if (lane == 0) atomicCAS(&a.hdr->status, 0u, kStatusTimeout);
                            s_abort = 1;
                            // the fast path has no CTA barrier per iteration: this warp leaves on its own,
                            // and the other warps of the cluster time out in turn (each wait bounded)
                            if (FAST) break;
                        }
                        // 128-thread CTAs load each slot's coordinates with its key, and the winner's
                        // arrive by shuffle instead of a shared load after the reduction (measured
                        // faster there, slower with 256 threads, whose lanes read four slots each)
                        constexpr bool SLOT_XYZ = NT == 128;
                        unsigned long long kk = 0ull, kk2 = 0ull;
                        uint32_t ki = 0, ki2 = 0;
                        float4 kx = make_float4(0.f, 0.f, 0.f, 0.f);
    #pragma unroll
                        for (int u = 0; u < NSLOT / 32; ++u) {   // every slot, unrolled; unused ones read as 0
                            const uint32_t q = static_cast<uint32_t>(u * 32 + lane);
                            const unsigned long long x = q < nslot ? s_ckey[buf][q] : 0ull;
                            float4 xq = make_float4(0.f, 0.f, 0.f, 0.f);
                            if constexpr (SLOT_XYZ) {
                                if (q < nslot) xq = s_cxyz[buf][q];
                            }
                            if (x > kk) {
                                kk2 = kk;
                                ki2 = ki;
                                kk = x;
                                ki = q;
                                kx = xq;
                            } else if (x > kk2) {
                                kk2 = x;
                                ki2 = q;
                            }
                        }
                        const int gl = warp_argmax_lane(kk, &gbest);
                        {
                            // Runner-up shortcut (exact): r, the best of the other slots, is the next
                            // sample if every other key is below it (the winning warp's bound), its
                            // distance is positive, and the update by this sample leaves it unchanged:
                            // every other key only decreases, and this sample's own becomes 0.
                            unsigned long long rk2;
                            const int gl2 = warp_argmax_lane(lane == gl ? kk2 : kk, &rk2);
                            const uint32_t si = __shfl_sync(0xffffffffu, lane == gl ? ki2 : ki, gl2);
                            const uint32_t wi = __shfl_sync(0xffffffffu, ki, gl);
                            const float4 r4 = s_cxyz[buf][si];
                            const float4 w4 = s_cxyz[buf][wi];
                            const float rd = key_d2(rk2);
                            nsc = j + 2 < c.m && !(COUNTERS && a.lost_iter != 0) && rk2 != 0ull && rd > 0.f &&
                                  rd > w4.w && sq_dist(r4.x, r4.y, r4.z, w4.x, w4.y, w4.z) >= rd;
                            nk2 = rk2;
                            ntx = r4.x;
                            nty = r4.y;
                            ntz = r4.z;
                        }
                        if constexpr (SLOT_XYZ) {
                            cxyz.x = __shfl_sync(0xffffffffu, kx.x, gl);
                            cxyz.y = __shfl_sync(0xffffffffu, kx.y, gl);
                            cxyz.z = __shfl_sync(0xffffffffu, kx.z, gl);
                        } else {
                            ki = __shfl_sync(0xffffffffu, ki, gl);
                            cxyz = s_cxyz[buf][ki];
                        }
                    }
                    sx = cxyz.x;
                    sy = cxyz.y;
                    sz = cxyz.z;
                    if (rank == 0 && t == 0) {
                        a.out[c.out_off + (resume ? j - 1 : j)] = static_cast<int64_t>(key_index(gbest)) - c.pt_off;
                        if (nsc) a.out[c.out_off + (resume ? j : j + 1)] = static_cast<int64_t>(key_index(nk2)) - c.pt_off;
                    }
                    two = nsc;
                    tx = ntx;
                    ty = nty;
                    tz = ntz;
                    const int64_t step = nsc ? 2 : 1;
                    if (COUNTERS) {
                        cn.iter += static_cast<uint64_t>(step);
                        ++cn.rounds;
                    }
                    j += step;
                }
            };
            if (!fast) iterate(IntC<0>{});
            else if (NT <= 256 && nb <= 1) iterate(IntC<NT <= 256 ? 1 : 3>{});
            else if (NT <= 256 && nb == 2) iterate(IntC<NT <= 256 ? 2 : 3>{});
            else iterate(IntC<3>{});
            if (a.save_state) {
                // state for a later resume: records kept in shared memory, resident points'
                // distances, and the last selected sample (every CTA holds the same one)
                __syncthreads();
                if (fast) {
                    for (uint32_t l = t; l < nloc; l += NT) {
                        const uint32_t k = v.g(l);
                        a.rec_key[k] = v.key[v.at(l)];
                        a.rec_best[k] = v.best[v.at(l)];
                        a.rec_thr[k] = v.ct[v.at(l)].w;
                    }
                    if (resident) {
                        for (uint32_t l = w; l < nloc; l += NW) {
                            const uint2 rg = v.rng[v.at(l)];
                            if (!(rg.x & kResident)) continue;
                            const uint32_t go = a.rec_rng[v.g(l)].x, so = rg.x & ~kResident;
                            for (uint32_t q = lane; q < rg.y; q += 32) a.pts4[go + q].w = s_pts[so + q].w;
                        }
                    }
                }   // the hierarchical path keeps its records in global memory throughout
                if (rank == 0 && t == 0) {
                    a.clouds[cloud].last[0] = sx;
                    a.clouds[cloud].last[1] = sy;
                    a.clouds[cloud].last[2] = sz;
                }
            }
        }
        if (CLUSTER) {
            // leave together: a CTA that gave up on a wait ends the loop for the whole cluster (one
            // that left alone would strand the others at the next cluster barrier).  Thread r reads
            // rank r's flag; the second barrier keeps every CTA alive until all have read.
            cluster_sync();
            uint32_t ab = 0;
            if (t < static_cast<int>(C)) ab = ld_cluster_u32(map_shared(&s_abort, static_cast<uint32_t>(t)));
            ab = __syncthreads_or(ab);
            cluster_sync();
            if (ab) break;
        } else {
            __syncthreads();
        }
    }
    if (COUNTERS) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[0]), cn.tests);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[1]), cn.pruned);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[2]), cn.visit);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[3]), cn.skip);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[4]), cn.upd);
        if (t == 0 && rank == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[5]), cn.iter);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[8]), cn.rounds);
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[6]), cn.pviol);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[7]), cn.sviol);
    }
}

// Register-record sampler for small clouds on one CTA (N <= NT * P): thread t holds the P sorted
// points [t P, t P + P) of the cloud in registers -- Morton-consecutive, so they are spatial
// neighbours -- and treats them as one record of its own: covering sphere (centre of their bounding
// box, radius measured over them as the build does for voxel records), Dist_v key (max point key)
// with the coordinates of its point, and the FP32-safe prune threshold.  An iteration is the same
// method as k_sample's (radius pruning of the record, point skip, strict update, Dist_v resync,
// Sec. 3.3-3.4) without shared-memory records or warp-serial visits: every thread tests its own
// record and, if it is not pruned, updates its own points; the selection is a warp argmax, one CTA
// barrier and an argmax over the warps.  On one SM the per-warp cost of the record-visiting
// loop sets the iteration time of small clouds (every warp runs ~280 instructions an iteration at
// 4,096 points on 512 threads), which this form avoids.  A record whose distances did not change
// keeps its key and threshold.
//
// FUSED: the kernel groups the cloud itself instead of reading the index build's sorted arrays:
// it reads the caller's points, checks that they are finite (RFPS_ENONFINITE otherwise), sorts
// them in shared memory by the Morton code of a 1,024^3 grid over their bounding box (bitonic sort
// of (code, row) pairs), and hands thread t the sorted points [tP, tP + P).  A call then launches
// two kernels (the cloud table and this one) instead of the index build's thirty.  Any grouping
// is correct, since the bound holds for any record sphere that covers its points; the Morton
// order keeps the records compact.  Not for a kept index, whose state lives in the build's arrays.
template <int NT, int P, bool COUNTERS, bool FUSED>
__global__ void __launch_bounds__(NT, 1) k_sample_regs(const SampleArgs a)
{
    constexpr int NW = NT / 32;
    __shared__ unsigned long long s_wkey[2][NW];
    __shared__ float4 s_wxyz[2][NW];
    __shared__ uint32_t s_item;
    __shared__ unsigned long long s_sort[FUSED ? NT * P : 1];
    __shared__ float s_box[6][NW];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    Cnt cn;
    for (;;) {
        if (t == 0) {
            uint32_t item = atomicAdd(&a.hdr->work, 1u);
            if (*static_cast<volatile uint32_t*>(&a.hdr->status) != 0u) item = 0xffffffffu;
            s_item = item;
        }
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();   // every thread has read s_item before thread 0 may rewrite it
        if (item >= a.n_clouds) break;
        const uint32_t cloud = a.order[item];
        const CloudDev c = a.clouds[cloud];
        if (c.valid && RFPS_IN(c.n <= static_cast<int64_t>(NT) * P)) {
            const bool resume = c.resume != 0;
            // the cloud's points occupy sorted positions [pt_off, pt_off + n)
            const uint32_t base = static_cast<uint32_t>(c.pt_off);
            const uint32_t n = static_cast<uint32_t>(c.n);
            const uint32_t q0 = static_cast<uint32_t>(t) * P;
            float px[P], py[P], pz[P], pd[P];
            uint32_t po[P];
            float lo[3] = {3.4028234e38f, 3.4028234e38f, 3.4028234e38f};
            float hi[3] = {-3.4028234e38f, -3.4028234e38f, -3.4028234e38f};
            bool grouped = true;
            if constexpr (FUSED) {
                // bounding box and finiteness of the caller's points
                const float* src = a.pts + 3 * c.pt_off;
                float mn[3] = {3.4028234e38f, 3.4028234e38f, 3.4028234e38f};
                float mx[3] = {-3.4028234e38f, -3.4028234e38f, -3.4028234e38f};
                int bad = 0;
                for (uint32_t i = t; i < n; i += NT) {
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const float x = src[3 * static_cast<size_t>(i) + ax];
                        bad |= !(fabsf(x) <= 3.4028234e38f);
                        mn[ax] = fminf(mn[ax], x);
                        mx[ax] = fmaxf(mx[ax], x);
                    }
                }
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    for (int o = 16; o > 0; o >>= 1) {
                        mn[ax] = fminf(mn[ax], __shfl_xor_sync(0xffffffffu, mn[ax], o));
                        mx[ax] = fmaxf(mx[ax], __shfl_xor_sync(0xffffffffu, mx[ax], o));
                    }
                    if (lane == 0) {
                        s_box[ax][w] = mn[ax];
                        s_box[3 + ax][w] = mx[ax];
                    }
                }
                if (__syncthreads_or(bad)) {
                    if (t == 0) atomicCAS(&a.hdr->status, 0u, kStatusNonFinite);
                    grouped = false;
                } else {
                    float sc[3];
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        for (int k = 0; k < NW; ++k) {
                            mn[ax] = fminf(mn[ax], s_box[ax][k]);
                            mx[ax] = fmaxf(mx[ax], s_box[3 + ax][k]);
                        }
                        const float e = mx[ax] - mn[ax];
                        sc[ax] = e > 0.f ? 1023.0f / e : 0.f;
                    }
                    // (Morton code << 32 | row) pairs, padded to a power of two with the largest key
                    const uint32_t np2 = n > 1 ? 1u << (32 - __clz(n - 1)) : 1u;
                    for (uint32_t i = t; i < np2; i += NT) {
                        unsigned long long kk = ~0ull;
                        if (i < n) {
                            uint32_t cq[3];
#pragma unroll
                            for (int ax = 0; ax < 3; ++ax) {
                                const float f = (src[3 * static_cast<size_t>(i) + ax] - mn[ax]) * sc[ax];
                                cq[ax] = static_cast<uint32_t>(fminf(1023.f, fmaxf(0.f, f)));
                            }
                            kk = (static_cast<unsigned long long>(morton3(cq[0], cq[1], cq[2])) << 32) |
                                 static_cast<uint32_t>(c.pt_off + i);
                        }
                        s_sort[i] = kk;
                    }
                    __syncthreads();
                    for (uint32_t k = 2; k <= np2; k <<= 1) {
                        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                            for (uint32_t i = t; i < np2; i += NT) {
                                const uint32_t ixj = i ^ j;
                                if (ixj > i) {
                                    const unsigned long long x = s_sort[i], y = s_sort[ixj];
                                    if ((x > y) == ((i & k) == 0)) {
                                        s_sort[i] = y;
                                        s_sort[ixj] = x;
                                    }
                                }
                            }
                            __syncthreads();
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const uint32_t q = q0 + u;
                px[u] = py[u] = pz[u] = 0.f;
                pd[u] = 0.f;
                po[u] = 0u;
                // (a cloud that failed its checks was not sorted: nothing of it is read)
                if (q < n && grouped) {
                    float4 p4;
                    if constexpr (FUSED) {
                        po[u] = static_cast<uint32_t>(s_sort[q]);   // row of the q-th point in Morton order
#ifdef RFPS_CHECKED
                        if (!RFPS_IN(po[u] >= c.pt_off && po[u] < c.pt_off + c.n)) po[u] = static_cast<uint32_t>(c.pt_off);
#endif
                        p4 = make_float4(a.pts[3 * static_cast<size_t>(po[u])], a.pts[3 * static_cast<size_t>(po[u]) + 1],
                                         a.pts[3 * static_cast<size_t>(po[u]) + 2], inf);
                    } else {
                        p4 = a.pts4[base + q];
                        po[u] = a.porig[base + q];
                    }
                    px[u] = p4.x;
                    py[u] = p4.y;
                    pz[u] = p4.z;
                    pd[u] = resume ? p4.w : inf;   // +inf: the initial update of Sec. 3.3
                    lo[0] = fminf(lo[0], p4.x);
                    lo[1] = fminf(lo[1], p4.y);
                    lo[2] = fminf(lo[2], p4.z);
                    hi[0] = fmaxf(hi[0], p4.x);
                    hi[1] = fmaxf(hi[1], p4.y);
                    hi[2] = fmaxf(hi[2], p4.z);
                }
            }
            const bool has = q0 < n && grouped;
            // covering sphere: any centre, radius r = max(fl(m (1 + 2^-20)), 2^-50) with
            // m = max over the members of sqrt(fl d2(p, c)) (the voxel records' rule)
            const float cx = __fmul_rn(__fadd_rn(lo[0], hi[0]), 0.5f);
            const float cy = __fmul_rn(__fadd_rn(lo[1], hi[1]), 0.5f);
            const float cz = __fmul_rn(__fadd_rn(lo[2], hi[2]), 0.5f);
            float m = 0.f;
#pragma unroll
            for (int u = 0; u < P; ++u)
                if (q0 + u < n) m = fmaxf(m, __fsqrt_rn(sq_dist(px[u], py[u], pz[u], cx, cy, cz)));
            const float rad = fmaxf(__fmul_rn(m, 0x1.00001p0f), 0x1p-50f);
            // Dist_v key of the record and its point, from the distances it starts with (+inf, or the
            // saved ones), and the second-largest point key; they change only when a distance does
            unsigned long long key = 0ull, key2 = 0ull;
            float bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
            for (int u = 0; u < P; ++u) {
                if (q0 + u < n) {
                    const unsigned long long kk = make_key(pd[u], po[u]);
                    if (kk > key) {
                        key2 = key;
                        key = kk;
                        bx = px[u];
                        by = py[u];
                        bz = pz[u];
                    } else if (kk > key2) {
                        key2 = kk;
                    }
                }
            }
            float4 ct = make_float4(cx, cy, cz, resume ? prune_threshold(rad, key) : nan);
            const int64_t g0 = c.pt_off + c.start;
            float sx = resume ? c.last[0] : a.pts[3 * g0 + 0];
            float sy = resume ? c.last[1] : a.pts[3 * g0 + 1];
            float sz = resume ? c.last[2] : a.pts[3 * g0 + 2];
            if (t == 0 && !resume) a.out[c.out_off] = c.start;
            // a second sample applied in the same round (the runner-up shortcut of k_sample's
            // clusters, here over the CTA's warps)
            bool two = false;
            float tx = 0.f, ty = 0.f, tz = 0.f;
            int64_t rnd = 0;
            for (int64_t j = 1; grouped && j < c.m; ++rnd) {   // (a cloud that failed its checks: none)
                const bool first = (j == 1) && !resume;
                const int par = static_cast<int>(rnd & 1);
                const bool keep_s = has && (first || !a.prune || !prune_by_threshold(ct, sx, sy, sz));
                const bool keep_t = has && two && (!a.prune || !prune_by_threshold(ct, tx, ty, tz));
                if (COUNTERS && !first && has) {
                    ++cn.tests;
                    if (!keep_s && !keep_t) ++cn.pruned;
#pragma unroll
                    for (int u = 0; u < P; ++u) {   // shadow check: no pruned point may improve
                        if (q0 + u < n && !keep_s && sq_dist(px[u], py[u], pz[u], sx, sy, sz) < pd[u]) ++cn.pviol;
                        if (q0 + u < n && two && !keep_t && sq_dist(px[u], py[u], pz[u], tx, ty, tz) < pd[u]) ++cn.pviol;
                    }
                }
                if (keep_s || keep_t) {
                    bool changed = false;
#pragma unroll
                    for (int u = 0; u < P; ++u) {
                        if (q0 + u < n) {
                            const float d0 = pd[u];
                            bool sk = true;   // every applied sample skipped the point
#pragma unroll
                            for (int q = 0; q < 2; ++q) {   // the round's samples in order
                                if (q == 0 ? !keep_s : !keep_t) continue;
                                const float dx = __fsub_rn(px[u], q == 0 ? sx : tx);
                                const float dy = __fsub_rn(py[u], q == 0 ? sy : ty);
                                const float dz = __fsub_rn(pz[u], q == 0 ? sz : tz);
                                const float xx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy), zz = __fmul_rn(dz, dz);
                                if (a.skip && skip_point(xx, yy, zz, pd[u])) {
                                    if (COUNTERS && __fadd_rn(__fadd_rn(xx, yy), zz) < pd[u]) ++cn.sviol;
                                } else {
                                    sk = false;
                                    const float nd = __fadd_rn(__fadd_rn(xx, yy), zz);
                                    if (nd < pd[u]) {
                                        pd[u] = nd;
                                        changed = true;
                                    }
                                }
                            }
                            if (COUNTERS) {
                                ++cn.visit;
                                if (sk) ++cn.skip;
                                if (pd[u] < d0) ++cn.upd;
                            }
                        }
                    }
                    // the Dist_v key and threshold change only when a distance did
                    if (changed) {
                        // max and second max over the points' keys as a pairwise tree (empty slots
                        // give key 0)
                        unsigned long long tk[P], t2[P];
                        float ux[P], uy[P], uz[P];
#pragma unroll
                        for (int u = 0; u < P; ++u) {
                            tk[u] = q0 + u < n ? make_key(pd[u], po[u]) : 0ull;
                            t2[u] = 0ull;
                            ux[u] = px[u];
                            uy[u] = py[u];
                            uz[u] = pz[u];
                        }
#pragma unroll
                        for (int h = 1; h < P; h <<= 1) {
#pragma unroll
                            for (int u = 0; u + h < P; u += 2 * h) {
                                if (tk[u + h] > tk[u]) {
                                    t2[u] = max(tk[u], t2[u + h]);
                                    tk[u] = tk[u + h];
                                    ux[u] = ux[u + h];
                                    uy[u] = uy[u + h];
                                    uz[u] = uz[u + h];
                                } else {
                                    t2[u] = max(t2[u], tk[u + h]);
                                }
                            }
                        }
                        key = tk[0];
                        key2 = t2[0];
                        bx = ux[0];
                        by = uy[0];
                        bz = uz[0];
                        ct.w = prune_threshold(rad, key);
                    }
                }
                // selection: warp argmax, one CTA barrier, argmax over the warps.  Each warp also
                // publishes a bound on its other keys (the winning lane's second key, the other
                // lanes' keys) for the runner-up shortcut.
                unsigned long long wk;
                const int wl = warp_argmax_lane(key, &wk);
                const float wbd = key_d2(warp_max_u64(lane == wl ? key2 : key));
                const float wx = __shfl_sync(0xffffffffu, bx, wl);
                const float wy = __shfl_sync(0xffffffffu, by, wl);
                const float wz = __shfl_sync(0xffffffffu, bz, wl);
                if (lane == 0) {
                    s_wkey[par][w] = wk;
                    s_wxyz[par][w] = make_float4(wx, wy, wz, wbd);
                }
                __syncthreads();
                unsigned long long gbest, rk2;
                const unsigned long long ck = lane < NW ? s_wkey[par][lane] : 0ull;
                const int cl = warp_argmax_lane(ck, &gbest);
                const int cl2 = warp_argmax_lane(lane == cl ? 0ull : ck, &rk2);   // the best of the other warps
                const float4 cxyz = s_wxyz[par][cl];
                const float4 rxyz = s_wxyz[par][cl2];
                sx = cxyz.x;
                sy = cxyz.y;
                sz = cxyz.z;
                // the runner-up r is the next sample too (exact) if it beats the winning warp's bound,
                // its distance is positive and the update with this sample leaves it unchanged
                const float rd = key_d2(rk2);
                const bool nsc = j + 2 < c.m && rk2 != 0ull && rd > 0.f && rd > cxyz.w &&
                                 sq_dist(rxyz.x, rxyz.y, rxyz.z, cxyz.x, cxyz.y, cxyz.z) >= rd;
                if (t == 0) {
                    a.out[c.out_off + (resume ? j - 1 : j)] = static_cast<int64_t>(key_index(gbest)) - c.pt_off;
                    if (nsc) a.out[c.out_off + (resume ? j : j + 1)] = static_cast<int64_t>(key_index(rk2)) - c.pt_off;
                }
                two = nsc;
                tx = rxyz.x;
                ty = rxyz.y;
                tz = rxyz.z;
                if (COUNTERS && t == 0) {
                    cn.iter += nsc ? 2 : 1;
                    ++cn.rounds;
                }
                j += nsc ? 2 : 1;
            }
            if (a.save_state) {   // the distances and the last sample, for a later resume
#pragma unroll
                for (int u = 0; u < P; ++u)
                    if (q0 + u < n) a.pts4[base + q0 + u].w = pd[u];
                if (t == 0) {
                    a.clouds[cloud].last[0] = sx;
                    a.clouds[cloud].last[1] = sy;
                    a.clouds[cloud].last[2] = sz;
                }
            }
        }
        __syncthreads();
    }
    if (COUNTERS) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[0]), cn.tests);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[1]), cn.pruned);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[2]), cn.visit);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[3]), cn.skip);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[4]), cn.upd);
        if (t == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[5]), cn.iter);
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[8]), cn.rounds);
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[6]), cn.pviol);
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->counters[7]), cn.sviol);
    }
}

// The per-iteration synchronisation floor of k_sample: the same selection
// tail (warp argmax, CTA slots or DSMEM push, one __syncthreads or one
// barrier.cluster, slot reduction) with no record work.  `sink` receives a
// value that depends on every round so the loop cannot be elided.
template <int NT, bool CLUSTER>
__global__ void __launch_bounds__(NT, 1) k_sync_floor(int64_t iters, unsigned long long* sink, uint32_t* status)
{
    constexpr int NW = NT / 32;
    constexpr int NSLOT = CLUSTER ? kMaxCluster * NW : 1;
    __shared__ unsigned long long s_wkey[2][NW];
    __shared__ unsigned long long s_ckey[2][NSLOT];
    __shared__ float4 s_cxyz[2][NSLOT];
    __shared__ unsigned long long s_mbar[2];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t C = CLUSTER ? cluster_nctarank() : 1u;
    if (CLUSTER && t == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        fence_mbar_init_cluster();
    }
    if (CLUSTER) cluster_sync();
    unsigned long long acc = 0ull;
    unsigned long long pk = make_key(static_cast<float>(t), blockIdx.x * NT + t);
    float sx = 0.f;
    for (int64_t j = 1; j < iters; ++j) {   // a timed-out wait is recorded; every round stays bounded
        const int par = static_cast<int>(j & 1);
        pk = (pk ^ static_cast<unsigned long long>(j)) + static_cast<unsigned long long>(__float_as_uint(sx) & 1u);
        unsigned long long wk, gbest;
        warp_argmax_lane(pk, &wk);
        if (!CLUSTER) {
            if (lane == 0) s_wkey[par][w] = wk;
            __syncthreads();
            const unsigned long long ck = lane < NW ? s_wkey[par][lane] : 0ull;
            warp_argmax_lane(ck, &gbest);
        } else {
            const uint32_t buf = static_cast<uint32_t>(j - 1) & 1u, ph = (static_cast<uint32_t>(j - 1) >> 1) & 1u;
            const uint32_t nslot = C * NW;
            if (t == 0) mbar_arrive_expect_tx(&s_mbar[buf], 24u * nslot);
            if (lane < static_cast<int>(C)) {
                const uint32_t rb = map_shared(&s_mbar[buf], lane);
                st_async_u64(map_shared(&s_ckey[buf][rank * NW + w], lane), wk, rb);
                st_async_f32x4(map_shared(&s_cxyz[buf][rank * NW + w], lane), make_float4(sx, sx, sx, 0.f), rb);
            }
            if (!mbar_wait_bounded(&s_mbar[buf], ph, kSpinLimit)) atomicCAS(status, 0u, kStatusTimeout);
            unsigned long long kk = 0ull;
            uint32_t ki = 0;
            for (uint32_t q = lane; q < nslot; q += 32) {
                const unsigned long long x = s_ckey[buf][q];
                if (x > kk) {
                    kk = x;
                    ki = q;
                }
            }
            const int gl = warp_argmax_lane(kk, &gbest);
            ki = __shfl_sync(0xffffffffu, ki, gl);
            sx = s_cxyz[buf][ki].x + 1.0f;
        }
        acc += gbest;
    }
    if (CLUSTER) cluster_sync();
    if (t == 0) sink[blockIdx.x] = acc;
}

template <int NT, bool CLUSTER, bool COUNTERS>
cudaError_t launch_one(SampleArgs args, int C, int64_t n_clouds, cudaStream_t st)
{
    auto kern = k_sample<NT, CLUSTER, COUNTERS>;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const size_t dyn = static_cast<size_t>(optin) - fa.sharedSizeBytes - 1024;
    args.smem_bytes = dyn;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
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
    if (NT == 128) return launch_one<128, CLUSTER, COUNTERS>(args, C, n_clouds, st);
    return NT == 256 ? launch_one<256, CLUSTER, COUNTERS>(args, C, n_clouds, st)
                     : launch_one<512, CLUSTER, COUNTERS>(args, C, n_clouds, st);
}

// Clouds of at most kRegsNT * kRegsP points on one CTA with records held in registers
// (k_sample_regs), chosen by the options cluster 1, threads 512.  Fewer points per thread shorten
// the chain of an unpruned record: 1,024 threads of 4 points measured 3-5 % faster than 512 of 8
// on 1k-4k-point clouds, 256 of 16 about 40 % slower, and 512 of 16 (to 8,192 points) lost to a
// 16-CTA cluster (6,000-point clouds: 2.2 against 1.8 ms).
constexpr int kRegsNT = 1024;
constexpr int kRegsP = 4;

template <int P, bool COUNTERS, bool FUSED>
cudaError_t launch_regs(const SampleArgs& args, int64_t n_clouds, cudaStream_t st)
{
    auto kern = k_sample_regs<kRegsNT, P, COUNTERS, FUSED>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRegsNT, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = static_cast<int64_t>(per_sm) * sms;
    kern<<<static_cast<unsigned>(n_clouds < cap ? n_clouds : cap), kRegsNT, 0, st>>>(args);
    note_launches(1);
    return cudaGetLastError();
}

template <int NT, bool CLUSTER>
cudaError_t launch_floor(int C, int64_t iters, unsigned long long* sink, cudaStream_t st)
{
    auto kern = k_sync_floor<NT, CLUSTER>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(NT);
    cfg.gridDim = dim3(CLUSTER ? C : 1);
    cfg.stream = st;
    if (CLUSTER) {
        if (C > 8) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, iters, sink, reinterpret_cast<uint32_t*>(sink + 16));
    note_launches(1);
    return e;
}

}  // namespace

cudaError_t launch_sample(char* ws, const WsLayout& L, const float* points, int64_t* out, const rfps_opts& o,
                          int64_t n_clouds, int64_t max_n, cudaStream_t st, bool save_state, int64_t lost_iter,
                          uint32_t spin_limit)
{
    SampleArgs a;
    a.hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    a.clouds = reinterpret_cast<CloudDev*>(ws + L.clouds);
    a.order = reinterpret_cast<const uint32_t*>(ws + L.order);
    a.n_clouds = n_clouds;
    a.pts = points;
    a.pts4 = reinterpret_cast<float4*>(ws + L.pts4);
    a.porig = reinterpret_cast<const uint32_t*>(ws + L.porig);
    a.rec_sph = reinterpret_cast<const float4*>(ws + L.rec_sph);
    a.rec_rng = reinterpret_cast<const uint2*>(ws + L.rec_rng);
    a.rec_key = reinterpret_cast<unsigned long long*>(ws + L.rec_key);
    a.rec_best = reinterpret_cast<float4*>(ws + L.rec_best);
    a.rec_thr = reinterpret_cast<float*>(ws + L.rec_thr);
    a.out = out;
    a.prune = o.prune;
    a.skip = o.skip;
    a.smem_bytes = 0;   // set per instantiation from the device's opt-in limit
    a.resident = 1;
    a.save_state = save_state ? 1 : 0;
    a.lost_iter = lost_iter;
    a.spin_limit = spin_limit ? spin_limit : kSpinLimit;
#ifdef RFPS_CHECKED
    a.n_total = static_cast<uint32_t>(L.total_n);
#endif
    const int C = o.cluster;
    const bool cl = C > 1;
    if (regs_path(o, max_n)) {
        // small clouds on one CTA: every thread's points are a record in its registers; without a
        // kept index the kernel groups the points itself (no index build ran)
        if (save_state)
            return o.counters ? launch_regs<kRegsP, true, false>(a, n_clouds, st)
                              : launch_regs<kRegsP, false, false>(a, n_clouds, st);
        return o.counters ? launch_regs<kRegsP, true, true>(a, n_clouds, st)
                          : launch_regs<kRegsP, false, true>(a, n_clouds, st);
    }
    if (o.counters || lost_iter != 0) {   // the failure-path test runs in the counting kernels
        return cl ? launch_nt<true, true>(a, o.threads, C, n_clouds, st)
                  : launch_nt<false, true>(a, o.threads, C, n_clouds, st);
    }
    return cl ? launch_nt<true, false>(a, o.threads, C, n_clouds, st)
              : launch_nt<false, false>(a, o.threads, C, n_clouds, st);
}

bool regs_path(const rfps_opts& o, int64_t max_n)
{
    return o.cluster == 1 && o.threads == 512 && max_n <= static_cast<int64_t>(kRegsNT) * kRegsP;
}

cudaError_t launch_sync_floor(int C, int NT, int64_t iters, unsigned long long* sink, cudaStream_t st)
{
    if (C > 1) {
        if (NT == 128) return launch_floor<128, true>(C, iters, sink, st);
        return NT == 256 ? launch_floor<256, true>(C, iters, sink, st) : launch_floor<512, true>(C, iters, sink, st);
    }
    if (NT == 128) return launch_floor<128, false>(1, iters, sink, st);
    return NT == 256 ? launch_floor<256, false>(1, iters, sink, st) : launch_floor<512, false>(1, iters, sink, st);
}

}  // namespace rfps
