// rfps_build.cu -- on-device construction of the spherical-voxel index
// (Sec. 3.2 preprocessing; the GPU pipeline of Alg. voxelization_gpu).
//
// Pipeline (one stream, every cloud of a batch at once):
//   k_setup      cloud table, device checks of the caller's arrays, n_vox per
//                cloud, global cell numbering, largest-first cloud order
//   k_bbox       bounding box per cloud + non-finite detection        (Alg. 2, bounds)
//   k_grid       L = alpha * max(E) / n_vox  (Eq. voxel_size)          (Alg. 2, voxel size)
//   k_bin        clamped floor binning (Alg. 2 Phase 1); the sort key is the cell's Morton
//                code rather than v_z n^2 + v_y n + v_x, so sorted neighbours are 3-D compact
//   radix sort   stable LSD sort of (global cell id, point index)      (Alg. 2 sort)
//   records      active voxels, split into records of <= chunk points,
//                with offset / count (Phase 3), centre c_k, a radius that
//                covers every member (Eq. preprocess_voxel_radius, see
//                below), and the gather into a float4 (x, y, z, d2) layout
//                sorted by voxel (Phase 2, with d2 riding in .w instead of
//                a separate SoA array).
#include <cfloat>
#include <cmath>

#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {

__device__ __forceinline__ void set_status(WsHeader* h, uint32_t code)
{
    atomicCAS(&h->status, 0u, code);
}

// ---------------------------------------------------------------------------
// Cloud table.  One block: the header is reset before any check can write it.
__global__ void k_setup(WsHeader* hdr, CloudDev* clouds, uint32_t* order, const int64_t* offsets,
                        const int64_t* out_offsets, const int64_t* starts, int64_t n_clouds,
                        int64_t total_n, int64_t n1, int64_t m1, int64_t start1, int64_t max_n,
                        int n_vox_opt, int n_vox_cap, float auto_k, int sort_clouds)
{
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_bad;
    __shared__ uint32_t s_cells[256];
    const int t = threadIdx.x;
    if (t == 0) {
        hdr->status = 0;
        hdr->work = 0;
        hdr->n_records = 0;
        hdr->total_cells = 0;
        for (int i = 0; i < 9; ++i) hdr->counters[i] = 0;
        hdr->grid_arrive = 0;
        s_carry = 0;
        s_bad = 0;
    }
    __syncthreads();
    const bool single = offsets == nullptr;
    for (int64_t b0 = 0; b0 < n_clouds; b0 += blockDim.x) {
        const int64_t b = b0 + t;
        uint32_t cells = 0;
        if (b < n_clouds) {
            CloudDev c;
            if (single) {
                c.pt_off = 0; c.n = n1; c.out_off = 0; c.m = m1; c.start = start1;
            } else {
                c.pt_off = offsets[b];
                c.n = offsets[b + 1] - offsets[b];
                c.out_off = out_offsets[b];
                c.m = out_offsets[b + 1] - out_offsets[b];
                c.start = starts[b];
            }
            bool ok = c.n >= 1 && c.n < (int64_t(1) << 31) && c.m >= 1 && c.m <= c.n && c.start >= 0 &&
                      c.start < c.n && c.pt_off >= 0 && c.pt_off + c.n <= total_n && c.out_off >= 0 &&
                      c.n <= max_n;
            if (!single) {
                if (b == 0 && offsets[0] != 0) ok = false;
                if (b == n_clouds - 1 && offsets[n_clouds] != total_n) ok = false;
                if (b == 0 && out_offsets[0] != 0) ok = false;
            }
            int nv = n_vox_opt;
            if (nv <= 0) {
                nv = static_cast<int>(rintf(auto_k * cbrtf(static_cast<float>(c.n))));
            }
            nv = max(1, min(nv, n_vox_cap));
            c.n_vox = nv;
            c.rec_off = 0;
            c.rec_end = 0;
            c.gmin[0] = c.gmin[1] = c.gmin[2] = 0.0f;
            c.L = 1.0f;
            for (int a = 0; a < 3; ++a) {
                c.bbox[a] = 0xffffffffu;   // running min (ordered encoding)
                c.bbox[3 + a] = 0u;        // running max
            }
            c.valid = ok ? 1u : 0u;
            c.resume = 0;
            c.last[0] = c.last[1] = c.last[2] = 0.0f;
            c.pad2 = 0;
            cells = 1u << (3 * morton_bits(nv));   // Morton-ordered cell ids of this cloud
            if (!ok) atomicOr(&s_bad, 1u);
            clouds[b] = c;
        }
        // exclusive prefix of cells over this chunk (cell_base), carried across chunks
        s_cells[t] = cells;
        __syncthreads();
        if (t == 0) {
            uint32_t run = s_carry;
            const int64_t rem = n_clouds - b0;
            const int lim = static_cast<int>(rem < static_cast<int64_t>(blockDim.x) ? rem : blockDim.x);
            for (int i = 0; i < lim; ++i) {
                const uint32_t c = s_cells[i];
                s_cells[i] = run;
                if (run + c < run) s_bad |= 2u;   // more than 2^32 cells
                run += c;
            }
            s_carry = run;
        }
        __syncthreads();
        if (b < n_clouds) clouds[b].cell_base = s_cells[t];
        __syncthreads();
    }
    if (t == 0) {
        hdr->total_cells = s_carry;
        if (s_bad) hdr->status = kStatusInval;
    }
    // largest-first work order (ties by index); identity when not sorting
    __syncthreads();
    for (int64_t b = t; b < n_clouds; b += blockDim.x) {
        if (!sort_clouds) {
            order[b] = static_cast<uint32_t>(b);
            continue;
        }
        const int64_t nb = single ? n1 : offsets[b + 1] - offsets[b];
        uint32_t rank = 0;
        for (int64_t o = 0; o < n_clouds; ++o) {
            const int64_t no = offsets[o + 1] - offsets[o];
            rank += (no > nb || (no == nb && o < b)) ? 1u : 0u;
        }
        order[rank] = static_cast<uint32_t>(b);
    }
}

// ---------------------------------------------------------------------------
// Bounding box per cloud (Sec. 3.2) and the non-finite check.
constexpr int kBoxNT = 256;
__global__ void __launch_bounds__(kBoxNT) k_bbox(WsHeader* hdr, CloudDev* clouds, const float* pts,
                                                 int64_t n_clouds)
{
    __shared__ float s_red[6][kBoxNT / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int64_t b = blockIdx.y; b < n_clouds; b += gridDim.y) {
        const CloudDev c = clouds[b];
        if (!c.valid) continue;
        float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        bool bad = false;
        const float* p = pts + 3 * c.pt_off;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBoxNT + t; i < c.n;
             i += static_cast<int64_t>(gridDim.x) * kBoxNT) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float v = p[3 * i + a];
                bad |= !isfinite(v);
                mn[a] = fminf(mn[a], v);
                mx[a] = fmaxf(mx[a], v);
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(hdr, kStatusNonFinite);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            for (int o = 16; o > 0; o >>= 1) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
            }
        }
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) {
                s_red[a][w] = mn[a];
                s_red[3 + a][w] = mx[a];
            }
        }
        __syncthreads();
        if (t < 6) {
            float v = s_red[t][0];
            for (int i = 1; i < kBoxNT / 32; ++i) v = (t < 3) ? fminf(v, s_red[t][i]) : fmaxf(v, s_red[t][i]);
            const uint32_t e = float_to_ordered(v);
            if (t < 3) atomicMin(&clouds[b].bbox[t], e);
            else atomicMax(&clouds[b].bbox[t], e);
        }
        __syncthreads();
    }
}

// L = alpha * max(E) / n_vox with alpha = 1 + 2^-10 (Eq. voxel_size; the paper
// leaves eps unstated).  max(E) = 0 (every point equal) gives L = 1.
__global__ void k_grid(CloudDev* clouds, int64_t n_clouds)
{
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= n_clouds) return;
    CloudDev& c = clouds[b];
    if (!c.valid) return;
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = ordered_to_float(c.bbox[a]);
        mx[a] = ordered_to_float(c.bbox[3 + a]);
    }
    const float ex = __fsub_rn(mx[0], mn[0]);
    const float ey = __fsub_rn(mx[1], mn[1]);
    const float ez = __fsub_rn(mx[2], mn[2]);
    float e = ex;
    if (ey > e) e = ey;
    if (ez > e) e = ez;
    float L = 1.0f;
    if (e > 0.0f) L = __fdiv_rn(__fmul_rn(1.0009765625f, e), static_cast<float>(c.n_vox));
    c.gmin[0] = mn[0];
    c.gmin[1] = mn[1];
    c.gmin[2] = mn[2];
    c.L = L;
}

__device__ __forceinline__ uint32_t bin_coord(float p, float mn, float L, int n_vox)
{
    float f = floorf(__fdiv_rn(__fsub_rn(p, mn), L));
    f = fmaxf(f, 0.0f);                                  // also maps NaN to 0
    f = fminf(f, static_cast<float>(n_vox - 1));
    return static_cast<uint32_t>(f);
}

// Phase 1: voxel coordinates per point; sort key = cell_base + Morton code of the cell,
// value = point row.
__global__ void __launch_bounds__(kBoxNT) k_bin(const WsHeader* hdr, const CloudDev* clouds, const float* pts,
                                                int64_t n_clouds, uint32_t* keys, uint32_t* vals)
{
    if (hdr->status != 0) return;
    for (int64_t b = blockIdx.y; b < n_clouds; b += gridDim.y) {
        const CloudDev c = clouds[b];
        const float* p = pts + 3 * c.pt_off;
        const uint32_t nv = static_cast<uint32_t>(c.n_vox);
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * kBoxNT + threadIdx.x; i < c.n;
             i += static_cast<int64_t>(gridDim.x) * kBoxNT) {
            const uint32_t vx = bin_coord(p[3 * i + 0], c.gmin[0], c.L, c.n_vox);
            const uint32_t vy = bin_coord(p[3 * i + 1], c.gmin[1], c.L, c.n_vox);
            const uint32_t vz = bin_coord(p[3 * i + 2], c.gmin[2], c.L, c.n_vox);
            keys[c.pt_off + i] = c.cell_base + morton3(vx, vy, vz);
            (void)nv;
            vals[c.pt_off + i] = static_cast<uint32_t>(c.pt_off + i);
        }
    }
}

// ---------------------------------------------------------------------------
// Block-wide scans (256 threads).
struct OpSum {
    __device__ static uint32_t id() { return 0u; }
    __device__ static uint32_t op(uint32_t a, uint32_t b) { return a + b; }
};
struct OpMax {
    __device__ static uint32_t id() { return 0u; }
    __device__ static uint32_t op(uint32_t a, uint32_t b) { return a > b ? a : b; }
};

template <class Op>
__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = Op::op(u, v);
    }
    return v;
}

// Exclusive scan of one value per thread over a 256-thread block; *total gets the block aggregate.
template <class Op>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* s_warp, uint32_t* total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t inc = warp_inclusive<Op>(v, lane);
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = lane < kScanNT / 32 ? s_warp[lane] : Op::id();
        x = warp_inclusive<Op>(x, lane);
        if (lane < kScanNT / 32) s_warp[lane] = x;
    }
    __syncthreads();
    const uint32_t before = w > 0 ? s_warp[w - 1] : Op::id();
    *total = s_warp[kScanNT / 32 - 1];
    const uint32_t exc_in_warp = __shfl_up_sync(0xffffffffu, inc, 1);
    const uint32_t exc = lane > 0 ? Op::op(before, exc_in_warp) : before;
    __syncthreads();
    return exc;
}

template <class Op>
__global__ void __launch_bounds__(kScanNT) k_scan_reduce(const uint32_t* in, uint32_t n, uint32_t* agg)
{
    __shared__ uint32_t s_warp[kScanNT / 32];
    const uint32_t base = blockIdx.x * kScanTile;
    uint32_t v = Op::id();
#pragma unroll
    for (int r = 0; r < kScanIPT; ++r) {
        const uint32_t i = base + r * kScanNT + threadIdx.x;
        if (i < n) v = Op::op(v, in[i]);
    }
    uint32_t total;
    block_exclusive<Op>(v, s_warp, &total);
    if (threadIdx.x == 0) agg[blockIdx.x] = total;
}

// Exclusive scan of agg[0..nt) in place by one block.
template <class Op>
__global__ void __launch_bounds__(kScanNT) k_scan_top(uint32_t* agg, uint32_t nt)
{
    __shared__ uint32_t s_warp[kScanNT / 32];
    uint32_t carry = Op::id();
    for (uint32_t base = 0; base < nt; base += kScanNT) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nt ? agg[i] : Op::id();
        uint32_t total;
        const uint32_t e = block_exclusive<Op>(v, s_warp, &total);
        if (i < nt) agg[i] = Op::op(carry, e);
        carry = Op::op(carry, total);
    }
}

// Tile scan plus the tile's prefix; in and out may alias.
template <class Op, bool Inclusive>
__global__ void __launch_bounds__(kScanNT) k_scan_down(const uint32_t* in, uint32_t* out, uint32_t n,
                                                       const uint32_t* agg)
{
    __shared__ uint32_t s_tile[kScanTile];
    __shared__ uint32_t s_warp[kScanNT / 32];
    const uint32_t base = blockIdx.x * kScanTile;
#pragma unroll
    for (int r = 0; r < kScanIPT; ++r) {
        const uint32_t i = base + r * kScanNT + threadIdx.x;
        s_tile[r * kScanNT + threadIdx.x] = i < n ? in[i] : Op::id();
    }
    __syncthreads();
    uint32_t x[kScanIPT];
    uint32_t acc = Op::id();
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        x[k] = s_tile[threadIdx.x * kScanIPT + k];
        acc = Op::op(acc, x[k]);
    }
    uint32_t total;
    uint32_t run = Op::op(agg[blockIdx.x], block_exclusive<Op>(acc, s_warp, &total));
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        const uint32_t inc = Op::op(run, x[k]);
        s_tile[threadIdx.x * kScanIPT + k] = Inclusive ? inc : run;
        run = inc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanIPT; ++r) {
        const uint32_t i = base + r * kScanNT + threadIdx.x;
        if (i < n) out[i] = s_tile[r * kScanNT + threadIdx.x];
    }
}

template <class Op, bool Inclusive>
void scan(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* agg, cudaStream_t st)
{
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<Op><<<tiles, kScanNT, 0, st>>>(in, n, agg);
    k_scan_top<Op><<<1, kScanNT, 0, st>>>(agg, tiles);
    k_scan_down<Op, Inclusive><<<tiles, kScanNT, 0, st>>>(in, out, n, agg);
    note_launches(3);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Digit-major histogram hist[d * tiles +
// tile]; its exclusive scan is the first output slot of each (digit, tile).
__global__ void __launch_bounds__(kRadixNT) k_radix_count(const WsHeader* hdr, const uint32_t* keys, uint32_t n,
                                                          int shift, uint32_t* hist, uint32_t tiles)
{
    __shared__ uint32_t s_cnt[256];
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixIPT; ++r) {
        const uint32_t i = base + r * kRadixNT + threadIdx.x;
        if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * tiles + blockIdx.x] = s_cnt[threadIdx.x];
    (void)hdr;
}

// Items of a tile are ranked in index order: round r, then warp, then lane.
__global__ void __launch_bounds__(kRadixNT) k_radix_scatter(const uint32_t* keys_in, const uint32_t* vals_in,
                                                            uint32_t n, int shift, const uint32_t* hist,
                                                            uint32_t tiles, uint32_t* keys_out, uint32_t* vals_out)
{
    constexpr int NW = kRadixNT / 32;
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_wh[NW][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    s_run[t] = hist[t * tiles + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t base = blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixIPT; ++r) {
#pragma unroll
        for (int k = 0; k < NW; ++k) s_wh[k][t] = 0;
        __syncthreads();
        const uint32_t i = base + r * kRadixNT + t;
        const bool valid = i < n;
        const uint32_t key = valid ? keys_in[i] : 0u;
        const uint32_t val = valid ? vals_in[i] : 0u;
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : (256u + lane));
        const uint32_t rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) s_wh[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = s_run[t];
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t c = s_wh[k][t];
                s_wh[k][t] = acc;
                acc += c;
            }
            s_run[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_wh[w][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Voxel records.
__global__ void k_cellhead(const WsHeader* hdr, const uint32_t* keys, uint32_t n, uint32_t* headpos)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    headpos[i] = (i == 0 || keys[i] != keys[i - 1]) ? i : 0u;
    (void)hdr;
}

__global__ void k_rechead(const uint32_t* cellstart, uint32_t n, uint32_t chunk_mask, uint32_t* flag)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = ((i - cellstart[i]) & chunk_mask) == 0u ? 1u : 0u;
}

__global__ void k_recoffs(WsHeader* hdr, const uint32_t* flag, const uint32_t* recidx, uint32_t n,
                          uint2* rec_rng)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) rec_rng[recidx[i]].x = i;
    if (i == n - 1) hdr->n_records = recidx[i] + flag[i];
}

__global__ void k_cloudrec(const WsHeader* hdr, CloudDev* clouds, int64_t n_clouds, const uint32_t* recidx)
{
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= n_clouds) return;
    if (hdr->status != 0) return;     // offsets are only trusted once every check passed
    CloudDev& c = clouds[b];
    c.rec_off = recidx[c.pt_off];
    c.rec_end = (b + 1 < n_clouds) ? recidx[clouds[b + 1].pt_off] : hdr->n_records;
}

// One warp per record: count, cloud, centre c_k = p_min + (v + 1/2) L, the
// gather into the sorted float4 layout, and a covering radius.
//
// The paper's radius sqrt(3)/2 L (Eq. preprocess_voxel_radius) covers the
// cube over the reals; a point can sit an ulp outside its nominal cube after
// the FP32 binning, and any radius with r >= |p - c| for every member is as
// correct.  Default: r = max(fl(m * (1 + 2^-20)), 2^-50), m = max over the
// members of sqrt(fl d2(p, c)).  With u = 2^-24, m >= (1 - 3.6u)|p - c| when
// |p - c| >= 2^-50, so fl(m (1 + 16u)) >= (1 + 11u)|p - c|; smaller
// distances are covered by the 2^-50 floor.  radius_mode 1 takes
// max(that, fl(sqrt(3)/2 * L)).
__global__ void k_records(const WsHeader* hdr, const CloudDev* clouds, int64_t n_clouds, const float* pts,
                          const uint32_t* skeys, const uint32_t* svals, uint32_t n_total, uint2* rec_rng,
                          float4* rec_sph, unsigned long long* rec_key, float4* rec_best, float4* pts4,
                          uint32_t* porig, int radius_mode)
{
    if (hdr->status != 0) return;
    const uint32_t R = hdr->n_records;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < R; r += warps) {
        const uint32_t off = rec_rng[r].x;
        const uint32_t end = (r + 1 < R) ? rec_rng[r + 1].x : n_total;
        const uint32_t cnt = end - off;
        // cloud of the record: last b with pt_off <= off
        int64_t lo = 0, hi = n_clouds - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (clouds[mid].pt_off <= static_cast<int64_t>(off)) lo = mid;
            else hi = mid - 1;
        }
        const CloudDev c = clouds[lo];
        const uint32_t code = skeys[off] - c.cell_base;   // Morton code of the cell
        const uint32_t v[3] = {morton_compact(code), morton_compact(code >> 1), morton_compact(code >> 2)};
        float cen[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            cen[a] = __fadd_rn(c.gmin[a], __fmul_rn(__fadd_rn(static_cast<float>(v[a]), 0.5f), c.L));
        float m = 0.0f;
        for (uint32_t q = lane; q < cnt; q += 32) {
            const uint32_t g = svals[off + q];
            const float x = pts[3 * static_cast<size_t>(g) + 0];
            const float y = pts[3 * static_cast<size_t>(g) + 1];
            const float z = pts[3 * static_cast<size_t>(g) + 2];
            pts4[off + q] = make_float4(x, y, z, __int_as_float(0x7f800000));
            porig[off + q] = g;
            m = fmaxf(m, __fsqrt_rn(sq_dist(x, y, z, cen[0], cen[1], cen[2])));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            float rad = fmaxf(__fmul_rn(m, 0x1.00001p0f), 0x1p-50f);
            if (radius_mode == 1) rad = fmaxf(rad, __fmul_rn(0.8660254037844386f, c.L));
            rec_rng[r].y = cnt;
            rec_sph[r] = make_float4(cen[0], cen[1], cen[2], rad);
            const uint32_t g0 = svals[off];
            rec_key[r] = make_key(__int_as_float(0x7f800000), g0);
            rec_best[r] = make_float4(pts[3 * static_cast<size_t>(g0)], pts[3 * static_cast<size_t>(g0) + 1],
                                      pts[3 * static_cast<size_t>(g0) + 2], 0.0f);
        }
    }
}

}  // namespace

cudaError_t launch_setup(char* ws, const WsLayout& L, const int64_t* offsets, const int64_t* out_offsets,
                         const int64_t* starts, int64_t n_clouds, int64_t total_n, int64_t n, int64_t m,
                         int64_t start, int64_t max_n, const rfps_opts& o, cudaStream_t st)
{
    auto* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    auto* clouds = reinterpret_cast<CloudDev*>(ws + L.clouds);
    auto* order = reinterpret_cast<uint32_t*>(ws + L.order);
    const int sort_clouds = (offsets != nullptr && n_clouds > 1 && n_clouds <= 8192) ? 1 : 0;
    // cap n_vox so that the global cell ids of all clouds fit 32 bits
    int cap = kMaxNVox;
    while (cap > 1 && std::ldexp(1.0, 3 * morton_bits(cap)) * static_cast<double>(n_clouds) >= 4294967295.0) --cap;
    k_setup<<<1, 256, 0, st>>>(hdr, clouds, order, offsets, out_offsets, starts, n_clouds, total_n, n, m, start,
                               max_n, o.n_vox, cap, static_cast<float>(o.nvox_scale) / 100.0f, sort_clouds);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_build(char* ws, const WsLayout& L, const float* points, const rfps_opts& o, int64_t max_n,
                         cudaStream_t st)
{
    auto* hdr = reinterpret_cast<WsHeader*>(ws + L.header);
    auto* clouds = reinterpret_cast<CloudDev*>(ws + L.clouds);
    const int64_t B = L.n_clouds;
    const uint32_t N = static_cast<uint32_t>(L.total_n);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(ws + L.keys0), reinterpret_cast<uint32_t*>(ws + L.keys1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(ws + L.vals0), reinterpret_cast<uint32_t*>(ws + L.vals1)};
    auto* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
    auto* agg = reinterpret_cast<uint32_t*>(ws + L.scan_agg);
    auto* aux = reinterpret_cast<uint32_t*>(ws + L.aux);

    const int gy = static_cast<int>(B < 65535 ? B : 65535);
    const int64_t per_cloud_blocks = (max_n + kBoxNT * 8 - 1) / (kBoxNT * 8);
    const int gx = static_cast<int>(per_cloud_blocks < 1024 ? (per_cloud_blocks > 0 ? per_cloud_blocks : 1) : 1024);
    k_bbox<<<dim3(gx, gy), kBoxNT, 0, st>>>(hdr, clouds, points, B);
    k_grid<<<static_cast<unsigned>((B + 255) / 256), 256, 0, st>>>(clouds, B);
    k_bin<<<dim3(gx, gy), kBoxNT, 0, st>>>(hdr, clouds, points, B, keys[0], vals[0]);
    note_launches(3);

    // radix sort over the global cell ids
    const uint32_t tiles = static_cast<uint32_t>(L.radix_tiles);
    int cur = 0;
    for (int p = 0; p < L.radix_passes; ++p) {
        const int shift = p * kRadixBits;
        k_radix_count<<<tiles, kRadixNT, 0, st>>>(hdr, keys[cur], N, shift, hist, tiles);
        note_launches(1);
        scan<OpSum, false>(hist, hist, 256u * tiles, agg, st);
        k_radix_scatter<<<tiles, kRadixNT, 0, st>>>(keys[cur], vals[cur], N, shift, hist, tiles, keys[cur ^ 1],
                                                    vals[cur ^ 1]);
        note_launches(1);
        cur ^= 1;
    }
    uint32_t* skeys = keys[cur];
    uint32_t* svals = vals[cur];
    uint32_t* flag = keys[cur ^ 1];
    uint32_t* recidx = vals[cur ^ 1];
    auto* rec_rng = reinterpret_cast<uint2*>(ws + L.rec_rng);
    const unsigned eb = (N + 255) / 256;
    k_cellhead<<<eb, 256, 0, st>>>(hdr, skeys, N, aux);
    note_launches(1);
    scan<OpMax, true>(aux, aux, N, agg, st);
    k_rechead<<<eb, 256, 0, st>>>(aux, N, static_cast<uint32_t>(o.chunk - 1), flag);
    note_launches(1);
    scan<OpSum, false>(flag, recidx, N, agg, st);
    k_recoffs<<<eb, 256, 0, st>>>(hdr, flag, recidx, N, rec_rng);
    k_cloudrec<<<static_cast<unsigned>((B + 255) / 256), 256, 0, st>>>(hdr, clouds, B, recidx);
    note_launches(2);
    const int64_t rb = (L.max_records * 32 + 255) / 256;
    k_records<<<static_cast<unsigned>(rb < 4096 ? rb : 4096), 256, 0, st>>>(
        hdr, clouds, B, points, skeys, svals, N, rec_rng, reinterpret_cast<float4*>(ws + L.rec_sph),
        reinterpret_cast<unsigned long long*>(ws + L.rec_key), reinterpret_cast<float4*>(ws + L.rec_best),
        reinterpret_cast<float4*>(ws + L.pts4), reinterpret_cast<uint32_t*>(ws + L.porig), o.radius_mode);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rfps
