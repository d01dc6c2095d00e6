// rfps_internal.h -- workspace layout and launcher declarations shared by the
// translation units of librfps.so (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rfps.h"

namespace rfps {

// Per-cloud descriptor kept in the workspace.
struct CloudDev {
    int64_t pt_off;    // first point (row) of the cloud in the concatenated input
    int64_t n;         // points
    int64_t out_off;   // first output slot
    int64_t m;         // samples
    int64_t start;     // start index, cloud-local
    uint32_t rec_off;  // first voxel record
    uint32_t rec_end;  // one past the last voxel record
    float gmin[3];     // bounding-box minimum (Sec. 3.2)
    float L;           // voxel side (Eq. voxel_size)
    int32_t n_vox;     // bins per axis
    uint32_t cell_base;// first global cell id of the cloud
    uint32_t bbox[6];  // order-preserving encodings of min xyz / max xyz during the reduction
    uint32_t valid;    // 1 if the cloud passed the device-side checks
    uint32_t resume;   // 1: continue a saved sampling state instead of starting from `start`
    float last[3];     // coordinates of the last selected sample (saved state)
    uint32_t pad2;
};
static_assert(sizeof(CloudDev) % 8 == 0, "CloudDev alignment");

// Header at the start of every workspace.
struct WsHeader {
    uint32_t status;        // first device-recorded error (rfps_status), 0 = ok
    uint32_t work;          // sampler work-queue counter
    uint32_t n_records;     // voxel records built
    uint32_t total_cells;   // sum of n_vox^3 over the clouds
    uint64_t counters[9];   // rfps_counters fields
    uint32_t grid_arrive;   // plain variant 2: grid-barrier arrival counter
    uint32_t pad[13];
};

constexpr int kMaxNVox = 256;
constexpr int kRadixBits = 8;
constexpr int kRadixNT = 256;
constexpr int kRadixIPT = 8;
constexpr int kRadixTile = kRadixNT * kRadixIPT;
constexpr int kScanNT = 256;
constexpr int kScanIPT = 8;
constexpr int kScanTile = kScanNT * kScanIPT;

// Byte offsets of the workspace regions (all 256-byte aligned).
struct WsLayout {
    size_t header, clouds, order;
    size_t keys0, vals0, keys1, vals1;
    size_t hist, scan_agg, aux;
    size_t pts4, porig;
    size_t rec_sph, rec_rng, rec_key, rec_best, rec_thr;
    size_t host_points, host_out;   // only for rfps_fps_host
    size_t total;
    int64_t total_n, n_clouds, max_records, radix_passes, radix_tiles;
};

WsLayout make_layout(int64_t total_n, int64_t n_clouds, int64_t max_n, const rfps_opts& o,
                     bool host_buffers, int64_t host_m);

// Effective options after the automatic choices for a cloud of max_n points.
rfps_opts resolve_opts(const rfps_opts* in, int64_t max_n);

// Build the voxel index of every cloud described in ws (clouds already set up).
cudaError_t launch_build(char* ws, const WsLayout& L, const float* points, const rfps_opts& o,
                         int64_t max_n, cudaStream_t st);
// Persistent sampling launch over the clouds of ws.
// lost_iter > 0 (failure-path test, counting kernels): exchange round lost_iter sends nothing and
// its waits give up after spin_limit polls (0: the default limit).
cudaError_t launch_sample(char* ws, const WsLayout& L, const float* points, int64_t* out,
                          const rfps_opts& o, int64_t n_clouds, int64_t max_n, cudaStream_t st,
                          bool save_state = false, int64_t lost_iter = 0, uint32_t spin_limit = 0);
// True when the options send clouds of at most max_n points to the register-record sampler,
// which groups the points itself unless a kept index is sampled: the caller then skips the
// index build (launch_build) for a launch without save_state.
bool regs_path(const rfps_opts& o, int64_t max_n);
// Synchronisation floor of the sampling loop (same tail, no record work).
cudaError_t launch_sync_floor(int C, int NT, int64_t iters, unsigned long long* sink, cudaStream_t st);
// On-chip bandwidth probe (rfps_probe.cu): kind 0 L2 reads of `buf`, kind 1 shared-memory reads.
cudaError_t launch_bw_probe(int kind, const void* buf, int64_t bytes, int reps, unsigned long long* sink,
                            cudaStream_t st, int64_t* moved, int* sms_out);
// Plain FPS launches.
cudaError_t launch_plain(char* ws, const WsLayout& L, const float* points, int64_t* out, int variant,
                         int64_t n_clouds, int64_t max_n, cudaStream_t st);
// Fill the cloud table from device arrays (batched) or scalars (single cloud).
cudaError_t launch_setup(char* ws, const WsLayout& L, const int64_t* offsets, const int64_t* out_offsets,
                         const int64_t* starts, int64_t n_clouds, int64_t total_n, int64_t n, int64_t m,
                         int64_t start, int64_t max_n, const rfps_opts& o, cudaStream_t st);

// Kernel launch accounting (rfps_launch_count).
void note_launches(int64_t k);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Cells are numbered in Morton (Z) order so that records that are consecutive
// in sort order are compact in space (the hierarchical path groups 32 of
// them).  With b = ceil(log2 n_vox) bits per axis a cloud spans 8^b cell ids.
__host__ __device__ inline int morton_bits(int n_vox)
{
    int b = 0;
    while ((1 << b) < n_vox) ++b;
    return b;
}
__host__ __device__ inline uint32_t morton_spread(uint32_t v)   // 10 bits -> every third bit
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ inline uint32_t morton_compact(uint32_t v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}
__host__ __device__ inline uint32_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    return morton_spread(x) | (morton_spread(y) << 1) | (morton_spread(z) << 2);
}

}  // namespace rfps
