// rfps_api.cu -- the extern "C" entry points of librfps.so (declared in
// include/rfps.h): argument checks, workspace layout, launches, device
// status, and the persistent index used for serving.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "rfps_common.cuh"
#include "rfps_internal.h"

namespace rfps {

namespace {
std::atomic<int64_t> g_launches{0};

// Cells per axis chosen when opts.n_vox == 0: about nvox_scale / 100 * cbrt(N),
// the value the device computes per cloud (k_setup); the host only needs an
// upper bound.
int auto_nvox_bound(int64_t n, int scale_pct, int cap)
{
    const double v = std::rint(scale_pct / 100.0 * std::cbrt(static_cast<double>(n))) + 1.0;
    const int nv = static_cast<int>(v < 1.0 ? 1.0 : v);
    return nv < cap ? nv : cap;
}

int nvox_cap(int64_t n_clouds)
{
    int cap = kMaxNVox;
    while (cap > 1 && std::ldexp(1.0, 3 * morton_bits(cap)) * static_cast<double>(n_clouds) >= 4294967295.0) --cap;
    return cap;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

__global__ void k_rearm(WsHeader* hdr, CloudDev* clouds, int64_t m, int64_t start, uint32_t resume)
{
    hdr->status = 0;
    hdr->work = 0;
    for (int i = 0; i < 9; ++i) hdr->counters[i] = 0;
    clouds[0].m = m;
    clouds[0].start = start;
    clouds[0].out_off = 0;
    clouds[0].resume = resume;
}

// Each point's stored distance (sorted position i, .w of the float4) back to its original row.
__global__ void k_index_d2(const float4* pts4, const uint32_t* porig, int64_t n, float* d2)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        d2[porig[i]] = pts4[i].w;
}

rfps_status from_cuda(cudaError_t e) { return e == cudaSuccess ? RFPS_OK : RFPS_ECUDA; }

rfps_status device_check()
{
    static int ok = -1;
    if (ok < 0) {
        int dev = 0;
        cudaDeviceProp prop;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return RFPS_ECUDA;
        ok = (prop.major == 10 && prop.minor == 3) ? 1 : 0;
    }
    return ok ? RFPS_OK : RFPS_EUNSUPPORTED;
}
}  // namespace

void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

rfps_opts resolve_opts(const rfps_opts* in, int64_t max_n)
{
    rfps_opts o;
    rfps_opts_default(&o);
    if (in) o = *in;
    // Defaults from launch-shape sweeps on GB300: up to 4,096 points one CTA of 512
    // threads, whose threads hold the points as records in registers, is fastest (uniform,
    // room and LiDAR clouds of 1k-4k points); above, the per-iteration cost is the cluster
    // exchange plus the unpruned records' work, and 16 CTAs of 256 threads were fastest.
    const bool small = max_n <= 4096 && (o.cluster <= 1) && (o.threads <= 0 || o.threads == 512);
    if (o.threads != 128 && o.threads != 256 && o.threads != 512) o.threads = small ? 512 : 256;
    if (o.cluster <= 0) o.cluster = (small || max_n < 2048) ? 1 : 16;
    if (o.chunk <= 0) o.chunk = 128;
    if (o.nvox_scale <= 0) o.nvox_scale = 70;
    return o;
}

WsLayout make_layout(int64_t total_n, int64_t n_clouds, int64_t max_n, const rfps_opts& o, bool host_buffers,
                     int64_t host_m)
{
    WsLayout L;
    std::memset(&L, 0, sizeof(L));
    const size_t N = static_cast<size_t>(total_n);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.header = take(sizeof(WsHeader));
    L.clouds = take(static_cast<size_t>(n_clouds) * sizeof(CloudDev));
    L.order = take(static_cast<size_t>(n_clouds) * 4);
    L.keys0 = take(N * 4);
    L.vals0 = take(N * 4);
    L.keys1 = take(N * 4);
    L.vals1 = take(N * 4);
    L.radix_tiles = static_cast<int64_t>((N + kRadixTile - 1) / kRadixTile);
    L.hist = take(static_cast<size_t>(L.radix_tiles) * 256 * 4);
    const size_t agg_n = std::max((N + kScanTile - 1) / kScanTile,
                                  (static_cast<size_t>(L.radix_tiles) * 256 + kScanTile - 1) / kScanTile) + 1;
    L.scan_agg = take(agg_n * 4);
    L.aux = take(N * 4);
    L.pts4 = take(N * 16);
    L.porig = take(N * 4);
    L.max_records = total_n;
    L.rec_sph = take(N * 16);
    L.rec_rng = take(N * 8);
    L.rec_key = take(N * 8);
    L.rec_best = take(N * 16);
    L.rec_thr = take(N * 4);
    L.host_points = host_buffers ? take(N * 12) : 0;
    L.host_out = host_buffers ? take(static_cast<size_t>(host_m) * 8) : 0;
    L.total = off;
    L.total_n = total_n;
    L.n_clouds = n_clouds;
    // sort key bits: global cell ids < n_clouds * n_vox_max^3
    const int cap = nvox_cap(n_clouds);
    const int nv = o.n_vox > 0 ? std::min(o.n_vox, cap) : auto_nvox_bound(max_n, o.nvox_scale, cap);
    const double cells = std::ldexp(1.0, 3 * morton_bits(nv)) * static_cast<double>(n_clouds);
    int bits = 1;
    while (bits < 32 && std::ldexp(1.0, bits) < cells) ++bits;
    L.radix_passes = (bits + kRadixBits - 1) / kRadixBits;
    return L;
}

// Plain FPS workspace: header, cloud table, order, d2 per point, grid slots.
static WsLayout make_plain_layout(int64_t total_n, int64_t n_clouds)
{
    WsLayout L;
    std::memset(&L, 0, sizeof(L));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.header = take(sizeof(WsHeader));
    L.clouds = take(static_cast<size_t>(n_clouds) * sizeof(CloudDev));
    L.order = take(static_cast<size_t>(n_clouds) * 4);
    L.keys0 = take(static_cast<size_t>(total_n) * 4);
    L.hist = take(2 * 1024 * 8);       // grid-barrier slot keys
    L.rec_best = take(2 * 1024 * 16);  // grid-barrier slot coordinates
    L.total = off;
    L.total_n = total_n;
    L.n_clouds = n_clouds;
    return L;
}

}  // namespace rfps

using namespace rfps;

struct rfps_index {
    void* mem;
    size_t bytes;
    WsLayout L;
    rfps_opts o;
    int64_t n;
    cudaStream_t stream;
    int sorted_buf;
    int64_t taken;   // samples of the current sequence so far (0: no saved state)
};

static rfps_status check_opts(const rfps_opts* o)
{
    if (!o) return RFPS_OK;
    if (o->n_vox < 0 || o->n_vox > kMaxNVox) return RFPS_EINVAL;
    if (o->cluster != 0 && o->cluster != 1 && o->cluster != 2 && o->cluster != 4 && o->cluster != 8 &&
        o->cluster != 16)
        return RFPS_EINVAL;
    if (o->threads != 0 && o->threads != 128 && o->threads != 256 && o->threads != 512) return RFPS_EINVAL;
    if (o->chunk != 0 && (!is_pow2(o->chunk) || o->chunk < 32 || o->chunk > 4096)) return RFPS_EINVAL;
    if (o->radius_mode != 0 && o->radius_mode != 1) return RFPS_EINVAL;
    if (o->nvox_scale < 0 || o->nvox_scale > 1000) return RFPS_EINVAL;
    return RFPS_OK;
}

static bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

extern "C" {

void rfps_opts_default(rfps_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prune = 1;
    o->skip = 1;
    o->radius_mode = 0;
}

const char* rfps_status_str(int s)
{
    switch (s) {
    case RFPS_OK: return "ok";
    case RFPS_EINVAL: return "invalid argument";
    case RFPS_ENONFINITE: return "non-finite coordinate";
    case RFPS_ENOMEM: return "out of memory (workspace too small or allocation failed)";
    case RFPS_ECUDA: return "CUDA runtime error";
    case RFPS_ETIMEOUT: return "device-side wait timed out";
    case RFPS_EUNSUPPORTED: return "unsupported device or launch shape";
    case RFPS_EBOUNDS: return "index out of range (bounds-checked build)";
    default: return "unknown status";
    }
}

int rfps_version(void) { return 3; }

rfps_status rfps_opts_resolve(int64_t n, const rfps_opts* in, rfps_opts* out)
{
    if (!out || n < 1) return RFPS_EINVAL;
    const rfps_status s = check_opts(in);
    if (s != RFPS_OK) return s;
    *out = resolve_opts(in, n);
    return RFPS_OK;
}

int64_t rfps_launch_count(void) { return g_launches.load(); }



size_t rfps_fps_workspace_size(int64_t n, const rfps_opts* opts)
{
    if (n < 1 || check_opts(opts) != RFPS_OK) return 0;
    const rfps_opts o = resolve_opts(opts, n);
    return make_layout(n, 1, n, o, false, 0).total;
}

rfps_status rfps_fps(const float* points, int64_t n, int64_t m, int64_t start, int64_t* out_idx,
                     const rfps_opts* opts, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!points || !out_idx || !workspace || n < 1 || n >= (int64_t(1) << 31) || m < 1 || m > n || start < 0 ||
        start >= n || !aligned256(workspace))
        return RFPS_EINVAL;
    rfps_status s = check_opts(opts);
    if (s != RFPS_OK) return s;
    if ((s = device_check()) != RFPS_OK) return s;
    const rfps_opts o = resolve_opts(opts, n);
    const WsLayout L = make_layout(n, 1, n, o, false, 0);
    if (workspace_bytes < L.total) return RFPS_ENOMEM;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_setup(ws, L, nullptr, nullptr, nullptr, 1, n, n, m, start, n, o, st);
    if (e == cudaSuccess && !regs_path(o, n)) e = launch_build(ws, L, points, o, n, st);
    if (e == cudaSuccess) e = launch_sample(ws, L, points, out_idx, o, 1, n, st);
    return from_cuda(e);
}

rfps_status rfps_fps_lost_round(const float* points, int64_t n, int64_t m, int64_t start, int64_t* out_idx,
                                const rfps_opts* opts, void* workspace, size_t workspace_bytes, int64_t lost_iteration,
                                uint32_t spin_limit, void* stream)
{
    if (!points || !out_idx || !workspace || n < 1 || n >= (int64_t(1) << 31) || m < 2 || m > n || start < 0 ||
        start >= n || !aligned256(workspace) || lost_iteration < 1 || lost_iteration >= m || spin_limit < 1 ||
        spin_limit > (1u << 22))
        return RFPS_EINVAL;
    rfps_status s = check_opts(opts);
    if (s != RFPS_OK) return s;
    if ((s = device_check()) != RFPS_OK) return s;
    rfps_opts o = resolve_opts(opts, n);
    if (o.cluster < 2) return RFPS_EINVAL;   // one CTA has no exchange to lose
    o.counters = 1;
    const WsLayout L = make_layout(n, 1, n, o, false, 0);
    if (workspace_bytes < L.total) return RFPS_ENOMEM;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_setup(ws, L, nullptr, nullptr, nullptr, 1, n, n, m, start, n, o, st);
    if (e == cudaSuccess) e = launch_build(ws, L, points, o, n, st);
    if (e == cudaSuccess) e = launch_sample(ws, L, points, out_idx, o, 1, n, st, false, lost_iteration, spin_limit);
    return from_cuda(e);
}

size_t rfps_fps_host_workspace_size(int64_t n, const rfps_opts* opts)
{
    if (n < 1 || check_opts(opts) != RFPS_OK) return 0;
    const rfps_opts o = resolve_opts(opts, n);
    return make_layout(n, 1, n, o, true, n).total;
}

rfps_status rfps_fps_host(const float* host_points, int64_t n, int64_t m, int64_t start, int64_t* host_out,
                          const rfps_opts* opts, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!host_points || !host_out || !workspace || n < 1 || n >= (int64_t(1) << 31) || m < 1 || m > n ||
        start < 0 || start >= n || !aligned256(workspace))
        return RFPS_EINVAL;
    rfps_status s = check_opts(opts);
    if (s != RFPS_OK) return s;
    if ((s = device_check()) != RFPS_OK) return s;
    const rfps_opts o = resolve_opts(opts, n);
    // the host layout reserves room for n output slots; m <= n
    const WsLayout L = make_layout(n, 1, n, o, true, n);
    if (workspace_bytes < L.total) return RFPS_ENOMEM;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* dpts = reinterpret_cast<float*>(ws + L.host_points);
    int64_t* dout = reinterpret_cast<int64_t*>(ws + L.host_out);
    cudaError_t e = cudaMemcpyAsync(dpts, host_points, static_cast<size_t>(n) * 12, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_setup(ws, L, nullptr, nullptr, nullptr, 1, n, n, m, start, n, o, st);
    if (e == cudaSuccess && !regs_path(o, n)) e = launch_build(ws, L, dpts, o, n, st);
    if (e == cudaSuccess) e = launch_sample(ws, L, dpts, dout, o, 1, n, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, dout, static_cast<size_t>(m) * 8, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return RFPS_ECUDA;
    return rfps_status_read(workspace, stream);
}

size_t rfps_batch_workspace_size(int64_t total_n, int64_t b, int64_t max_n, const rfps_opts* opts)
{
    if (total_n < 1 || b < 1 || max_n < 1 || check_opts(opts) != RFPS_OK) return 0;
    const rfps_opts o = resolve_opts(opts, max_n);
    return make_layout(total_n, b, max_n, o, false, 0).total;
}

rfps_status rfps_fps_batched(const float* points, int64_t total_n, const int64_t* offsets, int64_t b,
                             const int64_t* out_offsets, const int64_t* starts, int64_t max_n, int64_t* out_idx,
                             const rfps_opts* opts, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!points || !offsets || !out_offsets || !starts || !out_idx || !workspace || b < 1 || total_n < 1 ||
        total_n >= (int64_t(1) << 31) || max_n < 1 || !aligned256(workspace))
        return RFPS_EINVAL;
    rfps_status s = check_opts(opts);
    if (s != RFPS_OK) return s;
    if ((s = device_check()) != RFPS_OK) return s;
    const rfps_opts o = resolve_opts(opts, max_n);
    const WsLayout L = make_layout(total_n, b, max_n, o, false, 0);
    if (workspace_bytes < L.total) return RFPS_ENOMEM;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_setup(ws, L, offsets, out_offsets, starts, b, total_n, 0, 0, 0, max_n, o, st);
    if (e == cudaSuccess && !regs_path(o, max_n)) e = launch_build(ws, L, points, o, max_n, st);
    if (e == cudaSuccess) e = launch_sample(ws, L, points, out_idx, o, b, max_n, st);
    return from_cuda(e);
}

size_t rfps_plain_workspace_size(int64_t total_n, int64_t b)
{
    if (total_n < 1 || b < 1) return 0;
    return make_plain_layout(total_n, b).total;
}

static rfps_status plain_common(const float* points, int64_t total_n, const int64_t* offsets, int64_t b,
                                const int64_t* out_offsets, const int64_t* starts, int64_t n, int64_t m,
                                int64_t start, int64_t max_n, int64_t* out, int32_t variant, void* workspace,
                                size_t workspace_bytes, void* stream)
{
    if (variant < 0 || variant > 2 || (variant == 2 && b != 1)) return RFPS_EINVAL;
    rfps_status s = device_check();
    if (s != RFPS_OK) return s;
    const WsLayout L = make_plain_layout(total_n, b);
    if (workspace_bytes < L.total) return RFPS_ENOMEM;
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rfps_opts o;
    rfps_opts_default(&o);
    o.n_vox = 1;
    cudaError_t e = launch_setup(ws, L, offsets, out_offsets, starts, b, total_n, n, m, start, max_n, o, st);
    if (e == cudaSuccess) e = launch_plain(ws, L, points, out, variant, b, max_n, st);
    return from_cuda(e);
}

rfps_status rfps_plain_fps(const float* points, int64_t n, int64_t m, int64_t start, int64_t* out_idx,
                           int32_t variant, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!points || !out_idx || !workspace || n < 1 || n >= (int64_t(1) << 31) || m < 1 || m > n || start < 0 ||
        start >= n || !aligned256(workspace))
        return RFPS_EINVAL;
    return plain_common(points, n, nullptr, 1, nullptr, nullptr, n, m, start, n, out_idx, variant, workspace,
                        workspace_bytes, stream);
}

rfps_status rfps_plain_fps_batched(const float* points, int64_t total_n, const int64_t* offsets, int64_t b,
                                   const int64_t* out_offsets, const int64_t* starts, int64_t max_n,
                                   int64_t* out_idx, int32_t variant, void* workspace, size_t workspace_bytes,
                                   void* stream)
{
    if (!points || !offsets || !out_offsets || !starts || !out_idx || !workspace || b < 1 || total_n < 1 ||
        total_n >= (int64_t(1) << 31) || max_n < 1 || !aligned256(workspace))
        return RFPS_EINVAL;
    return plain_common(points, total_n, offsets, b, out_offsets, starts, 0, 0, 0, max_n, out_idx, variant,
                        workspace, workspace_bytes, stream);
}

rfps_status rfps_sync_floor(int32_t cluster, int32_t threads, int64_t iterations, void* workspace,
                            size_t workspace_bytes, void* stream)
{
    if (!workspace || iterations < 1 || (threads != 128 && threads != 256 && threads != 512) ||
        (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8 && cluster != 16) ||
        workspace_bytes < 17 * sizeof(unsigned long long) || !aligned256(workspace))
        return RFPS_EINVAL;
    rfps_status s = device_check();
    if (s != RFPS_OK) return s;
    return from_cuda(launch_sync_floor(cluster, threads, iterations, static_cast<unsigned long long*>(workspace),
                                       static_cast<cudaStream_t>(stream)));
}

rfps_status rfps_bandwidth_probe(int32_t kind, const void* buf, int64_t bytes, int32_t reps, void* sink,
                                 int64_t* bytes_moved, int32_t* sm_count, void* stream)
{
    if ((kind != 0 && kind != 1) || reps < 1 || reps > (1 << 20) || !sink ||
        (reinterpret_cast<uintptr_t>(sink) & 7u) != 0)
        return RFPS_EINVAL;
    if (kind == 0 && (!buf || (reinterpret_cast<uintptr_t>(buf) & 15u) != 0 || bytes < 16 || bytes % 16 != 0 ||
                      bytes > (int64_t(1) << 40)))
        return RFPS_EINVAL;
    rfps_status s = device_check();
    if (s != RFPS_OK) return s;
    int64_t moved = 0;
    int sms = 0;
    const cudaError_t e = launch_bw_probe(kind, buf, bytes, reps, static_cast<unsigned long long*>(sink),
                                          static_cast<cudaStream_t>(stream), &moved, &sms);
    if (e != cudaSuccess) return from_cuda(e);
    if (bytes_moved) *bytes_moved = moved;
    if (sm_count) *sm_count = sms;
    return RFPS_OK;
}

rfps_status rfps_status_read(const void* workspace, void* stream)
{
    if (!workspace) return RFPS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader h;
    if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RFPS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RFPS_ECUDA;
    return static_cast<rfps_status>(h.status);
}

rfps_status rfps_counters_read(const void* workspace, rfps_counters* out, void* stream)
{
    if (!workspace || !out) return RFPS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader h;
    if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RFPS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RFPS_ECUDA;
    out->voxel_tests = h.counters[0];
    out->voxels_pruned = h.counters[1];
    out->points_visited = h.counters[2];
    out->points_skipped = h.counters[3];
    out->points_updated = h.counters[4];
    out->iterations = h.counters[5];
    out->prune_violations = h.counters[6];
    out->skip_violations = h.counters[7];
    out->rounds = h.counters[8];
    return RFPS_OK;
}

rfps_status rfps_index_build(const float* points, int64_t n, const rfps_opts* opts, rfps_index** out, void* stream)
{
    if (!points || !out || n < 1 || n >= (int64_t(1) << 31)) return RFPS_EINVAL;
    rfps_status s = check_opts(opts);
    if (s != RFPS_OK) return s;
    if ((s = device_check()) != RFPS_OK) return s;
    *out = nullptr;
    rfps_index* ix = new (std::nothrow) rfps_index;
    if (!ix) return RFPS_ENOMEM;
    ix->o = resolve_opts(opts, n);
    ix->L = make_layout(n, 1, n, ix->o, true, 0);
    ix->n = n;
    ix->stream = static_cast<cudaStream_t>(stream);
    ix->sorted_buf = static_cast<int>(ix->L.radix_passes & 1);
    ix->taken = 0;
    ix->bytes = ix->L.total;
    if (cudaMallocAsync(&ix->mem, ix->bytes, ix->stream) != cudaSuccess) {
        delete ix;
        return RFPS_ENOMEM;
    }
    char* ws = static_cast<char*>(ix->mem);
    float* own = reinterpret_cast<float*>(ws + ix->L.host_points);
    cudaError_t e = cudaMemcpyAsync(own, points, static_cast<size_t>(n) * 12, cudaMemcpyDeviceToDevice, ix->stream);
    if (e == cudaSuccess) e = launch_setup(ws, ix->L, nullptr, nullptr, nullptr, 1, n, n, 1, 0, n, ix->o, ix->stream);
    if (e == cudaSuccess) e = launch_build(ws, ix->L, own, ix->o, n, ix->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(ix->mem, ix->stream);
        delete ix;
        return RFPS_ECUDA;
    }
    *out = ix;
    return RFPS_OK;
}

rfps_status rfps_index_sample(rfps_index* ix, int64_t m, int64_t start, int64_t* out_idx, void* stream)
{
    if (!ix || !out_idx || m < 1 || m > ix->n || start < 0 || start >= ix->n) return RFPS_EINVAL;
    char* ws = static_cast<char*>(ix->mem);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_rearm<<<1, 1, 0, st>>>(reinterpret_cast<WsHeader*>(ws + ix->L.header),
                             reinterpret_cast<CloudDev*>(ws + ix->L.clouds), m, start, 0u);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    const float* own = reinterpret_cast<const float*>(ws + ix->L.host_points);
    if (e == cudaSuccess) e = launch_sample(ws, ix->L, own, out_idx, ix->o, 1, ix->n, st, true);
    ix->taken = e == cudaSuccess ? m : 0;
    return from_cuda(e);
}

rfps_status rfps_index_sample_more(rfps_index* ix, int64_t m_more, int64_t* out_idx, void* stream)
{
    if (!ix || !out_idx || m_more < 1 || ix->taken < 1 || ix->taken + m_more > ix->n) return RFPS_EINVAL;
    char* ws = static_cast<char*>(ix->mem);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // m_more iterations, each applying the pending sample's update and selecting the next one
    k_rearm<<<1, 1, 0, st>>>(reinterpret_cast<WsHeader*>(ws + ix->L.header),
                             reinterpret_cast<CloudDev*>(ws + ix->L.clouds), m_more + 1, 0, 1u);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    const float* own = reinterpret_cast<const float*>(ws + ix->L.host_points);
    if (e == cudaSuccess) e = launch_sample(ws, ix->L, own, out_idx, ix->o, 1, ix->n, st, true);
    if (e != cudaSuccess) {
        ix->taken = 0;
        return RFPS_ECUDA;
    }
    ix->taken += m_more;
    return RFPS_OK;
}

rfps_status rfps_index_distances(const rfps_index* ix, float* d2_out, void* stream)
{
    if (!ix || !d2_out || ix->taken < 1) return RFPS_EINVAL;
    const char* ws = static_cast<const char*>(ix->mem);
    const int64_t blocks = std::min<int64_t>((ix->n + 255) / 256, 4096);
    k_index_d2<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4*>(ws + ix->L.pts4), reinterpret_cast<const uint32_t*>(ws + ix->L.porig), ix->n,
        d2_out);
    note_launches(1);
    return from_cuda(cudaGetLastError());
}

rfps_status rfps_index_status_copy(const rfps_index* ix, int32_t* host_status, void* stream)
{
    if (!ix || !host_status) return RFPS_EINVAL;
    const WsHeader* h = reinterpret_cast<const WsHeader*>(static_cast<const char*>(ix->mem) + ix->L.header);
    return from_cuda(cudaMemcpyAsync(host_status, &h->status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     static_cast<cudaStream_t>(stream)));
}

size_t rfps_index_bytes(const rfps_index* ix) { return ix ? ix->bytes : 0; }

void rfps_index_free(rfps_index* ix)
{
    if (!ix) return;
    cudaFreeAsync(ix->mem, ix->stream);
    delete ix;
}

rfps_status rfps_index_export(const rfps_index* ix, int64_t* n_records, uint32_t* voxel_id, uint32_t* first,
                              uint32_t* count, float* sphere4, uint32_t* sorted_orig, float* grid4, int32_t* n_vox)
{
    if (!ix || !n_records) return RFPS_EINVAL;
    if (cudaStreamSynchronize(ix->stream) != cudaSuccess) return RFPS_ECUDA;
    const char* ws = static_cast<const char*>(ix->mem);
    WsHeader h;
    CloudDev c;
    if (cudaMemcpy(&h, ws + ix->L.header, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return RFPS_ECUDA;
    if (cudaMemcpy(&c, ws + ix->L.clouds, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return RFPS_ECUDA;
    if (h.status != 0) return static_cast<rfps_status>(h.status);
    const int64_t R = h.n_records;
    *n_records = R;
    const size_t n = static_cast<size_t>(ix->n);
    uint2* rng = static_cast<uint2*>(std::malloc(static_cast<size_t>(R) * sizeof(uint2)));
    uint32_t* keys = static_cast<uint32_t*>(std::malloc(n * 4));
    if (!rng || !keys) {
        std::free(rng);
        std::free(keys);
        return RFPS_ENOMEM;
    }
    const size_t kb = ix->sorted_buf ? ix->L.keys1 : ix->L.keys0;
    rfps_status s = RFPS_OK;
    if (cudaMemcpy(rng, ws + ix->L.rec_rng, R * sizeof(uint2), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(keys, ws + kb, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = RFPS_ECUDA;
    if (s == RFPS_OK) {
        for (int64_t r = 0; r < R; ++r) {
            if (voxel_id) {
                const uint32_t code = keys[rng[r].x] - c.cell_base;   // Morton code -> v_z n^2 + v_y n + v_x
                const uint32_t n = static_cast<uint32_t>(c.n_vox);
                voxel_id[r] = (morton_compact(code >> 2) * n + morton_compact(code >> 1)) * n + morton_compact(code);
            }
            if (first) first[r] = rng[r].x;
            if (count) count[r] = rng[r].y;
        }
        if (sphere4 && cudaMemcpy(sphere4, ws + ix->L.rec_sph, R * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            s = RFPS_ECUDA;
        if (sorted_orig && cudaMemcpy(sorted_orig, ws + ix->L.porig, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            s = RFPS_ECUDA;
        if (grid4) {
            grid4[0] = c.gmin[0];
            grid4[1] = c.gmin[1];
            grid4[2] = c.gmin[2];
            grid4[3] = c.L;
        }
        if (n_vox) *n_vox = c.n_vox;
    }
    std::free(rng);
    std::free(keys);
    return s;
}

}  // extern "C"
