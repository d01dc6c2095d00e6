/*
 * rfps.h -- C ABI of the GB300 (sm_103a) RadiusFPS library (librfps.so).
 *
 * Exact farthest point sampling (FPS) accelerated by spherical-voxel
 * pruning, after "RadiusFPS" (Sec. 3 and Sec. 4 of the paper).  Given a cloud
 * P = {p_0 .. p_{N-1}} in R^3, a sample count M and a start index, the
 * library returns the M indices that plain FPS (Alg. 1) selects, in
 * selection order, in the original indexing of P (Sec. 3.1, Notation).
 *
 * Arithmetic contract (identical results on every path of this library):
 *   - distances are FP32 squared distances (dx*dx + dy*dy) + dz*dz with
 *     dx = p.x - q.x etc., each operation rounded to nearest, no fused
 *     multiply-add, no flush-to-zero;
 *   - each point keeps its FP32 squared distance to the nearest sample and
 *     replaces it only by a strictly smaller value;
 *   - argmax ties go to the smallest original index (Sec. 3.1).
 * The voxel pruning (Sec. 3.4.2) and the point skip (Sec. 3.4.3) are
 * conservative in this arithmetic, so the RadiusFPS path returns exactly the
 * plain-FPS indices.
 *
 * Conventions for every call:
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary CPU memory;
 *   - points are an array of N x 3 float32 in (x, y, z) order, row-major
 *     (array of structures), 4-byte aligned; the library only reads them;
 *   - output indices are int64 in original (per-cloud) indexing;
 *   - the caller owns every buffer it passes; the library never frees or
 *     keeps a caller buffer beyond the call (rfps_index_* keeps its own copy);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is enqueued on it asynchronously unless a call
 *     says it synchronises;
 *   - a call that returns RFPS_OK has enqueued its work.  Argument errors are
 *     found on the host before anything is enqueued.  Errors only the device
 *     can see (a non-finite coordinate, an invalid per-cloud entry of a
 *     device array) are written to a status word in the workspace and read
 *     back with rfps_status_read();
 *   - no call traps, asserts on the device or waits without a bound.
 */
#ifndef RFPS_H
#define RFPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    RFPS_OK = 0,
    RFPS_EINVAL = 1,      /* invalid argument (host check, or device check of a device array) */
    RFPS_ENONFINITE = 2,  /* a coordinate is NaN or +-inf (found on the device) */
    RFPS_ENOMEM = 3,      /* workspace too small, or a device allocation failed */
    RFPS_ECUDA = 4,       /* a CUDA runtime call failed */
    RFPS_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    RFPS_EUNSUPPORTED = 6, /* no sm_103a device, or a launch shape the device cannot run */
    RFPS_EBOUNDS = 7      /* bounds-checked test builds only: an index taken from data was out of range */
} rfps_status;

/* Tuning knobs.  Zero means "choose automatically" for every field but the
 * three switches, whose defaults (from rfps_opts_default) are 1, 1, 0. */
typedef struct {
    int32_t n_vox;       /* voxel bins per axis, n_vox of Sec. 3.2 (v in Sec. 5.6.2); 1..256 */
    int32_t cluster;     /* CTAs working on one cloud (thread-block cluster size): 1,2,4,8,16 */
    int32_t threads;     /* threads per CTA of the sampling kernel: 128, 256 or 512.  With
                            cluster 1 and 512 threads, clouds of at most 4,096 points run on
                            the register-record path instead: one CTA of 1,024 threads, each
                            holding up to 4 consecutive sorted points as one record of its own
                            (radius_mode and chunk then apply to nothing) */
    int32_t chunk;       /* max points per voxel record (a voxel with more points is split
                            into several records): power of two in 32..4096; default 128 */
    int32_t prune;       /* 1: spherical-voxel radius pruning (Sec. 3.4.2) on */
    int32_t skip;        /* 1: coordinate-wise point skip (Sec. 3.4.3) on */
    int32_t radius_mode; /* 0: radius measured over the members (tighter, default);
                            1: the paper's sqrt(3)/2 * L (Eq. preprocess_voxel_radius),
                               raised to the measured value if rounding requires it */
    int32_t counters;    /* 1: accumulate work counters (rfps_counters_read); slower */
    int32_t nvox_scale;  /* automatic resolution (n_vox = 0): each cloud gets
                            n_vox = round(nvox_scale / 100 * cbrt(N)) bins per axis;
                            0 means 70, valid 1..1000.  Ignored when n_vox > 0 */
} rfps_opts;

/* Work counters of the sampling loop (Fig. samplestep / Tab. ablation
 * statistics), summed over all iterations and clouds of one call. */
typedef struct {
    uint64_t voxel_tests;     /* voxel-record prune tests */
    uint64_t voxels_pruned;   /* records skipped by Eq. radius_pruning_condition */
    uint64_t points_visited;  /* points of unpruned records, once per visit (a visit applies
                                 the one or two samples of its round) */
    uint64_t points_skipped;  /* visited points dropped by Eq. point_skip_condition for every
                                 sample the visit applied */
    uint64_t points_updated;  /* visited points whose stored distance decreased (effective
                                 updates) */
    uint64_t iterations;      /* sampling iterations (selections after the start point) */
    uint64_t prune_violations; /* shadow check: points of pruned records whose distance to the
                                  new sample was below their stored one (0 when the bound is safe) */
    uint64_t skip_violations;  /* shadow check: skipped points whose distance to the new sample was
                                  below their stored one (0 when the skip is exact) */
    uint64_t rounds;          /* selection rounds (cluster exchanges); a round selects two samples
                                  when the runner-up shortcut applies, so rounds <= iterations */
} rfps_counters;

/* Fills *opts with the defaults (all automatic, prune = skip = 1). */
void rfps_opts_default(rfps_opts *opts);

/* The options a call on a cloud of n points will use, automatic fields
 * resolved (host only, no device work): up to 4,096 points cluster 1 and
 * threads 512 (the register-record path), above that clusters of 16 CTAs of 256
 * threads; records of at most 128 points, nvox_scale 70; n_vox stays 0 when
 * automatic because the device picks it per cloud (nvox_scale / 100 *
 * cbrt(N)).  RFPS_EINVAL for invalid options. */
rfps_status rfps_opts_resolve(int64_t n, const rfps_opts *in, rfps_opts *out);

/* Human-readable name of a status code (static string, never NULL). */
const char *rfps_status_str(int status);

/* Library ABI version (increments when a signature or struct changes). */
int rfps_version(void);

/* Total kernels this process has launched through the library so far. */
int64_t rfps_launch_count(void);

/* ------------------------------------------------------------------------
 * Single cloud.
 *
 * rfps_fps: M samples of one cloud with RadiusFPS (Sec. 3, Sec. 4): the
 * device builds the spherical-voxel index (bounding box, Eq. voxel_size,
 * binning, active voxels with centre and radius -- Sec. 3.2, Alg.
 * voxelization_gpu), runs the initial update from `start` (Sec. 3.3), then
 * M - 1 iterations of select / radius prune / point skip / update / voxel
 * resync (Sec. 3.4) in one persistent kernel.
 *   points     device, N x 3 float32
 *   n          N >= 1, N < 2^31
 *   m          1 <= M <= N
 *   start      0 <= start < N (the paper draws it uniformly, Sec. 3.3; here the
 *              caller chooses it)
 *   out_idx    device, M int64, receives the indices; out_idx[0] = start
 *   opts       NULL for defaults
 *   workspace  device scratch of at least rfps_fps_workspace_size() bytes,
 *              256-byte aligned, owned by the caller, not read before the call
 *              (its status word is valid until the next call that uses it)
 * Errors: RFPS_EINVAL (bad argument, nothing enqueued), RFPS_ENOMEM
 * (workspace too small), RFPS_EUNSUPPORTED, RFPS_ECUDA; a non-finite
 * coordinate is reported by rfps_status_read() as RFPS_ENONFINITE and then
 * out_idx is left unspecified.
 * ---------------------------------------------------------------------- */
size_t rfps_fps_workspace_size(int64_t n, const rfps_opts *opts);
rfps_status rfps_fps(const float *points, int64_t n, int64_t m, int64_t start,
                     int64_t *out_idx, const rfps_opts *opts, void *workspace,
                     size_t workspace_bytes, void *stream);

/* rfps_fps_lost_round: a test of the device-side failure path of rfps_fps.
 * The same call with work counters on, except that in sampling iteration
 * `lost_iteration` (1 <= lost_iteration < M) no CTA sends its candidate to the
 * cluster exchange (Sec. 4.2's per-iteration synchronisation), as if those
 * messages were lost.  Every exchange wait of that iteration then gives up
 * after `spin_limit` polls (1 .. 2^22; rfps_fps uses 2^22), the launch records
 * RFPS_ETIMEOUT in the workspace's status word (rfps_status_read) and the CTAs
 * of the cluster leave the kernel together; out_idx is then unspecified.  No
 * exchange message is in flight when the waits give up: every earlier
 * iteration's messages have arrived (their waits completed) and the lost one
 * sends none.  The workspace can be used again by the next call.  Needs a
 * cluster of at least 2 CTAs (a single CTA has no exchange): RFPS_EINVAL
 * otherwise, as for M < 2.  Other arguments and errors as rfps_fps. */
rfps_status rfps_fps_lost_round(const float *points, int64_t n, int64_t m,
                                int64_t start, int64_t *out_idx,
                                const rfps_opts *opts, void *workspace,
                                size_t workspace_bytes, int64_t lost_iteration,
                                uint32_t spin_limit, void *stream);

/* rfps_fps_host: the same call on HOST buffers.  Copies the points into the
 * workspace (which must hold rfps_fps_host_workspace_size() bytes), samples,
 * copies the indices back to host_out, and synchronises `stream`.  Returns
 * the device status (so RFPS_ENONFINITE is reported directly). */
size_t rfps_fps_host_workspace_size(int64_t n, const rfps_opts *opts);
rfps_status rfps_fps_host(const float *host_points, int64_t n, int64_t m,
                          int64_t start, int64_t *host_out, const rfps_opts *opts,
                          void *workspace, size_t workspace_bytes, void *stream);

/* rfps_fps_noalloc: rfps_fps for callers that cannot allocate device memory
 * on their own path (a real-time loop that cannot afford an allocation's
 * implicit synchronisation and latency, a plug-in inside an application
 * whose allocator owns the device, code running while the device heap is
 * reserved).  The paper has no counterpart: it is an interface choice of this
 * library.  The scratch is a 64 MiB array compiled into librfps.so; each GPU
 * that loads the library holds it until the process exits.  The call takes
 * only the input and output buffers (same meaning as rfps_fps) and calls no
 * allocating routine.  N whose rfps_fps workspace exceeds 64 MiB (with
 * default options, N above 725,440 points) is rejected with RFPS_ENOMEM.  Every call on a GPU
 * shares the one array: calls whose work overlaps on the GPU race, so
 * serialise them (one stream, or events).  The kernels reset the state they
 * need at the start of each call.  Every call looks up the array's device
 * address (cudaGetSymbolAddress) on the current device; the first call on a
 * device may load the library's device code and should come before any stream
 * capture.  Errors only the device can see (a non-finite coordinate, a
 * cluster exchange wait that gave up) are not returned by this call: read
 * them with rfps_noalloc_status_read, after which the output of a failed call
 * is unspecified. */
rfps_status rfps_fps_noalloc(const float *points, int64_t n, int64_t m,
                             int64_t start, int64_t *out_idx,
                             const rfps_opts *opts, void *stream);
/* rfps_noalloc_status_read: the device status of the last rfps_fps_noalloc
 * call on the current device (RFPS_OK if it recorded no error), read from the
 * fixed array into a host variable; synchronises `stream`, which must be the
 * stream of that call or ordered after it.  Allocates nothing.  The paper has
 * no counterpart. */
rfps_status rfps_noalloc_status_read(void *stream);

/* ------------------------------------------------------------------------
 * Ragged batch: B clouds concatenated in one point array, sampled by one
 * persistent launch whose CTA clusters take clouds from a device work queue
 * (largest clouds first).
 *   points       device, total_n x 3 float32 (cloud b = rows offsets[b] ..
 *                offsets[b+1]-1)
 *   offsets      device int64[B+1], offsets[0] = 0, non-decreasing,
 *                offsets[B] = total_n, every cloud non-empty
 *   out_offsets  device int64[B+1]: cloud b writes M_b = out_offsets[b+1] -
 *                out_offsets[b] indices at out_idx + out_offsets[b];
 *                1 <= M_b <= N_b
 *   starts       device int64[B], start index of each cloud in its own indexing
 *   max_n        host-known upper bound on every N_b (sizes the launch)
 *   out_idx      device int64[out_offsets[B]], per-cloud (local) indices
 * Device-detected violations of the array contracts set RFPS_EINVAL in the
 * status word and skip the offending cloud.
 * ---------------------------------------------------------------------- */
size_t rfps_batch_workspace_size(int64_t total_n, int64_t b, int64_t max_n,
                                 const rfps_opts *opts);
rfps_status rfps_fps_batched(const float *points, int64_t total_n,
                             const int64_t *offsets, int64_t b,
                             const int64_t *out_offsets, const int64_t *starts,
                             int64_t max_n, int64_t *out_idx,
                             const rfps_opts *opts, void *workspace,
                             size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Plain O(N*M) GPU FPS (Alg. 1), the comparison baseline, same arithmetic
 * and tie rule.
 *   variant 0: one CTA per cloud streaming the cloud every iteration (the
 *              classic FPS kernel design);
 *   variant 1: one thread-block cluster per cloud with the cloud resident in
 *              the cluster's shared memory when it fits, else streamed from L2;
 *   variant 2: the whole GPU on one cloud: one CTA per SM, each holding a
 *              slice of the cloud in shared memory, with a bounded
 *              software grid barrier per iteration (single cloud only).
 * Batched form: same array contracts as rfps_fps_batched (variants 0 and 1).
 * ---------------------------------------------------------------------- */
size_t rfps_plain_workspace_size(int64_t total_n, int64_t b);
rfps_status rfps_plain_fps(const float *points, int64_t n, int64_t m,
                           int64_t start, int64_t *out_idx, int32_t variant,
                           void *workspace, size_t workspace_bytes, void *stream);
rfps_status rfps_plain_fps_batched(const float *points, int64_t total_n,
                                   const int64_t *offsets, int64_t b,
                                   const int64_t *out_offsets,
                                   const int64_t *starts, int64_t max_n,
                                   int64_t *out_idx, int32_t variant,
                                   void *workspace, size_t workspace_bytes,
                                   void *stream);

/* ------------------------------------------------------------------------
 * Measurement of the sampling loop's synchronisation floor: one CTA cluster
 * of `cluster` CTAs x `threads` threads runs `iterations` rounds of exactly
 * the selection step of the RadiusFPS kernel (warp argmax, CTA reduction, the
 * DSMEM exchange and one barrier per round) with no voxel or point work.
 * The caller times the launch (e.g. CUDA events on `stream`); time divided by
 * iterations is the per-iteration floor of the sampling loop (Sec. 4.2's
 * "only synchronization point" of each iteration).  `workspace`: device, at
 * least 136 bytes, 256-byte aligned: one value per CTA (16 x 8 bytes), then a
 * status word (RFPS_ETIMEOUT if a bounded wait gave up; the caller zeroes it).
 * cluster in {1, 2, 4, 8, 16}, threads in {128, 256, 512}.
 * ---------------------------------------------------------------------- */
rfps_status rfps_sync_floor(int32_t cluster, int32_t threads, int64_t iterations,
                            void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * On-chip bandwidth probe, the denominator of the sampling kernel's on-chip
 * roofline.  After the first touch, the per-iteration traffic of the loop
 * (record tests, point visits, updates; Sec. 3.3-3.4) is served from shared
 * memory and L2, not DRAM.  One launch on `stream`, timed by the caller.
 *   kind 0  L2 reads: every SM streams `bytes` of the device buffer `buf`
 *           (16-byte aligned, bytes a positive multiple of 16, read only)
 *           with L2-only loads, `reps` passes.  For the L2 figure the buffer
 *           must fit in L2 and have been touched once (a warm-up launch).
 *   kind 1  shared-memory reads: every resident CTA reads a 48 KiB array of
 *           its own `reps` times, conflict-free; `buf` and `bytes` unused.
 * reps in [1, 2^20].  `sink`: device, 8-byte aligned, 8 bytes; the probe XORs
 * what it read into it (its value has no meaning).  On return, the optional
 * host pointers receive the bytes the launch reads (`bytes_moved`) and the
 * device's SM count (`sm_count`); read bandwidth = bytes_moved / launch time.
 * Invalid arguments: RFPS_EINVAL, nothing launched.
 * ---------------------------------------------------------------------- */
rfps_status rfps_bandwidth_probe(int32_t kind, const void *buf, int64_t bytes,
                                 int32_t reps, void *sink, int64_t *bytes_moved,
                                 int32_t *sm_count, void *stream);

/* ------------------------------------------------------------------------
 * Device status and counters of a workspace.  Both synchronise `stream`.
 * rfps_status_read returns the first error the device recorded for the last
 * call that used `workspace` (RFPS_OK if none).
 * rfps_counters_read fills *out with the counters of the last call that ran
 * with opts.counters = 1 (zeros otherwise).
 * ---------------------------------------------------------------------- */
rfps_status rfps_status_read(const void *workspace, void *stream);
rfps_status rfps_counters_read(const void *workspace, rfps_counters *out,
                               void *stream);

/* ------------------------------------------------------------------------
 * Persistent index for serving: the spherical-voxel index (Sec. 3.2) of one
 * cloud is built once, kept on the device in library-owned memory, and
 * sampled any number of times with different M / start.
 *   rfps_index_build   copies nothing from the caller after it returns: the
 *                      index holds the sorted points it needs.  Allocates
 *                      device memory (cudaMallocAsync on `stream`).
 *   rfps_index_sample  M samples from the index (same contract as rfps_fps);
 *                      starts a new sequence and keeps its state on the device.
 *   rfps_index_bytes   device bytes the index holds.
 *   rfps_index_free    releases the index (stream-ordered on the stream it was
 *                      built on); NULL is ignored.
 *   rfps_index_export  copies the voxel records to HOST arrays for inspection
 *                      (synchronises): per record its voxel id (v_z n^2 + v_y n
 *                      + v_x), first sorted position, point count, centre and
 *                      radius (float4 each), plus each sorted position's
 *                      original index.  Pass NULL for arrays not wanted;
 *                      *n_records receives the record count.
 * ---------------------------------------------------------------------- */
typedef struct rfps_index rfps_index;
rfps_status rfps_index_build(const float *points, int64_t n,
                             const rfps_opts *opts, rfps_index **out,
                             void *stream);
rfps_status rfps_index_sample(rfps_index *index, int64_t m, int64_t start,
                              int64_t *out_idx, void *stream);
/* rfps_index_sample_more: incremental sampling.  Continues the sequence of the
 * last rfps_index_sample / rfps_index_sample_more call on this index and
 * writes the next m_more indices (device, int64) to out_idx.  The FPS state
 * stays on the device between calls: every point's distance to the samples so
 * far, each voxel record's Dist_v key, best point and prune threshold, and
 * the last sample, whose update Alg. 1 applies before the next selection.  The
 * result equals the corresponding slice of rfps_fps with M = (samples so far)
 * + m_more.  RFPS_EINVAL without a prior rfps_index_sample, or if the total
 * would exceed N.  One sequence per index at a time (stream-ordered). */
rfps_status rfps_index_sample_more(rfps_index *index, int64_t m_more,
                                   int64_t *out_idx, void *stream);
/* rfps_index_distances: the FPS state of the current sequence, Alg. 1's D:
 * every point's FP32 squared distance (canonical arithmetic) to the samples
 * whose update has been applied, i.e. all but the last sample taken (its
 * update opens the next rfps_index_sample_more).  Written to the DEVICE
 * array d2_out[n] in the caller's point order, stream-ordered on `stream`
 * after the sampling calls there.  RFPS_EINVAL before the first
 * rfps_index_sample. */
rfps_status rfps_index_distances(const rfps_index *index, float *d2_out,
                                 void *stream);
/* rfps_index_status_copy: enqueues on `stream` a copy of the index's device
 * status word (the first error recorded by its last build or sampling call,
 * RFPS_OK if none; the same codes as rfps_status_read) into *host_status.
 * Page-locked host memory keeps the copy asynchronous; read the value once
 * the stream has passed this point (e.g. after an event recorded behind it). */
rfps_status rfps_index_status_copy(const rfps_index *index,
                                   int32_t *host_status, void *stream);
size_t rfps_index_bytes(const rfps_index *index);
void rfps_index_free(rfps_index *index);
rfps_status rfps_index_export(const rfps_index *index, int64_t *n_records,
                              uint32_t *voxel_id, uint32_t *first,
                              uint32_t *count, float *sphere4,
                              uint32_t *sorted_orig, float *grid4,
                              int32_t *n_vox);

#ifdef __cplusplus
}
#endif

#endif /* RFPS_H */
