/*
 * CPU oracle for exact farthest point sampling (FPS) and for RadiusFPS.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously correct
 * reference the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library's
 * product path never calls it and shares no code with it.
 *
 * Arithmetic (the reading every caller relies on):
 *   - distances are FP32 SQUARED Euclidean distances, evaluated as
 *       dx = p.x - q.x, dy = ..., dz = ...   (each rounded to fp32)
 *       d2 = (dx*dx + dy*dy) + dz*dz          (each product and sum rounded)
 *     with no fused multiply-add: the file is compiled with
 *     -ffp-contract=off and without -ffast-math;
 *   - the running nearest-sample distance is stored in FP32;
 *   - argmax ties go to the smallest original index (Sec. 3.1, Notation);
 *   - a point's distance is replaced only by a strictly smaller value
 *     (Alg. 1 takes the min; Eq. radius_pruning_correctness relies on the
 *     strict update).
 *
 * Functions (each cites the passage it follows):
 *   oracle_fps          plain FPS, Alg. 1 and Sec. 3.1          (pinned)
 *   oracle_radiusfps    the paper's CPU RadiusFPS, Sec. 3.2-3.4  (pinned
 *                       against oracle_fps: identical indices)
 *   oracle_voxelize     the voxel grid of Sec. 3.2               (pinned)
 *   oracle_fps_f64      FP64 sqrt-domain FPS, information only   (pinned
 *                       by the same hand-worked examples)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENONFINITE 2
#define ORACLE_ENOMEM 3

/* Squared distance between p and q in the canonical FP32 order. */
static float sq_dist(const float *p, const float *q)
{
    float dx = p[0] - q[0];
    float dy = p[1] - q[1];
    float dz = p[2] - q[2];
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    return s + zz;
}

static int check_args(const float *pts, int64_t n, int64_t m, int64_t start)
{
    if (pts == NULL || n < 1 || m < 1 || m > n || start < 0 || start >= n)
        return ORACLE_EINVAL;
    if (n > (int64_t)0xFFFFFFF0LL)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(pts[i]))
            return ORACLE_ENONFINITE;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Plain FPS (Alg. 1; Sec. 2.1; Sec. 3.1 Notation and tie rule).
 *
 *   D[i] = +inf for all i; out[0] = start
 *   for j = 1 .. M-1:
 *       for all i: D[i] = min(D[i], d2(p_i, s_{j-1}))      (strict update)
 *       s_j = argmax_i D[i], ties -> smallest i
 *
 * The first pass of the loop (s_0 = start) is the paper's initial update
 * (Sec. 3.3): it sets D[i] = d2(p_i, s_0) and D[start] = 0.
 * threads <= 0 uses every OpenMP thread; 1 runs serially.  The result does
 * not depend on the thread count: the min is per point and the argmax is
 * combined with the same (value, then smaller index) rule.
 * d2_out (nullable) receives D after the last update (with s_{M-2}).
 * ---------------------------------------------------------------------- */
int oracle_fps(const float *pts, int64_t n, int64_t m, int64_t start,
               int64_t *out, float *d2_out, int threads)
{
    int rc = check_args(pts, n, m, start);
    if (rc != ORACLE_OK || out == NULL)
        return rc != ORACLE_OK ? rc : ORACLE_EINVAL;
    float *D = (float *)malloc((size_t)n * sizeof(float));
    if (D == NULL)
        return ORACLE_ENOMEM;
    for (int64_t i = 0; i < n; ++i)
        D[i] = INFINITY;
    out[0] = start;
    int64_t s = start;
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    int nt = 1;
    (void)threads;
#endif
    for (int64_t j = 1; j < m; ++j) {
        const float *ps = pts + 3 * s;
        float best_v = -1.0f;
        int64_t best_i = -1;
        if (nt == 1) {
            for (int64_t i = 0; i < n; ++i) {
                float d = sq_dist(pts + 3 * i, ps);
                if (d < D[i])
                    D[i] = d;
                if (D[i] > best_v) {      /* strict: keeps the smallest index */
                    best_v = D[i];
                    best_i = i;
                }
            }
        } else {
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
            {
                float tv = -1.0f;
                int64_t ti = -1;
#pragma omp for schedule(static)
                for (int64_t i = 0; i < n; ++i) {
                    float d = sq_dist(pts + 3 * i, ps);
                    if (d < D[i])
                        D[i] = d;
                    if (D[i] > tv) {
                        tv = D[i];
                        ti = i;
                    }
                }
#pragma omp critical
                {
                    if (ti >= 0 && (tv > best_v || (tv == best_v && ti < best_i))) {
                        best_v = tv;
                        best_i = ti;
                    }
                }
            }
#endif
        }
        s = best_i;
        out[j] = s;
    }
    if (d2_out != NULL)
        memcpy(d2_out, D, (size_t)n * sizeof(float));
    free(D);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Voxel grid of Sec. 3.2 (Eq. voxel_size and the clamped binning formula).
 *
 *   p_min, p_max = bounding box;  E = p_max - p_min
 *   L = alpha * max(E) / n_vox,  alpha = 1 + eps, eps = 2^-10
 *   v_a = min(n_vox - 1, max(0, floor((p_a - p_min_a) / L)))
 *   voxel id = v_z * n_vox^2 + v_y * n_vox + v_x   (Sec. 4.1)
 *
 * The paper leaves eps unstated ("eps << 1"); 2^-10 is this project's
 * choice.  If every point coincides (max(E) = 0) the paper's L would be 0;
 * then L = 1 and every point falls in voxel 0.
 * grid_out receives {min_x, min_y, min_z, max_x, max_y, max_z, L}.
 * ---------------------------------------------------------------------- */
static float voxel_side(const float *mn, const float *mx, int n_vox)
{
    float ex = mx[0] - mn[0], ey = mx[1] - mn[1], ez = mx[2] - mn[2];
    float e = ex;
    if (ey > e) e = ey;
    if (ez > e) e = ez;
    if (!(e > 0.0f))
        return 1.0f;
    const float alpha = 1.0f + 0.0009765625f; /* 1 + 2^-10 */
    float t = alpha * e;
    return t / (float)n_vox;
}

static uint32_t voxel_coord(float p, float mn, float L, int n_vox)
{
    float q = (p - mn) / L;
    float f = floorf(q);
    if (f < 0.0f)
        f = 0.0f;
    if (f > (float)(n_vox - 1))
        f = (float)(n_vox - 1);
    return (uint32_t)f;
}

int oracle_voxelize(const float *pts, int64_t n, int n_vox, float *grid_out,
                    uint32_t *vid_out)
{
    if (pts == NULL || n < 1 || n_vox < 1 || n_vox > 1024 || vid_out == NULL)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(pts[i]))
            return ORACLE_ENONFINITE;
    float mn[3] = {pts[0], pts[1], pts[2]};
    float mx[3] = {pts[0], pts[1], pts[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = pts[3 * i + a];
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    float L = voxel_side(mn, mx, n_vox);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t vx = voxel_coord(pts[3 * i + 0], mn[0], L, n_vox);
        uint32_t vy = voxel_coord(pts[3 * i + 1], mn[1], L, n_vox);
        uint32_t vz = voxel_coord(pts[3 * i + 2], mn[2], L, n_vox);
        vid_out[i] = (vz * (uint32_t)n_vox + vy) * (uint32_t)n_vox + vx;
    }
    if (grid_out != NULL) {
        for (int a = 0; a < 3; ++a) {
            grid_out[a] = mn[a];
            grid_out[3 + a] = mx[a];
        }
        grid_out[6] = L;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * CPU RadiusFPS (Sec. 3.2 - 3.4), steps in the paper's order:
 *   preprocessing (Sec. 3.2): voxel grid, active voxels, centres c_k,
 *       bounding-sphere radii r_k, Dist_p = +inf;
 *   initial update (Sec. 3.3): Dist_p[i] = d2(p_i, s_0) for all i, then
 *       Dist_v[k] = max over the voxel (Eq. preprocess_distv);
 *   for j = 1 .. M-1:
 *       select (Sec. 3.4.1): k* = argmax_k Dist_v[k] (Eq. best_voxel), then
 *           s_j = argmax over v_k* of Dist_p (Eq. best_point); ties at both
 *           levels go to the smallest original index, so the two-level
 *           choice equals the global one (Eq. global_equivalent_selection);
 *       for every active voxel:
 *           radius pruning (Sec. 3.4.2, Eq. radius_pruning_condition);
 *           point skip (Sec. 3.4.3, Eq. point_skip_condition);
 *           exact update (Eq. point_distance_update);
 *           Dist_v sync of visited voxels (Eq. point_skip_distv_sync).
 *
 * Readings of the paper in floating point (the paper states the tests over
 * the reals):
 *   - Distances are squared FP32, as in oracle_fps; Dist_v[k] holds the max
 *     squared distance of the voxel and the smallest index attaining it.
 *   - Point skip: skip p_i if fl(dx*dx) >= D[i] for some axis, with the same
 *     rounded terms that make up d2.  Because adding non-negative floats is
 *     monotone under round-to-nearest, d2 >= fl(da*da) >= D[i] then holds,
 *     so the strict update could not fire: the skip is exact.
 *   - Radius pruning is decided in double precision with margins.  With
 *     u = 2^-24, the FP32 d2 of any p satisfies d2 >= (1 - 5u)|p - s|^2 when
 *     |p - s|^2 >= 2^-100.  The bound lb <= |s - c_k| - r_k <= |p - s| is
 *     formed with relative slack 2^-48 on both terms (covering the double
 *     rounding of the distances), and the voxel is pruned only if
 *     lb^2 (1 - 2^-20) >= Dist_v[k] (and lb^2 >= 2^-100), which then implies
 *     d2(p, s) >= Dist_v[k] >= D[i] for every member: no update can fire.
 *     A voxel whose Dist_v is 0 cannot change either and is pruned.
 *   - r_k: radius_mode 0 measures the members (max |p - c_k| in double,
 *     times 1 + 2^-48); radius_mode 1 takes the paper's sqrt(3)/2 * L
 *     (Eq. preprocess_voxel_radius), raised to the measured value if a
 *     rounding of the binning left a member outside it.
 *   - c_k = p_min + (v + 1/2) L per axis (the voxel's geometric centre),
 *     evaluated in FP32.
 *
 * prune / skip switch the two filters (the ablation of Tab. ablation); the
 * result must not depend on them.  stats (nullable, 6 entries) receives:
 *   voxel tests, voxels pruned, points visited, points skipped, points
 *   updated, active voxels.
 * ---------------------------------------------------------------------- */
int oracle_radiusfps(const float *pts, int64_t n, int64_t m, int64_t start,
                     int n_vox, int prune, int skip, int radius_mode,
                     int64_t *out, int64_t *stats)
{
    int rc = check_args(pts, n, m, start);
    if (rc != ORACLE_OK)
        return rc;
    if (out == NULL || n_vox < 1 || n_vox > 1024)
        return ORACLE_EINVAL;

    /* Sec. 3.2: voxel grid and per-point voxel id */
    uint32_t *vid = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    float grid[7];
    if (vid == NULL)
        return ORACLE_ENOMEM;
    rc = oracle_voxelize(pts, n, n_vox, grid, vid);
    if (rc != ORACLE_OK) {
        free(vid);
        return rc;
    }
    const float L = grid[6];

    /* active voxels: sort point indices by (voxel id, index) -- a counting
       sort by voxel id that visits points in index order, so members of a
       voxel are listed in increasing original index */
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (order == NULL || tmp == NULL) {
        free(vid); free(order); free(tmp);
        return ORACLE_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i)
        order[i] = i;
    /* LSD radix sort on the voxel id, 8 bits per pass, stable */
    for (int shift = 0; shift < 32; shift += 8) {
        int64_t cnt[257];
        memset(cnt, 0, sizeof(cnt));
        for (int64_t i = 0; i < n; ++i)
            cnt[((vid[order[i]] >> shift) & 255u) + 1]++;
        for (int b = 0; b < 256; ++b)
            cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < n; ++i)
            tmp[cnt[(vid[order[i]] >> shift) & 255u]++] = order[i];
        int64_t *sw = order; order = tmp; tmp = sw;
    }
    free(tmp);
    int64_t K = 0;
    for (int64_t i = 0; i < n; ++i)
        if (i == 0 || vid[order[i]] != vid[order[i - 1]])
            ++K;
    int64_t *vbeg = (int64_t *)malloc((size_t)(K + 1) * sizeof(int64_t));
    float *cen = (float *)malloc((size_t)K * 3 * sizeof(float));
    double *rad = (double *)malloc((size_t)K * sizeof(double));
    float *dv = (float *)malloc((size_t)K * sizeof(float));
    int64_t *dv_idx = (int64_t *)malloc((size_t)K * sizeof(int64_t));
    float *D = (float *)malloc((size_t)n * sizeof(float));
    if (!vbeg || !cen || !rad || !dv || !dv_idx || !D) {
        free(vid); free(order); free(vbeg); free(cen); free(rad); free(dv); free(dv_idx); free(D);
        return ORACLE_ENOMEM;
    }
    K = 0;
    for (int64_t i = 0; i < n; ++i)
        if (i == 0 || vid[order[i]] != vid[order[i - 1]])
            vbeg[K++] = i;
    vbeg[K] = n;

    /* centres and bounding-sphere radii (Eq. preprocess_voxel_radius) */
    for (int64_t k = 0; k < K; ++k) {
        uint32_t id = vid[order[vbeg[k]]];
        uint32_t v[3] = {id % (uint32_t)n_vox, (id / (uint32_t)n_vox) % (uint32_t)n_vox,
                         id / ((uint32_t)n_vox * (uint32_t)n_vox)};
        for (int a = 0; a < 3; ++a)
            cen[3 * k + a] = grid[a] + ((float)v[a] + 0.5f) * L;
        double rmax = 0.0;
        for (int64_t q = vbeg[k]; q < vbeg[k + 1]; ++q) {
            const float *p = pts + 3 * order[q];
            double ex = (double)p[0] - (double)cen[3 * k + 0];
            double ey = (double)p[1] - (double)cen[3 * k + 1];
            double ez = (double)p[2] - (double)cen[3 * k + 2];
            double r = sqrt(ex * ex + ey * ey + ez * ez);
            if (r > rmax)
                rmax = r;
        }
        rmax *= 1.0 + ldexp(1.0, -48);
        if (radius_mode == 1) {
            double rp = sqrt(3.0) / 2.0 * (double)L;
            rad[k] = rp > rmax ? rp : rmax;
        } else {
            rad[k] = rmax;
        }
    }

    int64_t st[6] = {0, 0, 0, 0, 0, K};

    /* Sec. 3.3: initial update with s_0 = start, then Dist_v sync */
    const float *s = pts + 3 * start;
    for (int64_t i = 0; i < n; ++i) {
        float d = sq_dist(pts + 3 * i, s);
        D[i] = INFINITY;
        if (d < D[i])
            D[i] = d;
    }
    for (int64_t k = 0; k < K; ++k) {
        float bv = -1.0f;
        int64_t bi = -1;
        for (int64_t q = vbeg[k]; q < vbeg[k + 1]; ++q) {
            int64_t i = order[q];     /* members in increasing index */
            if (D[i] > bv) {
                bv = D[i];
                bi = i;
            }
        }
        dv[k] = bv;
        dv_idx[k] = bi;
    }
    out[0] = start;

    const double margin_lo = 1.0 - ldexp(1.0, -48);
    const double shrink = 1.0 - ldexp(1.0, -20);
    const double tiny = ldexp(1.0, -100);
    for (int64_t j = 1; j < m; ++j) {
        /* Sec. 3.4.1: two-level selection */
        int64_t kb = 0;
        for (int64_t k = 1; k < K; ++k)
            if (dv[k] > dv[kb] || (dv[k] == dv[kb] && dv_idx[k] < dv_idx[kb]))
                kb = k;
        float pv = -1.0f;
        int64_t sj = -1;
        for (int64_t q = vbeg[kb]; q < vbeg[kb + 1]; ++q) {
            int64_t i = order[q];
            if (D[i] > pv) {
                pv = D[i];
                sj = i;
            }
        }
        out[j] = sj;
        if (j == m - 1)
            break;   /* no later selection needs the last update */
        s = pts + 3 * sj;

        for (int64_t k = 0; k < K; ++k) {
            st[0]++;
            if (prune) {
                /* Sec. 3.4.2, Eq. spherical_voxel_bound and radius_pruning_condition */
                int pr = 0;
                if (dv[k] == 0.0f) {
                    pr = 1;
                } else {
                    double cx = (double)s[0] - (double)cen[3 * k + 0];
                    double cy = (double)s[1] - (double)cen[3 * k + 1];
                    double cz = (double)s[2] - (double)cen[3 * k + 2];
                    double dc = sqrt(cx * cx + cy * cy + cz * cz);
                    double lb = dc * margin_lo - rad[k] * (1.0 + ldexp(1.0, -48));
                    if (lb > 0.0) {
                        double lb2 = lb * lb;
                        if (lb2 >= tiny && lb2 * shrink >= (double)dv[k])
                            pr = 1;
                    }
                }
                if (pr) {
                    st[1]++;
                    continue;
                }
            }
            /* Sec. 3.4.3: point skip and exact update */
            for (int64_t q = vbeg[k]; q < vbeg[k + 1]; ++q) {
                int64_t i = order[q];
                const float *p = pts + 3 * i;
                st[2]++;
                float dx = p[0] - s[0];
                float dy = p[1] - s[1];
                float dz = p[2] - s[2];
                float xx = dx * dx, yy = dy * dy, zz = dz * dz;
                if (skip && (xx >= D[i] || yy >= D[i] || zz >= D[i])) {
                    st[3]++;
                    continue;
                }
                float sum = xx + yy;
                float d = sum + zz;
                if (d < D[i]) {
                    D[i] = d;
                    st[4]++;
                }
            }
            /* Eq. point_skip_distv_sync */
            float bv = -1.0f;
            int64_t bi = -1;
            for (int64_t q = vbeg[k]; q < vbeg[k + 1]; ++q) {
                int64_t i = order[q];
                if (D[i] > bv) {
                    bv = D[i];
                    bi = i;
                }
            }
            dv[k] = bv;
            dv_idx[k] = bi;
        }
    }
    if (stats != NULL)
        memcpy(stats, st, sizeof(st));
    free(vid); free(order); free(vbeg); free(cen); free(rad); free(dv); free(dv_idx); free(D);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * FP64 FPS in the paper's Euclidean (square-root) domain, Alg. 1 with
 * D[i] = min(D[i], |p_i - s|_2) evaluated in double.  Information only: it
 * measures how often the FP32 squared-distance reading picks a different
 * index from the real-number reading; it is never a parity gate.
 * ---------------------------------------------------------------------- */
int oracle_fps_f64(const float *pts, int64_t n, int64_t m, int64_t start,
                   int64_t *out, double *cover_out)
{
    int rc = check_args(pts, n, m, start);
    if (rc != ORACLE_OK || out == NULL)
        return rc != ORACLE_OK ? rc : ORACLE_EINVAL;
    double *D = (double *)malloc((size_t)n * sizeof(double));
    if (D == NULL)
        return ORACLE_ENOMEM;
    for (int64_t i = 0; i < n; ++i)
        D[i] = INFINITY;
    out[0] = start;
    if (cover_out != NULL)
        cover_out[0] = INFINITY;
    int64_t s = start;
    for (int64_t j = 1; j < m; ++j) {
        const float *ps = pts + 3 * s;
        double bv = -1.0;
        int64_t bi = -1;
        for (int64_t i = 0; i < n; ++i) {
            const float *p = pts + 3 * i;
            double dx = (double)p[0] - (double)ps[0];
            double dy = (double)p[1] - (double)ps[1];
            double dz = (double)p[2] - (double)ps[2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d < D[i])
                D[i] = d;
            if (D[i] > bv) {
                bv = D[i];
                bi = i;
            }
        }
        s = bi;
        out[j] = s;
        if (cover_out != NULL)
            cover_out[j] = bv;
    }
    free(D);
    return ORACLE_OK;
}

int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
