/* sanitize_main.c -- TEST INFRASTRUCTURE: a standalone driver that runs the
 * oracle's entry points over small and degenerate clouds, built together
 * with rfps_oracle.c under AddressSanitizer and UndefinedBehaviorSanitizer
 * by tests/test_oracle_sanitizers.py.  It checks that every call returns,
 * that every RadiusFPS switch combination reproduces plain FPS exactly
 * (Sec. 3: pruning and skipping never change the result), and that invalid
 * arguments are rejected with the documented codes.  Exit status 0 when
 * everything held; the sanitizers abort the run on any memory or UB error.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_fps(const float *pts, int64_t n, int64_t m, int64_t start, int64_t *out, float *d2_out, int threads);
int oracle_voxelize(const float *pts, int64_t n, int n_vox, float *grid_out, uint32_t *vid_out);
int oracle_radiusfps(const float *pts, int64_t n, int64_t m, int64_t start, int n_vox, int prune, int skip,
                     int radius_mode, int64_t *out, int64_t *stats);
int oracle_fps_f64(const float *pts, int64_t n, int64_t m, int64_t start, int64_t *out, double *cover_out);

static uint64_t g_state = 0x9e3779b97f4a7c15ull;
static float unit(void)   /* xorshift64*: a seeded stream for the test clouds only */
{
    g_state ^= g_state >> 12;
    g_state ^= g_state << 25;
    g_state ^= g_state >> 27;
    return (float)((g_state * 0x2545f4914f6cdd1dull) >> 40) / 16777216.0f;
}

static int g_fail = 0;
#define CHECK(cond, ...)                      \
    do {                                      \
        if (!(cond)) {                        \
            fprintf(stderr, __VA_ARGS__);     \
            fputc('\n', stderr);              \
            ++g_fail;                         \
        }                                     \
    } while (0)

static void run_cloud(const char *name, const float *p, int64_t n)
{
    const int64_t ms[3] = {1, n > 1 ? n / 2 : 1, n};
    int64_t *ref = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *got = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    float *d2 = (float *)malloc((size_t)n * sizeof(float));
    uint32_t *vid = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    double *cover = (double *)malloc((size_t)n * sizeof(double));
    for (int k = 0; k < 3; ++k) {
        const int64_t m = ms[k], start = (n - 1) / 3;
        CHECK(oracle_fps(p, n, m, start, ref, d2, 1) == 0, "%s: oracle_fps serial failed", name);
        CHECK(oracle_fps(p, n, m, start, got, NULL, 0) == 0, "%s: oracle_fps threaded failed", name);
        CHECK(memcmp(ref, got, (size_t)m * sizeof(int64_t)) == 0, "%s m=%lld: thread count changed the result",
              name, (long long)m);
        const int nvs[3] = {1, 3, 17};
        for (int v = 0; v < 3; ++v)
            for (int sw = 0; sw < 8; ++sw) {
                int64_t stats[6];
                const int rc = oracle_radiusfps(p, n, m, start, nvs[v], sw & 1, (sw >> 1) & 1, (sw >> 2) & 1, got,
                                                stats);
                CHECK(rc == 0, "%s: oracle_radiusfps rc %d", name, rc);
                CHECK(memcmp(ref, got, (size_t)m * sizeof(int64_t)) == 0,
                      "%s m=%lld n_vox=%d switches=%d: RadiusFPS differs from FPS", name, (long long)m, nvs[v], sw);
            }
        CHECK(oracle_fps_f64(p, n, m, start, got, cover) == 0, "%s: oracle_fps_f64 failed", name);
    }
    float grid[7];
    CHECK(oracle_voxelize(p, n, 9, grid, vid) == 0, "%s: oracle_voxelize failed", name);
    for (int64_t i = 0; i < n; ++i)
        CHECK(vid[i] < 9u * 9u * 9u, "%s: voxel id out of range", name);
    free(ref);
    free(got);
    free(d2);
    free(vid);
    free(cover);
}

int main(void)
{
    enum { N = 300 };
    float *p = (float *)malloc(3 * N * sizeof(float));
    /* uniform */
    for (int i = 0; i < 3 * N; ++i) p[i] = unit();
    run_cloud("uniform", p, N);
    /* duplicates: 20 distinct points repeated */
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) p[3 * i + a] = (float)((i % 20) * 7 % 13) * 0.25f + (float)a;
    run_cloud("duplicates", p, N);
    /* lattice (exact ties) */
    for (int i = 0; i < N; ++i) {
        p[3 * i + 0] = (float)(i % 7);
        p[3 * i + 1] = (float)((i / 7) % 7);
        p[3 * i + 2] = (float)(i / 49);
    }
    run_cloud("lattice", p, N);
    /* extreme scales and a flat cloud */
    for (int i = 0; i < 3 * N; ++i) p[i] = unit() * 1e18f;
    run_cloud("wide", p, N);
    for (int i = 0; i < 3 * N; ++i) p[i] = unit() * 1e-18f;
    run_cloud("tiny", p, N);
    for (int i = 0; i < N; ++i) p[3 * i + 2] = 0.5f;
    run_cloud("flat", p, N);
    /* one and two points */
    run_cloud("single", p, 1);
    run_cloud("pair", p, 2);
    /* invalid arguments */
    int64_t out[4];
    CHECK(oracle_fps(p, 0, 1, 0, out, NULL, 1) != 0, "n = 0 accepted");
    CHECK(oracle_fps(p, 3, 4, 0, out, NULL, 1) != 0, "m > n accepted");
    CHECK(oracle_fps(p, 3, 2, 3, out, NULL, 1) != 0, "start out of range accepted");
    CHECK(oracle_radiusfps(p, 3, 2, 0, 0, 1, 1, 0, out, NULL) != 0, "n_vox = 0 accepted");
    p[4] = NAN;
    CHECK(oracle_fps(p, 3, 2, 0, out, NULL, 1) != 0, "non-finite coordinate accepted");
    free(p);
    if (g_fail) fprintf(stderr, "%d check(s) failed\n", g_fail);
    else printf("oracle sanitizer run: all checks held\n");
    return g_fail ? 1 : 0;
}
