/*
 * A plain C99 program that drives libphd.so through its C ABI alone (no
 * Python, no PyTorch; device memory from the CUDA runtime): a 4-PE DCPFPHD
 * filter (Algorithm 1) tracks two targets moving on straight lines, seen by a
 * linear position sensor with detection probability 0.95 and clutter, for 40
 * scans through phd_step (device buffers), then 5 more through
 * phd_step_host (pageable host buffers).  It prints the counters and one
 * "tracked" line, and exits 0 when every call succeeded and, from scan 15 on,
 * each target had an estimate within 30 m in at least 80 % of the scans.
 *
 * Built and run by tests/test_gpu_c_abi.py; compiled (not run) by the CPU
 * tests.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "phd.h"

static unsigned long long rng_state = 0x9E3779B97F4A7C15ull;

static double urand(void) {
    rng_state = rng_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(rng_state >> 11) * (1.0 / 9007199254740992.0);
}

static double nrand(void) {
    double u1 = urand(), u2 = urand();
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

#define CHECK(call)                                                                     \
    do {                                                                                \
        phd_status s_ = (call);                                                         \
        if (s_ != PHD_OK) {                                                             \
            fprintf(stderr, "%s: %s (%s)\n", #call, phd_status_string(s_),              \
                    h ? phd_last_error_string(h) : "");                                 \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

#define CUDA(call)                                                                      \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                 \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

enum { SCANS = 40, HOST_SCANS = 5, M_MAX = 128, CLUTTER = 10 };

/* Scan k: detections of the live targets (p_D = 0.95) and CLUTTER uniform
 * points over the region, shuffled; returns M. */
static int make_scan(double truth[2][4], float *Z) {
    int M = 0;
    for (int t = 0; t < 2; ++t)
        if (urand() < 0.95) {
            Z[2 * M] = (float)(truth[t][0] + 10.0 * nrand());
            Z[2 * M + 1] = (float)(truth[t][2] + 10.0 * nrand());
            ++M;
        }
    for (int c = 0; c < CLUTTER; ++c) {
        Z[2 * M] = (float)(-1000.0 + 2000.0 * urand());
        Z[2 * M + 1] = (float)(-1000.0 + 2000.0 * urand());
        ++M;
    }
    for (int i = M - 1; i > 0; --i) {
        int j = (int)(urand() * (i + 1));
        float a = Z[2 * i], b = Z[2 * i + 1];
        Z[2 * i] = Z[2 * j];
        Z[2 * i + 1] = Z[2 * j + 1];
        Z[2 * j] = a;
        Z[2 * j + 1] = b;
    }
    return M;
}

static void move(double truth[2][4]) {
    for (int t = 0; t < 2; ++t) {
        truth[t][0] += truth[t][1];
        truth[t][2] += truth[t][3];
    }
}

/* Whether estimate rows (x, vx, y, vy) hold one within 30 m of each target. */
static int near(double truth[2][4], const float *S, int n, int t) {
    for (int i = 0; i < n; ++i) {
        double dx = S[4 * i] - truth[t][0], dy = S[4 * i + 2] - truth[t][2];
        if (dx * dx + dy * dy < 900.0) return 1;
    }
    return 0;
}

int main(void) {
    phd_handle *h = NULL;
    phd_config c;
    memset(&c, 0, sizeof c);
    c.meas_model = PHD_MEAS_LINEAR;
    c.precision = PHD_FP32;
    c.num_pe = 4;
    c.ck_mode = PHD_CK_LOCAL;
    c.pe_cap = 2048;
    c.m_max = M_MAX;
    c.birth_count = 800;
    c.dt = 1.0;
    c.sigma_a = 2.0;
    c.sigma_z[0] = c.sigma_z[1] = 10.0;
    c.region[0] = -1000.0;
    c.region[1] = 1000.0;
    c.region[2] = -1000.0;
    c.region[3] = 1000.0;
    c.r_max = 1414.0;
    c.p_s = 0.99;
    c.p_d = 0.95;
    c.clutter_rate = CLUTTER;
    c.birth_mass = 0.2;
    c.birth_vel_sigma = 20.0;
    c.particles_per_target = 1000.0;
    c.exchange_frac = 0.1;
    c.seed = 7;

    size_t bytes = 0;
    CHECK(phd_workspace_size(&c, &bytes));
    void *ws = NULL;
    CUDA(cudaMalloc(&ws, bytes));
    CHECK(phd_init(&h, &c, ws, bytes, NULL));

    float *dZ = NULL, *dS = NULL;
    int32_t *dL = NULL, *dN = NULL;
    CUDA(cudaMalloc((void **)&dZ, sizeof(float) * 2 * M_MAX));
    CUDA(cudaMalloc((void **)&dS, sizeof(float) * 4 * M_MAX));
    CUDA(cudaMalloc((void **)&dL, sizeof(int32_t) * M_MAX));
    CUDA(cudaMalloc((void **)&dN, sizeof(int32_t)));
    float Z[2 * M_MAX], S[4 * M_MAX];
    int32_t L[M_MAX];

    double truth[2][4] = {{-300.0, 10.0, 200.0, -5.0}, {400.0, -8.0, -100.0, 12.0}};
    int hits[2] = {0, 0}, scored = 0;
    for (int k = 0; k < SCANS + HOST_SCANS; ++k) {
        move(truth);
        const int M = make_scan(truth, Z);
        int32_t n = 0;
        if (k < SCANS) {
            CUDA(cudaMemcpy(dZ, Z, sizeof(float) * 2 * M, cudaMemcpyHostToDevice));
            CHECK(phd_step(h, dZ, M, dS, dL, M_MAX, dN, &n));
            CUDA(cudaMemcpy(S, dS, sizeof(float) * 4 * (size_t)n, cudaMemcpyDeviceToHost));
        } else {
            CHECK(phd_step_host(h, Z, M, S, L, M_MAX, &n));
        }
        if (k >= 15) {
            ++scored;
            for (int t = 0; t < 2; ++t) hits[t] += near(truth, S, n, t);
        }
        if (k % 10 == 9) printf("scan %d: %d measurements, %d estimates\n", k + 1, M, (int)n);
    }
    phd_stats st;
    CHECK(phd_get_stats(h, &st));
    int32_t path = 0;
    CHECK(phd_get_path(h, &path));
    printf("updates %llu, pairs %llu, launches %llu, path %s\n", (unsigned long long)st.updates,
           (unsigned long long)st.pairs, (unsigned long long)st.launches,
           path == PHD_PATH_FUSED ? "fused" : "staged");
    CHECK(phd_destroy(h));
    h = NULL;
    CUDA(cudaFree(dZ));
    CUDA(cudaFree(dS));
    CUDA(cudaFree(dL));
    CUDA(cudaFree(dN));
    CUDA(cudaFree(ws));
    const int ok = hits[0] * 10 >= scored * 8 && hits[1] * 10 >= scored * 8;
    printf("tracked %d/%d and %d/%d scans: %s\n", hits[0], scored, hits[1], scored, ok ? "ok" : "FAIL");
    return ok ? 0 : 2;
}
