/*
 * rsa.c -- seeded input generator: random sequential addition of N hard-sphere
 * centres, uniform in a ball, none closer than sigma (the initial state of the
 * paper's production runs is ions placed uniformly with hard-core rejection,
 * Sec. 5.2).  This file holds no Monte Carlo arithmetic; it only produces
 * starting configurations that both the oracle and the CUDA path consume.
 *
 * Validity uses the same definitions the simulation checks: the FP32 centre p
 * satisfies ((double)p_x^2 + (double)p_y^2) + (double)p_z^2 <= Rc^2 and every
 * pair has FP64 squared distance >= sigma^2, both formed from the FP32 values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unif(uint64_t *s)
{
    return (double)(splitmix64(s) >> 11) * 0x1p-53;
}

/* Returns the number of centres placed (== n on success). */
int64_t rsa_place(int64_t n, double sigma, double Rc, uint64_t seed, int64_t max_attempts, float *out)
{
    if (n <= 0) return 0;
    double sig2 = sigma * sigma, Rc2 = Rc * Rc;
    double cell = sigma;
    int64_t m = (int64_t)floor(2.0 * Rc / cell);
    if (m < 1) m = 1;
    if (m > 1024) m = 1024;
    cell = 2.0 * Rc / (double)m;
    if (cell < sigma) {
        m = (int64_t)floor(2.0 * Rc / sigma);
        if (m < 1) m = 1;
        cell = 2.0 * Rc / (double)m;
    }
    int64_t ncell = m * m * m;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!head || !next) {
        free(head);
        free(next);
        return -1;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    uint64_t st = seed ^ 0x5A17F00Dull;
    int64_t placed = 0;
    for (int64_t att = 0; placed < n && att < max_attempts; ++att) {
        float p[3];
        for (int k = 0; k < 3; ++k) p[k] = (float)((2.0 * unif(&st) - 1.0) * Rc);
        double r2 = ((double)p[0] * (double)p[0] + (double)p[1] * (double)p[1]) + (double)p[2] * (double)p[2];
        if (!(r2 <= Rc2)) continue;
        int64_t ci[3];
        for (int k = 0; k < 3; ++k) {
            int64_t v = (int64_t)floor(((double)p[k] + Rc) / cell);
            ci[k] = v < 0 ? 0 : (v >= m ? m - 1 : v);
        }
        int ok = 1;
        for (int64_t dx = -1; dx <= 1 && ok; ++dx)
            for (int64_t dy = -1; dy <= 1 && ok; ++dy)
                for (int64_t dz = -1; dz <= 1 && ok; ++dz) {
                    int64_t cx = ci[0] + dx, cy = ci[1] + dy, cz = ci[2] + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= m || cy >= m || cz >= m) continue;
                    for (int64_t j = head[(cx * m + cy) * m + cz]; j >= 0; j = next[j]) {
                        double d0 = (double)p[0] - (double)out[3 * j];
                        double d1 = (double)p[1] - (double)out[3 * j + 1];
                        double d2 = (double)p[2] - (double)out[3 * j + 2];
                        if ((d0 * d0 + d1 * d1) + d2 * d2 < sig2) {
                            ok = 0;
                            break;
                        }
                    }
                }
        if (!ok) continue;
        out[3 * placed] = p[0];
        out[3 * placed + 1] = p[1];
        out[3 * placed + 2] = p[2];
        int64_t c = (ci[0] * m + ci[1]) * m + ci[2];
        next[placed] = head[c];
        head[c] = placed;
        placed++;
    }
    free(head);
    free(next);
    return placed;
}
