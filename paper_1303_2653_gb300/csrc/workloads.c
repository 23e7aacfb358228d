/*
 * Seeded synthetic inputs for fluidised-bed workloads.
 *
 * This file holds no arithmetic of the simulation method: it only draws random
 * numbers and places non-overlapping discs/spheres.  Both the CPU oracle tests
 * and the GPU library consume its output (SI positions and velocities), each
 * converting to lattice units on its own.
 *
 *  - splitmix64 stream (Steele, Lea and Flood, "Fast splittable pseudorandom
 *    number generators", OOPSLA 2014): 64-bit counter advanced by the golden
 *    gamma, then a two-round xor-shift-multiply finaliser.
 *  - uniform doubles from the top 53 bits.
 *  - normal deviates by the Box-Muller transform.
 *  - random sequential addition (RSA): candidates drawn uniformly in a box are
 *    accepted when no already-placed centre lies closer than the minimum
 *    separation (minimum image across periodic axes); a uniform cell grid of
 *    spacing >= separation makes each test O(1).
 *
 * Units are whatever the caller passes (the Python front end passes metres).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double sm64_uniform(uint64_t *state)
{
    return (double)(sm64_next(state) >> 11) * 0x1.0p-53;
}

/* n uniform doubles in [0,1): exported so tests can check the stream. */
void wl_uniform(uint64_t seed, int64_t n, double *out)
{
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = sm64_uniform(&s);
}

/*
 * Maxwellian velocities: each of dim components ~ N(mean[a], sigma^2).
 * Box-Muller on pairs of uniforms; u1 is mapped to (0,1] so log() is finite.
 */
void wl_maxwellian(int dim, int64_t n, const double *mean, double sigma,
                   uint64_t seed, double *vel)
{
    uint64_t s = seed;
    const double two_pi = 6.283185307179586476925286766559;
    int64_t total = n * dim;
    for (int64_t k = 0; k < total; k += 2) {
        double u1 = 1.0 - sm64_uniform(&s);
        double u2 = sm64_uniform(&s);
        double rad = sqrt(-2.0 * log(u1));
        double z0 = rad * cos(two_pi * u2);
        double z1 = rad * sin(two_pi * u2);
        vel[k] = mean[k % dim] + sigma * z0;
        if (k + 1 < total) vel[k + 1] = mean[(k + 1) % dim] + sigma * z1;
    }
}

/*
 * Random sequential addition of n centres.
 *   dim        2 or 3
 *   box[a]     periodic length of axis a (used for the grid and minimum image)
 *   lo[a],hi[a] sampling interval of axis a (subset of [0, box[a]])
 *   periodic[a] nonzero: distances wrap with period box[a]
 *   sep        minimum centre distance (accepted pairs have dist >= sep)
 * Returns the number placed (== n on success, less if max_attempts ran out).
 */
int64_t wl_rsa(int dim, const double *box, const double *lo, const double *hi,
               const int *periodic, double sep, int64_t n, uint64_t seed,
               int64_t max_attempts, double *pos)
{
    int64_t ng[3] = {1, 1, 1};
    double gs[3] = {1.0, 1.0, 1.0};
    for (int a = 0; a < dim; ++a) {
        int64_t m = (int64_t)floor(box[a] / sep);
        if (m < 1) m = 1;
        if (m > 4096) m = 4096;
        ng[a] = m;
        gs[a] = box[a] / (double)m;
    }
    int64_t ncell = ng[0] * ng[1] * ng[2];
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!head || !next) { free(head); free(next); return -1; }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;

    uint64_t s = seed;
    const double sep2 = sep * sep;
    int64_t placed = 0, attempts = 0;
    while (placed < n && attempts < max_attempts) {
        ++attempts;
        double p[3] = {0.0, 0.0, 0.0};
        int64_t g[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            p[a] = lo[a] + (hi[a] - lo[a]) * sm64_uniform(&s);
            int64_t gi = (int64_t)floor(p[a] / gs[a]);
            if (gi < 0) gi = 0;
            if (gi >= ng[a]) gi = ng[a] - 1;
            g[a] = gi;
        }
        /* distinct neighbour grid indices per axis (wrapped when periodic) */
        int64_t nb[3][3];
        int nnb[3] = {1, 1, 1};
        for (int a = 0; a < 3; ++a) nb[a][0] = g[a];
        for (int a = 0; a < dim; ++a) {
            nnb[a] = 0;
            for (int off = -1; off <= 1; ++off) {
                int64_t q = g[a] + off;
                if (q < 0 || q >= ng[a]) {
                    if (!periodic[a]) continue;
                    q = (q + ng[a]) % ng[a];
                }
                int dup = 0;
                for (int t = 0; t < nnb[a]; ++t) if (nb[a][t] == q) dup = 1;
                if (!dup) nb[a][nnb[a]++] = q;
            }
        }
        int ok = 1;
        for (int iz = 0; iz < nnb[2] && ok; ++iz)
        for (int iy = 0; iy < nnb[1] && ok; ++iy)
        for (int ix = 0; ix < nnb[0] && ok; ++ix) {
            int64_t c = nb[0][ix] + ng[0] * (nb[1][iy] + ng[1] * nb[2][iz]);
            for (int32_t j = head[c]; j >= 0; j = next[j]) {
                double d2 = 0.0;
                for (int a = 0; a < dim; ++a) {
                    double dd = p[a] - pos[(int64_t)j * dim + a];
                    if (periodic[a]) {
                        if (dd > 0.5 * box[a]) dd -= box[a];
                        else if (dd < -0.5 * box[a]) dd += box[a];
                    }
                    d2 += dd * dd;
                }
                if (d2 < sep2) { ok = 0; break; }
            }
        }
        if (!ok) continue;
        for (int a = 0; a < dim; ++a) pos[placed * dim + a] = p[a];
        int64_t c = g[0] + ng[0] * (g[1] + ng[1] * g[2]);
        next[placed] = head[c];
        head[c] = (int32_t)placed;
        ++placed;
    }
    free(head);
    free(next);
    return placed;
}
