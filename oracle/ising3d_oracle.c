/*
 * ising3d_oracle.c -- plain CPU oracle for the checkerboard Metropolis sweep of
 * the three-dimensional Ising model (simple cubic, periodic L x L x L, J = 1,
 * h = 0, six nearest neighbours).
 *
 * TEST INFRASTRUCTURE ONLY (like ising_oracle.c, whose Philox4x32-10 it
 * calls): nothing in the product library links, loads or calls this file.
 *
 * The paper's Hamiltonian (Section 1) is written for any dimension, with the
 * number of neighbours set by the lattice (four in 2D, six in 3D).  The same
 * rule as in 2D: a site flips iff dE <= 0 or r < thr[dE], with
 * thr = min(floor(2^32 exp(-dE/T)), 2^32 - 1) for dE in {4, 8, 12}; sites of
 * colour (x + y + z) & 1 == 0 ("black") are updated first, then colour 1.
 * Draws (this project's definitions): Philox4x32-10, key (lo32, hi32 of the
 * seed), counter (p >> 2, t, s, phase), lane p & 3, p = the site's rank among
 * the same-colour sites in (z, y, x) row-major order, p = (z L + y) (L/2) +
 * (x >> 1); phase 0/1 for the half-sweeps; the random initial state draws
 * phase 2 with p = (z L + y) L + x and sets +1 iff the top bit is 0.
 * sigma[(z L + y) L + x] in {+1, -1}.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

uint32_t oracle_site_random(uint64_t seed, uint32_t p, uint32_t t, uint32_t s, uint32_t phase);

static inline int wrap3(int i, int L) { return ((i % L) + L) % L; }
static inline size_t at3(int L, int x, int y, int z)
{
    return ((size_t)wrap3(z, L) * L + (size_t)wrap3(y, L)) * L + (size_t)wrap3(x, L);
}

/* thr[k] for dE = 4 (k + 1), k = 0, 1, 2; -1 for a T that is not positive
 * and finite. */
int oracle3d_thresholds(double T, uint32_t thr[3])
{
    if (!(T > 0.0) || !isfinite(T)) return -1;
    for (int k = 0; k < 3; ++k) {
        double v = ldexp(exp(-4.0 * (double)(k + 1) / T), 32);
        thr[k] = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)floor(v);
    }
    return 0;
}

int oracle3d_init(int L, uint64_t seed, uint32_t s, int mode, int8_t* sigma)
{
    if (L < 2 || (L & 1)) return -1;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int8_t v = 1;
                if (mode == 0) {
                    uint32_t p = ((uint32_t)z * (uint32_t)L + (uint32_t)y) * (uint32_t)L + (uint32_t)x;
                    v = (oracle_site_random(seed, p, 0u, s, 2u) >> 31) ? (int8_t)-1 : (int8_t)1;
                }
                sigma[at3(L, x, y, z)] = v;
            }
    return 0;
}

/* H = -sum over every site of sigma (right + down + back neighbour): each
 * bond once. */
int64_t oracle3d_energy(int L, const int8_t* sigma)
{
    int64_t e = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int s0 = sigma[at3(L, x, y, z)];
                int n = sigma[at3(L, x + 1, y, z)] + sigma[at3(L, x, y + 1, z)] + sigma[at3(L, x, y, z + 1)];
                e -= (int64_t)(s0 * n);
            }
    return e;
}

int64_t oracle3d_magnetization(int L, const int8_t* sigma)
{
    int64_t m = 0;
    for (size_t i = 0; i < (size_t)L * L * L; ++i) m += sigma[i];
    return m;
}

static void half_sweep3(int L, int8_t* sigma, int c, const uint32_t thr[3], uint64_t seed, uint32_t s,
                        uint32_t t)
{
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + z) & 1) != c) continue;
                size_t i = at3(L, x, y, z);
                int h = sigma[at3(L, x - 1, y, z)] + sigma[at3(L, x + 1, y, z)] + sigma[at3(L, x, y - 1, z)] +
                        sigma[at3(L, x, y + 1, z)] + sigma[at3(L, x, y, z - 1)] + sigma[at3(L, x, y, z + 1)];
                int dE = 2 * sigma[i] * h;
                int flip;
                if (dE <= 0) {
                    flip = 1;
                } else {
                    uint32_t p = ((uint32_t)z * (uint32_t)L + (uint32_t)y) * (uint32_t)(L / 2) + (uint32_t)(x >> 1);
                    flip = oracle_site_random(seed, p, t, s, (uint32_t)c) < thr[dE / 4 - 1];
                }
                if (flip) sigma[i] = (int8_t)(-sigma[i]);
            }
}

/* n sweeps with indices t0 .. t0+n-1; E, M after each (either may be NULL). */
void oracle3d_sweeps(int L, int8_t* sigma, const uint32_t thr[3], uint64_t seed, uint32_t s, uint32_t t0,
                     int64_t n, int64_t* E, int64_t* M)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t t = t0 + (uint32_t)i;
        half_sweep3(L, sigma, 0, thr, seed, s, t);
        half_sweep3(L, sigma, 1, thr, seed, s, t);
        if (E) E[i] = oracle3d_energy(L, sigma);
        if (M) M[i] = oracle3d_magnetization(L, sigma);
    }
}

/* Many lattices, one OpenMP thread per lattice at a time; lattice j uses
 * thrs[3j..3j+2], seeds[j], sims[j]; traces [n_lat][n]. */
void oracle3d_sweeps_batch(int n_lat, const int* Ls, int8_t* const* sigmas, const uint32_t* thrs,
                           const uint64_t* seeds, const uint32_t* sims, uint32_t t0, int64_t n, int64_t* E,
                           int64_t* M, int n_threads)
{
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) if (n_threads > 1)
#endif
    for (int j = 0; j < n_lat; ++j)
        oracle3d_sweeps(Ls[j], sigmas[j], thrs + 3 * j, seeds[j], sims[j], t0, n,
                        E ? E + (size_t)j * n : NULL, M ? M + (size_t)j * n : NULL);
    (void)n_threads;
}
