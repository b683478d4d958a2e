/*
 * cluster_oracle.c -- plain CPU oracle for the Swendsen-Wang cluster update.
 *
 * TEST INFRASTRUCTURE ONLY (like ising_oracle.c, whose Philox4x32-10 and
 * energy / magnetization it calls): nothing in the product library links,
 * loads or calls this file.  It shares no code with the CUDA path.
 *
 * The paper names cluster algorithms (Swendsen-Wang, Wolff) as the cure for
 * the critical slowing down of single-site Metropolis (Section 1).  This file
 * writes out the Swendsen-Wang step (Swendsen and Wang, PRL 58, 86, 1987) for
 * J = 1, h = 0 on the periodic L x L lattice:
 *   1. every nearest-neighbour pair of equal spins is joined by an active
 *      bond with probability p = 1 - exp(-2 J / T), independently;
 *   2. clusters are the connected components of the active bonds;
 *   3. every cluster is flipped with probability 1/2, independently.
 *
 * Draws (this project's definitions; Philox4x32-10 keyed by the lattice seed,
 * counter (q, t, s, phase), t = the step's index in the handle's sweep
 * counter, s = simulation index):
 *   - bonds, phase 7: site p = y*L + x owns the bonds to its right and down
 *     neighbours; q = p >> 1, lane 2*(p & 1) is the right bond's draw and
 *     lane 2*(p & 1) + 1 the down bond's; a bond between equal spins is
 *     active iff its draw r < thr, thr = min(floor(2^32 p), 2^32 - 1);
 *   - cluster coin, phase 8: a cluster is named by its smallest site index
 *     r0 (its root); it flips iff the top bit of lane r0 & 3 of block
 *     q = r0 >> 2 is 1.
 * Both sides compute the same clusters (a partition is unique) and the same
 * root (the minimum), so the result of a step is a single defined lattice.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t oracle_site_random(uint64_t seed, uint32_t p, uint32_t t, uint32_t s, uint32_t phase);
int64_t oracle_energy(int L, const int8_t* sigma);
int64_t oracle_magnetization(int L, const int8_t* sigma);

#define ORC_SW_PHASE_BOND 7u
#define ORC_SW_PHASE_COIN 8u
#define ORC_SW_NO_LABEL 0xFFFFFFFFu

/* Bond threshold at temperature T: floor(2^32 (1 - exp(-2/T))), at most
 * 2^32 - 1.  expm1 keeps the small-p end exact to double rounding.  Returns
 * 0 and leaves *thr alone for T that is not positive and finite. */
int oracle_sw_threshold(double T, uint32_t* thr)
{
    if (!(T > 0.0) || !isfinite(T)) return -1;
    double p = -expm1(-2.0 / T);
    double v = ldexp(p, 32);
    *thr = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)floor(v);
    return 0;
}

/* Active bonds of one step: bonds[p] bit 0 = bond (x, y)-(x+1, y), bit 1 =
 * bond (x, y)-(x, y+1), indices mod L. */
void oracle_sw_bonds(int L, const int8_t* sigma, uint64_t seed, uint32_t t, uint32_t s,
                     uint32_t thr, uint8_t* bonds)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            uint32_t p = (uint32_t)y * (uint32_t)L + (uint32_t)x;
            uint32_t ctr[4] = { p >> 1, t, s, ORC_SW_PHASE_BOND };
            uint32_t out[4];
            oracle_philox4x32_10(ctr, key, out);
            uint32_t r_right = out[2u * (p & 1u)];
            uint32_t r_down = out[2u * (p & 1u) + 1u];
            int8_t me = sigma[p];
            int8_t right = sigma[(size_t)y * L + (x + 1) % L];
            int8_t down = sigma[(size_t)((y + 1) % L) * L + x];
            uint8_t b = 0;
            if (me == right && r_right < thr) b |= 1u;
            if (me == down && r_down < thr) b |= 2u;
            bonds[p] = b;
        }
}

/* Cluster labels: label[p] = the smallest site index of p's cluster.  Sites
 * are visited in increasing index; an unlabelled site starts a breadth-first
 * search, so it is the smallest index of the cluster it labels.  Returns the
 * number of clusters, or -1 if the queue cannot be allocated. */
int64_t oracle_sw_labels(int L, const uint8_t* bonds, uint32_t* label)
{
    size_t N = (size_t)L * L;
    uint32_t* queue = (uint32_t*)malloc(N * sizeof(uint32_t));
    if (!queue) return -1;
    for (size_t i = 0; i < N; ++i) label[i] = ORC_SW_NO_LABEL;
    int64_t clusters = 0;
    for (size_t start = 0; start < N; ++start) {
        if (label[start] != ORC_SW_NO_LABEL) continue;
        ++clusters;
        size_t head = 0, tail = 0;
        label[start] = (uint32_t)start;
        queue[tail++] = (uint32_t)start;
        while (head < tail) {
            uint32_t u = queue[head++];
            int x = (int)(u % (uint32_t)L), y = (int)(u / (uint32_t)L);
            uint32_t right = (uint32_t)y * L + (uint32_t)((x + 1) % L);
            uint32_t left = (uint32_t)y * L + (uint32_t)((x + L - 1) % L);
            uint32_t down = (uint32_t)((y + 1) % L) * L + (uint32_t)x;
            uint32_t up = (uint32_t)((y + L - 1) % L) * L + (uint32_t)x;
            uint32_t nb[4];
            int k = 0;
            if (bonds[u] & 1u) nb[k++] = right;
            if (bonds[left] & 1u) nb[k++] = left;
            if (bonds[u] & 2u) nb[k++] = down;
            if (bonds[up] & 2u) nb[k++] = up;
            for (int i = 0; i < k; ++i)
                if (label[nb[i]] == ORC_SW_NO_LABEL) {
                    label[nb[i]] = (uint32_t)start;
                    queue[tail++] = nb[i];
                }
        }
    }
    free(queue);
    return clusters;
}

/* One Swendsen-Wang step with index t.  bonds / label are caller scratch of
 * L*L entries (left holding this step's bonds and labels). */
int oracle_sw_step(int L, int8_t* sigma, uint32_t thr, uint64_t seed, uint32_t s, uint32_t t,
                   uint8_t* bonds, uint32_t* label)
{
    size_t N = (size_t)L * L;
    oracle_sw_bonds(L, sigma, seed, t, s, thr, bonds);
    if (oracle_sw_labels(L, bonds, label) < 0) return -1;
    for (size_t p = 0; p < N; ++p) {
        uint32_t root = label[p];
        uint32_t coin = oracle_site_random(seed, root, t, s, ORC_SW_PHASE_COIN) >> 31;
        if (coin) sigma[p] = (int8_t)(-sigma[p]);
    }
    return 0;
}

/* n steps with indices t0 .. t0+n-1; E and M after each step (either may be
 * NULL). */
int oracle_sw_sweeps(int L, int8_t* sigma, uint32_t thr, uint64_t seed, uint32_t s, uint32_t t0,
                     int64_t n, int64_t* E, int64_t* M)
{
    size_t N = (size_t)L * L;
    uint8_t* bonds = (uint8_t*)malloc(N);
    uint32_t* label = (uint32_t*)malloc(N * sizeof(uint32_t));
    int rc = 0;
    if (!bonds || !label) rc = -1;
    for (int64_t i = 0; i < n && rc == 0; ++i) {
        rc = oracle_sw_step(L, sigma, thr, seed, s, t0 + (uint32_t)i, bonds, label);
        if (E) E[i] = oracle_energy(L, sigma);
        if (M) M[i] = oracle_magnetization(L, sigma);
    }
    free(bonds);
    free(label);
    return rc;
}

/* Many independent lattices, one OpenMP thread per lattice at a time; lattice
 * j uses thrs[j], seeds[j], sims[j]; traces are [n_lat][n].  Returns the
 * number of lattices that failed (allocation). */
int oracle_sw_sweeps_batch(int n_lat, const int* Ls, int8_t* const* sigmas, const uint32_t* thrs,
                           const uint64_t* seeds, const uint32_t* sims, uint32_t t0, int64_t n,
                           int64_t* E, int64_t* M, int n_threads)
{
    int failed = 0;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) if (n_threads > 1) reduction(+ : failed)
#endif
    for (int j = 0; j < n_lat; ++j)
        failed += oracle_sw_sweeps(Ls[j], sigmas[j], thrs[j], seeds[j], sims[j], t0, n,
                                   E ? E + (size_t)j * n : NULL, M ? M + (size_t)j * n : NULL) != 0;
    (void)n_threads;
    return failed;
}
