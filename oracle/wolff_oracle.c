/*
 * wolff_oracle.c -- plain CPU oracle for the Wolff single-cluster update.
 *
 * TEST INFRASTRUCTURE ONLY (like ising_oracle.c, whose Philox4x32-10 and
 * energy / magnetization it calls): nothing in the product library links,
 * loads or calls this file.  It shares no code with the CUDA path.
 *
 * The paper names cluster algorithms (Swendsen-Wang, Wolff) as the cure for
 * the critical slowing down of single-site Metropolis (Section 1).  This file
 * writes out Wolff's step (Wolff, PRL 62, 361, 1989) for J = 1, h = 0 on the
 * periodic L x L lattice: pick a seed site; grow a cluster from it, adding a
 * neighbour j of a cluster site i when sigma_j = sigma_i and the bond (i, j)
 * is active, which it is with probability p = 1 - exp(-2 J / T); flip the
 * whole cluster.
 *
 * Draws (this project's definitions; Philox4x32-10 keyed by the lattice seed,
 * counter (q, t, s, phase), t = the step's index in the handle's sweep
 * counter, s = simulation index):
 *   - seed, phase 9: r = lane 0 of block q = 0; the seed is site
 *     p0 = floor(r L^2 / 2^32) (p = y*L + x);
 *   - bonds, phase 10: site p owns the bonds to its right and down
 *     neighbours; q = p >> 1, lane 2*(p & 1) is the right bond's draw and
 *     lane 2*(p & 1) + 1 the down bond's; a bond is active iff its draw
 *     r < thr, thr = min(floor(2^32 p), 2^32 - 1) (the Swendsen-Wang bond
 *     threshold).
 * Every bond has one draw, so a bond is tried at most once, as in Wolff's
 * growth; and the cluster is the connected component of the seed among equal
 * spins joined by active bonds, whatever the order of the growth.  Here the
 * growth is a first-in first-out queue.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int64_t oracle_energy(int L, const int8_t* sigma);
int64_t oracle_magnetization(int L, const int8_t* sigma);

#define ORC_WOLFF_PHASE_SEED 9u
#define ORC_WOLFF_PHASE_BOND 10u

static uint32_t wolff_draw(uint64_t seed, uint32_t q, uint32_t t, uint32_t s, uint32_t phase, uint32_t lane)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { q, t, s, phase };
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[lane];
}

/* The seed site of step t. */
uint32_t oracle_wolff_seed(int L, uint64_t seed, uint32_t s, uint32_t t)
{
    uint64_t r = wolff_draw(seed, 0u, t, s, ORC_WOLFF_PHASE_SEED, 0u);
    return (uint32_t)((r * (uint64_t)L * (uint64_t)L) >> 32);
}

/* Is the bond owned by site p in direction dir (0 = right, 1 = down) active
 * in step t (its draw only; the caller checks the spins)? */
static int wolff_bond_active(uint64_t seed, uint32_t s, uint32_t t, uint32_t thr, uint32_t p, int dir)
{
    uint32_t r = wolff_draw(seed, p >> 1, t, s, ORC_WOLFF_PHASE_BOND, 2u * (p & 1u) + (uint32_t)dir);
    return r < thr;
}

/* One step on sigma (in place).  Returns the cluster size, or -1 if memory
 * runs out. */
int64_t oracle_wolff_step(int L, int8_t* sigma, uint32_t thr, uint64_t seed, uint32_t s, uint32_t t)
{
    const size_t N = (size_t)L * (size_t)L;
    uint32_t* queue = (uint32_t*)malloc(N * sizeof(uint32_t));
    uint8_t* in = (uint8_t*)calloc(N, 1);
    if (!queue || !in) {
        free(queue);
        free(in);
        return -1;
    }
    const uint32_t p0 = oracle_wolff_seed(L, seed, s, t);
    const int8_t s0 = sigma[p0];
    size_t head = 0, tail = 0;
    queue[tail++] = p0;
    in[p0] = 1;
    while (head < tail) {
        const uint32_t p = queue[head++];
        const int x = (int)(p % (uint32_t)L), y = (int)(p / (uint32_t)L);
        /* the four neighbours with the owner and direction of each bond */
        const uint32_t right = (uint32_t)y * L + (uint32_t)((x + 1) % L);
        const uint32_t left = (uint32_t)y * L + (uint32_t)((x + L - 1) % L);
        const uint32_t down = (uint32_t)((y + 1) % L) * L + (uint32_t)x;
        const uint32_t up = (uint32_t)((y + L - 1) % L) * L + (uint32_t)x;
        const uint32_t nb[4] = { right, left, down, up };
        const uint32_t owner[4] = { p, left, p, up };
        const int dir[4] = { 0, 0, 1, 1 };
        for (int k = 0; k < 4; ++k) {
            const uint32_t j = nb[k];
            if (in[j] || sigma[j] != s0) continue;
            if (!wolff_bond_active(seed, s, t, thr, owner[k], dir[k])) continue;
            in[j] = 1;
            queue[tail++] = j;
        }
    }
    for (size_t i = 0; i < tail; ++i) sigma[queue[i]] = (int8_t)(-s0);
    free(queue);
    free(in);
    return (int64_t)tail;
}

/* n steps with indices t0 .. t0+n-1; E, M and the cluster sizes after each
 * (any may be NULL).  Returns 0, or -1 if memory runs out. */
int oracle_wolff_steps(int L, int8_t* sigma, uint32_t thr, uint64_t seed, uint32_t s, uint32_t t0, int64_t n,
                       int64_t* E, int64_t* M, int64_t* size)
{
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = oracle_wolff_step(L, sigma, thr, seed, s, t0 + (uint32_t)i);
        if (c < 0) return -1;
        if (size) size[i] = c;
        if (E) E[i] = oracle_energy(L, sigma);
        if (M) M[i] = oracle_magnetization(L, sigma);
    }
    return 0;
}

/* Many lattices, one OpenMP thread per lattice at a time; lattice j uses
 * thrs[j], seeds[j], sims[j]; traces [n_lat][n]. */
int oracle_wolff_steps_batch(int n_lat, const int* Ls, int8_t* const* sigmas, const uint32_t* thrs,
                             const uint64_t* seeds, const uint32_t* sims, uint32_t t0, int64_t n, int64_t* E,
                             int64_t* M, int n_threads)
{
    int bad = 0;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(| : bad) if (n_threads > 1)
#endif
    for (int j = 0; j < n_lat; ++j)
        bad |= oracle_wolff_steps(Ls[j], sigmas[j], thrs[j], seeds[j], sims[j], t0, n,
                                  E ? E + (size_t)j * n : NULL, M ? M + (size_t)j * n : NULL, NULL) != 0;
    (void)n_threads;
    return bad ? -1 : 0;
}
