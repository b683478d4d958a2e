/*
 * ising_oracle.c -- plain CPU oracle for the checkerboard Metropolis sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, __graft_entry__.smoke() and the CPU
 * baseline arm of bench.py do.  It shares no code, header, table or constant
 * generator with the CUDA path: every definition below is written out here
 * from the paper and from the published definition of Philox4x32-10.
 *
 * Representation: one signed byte per spin, sigma[y*L + x] in {+1, -1},
 * periodic L x L lattice, J = 1, h = 0.  No packing, no blocking, no reuse of
 * random blocks between sites: every site that needs a random number calls
 * the generator on its own counter.
 *
 * What each function follows:
 *   - Hamiltonian H = -J sum_<ij> s_i s_j over nearest neighbours, 4 in 2D
 *     (Section 1, Ising Hamiltonian).
 *   - Metropolis rule: accept iff ran() < exp(-beta dE) (Section 1), applied
 *     with an unsigned 32-bit uniform r and threshold
 *     thr = min(floor(2^32 exp(-dE/T)), 2^32-1); moves with dE <= 0 are
 *     always accepted and draw nothing.
 *   - Checkerboard order: red = (x+y) even first, then blue = (x+y) odd
 *     (Algorithm 5, supplementary); here red is called "black" (colour 0)
 *     and blue "white" (colour 1).  All four neighbours enter the local field
 *     (the sum printed in Algorithms 4/5 lists three; the text of Section 1
 *     fixes four).
 *   - The paper's hardware generator is not public (supplementary, PRNG
 *     tests); it is replaced by Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     SC'11), keyed by the 64-bit seed (key = lo32, hi32) with counter
 *     (q, t, s, phase): t = sweep index, s = simulation index, phase 0/1 =
 *     black/white half-sweep, 2 = initial state; q = p >> 2 and output lane
 *     p & 3, where p is the site's rank among same-colour sites of the
 *     lattice in row-major order, p = y*(L/2) + (x >> 1) (for the initial
 *     state p = y*L + x over all sites).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Philox4x32 constants: the two round multipliers and the two Weyl key
 * increments (golden ratio and sqrt(3)-1 in 32-bit fixed point), as
 * published by Salmon et al. 2011. */
#define ORC_PHILOX_MUL_A 0xD2511F53u
#define ORC_PHILOX_MUL_B 0xCD9E8D57u
#define ORC_PHILOX_WEYL_A 0x9E3779B9u
#define ORC_PHILOX_WEYL_B 0xBB67AE85u

/* One Philox4x32 block with 10 rounds.  Each round: two 32x32->64 products
 * of counter words 0 and 2 with the multipliers; the new counter is
 * (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0)); the key is
 * advanced by the Weyl increments between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_WEYL_A;
            k1 += ORC_PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)ORC_PHILOX_MUL_A * (uint64_t)c0;
        uint64_t prod_b = (uint64_t)ORC_PHILOX_MUL_B * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod_b >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod_b;
        uint32_t n2 = (uint32_t)(prod_a >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The uniform 32-bit draw for rank p in (sweep t, simulation s, phase). */
uint32_t oracle_site_random(uint64_t seed, uint32_t p, uint32_t t, uint32_t s, uint32_t phase)
{
    uint32_t ctr[4] = { p >> 2, t, s, phase };
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[p & 3u];
}

/* Acceptance thresholds for dE = 4 (thr[0]) and dE = 8 (thr[1]) at
 * temperature T (J = 1, k_B = 1): thr = min(floor(2^32 exp(-dE/T)), 2^32-1).
 * Returns -1 for T that is not a positive finite number. */
int oracle_thresholds(double T, uint32_t thr[2])
{
    if (!(T > 0.0) || !isfinite(T)) return -1;
    for (int k = 0; k < 2; ++k) {
        double dE = 4.0 * (double)(k + 1);
        double v = ldexp(exp(-dE / T), 32);
        thr[k] = (v >= 4294967296.0) ? 0xFFFFFFFFu : (uint32_t)floor(v);
    }
    return 0;
}

static inline int wrap(int i, int L) { return ((i % L) + L) % L; }

/* H = -sum over every site of sigma * (right + down neighbour): each bond
 * once. */
int64_t oracle_energy(int L, const int8_t* sigma)
{
    int64_t e = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int s = sigma[(size_t)y * L + x];
            int r = sigma[(size_t)y * L + wrap(x + 1, L)];
            int d = sigma[(size_t)wrap(y + 1, L) * L + x];
            e -= (int64_t)(s * (r + d));
        }
    return e;
}

int64_t oracle_magnetization(int L, const int8_t* sigma)
{
    int64_t m = 0;
    for (size_t i = 0; i < (size_t)L * L; ++i) m += sigma[i];
    return m;
}

/* Metropolis decision for one site of colour c in sweep t. */
static inline void update_site(int L, int8_t* sigma, int x, int y, int c,
                               const uint32_t thr[2], uint64_t seed,
                               uint32_t s, uint32_t t)
{
    size_t i = (size_t)y * L + x;
    int h = sigma[(size_t)wrap(y - 1, L) * L + x] + sigma[(size_t)wrap(y + 1, L) * L + x]
          + sigma[(size_t)y * L + wrap(x - 1, L)] + sigma[(size_t)y * L + wrap(x + 1, L)];
    int dE = 2 * sigma[i] * h;
    int flip;
    if (dE <= 0) {
        flip = 1;
    } else {
        uint32_t p = (uint32_t)y * (uint32_t)(L / 2) + (uint32_t)(x >> 1);
        uint32_t r = oracle_site_random(seed, p, t, s, (uint32_t)c);
        flip = r < thr[dE == 8 ? 1 : 0];
    }
    if (flip) sigma[i] = (int8_t)(-sigma[i]);
}

/* One half-sweep over every site of colour c ((x+y) % 2 == c).  Sites of one
 * colour never neighbour each other, so rows may be split across threads
 * without changing any result. */
void oracle_half_sweep(int L, int8_t* sigma, int c, const uint32_t thr[2],
                       uint64_t seed, uint32_t s, uint32_t t, int n_threads)
{
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(static) num_threads(n_threads) if (n_threads > 1)
#endif
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            if (((x + y) & 1) == c) update_site(L, sigma, x, y, c, thr, seed, s, t);
    (void)n_threads;
}

/* n full sweeps (black then white), sweep indices t0 .. t0+n-1; after each
 * sweep E and M are written to the traces (either may be NULL). */
void oracle_sweeps(int L, int8_t* sigma, const uint32_t thr[2], uint64_t seed,
                   uint32_t s, uint32_t t0, int64_t n, int64_t* E, int64_t* M,
                   int n_threads)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t t = t0 + (uint32_t)i;
        oracle_half_sweep(L, sigma, 0, thr, seed, s, t, n_threads);
        oracle_half_sweep(L, sigma, 1, thr, seed, s, t, n_threads);
        if (E) E[i] = oracle_energy(L, sigma);
        if (M) M[i] = oracle_magnetization(L, sigma);
    }
}

/* Many independent lattices (possibly of different L); one OpenMP thread per
 * lattice at a time.  Lattice j uses simulation index sims[j], key seeds[j],
 * thresholds thr[2j..2j+1]; traces are [n_lat][n]. */
void oracle_sweeps_batch(int n_lat, const int* Ls, int8_t* const* sigmas,
                         const uint32_t* thr, const uint64_t* seeds,
                         const uint32_t* sims, uint32_t t0, int64_t n,
                         int64_t* E, int64_t* M, int n_threads)
{
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) if (n_threads > 1)
#endif
    for (int j = 0; j < n_lat; ++j)
        oracle_sweeps(Ls[j], sigmas[j], thr + 2 * j, seeds[j], sims[j], t0, n,
                      E ? E + (size_t)j * n : NULL, M ? M + (size_t)j * n : NULL, 1);
    (void)n_threads;
}

/* ---------------------------------------------------------------------------
 * Light-cone window.  The value of a site after n sweeps depends only on the
 * initial values within lattice distance 2n (each half-sweep reads nearest
 * neighbours only).  These two functions apply the very same definitions to a
 * h x w window whose top-left corner is the global site (x0, y0) (indices mod
 * L): draws use global coordinates, the window's outermost ring is never
 * updated.  After n sweeps every window site at distance >= 2n+1 from the
 * window edge holds exactly the value the full-lattice definition gives.
 * ------------------------------------------------------------------------- */
int oracle_window_init(int L, uint64_t seed, uint32_t s, int mode,
                       int y0, int x0, int h, int w, int8_t* win)
{
    if (L < 2 || (L & 1)) return -1;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            int y = wrap(y0 + i, L), x = wrap(x0 + j, L);
            int8_t v = 1;
            if (mode == 0) {
                uint32_t p = (uint32_t)y * (uint32_t)L + (uint32_t)x;
                v = (oracle_site_random(seed, p, 0u, s, 2u) >> 31) ? (int8_t)-1 : (int8_t)1;
            }
            win[(size_t)i * w + j] = v;
        }
    return 0;
}

void oracle_window_sweeps(int L, int8_t* win, int y0, int x0, int h, int w,
                          const uint32_t thr[2], uint64_t seed, uint32_t s,
                          uint32_t t0, int64_t n)
{
    for (int64_t it = 0; it < n; ++it) {
        uint32_t t = t0 + (uint32_t)it;
        for (int c = 0; c < 2; ++c) {
            for (int i = 1; i < h - 1; ++i)
                for (int j = 1; j < w - 1; ++j) {
                    int y = wrap(y0 + i, L), x = wrap(x0 + j, L);
                    if (((x + y) & 1) != c) continue;
                    size_t k = (size_t)i * w + j;
                    int hf = win[k - w] + win[k + w] + win[k - 1] + win[k + 1];
                    int dE = 2 * win[k] * hf;
                    int flip;
                    if (dE <= 0) {
                        flip = 1;
                    } else {
                        uint32_t p = (uint32_t)y * (uint32_t)(L / 2) + (uint32_t)(x >> 1);
                        flip = oracle_site_random(seed, p, t, s, (uint32_t)c) < thr[dE == 8 ? 1 : 0];
                    }
                    if (flip) win[k] = (int8_t)(-win[k]);
                }
        }
    }
}

/* Initial state: mode 1 = cold (all +1); mode 0 = random, sigma = +1 iff the
 * top bit of the site's draw (phase 2, sweep 0, p = y*L + x) is 0.  Rows may
 * be split across threads: every site has its own draw. */
int oracle_init_parallel(int L, uint64_t seed, uint32_t s, int mode, int8_t* sigma, int n_threads)
{
    if (L < 2 || (L & 1)) return -1;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(static) num_threads(n_threads) if (n_threads > 1)
#endif
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int8_t v = 1;
            if (mode == 0) {
                uint32_t p = (uint32_t)y * (uint32_t)L + (uint32_t)x;
                v = (oracle_site_random(seed, p, 0u, s, 2u) >> 31) ? (int8_t)-1 : (int8_t)1;
            }
            sigma[(size_t)y * L + x] = v;
        }
    (void)n_threads;
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
