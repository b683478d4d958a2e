// ising_cluster.cu -- sm_103a kernels of the Swendsen-Wang cluster step.
//
// The paper names cluster algorithms (Swendsen-Wang, Wolff) as the remedy for
// the critical slowing down of single-site Metropolis (Section 1).  One
// Swendsen-Wang step (Swendsen and Wang 1987), J = 1, h = 0, periodic L x L:
//   1. every nearest-neighbour pair of equal spins gets an active bond with
//      probability 1 - exp(-2/T);
//   2. clusters = connected components of the active bonds;
//   3. each cluster flips with probability 1/2.
// Draws: Philox4x32-10 keyed by the lattice seed, counter (q, t, s, phase).
// Bonds (phase 7): site p = y*L + x owns its right and down bonds, q = p >> 1,
// lane 2*(p & 1) for the right bond and 2*(p & 1) + 1 for the down bond; a
// bond between equal spins is active iff its draw is below the threshold.
// Coins (phase 8): a cluster is named by its smallest site index r0 and flips
// iff the top bit of lane r0 & 3 of block r0 >> 2 is set.  The partition and
// its minimum-index roots are unique, so the step is bit-reproducible
// whatever the labelling order.
//
// Labelling is a lock-free union-find whose links always point from a larger
// to a smaller index (atomicMin on the larger root), so that a component's
// final root is its smallest index:
//   sw_local_kernel   one warp per 64 x kSwTileH tile, rows in order: spins
//                     from the packed words, bonds; each row's runs of right
//                     bonds label themselves by their first site and join
//                     the runs above through the down bonds (union-find in
//                     shared memory); the global labels (every site -> its
//                     tile-local root), a bit mask of the tile-local roots
//                     and the edge bonds;
//   sw_merge_kernel   unions over the bonds that cross tile edges (global);
//   sw_resolve_kernel every tile-local root -> its final root, whose coin it
//                     takes over (one bit per tile-local root);
//   sw_flip_kernel    both colour words of (y, k) flipped by the coin bit of
//                     each site's tile-local root.
// Every pointer walk and union retry is bounded; running past a bound (which
// the strictly decreasing links make impossible for a consistent array) sets
// the error word and leaves the labels in range.
#include "ising_internal.h"
#include "ising_device.cuh"

#include <cuda_runtime.h>
#include <cstdint>

namespace ising {
namespace {

constexpr int kTileW = kSwTileW, kTileH = kSwTileH, kTileSites = kTileW * kTileH;
static_assert(kTileW == 64 && kTileH <= 32 && kSwThreads % 32 == 0, "one 64-bit word per tile row, edge rows in 32 bits");
constexpr int kWordsPerTile = kTileSites / 32;     // resolve: one thread per 32 sites
constexpr int kPairsPerTile = kTileSites / 64;     // flip: one thread per 64 sites
constexpr int kEdgeSites = kTileH + kTileW;        // merge: right edge rows + bottom edge columns
constexpr uint32_t kPhaseCoin = 8u, kPhaseWolffSeed = 9u, kPhaseWolffBond = kWolffBondPhase;
constexpr int kMaxChain = 1 << 26;                 // bound on one parent-pointer walk
constexpr int kMaxRetry = 1 << 22;                 // bound on the retries of one union
constexpr int kErrUnionBound = 3;                  // error word value

// Lattice of a tile: the last lattice with tile_begin <= tile.
__device__ __forceinline__ int lattice_of_tile(const SwLat* lat, int n, uint32_t tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lat[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The 64-bit mask of a tile row in natural order (bit j <-> x0 + j) from each
// lane's two sites x0 + 2l (bit 0 of v) and x0 + 2l + 1 (bit 1): lanes 0..15
// fill the low word, lanes 16..31 the high one (two warp OR-reductions).
__device__ __forceinline__ uint64_t row_mask(uint32_t v, uint32_t lane) {
    const uint32_t sh = v << (2u * (lane & 15u));
    const uint32_t lo = __reduce_or_sync(0xffffffffu, lane < 16u ? sh : 0u);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, lane < 16u ? 0u : sh);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// The 32 bits of v moved to the even bit positions of a 64-bit word.
__device__ __forceinline__ uint64_t spread_even(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// Sites x in [64k, 64k + 64) of row y in natural order (bit i <-> x = 64k + i):
// colour c holds x = 2(32k + b) + ((y + c) & 1), so even x come from colour
// y & 1 and odd x from the other one.
__device__ __forceinline__ uint64_t natural_row(const uint32_t* base, uint32_t L, uint32_t wn, uint32_t y,
                                                uint32_t k) {
    const uint32_t ce = y & 1u;
    const uint32_t we = base[((size_t)ce * L + y) * wn + k];
    const uint32_t wo = base[((size_t)(ce ^ 1u) * L + y) * wn + k];
    return spread_even(we) | (spread_even(wo) << 1);
}

// --- union-find in shared memory (one tile, indices < kTileSites) ---------
// Path halving by atomicMin: a link only ever moves down to an ancestor, so a
// walk ends within kTileSites steps.
__device__ __forceinline__ uint32_t find_tile(uint32_t* lab, uint32_t x) {
    const volatile uint32_t* v = lab;
    uint32_t p = v[x];
    for (int it = 0; it < kTileSites && p != x; ++it) {
        const uint32_t gp = v[p];
        if (gp != p) atomicMin(&lab[x], gp);
        x = p;
        p = gp;
    }
    return x;
}

__device__ __forceinline__ void unite_tile(uint32_t* lab, uint32_t a, uint32_t b) {
    for (int it = 0; it < kTileSites; ++it) {
        a = find_tile(lab, a);
        b = find_tile(lab, b);
        if (a == b) return;
        if (a > b) { const uint32_t s = a; a = b; b = s; }
        const uint32_t old = atomicMin(&lab[b], a);
        if (old == b) return;     // b was a root and now hangs under a
        b = old;                  // b had been linked meanwhile: merge a with its parent
    }
}

// --- union-find in global memory (one lattice) ----------------------------
// Path halving by atomicMin: a link only ever moves down to an ancestor.
// Returns the root, or ~0u if the walk ran past its bound.
__device__ __forceinline__ uint32_t find_global(uint32_t* lab, uint32_t x) {
    const volatile uint32_t* v = lab;
    uint32_t p = v[x];
    for (int it = 0; it < kMaxChain; ++it) {
        if (p == x) return x;
        const uint32_t gp = v[p];
        if (gp != p) atomicMin(&lab[x], gp);
        x = p;
        p = gp;
    }
    return ~0u;
}

__device__ __forceinline__ bool unite_global(uint32_t* lab, uint32_t a, uint32_t b) {
    for (int it = 0; it < kMaxRetry; ++it) {
        a = find_global(lab, a);
        b = find_global(lab, b);
        if (a == ~0u || b == ~0u) return false;
        if (a == b) return true;
        if (a > b) { const uint32_t s = a; a = b; b = s; }
        const uint32_t old = atomicMin(&lab[b], a);
        if (old == b) return true;
        b = old;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Bonds and tile-local labels: one warp per tile, rows in order.  Lane l owns
// the sites x0 + 2l and x0 + 2l + 1 of every row, whose four bond draws are
// one Philox block (q = p >> 1 with p = y*L + x0 + 2l even).  Row k: the
// row's right / down bond masks come from two warp OR-reductions each
// (row_mask); every site of a
// run of right bonds is labelled by the run's first site; the runs are joined
// to the runs of row k - 1 through the down bonds of row k - 1 (one union per
// pair of runs, lanes in parallel).  The tile is flattened at the end by
// pointer jumping.
// ---------------------------------------------------------------------------
constexpr int kTilesPerBlock = kSwThreads / 32;

__global__ void __launch_bounds__(kSwThreads) sw_local_kernel(DevState st, SwState sw) {
    __shared__ uint32_t s_lab[kTilesPerBlock][kTileSites];
    __shared__ uint64_t s_row[kTilesPerBlock][kTileH + 1];   // natural-order spins of rows y0 .. y0 + kTileH
    __shared__ uint64_t s_R[kTilesPerBlock][kTileH];         // right bonds per row (bit 63 leaves the tile)
    __shared__ uint64_t s_D[kTilesPerBlock][kTileH];         // down bonds per row (the last row leaves it)
    __shared__ uint32_t s_rbit[kTilesPerBlock][kTileH];      // spin of the site right of the tile, per row
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t tile = blockIdx.x * kTilesPerBlock + warp;
    if (tile >= sw.total_tiles) return;              // whole warps only; no block barrier below
    uint32_t* lab = s_lab[warp];
    const SwLat d = sw.lat[lattice_of_tile(sw.lat, sw.n, tile)];
    const uint32_t L = d.L, wn = d.wn;
    const uint32_t local = tile - d.tile_begin;
    const uint32_t tx = local % wn, ty = local / wn;     // L / 64 tiles per tile row
    const uint32_t x0 = kTileW * tx, y0 = kTileH * ty;
    const uint32_t* base = st.spins + d.word_off;
    const uint32_t t = (uint32_t)st.ctl->t;
    const uint32_t xe = 2u * lane, xo = xe + 1u;

    // all rows of the tile at once (the last one wraps at the lattice edge)
    if (lane <= (uint32_t)kTileH) {
        uint32_t y = y0 + lane;
        if (y >= L) y -= L;
        s_row[warp][lane] = natural_row(base, L, wn, y, tx);
        if (lane < (uint32_t)kTileH) {
            const uint32_t kr = (tx + 1 == wn) ? 0u : tx + 1;   // x = 64 kr: even, colour y & 1
            s_rbit[warp][lane] = base[((size_t)(y & 1u) * L + y) * wn + kr] & 1u;
        }
    }
    __syncwarp();
    // bonds of every row: the four draws of lane l's two sites are one block
#pragma unroll 4
    for (uint32_t k = 0; k < (uint32_t)kTileH; ++k) {
        const uint64_t row = s_row[warp][k], below = s_row[warp][k + 1];
        const uint64_t al_r = ~(row ^ ((row >> 1) | ((uint64_t)s_rbit[warp][k] << 63)));
        const uint64_t al_d = ~(row ^ below);
        const uint32_t p = (y0 + k) * L + x0 + xe;
        const uint4 r = philox(p >> 1, t, d.sim, sw.bond_phase, d.key0, d.key1);
        const uint32_t vr = (uint32_t)(((al_r >> xe) & 1u) && r.x < d.thr) |
                            ((uint32_t)(((al_r >> xo) & 1u) && r.z < d.thr) << 1);
        const uint32_t vd = (uint32_t)(((al_d >> xe) & 1u) && r.y < d.thr) |
                            ((uint32_t)(((al_d >> xo) & 1u) && r.w < d.thr) << 1);
        const uint64_t mr = row_mask(vr, lane), md = row_mask(vd, lane);
        if (lane == 0) {
            s_R[warp][k] = mr;
            s_D[warp][k] = md;
        }
    }
    __syncwarp();

    // rows in order: runs label themselves and join the runs above
    const uint64_t upto_e = ~0ull >> (63u - xe), upto_o = ~0ull >> (63u - xo);
    uint64_t inner_prev = 0;
#pragma unroll 1
    for (uint32_t k = 0; k < (uint32_t)kTileH; ++k) {
        const uint64_t inner = s_R[warp][k] & 0x7FFFFFFFFFFFFFFFull;
        const uint64_t starts = ~(inner << 1);         // bit j: no bond into site j
        const uint32_t i0 = k * kTileW;
        lab[i0 + xe] = i0 + 63u - (uint32_t)__clzll((long long)(starts & upto_e));
        lab[i0 + xo] = i0 + 63u - (uint32_t)__clzll((long long)(starts & upto_o));
        __syncwarp();
        if (k > 0) {
            // one contact per pair of runs: a down bond at x is skipped when
            // the down bond at x - 1 joins the same two runs
            const uint64_t down = s_D[warp][k - 1];
            const uint64_t need = down & ~((down & inner_prev & inner) << 1);
            if ((need >> xe) & 1u) unite_tile(lab, i0 - kTileW + xe, i0 + xe);
            if ((need >> xo) & 1u) unite_tile(lab, i0 - kTileW + xo, i0 + xo);
            __syncwarp();
        }
        inner_prev = inner;
    }
    // final flatten by pointer jumping (depth < kTileSites <= 2^11)
#pragma unroll 1
    for (int round = 0; round < 12; ++round) {
        bool changed = false;
        for (uint32_t i = lane; i < (uint32_t)kTileSites; i += 32u) {
            const uint32_t q = lab[i], gq = lab[q];
            if (gq != q) {
                lab[i] = gq;
                changed = true;
            }
        }
        if (!__any_sync(0xffffffffu, changed)) break;
        __syncwarp();
    }
    __syncwarp();
    // global labels (site -> tile-local root), root mask, edge bonds
    uint32_t* glab = sw.label + d.site_off;
#pragma unroll 4
    for (uint32_t k = 0; k < (uint32_t)kTileH; ++k) {
        const uint32_t i0 = k * kTileW;
        const uint32_t re = lab[i0 + xe], ro = lab[i0 + xo];
        const uint32_t pe = (y0 + k) * L + x0 + xe;
        *reinterpret_cast<uint2*>(glab + pe) = make_uint2((y0 + (re >> 6)) * L + x0 + (re & 63u),
                                                          (y0 + (ro >> 6)) * L + x0 + (ro & 63u));
        const uint64_t roots = row_mask((uint32_t)(re == i0 + xe) | ((uint32_t)(ro == i0 + xo) << 1), lane);
        if (lane < 2) sw.coins[(d.site_off + (uint64_t)(y0 + k) * L + x0) / 32 + lane] = (uint32_t)(roots >> (32 * lane));
    }
    if (lane == 0) {
        uint32_t edge_r = 0;
        for (int k = 0; k < kTileH; ++k) edge_r |= (uint32_t)(s_R[warp][k] >> 63) << k;
        const uint64_t edge_d = s_D[warp][kTileH - 1];
        sw.edges[tile] = make_uint4(edge_r, 0u, (uint32_t)edge_d, (uint32_t)(edge_d >> 32));
    }
}

// ---------------------------------------------------------------------------
// Unions over the bonds leaving each tile to the right and downwards.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sw_merge_kernel(DevState st, SwState sw) {
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t tile = gid / kEdgeSites;
    if (tile >= sw.total_tiles) return;
    const uint32_t e = (uint32_t)(gid - tile * kEdgeSites);
    const uint4 ed = sw.edges[tile];
    const bool on = (e < (uint32_t)kTileH) ? ((ed.x >> e) & 1u) != 0
                                          : ((e - kTileH < 32u) ? ((ed.z >> (e - kTileH)) & 1u) != 0
                                                                : ((ed.w >> (e - kTileH - 32u)) & 1u) != 0);
    if (!on) return;
    const SwLat d = sw.lat[lattice_of_tile(sw.lat, sw.n, (uint32_t)tile)];
    const uint32_t L = d.L, wn = d.wn;
    const uint32_t local = (uint32_t)tile - d.tile_begin;
    const uint32_t x0 = kTileW * (local % wn), y0 = kTileH * (local / wn);
    uint32_t a, b;
    if (e < (uint32_t)kTileH) {
        const uint32_t y = y0 + e, xr = (x0 + kTileW == L) ? 0u : x0 + kTileW;
        a = y * L + x0 + kTileW - 1;
        b = y * L + xr;
    } else {
        const uint32_t x = x0 + (e - kTileH), yb = (y0 + kTileH == L) ? 0u : y0 + kTileH;
        a = (y0 + kTileH - 1) * L + x;
        b = yb * L + x;
    }
    if (!unite_global(sw.label + d.site_off, a, b)) atomicExch(&st.ctl->error, kErrUnionBound);
}

// ---------------------------------------------------------------------------
// Every tile-local root (bit mask left in the coin array by sw_local_kernel)
// is resolved to its final root f and takes f's coin (the top bit of lane
// f & 3 of block f >> 2), which replaces the mask bit; the flip then needs
// only the coin bit of each site's tile-local root.  One warp per tile (a
// tile is 32 coin words): the tile's roots are dealt out evenly over the
// lanes -- root j of the tile (in word order) goes to lane j mod 32, which
// finds its word by a search over the warp's prefix counts and its bit by a
// popcount search -- and the coins are gathered back per word in shared
// memory.
// ---------------------------------------------------------------------------
static_assert(kWordsPerTile == 32, "one warp per tile in sw_resolve_kernel");
// Position of the k-th (from 0) set bit of m, which has more than k set bits:
// halve the window five times, skipping the low half when it holds <= k bits.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (int width = 16; width > 0; width >>= 1) {
        const uint32_t c = __popc(m & ((1u << width) - 1u));
        if (k >= c) {
            k -= c;
            m >>= width;
            pos += (uint32_t)width;
        }
    }
    return pos;
}
__global__ void __launch_bounds__(256) sw_resolve_kernel(DevState st, SwState sw) {
    __shared__ uint32_t s_coin[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t tile = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= sw.total_tiles) return;                 // whole warps
    const SwLat d = sw.lat[lattice_of_tile(sw.lat, sw.n, (uint32_t)tile)];
    const uint32_t w = (uint32_t)((tile - d.tile_begin) * kWordsPerTile) + (uint32_t)lane;   // word in the lattice
    uint32_t* lab = sw.label + d.site_off;
    uint32_t* coin_word = sw.coins + d.site_off / 32 + w;
    const uint32_t t = (uint32_t)st.ctl->t;
    const uint32_t m = *coin_word;
    uint32_t incl = __popc(m);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - __popc(m), total = __shfl_sync(0xffffffffu, incl, 31);
    s_coin[warp][lane] = 0u;
    __syncwarp();
    bool failed = false;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        // owner lane: the last lane whose exclusive count is <= j
        int o = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t e = __shfl_sync(0xffffffffu, excl, o + step);
            if (e <= j) o += step;
        }
        const uint32_t mo = __shfl_sync(0xffffffffu, m, o), eo = __shfl_sync(0xffffffffu, excl, o);
        if (j >= total) continue;
        const uint32_t i = nth_set_bit(mo, j - eo);
        const uint32_t r = 32u * (w - (uint32_t)lane + (uint32_t)o) + i;
        const uint32_t f = find_global(lab, r);
        if (f == ~0u) {
            failed = true;
            continue;
        }
        if (f != r) lab[r] = f;
        bool flip;
        if (sw.seed_root) {
            flip = f == sw.seed_root[d.sim];           // Wolff: only the seed's cluster
        } else {
            const uint4 v = philox(f >> 2, t, d.sim, kPhaseCoin, d.key0, d.key1);
            const uint32_t ln = f & 3u;
            flip = ((ln == 0 ? v.x : ln == 1 ? v.y : ln == 2 ? v.z : v.w) >> 31) != 0;
        }
        if (flip) atomicOr(&s_coin[warp][o], 1u << i);
    }
    if (failed) atomicExch(&st.ctl->error, kErrUnionBound);
    __syncwarp();
    *coin_word = s_coin[warp][lane];
}

// Wolff by labelling: the seed of each lattice (phase 9, as the growth
// kernel draws it) resolved to its final root.  One thread per lattice.
__global__ void wolff_seed_kernel(DevState st, SwState sw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sw.n) return;
    const SwLat d = sw.lat[i];
    const uint32_t t = (uint32_t)st.ctl->t;
    const uint32_t N = d.L * d.L;
    const uint32_t r = philox(0u, t, d.sim, kPhaseWolffSeed, d.key0, d.key1).x;
    const uint32_t p0 = (uint32_t)(((uint64_t)r * N) >> 32);
    const uint32_t f = find_global(sw.label + d.site_off, p0);
    if (f == ~0u) atomicExch(&st.ctl->error, kErrUnionBound);
    sw.seed_root[d.sim] = f;
}

// Every site points at its final root (only for ising_sw_labels): the link
// of a site is a tile-local root (of its own tile, or of another one after a
// path-halving step of the merge), whose link is final after
// sw_resolve_kernel.
__global__ void __launch_bounds__(256) sw_compress_kernel(SwState sw, uint64_t sites) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sites) return;
    const SwLat d = sw.lat[lattice_of_tile(sw.lat, sw.n, (uint32_t)(g / kTileSites))];
    uint32_t* lab = sw.label + d.site_off;
    const uint32_t p = (uint32_t)(g - d.site_off);
    lab[p] = lab[lab[p]];
}

// ---------------------------------------------------------------------------
// Flip: both colour words of (y, k), i.e. the 64 sites x in [64k, 64k + 64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sw_flip_kernel(DevState st, SwState sw) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)sw.total_tiles * kPairsPerTile) return;
    const SwLat d = sw.lat[lattice_of_tile(sw.lat, sw.n, (uint32_t)(g / kPairsPerTile))];
    const uint32_t i = (uint32_t)(g - (uint64_t)d.tile_begin * kPairsPerTile);
    const uint32_t L = d.L, wn = d.wn;
    const uint32_t y = i / wn, k = i - y * wn;
    const uint32_t p0 = y * L + 64u * k;
    const uint4* lab = reinterpret_cast<const uint4*>(sw.label + d.site_off + p0);
    const uint32_t* coins = sw.coins + d.site_off / 32;   // coin of each tile-local root's cluster
    uint32_t m_even = 0, m_odd = 0;
#pragma unroll 4
    for (uint32_t q = 0; q < 16; ++q) {
        const uint4 r = lab[q];
        const uint32_t c0 = (coins[r.x >> 5] >> (r.x & 31u)) & 1u;
        const uint32_t c1 = (coins[r.y >> 5] >> (r.y & 31u)) & 1u;
        const uint32_t c2 = (coins[r.z >> 5] >> (r.z & 31u)) & 1u;
        const uint32_t c3 = (coins[r.w >> 5] >> (r.w & 31u)) & 1u;
        m_even |= (c0 << (2 * q)) | (c2 << (2 * q + 1));
        m_odd |= (c1 << (2 * q)) | (c3 << (2 * q + 1));
    }
    uint32_t* base = st.spins + d.word_off;
    const uint32_t ce = y & 1u;
    base[((size_t)ce * L + y) * wn + k] ^= m_even;
    base[((size_t)(ce ^ 1u) * L + y) * wn + k] ^= m_odd;
}

// E, M of the step from the observables kernel's sums (aligned bonds, -1
// spins; the sums are cleared) into obs, the trace and the moments; then
// advance the device sweep counter.  One block.
__global__ void sw_record_kernel(DevState st, int n_lat) {
    const unsigned long long t = st.ctl->t;
    for (int lat = threadIdx.x; lat < n_lat; lat += blockDim.x) {
        const uint32_t L = st.lat[lat].L;
        const long long N = (long long)L * L;
        const unsigned long long sa = st.acc[2 * lat], sp = st.acc[2 * lat + 1];
        st.acc[2 * lat] = 0;
        st.acc[2 * lat + 1] = 0;
        record_em(st, (uint32_t)lat, L, 2 * N - 2 * (long long)sa, N - 2 * (long long)sp, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) st.ctl->t = t + 1;
}

// ---------------------------------------------------------------------------
// Wolff single-cluster step (Wolff 1989), every lattice at once, one block
// per lattice and all steps of a call in one launch.  Draws: the seed site is
// floor(r L^2 / 2^32), r = lane 0 of block 0, phase 9; site p owns its right
// and down bonds, whose draws are lanes 2(p & 1) and 2(p & 1) + 1 of block
// p >> 1, phase 10, active iff below the Swendsen-Wang bond threshold.  With
// one draw per bond the cluster is the seed's connected component among
// equal spins joined by active bonds, so a parallel breadth-first growth
// finds exactly the cluster of a sequential one.  Per step: levels of the
// growth (a queue of sites, a visited bit per site claimed by atomicOr); then
// the energy change from the bonds leaving the cluster, the flips (atomicXor
// on the packed words), the visited bits cleared, E and M recorded.  Every
// loop is bounded by L^2.
//
// The growth is a chain of dependent steps (a site is found only after its
// parent), so the latency of each hop sets the time.  Lattices with
// L <= kWolffSmemMaxL run entirely in shared memory (packed spins, visited
// bits, a queue of 16-bit site indices: 2.25 L^2 bytes, 144 KB at 256^2),
// loaded once per call and written back at its end; larger ones keep the
// queue in the cluster scratch's labels and the visited bits in its coins,
// and read spins, visited bits and queue from L2 (__ldcg): the flips and the
// claims are atomics, which act in L2, and an L1 line read earlier in the
// launch could be stale.
// ---------------------------------------------------------------------------
constexpr int kWolffThreads = 512;
constexpr uint32_t kWolffSmemMaxL = 256;

template <bool SMEM>
struct WolffStore {
    uint32_t* words;      // packed spins of the lattice
    uint32_t* vis;        // visited bits
    uint32_t* q32;        // queue (global)
    uint16_t* q16;        // queue (shared)
    uint32_t L, wn;
    __device__ __forceinline__ uint32_t load(const uint32_t* a) const { return SMEM ? *a : __ldcg(a); }
    __device__ __forceinline__ uint32_t word_index(uint32_t x, uint32_t y) const {
        return ((x + y) & 1u) * L * wn + y * wn + (x >> 6);
    }
    __device__ __forceinline__ uint32_t spin(uint32_t x, uint32_t y) const {
        return (load(&words[word_index(x, y)]) >> ((x >> 1) & 31u)) & 1u;
    }
    __device__ __forceinline__ bool visited(uint32_t v) const { return (load(&vis[v >> 5]) >> (v & 31u)) & 1u; }
    __device__ __forceinline__ bool claim(uint32_t v) {      // true if this call set the bit
        const uint32_t bit = 1u << (v & 31u);
        return !(atomicOr(&vis[v >> 5], bit) & bit);
    }
    __device__ __forceinline__ void unclaim(uint32_t v) { atomicAnd(&vis[v >> 5], ~(1u << (v & 31u))); }
    __device__ __forceinline__ uint32_t get(uint32_t k) const { return SMEM ? (uint32_t)q16[k] : __ldcg(&q32[k]); }
    __device__ __forceinline__ void put(uint32_t k, uint32_t v) {
        if (SMEM) q16[k] = (uint16_t)v;
        else q32[k] = v;
    }
    __device__ __forceinline__ void flip(uint32_t x, uint32_t y) {
        atomicXor(&words[word_index(x, y)], 1u << ((x >> 1) & 31u));
    }
};

template <bool SMEM>
__global__ void __launch_bounds__(kWolffThreads, 1) wolff_kernel(DevState st, SwState sw, long long n_steps) {
    extern __shared__ __align__(16) uint32_t wolff_smem[];
    __shared__ uint32_t s_tail, s_b0;
    __shared__ long long s_acc[kWolffThreads / 32];
    if ((int)blockIdx.x >= sw.n) return;
    const uint32_t lat = blockIdx.x;
    const SwLat d = sw.lat[lat];
    const uint32_t L = d.L, wn = d.wn;
    if ((L <= kWolffSmemMaxL) != SMEM) return;              // the other kernel takes this lattice
    const uint32_t N = L * L;
    const uint32_t n_words = N / 32;                         // packed words of the lattice
    uint32_t* gwords = st.spins + d.word_off;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    WolffStore<SMEM> S;
    S.L = L;
    S.wn = wn;
    if (SMEM) {
        S.words = wolff_smem;
        S.vis = wolff_smem + n_words;
        S.q16 = reinterpret_cast<uint16_t*>(wolff_smem + 2 * n_words);
        S.q32 = nullptr;
        for (uint32_t i = tid; i < n_words; i += kWolffThreads) {
            S.words[i] = gwords[i];
            S.vis[i] = 0u;
        }
    } else {
        S.words = gwords;
        S.vis = sw.coins + d.site_off / 32;                 // zero between steps
        S.q32 = sw.label + d.site_off;                       // up to L^2 sites
        S.q16 = nullptr;
    }
    __syncthreads();
    const unsigned long long t0 = st.ctl->t;
    for (long long step = 0; step < n_steps; ++step) {
        const uint32_t t = (uint32_t)(t0 + (unsigned long long)step);
        if (tid == 0) {
            const uint32_t r = philox(0u, t, d.sim, kPhaseWolffSeed, d.key0, d.key1).x;
            const uint32_t p0 = (uint32_t)(((uint64_t)r * N) >> 32);
            s_b0 = S.spin(p0 % L, p0 / L);
            S.put(0, p0);
            S.claim(p0);
            s_tail = 1;
        }
        __syncthreads();
        const uint32_t b0 = s_b0;
        uint32_t head = 0, tail = 1;
        // the growth, level by level
        for (uint32_t level = 0; level < N && head < tail; ++level) {
            for (uint32_t k = head + tid; k < tail; k += kWolffThreads) {
                const uint32_t p = S.get(k);
                const uint32_t y = p / L, x = p - y * L;
                const uint32_t xr = (x + 1 == L) ? 0u : x + 1, xl = (x == 0) ? L - 1 : x - 1;
                const uint32_t yd = (y + 1 == L) ? 0u : y + 1, yu = (y == 0) ? L - 1 : y - 1;
#pragma unroll
                for (int n = 0; n < 4; ++n) {                // right, left, down, up
                    const uint32_t vx = n == 0 ? xr : (n == 1 ? xl : x), vy = n == 2 ? yd : (n == 3 ? yu : y);
                    const uint32_t v = vy * L + vx;
                    if (S.spin(vx, vy) != b0) continue;
                    if (S.visited(v)) continue;              // already claimed (decided by claim below)
                    // the bond's owner: this site for right / down, the neighbour for left / up
                    const uint32_t owner = (n == 0 || n == 2) ? p : v, dir = (n < 2) ? 0u : 1u;
                    const uint4 r4 = philox(owner >> 1, t, d.sim, kPhaseWolffBond, d.key0, d.key1);
                    // lane 2 (owner & 1) + dir, by two-way selects
                    const uint32_t r = (owner & 1u) ? (dir ? r4.w : r4.z) : (dir ? r4.y : r4.x);
                    if (r >= d.thr) continue;
                    if (S.claim(v)) S.put(atomicAdd(&s_tail, 1u), v);
                }
            }
            __syncthreads();
            head = tail;
            tail = s_tail;
            __syncthreads();          // every thread has read the tail before the next level grows it
        }
        // energy change: 2 * sum over bonds leaving the cluster of sigma_0 sigma_v
        long long acc = 0;
        for (uint32_t k = tid; k < tail; k += kWolffThreads) {
            const uint32_t p = S.get(k);
            const uint32_t y = p / L, x = p - y * L;
            const uint32_t xr = (x + 1 == L) ? 0u : x + 1, xl = (x == 0) ? L - 1 : x - 1;
            const uint32_t yd = (y + 1 == L) ? 0u : y + 1, yu = (y == 0) ? L - 1 : y - 1;
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const uint32_t vx = n == 0 ? xr : (n == 1 ? xl : x), vy = n == 2 ? yd : (n == 3 ? yu : y);
                if (S.visited(vy * L + vx)) continue;
                acc += (S.spin(vx, vy) == b0) ? 1 : -1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) s_acc[warp] = acc;
        __syncthreads();
        // flips and visited bits cleared
        for (uint32_t k = tid; k < tail; k += kWolffThreads) {
            const uint32_t p = S.get(k);
            const uint32_t y = p / L, x = p - y * L;
            S.flip(x, y);
            S.unclaim(p);
        }
        if (tid == 0) {
            long long de = 0;
            for (int w = 0; w < kWolffThreads / 32; ++w) de += s_acc[w];
            const long long E = st.obs[2 * lat] + 2 * de;
            const long long M = st.obs[2 * lat + 1] + (b0 ? 2ll : -2ll) * (long long)tail;
            record_em(st, lat, L, E, M, t0 + (unsigned long long)step);
        }
        __syncthreads();
    }
    if (SMEM)
        for (uint32_t i = tid; i < n_words; i += kWolffThreads) gwords[i] = S.words[i];
}

}  // namespace

cudaError_t launch_sw_clusters(const DevState& st, const SwState& sw, cudaStream_t stream) {
    if (sw.n <= 0 || sw.total_tiles == 0) return cudaSuccess;
    sw_local_kernel<<<(sw.total_tiles + kTilesPerBlock - 1) / kTilesPerBlock, kSwThreads, 0, stream>>>(st, sw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t edge_threads = (uint64_t)sw.total_tiles * kEdgeSites;
    sw_merge_kernel<<<(unsigned)((edge_threads + 255) / 256), 256, 0, stream>>>(st, sw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t words = (uint64_t)sw.total_tiles * kWordsPerTile;
    sw_resolve_kernel<<<(unsigned)((words + 255) / 256), 256, 0, stream>>>(st, sw);
    return cudaGetLastError();
}

cudaError_t launch_wolff_clusters(const DevState& st, const SwState& sw, cudaStream_t stream) {
    if (sw.n <= 0 || sw.total_tiles == 0 || !sw.seed_root) return cudaErrorInvalidValue;
    sw_local_kernel<<<(sw.total_tiles + kTilesPerBlock - 1) / kTilesPerBlock, kSwThreads, 0, stream>>>(st, sw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t edge_threads = (uint64_t)sw.total_tiles * kEdgeSites;
    sw_merge_kernel<<<(unsigned)((edge_threads + 255) / 256), 256, 0, stream>>>(st, sw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wolff_seed_kernel<<<(sw.n + 127) / 128, 128, 0, stream>>>(st, sw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t words = (uint64_t)sw.total_tiles * kWordsPerTile;
    sw_resolve_kernel<<<(unsigned)((words + 255) / 256), 256, 0, stream>>>(st, sw);
    return cudaGetLastError();
}

cudaError_t launch_sw_compress(const SwState& sw, cudaStream_t stream) {
    if (sw.n <= 0 || sw.total_tiles == 0) return cudaSuccess;
    const uint64_t sites = (uint64_t)sw.total_tiles * kTileSites;
    sw_compress_kernel<<<(unsigned)((sites + 255) / 256), 256, 0, stream>>>(sw, sites);
    return cudaGetLastError();
}

cudaError_t launch_sw_flip(const DevState& st, const SwState& sw, cudaStream_t stream) {
    if (sw.n <= 0 || sw.total_tiles == 0) return cudaSuccess;
    const uint64_t pairs = (uint64_t)sw.total_tiles * kPairsPerTile;
    sw_flip_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, stream>>>(st, sw);
    return cudaGetLastError();
}

cudaError_t launch_sw_record(const DevState& st, int n_lat, cudaStream_t stream) {
    if (n_lat <= 0) return cudaSuccess;
    sw_record_kernel<<<1, 256, 0, stream>>>(st, n_lat);
    return cudaGetLastError();
}

cudaError_t launch_wolff(const DevState& st, const SwState& sw, int64_t n_steps, uint32_t max_small_L, bool any_large,
                         cudaStream_t stream) {
    if (sw.n <= 0 || n_steps <= 0) return cudaSuccess;
    if (max_small_L > 0) {     // lattices with L <= kWolffSmemMaxL, in shared memory
        const size_t smem = (size_t)max_small_L * max_small_L / 32 * 2 * 4 + (size_t)max_small_L * max_small_L * 2;
        cudaError_t e = cudaFuncSetAttribute(wolff_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        wolff_kernel<true><<<sw.n, kWolffThreads, smem, stream>>>(st, sw, (long long)n_steps);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (any_large) {           // the others, with the queue and visited bits in the scratch
        wolff_kernel<false><<<sw.n, kWolffThreads, 0, stream>>>(st, sw, (long long)n_steps);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

uint32_t wolff_smem_max_L() { return kWolffSmemMaxL; }

}  // namespace ising
