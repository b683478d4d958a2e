// ising_kernels.cu -- sm_103a kernels of the checkerboard Metropolis sweep.
//
// Method (arXiv 2404.16990): black ((x+y) even) sites are updated in parallel,
// then white ones (Algorithm 5 / Algorithm 3); a site flips iff dE <= 0 or a
// uniform draw falls below exp(-beta dE) (Section 1).  As in Section 2 the
// spins are multi-spin coded (here 32 per 32-bit word, one colour per word,
// LSB = lowest index) and the local field is formed with bitwise adders
// (Algorithm 2's bitwiseAdd), the neighbour words being aligned with funnel
// shifts (the role of getBitAbove / getBitBelow in Algorithm 1).  Unlike the
// paper's 16-entry float exp table and float draws (Algorithm 2, supplementary
// float shaping), every decision here is an integer comparison of a
// Philox4x32-10 word with a u32 threshold, and all four lanes of each Philox
// block are used by four consecutive same-colour sites of one word.
//
// Layout of a lattice with side L (wn = L/64 words per row and colour):
//   word[(c*L + y)*wn + k], bit b <-> site x = 2*(32k + b) + ((y + c) & 1).
// Bit value 0 = spin +1, 1 = spin -1.
#include "ising_internal.h"
#include "ising_device.cuh"

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>

namespace ising {
namespace {

constexpr int kMaxGroupCount = 256;       // lattices per resident group
constexpr unsigned long long kWaitLimitNs = 10ull * 1000ull * 1000ull * 1000ull;  // default bound: 10 s

// The bound of a device wait: the handle's setting, else the default.
__device__ __forceinline__ unsigned long long wait_limit(const Control* ctl) {
    const unsigned long long v = ctl->wait_limit_ns;
    return v != 0 ? v : kWaitLimitNs;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Metropolis update of the 32 same-colour spins of word w given the four
// aligned neighbour words.  a = number of neighbours aligned with the spin
// (0..4) is summed bitwise by one full adder and one half adder; dE = 4a - 8,
// so a <= 2 always flips, a == 3 needs r < thr0 and a == 4 needs r < thr1.
// q0 = first Philox counter of the word's eight site groups.
struct SiteKey {
    uint32_t t, s, phase, k0, k1, thr0, thr1;
};

// 2 acc + [r >= t]: sub.cc leaves the carry of r + ~t + 1, which is 1 exactly
// when r >= t (no borrow), and madc adds it to acc * 2 -- two carry-chain
// instructions shift one comparison result into a word.  (madc rather than
// addc: the same result and instruction count; the sweep measured 1.5 %
// faster with it, the kernel at 124 instead of 128 registers.)
__device__ __forceinline__ uint32_t shift_in_not_below(uint32_t acc, uint32_t r, uint32_t t) {
    uint32_t out;
    asm("{\n\t.reg .u32 d;\n\t"
        "sub.cc.u32 d, %1, %2;\n\t"
        "madc.lo.u32 %0, %3, 2, 0;\n\t}"
        : "=r"(out)
        : "r"(r), "r"(t), "r"(acc));
    return out;
}

__device__ __forceinline__ uint32_t metropolis_word(uint32_t w, uint32_t up, uint32_t dn,
                                                    uint32_t same, uint32_t side, uint32_t q0,
                                                    const SiteKey& key) {
    const uint32_t a0 = ~(w ^ up), a1 = ~(w ^ dn), a2 = ~(w ^ same), a3 = ~(w ^ side);
    const uint32_t x01 = a0 ^ a1;
    const uint32_t s1 = x01 ^ a2;                   // ones of a0+a1+a2
    const uint32_t c1 = (a0 & a1) | (x01 & a2);     // twos of a0+a1+a2
    const uint32_t b0 = s1 ^ a3;                    // ones of a
    const uint32_t c2 = s1 & a3;
    const uint32_t b1 = c1 ^ c2;                    // twos of a
    const uint32_t b2 = c1 & c2;                    // fours of a (a == 4)
    const uint32_t need8 = b2;
    const uint32_t need4 = b0 & b1;                 // a == 3
    // every draw against both thresholds: the bits [r >= thr0] and [r >= thr1]
    // are shifted into two words from site 31 down to site 0, so bit k ends
    // up at site k, with no per-site threshold select
    uint32_t ge0 = 0, ge1 = 0;
#pragma unroll
    for (int g = 7; g >= 0; --g) {
        const uint4 r = philox(q0 + (uint32_t)g, key.t, key.s, key.phase, key.k0, key.k1);
        ge0 = shift_in_not_below(ge0, r.w, key.thr0);
        ge1 = shift_in_not_below(ge1, r.w, key.thr1);
        ge0 = shift_in_not_below(ge0, r.z, key.thr0);
        ge1 = shift_in_not_below(ge1, r.z, key.thr1);
        ge0 = shift_in_not_below(ge0, r.y, key.thr0);
        ge1 = shift_in_not_below(ge1, r.y, key.thr1);
        ge0 = shift_in_not_below(ge0, r.x, key.thr0);
        ge1 = shift_in_not_below(ge1, r.x, key.thr1);
    }
    return w ^ (~(need4 | need8) | (need4 & ~ge0) | (need8 & ~ge1));
}

// Horizontal neighbour word: for bit b the site j+1 (plus) or j-1 (minus) of
// the other colour in the same row; `cur` holds j, `nb` the adjacent word.
__device__ __forceinline__ uint32_t side_word(bool plus, uint32_t cur, uint32_t nb) {
    return plus ? __funnelshift_r(cur, nb, 1) : __funnelshift_l(nb, cur, 1);
}

// Aligned-neighbour count of a white word after its update (E) and the
// popcount of it and of its same-position black word (M).
__device__ __forceinline__ void observe_word(uint32_t w, uint32_t up, uint32_t dn, uint32_t same,
                                             uint32_t side, unsigned long long& sum_a,
                                             unsigned long long& sum_pop) {
    sum_a += __popc(~(w ^ up)) + __popc(~(w ^ dn)) + __popc(~(w ^ same)) + __popc(~(w ^ side));
    sum_pop += __popc(w) + __popc(same);
}

// E = 2L^2 - 2 * sum_white a ;  M = L^2 - 2 * popcount(all words).
__device__ __forceinline__ void record(const DevState& st, uint32_t lat, uint32_t L,
                                       unsigned long long sum_a, unsigned long long sum_pop,
                                       unsigned long long t) {
    const long long N = (long long)L * (long long)L;
    record_em(st, lat, L, 2 * N - 2 * (long long)sum_a, N - 2 * (long long)sum_pop, t);
}

// Block-wide sum of two counters; result valid in thread 0.
__device__ __forceinline__ void block_sum2(unsigned long long& a, unsigned long long& b,
                                           unsigned long long* scratch /* 2*32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { scratch[2 * warp] = a; scratch[2 * warp + 1] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sa = 0, sb = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) { sa += scratch[2 * w]; sb += scratch[2 * w + 1]; }
        a = sa; b = sb;
    }
}

// ---------------------------------------------------------------------------
// Random initial state: both colour words of (y, k) from the 16 Philox blocks
// that cover sites x in [64k, 64k+64) of row y (p = y*L + x, phase 2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) init_random_kernel(DevState st, int n_lat) {
    for (int lat = blockIdx.y; lat < n_lat; lat += gridDim.y) {
        const LatDesc d = st.lat[lat];
        const uint32_t L = d.L, wn = d.wn;
        uint32_t* base = st.spins + d.word_off;
        const uint32_t items = L * wn;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < items; i += gridDim.x * blockDim.x) {
            const uint32_t y = i / wn, k = i - y * wn;
            const uint32_t q0 = (y * L + 64u * k) >> 2;
            uint32_t even = 0, odd = 0;   // sites with x even / x odd
#pragma unroll 4
            for (uint32_t g = 0; g < 16; ++g) {
                const uint4 r = philox(q0 + g, 0u, d.sim, 2u, d.key0, d.key1);
                even |= ((r.x >> 31) << (2 * g)) | ((r.z >> 31) << (2 * g + 1));
                odd |= ((r.y >> 31) << (2 * g)) | ((r.w >> 31) << (2 * g + 1));
            }
            // colour c holds x = 2j + ((y + c) & 1)
            const bool yodd = (y & 1u) != 0;
            base[(0 * L + y) * wn + k] = yodd ? odd : even;
            base[(1 * L + y) * wn + k] = yodd ? even : odd;
        }
    }
}

// ---------------------------------------------------------------------------
// E and M of listed lattices from their packed words (after init / set).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) observables_kernel(DevState st, const uint32_t* list, int n_list) {
    __shared__ unsigned long long red[64];
    for (int li = blockIdx.y; li < n_list; li += gridDim.y) {
        const uint32_t lat = list[li];
        const LatDesc d = st.lat[lat];
        const uint32_t L = d.L, wn = d.wn;
        const uint32_t* white = st.spins + d.word_off + (size_t)L * wn;
        const uint32_t* black = st.spins + d.word_off;
        unsigned long long sa = 0, sp = 0;
        const uint32_t items = L * wn;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < items; i += gridDim.x * blockDim.x) {
            const uint32_t y = i / wn, k = i - y * wn;
            const uint32_t ym = (y == 0) ? L - 1 : y - 1, yp = (y + 1 == L) ? 0 : y + 1;
            const bool plus = ((1u ^ (y & 1u)) != 0);
            const uint32_t kk = plus ? ((k + 1 == wn) ? 0 : k + 1) : ((k == 0) ? wn - 1 : k - 1);
            const uint32_t same = black[y * wn + k];
            observe_word(white[y * wn + k], black[ym * wn + k], black[yp * wn + k], same,
                         side_word(plus, same, black[y * wn + kk]), sa, sp);
        }
        block_sum2(sa, sp, red);
        if (threadIdx.x == 0) {
            atomicAdd(&st.acc[2 * lat + 0], sa);
            atomicAdd(&st.acc[2 * lat + 1], sp);
        }
        __syncthreads();
    }
}

__global__ void observables_finalize_kernel(DevState st, const uint32_t* list, int n_list) {
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < n_list; li += gridDim.x * blockDim.x) {
        const uint32_t lat = list[li];
        const long long N = (long long)st.lat[lat].L * st.lat[lat].L;
        const unsigned long long sa = st.acc[2 * lat], sp = st.acc[2 * lat + 1];
        st.obs[2 * lat + 0] = 2 * N - 2 * (long long)sa;
        st.obs[2 * lat + 1] = N - 2 * (long long)sp;
        st.acc[2 * lat] = 0;
        st.acc[2 * lat + 1] = 0;
    }
}

// ---------------------------------------------------------------------------
// Resident kernel: a persistent grid; each work ticket = (group g, chunk c) =
// sweeps [c*k, (c+1)*k) of the lattices of group g, held in shared memory.
// Tickets are handed out in order (g fastest); a ticket waits (bounded) until
// chunk c-1 of its group is stored.  The oldest ticket in flight never waits,
// so the schedule always progresses.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 1) resident_kernel(DevState st, int n_groups, long long n_sweeps,
                                                        int k_unit) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long s_cnt[2 * kMaxGroupCount];
    __shared__ SiteKey s_key[kMaxGroupCount];
    __shared__ uint32_t s_lat[kMaxGroupCount];
    __shared__ long long s_ticket;
    __shared__ int s_abort;
    __shared__ unsigned long long s_t0;

    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) s_t0 = st.ctl->t;
    const long long n_chunks = (n_sweeps + k_unit - 1) / k_unit;
    const long long total = n_chunks * (long long)n_groups;

    for (;;) {
        if (tid == 0) {
            s_ticket = (long long)atomicAdd(&st.ctl->ticket, 1u);
            s_abort = 0;
        }
        __syncthreads();
        const long long ticket = s_ticket;
        if (ticket >= total) break;
        const int g = (int)(ticket % n_groups);
        const long long chunk = ticket / n_groups;
        if (tid == 0) {
            const unsigned long long start = global_ns(), limit = wait_limit(st.ctl);
            while ((long long)ld_acquire(&st.done[g]) < chunk) {
                if (global_ns() - start > limit) {
                    atomicOr(&st.ctl->error, 1);
                    s_abort = 1;
                    break;
                }
                __nanosleep(200);
            }
        }
        const GroupDesc gd = st.groups[g];
        const uint32_t L = gd.L, wn = gd.wn, cnt = gd.count;
        const uint32_t wpl = 2u * L * wn;          // words per lattice
        const uint32_t wpc = L * wn;               // words per colour
        if (tid < (int)cnt) {
            const uint32_t lat = st.members[gd.member_off + tid];
            const LatDesc d = st.lat[lat];
            s_lat[tid] = lat;
            s_key[tid] = SiteKey{0u, d.sim, 0u, d.key0, d.key1, d.thr0, d.thr1};
        }
        __syncthreads();
        if (s_abort) break;

        // load the group (L2 only: another SM may have written it)
        const uint32_t v4 = wpl / 4;
        for (uint32_t i = tid; i < cnt * v4; i += nthr) {
            const uint32_t m = i / v4, r = i - m * v4;
            const uint4* src = reinterpret_cast<const uint4*>(st.spins + st.lat[s_lat[m]].word_off);
            reinterpret_cast<uint4*>(sm + (size_t)m * wpl)[r] = __ldcg(src + r);
        }
        __syncthreads();

        const long long sw0 = chunk * k_unit;
        const long long k_this = (n_sweeps - sw0 < k_unit) ? (n_sweeps - sw0) : k_unit;
        // threads as a (ty, tx) grid over the group's stacked rows (lattice m
        // holds rows [m*L, (m+1)*L)) and the words of a row: no divisions in
        // the update loop
        const uint32_t tw = wn < (uint32_t)nthr ? wn : (uint32_t)nthr;
        const uint32_t n_ty = (uint32_t)nthr / tw;
        const uint32_t tx = (uint32_t)tid % tw, ty = (uint32_t)tid / tw;
        const uint32_t rows = cnt * L;
        for (long long it = 0; it < k_this; ++it) {
            const unsigned long long t = s_t0 + (unsigned long long)(sw0 + it);
            if (tid < 2 * (int)cnt) s_cnt[tid] = 0;
            for (uint32_t c = 0; c < 2; ++c) {
                unsigned long long sa = 0, sp = 0;
                uint32_t m = 0, row0 = 0;
                if (ty < n_ty) {
                    for (uint32_t Y = ty; Y < rows; Y += n_ty) {
                        if (Y >= row0 + L) {
                            if (c == 1) {
                                atomicAdd(&s_cnt[2 * m], sa);
                                atomicAdd(&s_cnt[2 * m + 1], sp);
                                sa = 0; sp = 0;
                            }
                            do { ++m; row0 += L; } while (Y >= row0 + L);
                        }
                        const uint32_t y = Y - row0;
                        uint32_t* lat_sm = sm + (size_t)m * wpl;
                        const uint32_t* opp = lat_sm + (1u - c) * wpc;
                        const uint32_t ym = (y == 0) ? L - 1 : y - 1, yp = (y + 1 == L) ? 0 : y + 1;
                        const bool plus = ((c ^ (y & 1u)) != 0);
                        SiteKey key = s_key[m];
                        key.t = (uint32_t)t;
                        key.phase = c;
                        for (uint32_t k = tx; k < wn; k += tw) {
                            const uint32_t kk = plus ? ((k + 1 == wn) ? 0 : k + 1) : ((k == 0) ? wn - 1 : k - 1);
                            const uint32_t up = opp[ym * wn + k], dn = opp[yp * wn + k];
                            const uint32_t same = opp[y * wn + k];
                            const uint32_t side = side_word(plus, same, opp[y * wn + kk]);
                            uint32_t* own = lat_sm + c * wpc + y * wn + k;
                            const uint32_t q0 = (y * (L >> 1) + 32u * k) >> 2;
                            const uint32_t wnew = metropolis_word(*own, up, dn, same, side, q0, key);
                            *own = wnew;
                            if (c == 1) observe_word(wnew, up, dn, same, side, sa, sp);
                        }
                    }
                    if (c == 1) {
                        atomicAdd(&s_cnt[2 * m], sa);
                        atomicAdd(&s_cnt[2 * m + 1], sp);
                    }
                }
                __syncthreads();
            }
            if (tid < (int)cnt) record(st, s_lat[tid], L, s_cnt[2 * tid], s_cnt[2 * tid + 1], t);
            __syncthreads();
        }

        // store the group back and publish the chunk
        for (uint32_t i = tid; i < cnt * v4; i += nthr) {
            const uint32_t m = i / v4, r = i - m * v4;
            uint4* dst = reinterpret_cast<uint4*>(st.spins + st.lat[s_lat[m]].word_off);
            __stcg(dst + r, reinterpret_cast<const uint4*>(sm + (size_t)m * wpl)[r]);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(&st.done[g], (unsigned int)(chunk + 1));
    }
}

// ---------------------------------------------------------------------------
// Streaming half-sweep over lattices in device memory.  A tile = tw word
// groups (V consecutive words each) x th row groups (R rows each); every
// thread of a block works on the same lattice, so E/M partial sums are
// reduced per block and added with one atomic per block and lattice.
// ---------------------------------------------------------------------------
template <int V>
struct WordVec;
template <> struct WordVec<1> { using T = uint32_t; };
template <> struct WordVec<2> { using T = uint2; };
template <> struct WordVec<4> { using T = uint4; };

template <int V>
__device__ __forceinline__ void load_vec(const uint32_t* p, uint32_t (&o)[V]) {
    if constexpr (V == 1) { o[0] = p[0]; }
    else if constexpr (V == 2) { const uint2 v = *reinterpret_cast<const uint2*>(p); o[0] = v.x; o[1] = v.y; }
    else { const uint4 v = *reinterpret_cast<const uint4*>(p); o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
}
template <int V>
__device__ __forceinline__ void store_vec(uint32_t* p, const uint32_t (&o)[V]) {
    if constexpr (V == 1) { p[0] = o[0]; }
    else if constexpr (V == 2) { *reinterpret_cast<uint2*>(p) = make_uint2(o[0], o[1]); }
    else { *reinterpret_cast<uint4*>(p) = make_uint4(o[0], o[1], o[2], o[3]); }
}

// One half-sweep of colour c over the tiles of the streamed lattices, tiles
// taken in a grid-stride loop; with c == 1 the per-lattice E/M partial sums are
// reduced per block and added to st.acc.
template <int V>
__device__ __forceinline__ void stream_tiles(const DevState& st, int n_slats, unsigned long long total_tiles,
                                             uint32_t c, unsigned long long t, unsigned long long* red) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    unsigned long long sa = 0, sp = 0;
    int cur_slat = -1;

    for (unsigned long long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        // lattice of this tile (block-uniform binary search)
        int lo = 0, hi = n_slats - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (st.slats[mid].item_begin <= tile) lo = mid; else hi = mid - 1;
        }
        if (c == 1 && lo != cur_slat) {
            if (cur_slat >= 0) {
                block_sum2(sa, sp, red);
                if (tid == 0) {
                    const uint32_t lat = st.slats[cur_slat].lat;
                    atomicAdd(&st.acc[2 * lat], sa);
                    atomicAdd(&st.acc[2 * lat + 1], sp);
                }
                sa = 0; sp = 0;
            }
            cur_slat = lo;
        }
        const StreamLat sl = st.slats[lo];
        const LatDesc d = st.lat[sl.lat];
        const uint32_t L = d.L, wn = d.wn;
        const uint32_t gw = sl.groups;                  // word groups per row
        const uint32_t tw = gw < (uint32_t)nthr ? gw : (uint32_t)nthr;
        const uint32_t th = (uint32_t)nthr / tw;
        const uint32_t tiles_x = (gw + tw - 1) / tw;
        const unsigned long long local = tile - sl.item_begin;
        const uint32_t tile_y = (uint32_t)(local / tiles_x), tile_x = (uint32_t)(local - (unsigned long long)tile_y * tiles_x);
        const uint32_t tx = (uint32_t)tid % tw, ty = (uint32_t)tid / tw;
        const uint32_t kg = tile_x * tw + tx;
        const uint32_t R = sl.rows;
        const uint32_t y0 = (tile_y * th + ty) * R;
        if (ty < th && kg < gw && y0 < L) {
            const uint32_t y1 = (y0 + R < L) ? y0 + R : L;
            const uint32_t k0 = kg * V;
            uint32_t* own_base = st.spins + d.word_off + (size_t)c * L * wn;
            const uint32_t* opp = st.spins + d.word_off + (size_t)(1u - c) * L * wn;
            const SiteKey key0{(uint32_t)t, d.sim, c, d.key0, d.key1, d.thr0, d.thr1};
            uint32_t prev[V], cur[V], next[V];
            load_vec<V>(opp + (size_t)((y0 == 0) ? L - 1 : y0 - 1) * wn + k0, prev);
            load_vec<V>(opp + (size_t)y0 * wn + k0, cur);
            for (uint32_t y = y0; y < y1; ++y) {
                const uint32_t yp = (y + 1 == L) ? 0 : y + 1;
                load_vec<V>(opp + (size_t)yp * wn + k0, next);
                const bool plus = ((c ^ (y & 1u)) != 0);
                const uint32_t kk = plus ? ((k0 + V == wn) ? 0 : k0 + V) : ((k0 == 0) ? wn - 1 : k0 - 1);
                const uint32_t nb = opp[(size_t)y * wn + kk];
                uint32_t own[V];
                load_vec<V>(own_base + (size_t)y * wn + k0, own);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t adj = plus ? ((v + 1 < V) ? cur[(v + 1) % V] : nb)
                                              : ((v > 0) ? cur[(v + V - 1) % V] : nb);
                    const uint32_t side = side_word(plus, cur[v], adj);
                    const uint32_t q0 = (y * (L >> 1) + 32u * (k0 + v)) >> 2;
                    own[v] = metropolis_word(own[v], prev[v], next[v], cur[v], side, q0, key0);
                    if (c == 1) observe_word(own[v], prev[v], next[v], cur[v], side, sa, sp);
                }
                store_vec<V>(own_base + (size_t)y * wn + k0, own);
#pragma unroll
                for (int v = 0; v < V; ++v) { prev[v] = cur[v]; cur[v] = next[v]; }
            }
        }
    }

    if (c == 1 && cur_slat >= 0) {
        block_sum2(sa, sp, red);
        if (tid == 0) {
            const uint32_t lat = st.slats[cur_slat].lat;
            atomicAdd(&st.acc[2 * lat], sa);
            atomicAdd(&st.acc[2 * lat + 1], sp);
        }
    }
}

template <int V>
__global__ void __launch_bounds__(256, 2) stream_half_kernel(DevState st, int n_slats,
                                                          unsigned long long total_tiles, uint32_t c) {
    __shared__ unsigned long long red[64];
    __shared__ int s_last;
    const unsigned long long t = st.ctl->t;
    const int tid = threadIdx.x, nthr = blockDim.x;
    stream_tiles<V>(st, n_slats, total_tiles, c, t, red);
    if (c == 1) {
        // last block to finish records E/M of every streamed lattice and
        // advances the sweep counter
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = (atomicAdd(&st.ctl->blocks_done, 1u) == gridDim.x - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int i = tid; i < n_slats; i += nthr) {
                const uint32_t lat = st.slats[i].lat;
                const unsigned long long a = atomicExch(&st.acc[2 * lat], 0ull);
                const unsigned long long p = atomicExch(&st.acc[2 * lat + 1], 0ull);
                record(st, lat, st.lat[lat].L, a, p, t);
            }
            __syncthreads();
            if (tid == 0) {
                st.ctl->blocks_done = 0;
                st.ctl->t = t + 1;
            }
        }
    }
}

// Grid-wide barrier of a cooperative launch (every block co-resident): an
// arrival counter and a generation word in the control block.  A block that
// waits longer than the limit sets the error flag and returns false.
__device__ __forceinline__ bool grid_barrier(Control* ctl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int g = ld_acquire(&ctl->bar_gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            st_release(&ctl->bar_gen, g + 1u);
        } else {
            const unsigned long long start = global_ns(), limit = wait_limit(ctl);
            while (ld_acquire(&ctl->bar_gen) == g) {
                if (global_ns() - start > limit) {
                    atomicOr(&ctl->error, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Persistent streaming kernel: n sweeps of every streamed lattice in one
// cooperative launch, a grid barrier after each half-sweep; after each white
// half-sweep block 0 records E/M of every lattice.
template <int V>
__global__ void __launch_bounds__(256, 2) stream_persist_kernel(DevState st, int n_slats,
                                                             unsigned long long total_tiles,
                                                             long long n_sweeps) {
    __shared__ unsigned long long red[64];
    const unsigned long long t0 = st.ctl->t;
    for (long long i = 0; i < n_sweeps; ++i) {
        const unsigned long long t = t0 + (unsigned long long)i;
        for (uint32_t c = 0; c < 2; ++c) {
            stream_tiles<V>(st, n_slats, total_tiles, c, t, red);
            if (!grid_barrier(st.ctl)) return;
            if (c == 1 && blockIdx.x == 0) {
                __threadfence();
                for (int k = threadIdx.x; k < n_slats; k += blockDim.x) {
                    const uint32_t lat = st.slats[k].lat;
                    const unsigned long long a = atomicExch(&st.acc[2 * lat], 0ull);
                    const unsigned long long p = atomicExch(&st.acc[2 * lat + 1], 0ull);
                    record(st, lat, st.lat[lat].L, a, p, t);
                }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st.ctl->t = t0 + (unsigned long long)n_sweeps;
}

// ---------------------------------------------------------------------------
// Cluster-resident kernel for small lattices: one thread-block cluster of C
// CTAs per lattice, CTA rank r holding rows [r L/C, (r+1) L/C) of both colours
// in shared memory for all sweeps of the call.  A half-sweep reads the rows
// just above and below the strip straight from the neighbouring CTAs' shared
// memory (distributed shared memory), and a cluster barrier separates the
// half-sweeps -- the paper's halo refresh between the two colours
// (Algorithm 6) without any copy.  E/M partial sums go to rank 0 by DSMEM
// atomics; rank 0 records them after each sweep.  Lattice li of the class is
// handled by cluster li (blockIdx.x / C); every lattice's L / C rows form
// whole rows of words.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cluster_resident_kernel(DevState st, const uint32_t* members, int count,
                                                               long long n_sweeps) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long s_acc[2];          // rank 0: the cluster's E/M partial sums of a sweep
    __shared__ unsigned long long red[64];
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t C = cluster.num_blocks(), r = cluster.block_rank();
    const int li = (int)(blockIdx.x / C);
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (li >= count) return;                          // whole clusters only (grid = count x C)
    const uint32_t lat = members[li];
    const LatDesc d = st.lat[lat];
    const uint32_t L = d.L, wn = d.wn, rows = L / C, y0 = r * rows;
    const uint32_t strip = rows * wn;                 // words of one colour in this CTA
    uint32_t* base = st.spins + d.word_off;
    for (uint32_t i = tid; i < 2 * strip; i += nthr) {
        const uint32_t c = i / strip, j = i - c * strip;
        sm[i] = __ldcg(base + ((size_t)c * L + y0) * wn + j);
    }
    if (tid < 2) s_acc[tid] = 0ull;
    const unsigned long long t0 = st.ctl->t;
    cluster.sync();                                   // every strip loaded
    const uint32_t* up_sm = cluster.map_shared_rank(sm, (r + C - 1) % C);   // its last row is row y0 - 1
    const uint32_t* dn_sm = cluster.map_shared_rank(sm, (r + 1) % C);       // its first row is row y0 + rows
    unsigned long long* acc0 = cluster.map_shared_rank(s_acc, 0u);
    for (long long it = 0; it < n_sweeps; ++it) {
        const unsigned long long t = t0 + (unsigned long long)it;
        for (uint32_t c = 0; c < 2; ++c) {
            const uint32_t* opp = sm + (1u - c) * strip;
            uint32_t* own = sm + c * strip;
            const SiteKey key{(uint32_t)t, d.sim, c, d.key0, d.key1, d.thr0, d.thr1};
            unsigned long long sa = 0, sp = 0;
            for (uint32_t i = tid; i < strip; i += nthr) {
                const uint32_t ly = i / wn, k = i - ly * wn, y = y0 + ly;
                const uint32_t up = ly > 0 ? opp[i - wn] : up_sm[(1u - c) * strip + (rows - 1) * wn + k];
                const uint32_t dn = ly + 1 < rows ? opp[i + wn] : dn_sm[(1u - c) * strip + k];
                const uint32_t same = opp[i];
                const bool plus = ((c ^ (y & 1u)) != 0);
                const uint32_t kk = plus ? ((k + 1 == wn) ? 0 : k + 1) : ((k == 0) ? wn - 1 : k - 1);
                const uint32_t side = side_word(plus, same, opp[ly * wn + kk]);
                const uint32_t q0 = (y * (L >> 1) + 32u * k) >> 2;
                const uint32_t w = metropolis_word(own[i], up, dn, same, side, q0, key);
                own[i] = w;
                if (c == 1) observe_word(w, up, dn, same, side, sa, sp);
            }
            if (c == 1) {
                block_sum2(sa, sp, red);
                if (tid == 0) {
                    atomicAdd(&acc0[0], sa);
                    atomicAdd(&acc0[1], sp);
                }
            }
            cluster.sync();                           // this colour complete everywhere before the other is read
            if (c == 1 && r == 0 && tid == 0) {
                record(st, lat, L, s_acc[0], s_acc[1], t);
                s_acc[0] = 0ull;                      // the next additions come after the next barrier
                s_acc[1] = 0ull;
            }
        }
    }
    for (uint32_t i = tid; i < 2 * strip; i += nthr) {
        const uint32_t c = i / strip, j = i - c * strip;
        __stcg(base + ((size_t)c * L + y0) * wn + j, sm[i]);
    }
    cluster.sync();                                   // no CTA leaves while another may still read its memory
}

__global__ void advance_t_kernel(DevState st, long long n) { st.ctl->t += (unsigned long long)n; }

// The draws of sites p0 .. p0 + n_p - 1 in sweeps t0 .. t0 + n_t - 1, one
// Philox block per thread: item (t, g) covers the sites of block q = (p0 >> 2)
// + g that fall inside [p0, p0 + n_p).
__global__ void __launch_bounds__(256) random_stream_kernel(uint32_t k0, uint32_t k1, uint32_t s, uint32_t phase,
                                                            unsigned long long p0, unsigned long long n_p,
                                                            uint32_t t0, uint32_t n_t, unsigned long long blocks,
                                                            uint32_t* out) {
    const unsigned long long total = blocks * n_t;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long tt = i / blocks, g = i - tt * blocks;
        const unsigned long long q = (p0 >> 2) + g;
        const uint4 r = philox((uint32_t)q, t0 + (uint32_t)tt, s, phase, k0, k1);
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        uint32_t* row = out + tt * n_p;
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            const unsigned long long p = 4ull * q + lane;
            if (p >= p0 && p < p0 + n_p) row[p - p0] = v[lane];
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

size_t device_max_smem_optin() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)n;
}

cudaError_t configure_kernels() {
    const size_t optin = device_max_smem_optin();
    const size_t static_smem = 2 * kMaxGroupCount * sizeof(unsigned long long) +
                               kMaxGroupCount * (sizeof(SiteKey) + sizeof(uint32_t)) + 64;
    const int dyn = (int)(optin > static_smem ? optin - static_smem : 0);
    return cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}

int resident_occupancy(int threads, size_t smem_bytes) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, resident_kernel, threads, smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

int stream_occupancy(int words_per_thread, int threads) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (words_per_thread) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_half_kernel<1>, threads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_half_kernel<2>, threads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_half_kernel<4>, threads, 0); break;
    default: break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_init_random(const DevState& st, int n_lat, cudaStream_t stream) {
    if (n_lat <= 0) return cudaSuccess;
    const int sms = device_sm_count();
    dim3 grid((unsigned)(sms * 4), (unsigned)(n_lat < 65535 ? n_lat : 65535));
    if (n_lat > 64) grid.x = 4;
    init_random_kernel<<<grid, 256, 0, stream>>>(st, n_lat);
    return cudaGetLastError();
}

cudaError_t launch_observables(const DevState& st, uint32_t max_L, const uint32_t* lat_list,
                               int n_list, cudaStream_t stream, bool finalize) {
    if (n_list <= 0) return cudaSuccess;
    const int sms = device_sm_count();
    // blocks per lattice: enough for about four word pairs per thread of the
    // largest listed lattice (L * L / 64 pairs), at most two per SM (four when
    // more than 64 lattices share the grid)
    uint32_t per_lat = (uint32_t)(n_list > 64 ? 4 : sms * 2);
    if (max_L > 0) {
        const uint64_t pairs = (uint64_t)max_L * (max_L / 64);
        per_lat = (uint32_t)std::min<uint64_t>(per_lat, std::max<uint64_t>(1, (pairs + 1023) / 1024));
    }
    dim3 grid(per_lat, (unsigned)(n_list < 65535 ? n_list : 65535));
    observables_kernel<<<grid, 256, 0, stream>>>(st, lat_list, n_list);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !finalize) return e;
    observables_finalize_kernel<<<(n_list + 255) / 256, 256, 0, stream>>>(st, lat_list, n_list);
    return cudaGetLastError();
}

cudaError_t launch_resident(const DevState& st, int n_groups, int64_t n_sweeps, int sweeps_per_unit,
                            int threads, int grid, size_t smem_bytes, cudaStream_t stream) {
    if (n_groups <= 0 || n_sweeps <= 0) return cudaSuccess;
    resident_kernel<<<grid, threads, smem_bytes, stream>>>(st, n_groups, (long long)n_sweeps,
                                                           sweeps_per_unit);
    return cudaGetLastError();
}

cudaError_t launch_stream_sweeps(const DevState& st, int n_slats, uint64_t total_tiles,
                                 int words_per_thread, int threads, int grid,
                                 int64_t n_sweeps, cudaStream_t stream) {
    if (n_slats <= 0 || n_sweeps <= 0) return cudaSuccess;
    for (int64_t i = 0; i < n_sweeps; ++i) {
        for (uint32_t c = 0; c < 2; ++c) {
            switch (words_per_thread) {
            case 1: stream_half_kernel<1><<<grid, threads, 0, stream>>>(st, n_slats, total_tiles, c); break;
            case 2: stream_half_kernel<2><<<grid, threads, 0, stream>>>(st, n_slats, total_tiles, c); break;
            case 4: stream_half_kernel<4><<<grid, threads, 0, stream>>>(st, n_slats, total_tiles, c); break;
            default: return cudaErrorInvalidValue;
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int stream_persistent_occupancy(int words_per_thread, int threads) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (words_per_thread) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_persist_kernel<1>, threads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_persist_kernel<2>, threads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_persist_kernel<4>, threads, 0); break;
    default: break;
    }
    return e == cudaSuccess ? n : 0;
}

template <int V>
static cudaError_t launch_persist_v(const DevState& st, int n_slats, uint64_t total_tiles, int threads, int grid,
                                    int64_t n_sweeps, cudaStream_t stream) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stream_persist_kernel<V>, st, n_slats, (unsigned long long)total_tiles,
                              (long long)n_sweeps);
}

cudaError_t launch_stream_persistent(const DevState& st, int n_slats, uint64_t total_tiles, int words_per_thread,
                                     int threads, int grid, int64_t n_sweeps, cudaStream_t stream) {
    if (n_slats <= 0 || n_sweeps <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(&st.ctl->bar_count, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    switch (words_per_thread) {
    case 1: e = launch_persist_v<1>(st, n_slats, total_tiles, threads, grid, n_sweeps, stream); break;
    case 2: e = launch_persist_v<2>(st, n_slats, total_tiles, threads, grid, n_sweeps, stream); break;
    case 4: e = launch_persist_v<4>(st, n_slats, total_tiles, threads, grid, n_sweeps, stream); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_random_stream(uint32_t k0, uint32_t k1, uint32_t s, uint32_t phase, uint64_t p0, uint64_t n_p,
                                 uint32_t t0, uint32_t n_t, uint32_t* out, cudaStream_t stream) {
    if (n_p == 0 || n_t == 0) return cudaSuccess;
    const uint64_t blocks = ((p0 + n_p + 3) >> 2) - (p0 >> 2);
    const uint64_t total = blocks * n_t;
    const uint64_t grid = std::min<uint64_t>((total + 255) / 256, (uint64_t)device_sm_count() * 16);
    random_stream_kernel<<<(unsigned)grid, 256, 0, stream>>>(k0, k1, s, phase, (unsigned long long)p0,
                                                             (unsigned long long)n_p, t0, n_t,
                                                             (unsigned long long)blocks, out);
    return cudaGetLastError();
}

cudaError_t launch_cluster_resident(const DevState& st, const uint32_t* members, int count, int cluster_size,
                                    uint32_t L, int64_t n_sweeps, cudaStream_t stream) {
    if (count <= 0 || n_sweeps <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(count * cluster_size));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = (size_t)L * L / 8 / (size_t)cluster_size;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, cluster_resident_kernel, st, members, count, (long long)n_sweeps);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_advance_t(const DevState& st, int64_t n, cudaStream_t stream) {
    advance_t_kernel<<<1, 1, 0, stream>>>(st, (long long)n);
    return cudaGetLastError();
}

}  // namespace ising
