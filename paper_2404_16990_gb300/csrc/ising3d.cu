// ising3d.cu -- the checkerboard Metropolis sweep on the simple cubic lattice
// (periodic L x L x L, J = 1, h = 0, six nearest neighbours): kernels and the
// ising3d_* entry points of the C ABI.
//
// The paper's Hamiltonian (Section 1) is written for any dimension, with the
// number of neighbours set by the lattice (four in 2D, six in 3D); the sweep
// is the 2D one of Algorithm 5 with one more axis.  Layout (L a multiple of
// 64): word[((c L + z) L + y) (L/64) + k], bit b <-> x = 2 (32 k + b) +
// ((y + z + c) & 1), bit 1 = spin -1.  The y and z neighbours of a word are
// the same word index of the other colour in rows (z, y +- 1) and
// (z +- 1, y); the x neighbours are the same word and a funnel-shifted
// neighbour word of the other colour in the same row.  Aligned neighbours
// a = 0..6 come from a bitsliced adder of six masks (two full adders, then a
// two-bit add); dE = 4a - 12: a <= 3 always flips, a = 4, 5, 6 need r below
// thr[0], thr[1], thr[2].  Draws: Philox4x32-10, counter (p >> 2, t, s,
// phase), lane p & 3, p = (z L + y) (L/2) + (x >> 1) (phase 0/1), and
// p = (z L + y) L + x for the random initial state (phase 2).
#include "../../include/ising.h"
#include "ising_internal.h"
#include "ising_device.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

namespace ising {
namespace {

struct Lat3 {
    uint64_t word_off;     // first word of the lattice
    uint64_t item_begin;   // first word item of the lattice (L^3 / 64 items per colour)
    uint32_t L, wn, sim, key0, key1;
    uint32_t thr[3];       // dE = 4, 8, 12
};

struct Ctl3 {
    unsigned long long t;
    long long trace_cap;
    int measure;
    int pad;
};

struct State3 {
    const Lat3* lat;
    uint32_t* spins;
    unsigned long long* acc;   // [n][2] aligned count (white), popcount
    long long* obs;            // [n][2] E, M
    long long* trace;          // [n][cap][2]
    Ctl3* ctl;
    int n;
    uint64_t items;            // words of one colour over all lattices
};

__device__ __forceinline__ int lattice_of_item(const Lat3* lat, int n, uint64_t item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lat[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// 2 acc + [r >= t] by the carry of r - t, as in the 2D sweep (madc for the
// shift-in: 0.6 % faster at 1024^3, 3-4 % at 256^3 and 512^3).
__device__ __forceinline__ uint32_t shift_in_not_below3(uint32_t acc, uint32_t r, uint32_t t) {
    uint32_t out;
    asm("{\n\t.reg .u32 d;\n\t"
        "sub.cc.u32 d, %1, %2;\n\t"
        "madc.lo.u32 %0, %3, 2, 0;\n\t}"
        : "=r"(out)
        : "r"(r), "r"(t), "r"(acc));
    return out;
}

// Bit planes (b0, b1, b2) of the number of set bits among six masks.
__device__ __forceinline__ void count6(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4,
                                       uint32_t a5, uint32_t& b0, uint32_t& b1, uint32_t& b2) {
    const uint32_t x1 = a0 ^ a1, s1 = x1 ^ a2, c1 = (a0 & a1) | (x1 & a2);   // a0+a1+a2 = s1 + 2 c1
    const uint32_t x2 = a3 ^ a4, s2 = x2 ^ a5, c2 = (a3 & a4) | (x2 & a5);   // a3+a4+a5 = s2 + 2 c2
    b0 = s1 ^ s2;
    const uint32_t k = s1 & s2;                                              // carry into the twos
    b1 = c1 ^ c2 ^ k;
    b2 = (c1 & c2) | (k & (c1 ^ c2));
}

struct Words6 {
    uint32_t w, yl, yh, zl, zh, same, side;
};

// The word of colour c at (z, y, k) and its six neighbour words.
__device__ __forceinline__ Words6 load6(const uint32_t* base, uint32_t L, uint32_t wn, uint32_t c, uint32_t z,
                                        uint32_t y, uint32_t k) {
    const uint32_t o = c ^ 1u;
    const uint32_t ym = (y == 0) ? L - 1 : y - 1, yp = (y + 1 == L) ? 0 : y + 1;
    const uint32_t zm = (z == 0) ? L - 1 : z - 1, zp = (z + 1 == L) ? 0 : z + 1;
    auto at = [&](uint32_t cc, uint32_t zz, uint32_t yy, uint32_t kk) {
        return base[(((size_t)cc * L + zz) * L + yy) * wn + kk];
    };
    Words6 r;
    r.w = at(c, z, y, k);
    r.yl = at(o, z, ym, k);
    r.yh = at(o, z, yp, k);
    r.zl = at(o, zm, y, k);
    r.zh = at(o, zp, y, k);
    r.same = at(o, z, y, k);
    // sites of colour c sit at x = 2j + e, e = (y + z + c) & 1: for e = 1 the
    // other x neighbour is j + 1 of the other colour, for e = 0 it is j - 1
    const bool plus = ((y + z + c) & 1u) != 0;
    const uint32_t kk = plus ? ((k + 1 == wn) ? 0 : k + 1) : ((k == 0) ? wn - 1 : k - 1);
    const uint32_t nb = at(o, z, y, kk);
    r.side = plus ? __funnelshift_r(r.same, nb, 1) : __funnelshift_l(nb, r.same, 1);
    return r;
}

// One half-sweep of colour c over every lattice: one thread per V consecutive
// words of a row (the x neighbours of inner words come from the thread's own
// loads).
template <int V>
__global__ void __launch_bounds__(256) half3d_kernel(State3 st, uint32_t c) {
    const uint32_t t = (uint32_t)st.ctl->t;
    const uint64_t groups = st.items / V;
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < groups;
         item += (uint64_t)gridDim.x * blockDim.x) {
        const Lat3 d = st.lat[lattice_of_item(st.lat, st.n, item * V)];
        const uint32_t L = d.L, wn = d.wn;
        const uint64_t i = item * V - d.item_begin;
        const uint32_t k0 = (uint32_t)(i % wn);
        const uint32_t y = (uint32_t)((i / wn) % L), z = (uint32_t)(i / ((uint64_t)wn * L));
        uint32_t* base = st.spins + d.word_off;
        const uint32_t o = c ^ 1u;
        const uint32_t ym = (y == 0) ? L - 1 : y - 1, yp = (y + 1 == L) ? 0 : y + 1;
        const uint32_t zm = (z == 0) ? L - 1 : z - 1, zp = (z + 1 == L) ? 0 : z + 1;
        auto row = [&](uint32_t cc, uint32_t zz, uint32_t yy) { return base + (((size_t)cc * L + zz) * L + yy) * wn; };
        uint32_t* own = row(c, z, y);
        const uint32_t *sm = row(o, z, y), *yl = row(o, z, ym), *yh = row(o, z, yp), *zl = row(o, zm, y), *zh = row(o, zp, y);
        const bool plus = ((y + z + c) & 1u) != 0;
        const uint32_t kk = plus ? ((k0 + V == wn) ? 0 : k0 + V) : ((k0 == 0) ? wn - 1 : k0 - 1);
        const uint32_t nb = sm[kk];
        uint32_t same[V];
#pragma unroll
        for (int v = 0; v < V; ++v) same[v] = sm[k0 + v];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t k = k0 + v;
            const uint32_t w = own[k];
            const uint32_t adj = plus ? ((v + 1 < V) ? same[(v + 1) % V] : nb) : ((v > 0) ? same[(v + V - 1) % V] : nb);
            const uint32_t side = plus ? __funnelshift_r(same[v], adj, 1) : __funnelshift_l(adj, same[v], 1);
            uint32_t b0, b1, b2;
            count6(~(w ^ yl[k]), ~(w ^ yh[k]), ~(w ^ zl[k]), ~(w ^ zh[k]), ~(w ^ same[v]), ~(w ^ side), b0, b1, b2);
            const uint32_t needA = b2 & ~b1 & ~b0, needB = b2 & ~b1 & b0, needC = b2 & b1;   // a = 4, 5, 6
            const uint32_t q0 = ((z * L + y) * (L / 2) + 32u * k) >> 2;
            // [r >= thr] shifted in from site 31 down to site 0 (as in the 2D sweep)
            uint32_t ge0 = 0, ge1 = 0, ge2 = 0;
#pragma unroll
            for (int g = 7; g >= 0; --g) {
                const uint4 r = philox(q0 + (uint32_t)g, t, d.sim, c, d.key0, d.key1);
                const uint32_t rr[4] = {r.w, r.z, r.y, r.x};
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    ge0 = shift_in_not_below3(ge0, rr[l], d.thr[0]);
                    ge1 = shift_in_not_below3(ge1, rr[l], d.thr[1]);
                    ge2 = shift_in_not_below3(ge2, rr[l], d.thr[2]);
                }
            }
            own[k] = w ^ (~b2 | (needA & ~ge0) | (needB & ~ge1) | (needC & ~ge2));
        }
    }
}

// E and M of every lattice from its words: for each white word, its six
// aligned bonds and the spins of both colours; block sums, one atomic per
// block and lattice (blockIdx.y = lattice).
__global__ void __launch_bounds__(256) obs3d_kernel(State3 st) {
    __shared__ unsigned long long red[2 * 8];
    for (int lat = blockIdx.y; lat < st.n; lat += gridDim.y) {
        const Lat3 d = st.lat[lat];
        const uint32_t L = d.L, wn = d.wn;
        const uint64_t items = (uint64_t)L * L * wn;
        const uint32_t* base = st.spins + d.word_off;
        unsigned long long sa = 0, sp = 0;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items;
             i += (uint64_t)gridDim.x * blockDim.x) {
            const uint32_t k = (uint32_t)(i % wn);
            const uint32_t y = (uint32_t)((i / wn) % L), z = (uint32_t)(i / ((uint64_t)wn * L));
            const Words6 v = load6(base, L, wn, 1u, z, y, k);
            sa += __popc(~(v.w ^ v.yl)) + __popc(~(v.w ^ v.yh)) + __popc(~(v.w ^ v.zl)) + __popc(~(v.w ^ v.zh)) +
                  __popc(~(v.w ^ v.same)) + __popc(~(v.w ^ v.side));
            sp += __popc(v.w) + __popc(v.same);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xffffffffu, sa, o);
            sp += __shfl_down_sync(0xffffffffu, sp, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) { red[2 * warp] = sa; red[2 * warp + 1] = sp; }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0, b = 0;
            for (int w = 0; w < (int)blockDim.x / 32; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
            atomicAdd(&st.acc[2 * (size_t)lat], a);
            atomicAdd(&st.acc[2 * (size_t)lat + 1], b);
        }
    }
}

// E = 3N - 2 sum(white aligned), M = N - 2 popcount; current values, trace
// slot t % cap; clear the sums; advance the sweep counter when `advance`.
__global__ void record3d_kernel(State3 st, int advance) {
    const unsigned long long t = st.ctl->t;
    for (int lat = threadIdx.x; lat < st.n; lat += blockDim.x) {
        const long long N = (long long)st.lat[lat].L * st.lat[lat].L * st.lat[lat].L;
        const long long E = 3 * N - 2 * (long long)st.acc[2 * lat];
        const long long M = N - 2 * (long long)st.acc[2 * lat + 1];
        st.acc[2 * lat] = 0;
        st.acc[2 * lat + 1] = 0;
        st.obs[2 * lat] = E;
        st.obs[2 * lat + 1] = M;
        const long long cap = st.ctl->trace_cap;
        if (advance && cap > 0) {
            const long long slot = (long long)(t % (unsigned long long)cap);
            st.trace[((long long)lat * cap + slot) * 2] = E;
            st.trace[((long long)lat * cap + slot) * 2 + 1] = M;
        }
    }
    __syncthreads();
    if (advance && threadIdx.x == 0) st.ctl->t = t + 1;
}

// Random initial state: both colour words of (z, y, k) from the 16 Philox
// blocks of sites x in [64 k, 64 k + 64), p = (z L + y) L + x, phase 2.
__global__ void __launch_bounds__(256) init3d_kernel(State3 st) {
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < st.items;
         item += (uint64_t)gridDim.x * blockDim.x) {
        const Lat3 d = st.lat[lattice_of_item(st.lat, st.n, item)];
        const uint32_t L = d.L, wn = d.wn;
        const uint64_t i = item - d.item_begin;
        const uint32_t k = (uint32_t)(i % wn);
        const uint32_t y = (uint32_t)((i / wn) % L), z = (uint32_t)(i / ((uint64_t)wn * L));
        const uint32_t q0 = ((z * L + y) * L + 64u * k) >> 2;
        uint32_t even = 0, odd = 0;
#pragma unroll 4
        for (uint32_t g = 0; g < 16; ++g) {
            const uint4 r = philox(q0 + g, 0u, d.sim, 2u, d.key0, d.key1);
            even |= ((r.x >> 31) << (2 * g)) | ((r.z >> 31) << (2 * g + 1));
            odd |= ((r.y >> 31) << (2 * g)) | ((r.w >> 31) << (2 * g + 1));
        }
        // colour c holds x = 2j + ((y + z + c) & 1)
        const bool e1 = ((y + z) & 1u) != 0;
        uint32_t* base = st.spins + d.word_off;
        base[(((size_t)0 * L + z) * L + y) * wn + k] = e1 ? odd : even;
        base[(((size_t)1 * L + z) * L + y) * wn + k] = e1 ? even : odd;
    }
}

}  // namespace
}  // namespace ising

// ===========================================================================
// Host side: the ising3d_* entry points
// ===========================================================================
using namespace ising;

namespace {

constexpr size_t kAlign3 = 256;
size_t align3(size_t x) { return (x + kAlign3 - 1) / kAlign3 * kAlign3; }

struct Layout3 {
    size_t ctl = 0, lat = 0, acc = 0, obs = 0, trace = 0, spins = 0, total = 0;
    std::vector<uint64_t> word_off;
    uint64_t words = 0;
};

bool layout3(int n, const int* Ls, int64_t cap, Layout3* out) {
    Layout3 l;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align3(off + b); return o; };
    l.ctl = take(sizeof(Ctl3));
    l.lat = take((size_t)n * sizeof(Lat3));
    l.acc = take((size_t)n * 2 * sizeof(unsigned long long));
    l.obs = take((size_t)n * 2 * sizeof(long long));
    if (cap > 0 && n > 0 && (size_t)cap > (SIZE_MAX / 32) / (size_t)n) return false;
    l.trace = take((size_t)n * (size_t)cap * 2 * sizeof(long long));
    l.spins = off;
    l.word_off.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
        l.word_off[(size_t)i] = l.words;
        l.words += (uint64_t)Ls[i] * Ls[i] * Ls[i] / 32;
    }
    off = align3(off + l.words * 4);
    l.total = off;
    *out = l;
    return true;
}

uint32_t thr3(double dE, double T) {
    const double v = std::ldexp(std::exp(-dE / T), 32);
    if (v >= 4294967296.0) return 0xFFFFFFFFu;
    return (uint32_t)std::floor(v);
}

bool valid_L3(int L) { return L >= 64 && L <= ISING3D_MAX_L && L % 64 == 0; }

}  // namespace

struct ising3d_handle {
    int n = 0;
    std::vector<int> L;
    int64_t cap = 0;
    int64_t t = 0;
    int64_t launches = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    Layout3 layout;
    State3 st{};
    int V = 1;
    bool graph = false;
    std::map<int64_t, cudaGraphExec_t> graphs;
    int grid = 0;
};

namespace {

int fail3(int code, const std::string& m) { return set_last_error(code, m.c_str()); }

int cuda_fail3(cudaError_t e, const char* what) {
    return fail3(ISING_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int enqueue_obs3(ising3d_handle* h, int advance) {
    const int gy = std::min(h->n, 65535);
    const int gx = std::max(1, std::min(1024, (int)(h->grid / std::max(1, h->n)) + 1));
    obs3d_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, h->stream>>>(h->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail3(e, "3d observables");
    record3d_kernel<<<1, 256, 0, h->stream>>>(h->st, advance);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail3(e, "3d record");
    return ISING_OK;
}

int enqueue_sweeps3(ising3d_handle* h, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        for (uint32_t c = 0; c < 2; ++c) {
            switch (h->V) {
            case 4: half3d_kernel<4><<<h->grid, 256, 0, h->stream>>>(h->st, c); break;
            case 2: half3d_kernel<2><<<h->grid, 256, 0, h->stream>>>(h->st, c); break;
            default: half3d_kernel<1><<<h->grid, 256, 0, h->stream>>>(h->st, c); break;
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail3(e, "3d half-sweep");
        }
        int rc = enqueue_obs3(h, 1);
        if (rc != ISING_OK) return rc;
    }
    return ISING_OK;
}

}  // namespace

extern "C" {

int ising3d_workspace_bytes(int n_sims, const int* Ls, int64_t trace_cap, size_t* bytes) {
    if (!bytes || n_sims < 0 || trace_cap < 0 || (n_sims > 0 && !Ls)) return fail3(ISING_EINVAL, "invalid arguments");
    for (int i = 0; i < n_sims; ++i)
        if (!valid_L3(Ls[i])) return fail3(ISING_EINVAL, "3d lattice sides must be multiples of 64 in [64, ISING3D_MAX_L]");
    Layout3 l;
    if (!layout3(n_sims, Ls, trace_cap, &l)) return fail3(ISING_EINVAL, "trace_cap too large");
    *bytes = l.total;
    return ISING_OK;
}

int ising3d_create(ising3d_t* out, int n_sims, const int* Ls, const double* temps, const uint64_t* seeds, int init,
                   int64_t trace_cap, void* dev_workspace, size_t ws_bytes, void* cuda_stream) {
    if (!out) return fail3(ISING_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_sims < 1 || !Ls || !temps || !seeds) return fail3(ISING_EINVAL, "need n_sims >= 1 and Ls, temps, seeds");
    if (init != ISING_INIT_RANDOM && init != ISING_INIT_COLD) return fail3(ISING_EINVAL, "init must be 0 or 1");
    if (trace_cap < 0) return fail3(ISING_EINVAL, "trace_cap must be >= 0");
    for (int i = 0; i < n_sims; ++i) {
        if (!valid_L3(Ls[i])) return fail3(ISING_EINVAL, "3d lattice sides must be multiples of 64 in [64, ISING3D_MAX_L]");
        if (!(temps[i] > 0.0) || !std::isfinite(temps[i])) return fail3(ISING_EINVAL, "temperatures must be positive and finite");
    }
    Layout3 lay;
    if (!layout3(n_sims, Ls, trace_cap, &lay)) return fail3(ISING_EINVAL, "trace_cap too large");
    if (!dev_workspace || ((uintptr_t)dev_workspace) % kAlign3 != 0) return fail3(ISING_EINVAL, "workspace must be 256-byte aligned device memory");
    if (ws_bytes < lay.total) return fail3(ISING_ENOMEM, "workspace too small");
    auto* h = new ising3d_handle();
    h->n = n_sims;
    h->L.assign(Ls, Ls + n_sims);
    h->cap = trace_cap;
    h->stream = (cudaStream_t)cuda_stream;
    h->ws = (char*)dev_workspace;
    h->layout = lay;
    std::vector<Lat3> tab((size_t)n_sims);
    uint64_t items = 0;
    for (int i = 0; i < n_sims; ++i) {
        Lat3 d{};
        d.word_off = lay.word_off[(size_t)i];
        d.item_begin = items;
        d.L = (uint32_t)Ls[i];
        d.wn = (uint32_t)(Ls[i] / 64);
        d.sim = (uint32_t)i;
        d.key0 = (uint32_t)(seeds[i] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(seeds[i] >> 32);
        for (int k = 0; k < 3; ++k) d.thr[k] = thr3(4.0 * (k + 1), temps[i]);
        tab[(size_t)i] = d;
        items += (uint64_t)Ls[i] * Ls[i] * (Ls[i] / 64);
    }
    State3& st = h->st;
    st.ctl = (Ctl3*)(h->ws + lay.ctl);
    st.lat = (const Lat3*)(h->ws + lay.lat);
    st.acc = (unsigned long long*)(h->ws + lay.acc);
    st.obs = (long long*)(h->ws + lay.obs);
    st.trace = (long long*)(h->ws + lay.trace);
    st.spins = (uint32_t*)(h->ws + lay.spins);
    st.n = n_sims;
    st.items = items;
    Ctl3 ctl{};
    ctl.trace_cap = trace_cap;
    int sms = device_sm_count();
    // words per thread: 2 (the fastest measured on 512^3 and 1024^3), or 1
    // when some row has an odd number of words
    h->V = 2;
    for (int i = 0; i < n_sims; ++i)
        if ((Ls[i] / 64) % 2 != 0) h->V = 1;
    h->grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((items / h->V + 255) / 256, (uint64_t)sms * 8));
    cudaError_t e = cudaMemsetAsync(h->ws, 0, lay.spins, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ws + lay.ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws + lay.lat, tab.data(), tab.size() * sizeof(Lat3), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        if (init == ISING_INIT_COLD) {
            e = cudaMemsetAsync(h->ws + lay.spins, 0, lay.words * 4, h->stream);
        } else {
            init3d_kernel<<<h->grid, 256, 0, h->stream>>>(st);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host table goes out of scope
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail3(e, "3d create");
    }
    int rc = enqueue_obs3(h, 0);
    if (rc == ISING_OK) {
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail3(e, "3d create");
    }
    if (rc != ISING_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return ISING_OK;
}

int ising3d_set_graph(ising3d_t h, int on) {
    if (!h) return fail3(ISING_EINVAL, "handle is NULL");
    if (on && h->stream == nullptr) return fail3(ISING_ESTATE, "graph replay needs a non-default stream");
    h->graph = on != 0;
    if (!h->graph) {
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
    }
    return ISING_OK;
}

int ising3d_sweep(ising3d_t h, int64_t n) {
    if (!h) return fail3(ISING_EINVAL, "handle is NULL");
    if (n < 0) return fail3(ISING_EINVAL, "n must be >= 0");
    if (n == 0) return ISING_OK;
    if (h->t + n > (int64_t)0xFFFFFFFFll) return fail3(ISING_EINVAL, "sweep counter would pass 2^32");
    if (h->graph) {
        auto it = h->graphs.find(n);
        if (it == h->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail3(e, "begin capture");
            int rc = enqueue_sweeps3(h, n);
            e = cudaStreamEndCapture(h->stream, &g);
            if (rc != ISING_OK) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail3(e, "end capture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail3(e, "graph instantiate");
            it = h->graphs.emplace(n, ex).first;
        }
        cudaError_t e = cudaGraphLaunch(it->second, h->stream);
        if (e != cudaSuccess) return cuda_fail3(e, "graph launch");
    } else {
        int rc = enqueue_sweeps3(h, n);
        if (rc != ISING_OK) return rc;
    }
    h->t += n;
    h->launches += 4 * n;
    return ISING_OK;
}

int64_t ising3d_sweeps_done(ising3d_t h) { return h ? h->t : -1; }

int64_t ising3d_kernel_launches(ising3d_t h) { return h ? h->launches : -1; }

int ising3d_observables(ising3d_t h, int64_t* E, int64_t* M) {
    if (!h || !E || !M) return fail3(ISING_EINVAL, "invalid arguments");
    std::vector<long long> buf(2 * (size_t)h->n);
    cudaError_t e = cudaMemcpyAsync(buf.data(), h->st.obs, buf.size() * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail3(e, "3d observables");
    for (int i = 0; i < h->n; ++i) { E[i] = buf[2 * (size_t)i]; M[i] = buf[2 * (size_t)i + 1]; }
    return ISING_OK;
}

int ising3d_trace(ising3d_t h, int64_t* E, int64_t* M, int64_t max_sweeps, int64_t* n_out) {
    if (!h || !n_out || max_sweeps < 0) return fail3(ISING_EINVAL, "invalid arguments");
    const int64_t k = std::min(std::min(h->t, h->cap), max_sweeps);
    *n_out = k;
    if (k == 0) return ISING_OK;
    if (!E || !M) return fail3(ISING_EINVAL, "E/M is NULL");
    std::vector<long long> buf((size_t)h->n * h->cap * 2);
    cudaError_t e = cudaMemcpyAsync(buf.data(), h->st.trace, buf.size() * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail3(e, "3d trace");
    for (int i = 0; i < h->n; ++i)
        for (int64_t j = 0; j < k; ++j) {
            const int64_t t = h->t - k + j;
            const size_t slot = (size_t)(t % h->cap);
            E[(size_t)i * k + j] = buf[((size_t)i * h->cap + slot) * 2];
            M[(size_t)i * k + j] = buf[((size_t)i * h->cap + slot) * 2 + 1];
        }
    return ISING_OK;
}

int ising3d_get_spins(ising3d_t h, int sim, int8_t* host_LLL) {
    if (!h || sim < 0 || sim >= h->n || !host_LLL) return fail3(ISING_EINVAL, "invalid arguments");
    const int L = h->L[(size_t)sim];
    const size_t wn = (size_t)L / 64, words = (size_t)L * L * L / 32;
    std::vector<uint32_t> w(words);
    cudaError_t e = cudaMemcpyAsync(w.data(), h->st.spins + h->layout.word_off[(size_t)sim], words * 4,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail3(e, "3d spins");
    for (int c = 0; c < 2; ++c)
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (size_t k = 0; k < wn; ++k) {
                    const uint32_t v = w[(((size_t)c * L + z) * L + y) * wn + k];
                    for (int b = 0; b < 32; ++b) {
                        const size_t x = 2 * (32 * k + (size_t)b) + (size_t)((y + z + c) & 1);
                        host_LLL[((size_t)z * L + y) * L + x] = ((v >> b) & 1u) ? -1 : 1;
                    }
                }
    return ISING_OK;
}

void ising3d_destroy(ising3d_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    delete h;
}

}  // extern "C"
