// ising_api.cu -- host side of the C ABI declared in include/ising.h.
//
// Owns no device memory: every device array lives in the caller's workspace,
// carved up by compute_layout().  Kernels are in ising_kernels.cu.
#include "../../include/ising.h"
#include "ising_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

using namespace ising;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(ISING_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                          \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kMaxGroup = 256;            // lattices per resident group (matches the kernel)
constexpr uint32_t kSaveMagic = 0x49534E47u;  // "ISNG"
constexpr uint32_t kSaveVersion = 1;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_L(int L) { return L >= ISING_MIN_L && L <= ISING_MAX_L && (L % 64) == 0; }


struct Layout {
    size_t lat = 0, groups = 0, members = 0, slats = 0, done = 0, acc = 0, obs = 0, trace = 0,
           mom = 0, ctl = 0, list = 0, spins = 0, total = 0;
    std::vector<uint64_t> word_off;  // per lattice, in 32-bit words from `spins`
    size_t spin_bytes = 0;
};

bool compute_layout(int n, const int* Ls, int64_t trace_cap, Layout* out) {
    Layout l;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t nn = (size_t)n;
    l.ctl = take(sizeof(Control));
    l.lat = take(nn * sizeof(LatDesc));
    l.groups = take(nn * sizeof(GroupDesc));
    l.members = take(nn * sizeof(uint32_t));
    l.slats = take(nn * sizeof(StreamLat));
    l.done = take(nn * sizeof(unsigned int));
    l.acc = take(nn * 2 * sizeof(unsigned long long));
    l.obs = take(nn * 2 * sizeof(long long));
    if (trace_cap > 0 && nn > 0 && (size_t)trace_cap > (SIZE_MAX / 32) / nn) return false;
    l.trace = take(nn * (size_t)trace_cap * 2 * sizeof(long long));
    l.mom = take(nn * 6 * sizeof(double));
    l.list = take(nn * sizeof(uint32_t));
    l.spins = off;
    uint64_t words = 0;
    l.word_off.resize(nn);
    for (int i = 0; i < n; ++i) {
        l.word_off[i] = words;
        words += (uint64_t)Ls[i] * (uint64_t)Ls[i] / 32;  // L*L/8 bytes
    }
    l.spin_bytes = (size_t)words * 4;
    off = align_up(off + l.spin_bytes);
    l.total = off;
    *out = l;
    return true;
}

struct Plan {
    int mode = ISING_PLAN_AUTO;
    int words_per_thread = 0;   // stream: V (0 = default)
    int rows_per_item = 0;      // stream: R (0 = default)
    int stream_threads = 256;
    int sweeps_per_unit = 0;    // resident: k (0 = default)
    int resident_threads = 0;   // 0 = from group size
};

}  // namespace

int ising::set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

// thr = min(floor(2^32 exp(-dE/T)), 2^32 - 1) in double precision.
uint32_t ising::threshold_u32(double dE, double T) {
    const double v = std::ldexp(std::exp(-dE / T), 32);
    if (v >= 4294967296.0) return 0xFFFFFFFFu;
    return (uint32_t)std::floor(v);
}

struct ising_handle {
    int n = 0;
    std::vector<int> L;
    std::vector<double> T;
    std::vector<uint64_t> seed;
    std::vector<uint32_t> thr;
    int64_t trace_cap = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    Layout layout;
    DevState st{};
    int64_t t = 0;
    int measure = 0;
    Plan plan;
    bool graph = false;
    std::map<int64_t, cudaGraphExec_t> graphs;
    // resolved execution tables
    bool tables_ready = false;
    int n_groups = 0;
    size_t group_smem = 0;
    int res_threads = 0;
    int res_grid = 0;
    // CLUSTER plan: classes of equal L, one thread-block cluster per lattice
    struct ClusterClass { uint32_t L; int cluster; int member_off; int count; };
    std::vector<ClusterClass> cl_classes;
    int n_slats = 0;
    uint64_t total_tiles = 0;
    int V = 1;                  // streaming tiling in use: words per thread and row,
    int R = 4;                  // and rows per thread
    int stream_grid = 0;
    int sms = 0;
    int64_t launches = 0;
    // Swendsen-Wang: per-lattice table (built once) and its upload target
    std::vector<SwLat> sw_table;
    uint64_t sw_tiles = 0, sw_sites = 0;
    std::map<std::pair<int64_t, const void*>, cudaGraphExec_t> sw_graphs;
    std::map<std::pair<int64_t, const void*>, cudaGraphExec_t> wolff_graphs;   // Wolff steps by labelling
    int wolff_method = ISING_WOLFF_AUTO;
    uint32_t* sw_seed_area = nullptr;    // seed roots in the last cluster scratch (set by sw_prepare)
};

namespace {

void drop_graphs(ising_handle* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    for (auto& kv : h->sw_graphs) cudaGraphExecDestroy(kv.second);
    h->sw_graphs.clear();
    for (auto& kv : h->wolff_graphs) cudaGraphExecDestroy(kv.second);
    h->wolff_graphs.clear();
}

int check_device_error(ising_handle* h) {
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, &h->st.ctl->error, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
             "read error flag");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    if (err == 3)
        return fail(ISING_ETIMEOUT, "a bounded union-find walk of the cluster step ran out (flag %d)", err);
    if (err != 0)
        return fail(ISING_ETIMEOUT, "a bounded device wait of the sweep kernels ran out (flag %d)", err);
    return ISING_OK;
}

// Build the resident groups and streamed lattice tables for the current plan
// and upload them (asynchronously, from host buffers kept alive by a sync).
int build_tables(ising_handle* h) {
    const int n = h->n;
    h->sms = device_sm_count();
    const size_t optin = device_max_smem_optin();
    const size_t static_smem = 16 * 1024;  // SiteKey/lattice tables and counters of the kernel
    const size_t res_budget = optin > static_smem ? optin - static_smem : 0;
    h->cl_classes.clear();
    if (h->plan.mode == ISING_PLAN_CLUSTER) {
        // one thread-block cluster per lattice: C CTAs of rows_per_item rows
        // (default 64), C the largest power of two <= min(8, L / rows)
        const int rows = h->plan.rows_per_item > 0 ? h->plan.rows_per_item : 64;
        std::map<int, std::vector<uint32_t>> by_L;
        for (int i = 0; i < n; ++i) {
            if (h->L[i] > ISING_CLUSTER_MAX_L)
                return fail(ISING_EINVAL, "cluster plan: lattice %d has L=%d > %d", i, h->L[i], ISING_CLUSTER_MAX_L);
            by_L[h->L[i]].push_back((uint32_t)i);
        }
        std::vector<uint32_t> members;
        for (auto& kv : by_L) {
            int c = 1;
            while (c * 2 <= 8 && c * 2 <= std::max(1, kv.first / rows)) c *= 2;
            h->cl_classes.push_back({(uint32_t)kv.first, c, (int)members.size(), (int)kv.second.size()});
            members.insert(members.end(), kv.second.begin(), kv.second.end());
        }
        h->n_groups = 0;
        h->n_slats = 0;
        h->total_tiles = 0;
        h->V = 1;
        h->R = rows;
        if (!members.empty())
            CUDA_TRY(cudaMemcpyAsync(h->ws + h->layout.members, members.data(), members.size() * sizeof(uint32_t),
                                     cudaMemcpyHostToDevice, h->stream), "upload cluster members");
        CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize after table upload");
        h->tables_ready = true;
        drop_graphs(h);
        return ISING_OK;
    }
    std::vector<int> resident, streamed;
    for (int i = 0; i < n; ++i) {
        const size_t bytes = (size_t)h->L[i] * h->L[i] / 8;
        bool res;
        if (h->plan.mode == ISING_PLAN_RESIDENT) {
            if (bytes > res_budget)
                return fail(ISING_EINVAL, "lattice %d (L=%d) does not fit in shared memory (%zu > %zu bytes)",
                            i, h->L[i], bytes, res_budget);
            res = true;
        } else if (h->plan.mode == ISING_PLAN_MIXED) {
            res = h->L[i] <= 1024 && bytes <= res_budget;
        } else {
            // STREAM, PERSIST and AUTO: streamed.  AUTO streams too: on GB300 the
            // resident kernel measured at best even with the streaming one (one
            // 64^2 lattice) and up to 17x slower (one 1024^2 lattice)
            res = false;
        }
        (res ? resident : streamed).push_back(i);
    }

    // resident groups: equal L, filled up to the shared-memory budget, then
    // split so that there are at least as many groups as SMs when possible
    std::vector<GroupDesc> groups;
    std::vector<uint32_t> members;
    h->group_smem = 0;
    if (!resident.empty()) {
        std::stable_sort(resident.begin(), resident.end(), [&](int a, int b) { return h->L[a] < h->L[b]; });
        double total_sites = 0;
        for (int i : resident) total_sites += (double)h->L[i] * h->L[i];
        size_t i0 = 0;
        int full_groups = 0;
        std::vector<std::pair<size_t, size_t>> classes;  // [begin, end) of equal L
        while (i0 < resident.size()) {
            size_t i1 = i0;
            while (i1 < resident.size() && h->L[resident[i1]] == h->L[resident[i0]]) ++i1;
            classes.push_back({i0, i1});
            const size_t bytes = (size_t)h->L[resident[i0]] * h->L[resident[i0]] / 8;
            const size_t maxg = std::min<size_t>(kMaxGroup, std::max<size_t>(1, res_budget / bytes));
            full_groups += (int)((i1 - i0 + maxg - 1) / maxg);
            i0 = i1;
        }
        for (auto [b, e] : classes) {
            const int Lc = h->L[resident[b]];
            const size_t bytes = (size_t)Lc * Lc / 8;
            size_t per = std::min<size_t>(kMaxGroup, std::max<size_t>(1, res_budget / bytes));
            const size_t cnt = e - b;
            if (full_groups < h->sms) {
                // spread this class over its share of the SMs
                const double share = (double)cnt * Lc * Lc / total_sites;
                const size_t want = std::max<size_t>(1, (size_t)std::floor(share * h->sms));
                per = std::min(per, std::max<size_t>(1, (cnt + want - 1) / want));
            }
            for (size_t j = b; j < e; j += per) {
                const size_t c = std::min(per, e - j);
                GroupDesc g{};
                g.member_off = (uint32_t)members.size();
                g.count = (uint32_t)c;
                g.L = (uint32_t)Lc;
                g.wn = (uint32_t)(Lc / 64);
                for (size_t q = j; q < j + c; ++q) members.push_back((uint32_t)resident[q]);
                groups.push_back(g);
                h->group_smem = std::max(h->group_smem, c * bytes);
            }
        }
    }
    h->n_groups = (int)groups.size();
    if (h->n_groups > 0) {
        size_t max_words = 0;
        for (auto& g : groups) max_words = std::max(max_words, (size_t)g.count * g.L * g.wn);
        int thr = h->plan.resident_threads;
        if (thr <= 0) thr = (int)std::min<size_t>(512, std::max<size_t>(64, (max_words + 31) / 32 * 32));
        if (thr > 512) return fail(ISING_EINVAL, "resident kernel runs at most 512 threads per block");
        h->res_threads = thr;
        const int occ = resident_occupancy(thr, h->group_smem);
        if (occ <= 0)
            return fail(ISING_EINVAL, "resident kernel cannot launch with %d threads and %zu bytes of shared memory",
                        thr, h->group_smem);
        h->res_grid = std::min(h->n_groups, h->sms * occ);
    }

    // streamed lattices: tiles of (tw word groups) x (th row groups of R rows)
    std::vector<StreamLat> slats;
    const int B = h->plan.stream_threads;
    auto divides = [&](int v) {
        for (int i : streamed)
            if ((h->L[i] / 64) % v != 0) return false;
        return true;
    };
    auto count_tiles = [&](int v, int r) {
        uint64_t n = 0;
        for (int i : streamed) {
            const uint32_t groups = (uint32_t)(h->L[i] / 64) / (uint32_t)v;
            const uint32_t tw = std::min<uint32_t>(groups, (uint32_t)B), th = (uint32_t)B / tw;
            const uint32_t rl = std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)r, (uint32_t)h->L[i] / th));
            n += (uint64_t)((groups + tw - 1) / tw) * (((uint32_t)h->L[i] + th * rl - 1) / (th * rl));
        }
        return n;
    };
    int V = h->plan.words_per_thread, R = h->plan.rows_per_item > 0 ? h->plan.rows_per_item : 4;
    if (V > 0) {
        while (V > 1 && !divides(V)) V /= 2;
    } else if (streamed.empty()) {
        V = 4;
    } else {
        // default tiling by the number of blocks it gives (256 threads), from
        // measurements of single lattices (flip/ns): 4 words x 4 rows per thread
        // only for large streamed workloads (six 16384^2: 1,461), 2 x 2 from
        // 1.5 blocks per SM (8192^2: 1,221 against 1,160 for 4 x 4; 4096^2:
        // 838 against 512), 1 x 2 from half a block per SM (2048^2: 479
        // against 125), else 1 x 1.  Rows stay as given if rows_per_item is set.
        const bool rows_free = h->plan.rows_per_item == 0;
        const uint64_t sms = (uint64_t)h->sms;
        const struct { int v, r; uint64_t min_tiles; } cand[4] = {
            {4, rows_free ? 4 : R, 4 * sms}, {2, rows_free ? 2 : R, 3 * sms / 2},
            {1, rows_free ? 2 : R, sms / 2}, {1, rows_free ? 1 : R, 0}};
        for (const auto& c : cand) {
            if (!divides(c.v)) continue;
            V = c.v;
            R = c.r;
            if (count_tiles(V, R) >= c.min_tiles) break;
        }
    }
    h->V = V;
    h->R = R;
    uint64_t tiles = 0;
    for (int i : streamed) {
        StreamLat s{};
        s.lat = (uint32_t)i;
        const uint32_t wn = (uint32_t)(h->L[i] / 64);
        s.groups = wn / (uint32_t)V;
        const uint32_t tw = std::min<uint32_t>(s.groups, (uint32_t)B);
        const uint32_t th = (uint32_t)B / tw;
        // rows per thread: at most R, and no more than keeps a whole tile within the lattice
        const uint32_t Rl = std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)R, (uint32_t)h->L[i] / th));
        s.rows = Rl;
        const uint32_t tiles_x = (s.groups + tw - 1) / tw;
        const uint32_t tiles_y = ((uint32_t)h->L[i] + th * Rl - 1) / (th * Rl);
        s.strips = tiles_y;
        s.item_begin = tiles;
        tiles += (uint64_t)tiles_x * tiles_y;
        slats.push_back(s);
    }
    h->n_slats = (int)slats.size();
    h->total_tiles = tiles;
    if (h->n_slats > 0) {
        const int occ = (h->plan.mode == ISING_PLAN_PERSIST) ? stream_persistent_occupancy(V, B)
                                                              : stream_occupancy(V, B);
        if (occ <= 0) return fail(ISING_EINVAL, "streaming kernel cannot launch with %d threads", B);
        // the persistent kernel needs every block co-resident (cooperative
        // launch); the per-half-sweep kernel runs one block per tile, so that
        // the block scheduler balances the tiles over the SMs (a grid of two
        // blocks per SM looping over tiles left SMs idle in its last round:
        // 12 % slower on three 16384^2 lattices)
        h->stream_grid = (h->plan.mode == ISING_PLAN_PERSIST)
                             ? (int)std::min<uint64_t>(tiles, (uint64_t)h->sms * occ)
                             : (int)std::min<uint64_t>(tiles, (uint64_t)0x7FFFFFFF);
    }

    if (!groups.empty())
        CUDA_TRY(cudaMemcpyAsync(h->ws + h->layout.groups, groups.data(), groups.size() * sizeof(GroupDesc),
                                 cudaMemcpyHostToDevice, h->stream), "upload groups");
    if (!members.empty())
        CUDA_TRY(cudaMemcpyAsync(h->ws + h->layout.members, members.data(), members.size() * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, h->stream), "upload members");
    if (!slats.empty())
        CUDA_TRY(cudaMemcpyAsync(h->ws + h->layout.slats, slats.data(), slats.size() * sizeof(StreamLat),
                                 cudaMemcpyHostToDevice, h->stream), "upload stream tables");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize after table upload");
    h->tables_ready = true;
    drop_graphs(h);
    return ISING_OK;
}

// Kernels one enqueue_sweeps(h, n) issues.
int64_t kernels_per_call(const ising_handle* h, int64_t n) {
    if (h->plan.mode == ISING_PLAN_CLUSTER) return (int64_t)h->cl_classes.size() + 1;
    int64_t k = 0;
    if (h->n_groups > 0) k += 1;
    if (h->n_slats > 0 && h->plan.mode == ISING_PLAN_PERSIST) k += 1;
    else if (h->n_slats > 0) k += 2 * n;
    else if (h->n_groups > 0) k += 1;
    return k;
}

int enqueue_sweeps(ising_handle* h, int64_t n) {
    if (h->plan.mode == ISING_PLAN_CLUSTER) {
        const uint32_t* members = (const uint32_t*)(h->ws + h->layout.members);
        for (const auto& c : h->cl_classes)
            CUDA_TRY(launch_cluster_resident(h->st, members + c.member_off, c.count, c.cluster, c.L, n, h->stream),
                     "cluster-resident kernel launch");
        CUDA_TRY(launch_advance_t(h->st, n, h->stream), "advance sweep counter");
        return ISING_OK;
    }
    if (h->n_groups > 0) {
        CUDA_TRY(cudaMemsetAsync(&h->st.ctl->ticket, 0, sizeof(unsigned int), h->stream), "reset tickets");
        CUDA_TRY(cudaMemsetAsync(h->st.done, 0, (size_t)h->n_groups * sizeof(unsigned int), h->stream),
                 "reset chunk flags");
        int k = h->plan.sweeps_per_unit;
        if (k <= 0) k = (int)std::min<int64_t>(n, 64);
        CUDA_TRY(launch_resident(h->st, h->n_groups, n, k, h->res_threads, h->res_grid, h->group_smem,
                                 h->stream), "resident kernel launch");
    }
    if (h->n_slats > 0 && h->plan.mode == ISING_PLAN_PERSIST) {
        CUDA_TRY(launch_stream_persistent(h->st, h->n_slats, h->total_tiles, h->V, h->plan.stream_threads,
                                          h->stream_grid, n, h->stream), "persistent streaming kernel launch");
    } else if (h->n_slats > 0) {
        CUDA_TRY(launch_stream_sweeps(h->st, h->n_slats, h->total_tiles, h->V, h->plan.stream_threads,
                                      h->stream_grid, n, h->stream),
                 "streaming kernel launch");
    } else if (h->n_groups > 0) {
        CUDA_TRY(launch_advance_t(h->st, n, h->stream), "advance sweep counter");
    }
    return ISING_OK;
}

int create_common(ising_t* out, int n, const int* Ls, const double* temps, const uint64_t* seeds,
                  uint64_t one_seed, int init, int64_t trace_cap, void* ws, size_t ws_bytes,
                  void* stream) {
    if (!out) return fail(ISING_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 0) return fail(ISING_EINVAL, "n_sims must be >= 0 (got %d)", n);
    if (trace_cap < 0) return fail(ISING_EINVAL, "trace_cap must be >= 0");
    if (init != ISING_INIT_RANDOM && init != ISING_INIT_COLD) return fail(ISING_EINVAL, "init must be 0 or 1");
    if (n > 0 && (!Ls || !temps)) return fail(ISING_EINVAL, "Ls/temps is NULL");
    for (int i = 0; i < n; ++i) {
        if (!valid_L(Ls[i]))
            return fail(ISING_EINVAL, "lattice %d: L=%d must be a multiple of 64 in [%d, %d]", i, Ls[i],
                        ISING_MIN_L, ISING_MAX_L);
        if (!(temps[i] > 0.0) || !std::isfinite(temps[i]))
            return fail(ISING_EINVAL, "lattice %d: temperature must be positive and finite", i);
    }
    Layout lay;
    if (!compute_layout(n, Ls, trace_cap, &lay)) return fail(ISING_EINVAL, "trace_cap too large");
    if (ws_bytes < lay.total)
        return fail(ISING_ENOMEM, "workspace too small: %zu bytes given, %zu needed", ws_bytes, lay.total);
    if (!ws) return fail(ISING_EINVAL, "workspace is NULL");
    if (((uintptr_t)ws) % kAlign != 0) return fail(ISING_EINVAL, "workspace must be 256-byte aligned");

    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    cudaPointerAttributes attr{};
    CUDA_TRY(cudaPointerGetAttributes(&attr, ws), "cudaPointerGetAttributes");
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(ISING_EINVAL, "workspace is not device memory");
    CUDA_TRY(configure_kernels(), "configure kernels");

    auto* h = new ising_handle();
    h->n = n;
    h->L.assign(Ls, Ls + n);
    h->T.assign(temps, temps + n);
    h->seed.resize(n);
    for (int i = 0; i < n; ++i) h->seed[i] = seeds ? seeds[i] : one_seed;
    h->thr.resize(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        h->thr[2 * i] = threshold_u32(4.0, temps[i]);
        h->thr[2 * i + 1] = threshold_u32(8.0, temps[i]);
    }
    h->trace_cap = trace_cap;
    h->stream = (cudaStream_t)stream;
    h->ws = (char*)ws;
    h->ws_bytes = ws_bytes;
    h->layout = lay;
    DevState& st = h->st;
    st.ctl = (Control*)(h->ws + lay.ctl);
    st.lat = (const LatDesc*)(h->ws + lay.lat);
    st.groups = (const GroupDesc*)(h->ws + lay.groups);
    st.members = (const uint32_t*)(h->ws + lay.members);
    st.slats = (const StreamLat*)(h->ws + lay.slats);
    st.done = (unsigned int*)(h->ws + lay.done);
    st.acc = (unsigned long long*)(h->ws + lay.acc);
    st.obs = (long long*)(h->ws + lay.obs);
    st.trace = (long long*)(h->ws + lay.trace);
    st.mom = (double*)(h->ws + lay.mom);
    st.spins = (uint32_t*)(h->ws + lay.spins);
    st.n = n;

    std::vector<LatDesc> descs(n);
    for (int i = 0; i < n; ++i) {
        LatDesc d{};
        d.word_off = lay.word_off[i];
        d.L = (uint32_t)Ls[i];
        d.wn = (uint32_t)(Ls[i] / 64);
        d.sim = (uint32_t)i;
        d.key0 = (uint32_t)(h->seed[i] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(h->seed[i] >> 32);
        d.thr0 = h->thr[2 * i];
        d.thr1 = h->thr[2 * i + 1];
        descs[i] = d;
    }
    std::vector<uint32_t> list(n);
    std::iota(list.begin(), list.end(), 0u);
    Control ctl{};
    ctl.trace_cap = trace_cap;

    auto cleanup = [&](int rc) { delete h; return rc; };
    // zero everything except the spin array, then fill tables
    cudaError_t e = cudaMemsetAsync(h->ws, 0, lay.spins, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ws + lay.ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(h->ws + lay.lat, descs.data(), n * sizeof(LatDesc), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(h->ws + lay.list, list.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && n > 0) {
        if (init == ISING_INIT_COLD)
            e = cudaMemsetAsync(h->ws + lay.spins, 0, lay.spin_bytes, h->stream);
        else
            e = launch_init_random(st, n, h->stream);
    }
    if (e == cudaSuccess && n > 0)
        e = launch_observables(st, (uint32_t)*std::max_element(h->L.begin(), h->L.end()),
                               (const uint32_t*)(h->ws + lay.list), n, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host buffers above go out of scope
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "create"));
    int rc = build_tables(h);
    if (rc != ISING_OK) return cleanup(rc);
    *out = h;
    return ISING_OK;
}

}  // namespace

extern "C" {

const char* ising_last_error(void) { return g_last_error.c_str(); }

const char* ising_version(void) { return "libising 0.1 (sm_103a)"; }

int ising_workspace_bytes(int L, int n_sims, int64_t trace_cap, size_t* bytes) {
    if (!bytes) return fail(ISING_EINVAL, "bytes is NULL");
    if (!valid_L(L)) return fail(ISING_EINVAL, "L=%d must be a multiple of 64 in [%d, %d]", L, ISING_MIN_L, ISING_MAX_L);
    if (n_sims < 0 || trace_cap < 0) return fail(ISING_EINVAL, "n_sims and trace_cap must be >= 0");
    std::vector<int> Ls((size_t)n_sims, L);
    Layout l;
    if (!compute_layout(n_sims, Ls.data(), trace_cap, &l)) return fail(ISING_EINVAL, "trace_cap too large");
    *bytes = l.total;
    return ISING_OK;
}

int ising_batch_workspace_bytes(int n_sims, const int* Ls, int64_t trace_cap, size_t* bytes) {
    if (!bytes) return fail(ISING_EINVAL, "bytes is NULL");
    if (n_sims < 0 || trace_cap < 0) return fail(ISING_EINVAL, "n_sims and trace_cap must be >= 0");
    if (n_sims > 0 && !Ls) return fail(ISING_EINVAL, "Ls is NULL");
    for (int i = 0; i < n_sims; ++i)
        if (!valid_L(Ls[i])) return fail(ISING_EINVAL, "lattice %d: L=%d invalid", i, Ls[i]);
    Layout l;
    if (!compute_layout(n_sims, Ls, trace_cap, &l)) return fail(ISING_EINVAL, "trace_cap too large");
    *bytes = l.total;
    return ISING_OK;
}

int ising_create(ising_t* out, int L, int n_sims, const double* temps, uint64_t seed, int init,
                 int64_t trace_cap, void* dev_workspace, size_t ws_bytes, void* cuda_stream) {
    if (n_sims > 0 && !valid_L(L))
        return fail(ISING_EINVAL, "L=%d must be a multiple of 64 in [%d, %d]", L, ISING_MIN_L, ISING_MAX_L);
    if (n_sims < 0) return fail(ISING_EINVAL, "n_sims must be >= 0");
    std::vector<int> Ls((size_t)n_sims, L);
    return create_common(out, n_sims, Ls.data(), temps, nullptr, seed, init, trace_cap, dev_workspace,
                         ws_bytes, cuda_stream);
}

int ising_create_batch(ising_t* out, int n_sims, const int* Ls, const double* temps, const uint64_t* seeds,
                       int init, int64_t trace_cap, void* dev_workspace, size_t ws_bytes, void* cuda_stream) {
    if (n_sims > 0 && !seeds) return fail(ISING_EINVAL, "seeds is NULL");
    return create_common(out, n_sims, Ls, temps, seeds, 0, init, trace_cap, dev_workspace, ws_bytes, cuda_stream);
}

int ising_sweep(ising_t h, int64_t n) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (n < 0) return fail(ISING_EINVAL, "n must be >= 0");
    if (n == 0 || h->n == 0) return ISING_OK;
    if (h->t + n > (int64_t)0xFFFFFFFFll)
        return fail(ISING_EINVAL, "sweep counter would pass 2^32 (Philox counter word 1)");
    if (!h->tables_ready) {
        int rc = build_tables(h);
        if (rc != ISING_OK) return rc;
    }
    if (h->n_groups > 0) {
        int k = h->plan.sweeps_per_unit > 0 ? h->plan.sweeps_per_unit : (int)std::min<int64_t>(n, 64);
        const int64_t tickets = ((n + k - 1) / k) * (int64_t)h->n_groups;
        if (tickets >= (int64_t)0x7FFFFFFF) return fail(ISING_EINVAL, "too many work units; call ising_sweep with fewer sweeps");
    }
    if (h->graph) {
        if (h->stream == nullptr) return fail(ISING_ESTATE, "graph replay needs a non-default stream");
        auto it = h->graphs.find(n);
        if (it == h->graphs.end()) {
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            int rc = enqueue_sweeps(h, n);
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (rc != ISING_OK) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            it = h->graphs.emplace(n, ex).first;
        }
        CUDA_TRY(cudaGraphLaunch(it->second, h->stream), "graph launch");
    } else {
        int rc = enqueue_sweeps(h, n);
        if (rc != ISING_OK) return rc;
    }
    h->t += n;
    h->launches += kernels_per_call(h, n);
    return ISING_OK;
}

int64_t ising_sweeps_done(ising_t h) { return h ? h->t : -1; }

int64_t ising_kernel_launches(ising_t h) { return h ? h->launches : -1; }

int ising_num_sims(ising_t h) { return h ? h->n : 0; }

int ising_lattice_size(ising_t h, int sim) {
    if (!h || sim < 0 || sim >= h->n) return 0;
    return h->L[sim];
}

int ising_observables(ising_t h, int64_t* E, int64_t* M) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (h->n == 0) return ISING_OK;
    if (!E || !M) return fail(ISING_EINVAL, "E/M is NULL");
    std::vector<long long> buf(2 * (size_t)h->n);
    CUDA_TRY(cudaMemcpyAsync(buf.data(), h->st.obs, buf.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream),
             "copy observables");
    int rc = check_device_error(h);
    if (rc != ISING_OK) return rc;
    for (int i = 0; i < h->n; ++i) { E[i] = buf[2 * i]; M[i] = buf[2 * i + 1]; }
    return ISING_OK;
}

int ising_trace(ising_t h, int64_t* E, int64_t* M, int64_t max_sweeps, int64_t* n_out) {
    if (!h || !n_out) return fail(ISING_EINVAL, "handle or n_out is NULL");
    *n_out = 0;
    if (max_sweeps < 0) return fail(ISING_EINVAL, "max_sweeps must be >= 0");
    const int64_t cap = h->trace_cap;
    const int64_t k = std::min(std::min(h->t, cap), max_sweeps);
    if (h->n == 0 || k == 0) { *n_out = 0; return ISING_OK; }
    if (!E || !M) return fail(ISING_EINVAL, "E/M is NULL");
    std::vector<long long> buf((size_t)h->n * cap * 2);
    CUDA_TRY(cudaMemcpyAsync(buf.data(), h->st.trace, buf.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                             h->stream), "copy trace");
    int rc = check_device_error(h);
    if (rc != ISING_OK) return rc;
    for (int i = 0; i < h->n; ++i)
        for (int64_t j = 0; j < k; ++j) {
            const int64_t t = h->t - k + j;
            const int64_t slot = t % cap;
            E[(size_t)i * k + j] = buf[((size_t)i * cap + slot) * 2];
            M[(size_t)i * k + j] = buf[((size_t)i * cap + slot) * 2 + 1];
        }
    *n_out = k;
    return ISING_OK;
}

int ising_get_spins(ising_t h, int sim, int8_t* out) {
    if (!h || !out) return fail(ISING_EINVAL, "handle or buffer is NULL");
    if (sim < 0 || sim >= h->n) return fail(ISING_EINVAL, "sim %d out of range", sim);
    const int L = h->L[sim];
    const size_t wn = (size_t)L / 64;
    std::vector<uint32_t> w((size_t)L * L / 32);
    CUDA_TRY(cudaMemcpyAsync(w.data(), h->st.spins + h->layout.word_off[sim], w.size() * 4,
                             cudaMemcpyDeviceToHost, h->stream), "copy spins");
    int rc = check_device_error(h);
    if (rc != ISING_OK) return rc;
    for (int c = 0; c < 2; ++c)
        for (int y = 0; y < L; ++y)
            for (size_t k = 0; k < wn; ++k) {
                const uint32_t word = w[((size_t)c * L + y) * wn + k];
                for (int b = 0; b < 32; ++b) {
                    const size_t x = 2 * (32 * k + b) + ((y + c) & 1);
                    out[(size_t)y * L + x] = ((word >> b) & 1u) ? (int8_t)-1 : (int8_t)1;
                }
            }
    return ISING_OK;
}

int ising_set_spins(ising_t h, int sim, const int8_t* in) {
    if (!h || !in) return fail(ISING_EINVAL, "handle or buffer is NULL");
    if (sim < 0 || sim >= h->n) return fail(ISING_EINVAL, "sim %d out of range", sim);
    const int L = h->L[sim];
    const size_t wn = (size_t)L / 64;
    std::vector<uint32_t> w((size_t)L * L / 32, 0u);
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const int8_t v = in[(size_t)y * L + x];
            if (v != 1 && v != -1) return fail(ISING_EINVAL, "spin (%d,%d) is %d, not +1/-1", x, y, (int)v);
            const int c = (x + y) & 1;
            const size_t j = (size_t)x >> 1, k = j / 32, b = j % 32;
            if (v == -1) w[((size_t)c * L + y) * wn + k] |= 1u << b;
        }
    CUDA_TRY(cudaMemcpyAsync(h->st.spins + h->layout.word_off[sim], w.data(), w.size() * 4, cudaMemcpyHostToDevice,
                             h->stream), "copy spins");
    CUDA_TRY(launch_observables(h->st, (uint32_t)h->L[sim], (const uint32_t*)(h->ws + h->layout.list) + sim, 1,
                                h->stream),
             "observables");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    return ISING_OK;
}

int ising_lattice_words(ising_t h, int sim, void** dev_words, size_t* n_words) {
    if (!h || !dev_words || !n_words) return fail(ISING_EINVAL, "NULL argument");
    if (sim < 0 || sim >= h->n) return fail(ISING_EINVAL, "sim %d out of range", sim);
    *dev_words = (void*)(h->st.spins + h->layout.word_off[sim]);
    *n_words = (size_t)h->L[sim] * h->L[sim] / 32;
    return ISING_OK;
}

int ising_snapshot(ising_t h, void* dev_dst, size_t bytes) {
    if (!h || !dev_dst) return fail(ISING_EINVAL, "NULL argument");
    if (bytes < h->layout.spin_bytes) return fail(ISING_EINVAL, "destination too small (%zu < %zu)", bytes,
                                                  h->layout.spin_bytes);
    if (h->n == 0) return ISING_OK;
    CUDA_TRY(cudaMemcpyAsync(dev_dst, h->st.spins, h->layout.spin_bytes, cudaMemcpyDeviceToDevice, h->stream),
             "snapshot");
    return ISING_OK;
}

int ising_get_thresholds(ising_t h, uint32_t* thr) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (h->n == 0) return ISING_OK;
    if (!thr) return fail(ISING_EINVAL, "thr is NULL");
    std::copy(h->thr.begin(), h->thr.end(), thr);
    return ISING_OK;
}

int ising_set_measure(ising_t h, int on) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    h->measure = on ? 1 : 0;
    CUDA_TRY(cudaMemcpyAsync(&h->st.ctl->measure, &h->measure, sizeof(int), cudaMemcpyHostToDevice, h->stream),
             "set measure");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    return ISING_OK;
}

int ising_set_wait_limit_ns(ising_t h, uint64_t ns) {
    if (ns > ISING_MAX_WAIT_LIMIT_NS) return fail(ISING_EINVAL, "wait limit must be at most %llu ns",
                                                 (unsigned long long)ISING_MAX_WAIT_LIMIT_NS);
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    const unsigned long long v = (unsigned long long)ns;
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    CUDA_TRY(cudaMemcpy(&h->st.ctl->wait_limit_ns, &v, sizeof(v), cudaMemcpyHostToDevice), "set wait limit");
    return ISING_OK;
}

int ising_reset_moments(ising_t h) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (h->n == 0) return ISING_OK;
    CUDA_TRY(cudaMemsetAsync(h->st.mom, 0, (size_t)h->n * 6 * sizeof(double), h->stream), "reset moments");
    return ISING_OK;
}

int ising_moments(ising_t h, double* out) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (h->n == 0) return ISING_OK;
    if (!out) return fail(ISING_EINVAL, "out is NULL");
    CUDA_TRY(cudaMemcpyAsync(out, h->st.mom, (size_t)h->n * 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "copy moments");
    return check_device_error(h);
}

namespace {
struct SaveHeader {
    uint32_t magic, version;
    int32_t n;
    int32_t pad;
    int64_t t;
    uint64_t spin_bytes;
};
}  // namespace

int ising_state_bytes(ising_t h, size_t* bytes) {
    if (!h || !bytes) return fail(ISING_EINVAL, "handle or bytes is NULL");
    *bytes = sizeof(SaveHeader) + (size_t)h->n * sizeof(int32_t) + h->layout.spin_bytes +
             (size_t)h->n * 2 * sizeof(long long) + (size_t)h->n * 6 * sizeof(double);
    return ISING_OK;
}

int ising_save(ising_t h, void* buf, size_t bytes) {
    size_t need = 0;
    int rc = ising_state_bytes(h, &need);
    if (rc != ISING_OK) return rc;
    if (!buf || bytes < need) return fail(ISING_EINVAL, "buffer too small (%zu < %zu)", bytes, need);
    char* p = (char*)buf;
    SaveHeader hd{kSaveMagic, kSaveVersion, h->n, 0, h->t, h->layout.spin_bytes};
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    for (int i = 0; i < h->n; ++i) { int32_t L = h->L[i]; memcpy(p, &L, 4); p += 4; }
    if (h->n > 0) {
        CUDA_TRY(cudaMemcpyAsync(p, h->st.spins, h->layout.spin_bytes, cudaMemcpyDeviceToHost, h->stream), "save spins");
        p += h->layout.spin_bytes;
        CUDA_TRY(cudaMemcpyAsync(p, h->st.obs, (size_t)h->n * 2 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream),
                 "save observables");
        p += (size_t)h->n * 2 * sizeof(long long);
        CUDA_TRY(cudaMemcpyAsync(p, h->st.mom, (size_t)h->n * 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                 "save moments");
    }
    return check_device_error(h);
}

int ising_load(ising_t h, const void* buf, size_t bytes) {
    size_t need = 0;
    int rc = ising_state_bytes(h, &need);
    if (rc != ISING_OK) return rc;
    if (!buf || bytes < need) return fail(ISING_EINVAL, "buffer too small (%zu < %zu)", bytes, need);
    const char* p = (const char*)buf;
    SaveHeader hd;
    memcpy(&hd, p, sizeof(hd));
    p += sizeof(hd);
    if (hd.magic != kSaveMagic || hd.version != kSaveVersion) return fail(ISING_EINVAL, "not an ising checkpoint");
    if (hd.n != h->n || hd.spin_bytes != h->layout.spin_bytes) return fail(ISING_EINVAL, "checkpoint shape differs");
    for (int i = 0; i < h->n; ++i) {
        int32_t L;
        memcpy(&L, p, 4);
        p += 4;
        if (L != h->L[i]) return fail(ISING_EINVAL, "checkpoint lattice %d has L=%d, handle has %d", i, L, h->L[i]);
    }
    if (hd.t < 0 || hd.t > (int64_t)0xFFFFFFFFll) return fail(ISING_EINVAL, "checkpoint sweep counter out of range");
    unsigned long long t = (unsigned long long)hd.t;
    if (h->n > 0) {
        CUDA_TRY(cudaMemcpyAsync(h->st.spins, p, h->layout.spin_bytes, cudaMemcpyHostToDevice, h->stream), "load spins");
        p += h->layout.spin_bytes;
        CUDA_TRY(cudaMemcpyAsync(h->st.obs, p, (size_t)h->n * 2 * sizeof(long long), cudaMemcpyHostToDevice, h->stream),
                 "load observables");
        p += (size_t)h->n * 2 * sizeof(long long);
        CUDA_TRY(cudaMemcpyAsync(h->st.mom, p, (size_t)h->n * 6 * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                 "load moments");
    }
    CUDA_TRY(cudaMemcpyAsync(&h->st.ctl->t, &t, sizeof(t), cudaMemcpyHostToDevice, h->stream), "load counter");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
    h->t = hd.t;
    return ISING_OK;
}

int ising_set_plan(ising_t h, int plan, int words_per_thread, int rows_per_item, int sweeps_per_unit,
                   int threads) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (plan != ISING_PLAN_AUTO && plan != ISING_PLAN_RESIDENT && plan != ISING_PLAN_STREAM &&
        plan != ISING_PLAN_PERSIST && plan != ISING_PLAN_MIXED && plan != ISING_PLAN_CLUSTER)
        return fail(ISING_EINVAL, "unknown plan %d", plan);
    if (words_per_thread != 0 && words_per_thread != 1 && words_per_thread != 2 && words_per_thread != 4)
        return fail(ISING_EINVAL, "words_per_thread must be 0, 1, 2 or 4");
    if (sweeps_per_unit < 0) return fail(ISING_EINVAL, "sweeps_per_unit must be >= 0");
    if (rows_per_item < 0 || rows_per_item > 1024) return fail(ISING_EINVAL, "rows_per_item must be in [0, 1024]");
    if (threads != 0 && (threads < 32 || threads > 1024 || threads % 32 != 0))
        return fail(ISING_EINVAL, "threads must be 0 or a multiple of 32 in [32, 1024]");
    Plan p = h->plan;
    p.mode = plan;
    p.words_per_thread = words_per_thread;
    p.sweeps_per_unit = sweeps_per_unit;
    p.rows_per_item = rows_per_item;
    if (plan == ISING_PLAN_STREAM || plan == ISING_PLAN_PERSIST || plan == ISING_PLAN_AUTO) {
        if (threads != 0 && threads > 256) return fail(ISING_EINVAL, "streaming kernel allows at most 256 threads");
        p.stream_threads = threads ? threads : 256;
    } else {
        p.resident_threads = threads;
    }
    Plan saved = h->plan;
    h->plan = p;
    int rc = build_tables(h);
    if (rc != ISING_OK) {
        h->plan = saved;
        build_tables(h);
        return rc;
    }
    return ISING_OK;
}

namespace {

struct TuneCand {
    int mode, V, R, k, threads;
};

std::string tune_key(const ising_handle* h) {
    std::vector<int> Ls = h->L;
    std::sort(Ls.begin(), Ls.end());
    std::string key;
    int run = 0;
    for (size_t i = 0; i < Ls.size(); ++i) {
        ++run;
        if (i + 1 == Ls.size() || Ls[i + 1] != Ls[i]) {
            key += std::to_string(Ls[i]) + "x" + std::to_string(run) + ",";
            run = 0;
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    key += "sm" + std::to_string(prop.major * 10 + prop.minor) + "n" + std::to_string(prop.multiProcessorCount);
    return key;
}

bool tune_cache_lookup(const std::string& key, TuneCand* c) {
    const char* path = getenv("ISING_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char kbuf[4096];
    TuneCand t{};
    bool found = false;
    while (fscanf(f, "%4095s %d %d %d %d %d", kbuf, &t.mode, &t.V, &t.R, &t.k, &t.threads) == 6)
        if (key == kbuf) { *c = t; found = true; }
    fclose(f);
    return found;
}

void tune_cache_store(const std::string& key, const TuneCand& c) {
    const char* path = getenv("ISING_TUNE_CACHE");
    if (!path || !*path || key.size() >= 4000) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), c.mode, c.V, c.R, c.k, c.threads);
    fclose(f);
}

int apply_cand(ising_handle* h, const TuneCand& c) {
    return ising_set_plan(h, c.mode, c.V, c.R, c.k, c.threads);
}

}  // namespace

int ising_autotune(ising_t h, int64_t probe_sweeps, int force, double* best_flips_per_ns) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (probe_sweeps < 1) return fail(ISING_EINVAL, "probe_sweeps must be >= 1");
    if (best_flips_per_ns) *best_flips_per_ns = 0.0;
    if (h->n == 0) return ISING_OK;
    const std::string key = tune_key(h);
    TuneCand cached{};
    if (!force && tune_cache_lookup(key, &cached)) {
        int rc = apply_cand(h, cached);
        if (rc == ISING_OK) return ISING_OK;
    }
    // candidates: the resident kernel with several unit sizes and block sizes
    // when some lattice has L <= 1024 (RESIDENT if all do, else MIXED), and
    // the streaming and persistent kernels with several tilings
    std::vector<TuneCand> cands;
    bool all_small = true, any_small = false;
    for (int L : h->L) {
        all_small &= (L <= 1024);
        any_small |= (L <= 1024);
    }
    if (any_small)
        for (int k : {8, 32, 128})
            for (int thr : {0, 256, 512})
                cands.push_back({all_small ? ISING_PLAN_RESIDENT : ISING_PLAN_MIXED, 0, 0, k, thr});
    if (all_small)
        for (int rows : {32, 64, 128}) cands.push_back({ISING_PLAN_CLUSTER, 0, rows, 0, 0});
    const int Vs[] = {1, 2, 4};
    for (int V : Vs) {
        bool ok = true;
        for (int L : h->L) ok &= ((L / 64) % V == 0);
        if (!ok) continue;
        for (int R : {1, 2, 4, 8})
            for (int thr : {128, 256}) {
                cands.push_back({ISING_PLAN_STREAM, V, R, 0, thr});
                cands.push_back({ISING_PLAN_PERSIST, V, R, 0, thr});
            }
    }
    size_t nbytes = 0;
    int rc = ising_state_bytes(h, &nbytes);
    if (rc != ISING_OK) return rc;
    std::vector<char> saved(nbytes);
    rc = ising_save(h, saved.data(), nbytes);
    if (rc != ISING_OK) return rc;
    const Plan plan0 = h->plan;   // candidates are timed the way sweeps will run (graph replay or not)
    double sites = 0;
    for (int L : h->L) sites += (double)L * L;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0), "event");
    CUDA_TRY(cudaEventCreate(&e1), "event");
    double best = -1.0;
    TuneCand best_c{};
    for (const TuneCand& c : cands) {
        if (apply_cand(h, c) != ISING_OK) continue;
        if (ising_load(h, saved.data(), nbytes) != ISING_OK) break;
        if (ising_sweep(h, probe_sweeps) != ISING_OK) continue;      // warm-up (captures the graph if on)
        if (ising_load(h, saved.data(), nbytes) != ISING_OK) break;
        cudaEventRecord(e0, h->stream);
        if (ising_sweep(h, probe_sweeps) != ISING_OK) continue;
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = sites * (double)probe_sweeps / ((double)ms * 1e6);
        if (rate > best) { best = rate; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        h->plan = plan0;
        build_tables(h);
        ising_load(h, saved.data(), nbytes);
        return fail(ISING_ECUDA, "autotune: no candidate ran");
    }
    rc = apply_cand(h, best_c);
    if (rc != ISING_OK) return rc;
    rc = ising_load(h, saved.data(), nbytes);   // the state is as before tuning
    if (rc != ISING_OK) return rc;
    tune_cache_store(key, best_c);
    if (best_flips_per_ns) *best_flips_per_ns = best;
    return ISING_OK;
}

int ising_get_plan(ising_t h, int* plan, int* words_per_thread, int* rows_per_item, int* sweeps_per_unit,
                   int* threads) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (plan) *plan = h->plan.mode;
    if (words_per_thread) *words_per_thread = h->V;
    if (rows_per_item) *rows_per_item = h->R;
    if (sweeps_per_unit) *sweeps_per_unit = h->plan.sweeps_per_unit;
    if (threads)
        *threads = (h->plan.mode == ISING_PLAN_STREAM || h->plan.mode == ISING_PLAN_PERSIST ||
                    h->plan.mode == ISING_PLAN_AUTO) ? h->plan.stream_threads
                   : h->plan.mode == ISING_PLAN_CLUSTER ? 256 : h->res_threads;
    return ISING_OK;
}

int ising_set_graph(ising_t h, int on) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (on && h->stream == nullptr) return fail(ISING_ESTATE, "graph replay needs a non-default stream");
    h->graph = on != 0;
    if (!h->graph) drop_graphs(h);
    return ISING_OK;
}

void ising_destroy(ising_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    delete h;
}

}  // extern "C"

extern "C" int ising_random_stream(uint64_t seed, uint32_t s, uint32_t phase, uint64_t p0, uint64_t n_p, uint32_t t0,
                                   uint32_t n_t, uint32_t* dev_out, void* cuda_stream) {
    if (!dev_out) return fail(ISING_EINVAL, "dev_out is NULL");
    if (((uintptr_t)dev_out) % 16 != 0) return fail(ISING_EINVAL, "dev_out must be 16-byte aligned");
    if (p0 + n_p < p0 || p0 + n_p > (1ull << 34)) return fail(ISING_EINVAL, "sites beyond 2^34");
    if ((uint64_t)t0 + n_t > (1ull << 32)) return fail(ISING_EINVAL, "sweeps beyond 2^32");
    if (n_p > 0 && n_t > 0 && n_p > (uint64_t)-1 / n_t) return fail(ISING_EINVAL, "n_p * n_t overflows");
    CUDA_TRY(launch_random_stream((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), s, phase, p0, n_p, t0, n_t,
                                  dev_out, (cudaStream_t)cuda_stream), "random stream kernel");
    return ISING_OK;
}

// ===========================================================================
// Swendsen-Wang cluster step (kernels in ising_cluster.cu)
// ===========================================================================
namespace {

constexpr int kSwTileSites = kSwTileW * kSwTileH;
constexpr int kSwKernels = 6;   // local, merge, resolve, flip, observables, record (with the E/M finish)

struct SwLayout {
    size_t lat = 0, edges = 0, coins = 0, label = 0, seeds = 0, total = 0;
};

// bond threshold floor(2^32 (1 - exp(-2/T))), at most 2^32 - 1
uint32_t sw_threshold_u32(double T) {
    const double v = std::ldexp(-std::expm1(-2.0 / T), 32);
    if (v >= 4294967296.0) return 0xFFFFFFFFu;
    return (uint32_t)std::floor(v);
}

int sw_build_table(ising_handle* h) {
    if (!h->sw_table.empty() || h->n == 0) return ISING_OK;
    uint64_t tiles = 0, sites = 0;
    std::vector<SwLat> tab((size_t)h->n);
    for (int i = 0; i < h->n; ++i) {
        if (h->L[i] > ISING_SW_MAX_L)
            return fail(ISING_EINVAL, "lattice %d: the cluster step takes L <= %d (L=%d)", i, ISING_SW_MAX_L, h->L[i]);
        SwLat d{};
        d.word_off = h->layout.word_off[i];
        d.site_off = sites;
        d.L = (uint32_t)h->L[i];
        d.wn = (uint32_t)(h->L[i] / 64);
        d.sim = (uint32_t)i;
        d.key0 = (uint32_t)(h->seed[i] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(h->seed[i] >> 32);
        d.thr = sw_threshold_u32(h->T[i]);
        d.tile_begin = (uint32_t)tiles;
        tab[i] = d;
        const uint64_t n2 = (uint64_t)h->L[i] * (uint64_t)h->L[i];
        sites += n2;
        tiles += n2 / kSwTileSites;
        if (tiles >= 0x7FFFFFFFull) return fail(ISING_EINVAL, "too many sites for one cluster step");
    }
    h->sw_tiles = tiles;
    h->sw_sites = sites;
    h->sw_table = std::move(tab);
    return ISING_OK;
}

SwLayout sw_layout(const ising_handle* h) {
    SwLayout l;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    l.lat = take((size_t)h->n * sizeof(SwLat));
    l.edges = take((size_t)h->sw_tiles * sizeof(uint4));
    l.coins = take((size_t)(h->sw_sites / 32) * sizeof(uint32_t));
    l.label = take((size_t)h->sw_sites * sizeof(uint32_t));
    l.seeds = take((size_t)h->n * sizeof(uint32_t));
    l.total = off;
    return l;
}

// Validate the scratch, upload the table, fill sw.
int sw_prepare(ising_handle* h, void* scratch, size_t bytes, SwState* sw) {
    int rc = sw_build_table(h);
    if (rc != ISING_OK) return rc;
    const SwLayout l = sw_layout(h);
    if (!scratch) return fail(ISING_EINVAL, "scratch is NULL");
    if (((uintptr_t)scratch) % kAlign != 0) return fail(ISING_EINVAL, "scratch must be 256-byte aligned");
    if (bytes < l.total) return fail(ISING_ENOMEM, "cluster scratch too small: %zu bytes given, %zu needed", bytes, l.total);
    char* base = (char*)scratch;
    // the table is tiny: upload it on every call, so that a scratch that was
    // freed and reallocated at the same address never runs with a stale one
    // (the host copy lives as long as the handle)
    CUDA_TRY(cudaMemcpyAsync(base + l.lat, h->sw_table.data(), h->sw_table.size() * sizeof(SwLat),
                             cudaMemcpyHostToDevice, h->stream), "upload cluster table");
    sw->lat = (const SwLat*)(base + l.lat);
    sw->n = h->n;
    sw->total_tiles = (uint32_t)h->sw_tiles;
    sw->edges = (uint4*)(base + l.edges);
    sw->coins = (uint32_t*)(base + l.coins);
    sw->label = (uint32_t*)(base + l.label);
    sw->bond_phase = kSwBondPhase;           // Wolff by labelling sets kWolffBondPhase
    sw->seed_root = nullptr;
    h->sw_seed_area = (uint32_t*)(base + l.seeds);
    return ISING_OK;
}

int enqueue_sw(ising_handle* h, const SwState& sw, int64_t n) {
    const uint32_t* list = (const uint32_t*)(h->ws + h->layout.list);
    const uint32_t max_L = (uint32_t)*std::max_element(h->L.begin(), h->L.end());
    for (int64_t i = 0; i < n; ++i) {
        CUDA_TRY(launch_sw_clusters(h->st, sw, h->stream), "cluster labelling");
        CUDA_TRY(launch_sw_flip(h->st, sw, h->stream), "cluster flip");
        CUDA_TRY(launch_observables(h->st, max_L, list, h->n, h->stream, false), "observables");
        CUDA_TRY(launch_sw_record(h->st, h->n, h->stream), "record");
    }
    return ISING_OK;
}

}  // namespace

extern "C" {

int ising_sw_scratch_bytes(ising_t h, size_t* bytes) {
    if (!h || !bytes) return fail(ISING_EINVAL, "handle or bytes is NULL");
    int rc = sw_build_table(h);
    if (rc != ISING_OK) return rc;
    *bytes = sw_layout(h).total;
    return ISING_OK;
}

int ising_sw_get_thresholds(ising_t h, uint32_t* thr) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (h->n > 0 && !thr) return fail(ISING_EINVAL, "thr is NULL");
    for (int i = 0; i < h->n; ++i) thr[i] = sw_threshold_u32(h->T[i]);
    return ISING_OK;
}

int ising_sw_sweep(ising_t h, int64_t n, void* dev_scratch, size_t scratch_bytes) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (n < 0) return fail(ISING_EINVAL, "n must be >= 0");
    if (h->n == 0) return ISING_OK;
    if (h->t + n > (int64_t)0xFFFFFFFFll)
        return fail(ISING_EINVAL, "sweep counter would pass 2^32 (Philox counter word 1)");
    SwState sw{};
    int rc = sw_prepare(h, dev_scratch, scratch_bytes, &sw);
    if (rc != ISING_OK || n == 0) return rc;
    if (h->graph) {
        if (h->stream == nullptr) return fail(ISING_ESTATE, "graph replay needs a non-default stream");
        const auto key = std::make_pair(n, (const void*)dev_scratch);
        auto it = h->sw_graphs.find(key);
        if (it == h->sw_graphs.end()) {
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            rc = enqueue_sw(h, sw, n);
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (rc != ISING_OK) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            it = h->sw_graphs.emplace(key, ex).first;
        }
        CUDA_TRY(cudaGraphLaunch(it->second, h->stream), "graph launch");
    } else {
        rc = enqueue_sw(h, sw, n);
        if (rc != ISING_OK) return rc;
    }
    h->t += n;
    h->launches += kSwKernels * n;
    return ISING_OK;
}

namespace {

// Wolff steps by labelling: the Swendsen-Wang labelling of the Wolff bonds
// (phase 10), the seed's root, the seed's component flipped; E and M from the
// observables kernel, recorded as after a sweep.
int enqueue_wolff_labels(ising_handle* h, const SwState& sw, int64_t n) {
    const uint32_t* list = (const uint32_t*)(h->ws + h->layout.list);
    const uint32_t max_L = (uint32_t)*std::max_element(h->L.begin(), h->L.end());
    for (int64_t i = 0; i < n; ++i) {
        CUDA_TRY(launch_wolff_clusters(h->st, sw, h->stream), "Wolff cluster labelling");
        CUDA_TRY(launch_sw_flip(h->st, sw, h->stream), "Wolff cluster flip");
        CUDA_TRY(launch_observables(h->st, max_L, list, h->n, h->stream, false), "observables");
        CUDA_TRY(launch_sw_record(h->st, h->n, h->stream), "record");
    }
    return ISING_OK;
}

// The way ising_wolff_sweep runs: growth, or labelling (when some lattice is
// at T < kWolffLabelsBelowT under the automatic choice).
constexpr double kWolffLabelsBelowT = 2.3;
bool wolff_by_labels(const ising_handle* h) {
    if (h->wolff_method == ISING_WOLFF_LABELS) return true;
    if (h->wolff_method == ISING_WOLFF_GROWTH) return false;
    return *std::min_element(h->T.begin(), h->T.end()) < kWolffLabelsBelowT;
}

}  // namespace

int ising_wolff_sweep(ising_t h, int64_t n, void* dev_scratch, size_t scratch_bytes) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (n < 0) return fail(ISING_EINVAL, "n must be >= 0");
    if (h->n == 0) return ISING_OK;
    if (h->t + n > (int64_t)0xFFFFFFFFll)
        return fail(ISING_EINVAL, "sweep counter would pass 2^32 (Philox counter word 1)");
    SwState sw{};
    int rc = sw_prepare(h, dev_scratch, scratch_bytes, &sw);
    if (rc != ISING_OK || n == 0) return rc;
    if (wolff_by_labels(h)) {
        sw.bond_phase = kWolffBondPhase;
        sw.seed_root = h->sw_seed_area;
        if (h->graph) {
            if (h->stream == nullptr) return fail(ISING_ESTATE, "graph replay needs a non-default stream");
            const auto key = std::make_pair(n, (const void*)dev_scratch);
            auto it = h->wolff_graphs.find(key);
            if (it == h->wolff_graphs.end()) {
                cudaGraph_t g = nullptr;
                CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                rc = enqueue_wolff_labels(h, sw, n);
                cudaError_t e = cudaStreamEndCapture(h->stream, &g);
                if (rc != ISING_OK) { if (g) cudaGraphDestroy(g); return rc; }
                if (e != cudaSuccess) return cuda_fail(e, "end capture");
                cudaGraphExec_t ex = nullptr;
                e = cudaGraphInstantiate(&ex, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
                it = h->wolff_graphs.emplace(key, ex).first;
            }
            CUDA_TRY(cudaGraphLaunch(it->second, h->stream), "graph launch");
        } else {
            rc = enqueue_wolff_labels(h, sw, n);
            if (rc != ISING_OK) return rc;
        }
        h->t += n;
        h->launches += 7 * n;
        return ISING_OK;
    }
    // growth: the visited bits (the coin region of the scratch) start at
    // zero; each step clears the bits it set
    CUDA_TRY(cudaMemsetAsync(sw.coins, 0, (size_t)(h->sw_sites / 8), h->stream), "clear visited bits");
    uint32_t max_small = 0;
    bool any_large = false;
    for (int L : h->L) {
        if ((uint32_t)L <= wolff_smem_max_L()) max_small = std::max(max_small, (uint32_t)L);
        else any_large = true;
    }
    CUDA_TRY(launch_wolff(h->st, sw, n, max_small, any_large, h->stream), "Wolff steps");
    CUDA_TRY(launch_advance_t(h->st, n, h->stream), "advance sweep counter");
    h->t += n;
    h->launches += 2;
    return ISING_OK;
}

int ising_wolff_set_method(ising_t h, int method) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (method != ISING_WOLFF_AUTO && method != ISING_WOLFF_GROWTH && method != ISING_WOLFF_LABELS)
        return fail(ISING_EINVAL, "unknown Wolff method %d", method);
    h->wolff_method = method;
    return ISING_OK;
}

int ising_sw_labels(ising_t h, int sim, void* dev_scratch, size_t scratch_bytes, uint32_t* host_labels) {
    if (!h) return fail(ISING_EINVAL, "handle is NULL");
    if (sim < 0 || sim >= h->n) return fail(ISING_EINVAL, "sim %d out of range", sim);
    if (!host_labels) return fail(ISING_EINVAL, "host_labels is NULL");
    SwState sw{};
    int rc = sw_prepare(h, dev_scratch, scratch_bytes, &sw);
    if (rc != ISING_OK) return rc;
    CUDA_TRY(launch_sw_clusters(h->st, sw, h->stream), "cluster labelling");
    CUDA_TRY(launch_sw_compress(sw, h->stream), "label compression");
    h->launches += 4;
    const SwLat& d = h->sw_table[sim];
    CUDA_TRY(cudaMemcpyAsync(host_labels, sw.label + d.site_off, (size_t)d.L * d.L * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, h->stream), "copy labels");
    return check_device_error(h);
}

}  // extern "C"

// ===========================================================================
// Learned patch proposal: network handle and round
// ===========================================================================
struct ising_net {
    int max_windows = 0, max_lattices = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    NetState ns{};
    int8_t* win = nullptr;
    int8_t* win2 = nullptr;
    float* z = nullptr;
    float* lq = nullptr;
    float* lq2 = nullptr;
    __nv_bfloat16* h = nullptr;
    LearnedKey* keys = nullptr;
    LearnedLat* ll = nullptr;
    unsigned long long* accepted = nullptr;
    int step = 0;
    int precision = ISING_NET_BF16;
    bool fp8_stale = true;                        // masters changed since the e4m3 copy was made
    const ising_handle* table_owner = nullptr;   // handle whose lattice table is on the device
    std::vector<LearnedLat> table;
    int table_windows = 0;
};

namespace {

struct NetLayout {
    size_t w, m, v, g, wb, loss, wq, wscale, win, win2, z, lq, lq2, h, keys, ll, acc, total;
};

NetLayout net_layout(int W, int NB, int NL) {
    NetLayout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t P = ISING_NET_PARAMS, w = (size_t)W;
    l.w = take(P * 4); l.m = take(P * 4); l.v = take(P * 4); l.g = take(P * 4); l.wb = take(P * 2);
    l.loss = take(16);
    l.wq = take(P);
    l.wscale = take(16);
    l.win = take(w * 100); l.win2 = take(w * 100);
    l.z = take((size_t)NB * 100 * 4);
    l.lq = take(w * 4); l.lq2 = take(w * 4);
    l.h = take(3 * (size_t)NB * 100 * 16 * 2);
    l.keys = take(w * sizeof(LearnedKey));
    l.ll = take((size_t)NL * sizeof(LearnedLat));
    l.acc = take((size_t)NL * 8);
    l.total = off;
    return l;
}

int net_upload_windows(ising_net* net, const int8_t* host, int n) {
    if (n < 1 || n > net->max_windows) return fail(ISING_EINVAL, "n must be in [1, max_windows=%d]", net->max_windows);
    if (!host) return fail(ISING_EINVAL, "windows is NULL");
    for (size_t i = 0; i < (size_t)n * 100; ++i)
        if (host[i] != 1 && host[i] != -1) return fail(ISING_EINVAL, "window spins must be +1/-1");
    CUDA_TRY(cudaMemcpyAsync(net->win, host, (size_t)n * 100, cudaMemcpyHostToDevice, net->stream), "upload windows");
    return ISING_OK;
}

// Per-layer power-of-two scales of the e4m3 weight copy: the largest |W| of a
// layer times its scale is at most 448 (the largest finite e4m3 value).
int net_refresh_fp8(ising_net* net) {
    if (!net->fp8_stale) return ISING_OK;
    std::vector<float> w(ISING_NET_PARAMS);
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    CUDA_TRY(cudaMemcpy(w.data(), net->ns.w, w.size() * sizeof(float), cudaMemcpyDeviceToHost), "read params");
    const int lo[4] = {0, 272, 1568, 2864}, hi[4] = {256, 1552, 2848, 2944};
    float scale[4];
    for (int l = 0; l < 4; ++l) {
        double mx = 0.0;
        for (int i = lo[l]; i < hi[l]; ++i) mx = std::max(mx, (double)std::fabs(w[i]));
        double e = mx > 0.0 ? std::floor(std::log2(448.0 / mx)) : 0.0;
        e = std::min(std::max(e, -60.0), 60.0);
        scale[l] = (float)std::ldexp(1.0, (int)e);
    }
    CUDA_TRY(cudaMemcpy(net->ns.wscale, scale, sizeof(scale), cudaMemcpyHostToDevice), "upload scales");
    CUDA_TRY(launch_to_fp8(net->ns, net->stream), "e4m3 copy");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    net->fp8_stale = false;
    return ISING_OK;
}

// log q (and logits) of n windows on the tensor cores, in the net's precision
cudaError_t net_score(ising_net* net, const int8_t* win, int n, float* lq, float* z, cudaStream_t st) {
    return launch_net_score_tc(net->ns, net->precision == ISING_NET_FP8, win, n, lq, z, nullptr, nullptr, st);
}

// ISING_ETIMEOUT if a bounded wait of a tensor-core kernel ran out (reads the
// flag after the stream's work so far; synchronises)
int net_check_error(ising_net* net, cudaStream_t st) {
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, net->ns.err, sizeof(int), cudaMemcpyDeviceToHost, st), "read error flag");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
    if (err != 0) return fail(ISING_ETIMEOUT, "a bounded wait of the tensor-core scoring kernel ran out");
    return ISING_OK;
}

cudaError_t net_sample(ising_net* net, int8_t* win, int n, float* lq, uint32_t round_t, cudaStream_t st) {
    if (net->precision == ISING_NET_FP8) return launch_net_sample_fp8(net->ns, win, n, lq, net->keys, round_t, st);
    return launch_net_sample(net->ns, win, n, lq, net->keys, round_t, st);
}

}  // namespace

extern "C" {

int ising_net_set_precision(ising_net_t net, int precision) {
    if (!net) return fail(ISING_EINVAL, "net is NULL");
    if (precision != ISING_NET_BF16 && precision != ISING_NET_FP8)
        return fail(ISING_EINVAL, "precision must be ISING_NET_BF16 or ISING_NET_FP8");
    net->precision = precision;
    if (precision == ISING_NET_FP8) return net_refresh_fp8(net);
    return ISING_OK;
}

int ising_net_workspace_bytes(int max_windows, int max_batch, int max_lattices, size_t* bytes) {
    if (!bytes || max_windows < 1 || max_batch < 1 || max_lattices < 1)
        return fail(ISING_EINVAL, "max_windows, max_batch and max_lattices must be >= 1");
    *bytes = net_layout(max_windows, max_batch, max_lattices).total;
    return ISING_OK;
}

int ising_net_create(ising_net_t* out, int max_windows, int max_batch, int max_lattices, void* dev_ws,
                     size_t ws_bytes, void* cuda_stream) {
    if (!out) return fail(ISING_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_windows < 1 || max_batch < 1 || max_lattices < 1)
        return fail(ISING_EINVAL, "max_windows, max_batch and max_lattices must be >= 1");
    const NetLayout l = net_layout(max_windows, max_batch, max_lattices);
    if (ws_bytes < l.total) return fail(ISING_ENOMEM, "net workspace too small: %zu < %zu", ws_bytes, l.total);
    if (!dev_ws || ((uintptr_t)dev_ws) % kAlign) return fail(ISING_EINVAL, "workspace NULL or not 256-byte aligned");
    CUDA_TRY(configure_learned_kernels(), "configure learned kernels");
    auto* net = new ising_net();
    char* b = (char*)dev_ws;
    net->max_windows = max_windows;
    net->max_batch = max_batch;
    net->max_lattices = max_lattices;
    net->stream = (cudaStream_t)cuda_stream;
    net->ws = b;
    net->ns = NetState{(float*)(b + l.w), (float*)(b + l.m), (float*)(b + l.v), (float*)(b + l.g),
                       (__nv_bfloat16*)(b + l.wb), (float*)(b + l.loss), (uint8_t*)(b + l.wq),
                       (float*)(b + l.wscale), (int*)(b + l.loss + 8)};
    net->win = (int8_t*)(b + l.win);
    net->win2 = (int8_t*)(b + l.win2);
    net->z = (float*)(b + l.z);
    net->lq = (float*)(b + l.lq);
    net->lq2 = (float*)(b + l.lq2);
    net->h = (__nv_bfloat16*)(b + l.h);
    net->keys = (LearnedKey*)(b + l.keys);
    net->ll = (LearnedLat*)(b + l.ll);
    net->accepted = (unsigned long long*)(b + l.acc);
    cudaError_t e = cudaMemsetAsync(b, 0, l.total, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) { delete net; return cuda_fail(e, "net create"); }
    *out = net;
    return ISING_OK;
}

void ising_net_destroy(ising_net_t net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    delete net;
}

int ising_net_set_params(ising_net_t net, const float* host) {
    if (!net || !host) return fail(ISING_EINVAL, "NULL argument");
    for (int i = 0; i < ISING_NET_PARAMS; ++i)
        if (!std::isfinite(host[i])) return fail(ISING_EINVAL, "parameter %d is not finite", i);
    const size_t nb = ISING_NET_PARAMS * sizeof(float);
    CUDA_TRY(cudaMemcpyAsync(net->ns.w, host, nb, cudaMemcpyHostToDevice, net->stream), "set params");
    CUDA_TRY(cudaMemsetAsync(net->ns.m, 0, nb, net->stream), "zero m");
    CUDA_TRY(cudaMemsetAsync(net->ns.v, 0, nb, net->stream), "zero v");
    CUDA_TRY(launch_to_bf16(net->ns, net->stream), "bf16 copy");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    net->step = 0;
    net->fp8_stale = true;
    if (net->precision == ISING_NET_FP8) return net_refresh_fp8(net);
    return ISING_OK;
}

int ising_net_get_params(ising_net_t net, float* host) {
    if (!net || !host) return fail(ISING_EINVAL, "NULL argument");
    CUDA_TRY(cudaMemcpyAsync(host, net->ns.w, ISING_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, net->stream),
             "get params");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    return ISING_OK;
}

int ising_net_score(ising_net_t net, const int8_t* host_windows, int n, float* host_logq, float* host_z) {
    if (!net || !host_logq) return fail(ISING_EINVAL, "NULL argument");
    if (host_z && n > net->max_batch) return fail(ISING_EINVAL, "logits need n <= max_batch=%d", net->max_batch);
    int rc = net_upload_windows(net, host_windows, n);
    if (rc != ISING_OK) return rc;
    CUDA_TRY(net_score(net, net->win, n, net->lq, host_z ? net->z : nullptr, net->stream), "score");
    CUDA_TRY(cudaMemcpyAsync(host_logq, net->lq, (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream), "copy logq");
    if (host_z)
        CUDA_TRY(cudaMemcpyAsync(host_z, net->z, (size_t)n * 400, cudaMemcpyDeviceToHost, net->stream), "copy z");
    return net_check_error(net, net->stream);
}

int ising_net_sample(ising_net_t net, int8_t* host_windows, int n, const uint32_t* host_keys, uint32_t round_index,
                     float* host_logq) {
    if (!net || !host_keys || !host_logq) return fail(ISING_EINVAL, "NULL argument");
    int rc = net_upload_windows(net, host_windows, n);
    if (rc != ISING_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(net->keys, host_keys, (size_t)n * sizeof(LearnedKey), cudaMemcpyHostToDevice,
                             net->stream), "upload keys");
    CUDA_TRY(net_sample(net, net->win, n, net->lq, round_index, net->stream), "sample");
    CUDA_TRY(cudaMemcpyAsync(host_windows, net->win, (size_t)n * 100, cudaMemcpyDeviceToHost, net->stream),
             "copy windows");
    CUDA_TRY(cudaMemcpyAsync(host_logq, net->lq, (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream), "copy logq");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    return ISING_OK;
}

int ising_net_grad(ising_net_t net, const int8_t* host_windows, int n, float* host_grad, float* host_loss) {
    if (!net || !host_grad) return fail(ISING_EINVAL, "NULL argument");
    if (n > net->max_batch) return fail(ISING_EINVAL, "n must be <= max_batch=%d", net->max_batch);
    int rc = net_upload_windows(net, host_windows, n);
    if (rc != ISING_OK) return rc;
    CUDA_TRY(cudaMemsetAsync(net->ns.g, 0, ISING_NET_PARAMS * sizeof(float), net->stream), "zero grad");
    CUDA_TRY(cudaMemsetAsync(net->ns.loss, 0, sizeof(float), net->stream), "zero loss");
    CUDA_TRY(launch_net_forward(net->ns, net->win, n, net->lq, net->z, net->h, net->stream), "forward");
    CUDA_TRY(launch_net_backward(net->ns, net->win, n, net->z, net->h, net->ns.g, net->ns.loss, net->stream),
             "backward");
    CUDA_TRY(cudaMemcpyAsync(host_grad, net->ns.g, ISING_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost,
                             net->stream), "copy grad");
    if (host_loss)
        CUDA_TRY(cudaMemcpyAsync(host_loss, net->ns.loss, sizeof(float), cudaMemcpyDeviceToHost, net->stream),
                 "copy loss");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    return ISING_OK;
}

int ising_net_train(ising_net_t net, const void* dev_pool_words, int n_snap, int L, int64_t steps, int batch,
                    float lr, uint64_t seed, float* host_losses) {
    if (!net || !dev_pool_words) return fail(ISING_EINVAL, "NULL argument");
    if (n_snap < 1 || !valid_L(L)) return fail(ISING_EINVAL, "need n_snap >= 1 and a valid L");
    if (batch < 1 || batch > net->max_batch || batch > net->max_windows)
        return fail(ISING_EINVAL, "batch must be in [1, min(max_batch, max_windows)]");
    if (steps < 0 || !(lr > 0.f) || !std::isfinite(lr)) return fail(ISING_EINVAL, "invalid steps or lr");
    std::vector<float> losses;
    for (int64_t s = 0; s < steps; ++s) {
        const uint32_t step_id = (uint32_t)(net->step);
        CUDA_TRY(launch_train_windows((const uint32_t*)dev_pool_words, n_snap, (uint32_t)L, batch, seed, step_id,
                                      net->win, net->stream), "training windows");
        CUDA_TRY(cudaMemsetAsync(net->ns.g, 0, ISING_NET_PARAMS * sizeof(float), net->stream), "zero grad");
        CUDA_TRY(cudaMemsetAsync(net->ns.loss, 0, sizeof(float), net->stream), "zero loss");
        CUDA_TRY(launch_net_forward(net->ns, net->win, batch, net->lq, net->z, net->h, net->stream), "forward");
        CUDA_TRY(launch_net_backward(net->ns, net->win, batch, net->z, net->h, net->ns.g, net->ns.loss, net->stream),
                 "backward");
        net->step += 1;
        CUDA_TRY(launch_adam(net->ns, lr, net->step, net->stream), "adam");
        if (host_losses)
            CUDA_TRY(cudaMemcpyAsync(host_losses + s, net->ns.loss, sizeof(float), cudaMemcpyDeviceToHost,
                                     net->stream), "copy loss");
    }
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    net->fp8_stale = true;
    if (net->precision == ISING_NET_FP8 && steps > 0) return net_refresh_fp8(net);
    return ISING_OK;
}

int ising_net_train_windows(ising_net_t net, const void* dev_pool_words, int n_snap, int L, int64_t step,
                            int batch, uint64_t seed, int8_t* host_windows) {
    if (!net || !dev_pool_words || !host_windows) return fail(ISING_EINVAL, "NULL argument");
    if (n_snap < 1 || !valid_L(L)) return fail(ISING_EINVAL, "need n_snap >= 1 and a valid L");
    if (batch < 1 || batch > net->max_windows) return fail(ISING_EINVAL, "batch must be in [1, max_windows=%d]",
                                                           net->max_windows);
    if (step < 0 || step > (int64_t)0xFFFFFFFFll) return fail(ISING_EINVAL, "step must be in [0, 2^32)");
    CUDA_TRY(launch_train_windows((const uint32_t*)dev_pool_words, n_snap, (uint32_t)L, batch, seed, (uint32_t)step,
                                  net->win, net->stream), "training windows");
    CUDA_TRY(cudaMemcpyAsync(host_windows, net->win, (size_t)batch * 100, cudaMemcpyDeviceToHost, net->stream),
             "copy windows");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    return ISING_OK;
}

int ising_net_apply_grad(ising_net_t net, const float* host_grad, float lr) {
    if (!net || !host_grad) return fail(ISING_EINVAL, "NULL argument");
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(ISING_EINVAL, "lr must be positive and finite");
    for (int i = 0; i < ISING_NET_PARAMS; ++i)
        if (!std::isfinite(host_grad[i])) return fail(ISING_EINVAL, "gradient entry %d is not finite", i);
    CUDA_TRY(cudaMemcpyAsync(net->ns.g, host_grad, ISING_NET_PARAMS * sizeof(float), cudaMemcpyHostToDevice,
                             net->stream), "upload gradient");
    net->step += 1;
    CUDA_TRY(launch_adam(net->ns, lr, net->step, net->stream), "adam");
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");   // the host gradient may go out of scope
    net->fp8_stale = true;
    if (net->precision == ISING_NET_FP8) return net_refresh_fp8(net);
    return ISING_OK;
}

int ising_learned_round(ising_t h, ising_net_t net, int64_t round_index, int64_t* host_accepted) {
    if (!h || !net) return fail(ISING_EINVAL, "NULL handle");
    if (round_index < 0 || round_index > (int64_t)0xFFFFFFFFll) return fail(ISING_EINVAL, "round_index out of range");
    if (h->n == 0) return ISING_OK;
    if (h->n > net->max_lattices) return fail(ISING_EINVAL, "handle has %d lattices, net allows %d", h->n, net->max_lattices);
    // the lattice table depends only on the handle: upload it when the handle
    // changes, from a host copy that lives as long as the net
    if (net->table_owner != h) {
        net->table.assign(h->n, LearnedLat{});
        int64_t nwin = 0;
        for (int i = 0; i < h->n; ++i) {
            LearnedLat d{};
            d.word_off = h->layout.word_off[i];
            d.L = (uint32_t)h->L[i];
            d.lat = (uint32_t)i;
            d.sim = (uint32_t)i;
            d.key0 = (uint32_t)(h->seed[i] & 0xFFFFFFFFull);
            d.key1 = (uint32_t)(h->seed[i] >> 32);
            d.patch_begin = (uint32_t)nwin;
            d.beta = 1.0 / h->T[i];
            net->table[i] = d;
            nwin += (int64_t)(h->L[i] / 16) * (h->L[i] / 16);
        }
        if (nwin > net->max_windows)
            return fail(ISING_EINVAL, "round needs %lld windows, net allows %d", (long long)nwin, net->max_windows);
        CUDA_TRY(cudaStreamSynchronize(h->stream), "synchronize");
        CUDA_TRY(cudaMemcpy(net->ll, net->table.data(), net->table.size() * sizeof(LearnedLat), cudaMemcpyHostToDevice),
                 "upload lattice table");
        CUDA_TRY(cudaMemset(net->accepted, 0, (size_t)net->max_lattices * 8), "zero counters");
        net->table_owner = h;
        net->table_windows = (int)nwin;
    }
    static const uint32_t off[4][2] = {{0, 0}, {8, 8}, {0, 8}, {8, 0}};
    const uint32_t ox = off[round_index % 4][0], oy = off[round_index % 4][1];
    const uint32_t rt = (uint32_t)round_index;
    const int nwin = net->table_windows;
    if (host_accepted)
        CUDA_TRY(cudaMemsetAsync(net->accepted, 0, (size_t)h->n * 8, h->stream), "zero counters");
    CUDA_TRY(launch_gather_patches(h->st, net->ll, h->n, nwin, ox, oy, net->win, net->win2, net->keys, h->stream),
             "gather patches");
    // the sampler's own log q is not needed: both patches are scored below
    CUDA_TRY(net_sample(net, net->win2, nwin, net->precision == ISING_NET_FP8 ? net->lq2 : nullptr, rt, h->stream),
             "sample");
    // log q of the current and of the proposed patch from the same function,
    // in one launch of the tensor-core scoring kernel (in the net's precision)
    CUDA_TRY(launch_net_score_tc(net->ns, net->precision == ISING_NET_FP8, net->win, nwin, net->lq, nullptr, net->win2,
                                 net->lq2, h->stream), "score");
    CUDA_TRY(launch_mh_apply(h->st, net->ll, h->n, nwin, ox, oy, net->win, net->win2, net->lq, net->lq2, rt,
                             net->accepted, h->stream), "accept");
    if (host_accepted) {
        std::vector<unsigned long long> acc(h->n);
        CUDA_TRY(cudaMemcpyAsync(acc.data(), net->accepted, (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream),
                 "copy counters");
        int rc = net_check_error(net, h->stream);
        if (rc != ISING_OK) return rc;
        for (int i = 0; i < h->n; ++i) host_accepted[i] = (int64_t)acc[i];
        CUDA_TRY(cudaMemsetAsync(net->accepted, 0, (size_t)h->n * 8, h->stream), "zero counters");
    }
    return ISING_OK;
}

int ising_net_accepted(ising_net_t net, int64_t* host_accepted, int n, int reset) {
    if (!net || !host_accepted || n < 0 || n > net->max_lattices) return fail(ISING_EINVAL, "invalid arguments");
    std::vector<unsigned long long> acc((size_t)std::max(n, 1));
    CUDA_TRY(cudaStreamSynchronize(net->stream), "synchronize");
    CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
    CUDA_TRY(cudaMemcpy(acc.data(), net->accepted, (size_t)n * 8, cudaMemcpyDeviceToHost), "copy counters");
    int rc = net_check_error(net, net->stream);
    if (rc != ISING_OK) return rc;
    for (int i = 0; i < n; ++i) host_accepted[i] = (int64_t)acc[i];
    if (reset) CUDA_TRY(cudaMemset(net->accepted, 0, (size_t)net->max_lattices * 8), "zero counters");
    return ISING_OK;
}

}  // extern "C"
