// ising_noalloc.cu -- ising_sweep_noalloc: the streaming sweep for callers
// that cannot allocate device memory.
//
// Every other entry point of this library takes its device scratch (lattice
// descriptors, per-lattice partial sums, the block counter of the last-block
// reduction) from a workspace the caller allocates.  Some callers cannot make
// that allocation: code that runs inside a host application owning all device
// memory through its own pool, or a latency-critical path where cudaMalloc may
// block or synchronise the device.  This entry point keeps its scratch in a
// fixed, file-scope device array instead, so the caller only passes the
// packed lattices (input and output) and the device array for E and M.
#include "../../include/ising.h"
#include "ising_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

using namespace ising;

namespace {

// Scratch layout inside the static array (byte offsets).
constexpr size_t kCtlOff = 0;
constexpr size_t kLatOff = 256;
constexpr size_t kSlatOff = kLatOff + ISING_NOALLOC_MAX_LATTICES * sizeof(LatDesc);
constexpr size_t kAccOff = kSlatOff + ISING_NOALLOC_MAX_LATTICES * sizeof(StreamLat);
constexpr size_t kScratchBytes = kAccOff + ISING_NOALLOC_MAX_LATTICES * 2 * sizeof(unsigned long long);
static_assert(sizeof(Control) <= kLatOff, "control block must fit before the descriptors");
static_assert(kLatOff % 16 == 0 && kSlatOff % 16 == 0 && kAccOff % 16 == 0, "aligned sections");

// The scratch itself.  Every GPU that loads this library holds one copy until
// the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Descriptors of up to kSetupChunk lattices, passed by value as a kernel
// parameter: the launch copies them, so no host buffer has to outlive the
// call and no host-to-device copy is issued.
constexpr int kSetupChunk = 16;
struct SetupBlock {
    Control ctl;                  // written by the chunk with first == 0
    int first, count;             // lattices first .. first + count - 1
    LatDesc lat[kSetupChunk];
    StreamLat sl[kSetupChunk];
};
static_assert(sizeof(SetupBlock) <= 4096, "setup block must fit the classic kernel parameter limit");

// Writes one chunk of descriptors into the scratch and zeroes those
// lattices' partial sums (device code names the array directly).
__global__ void noalloc_setup_kernel(const __grid_constant__ SetupBlock b) {
    unsigned char* base = g_noalloc_scratch;
    const int i = threadIdx.x;
    if (i == 0 && b.first == 0) *reinterpret_cast<Control*>(base + kCtlOff) = b.ctl;
    if (i < b.count) {
        const int k = b.first + i;
        reinterpret_cast<LatDesc*>(base + kLatOff)[k] = b.lat[i];
        reinterpret_cast<StreamLat*>(base + kSlatOff)[k] = b.sl[i];
        unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + kAccOff);
        acc[2 * k] = 0ull;
        acc[2 * k + 1] = 0ull;
    }
}

// Device address of the scratch on the current device (set up once per device).
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(ISING_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(ISING_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return set_last_error(ISING_ECUDA, "cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ISING_OK;
}

}  // namespace

extern "C" int ising_sweep_noalloc(uint32_t* dev_words, int n_lat, const int* Ls, const double* temps,
                                   const uint64_t* seeds, int64_t t0, int64_t n, int64_t* dev_EM,
                                   void* cuda_stream) {
    if (n_lat < 1 || n_lat > ISING_NOALLOC_MAX_LATTICES)
        return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: n_lat must be in [1, ISING_NOALLOC_MAX_LATTICES]");
    if (!dev_words || !dev_EM || !Ls || !temps || !seeds)
        return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: NULL argument");
    if (n < 0 || t0 < 0 || t0 + n > (int64_t)0xFFFFFFFFll)
        return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: need n >= 0, t0 >= 0 and t0 + n < 2^32");
    if (((uintptr_t)dev_words) % 16 != 0)
        return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: dev_words must be 16-byte aligned");
    for (int i = 0; i < n_lat; ++i) {
        if (Ls[i] < ISING_MIN_L || Ls[i] > ISING_MAX_L || Ls[i] % 64 != 0)
            return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: every L must be a multiple of 64 in [64, 65536]");
        if (!(temps[i] > 0.0) || !std::isfinite(temps[i]))
            return set_last_error(ISING_EINVAL, "ising_sweep_noalloc: temperatures must be positive and finite");
    }
    if (n == 0) return ISING_OK;

    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != ISING_OK) return rc;
    char* base = (char*)scratch;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // descriptors and tiles, as the workspace-based path builds them
    const int threads = 256, rows = 4;
    int V = 2;
    for (int i = 0; i < n_lat; ++i)
        if ((Ls[i] / 64) % 2 != 0) V = 1;
    std::vector<SetupBlock> chunks((size_t)((n_lat + kSetupChunk - 1) / kSetupChunk));
    uint64_t off = 0, tiles = 0;
    for (int i = 0; i < n_lat; ++i) {
        const uint32_t L = (uint32_t)Ls[i], wn = L / 64;
        LatDesc d{};
        d.word_off = off;
        d.L = L;
        d.wn = wn;
        d.sim = (uint32_t)i;
        d.key0 = (uint32_t)(seeds[i] & 0xFFFFFFFFull);
        d.key1 = (uint32_t)(seeds[i] >> 32);
        d.thr0 = threshold_u32(4.0, temps[i]);
        d.thr1 = threshold_u32(8.0, temps[i]);
        SetupBlock& b = chunks[(size_t)(i / kSetupChunk)];
        b.lat[i % kSetupChunk] = d;
        off += (uint64_t)L * L / 32;
        StreamLat s{};
        s.lat = (uint32_t)i;
        s.groups = wn / (uint32_t)V;
        const uint32_t tw = std::min<uint32_t>(s.groups, (uint32_t)threads);
        const uint32_t th = (uint32_t)threads / tw;
        const uint32_t tiles_x = (s.groups + tw - 1) / tw;
        const uint32_t Rl = std::max<uint32_t>(1u, std::min<uint32_t>((uint32_t)rows, L / th));
        s.rows = Rl;
        const uint32_t tiles_y = (L + th * Rl - 1) / (th * Rl);
        s.strips = tiles_y;
        s.item_begin = tiles;
        tiles += (uint64_t)tiles_x * tiles_y;
        b.sl[i % kSetupChunk] = s;
    }
    for (size_t c = 0; c < chunks.size(); ++c) {
        SetupBlock& b = chunks[c];
        b.first = (int)c * kSetupChunk;
        b.count = std::min(kSetupChunk, n_lat - b.first);
        b.ctl = Control{};
        b.ctl.t = (unsigned long long)t0;   // trace_cap = 0 and measure = 0: only E/M are written
        noalloc_setup_kernel<<<1, kSetupChunk, 0, stream>>>(b);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(ISING_ECUDA, cudaGetErrorString(e));

    DevState st{};
    st.ctl = (Control*)(base + kCtlOff);
    st.lat = (const LatDesc*)(base + kLatOff);
    st.slats = (const StreamLat*)(base + kSlatOff);
    st.acc = (unsigned long long*)(base + kAccOff);
    st.spins = dev_words;
    st.obs = (long long*)dev_EM;
    st.n = n_lat;
    const int occ = stream_occupancy(V, threads);
    if (occ <= 0) return set_last_error(ISING_ECUDA, "streaming kernel occupancy query failed");
    const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)device_sm_count() * occ);
    e = launch_stream_sweeps(st, n_lat, tiles, V, threads, grid, n, stream);
    if (e != cudaSuccess) return set_last_error(ISING_ECUDA, cudaGetErrorString(e));
    return ISING_OK;
}
