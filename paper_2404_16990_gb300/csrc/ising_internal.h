// ising_internal.h -- device data structures shared by the host side of the
// C ABI (ising_api.cu) and the kernels (ising_kernels.cu).  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ising {

// Per-lattice descriptor (device, read-only during sweeps).
struct LatDesc {
    uint64_t word_off;   // first 32-bit word of the lattice in the spin array
    uint32_t L;          // side
    uint32_t wn;         // 32-bit words per row and colour = L / 64
    uint32_t sim;        // simulation index s (Philox counter word 2)
    uint32_t key0;       // lo32(seed)
    uint32_t key1;       // hi32(seed)
    uint32_t thr0;       // threshold for dE = 4
    uint32_t thr1;       // threshold for dE = 8
    uint32_t pad;
};

// A group of equal-size lattices that one CTA keeps in shared memory.
struct GroupDesc {
    uint32_t member_off; // first entry of the group in the member list
    uint32_t count;      // lattices in the group
    uint32_t L;
    uint32_t wn;
};

// A lattice handled by the streaming kernels, with the prefix of work items.
struct StreamLat {
    uint32_t lat;        // lattice index
    uint32_t strips;     // tile rows of the lattice
    uint32_t groups;     // wn / words_per_thread
    uint32_t rows;       // rows per thread (clamped so that a tile never exceeds the lattice)
    uint64_t item_begin; // first work item of this lattice
};

// Small device-side control block (first bytes of the workspace scratch).
struct Control {
    unsigned long long t;        // sweep index of the next sweep
    unsigned int ticket;         // resident kernel: next work ticket
    unsigned int blocks_done;    // stream kernel: blocks finished (last-block pattern)
    int error;                   // nonzero: a bounded wait ran out (code in low bits)
    int measure;                 // accumulate moments if nonzero
    long long trace_cap;         // trace entries per lattice (0 = none)
    unsigned int bar_count;      // persistent kernel: blocks arrived at the grid barrier
    unsigned int bar_gen;        // persistent kernel: grid barrier generation
    unsigned long long wait_limit_ns;  // bound of every device wait; 0 = the default (10 s)
    unsigned int pad[4];
};
static_assert(sizeof(Control) == 64, "control block layout");

// Device pointers of one handle, passed by value to kernels.
struct DevState {
    const LatDesc* lat;
    uint32_t* spins;
    long long* obs;              // [n][2]  current E, M
    long long* trace;            // [n][cap][2]
    double* mom;                 // [n][6]  count, sum|m|, sum m^2, sum m^4, sum e, sum e^2
    unsigned long long* acc;     // [n][2]  streaming partial sums (aligned-count, popcount)
    Control* ctl;
    unsigned int* done;          // resident: chunks done per group
    const GroupDesc* groups;
    const uint32_t* members;
    const StreamLat* slats;
    int n;
};

// Learned proposal: per-window Philox key of a patch (sampling draws).
struct LearnedKey {
    uint32_t key0, key1, sim, j;   // lattice seed (lo, hi), simulation index, patch index
};

// Learned proposal: per-lattice description for one round.
struct LearnedLat {
    uint64_t word_off;     // first word of the lattice
    uint32_t L, lat, sim, key0, key1, patch_begin;
    double beta;           // 1 / T
};

// Learned proposal: device pointers of a network (all in the net workspace).
struct NetState {
    float* w;              // fp32 master parameters [ISING_NET_PARAMS]
    float* m;              // Adam first moments
    float* v;              // Adam second moments
    float* g;              // gradient accumulator
    __nv_bfloat16* wb;     // bf16 copy used by the tensor-core kernels
    float* loss;           // scalar
    uint8_t* wq;           // e4m3 copy of the weights, scaled per layer (FP8 inference)
    float* wscale;         // [4] per-layer power-of-two weight scales of the e4m3 copy
    int* err;              // nonzero: a bounded wait of a tensor-core kernel ran out
};

// Swendsen-Wang step: tiles of kSwTileW x kSwTileH sites (x in [64 tx,
// 64 tx + 64), y in [kSwTileH ty, kSwTileH (ty + 1))), numbered row-major
// within a lattice and consecutively over lattices; one warp labels a tile,
// kSwThreads / 32 tiles per CTA.
constexpr int kSwTileW = 64;
constexpr int kSwTileH = 16;
constexpr int kSwThreads = 128;

// Philox phases of the bond draws of a Swendsen-Wang step and of a Wolff step.
constexpr uint32_t kSwBondPhase = 7u, kWolffBondPhase = 10u;

// Per-lattice description (device, in the caller's SW scratch).
struct SwLat {
    uint64_t word_off;     // first packed word of the lattice
    uint64_t site_off;     // first label of the lattice (sum of the earlier L^2)
    uint32_t L, wn, sim, key0, key1;
    uint32_t thr;          // bond threshold floor(2^32 (1 - exp(-2/T))), clamped
    uint32_t tile_begin;   // first tile of the lattice
    uint32_t pad;
};

// Device pointers of one SW scratch area.
struct SwState {
    const SwLat* lat;
    int n;
    uint32_t total_tiles;
    uint4* edges;          // [tiles] right-edge bonds (x), bottom-edge bonds (z | w << 32)
    uint32_t* coins;       // [sites / 32] tile-local root mask, then each tile-local root's cluster coin
    uint32_t* label;       // [sites] parent pointers (site -> tile-local root -> cluster root)
    uint32_t bond_phase;   // Philox phase of the bond draws: kSwBondPhase or kWolffBondPhase
    uint32_t* seed_root;   // [n] Wolff by labelling: the final root of each lattice's seed, else null
};

// Launch wrappers (ising_kernels.cu).  All asynchronous on `stream`.
cudaError_t launch_init_random(const DevState& st, int n_lat, cudaStream_t stream);
// E, M of the listed lattices into obs; max_L = the largest listed side
// (sizes the grid; 0: as for the largest lattices).  finalize = false leaves
// the sums in acc for a kernel that turns them into E and M itself.
cudaError_t launch_observables(const DevState& st, uint32_t max_L, const uint32_t* lat_list,
                               int n_list, cudaStream_t stream, bool finalize = true);
cudaError_t launch_resident(const DevState& st, int n_groups, int64_t n_sweeps,
                            int sweeps_per_unit, int threads, int grid, size_t smem_bytes,
                            cudaStream_t stream);
cudaError_t launch_stream_sweeps(const DevState& st, int n_slats, uint64_t total_items,
                                 int words_per_thread, int threads, int grid, int64_t n_sweeps,
                                 cudaStream_t stream);
cudaError_t launch_stream_persistent(const DevState& st, int n_slats, uint64_t total_tiles,
                                     int words_per_thread, int threads, int grid, int64_t n_sweeps,
                                     cudaStream_t stream);
int stream_persistent_occupancy(int words_per_thread, int threads);
// One thread-block cluster of cluster_size CTAs per lattice (members[0 ..
// count)), all of side L, all n_sweeps sweeps in one launch.
cudaError_t launch_cluster_resident(const DevState& st, const uint32_t* members, int count, int cluster_size,
                                    uint32_t L, int64_t n_sweeps, cudaStream_t stream);
cudaError_t launch_advance_t(const DevState& st, int64_t n, cudaStream_t stream);
cudaError_t launch_random_stream(uint32_t k0, uint32_t k1, uint32_t s, uint32_t phase, uint64_t p0, uint64_t n_p,
                                 uint32_t t0, uint32_t n_t, uint32_t* out, cudaStream_t stream);

// Record a message for ising_last_error() and return code (ising_api.cu).
int set_last_error(int code, const char* msg);

// Metropolis acceptance threshold min(floor(2^32 exp(-dE/T)), 2^32 - 1),
// evaluated in double precision (ising_api.cu); the one table builder of
// every sweep path.
uint32_t threshold_u32(double dE, double T);

// Learned-proposal launch wrappers (ising_learned.cu).
cudaError_t configure_learned_kernels();
cudaError_t launch_net_forward(const NetState& ns, const int8_t* win, int n, float* lq, float* z,
                               __nv_bfloat16* h, cudaStream_t stream);
cudaError_t launch_net_sample(const NetState& ns, int8_t* win, int n, float* lq, const LearnedKey* keys,
                              uint32_t round_t, cudaStream_t stream);
// Teacher-forced log q on the tcgen05 tensor cores (ising_learned_tc.cu), in
// BF16 or FP8: windows [0, n) of win (log q to lq, logits to z if given) and,
// with win_b, [0, n) of win_b (log q to lq_b), in one launch.
cudaError_t launch_net_score_tc(const NetState& ns, bool fp8, const int8_t* win, int n, float* lq, float* z,
                                const int8_t* win_b, float* lq_b, cudaStream_t stream);
cudaError_t launch_net_backward(const NetState& ns, const int8_t* win, int n, const float* z,
                                const __nv_bfloat16* h, float* grad, float* loss, cudaStream_t stream);
cudaError_t launch_adam(const NetState& ns, float lr, int step, cudaStream_t stream);
cudaError_t launch_to_bf16(const NetState& ns, cudaStream_t stream);
cudaError_t launch_to_fp8(const NetState& ns, cudaStream_t stream);
cudaError_t launch_net_sample_fp8(const NetState& ns, int8_t* win, int n, float* lq, const LearnedKey* keys,
                                  uint32_t round_t, cudaStream_t stream);
cudaError_t launch_train_windows(const uint32_t* pool, int n_snap, uint32_t L, int nwin, uint64_t seed,
                                 uint32_t step, int8_t* win, cudaStream_t stream);
cudaError_t launch_gather_patches(const DevState& st, const LearnedLat* ll, int n_lat, int nwin, uint32_t ox,
                                  uint32_t oy, int8_t* win, int8_t* win2, LearnedKey* keys, cudaStream_t stream);
cudaError_t launch_mh_apply(const DevState& st, const LearnedLat* ll, int n_lat, int nwin, uint32_t ox,
                            uint32_t oy, const int8_t* win_old, const int8_t* win_new, const float* lq_old,
                            const float* lq_new, uint32_t round_t, unsigned long long* accepted,
                            cudaStream_t stream);

// Swendsen-Wang launch wrappers (ising_cluster.cu).  sw_clusters: bonds,
// labels (every site -> a tile-local root -> the final root) and the root
// coins of the current step; sw_flip: flip every cluster by its root's coin; sw_record: E, M after the step into the trace / moments
// and advance the device sweep counter.
cudaError_t launch_sw_clusters(const DevState& st, const SwState& sw, cudaStream_t stream);
cudaError_t launch_sw_flip(const DevState& st, const SwState& sw, cudaStream_t stream);
cudaError_t launch_sw_record(const DevState& st, int n_lat, cudaStream_t stream);
cudaError_t launch_sw_compress(const SwState& sw, cudaStream_t stream);   // labels -> final roots
// Wolff by labelling: after launch_sw_clusters' local and merge kernels have
// linked the components of the Wolff bonds (bond_phase 10), each lattice's
// seed (phase 9) is resolved to its final root into sw.seed_root, and the
// resolve kernel sets "coin" 1 exactly for the tile-local roots of that
// component.  One launch of the whole step: local, merge, seed, resolve.
cudaError_t launch_wolff_clusters(const DevState& st, const SwState& sw, cudaStream_t stream);
// Wolff single-cluster steps of every lattice (ising_cluster.cu); the scratch
// of the cluster step serves as queue (labels) and visited bits (coins).
// Lattices with L <= wolff_smem_max_L() run in shared memory (max_small_L =
// the largest of them, 0 if none); any_large: some lattice is larger.
cudaError_t launch_wolff(const DevState& st, const SwState& sw, int64_t n_steps, uint32_t max_small_L, bool any_large,
                         cudaStream_t stream);
uint32_t wolff_smem_max_L();

int resident_occupancy(int threads, size_t smem_bytes);
int stream_occupancy(int words_per_thread, int threads);
int device_sm_count();
size_t device_max_smem_optin();
cudaError_t configure_kernels();

}  // namespace ising
