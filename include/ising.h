/*
 * ising.h -- C ABI of libising, a GB300 (sm_103a) simulator of the 2D Ising
 * model with checkerboard Metropolis sweeps on multi-spin-coded lattices.
 *
 * The model and method follow arXiv 2404.16990:
 *   - Hamiltonian H = -J sum_<ij> s_i s_j over the four nearest neighbours of
 *     a square periodic L x L lattice, J = 1, no field (Section 1).
 *   - Metropolis rule, accept iff ran() < exp(-beta dE) (Section 1).
 *   - Checkerboard order: all red/black sites ((x+y) even) in parallel, then
 *     all blue/white sites ((x+y) odd) (Algorithm 5; Algorithm 3 is the same
 *     loop at PE level).  One sweep attempts every spin once; the flip rate is
 *     spins x sweeps / time (Section 3.2, Table 1).
 *   - Many independent simulations advance at once (Section 2: one lattice
 *     per PE column, up to 754 in Section 3.2).
 *
 * Definitions this library fixes where the paper leaves them open:
 *   - Spins are stored one bit each (bit 0 = +1, bit 1 = -1), 32 per 32-bit
 *     word, least significant bit = lowest index (the bit order of Section 2,
 *     where 16 spins share an int16).  Lattice layout in device memory:
 *     word[(c*L + y)*(L/64) + k] holds the sites of colour c in row y with
 *     x = 2j + ((y+c) & 1), j = 32k + bit.  One lattice = L*L/8 bytes.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) replaces the
 *     paper's hardware generator.  Key = (lo32(seed), hi32(seed)); counter =
 *     (p >> 2, t, s, phase) with t the sweep index counted over the life of
 *     the handle, s the simulation index, phase 0/1 = black/white half-sweep,
 *     2 = random initial state; output lane p & 3.  p is the rank of the
 *     site among the same-colour sites of its lattice in row-major order,
 *     p = y*(L/2) + (x >> 1); for the initial state p = y*L + x.
 *   - A site with dE <= 0 always flips; with dE in {4, 8} it flips iff
 *     r < thr[dE/4 - 1], thr = min(floor(2^32 exp(-dE/T)), 2^32-1), computed
 *     on the host in double precision.  Random start: s = +1 iff the top bit
 *     of the site's phase-2 draw is 0.
 *   - E = -sum over bonds s_i s_j and M = sum s_i are exact 64-bit integers.
 *
 * Conventions for every call:
 *   - Return 0 (ISING_OK) on success, a negative ISING_E* code on failure;
 *     ising_last_error() then gives a message (thread-local, valid until the
 *     next failing call on the same thread).
 *   - Device memory is owned by the caller: it passes one workspace of at
 *     least the size the *_workspace_bytes call reports; the library never
 *     allocates device memory and never frees the workspace.  Host arrays are
 *     owned by the caller and read/written only during the call.
 *   - Every device operation is issued on the CUDA stream given at creation
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).  Calls
 *     that return host data synchronise that stream first.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - Lattice sizes: L even, 64 <= L <= 65536 and L a multiple of 64.
 *     Temperatures: positive and finite.  Anything else is ISING_EINVAL.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISING_OK 0
#define ISING_EINVAL (-1)    /* invalid argument */
#define ISING_ENOMEM (-2)    /* workspace smaller than required */
#define ISING_ECUDA (-3)     /* a CUDA call failed; see ising_last_error() */
#define ISING_ETIMEOUT (-4)  /* a bounded device-side wait ran out */
#define ISING_ESTATE (-5)    /* handle in a state that does not allow the call */

#define ISING_INIT_RANDOM 0
#define ISING_INIT_COLD 1

#define ISING_MIN_L 64
#define ISING_MAX_L 65536

typedef struct ising_handle* ising_t;

/* Message of the last failing call on this thread ("" if none). */
const char* ising_last_error(void);

/* Library version string. */
const char* ising_version(void);

/* Bytes of device workspace for n_sims lattices of side L with a per-sweep
 * E/M trace ring of trace_cap entries per lattice (0 = no trace).
 * Errors: ISING_EINVAL for an invalid L, n_sims < 0 or trace_cap < 0. */
int ising_workspace_bytes(int L, int n_sims, int64_t trace_cap, size_t* bytes);

/* Same for a batch of lattices of possibly different sides Ls[0..n_sims-1]. */
int ising_batch_workspace_bytes(int n_sims, const int* Ls, int64_t trace_cap, size_t* bytes);

/* Create n_sims independent L x L lattices (Algorithm 5's P, one per
 * simulation as in Algorithm 3's (gamma, beta) pairs).  temps[n_sims] are the
 * temperatures (J = 1); seed keys every lattice's generator, simulation i
 * uses s = i.  init = ISING_INIT_RANDOM or ISING_INIT_COLD.  dev_workspace
 * is a device pointer (256-byte aligned) of ws_bytes >= the size reported by
 * ising_workspace_bytes.  The initial state and its E, M are computed on
 * cuda_stream before the call returns (asynchronously).  n_sims may be 0: the
 * handle then does nothing.  *out receives the handle; free it with
 * ising_destroy (the workspace stays the caller's). */
int ising_create(ising_t* out, int L, int n_sims, const double* temps, uint64_t seed,
                 int init, int64_t trace_cap, void* dev_workspace, size_t ws_bytes,
                 void* cuda_stream);

/* Create a batch of lattices of uneven side and temperature: lattice i has
 * side Ls[i], temperature temps[i], key seeds[i] and simulation index s = i. */
int ising_create_batch(ising_t* out, int n_sims, const int* Ls, const double* temps,
                       const uint64_t* seeds, int init, int64_t trace_cap,
                       void* dev_workspace, size_t ws_bytes, void* cuda_stream);

/* Advance every lattice by n >= 0 full sweeps (black half-sweep, then white
 * half-sweep; Algorithm 3's loop body).  Asynchronous on the handle's stream:
 * returns after enqueueing.  After each sweep E and M are recorded (current
 * values, trace ring, and the FP64 moment sums if measuring is on).  If a
 * bounded device-side wait of the resident kernel or of the persistent
 * streaming kernel runs out (ising_set_wait_limit_ns), the next call that
 * synchronises returns ISING_ETIMEOUT and the state is undefined.  The sweep
 * counter must stay below 2^32 (ISING_EINVAL otherwise). */
int ising_sweep(ising_t h, int64_t n);

/* Sweeps done since creation (the t of the next sweep). */
int64_t ising_sweeps_done(ising_t h);

/* Kernels this handle has enqueued so far (each CUDA-graph replay counts the
 * kernels of the graph); -1 for a NULL handle.  A diagnostic for profiling. */
int64_t ising_kernel_launches(ising_t h);

/* Current E[n_sims], M[n_sims] (host arrays, caller-owned).  Synchronises. */
int ising_observables(ising_t h, int64_t* E, int64_t* M);

/* The last n = min(sweeps recorded, trace_cap, max_sweeps) trace entries of
 * every lattice, oldest first: E[i*n + j], M[i*n + j] for lattice i.  *n_out
 * receives n.  Synchronises. */
int ising_trace(ising_t h, int64_t* E, int64_t* M, int64_t max_sweeps, int64_t* n_out);

/* Unpacked spins (+1/-1, row-major L x L) of lattice sim.  Synchronises. */
int ising_get_spins(ising_t h, int sim, int8_t* host_LxL);

/* Overwrite lattice sim with host spins (+1/-1; any other value is
 * ISING_EINVAL); its E and M are recomputed on the device. */
int ising_set_spins(ising_t h, int sim, const int8_t* host_LxL);

/* Device address and length (in 32-bit words, L*L/32) of the packed spins of
 * lattice sim, in the layout described at the top of this file.  The memory
 * belongs to the caller's workspace; reading it is safe once the handle's
 * stream has finished the sweeps that write it. */
int ising_lattice_words(ising_t h, int sim, void** dev_words, size_t* n_words);

/* The acceptance thresholds thr[2*i], thr[2*i+1] (dE = 4, 8) of every lattice. */
int ising_get_thresholds(ising_t h, uint32_t* thr);

/* Lattice side of simulation sim (0 if out of range). */
int ising_lattice_size(ising_t h, int sim);

/* Number of simulations of the handle. */
int ising_num_sims(ising_t h);

/* Turn the accumulation of FP64 moments on (1) or off (0). */
int ising_set_measure(ising_t h, int on);

/* Bound of every device-side wait of the handle's sweep kernels, in
 * nanoseconds of the GPU's global timer: the resident kernel's wait for the
 * previous chunk of its lattice group and the persistent streaming kernel's
 * grid barrier.  ns = 0 restores the default of 10 s; at most
 * ISING_MAX_WAIT_LIMIT_NS.  A wait that runs out sets the handle's error word
 * and its kernel returns without finishing the sweeps; from then on every
 * synchronising call on the handle (ising_observables, ising_trace,
 * ising_moments, ising_get_spins, ...) returns ISING_ETIMEOUT and the
 * handle's lattices are undefined (make a new handle).  A short limit exists
 * for testing that path: failure detection in the sense of the paper's
 * long-running validation scans (Section 3.1), where a stalled kernel must
 * end with an error rather than hold the GPU.  Synchronises the stream. */
#define ISING_MAX_WAIT_LIMIT_NS 600000000000ull
int ising_set_wait_limit_ns(ising_t h, uint64_t ns);

/* Zero the moment sums. */
int ising_reset_moments(ising_t h);

/* Moment sums of every lattice over the measured sweeps, 6 doubles each:
 * out[6*i + 0..5] = count, sum |m|, sum m^2, sum m^4, sum e, sum e^2 with
 * m = M/L^2 and e = E/L^2.  Synchronises. */
int ising_moments(ising_t h, double* out);

/* Binder cumulant U = 1 - <m^4> / (3 <m^2>^2) of every lattice from the
 * moment sums of ising_moments (moments[6*i + 0..5]); U[i] is NaN where no
 * sweep was measured.  Host-only. */
int ising_binder(const double* moments, int n_sims, double* U);

/* Integrated autocorrelation time of the series x[0..n-1] (n >= 2), host-only:
 * tau = 1/2 + sum_{t=1..W} rho(t) with rho the normalised autocovariance and W
 * the smallest lag with W >= c * tau(W) (automatic window of Madras and Sokal,
 * c ~ 5..6).  tau_err (may be NULL) = tau * sqrt(2(2W+1)/n), window (may be
 * NULL) = W.  A constant series gives tau = 1/2.  The paper averages |M| over
 * long runs (Section 3.1); effective independent samples = n / (2 tau). */
int ising_tau_int(const double* x, int64_t n, double c, double* tau, double* tau_err,
                  int64_t* window);

/* Statistical inefficiency of x[0..n-1] (host arrays, n >= 2), after Chodera,
 * J. Chem. Theory Comput. 12, 1799 (2016): g = 1 + 2 sum_{t>=1} (1 - t/n) C(t)
 * with C(t) the fluctuation autocorrelation about the series' own mean,
 * C(t) = [sum_{i<n-t} d_i d_{i+t} / (n - t)] / [sum_i d_i^2 / n], the sum
 * stopping before the first lag with C(t) <= 0; g >= 1 (1 for a constant
 * series).  n / g is the number of effectively independent samples. */
int ising_stat_inefficiency(const double* x, int64_t n, double* g);

/* Automatic equilibration detection (the same reference; the method Section
 * 3.1 uses to discard non-equilibrated data): over the candidate starts
 * t = 0, stride, 2 stride, ... <= n - 2, *t0 receives the t that maximises
 * the effective sample count (n - t) / g(x[t..n-1]) (the smallest such t on
 * ties), *g and *n_eff (either may be NULL) its g and count.  stride = 0
 * picks max(1, n / 256).  Host-only; ISING_EINVAL for n < 2 or stride < 0. */
int ising_equilibration(const double* x, int64_t n, int64_t stride, int64_t* t0, double* g, double* n_eff);

/* Size of a checkpoint of the handle (spins, sweep counter, current E/M,
 * moment sums), and save/load through a host buffer of that size.  Loading
 * into a handle of a different shape is ISING_EINVAL.  Because the generator
 * is counter-based, n sweeps, save, load, m sweeps give the same bits as
 * n + m sweeps. */
int ising_state_bytes(ising_t h, size_t* bytes);
int ising_save(ising_t h, void* host_buf, size_t bytes);
int ising_load(ising_t h, const void* host_buf, size_t bytes);

/* Execution plan.  ISING_PLAN_AUTO (the default) streams every lattice with
 * the default tiling: on GB300 the resident kernel measured at best even with
 * the streaming one and up to 17x slower (one 1024^2 lattice).  The others
 * force one kernel for every lattice: RESIDENT keeps each lattice (or group
 * of equal-size lattices) in shared memory for many sweeps (up to the
 * shared-memory limit, else ISING_EINVAL); STREAM runs one launch per
 * half-sweep over the lattices in device memory.  Tuning knobs (0 = default):
 * words_per_thread in {1, 2, 4} = 32-bit words per streaming thread and row;
 * rows_per_item = rows per streaming thread (lowered per lattice so that one tile
 * of a block never spans more rows than the lattice has).  By default the
 * streaming tiling follows the number of blocks of 256 threads it gives:
 * 4 words x 4 rows per thread from 4 blocks per SM, else 2 x 2 from 1.5, else
 * 1 x 2 from 0.5, else 1 x 1 (rows as given when rows_per_item is set);
 * ising_get_plan reports the tiling in use.  sweeps_per_unit = sweeps a
 * resident work unit runs before its group is stored; threads = block size
 * (a multiple of 32, at most 512 resident / 256 streaming).  No choice
 * changes any result bit. */
#define ISING_PLAN_AUTO 0
#define ISING_PLAN_RESIDENT 1
#define ISING_PLAN_STREAM 2
#define ISING_PLAN_PERSIST 3
/* ISING_PLAN_MIXED: lattices with L <= 1024 resident (as RESIDENT, grouped by
 * size), larger ones streamed (as STREAM), in the same sweeps. */
#define ISING_PLAN_MIXED 4
/* ISING_PLAN_CLUSTER: every lattice (L <= ISING_CLUSTER_MAX_L, else
 * ISING_EINVAL) is held by one thread-block cluster of C CTAs for all sweeps
 * of a call, CTA r owning rows [r L/C, (r+1) L/C) of both colours in shared
 * memory; a half-sweep reads the rows next to its strip from the neighbouring
 * CTAs' shared memory (distributed shared memory) and a cluster barrier
 * separates the half-sweeps.  C is the largest power of two <= min(8,
 * L / rows_per_item) (rows_per_item 0 = 64).  One launch per distinct L, all
 * lattices of that size in it, then one to advance the sweep counter. */
#define ISING_PLAN_CLUSTER 5
#define ISING_CLUSTER_MAX_L 1024
int ising_set_plan(ising_t h, int plan, int words_per_thread, int rows_per_item,
                   int sweeps_per_unit, int threads);

/* Autotuner: time candidate plans (resident with sweeps_per_unit in {8, 32,
 * 128} and block sizes {auto, 256, 512} when some lattice has L <= 1024 --
 * RESIDENT if every lattice has, else MIXED; CLUSTER with rows_per_item in
 * {32, 64, 128} when every lattice has L <= 1024;
 * streaming with words_per_thread in {1, 2, 4}, rows_per_item in {1, 2, 4, 8},
 * threads in {128, 256}, and the persistent streaming kernel with the same
 * tilings) for probe_sweeps sweeps each on the handle's stream
 * (through CUDA graphs if ising_set_graph is on, as the sweeps will run) and
 * keep the fastest.  The lattices and the sweep counter are saved before
 * and restored after, so tuning changes no result.  If the environment
 * variable ISING_TUNE_CACHE names a file, the choice is appended to it keyed by
 * the multiset of lattice sizes and the device, and a later call with
 * force = 0 reuses it without timing.  *best_flips_per_ns (may be NULL)
 * receives the winner's probe rate (0 when taken from the cache). */
int ising_autotune(ising_t h, int64_t probe_sweeps, int force, double* best_flips_per_ns);

/* The plan in use (any pointer may be NULL). */
int ising_get_plan(ising_t h, int* plan, int* words_per_thread, int* rows_per_item,
                   int* sweeps_per_unit, int* threads);

/* Replay the sweeps of each later ising_sweep(h, n) call through a CUDA graph
 * captured for that n (1 = on, 0 = off).  Results are identical either way. */
int ising_set_graph(ising_t h, int on);

/* Copy the packed spins of every lattice (the handle's whole spin array, sum of
 * L*L/8 bytes, lattices one after another) to dev_dst on the handle's stream;
 * bytes must be at least that size.  Used to collect training snapshots. */
int ising_snapshot(ising_t h, void* dev_dst, size_t bytes);

/* ------------------------------------------------------------------------
 * Learned patch proposal.  The paper has no learned component; it motivates
 * improving on local moves by the critical slowing down of single-site
 * updates near T_c (Section 1).  Definitions:
 *
 * Window: an 8x8 interior patch plus its one-site ring, 10x10 spins (+1/-1,
 * int8, row-major), positions p = (r, c) in raster order; interior =
 * 1 <= r, c <= 8.
 * Net (ISING_NET_PARAMS fp32 parameters, flat order W1[16][16], b1[16],
 * W2[5][16][16], b2[16], W3[5][16][16], b3[16], W4[5][16], b4[1]): a masked
 * 3x3-convolution autoregressive model with 16 channels.  Layer 1 reads 16
 * features per position: the interior spins at the 4 taps before p in raster
 * order, (dy,dx) in {(-1,-1),(-1,0),(-1,1),(0,-1)}, the ring spins at the 9
 * taps (dy,dx) in {-1,0,1}^2 (row-major), then 3 zeros (positions outside the
 * window read 0).  Layers 2, 3 (16 -> 16) and 4 (16 -> 1) sum over the 5 taps
 * {(-1,-1),(-1,0),(-1,1),(0,-1),(0,0)}; W[t][ci][co].  Hidden activations are
 * bf16(relu(.)), weights enter as bf16, sums are fp32 (tensor cores).  z(p) is
 * the logit of P(spin = +1) at interior p given the ring and earlier interior
 * spins; log q(window) = sum over interior p of log sigmoid(s_p z(p)) (fp32).
 * Sampling: s_p = +1 iff r_p < floor(2^32 sigmoid(z(p))) (sigmoid in fp32),
 * r_p = lane i%4 of Philox counter (16 j + i/4, round, s, 4), i = 8(r-1)+(c-1),
 * j the patch index, key = the lattice seed.
 * Round (ising_learned_round): patches with interior top-left site
 * (16a + ox, 16b + oy), a, b in [0, L/16), patch index j = b L/16 + a,
 * (ox, oy) = (0,0), (8,8), (0,8), (8,0) for round % 4 = 0..3; every ring
 * avoids every other interior, so all patches move at once.  Each patch
 * proposes x' ~ q(. | ring), accepted iff log u < log alpha with
 * log alpha = -dE/T + log q(x) - log q(x') in FP64 (dE over the bonds touching
 * the interior) and u = ((r0 >> 5) 2^26 + (r1 >> 6) + 0.5) / 2^53 (FP64
 * arithmetic: in (0, 1], 1.0 only for the top code) from lanes 0, 1 of
 * Philox counter (j, round, s, 5).  E and M are updated exactly.
 * ------------------------------------------------------------------------ */
#define ISING_NET_PARAMS 2945
typedef struct ising_net* ising_net_t;

/* Device workspace of a net that handles up to max_windows windows per call
 * (patches of one round: sum over lattices of (L/16)^2, ~0.25 KB each), a
 * training batch / gradient / logits call of up to max_batch windows (~10 KB
 * each: activations kept for the backward pass), and rounds over up to
 * max_lattices lattices. */
int ising_net_workspace_bytes(int max_windows, int max_batch, int max_lattices, size_t* bytes);
int ising_net_create(ising_net_t* out, int max_windows, int max_batch, int max_lattices,
                     void* dev_workspace, size_t ws_bytes, void* cuda_stream);
void ising_net_destroy(ising_net_t net);

/* Arithmetic of scoring, sampling and rounds (training is always BF16):
 * ISING_NET_BF16 as above, or ISING_NET_FP8: weights enter as
 * e4m3(W * s_l) with s_l = 2^floor(log2(448 / max|W of layer l|)) (layers 1..4),
 * hidden activations as e4m3(relu(.)) (round to nearest even, saturating),
 * products summed in fp32 and divided by s_l before the fp32 bias.  Scoring
 * (ising_net_score, and both log q of a round) runs on the tcgen05 tensor
 * cores in either precision (one MMA per tap in BF16, one per pair of taps
 * in FP8); the MH correction evaluates log q of x and x' in one launch of
 * that kernel.  The proposal is drawn by a separate kernel (a wavefront
 * sampler, mma.sync BF16 or E4M3) whose logits equal the scoring kernel's up
 * to the order of the fp32 sums.  Either precision therefore samples the
 * Boltzmann distribution up to a relative bias of about 1e-6 (and the 2^-32
 * quantization of the sampling thresholds); FP8 changes the acceptance rate
 * and the cost.  A bounded wait of the scoring kernel that runs out (1 s)
 * makes the next synchronising net call return ISING_ETIMEOUT. */
#define ISING_NET_BF16 0
#define ISING_NET_FP8 1
int ising_net_set_precision(ising_net_t net, int precision);

/* fp32 parameters in/out (host, ISING_NET_PARAMS); set also zeroes the Adam
 * moments and its step count. */
int ising_net_set_params(ising_net_t net, const float* host_params);
int ising_net_get_params(ising_net_t net, float* host_params);

/* Teacher-forced scoring of n host windows: log q per window (host [n]) and,
 * if host_z is not NULL, the logits of all 100 positions (host [n][100]). */
int ising_net_score(ising_net_t net, const int8_t* host_windows, int n, float* host_logq, float* host_z);

/* Sample the interiors of n host windows given their rings (in place) with
 * keys[4*w + 0..3] = (key0, key1, s, j) and the round index; log q of the
 * samples to host_logq [n]. */
int ising_net_sample(ising_net_t net, int8_t* host_windows, int n, const uint32_t* host_keys,
                     uint32_t round_index, float* host_logq);

/* Gradient of the mean negative log-likelihood of n host windows (host
 * [ISING_NET_PARAMS]) and that loss; does not change the parameters. */
int ising_net_grad(ising_net_t net, const int8_t* host_windows, int n, float* host_grad, float* host_loss);

/* Train with Adam (lr; beta1 0.9, beta2 0.999, eps 1e-8): each step draws
 * `batch` windows from n_snap packed L x L lattices at dev_pool_words (one
 * after another, L*L/32 words each; e.g. snapshots taken with
 * ising_lattice_words) -- window b of step s takes snapshot r.x % n_snap and
 * top-left interior site (r.y % L, r.z % L), r = Philox counter (b, step, 0,
 * 6) keyed by seed -- then runs forward, backward and the update.  The
 * per-step losses go to host_losses [steps] if not NULL. */
int ising_net_train(ising_net_t net, const void* dev_pool_words, int n_snap, int L, int64_t steps,
                    int batch, float lr, uint64_t seed, float* host_losses);

/* The windows that training step `step` of ising_net_train draws: batch
 * (<= max_windows) windows into host_windows [batch][100], by the rule given
 * for ising_net_train (the same kernel).  Does not change the net.  For
 * inspecting and checking the training data. */
int ising_net_train_windows(ising_net_t net, const void* dev_pool_words, int n_snap, int L, int64_t step,
                            int batch, uint64_t seed, int8_t* host_windows);

/* One Adam step of the fp32 masters with a caller-given gradient (host
 * [ISING_NET_PARAMS]) by the same update kernel as ising_net_train: with k
 * the net's step count after incrementing it, m = 0.9 m + 0.1 g, v = 0.999 v
 * + 0.001 g^2, w -= lr (m / (1 - 0.9^k)) / (sqrt(v / (1 - 0.999^k)) + 1e-8)
 * (Kingma and Ba 2015), all in fp32; then the bf16 (and, if in use, e4m3)
 * copies are refreshed.  Synchronises. */
int ising_net_apply_grad(ising_net_t net, const float* host_grad, float lr);

/* One learned patch round over every lattice of h (round index round_index;
 * L must be a multiple of 16, which every valid L is), on h's stream: gather
 * the patches' windows, sample proposals, score the current and the proposed
 * windows (in BF16 both in one launch), accept or reject in FP64.  With
 * host_accepted [n_sims] not NULL the call synchronises and returns the
 * patches accepted in this round; with NULL it only enqueues the round and the
 * per-lattice counts accumulate on the device (read them with
 * ising_net_accepted).  The first round with a handle uploads its lattice
 * table (synchronising once).  The handle's sweep counter is unchanged; its
 * current E and M are updated exactly. */
int ising_learned_round(ising_t h, ising_net_t net, int64_t round_index, int64_t* host_accepted);

/* Accepted patches per lattice accumulated by rounds enqueued without a host
 * buffer (host [n]); reset = 1 zeroes the counters.  Synchronises the device. */
int ising_net_accepted(ising_net_t net, int64_t* host_accepted, int n, int reset);

/* Allocation-free streaming sweep.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code running
 * inside a host application that owns all device memory through its own pool,
 * or a latency-critical path where cudaMalloc may block or synchronise the
 * device -- and so cannot provide the workspace the other calls need.
 *
 * It runs the same streaming half-sweep kernel as ising_sweep, with the
 * kernel's scratch (lattice descriptors, per-lattice partial sums of E and M,
 * the sweep counter and block counter) in one fixed device array inside the
 * library of about 5.4 KB, sized for at most ISING_NOALLOC_MAX_LATTICES
 * lattices; a larger n_lat is ISING_EINVAL.  Every GPU that loads the library
 * holds that array until the process exits.  No cudaMalloc, cudaFree or other
 * allocating routine is called.
 *
 *   dev_words  device, 16-byte aligned: the packed lattices one after another,
 *              lattice i (side Ls[i]) taking Ls[i]^2/32 32-bit words in the
 *              layout described at the top of this file; updated in place.
 *   Ls, temps, seeds  host arrays [n_lat]; lattice i uses key seeds[i] and
 *              simulation index s = i (as ising_create_batch).
 *   t0, n      sweeps t0 .. t0+n-1 (t0 is the Philox sweep counter of the
 *              first sweep; t0 + n < 2^32).  n = 0 does nothing.
 *   dev_EM     device int64[2*n_lat]: E and M of lattice i after the last
 *              sweep at [2i] and [2i+1].
 *
 * Asynchronous on cuda_stream.  All calls share the one scratch array, which
 * keeps the last call's contents; each call clears what must start at zero.
 * Calls that overlap on the GPU (other streams, or other host threads without
 * ordering between them) race on the array and give undefined results.  The
 * first call on each device looks the array's device address up
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Results are bit-identical to ising_create_batch
 * followed by ising_sweep on the same lattices when ising_sweeps_done == t0. */
#define ISING_NOALLOC_MAX_LATTICES 64
int ising_sweep_noalloc(uint32_t* dev_words, int n_lat, const int* Ls, const double* temps,
                        const uint64_t* seeds, int64_t t0, int64_t n, int64_t* dev_EM,
                        void* cuda_stream);

/* ---- Swendsen-Wang cluster step -----------------------------------------
 * Section 1 names cluster algorithms (Swendsen-Wang, Wolff) as the cure for
 * the critical slowing down of single-site Metropolis.  One step (Swendsen
 * and Wang, PRL 58, 86 (1987)), J = 1, h = 0: every nearest-neighbour pair of
 * equal spins gets an active bond with probability p = 1 - exp(-2/T); the
 * clusters are the connected components of the active bonds; each cluster
 * flips with probability 1/2.  Draws (Philox4x32-10 keyed by the lattice's
 * seed, counter (q, t, s, phase), t = the step's index in the handle's sweep
 * counter, s = simulation index):
 *   bonds, phase 7: site p = y*L + x owns the bonds to (x+1, y) and (x, y+1)
 *     (indices mod L); q = p >> 1, lane 2*(p & 1) is the right bond's draw,
 *     lane 2*(p & 1) + 1 the down bond's; a bond between equal spins is
 *     active iff its draw is below floor(2^32 p) (at most 2^32 - 1);
 *   coins, phase 8: a cluster is named by its smallest site index r0 (its
 *     root) and flips iff the top bit of lane r0 & 3 of block r0 >> 2 is 1.
 * Steps and Metropolis sweeps share the sweep counter and may be mixed. */
#define ISING_SW_MAX_L 32768

/* Bytes of device scratch one cluster step of this handle needs: the
 * per-lattice table and a 32-bit word per lattice, 16 bytes per 64 x 16
 * tile, one coin bit and one 32-bit label per site (about 4.14 bytes per
 * site).  ISING_EINVAL if a lattice has
 * L > ISING_SW_MAX_L. */
int ising_sw_scratch_bytes(ising_t h, size_t* bytes);

/* The bond thresholds floor(2^32 (1 - exp(-2/T))) of every lattice (host
 * array thr[n_sims], caller-owned). */
int ising_sw_get_thresholds(ising_t h, uint32_t* thr);

/* Advance every lattice by n >= 0 Swendsen-Wang steps.  dev_scratch: device
 * memory (256-byte aligned, caller-owned, contents need not be kept between
 * calls) of scratch_bytes >= ising_sw_scratch_bytes; it must not be used by
 * anything else while the steps run.  Asynchronous on the handle's stream;
 * after each step E and M are recorded exactly as after a sweep (current
 * values, trace ring, FP64 moments if measuring) and the sweep counter
 * advances by one.  Graph replay (ising_set_graph) captures n steps per
 * (n, scratch) pair.  ISING_ENOMEM if the scratch is too small; a union-find
 * walk that runs past its bound (impossible for a consistent label array)
 * makes the next synchronising call return ISING_ETIMEOUT. */
int ising_sw_sweep(ising_t h, int64_t n, void* dev_scratch, size_t scratch_bytes);

/* Advance every lattice by n >= 0 Wolff single-cluster steps (Wolff, PRL 62,
 * 361 (1989)): a seed site is chosen, its cluster grown over nearest
 * neighbours of equal spin joined by active bonds, and flipped.  Draws
 * (Philox4x32-10 keyed by the lattice's seed, counter (q, t, s, phase), t =
 * the step's index in the handle's sweep counter, s = simulation index):
 *   seed, phase 9: r = lane 0 of block q = 0; the seed is site
 *     p0 = floor(r L^2 / 2^32) (p = y*L + x);
 *   bonds, phase 10: site p owns the bonds to (x+1, y) and (x, y+1); q =
 *     p >> 1, lane 2*(p & 1) is the right bond's draw, lane 2*(p & 1) + 1 the
 *     down bond's; a bond is active iff its draw is below the Swendsen-Wang
 *     bond threshold (ising_sw_get_thresholds).
 * With one draw per bond, each bond is tried at most once and the cluster is
 * the seed's connected component among equal spins joined by active bonds.
 * Scratch as for ising_sw_sweep (same size, same rules).  Asynchronous on the
 * handle's stream; after each step E and M are recorded exactly as after a
 * sweep and the sweep counter advances by one.  Steps, Swendsen-Wang steps
 * and Metropolis sweeps share the counter and may be mixed.  Two ways to
 * find the cluster, with the same result bit for bit (ising_wolff_set_method):
 *   growth: one launch for all n steps of every lattice, a block per lattice
 *     growing the cluster level by level -- fast when clusters are small
 *     (above T_c), slow when one spans much of a large lattice;
 *   labelling: the Swendsen-Wang step's labelling of all components of the
 *     Wolff bonds over every SM, the seed's root looked up, and only that
 *     component flipped (seven launches per step; graph replay as for
 *     ising_sw_sweep) -- a fixed cost per site whatever the cluster's size.
 * ISING_WOLFF_AUTO (the default) labels when some lattice of the handle is
 * at T < 2.3, else grows. */
#define ISING_WOLFF_AUTO 0
#define ISING_WOLFF_GROWTH 1
#define ISING_WOLFF_LABELS 2
int ising_wolff_sweep(ising_t h, int64_t n, void* dev_scratch, size_t scratch_bytes);

/* Choose how ising_wolff_sweep finds its clusters (ISING_WOLFF_AUTO, _GROWTH
 * or _LABELS); ISING_EINVAL otherwise. */
int ising_wolff_set_method(ising_t h, int method);

/* Cluster labels of lattice `sim` for the step the handle would take next
 * (its current sweep counter), without taking it: host_labels[L*L]
 * (caller-owned) receives, for every site p = y*L + x, the smallest site
 * index of its cluster.  Synchronises the stream.  The spins and the sweep
 * counter are unchanged. */
int ising_sw_labels(ising_t h, int sim, void* dev_scratch, size_t scratch_bytes, uint32_t* host_labels);

/* ---- Random streams and their quality battery ----------------------------
 * The paper checks its hardware generator's bit stream with the NIST SP
 * 800-22 tests and floats shaped from it for uniformity in 100 bins, lag-1
 * independence and the bits "float >= median" (supplementary, PRNG tests).
 * These calls give the same checks for the Philox4x32-10 stream this library
 * draws. */

/* The draws of sites p0 .. p0 + n_p - 1 in sweeps t0 .. t0 + n_t - 1 for key
 * `seed`, simulation s and phase (0/1 black/white half-sweep, 2 initial
 * state, 4..8 learned proposal and cluster step), exactly as the kernels use
 * them: dev_out[(t - t0) * n_p + (p - p0)] = lane p & 3 of the block with
 * counter (p >> 2, t, s, phase).  dev_out: device memory of n_p * n_t words,
 * 16-byte aligned, caller-owned.  Needs p0 + n_p <= 2^34 and t0 + n_t <= 2^32
 * (ISING_EINVAL otherwise).  Asynchronous on cuda_stream. */
int ising_random_stream(uint64_t seed, uint32_t s, uint32_t phase, uint64_t p0, uint64_t n_p, uint32_t t0,
                        uint32_t n_t, uint32_t* dev_out, void* cuda_stream);

/* The battery on n_words >= 4096 host words (at most 2^30): the bit stream is
 * every word most significant bit first, floats are the paper's shaping
 * (w & 0x7FFFFF) / 2^23.  pvalues[ISING_PRNG_TESTS] (and statistics, if not
 * NULL) receive, in order: frequency (statistic S = ones - zeros), block
 * frequency with 128-bit blocks (chi2), runs (number of runs V; p = 0 when the
 * frequency pre-test fails), longest run of ones in 128-bit blocks in the
 * classes <= 4, 5, 6, 7, 8, >= 9 with exact class probabilities (chi2),
 * spectral on the first 2^k <= min(bits, ISING_PRNG_SPECTRAL_MAX_BITS) bits (d),
 * cumulative sums forward and backward (max excursion z), float uniformity in
 * 100 bins (chi2), non-overlapping float pairs in a 10 x 10 grid (chi2), and
 * runs and longest run of the bits "float >= median".  Host-only. */
#define ISING_PRNG_TESTS 11
#define ISING_PRNG_SPECTRAL_MAX_BITS (1 << 20)
int ising_prng_battery(const uint32_t* words, int64_t n_words, double* pvalues, double* statistics);

/* ---- The three-dimensional sweep -----------------------------------------
 * The paper's Hamiltonian (Section 1) for the simple cubic lattice: periodic
 * L x L x L, J = 1, h = 0, six nearest neighbours; the checkerboard sweep of
 * Algorithm 5 with colours (x + y + z) & 1 (0 = black first).  A site flips
 * iff dE <= 0 or r < thr[dE/4 - 1], thr = min(floor(2^32 exp(-dE/T)),
 * 2^32 - 1) for dE = 4, 8, 12.  Layout: word[((c L + z) L + y) (L/64) + k],
 * bit b <-> x = 2 (32 k + b) + ((y + z + c) & 1), bit 1 = spin -1.  Draws:
 * Philox4x32-10, key (lo32, hi32 of seeds[i]), counter (p >> 2, t, i, phase),
 * lane p & 3, p = (z L + y) (L/2) + (x >> 1) in the half-sweeps (phase 0/1)
 * and p = (z L + y) L + x for the random start (phase 2, +1 iff the top bit
 * is 0).  E = -sum over bonds, M = sum of spins, exact 64-bit integers.
 * Sides: multiples of 64 in [64, ISING3D_MAX_L].  Conventions (errors,
 * ownership, streams) as for the 2D calls above. */
#define ISING3D_MAX_L 1024
typedef struct ising3d_handle* ising3d_t;
int ising3d_workspace_bytes(int n_sims, const int* Ls, int64_t trace_cap, size_t* bytes);
int ising3d_create(ising3d_t* out, int n_sims, const int* Ls, const double* temps, const uint64_t* seeds, int init,
                   int64_t trace_cap, void* dev_workspace, size_t ws_bytes, void* cuda_stream);
/* n sweeps (black then white half-sweep, then E and M into the trace ring);
 * asynchronous; graph replay per n when ising3d_set_graph is on. */
int ising3d_sweep(ising3d_t h, int64_t n);
int ising3d_set_graph(ising3d_t h, int on);
int64_t ising3d_sweeps_done(ising3d_t h);
int64_t ising3d_kernel_launches(ising3d_t h);
int ising3d_observables(ising3d_t h, int64_t* E, int64_t* M);
int ising3d_trace(ising3d_t h, int64_t* E, int64_t* M, int64_t max_sweeps, int64_t* n_out);
/* Unpacked spins of lattice sim, host_LLL[(z L + y) L + x] in {+1, -1}. */
int ising3d_get_spins(ising3d_t h, int sim, int8_t* host_LLL);
void ising3d_destroy(ising3d_t h);

/* Free the handle (not the workspace).  Synchronises its stream. */
void ising_destroy(ising_t h);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */
