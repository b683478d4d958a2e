// ising_learned.cu -- learned patch proposal: a masked-convolution
// autoregressive network over 8x8 patches conditioned on their one-site ring,
// trained by the library's own forward/backward/Adam kernels, used as an
// independence proposal accepted by exact Metropolis-Hastings.
//
// The paper has no learned component; it motivates improving on local moves by
// the critical slowing down of single-site updates near T_c (Section 1).  The
// net, its masks, the move and its random-number keying are defined in
// include/ising.h (ising_net_* and ising_learned_round).
//
// Tensor cores: every layer of the net is a masked 3x3 convolution, i.e. a
// contraction over (tap, input channel).  Teacher-forced scoring of known
// windows -- every position at once, M = 128 rows per window -- runs on the
// tcgen05 tensor cores (ising_learned_tc.cu).  The kernels here are the
// sequential ones: the training forward (which also keeps the activations for
// the backward pass) and the samplers, whose positions depend on each other.
// They run mma.sync (BF16 m16n8k16, E4M3 m16n8k32, FP32 accumulate), whose
// register-level hand-off from one layer's accumulator fragment to the next
// layer's operand fragment suits their short dependent chains: the M dimension
// holds the windows of one warp (8 of the 16 rows in the sequential forward),
// K = 16 input channels of one tap (a k-step per tap), N = 16 output channels
// (two n-tiles).
#include "../../include/ising.h"
#include "ising_internal.h"
#include "ising_device.cuh"

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace ising {
namespace {

constexpr int kS = 10;          // window side
constexpr int kNPos = kS * kS;  // window positions
constexpr int kP = 8;           // interior side
constexpr int kC = 16;          // channels
constexpr int kSlots = 12;      // activation ring buffer (taps reach 11 positions back)
constexpr int kOffW1 = 0, kOffB1 = 256, kOffW2 = 272, kOffB2 = 1552, kOffW3 = 1568, kOffB3 = 2848,
              kOffW4 = 2864, kOffB4 = 2944;
constexpr int kNParams = ISING_NET_PARAMS;
static_assert(kOffB4 + 1 == ISING_NET_PARAMS, "parameter layout");
constexpr int kWarpsFwd = 4;
constexpr int kWin = 8;                                       // windows per warp (rows 0..7 of the m16 tile)
constexpr int kRowH = 24;                                     // bf16 per activation row: 16 + 8 padding
// per-warp shared memory of the sequential BF16 forward kernel: spins [8][100]
// int8 and the activation ring [3 layers][12 slots][8 windows][24] bf16 (rows
// padded so the fragment loads of 8 rows x 4 lanes hit 32 distinct banks)
constexpr int kSpinBytes = kWin * kNPos;                      // 800
constexpr int kRingBytes = 3 * kSlots * kWin * kRowH * 2;     // 13824
constexpr int kWarpSmem = kSpinBytes + kRingBytes;            // 14624 (multiple of 16)

// (dy, dx) of the "mask B" taps and of the layer-1 features
__constant__ int8_t c_tapB[5][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 0}};
__constant__ int8_t c_feat[16][3] = {
    // dy, dx, kind (0 = interior spin, 1 = ring spin, 2 = zero)
    {-1, -1, 0}, {-1, 0, 0}, {-1, 1, 0}, {0, -1, 0},
    {-1, -1, 1}, {-1, 0, 1}, {-1, 1, 1}, {0, -1, 1}, {0, 0, 1}, {0, 1, 1}, {1, -1, 1}, {1, 0, 1}, {1, 1, 1},
    {0, 0, 2}, {0, 0, 2}, {0, 0, 2}};

__device__ __forceinline__ bool interior(int r, int c) { return r >= 1 && r <= kP && c >= 1 && c <= kP; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float log_sigmoid(float t) {
    return -(fmaxf(-t, 0.0f) + log1pf(expf(-fabsf(t))));
}

// B fragment of a K x N = 16 x 8 slice of a row-major [k][n] bf16 matrix
// (row stride ld): k = 2*(lane%4) + {0,1} and +8, n = lane/4.
__device__ __forceinline__ void load_b(const __nv_bfloat16* m, int ld, int n0, int ncols, uint32_t (&b)[2]) {
    const int lane = threadIdx.x & 31, k = 2 * (lane & 3), n = n0 + (lane >> 2);
    auto at = [&](int kk) -> float { return n < ncols ? __bfloat162float(m[kk * ld + n]) : 0.0f; };
    b[0] = pack_bf16(at(k), at(k + 1));
    b[1] = pack_bf16(at(k + 8), at(k + 9));
}

struct NetPtrs {
    const __nv_bfloat16* wb;  // bf16 copy of the parameters (weights used by the mma)
    const float* wf;          // fp32 master parameters (biases)
};

// ---------------------------------------------------------------------------
// Sequential teacher-forced forward over the 100 window positions for 8
// windows per warp (rows 0..7 of each m16 tile; rows 8..15 are zero), the
// forward pass of training.  Writes lq[w] = log q(window w) (fp32 sum), and
// optionally the logits z[w][p] and the activations h[l][w][p][c] that the
// backward kernel reads.
//
// In the m16n8k16 layout the C fragment a thread holds for an output position
// (row g, channels 2tq, 2tq+1, 8+2tq, 9+2tq) is exactly the A fragment the next
// layer needs from that position, so the (0,0) and (0,-1) taps of layers 2-4
// come from registers; only the three taps of the previous row go through a
// shared-memory ring written once per position and read about ten positions
// later.  Layers 2-4 accumulate their taps in independent chains summed at
// the end.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsFwd * 32) ar_net_kernel(NetPtrs net, const int8_t* win, int n, float* lq,
                                                                 float* z_out, __nv_bfloat16* h_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int w0 = (blockIdx.x * kWarpsFwd + warp) * kWin;
    if (w0 >= n) return;
    unsigned char* wbase = smem + warp * kWarpSmem;
    int8_t* sp = reinterpret_cast<int8_t*>(wbase);
    __nv_bfloat16* ring = reinterpret_cast<__nv_bfloat16*>(wbase + kSpinBytes);
    auto H = [&](int layer, int slot, int row) -> __nv_bfloat16* {
        return ring + ((layer * kSlots + slot) * kWin + row) * kRowH;
    };
    for (int i = lane; i < kWin * kNPos; i += 32) {
        const int row = i / kNPos;
        sp[i] = (w0 + row < n) ? win[(size_t)(w0 + row) * kNPos + (i - row * kNPos)] : (int8_t)0;
    }
    // weights -> B fragments (registers)
    uint32_t bw1[2][2], bw2[5][2][2], bw3[5][2][2], bw4[5][2];
    load_b(net.wb + kOffW1, kC, 0, kC, bw1[0]);
    load_b(net.wb + kOffW1, kC, 8, kC, bw1[1]);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        load_b(net.wb + kOffW2 + t * 256, kC, 0, kC, bw2[t][0]);
        load_b(net.wb + kOffW2 + t * 256, kC, 8, kC, bw2[t][1]);
        load_b(net.wb + kOffW3 + t * 256, kC, 0, kC, bw3[t][0]);
        load_b(net.wb + kOffW3 + t * 256, kC, 8, kC, bw3[t][1]);
        load_b(net.wb + kOffW4 + t * kC, 1, 0, 1, bw4[t]);     // N = 1 (column 0 only)
    }
    float bias[3][2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int co = nt * 8 + 2 * tq + e;
            bias[0][nt][e] = net.wf[kOffB1 + co];
            bias[1][nt][e] = net.wf[kOffB2 + co];
            bias[2][nt][e] = net.wf[kOffB3 + co];
        }
    const float b4 = net.wf[kOffB4];
    // this thread's four layer-1 features: k = 2tq, 2tq+1, 2tq+8, 2tq+9
    int fdy[4], fdx[4], fkind[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 2 * tq + (e & 1) + ((e >> 1) ? 8 : 0);
        fdy[e] = c_feat[k][0];
        fdx[e] = c_feat[k][1];
        fkind[e] = c_feat[k][2];
    }
    float lq_acc = 0.0f;
    __syncwarp();

    uint32_t hprev[3][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}};   // layer outputs at the previous column
    float xprev = 0.0f;                                          // window g's spin at the previous column
    for (int r = 0; r < kS; ++r) {
#pragma unroll
        for (int c = 0; c < kS; ++c) {
            const int p = r * kS + c, slot = p % kSlots;
            // ---- layer 1: features (mask A interior taps + ring taps) ----
            uint32_t a[4];
            {
                const int8_t* s = sp + g * kNPos;
                float f[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int yy = r + fdy[e], xx = c + fdx[e];
                    float v = 0.0f;
                    if (fkind[e] != 2 && yy >= 0 && yy < kS && xx >= 0 && xx < kS) {
                        const bool in = interior(yy, xx);
                        if ((fkind[e] == 0) == in) {
                            // the left neighbour in the current row is the spin just decided
                            v = (fdy[e] == 0 && fkind[e] == 0) ? xprev : (float)s[yy * kS + xx];
                        }
                    }
                    f[e] = v;
                }
                a[0] = pack_bf16(f[0], f[1]);
                a[1] = 0u;
                a[2] = pack_bf16(f[2], f[3]);
                a[3] = 0u;
            }
            uint32_t hcur[3][2];
#pragma unroll
            for (int layer = 0; layer < 3; ++layer) {
                float d[5][2][4] = {};   // one accumulator per tap: every mma of a layer is independent
                if (layer == 0) {
                    mma16816(d[0][0], a, bw1[0]);
                    mma16816(d[0][1], a, bw1[1]);
                } else {
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        const int dy = (t < 3) ? -1 : 0, dx = (t < 3) ? t - 1 : (t == 3 ? -1 : 0);
                        const int yy = r + dy, xx = c + dx;
                        if (yy < 0 || xx < 0 || xx >= kS) continue;
                        uint32_t at[4];
                        if (t < 3) {            // previous row: from the ring
                            const int sl = (p + dy * kS + dx + kSlots) % kSlots;
                            const __nv_bfloat16* h0 = H(layer - 1, sl, g);
                            at[0] = *reinterpret_cast<const uint32_t*>(h0 + 2 * tq);
                            at[2] = *reinterpret_cast<const uint32_t*>(h0 + 2 * tq + 8);
                        } else if (t == 3) {    // previous column: registers
                            at[0] = hprev[layer - 1][0];
                            at[2] = hprev[layer - 1][1];
                        } else {                // this position: registers
                            at[0] = hcur[layer - 1][0];
                            at[2] = hcur[layer - 1][1];
                        }
                        at[1] = 0u;
                        at[3] = 0u;
                        if (layer == 1) { mma16816(d[t][0], at, bw2[t][0]); mma16816(d[t][1], at, bw2[t][1]); }
                        else { mma16816(d[t][0], at, bw3[t][0]); mma16816(d[t][1], at, bw3[t][1]); }
                    }
                }
                // bias, relu, bf16: the A fragment of the next layer
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const float s0 = ((d[0][nt][0] + d[1][nt][0]) + (d[2][nt][0] + d[3][nt][0])) + d[4][nt][0];
                    const float s1 = ((d[0][nt][1] + d[1][nt][1]) + (d[2][nt][1] + d[3][nt][1])) + d[4][nt][1];
                    const uint32_t v0 = pack_bf16(fmaxf(s0 + bias[layer][nt][0], 0.f),
                                                  fmaxf(s1 + bias[layer][nt][1], 0.f));
                    hcur[layer][nt] = v0;
                    *reinterpret_cast<uint32_t*>(H(layer, slot, g) + nt * 8 + 2 * tq) = v0;
                    if (h_out && w0 + g < n)
                        *reinterpret_cast<uint32_t*>(h_out + (((size_t)layer * n + w0 + g) * kNPos + p) * kC +
                                                     nt * 8 + 2 * tq) = v0;
                }
            }
            // ---- layer 4: the logit ----
            float d4[5][4] = {};
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const int dy = (t < 3) ? -1 : 0, dx = (t < 3) ? t - 1 : (t == 3 ? -1 : 0);
                const int yy = r + dy, xx = c + dx;
                if (yy < 0 || xx < 0 || xx >= kS) continue;
                uint32_t at[4];
                if (t < 3) {
                    const int sl = (p + dy * kS + dx + kSlots) % kSlots;
                    const __nv_bfloat16* h0 = H(2, sl, g);
                    at[0] = *reinterpret_cast<const uint32_t*>(h0 + 2 * tq);
                    at[2] = *reinterpret_cast<const uint32_t*>(h0 + 2 * tq + 8);
                } else if (t == 3) {
                    at[0] = hprev[2][0];
                    at[2] = hprev[2][1];
                } else {
                    at[0] = hcur[2][0];
                    at[2] = hcur[2][1];
                }
                at[1] = 0u;
                at[3] = 0u;
                mma16816(d4[t], at, bw4[t]);
            }
            const float z = (((d4[0][0] + d4[1][0]) + (d4[2][0] + d4[3][0])) + d4[4][0]) + b4;   // lanes tq == 0
            float xs = 0.0f;
            if (interior(r, c)) {
                const int8_t x = sp[g * kNPos + p];
                if (tq == 0 && w0 + g < n) lq_acc += log_sigmoid((float)x * z);
                xs = (float)x;
            }
            if (tq == 0 && w0 + g < n && z_out) z_out[(size_t)(w0 + g) * kNPos + p] = z;
#pragma unroll
            for (int layer = 0; layer < 3; ++layer) { hprev[layer][0] = hcur[layer][0]; hprev[layer][1] = hcur[layer][1]; }
            xprev = xs;
            __syncwarp();
        }
    }
    if (tq == 0 && w0 + g < n) lq[w0 + g] = lq_acc;
}

// ---------------------------------------------------------------------------
// Padded window layout shared by the sampler: position (r, c) is row
// (r + 1) * 11 + c + 1 of a buffer whose rows 0 .. 11 and every multiple of 11
// are zero (the column left of a window row is the one right of the
// previous), so every input outside the window is a zero row and tap (dy, dx)
// of row q is row q + 11 dy + dx.  Activation rows are 24 bf16 (16 channels +
// 8 padding, 48 bytes: 16-byte aligned, conflict-free ldmatrix phases).
// (Teacher-forced scoring of known windows runs on the tcgen05 tensor cores,
// ising_learned_tc.cu.)
// ---------------------------------------------------------------------------
constexpr int kPW = kS + 1;                                      // padded row pitch (11)
constexpr int kRow0 = kPW + 1;                                   // row of position (0, 0): 12
constexpr int kRowBytes = kRowH * 2;                             // 48: rows stay 16-byte aligned
constexpr int kSpinRows = kRow0 + 112 + kPW + 1;                 // padded spins, room for dy = +1 taps (136)

__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void stmatrix_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};\n"
                 :: "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3) : "memory");
}
__device__ __forceinline__ int padded_row(int p) { return p + p / kS + kRow0; }

// ---------------------------------------------------------------------------
// Autoregressive sampling by wavefronts.  The logit of position (r, c)
// depends on spins and activations at (r', c') with r' < r and c' <= c + (r - r')
// (c' <= c in row r - 1) or r' = r, c' < c, so every position on the line
// s = c + 2r can be sampled at once once the lines before it are done: 28
// steps of at most five positions replace the 100 sequential positions, with
// the same arithmetic at every position (the sampled spins equal the raster
// order's).  One warp carries three windows; the rows of its m16 tile are
// (window w, k-th position of the step), row 5w + k (row 15 idle).
//
// Per step: the four taps of layers 2 and 3 that come from the three previous
// steps are gathered by ldmatrix from per-window rings (the last four steps'
// layer-1 and layer-2 outputs) and multiplied first, into accumulators that
// start at the bias; then layer 1 (A fragment from padded spin arrays of
// interior and ring sites, as in the scoring kernel), and the (0, 0) taps of
// layers 2 and 3 straight from registers (the C fragment of a layer is the A
// fragment of the next); layer 4 is one n8 mma giving u[t] = H3 . W4[t] per
// row, kept in a ring, and the logit is b4 + sum_t u[source_t][t].  Lanes
// 0 .. 14 then sample their row's site from its draw.  Rows that are idle in
// a step read the zero slot and write a trash slot.  Per-step row geometry
// comes from two block-shared tables.
// ---------------------------------------------------------------------------
constexpr int kSteps = 3 * kS - 2;                     // s = c + 2r in [0, 27]
constexpr int kPerStep = 5;
constexpr int kWinT = 3;                               // windows per warp
constexpr int kWarpsSmp = 4;
constexpr int kRingSlots = 4 * kPerStep;               // rows of the last four steps
constexpr int kZeroSlot = kRingSlots, kTrashSlot = kRingSlots + 1;
constexpr int kLayerRows = kRingSlots + 2;             // 22 rows of one layer's ring
constexpr int kSmpRing = 2 * kLayerRows * kRowBytes;   // layers 1 and 2: 2112 bytes
constexpr int kSmpSpin = kSmpRing;                     // interior then ring spins, bf16 bits
constexpr int kSmpU = kSmpSpin + 2 * 2 * kSpinRows;    // u ring: kLayerRows x 5 floats (+2)
constexpr int kSmpDraws = kSmpU + 112 * 4;             // 64 draws
constexpr int kSmpWinBytes = kSmpDraws + 64 * 4;       // 3360
// window stride: 16-byte chunk index = 7 (mod 8), so that the tile rows 5w + k
// of one step fall into distinct bank groups at the 48-byte row pitch
constexpr int kSmpWinStride = (kSmpWinBytes / 16 + (15 - (kSmpWinBytes / 16) % 8) % 8) * 16;   // 3440
static_assert(kSmpWinBytes % 16 == 0 && kSmpWinStride >= kSmpWinBytes && kSmpWinStride - kSmpWinBytes < 128 &&
                  (kSmpWinStride / 16) % 8 == 7, "window stride");
static_assert(kLayerRows * 5 <= 112, "u ring");
// tables: per (step, tile row) 8 bytes {source slot of taps 0..4, own slot (or
// trash), draw index (0xFF: nothing to sample), padded site row}; per (step,
// g) 4 bytes {padded site rows of tile rows g and g + 8, their own slots}
constexpr int kSmpTabR = kSteps * 16 * 8;
constexpr int kSmpTabC = kSteps * 8 * 4;
constexpr int kSmpSmem = kWarpsSmp * kWinT * kSmpWinStride + kSmpTabR + kSmpTabC;

__device__ __forceinline__ int step_rmin(int s) { return s >= 9 ? (s - 8) / 2 : 0; }
__device__ __forceinline__ int step_count(int s) { return min(kS - 1, s / 2) - step_rmin(s) + 1; }
// d = a b + c with c = (c0, c1) in both row halves: the bias as the accumulator input
__device__ __forceinline__ void mma16816_bias(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2],
                                              float c0, float c1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%10,%11};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(c0), "f"(c1));
}

// Per-step row tables of the wavefront samplers, filled by the whole block:
// per (step, tile row) 8 bytes {source slot of taps 0..4, own slot (or
// trash), draw index (0xFF: nothing to sample), padded site row}; per (step,
// g) 4 bytes {padded site rows of tile rows g and g + 8, their own slots}.
__device__ void fill_sampler_tables(uint2* tabR, uint32_t* tabC) {
    for (int i = threadIdx.x; i < kSteps * 16; i += blockDim.x) {
        const int st = i >> 4, row = i & 15, k = row % kPerStep;
        uint32_t b[8] = {kZeroSlot, kZeroSlot, kZeroSlot, kZeroSlot, kZeroSlot, kTrashSlot, 0xFFu, kRow0};
        if (row < kPerStep * kWinT && k < step_count(st)) {
            const int r = step_rmin(st) + k, c = st - 2 * r;
#pragma unroll 1
            for (int t = 0; t < 5; ++t) {
                const int y = r + c_tapB[t][0], x = c + c_tapB[t][1];
                if (y >= 0 && x >= 0 && x < kS) b[t] = kPerStep * ((x + 2 * y) & 3) + (y - step_rmin(x + 2 * y));
            }
            b[5] = kPerStep * (st & 3) + k;
            if (interior(r, c)) b[6] = (r - 1) * kP + (c - 1);
            b[7] = (r + 1) * kPW + c + 1;
        }
        tabR[i] = make_uint2(b[0] | b[1] << 8 | b[2] << 16 | b[3] << 24, b[4] | b[5] << 8 | b[6] << 16 | b[7] << 24);
    }
    for (int i = threadIdx.x; i < kSteps * 8; i += blockDim.x) {
        const int st = i >> 3, gg = i & 7;
        uint32_t v = 0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int row = gg + 8 * h, k = row % kPerStep;
            uint32_t q = kRow0, own = kTrashSlot;
            if (row < kPerStep * kWinT && k < step_count(st)) {
                const int r = step_rmin(st) + k, c = st - 2 * r;
                q = (r + 1) * kPW + c + 1;
                own = kPerStep * (st & 3) + k;
            }
            v |= q << (8 * h) | own << (16 + 8 * h);
        }
        tabC[i] = v;
    }
}

__global__ void __launch_bounds__(kWarpsSmp * 32, 4) ar_sample_kernel(NetPtrs net, int8_t* win, int n, float* lq,
                                                                  const LearnedKey* keys, uint32_t round_t) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    uint2* tabR = reinterpret_cast<uint2*>(smem + kWarpsSmp * kWinT * kSmpWinStride);
    uint32_t* tabC = reinterpret_cast<uint32_t*>(smem + kWarpsSmp * kWinT * kSmpWinStride + kSmpTabR);
    fill_sampler_tables(tabR, tabC);
    unsigned char* wb = smem + warp * kWinT * kSmpWinStride;
    auto wbase = [&](int w) -> unsigned char* { return wb + w * kSmpWinStride; };
    uint32_t bw1[2][2], bw2[5][2][2], bw3[5][2][2], bw4[2];
    load_b(net.wb + kOffW1, kC, 0, kC, bw1[0]);
    load_b(net.wb + kOffW1, kC, 8, kC, bw1[1]);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        load_b(net.wb + kOffW2 + t * 256, kC, 0, kC, bw2[t][0]);
        load_b(net.wb + kOffW2 + t * 256, kC, 8, kC, bw2[t][1]);
        load_b(net.wb + kOffW3 + t * 256, kC, 0, kC, bw3[t][0]);
        load_b(net.wb + kOffW3 + t * 256, kC, 8, kC, bw3[t][1]);
    }
    {
        auto at = [&](int k) -> float { return g < 5 ? __bfloat162float(net.wb[kOffW4 + g * kC + k]) : 0.0f; };
        bw4[0] = pack_bf16(at(2 * tq), at(2 * tq + 1));
        bw4[1] = pack_bf16(at(2 * tq + 8), at(2 * tq + 9));
    }
    float bias[3][2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int co = nt * 8 + 2 * tq + e;
            bias[0][nt][e] = net.wf[kOffB1 + co];
            bias[1][nt][e] = net.wf[kOffB2 + co];
            bias[2][nt][e] = net.wf[kOffB3 + co];
        }
    const float b4 = net.wf[kOffB4];
    // this lane's four layer-1 features (2tq, 2tq+1, 2tq+8, 2tq+9): offsets into
    // the window's spin arrays (the ring copy kSpinRows further) and masks
    int foff[4];
    uint32_t fmask[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 2 * tq + (e & 1) + ((e >> 1) ? 8 : 0), kind = c_feat[k][2];
        foff[e] = kind == 2 ? 0 : (kind == 1 ? kSpinRows : 0) + c_feat[k][0] * kPW + c_feat[k][1];
        fmask[e] = kind == 2 ? 0u : 0xFFFFu;
    }
    // the window of this lane's ldmatrix row (lane & 15; row 15 idle -> window 2) and of its C rows g, g + 8
    const int lr = lane & 15, lwc = min(lr / kPerStep, kWinT - 1);
    const int cw0 = g / kPerStep, cw1c = min((g + 8) / kPerStep, kWinT - 1);
    const uint32_t ring_l = (uint32_t)__cvta_generic_to_shared(wbase(lwc)) + (uint32_t)(lane >> 4) * 16u;
    const uint16_t* spin0 = reinterpret_cast<const uint16_t*>(wbase(cw0) + kSmpSpin);
    const uint16_t* spin1 = reinterpret_cast<const uint16_t*>(wbase(cw1c) + kSmpSpin);
    float* u0 = reinterpret_cast<float*>(wbase(cw0) + kSmpU);
    float* u1 = reinterpret_cast<float*>(wbase(cw1c) + kSmpU);
    unsigned char* wl = wbase(lwc);
    const float* ul = reinterpret_cast<const float*>(wl + kSmpU);
    __syncthreads();

    constexpr uint32_t kL2 = kLayerRows * kRowBytes;       // the layer-2 ring after the layer-1 ring
    // persistent over groups of three windows
    for (int w0 = (blockIdx.x * kWarpsSmp + warp) * kWinT; w0 < n; w0 += gridDim.x * kWarpsSmp * kWinT) {
    // zero the rings (zero slots included), spins, u ring; the input window's ring sites; the draws
    for (int i = lane; i < kWinT * kSmpWinStride / 4; i += 32) reinterpret_cast<uint32_t*>(wb)[i] = 0u;
    __syncwarp();
    for (int i = lane; i < kWinT * kNPos; i += 32) {
        const int w = i / kNPos, p = i - w * kNPos;
        if (w0 + w < n && !interior(p / kS, p % kS)) {
            const int8_t x = win[(size_t)(w0 + w) * kNPos + p];
            reinterpret_cast<uint16_t*>(wbase(w) + kSmpSpin)[kSpinRows + padded_row(p)] =
                x > 0 ? 0x3F80u : (x < 0 ? 0xBF80u : 0u);
        }
    }
    for (int bq = lane; bq < kWinT * 16; bq += 32) {
        const int w = bq >> 4, q = bq & 15;
        if (w0 + w < n) {
            const LearnedKey k = keys[w0 + w];
            const uint4 rv = philox(16u * k.j + (uint32_t)q, round_t, k.sim, 4u, k.key0, k.key1);
            uint32_t* d = reinterpret_cast<uint32_t*>(wbase(w) + kSmpDraws) + 4 * q;
            d[0] = rv.x; d[1] = rv.y; d[2] = rv.z; d[3] = rv.w;
        }
    }
    __syncwarp();
    float lq_acc = 0.0f;
#pragma unroll 1
    for (int s = 0; s < kSteps; ++s) {
        const uint2 dr = tabR[s * 16 + lr];
        const uint32_t dc = tabC[s * 8 + g];
        const uint32_t sl0 = dr.x & 0xFF, sl1 = (dr.x >> 8) & 0xFF, sl2 = (dr.x >> 16) & 0xFF, sl3 = dr.x >> 24;
        const uint32_t sl4 = dr.y & 0xFF, own = (dr.y >> 8) & 0xFF;
        // ---- the ring taps of layers 2 and 3, into bias-initialised accumulators ----
        float d2[2][4], d3[2][4];
        {
            uint32_t at[4][4];
            ldmatrix_x4(at[0], ring_l + sl0 * kRowBytes);
            ldmatrix_x4(at[1], ring_l + sl1 * kRowBytes);
            ldmatrix_x4(at[2], ring_l + sl2 * kRowBytes);
            ldmatrix_x4(at[3], ring_l + sl3 * kRowBytes);
            mma16816_bias(d2[0], at[0], bw2[0][0], bias[1][0][0], bias[1][0][1]);
            mma16816_bias(d2[1], at[0], bw2[0][1], bias[1][1][0], bias[1][1][1]);
#pragma unroll
            for (int t = 1; t < 4; ++t) { mma16816(d2[0], at[t], bw2[t][0]); mma16816(d2[1], at[t], bw2[t][1]); }
            ldmatrix_x4(at[0], ring_l + kL2 + sl0 * kRowBytes);
            ldmatrix_x4(at[1], ring_l + kL2 + sl1 * kRowBytes);
            ldmatrix_x4(at[2], ring_l + kL2 + sl2 * kRowBytes);
            ldmatrix_x4(at[3], ring_l + kL2 + sl3 * kRowBytes);
            mma16816_bias(d3[0], at[0], bw3[0][0], bias[2][0][0], bias[2][0][1]);
            mma16816_bias(d3[1], at[0], bw3[0][1], bias[2][1][0], bias[2][1][1]);
#pragma unroll
            for (int t = 1; t < 4; ++t) { mma16816(d3[0], at[t], bw3[t][0]); mma16816(d3[1], at[t], bw3[t][1]); }
        }
        // ---- layer 1 ----
        const int q0 = dc & 0xFF, q1 = (dc >> 8) & 0xFF;
        uint32_t h[4];
        {
            uint32_t f0[4], f1[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                f0[e] = spin0[q0 + foff[e]] & fmask[e];
                f1[e] = spin1[q1 + foff[e]] & fmask[e];
            }
            const uint32_t a[4] = {f0[0] | (f0[1] << 16), f1[0] | (f1[1] << 16), f0[2] | (f0[3] << 16),
                                   f1[2] | (f1[3] << 16)};
            float d[2][4];
            mma16816_bias(d[0], a, bw1[0], bias[0][0][0], bias[0][0][1]);
            mma16816_bias(d[1], a, bw1[1], bias[0][1][0], bias[0][1][1]);
            h[0] = pack_bf16_relu(d[0][0], d[0][1]); h[1] = pack_bf16_relu(d[0][2], d[0][3]);
            h[2] = pack_bf16_relu(d[1][0], d[1][1]); h[3] = pack_bf16_relu(d[1][2], d[1][3]);
            stmatrix_x4(ring_l + own * kRowBytes, h[0], h[1], h[2], h[3]);
        }
        // ---- layers 2 and 3: the (0, 0) taps ----
        mma16816(d2[0], h, bw2[4][0]);
        mma16816(d2[1], h, bw2[4][1]);
        h[0] = pack_bf16_relu(d2[0][0], d2[0][1]); h[1] = pack_bf16_relu(d2[0][2], d2[0][3]);
        h[2] = pack_bf16_relu(d2[1][0], d2[1][1]); h[3] = pack_bf16_relu(d2[1][2], d2[1][3]);
        stmatrix_x4(ring_l + kL2 + own * kRowBytes, h[0], h[1], h[2], h[3]);
        mma16816(d3[0], h, bw3[4][0]);
        mma16816(d3[1], h, bw3[4][1]);
        h[0] = pack_bf16_relu(d3[0][0], d3[0][1]); h[1] = pack_bf16_relu(d3[0][2], d3[0][3]);
        h[2] = pack_bf16_relu(d3[1][0], d3[1][1]); h[3] = pack_bf16_relu(d3[1][2], d3[1][3]);
        // ---- layer 4: u[t] of rows g, g + 8 (columns 2tq, 2tq + 1) into the u ring ----
        {
            float d4[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816(d4, h, bw4);
            const int c0 = 2 * tq, o0 = (int)((dc >> 16) & 0xFF) * 5 + c0, o1 = (int)(dc >> 24) * 5 + c0;
            if (c0 < 5) { u0[o0] = d4[0]; u1[o1] = d4[2]; }
            if (c0 + 1 < 5) { u0[o0 + 1] = d4[1]; u1[o1 + 1] = d4[3]; }
        }
        __syncwarp();
        // ---- sample: lane lr < 15 takes its row's site when it has one ----
        const uint32_t di = (dr.y >> 16) & 0xFF;
        if (lane < 16 && di != 0xFFu) {
            const float z = b4 + ul[sl0 * 5 + 0] + ul[sl1 * 5 + 1] + ul[sl2 * 5 + 2] + ul[sl3 * 5 + 3] + ul[sl4 * 5 + 4];
            const uint32_t draw = reinterpret_cast<const uint32_t*>(wl + kSmpDraws)[di];
            const float sg = __frcp_rn(1.0f + expf(-z));        // = 1 / (1 + e^-z), correctly rounded
            const uint32_t thr = (sg >= 1.0f) ? 0xFFFFFFFFu : (uint32_t)(sg * 4294967296.0f);
            const float x = draw < thr ? 1.0f : -1.0f;
            reinterpret_cast<uint16_t*>(wl + kSmpSpin)[dr.y >> 24] = x > 0.f ? 0x3F80u : 0xBF80u;
            if (lq) lq_acc += log_sigmoid(x * z);
        }
        __syncwarp();
    }
    // log q per window: lanes 5w .. 5w + 4
    float* lqs = reinterpret_cast<float*>(wb + kSmpU);     // window 0's u ring is free now
    if (lane < 16) lqs[lane] = lq_acc;
    __syncwarp();
    if (lane < kWinT && w0 + lane < n && lq) {
        float t = 0.0f;
        for (int k = 0; k < kPerStep; ++k) t += lqs[kPerStep * lane + k];
        lq[w0 + lane] = t;
    }
    // the sampled interiors back into the windows
    for (int i = lane; i < kWinT * kNPos; i += 32) {
        const int w = i / kNPos, p = i - w * kNPos;
        if (w0 + w < n && interior(p / kS, p % kS)) {
            const uint16_t v = reinterpret_cast<const uint16_t*>(wbase(w) + kSmpSpin)[padded_row(p)];
            win[(size_t)(w0 + w) * kNPos + p] = v == 0x3F80u ? (int8_t)1 : (int8_t)-1;
        }
    }
    __syncwarp();                       // the window buffers are cleared for the next group
    }
}

// ---------------------------------------------------------------------------
// FP8 (E4M3) helpers: 16-byte activation rows, mma.sync.m16n8k32 e4m3 x e4m3 ->
// f32, and B fragments from the e4m3 weight copy.
// ---------------------------------------------------------------------------
constexpr int kRowQ = 16;                                     // fp8 per activation row (16 channels)

__device__ __forceinline__ void mma16832_e4m3(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragment (K x N = 32 x 8, 8-bit) from the fp8 weight copy: k = 4*(lane%4)
// + {0..3} and 16 + that, n = lane/4.  wk(k, n) returns the byte of row k.
template <typename F>
__device__ __forceinline__ void load_b8(F wk, uint32_t (&b)[2]) {
    const int lane = threadIdx.x & 31, k = 4 * (lane & 3), n = lane >> 2;
    uint32_t r0 = 0, r1 = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        r0 |= (uint32_t)wk(k + e, n) << (8 * e);
        r1 |= (uint32_t)wk(16 + k + e, n) << (8 * e);
    }
    b[0] = r0;
    b[1] = r1;
}

// ---------------------------------------------------------------------------
// FP8 (E4M3) autoregressive sampling by wavefronts: the schedule, tables and
// window grouping of ar_sample_kernel (28 steps of at most five positions,
// three windows per warp, rows 5w + k of the m16 tile), with the FP8
// arithmetic of the sequential FP8 kernel: e4m3 activations, e4m3 weights
// times their power-of-two layer scale, mma.sync.m16n8k32 e4m3 x e4m3 -> f32.
// One k32 step takes two taps: the four taps of the previous steps pair up as
// (0, 1) and (2, 3), gathered by ldmatrix from per-window rings of 16-byte
// rows (lanes 0-15 address the first tap's rows, lanes 16-31 the second's);
// the (0, 0) tap is this step's own output, with a zero second half.  An
// m16n8k32 accumulator fragment holds channels 2tq, 2tq + 1, 8 + 2tq, 9 + 2tq
// of rows g, g + 8, while an operand fragment holds k = 4tq .. 4tq + 3.  The
// hidden layers' channels are internal, so their operand order is permuted to
// match (k = 4tq + e is channel chan_perm(k); the weight rows of layers 2-4
// are permuted the same way): each lane's rounded accumulators are its operand
// word as they stand, for the own-tap product and for the stmatrix into the
// ring, with no exchange between lanes.
// Accumulators start at bias x s_l (exact: s_l is a power of two) and are
// scaled by 1 / s_l before relu and the e4m3 rounding, as (sum / s_l) + bias.
// ---------------------------------------------------------------------------
constexpr int kSmpQRing = 2 * kLayerRows * kRowQ;               // layers 1 and 2: 704 bytes
constexpr int kSmpQSpin = kSmpQRing;                            // interior then ring spins, e4m3 codes
constexpr int kSmpQU = kSmpQSpin + 2 * kSpinRows;               // u ring: kLayerRows x 5 floats (+2)
constexpr int kSmpQDraws = kSmpQU + 112 * 4;                    // 64 draws
constexpr int kSmpQWinBytes = kSmpQDraws + 64 * 4;              // 1680 = 105 16-byte chunks (odd)
constexpr int kSmpQSmem = kWarpsSmp * kWinT * kSmpQWinBytes + kSmpTabR + kSmpTabC;
static_assert(kSmpQU % 16 == 0 && kSmpQWinBytes % 16 == 0 && (kSmpQWinBytes / 16) % 2 == 1, "fp8 sampler layout");
constexpr uint8_t kE4m3Plus = 0x38, kE4m3Minus = 0xB8;          // +1, -1

__device__ __forceinline__ void stmatrix_x2(uint32_t addr, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.shared.b16 [%0], {%1, %2};\n" :: "r"(addr), "r"(r0), "r"(r1) : "memory");
}

// The hidden channel behind operand index k = 4tq + e: the accumulator
// fragment's channels 2tq, 2tq + 1, 8 + 2tq, 9 + 2tq for e = 0 .. 3.
__host__ __device__ constexpr int chan_perm(int k) { return 2 * (k >> 2) + (k & 1) + ((k & 2) ? 8 : 0); }

// relu(d / s) rounded to e4m3 for the two n-tiles of a row pair: out[0] = row
// g, out[1] = row g + 8, bytes in chan_perm order (operand words of this lane)
__device__ __forceinline__ void layer_out_e4m3(const float (&d)[2][4], float inv_s, uint32_t (&out)[2]) {
    auto p = [&](float a, float b) -> uint32_t {       // a in the low byte
        uint16_t r;
        asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(b * inv_s), "f"(a * inv_s));
        return r;
    };
    out[0] = p(d[0][0], d[0][1]) | (p(d[1][0], d[1][1]) << 16);
    out[1] = p(d[0][2], d[0][3]) | (p(d[1][2], d[1][3]) << 16);
}

__global__ void __launch_bounds__(kWarpsSmp * 32, 4) ar_sample_fp8_kernel(const uint8_t* wq, const float* wscale,
                                                                       const float* wf, int8_t* win, int n, float* lq,
                                                                       const LearnedKey* keys, uint32_t round_t) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    uint2* tabR = reinterpret_cast<uint2*>(smem + kWarpsSmp * kWinT * kSmpQWinBytes);
    uint32_t* tabC = reinterpret_cast<uint32_t*>(smem + kWarpsSmp * kWinT * kSmpQWinBytes + kSmpTabR);
    fill_sampler_tables(tabR, tabC);
    unsigned char* wb = smem + warp * kWinT * kSmpQWinBytes;
    auto wbase = [&](int w) -> unsigned char* { return wb + w * kSmpQWinBytes; };
    const float s1 = wscale[0], s2 = wscale[1], s3 = wscale[2];
    const float inv_s[4] = {1.0f / wscale[0], 1.0f / wscale[1], 1.0f / wscale[2], 1.0f / wscale[3]};
    // B fragments: layer 1 (features | zero), layers 2/3: (tap 0 | tap 1), (tap 2 | tap 3), (tap 4 | zero);
    // layer 4: k = channel (| zero), n = tap
    uint32_t bq1[2][2], bq2[3][2][2], bq3[3][2][2], bq4[2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        load_b8([&](int k, int nn) -> uint8_t { return k < 16 ? wq[kOffW1 + k * kC + nt * 8 + nn] : 0; }, bq1[nt]);
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
            load_b8([&](int k, int nn) -> uint8_t {
                const int t = pr < 2 ? 2 * pr + (k >> 4) : (k < 16 ? 4 : -1), ci = chan_perm(k & 15);
                return t >= 0 ? wq[kOffW2 + t * 256 + ci * kC + nt * 8 + nn] : 0;
            }, bq2[pr][nt]);
            load_b8([&](int k, int nn) -> uint8_t {
                const int t = pr < 2 ? 2 * pr + (k >> 4) : (k < 16 ? 4 : -1), ci = chan_perm(k & 15);
                return t >= 0 ? wq[kOffW3 + t * 256 + ci * kC + nt * 8 + nn] : 0;
            }, bq3[pr][nt]);
        }
    }
    load_b8([&](int k, int nn) -> uint8_t {
        return (k < 16 && nn < 5) ? wq[kOffW4 + nn * kC + chan_perm(k)] : 0;
    }, bq4);
    float bias_s[3][2][2];                         // bias x s_l: the accumulators' start
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int co = nt * 8 + 2 * tq + e;
            bias_s[0][nt][e] = wf[kOffB1 + co] * s1;
            bias_s[1][nt][e] = wf[kOffB2 + co] * s2;
            bias_s[2][nt][e] = wf[kOffB3 + co] * s3;
        }
    const float b4 = wf[kOffB4];
    // this lane's four layer-1 features 4tq .. 4tq + 3: offsets into the window's
    // spin codes (ring codes kSpinRows further) and whether the feature is zero
    int foff[4];
    bool fzero[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = 4 * tq + e, kind = c_feat[k][2];
        foff[e] = kind == 2 ? 0 : (kind == 1 ? kSpinRows : 0) + c_feat[k][0] * kPW + c_feat[k][1];
        fzero[e] = kind == 2;
    }
    const int lr = lane & 15, lwc = min(lr / kPerStep, kWinT - 1);
    const int cw0 = g / kPerStep, cw1c = min((g + 8) / kPerStep, kWinT - 1);
    const uint32_t ring_l = (uint32_t)__cvta_generic_to_shared(wbase(lwc));
    const uint8_t* spin0 = wbase(cw0) + kSmpQSpin;
    const uint8_t* spin1 = wbase(cw1c) + kSmpQSpin;
    float* u0 = reinterpret_cast<float*>(wbase(cw0) + kSmpQU);
    float* u1 = reinterpret_cast<float*>(wbase(cw1c) + kSmpQU);
    unsigned char* wl = wbase(lwc);
    const float* ul = reinterpret_cast<const float*>(wl + kSmpQU);
    __syncthreads();

    constexpr uint32_t kL2 = kLayerRows * kRowQ;         // the layer-2 ring after the layer-1 ring
    for (int w0 = (blockIdx.x * kWarpsSmp + warp) * kWinT; w0 < n; w0 += gridDim.x * kWarpsSmp * kWinT) {
        for (int i = lane; i < kWinT * kSmpQWinBytes / 4; i += 32) reinterpret_cast<uint32_t*>(wb)[i] = 0u;
        __syncwarp();
        for (int i = lane; i < kWinT * kNPos; i += 32) {
            const int w = i / kNPos, p = i - w * kNPos;
            if (w0 + w < n && !interior(p / kS, p % kS)) {
                const int8_t x = win[(size_t)(w0 + w) * kNPos + p];
                (wbase(w) + kSmpQSpin)[kSpinRows + padded_row(p)] = x > 0 ? kE4m3Plus : (x < 0 ? kE4m3Minus : 0);
            }
        }
        for (int bq = lane; bq < kWinT * 16; bq += 32) {
            const int w = bq >> 4, q = bq & 15;
            if (w0 + w < n) {
                const LearnedKey k = keys[w0 + w];
                const uint4 rv = philox(16u * k.j + (uint32_t)q, round_t, k.sim, 4u, k.key0, k.key1);
                uint32_t* d = reinterpret_cast<uint32_t*>(wbase(w) + kSmpQDraws) + 4 * q;
                d[0] = rv.x; d[1] = rv.y; d[2] = rv.z; d[3] = rv.w;
            }
        }
        __syncwarp();
        float lq_acc = 0.0f;
#pragma unroll 1
        for (int s = 0; s < kSteps; ++s) {
            const uint2 dr = tabR[s * 16 + lr];
            const uint32_t dc = tabC[s * 8 + g];
            const uint32_t sl0 = dr.x & 0xFF, sl1 = (dr.x >> 8) & 0xFF, sl2 = (dr.x >> 16) & 0xFF, sl3 = dr.x >> 24;
            const uint32_t sl4 = dr.y & 0xFF, own = (dr.y >> 8) & 0xFF;
            // ---- ring taps of layers 2 and 3 (pairs (0 | 1), (2 | 3)) into accumulators at bias x s ----
            float d2[2][4], d3[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                d2[nt][0] = d2[nt][2] = bias_s[1][nt][0]; d2[nt][1] = d2[nt][3] = bias_s[1][nt][1];
                d3[nt][0] = d3[nt][2] = bias_s[2][nt][0]; d3[nt][1] = d3[nt][3] = bias_s[2][nt][1];
            }
            {
                const uint32_t pa = (lane < 16 ? sl0 : sl1) * kRowQ, pb = (lane < 16 ? sl2 : sl3) * kRowQ;
                uint32_t at[4];
                ldmatrix_x4(at, ring_l + pa);
                mma16832_e4m3(d2[0], at, bq2[0][0]); mma16832_e4m3(d2[1], at, bq2[0][1]);
                ldmatrix_x4(at, ring_l + pb);
                mma16832_e4m3(d2[0], at, bq2[1][0]); mma16832_e4m3(d2[1], at, bq2[1][1]);
                ldmatrix_x4(at, ring_l + kL2 + pa);
                mma16832_e4m3(d3[0], at, bq3[0][0]); mma16832_e4m3(d3[1], at, bq3[0][1]);
                ldmatrix_x4(at, ring_l + kL2 + pb);
                mma16832_e4m3(d3[0], at, bq3[1][0]); mma16832_e4m3(d3[1], at, bq3[1][1]);
            }
            // ---- layer 1: features 4tq .. 4tq + 3 of rows g, g + 8 ----
            const int q0 = dc & 0xFF, q1 = (dc >> 8) & 0xFF;
            uint32_t h[2];
            {
                uint32_t f0 = 0, f1 = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (fzero[e]) continue;
                    f0 |= (uint32_t)spin0[q0 + foff[e]] << (8 * e);
                    f1 |= (uint32_t)spin1[q1 + foff[e]] << (8 * e);
                }
                const uint32_t a[4] = {f0, f1, 0u, 0u};
                float d[2][4];
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    d[nt][0] = d[nt][2] = bias_s[0][nt][0]; d[nt][1] = d[nt][3] = bias_s[0][nt][1];
                    mma16832_e4m3(d[nt], a, bq1[nt]);
                }
                layer_out_e4m3(d, inv_s[0], h);
                stmatrix_x2(ring_l + own * kRowQ, h[0], h[1]);
            }
            // ---- layers 2 and 3: the (0, 0) taps ----
            {
                const uint32_t a[4] = {h[0], h[1], 0u, 0u};
                mma16832_e4m3(d2[0], a, bq2[2][0]); mma16832_e4m3(d2[1], a, bq2[2][1]);
            }
            layer_out_e4m3(d2, inv_s[1], h);
            stmatrix_x2(ring_l + kL2 + own * kRowQ, h[0], h[1]);
            {
                const uint32_t a[4] = {h[0], h[1], 0u, 0u};
                mma16832_e4m3(d3[0], a, bq3[2][0]); mma16832_e4m3(d3[1], a, bq3[2][1]);
            }
            layer_out_e4m3(d3, inv_s[2], h);
            // ---- layer 4: u[t] (unscaled) of rows g, g + 8 into the u ring ----
            {
                const uint32_t a[4] = {h[0], h[1], 0u, 0u};
                float d4[4] = {0.f, 0.f, 0.f, 0.f};
                mma16832_e4m3(d4, a, bq4);
                const int c0 = 2 * tq, o0 = (int)((dc >> 16) & 0xFF) * 5 + c0, o1 = (int)(dc >> 24) * 5 + c0;
                if (c0 < 5) { u0[o0] = d4[0]; u1[o1] = d4[2]; }
                if (c0 + 1 < 5) { u0[o0 + 1] = d4[1]; u1[o1 + 1] = d4[3]; }
            }
            __syncwarp();
            // ---- sample: lane lr < 15 takes its row's site when it has one ----
            const uint32_t di = (dr.y >> 16) & 0xFF;
            if (lane < 16 && di != 0xFFu) {
                const float z = (ul[sl0 * 5 + 0] + ul[sl1 * 5 + 1] + ul[sl2 * 5 + 2] + ul[sl3 * 5 + 3] + ul[sl4 * 5 + 4]) *
                                    inv_s[3] + b4;
                const uint32_t draw = reinterpret_cast<const uint32_t*>(wl + kSmpQDraws)[di];
                const float sg = __frcp_rn(1.0f + expf(-z));
                const uint32_t thr = (sg >= 1.0f) ? 0xFFFFFFFFu : (uint32_t)(sg * 4294967296.0f);
                const float x = draw < thr ? 1.0f : -1.0f;
                (wl + kSmpQSpin)[dr.y >> 24] = x > 0.f ? kE4m3Plus : kE4m3Minus;
                if (lq) lq_acc += log_sigmoid(x * z);
            }
            __syncwarp();
        }
        float* lqs = reinterpret_cast<float*>(wb + kSmpQU);
        if (lane < 16) lqs[lane] = lq_acc;
        __syncwarp();
        if (lane < kWinT && w0 + lane < n && lq) {
            float t = 0.0f;
            for (int k = 0; k < kPerStep; ++k) t += lqs[kPerStep * lane + k];
            lq[w0 + lane] = t;
        }
        for (int i = lane; i < kWinT * kNPos; i += 32) {
            const int w = i / kNPos, p = i - w * kNPos;
            if (w0 + w < n && interior(p / kS, p % kS))
                win[(size_t)(w0 + w) * kNPos + p] = (wbase(w) + kSmpQSpin)[padded_row(p)] == kE4m3Plus ? (int8_t)1 : (int8_t)-1;
        }
        __syncwarp();
    }
}

// fp8 weight copy: e4m3(W * s_layer) for the weights of each layer (biases
// stay fp32 and are read from the masters).
__global__ void to_fp8_kernel(const float* w, const float* wscale, uint8_t* wq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    const int layer = i < kOffW2 ? 0 : i < kOffW3 ? 1 : i < kOffW4 ? 2 : 3;
    wq[i] = __nv_cvt_float_to_fp8(w[i] * wscale[layer], __NV_SATFINITE, __NV_E4M3);
}

// ---------------------------------------------------------------------------
// Backward pass (FP32 CUDA cores), one warp per window: gradient of the mean
// negative log-likelihood through the bf16 weights; weight gradients summed
// per block in shared memory, then added to `grad`.
// ---------------------------------------------------------------------------
constexpr int kWarpsBwd = 4;

__global__ void __launch_bounds__(kWarpsBwd * 32) net_backward_kernel(NetPtrs net, const int8_t* win, int n,
                                                                      const float* z, const __nv_bfloat16* h,
                                                                      float* grad, float* loss, float inv_batch) {
    extern __shared__ __align__(16) float fsm[];
    float* gacc = fsm;                                          // [kNParams]
    float* wbuf = fsm + ((kNParams + 3) / 4) * 4;               // per warp: dA [100][16], dH [100][16]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) gacc[i] = 0.f;
    __syncthreads();
    float* dA = wbuf + warp * 2 * kNPos * kC;
    float* dH = dA + kNPos * kC;
    float loss_acc = 0.f;
    auto Wb = [&](int off) { return __bfloat162float(net.wb[off]); };

    for (int w = blockIdx.x * kWarpsBwd + warp; w < n; w += gridDim.x * kWarpsBwd) {
        const int8_t* x = win + (size_t)w * kNPos;
        const __nv_bfloat16* H1 = h + ((size_t)0 * n + w) * kNPos * kC;
        const __nv_bfloat16* H2 = h + ((size_t)1 * n + w) * kNPos * kC;
        const __nv_bfloat16* H3 = h + ((size_t)2 * n + w) * kNPos * kC;
        // dz (stored in dA[p][0])
        for (int p = lane; p < kNPos; p += 32) {
            const int r = p / kS, c = p % kS;
            float dz = 0.f;
            if (interior(r, c)) {
                const float zz = z[(size_t)w * kNPos + p], xv = (float)x[p];
                dz = (1.0f / (1.0f + expf(-zz)) - 0.5f * (xv + 1.0f)) * inv_batch;
                loss_acc -= log_sigmoid(xv * zz) * inv_batch;
            }
            dA[p * kC] = dz;
        }
        __syncwarp();
        // layer 4: dW4, db4, dH3
        for (int e = lane; e < 5 * kC; e += 32) {
            const int t = e / kC, ci = e % kC;
            float s = 0.f;
            for (int p = 0; p < kNPos; ++p) {
                const int r = p / kS, c = p % kS, yy = r + c_tapB[t][0], xx = c + c_tapB[t][1];
                if (!interior(r, c) || yy < 0 || xx < 0 || xx >= kS) continue;
                s += dA[p * kC] * __bfloat162float(H3[(yy * kS + xx) * kC + ci]);
            }
            atomicAdd(&gacc[kOffW4 + e], s);
        }
        if (lane == 0) {
            float s = 0.f;
            for (int p = 0; p < kNPos; ++p) s += dA[p * kC];
            atomicAdd(&gacc[kOffB4], s);
        }
        for (int e = lane; e < kNPos * kC; e += 32) {
            const int q = e / kC, ci = e % kC, qr = q / kS, qc = q % kS;
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const int pr = qr - c_tapB[t][0], pc = qc - c_tapB[t][1];
                if (pr < 0 || pr >= kS || pc < 0 || pc >= kS || !interior(pr, pc)) continue;
                s += Wb(kOffW4 + t * kC + ci) * dA[(pr * kS + pc) * kC];
            }
            dH[e] = (__bfloat162float(H3[e]) > 0.f) ? s : 0.f;   // dA3
        }
        __syncwarp();
        // layers 3 and 2: dW, db, dA of the layer below
        for (int layer = 3; layer >= 2; --layer) {
            const __nv_bfloat16* Hin = (layer == 3) ? H2 : H1;
            const int offW = (layer == 3) ? kOffW3 : kOffW2, offB = (layer == 3) ? kOffB3 : kOffB2;
            const float* dAl = dH;      // dA of this layer
            float* dAn = dA;            // dA of the layer below (overwrites the buffer)
            for (int e = lane; e < 5 * kC * kC; e += 32) {
                const int t = e / (kC * kC), ci = (e / kC) % kC, co = e % kC;
                float s = 0.f;
                for (int p = 0; p < kNPos; ++p) {
                    const int r = p / kS, c = p % kS, yy = r + c_tapB[t][0], xx = c + c_tapB[t][1];
                    if (yy < 0 || xx < 0 || xx >= kS) continue;
                    s += dAl[p * kC + co] * __bfloat162float(Hin[(yy * kS + xx) * kC + ci]);
                }
                atomicAdd(&gacc[offW + e], s);
            }
            if (lane < kC) {
                float s = 0.f;
                for (int p = 0; p < kNPos; ++p) s += dAl[p * kC + lane];
                atomicAdd(&gacc[offB + lane], s);
            }
            __syncwarp();
            for (int e = lane; e < kNPos * kC; e += 32) {
                const int q = e / kC, ci = e % kC, qr = q / kS, qc = q % kS;
                float s = 0.f;
                for (int t = 0; t < 5; ++t) {
                    const int pr = qr - c_tapB[t][0], pc = qc - c_tapB[t][1];
                    if (pr < 0 || pr >= kS || pc < 0 || pc >= kS) continue;
                    const float* dap = dAl + (pr * kS + pc) * kC;
                    const int wo = offW + t * kC * kC + ci * kC;
#pragma unroll 4
                    for (int co = 0; co < kC; ++co) s += Wb(wo + co) * dap[co];
                }
                dAn[e] = (__bfloat162float(Hin[e]) > 0.f) ? s : 0.f;
            }
            __syncwarp();
            // move dA of the layer below into dH for the next iteration
            for (int e = lane; e < kNPos * kC; e += 32) dH[e] = dAn[e];
            __syncwarp();
        }
        // layer 1: dW1, db1 from the features
        for (int e = lane; e < 13 * kC; e += 32) {
            const int k = e / kC, co = e % kC;
            const int kind = c_feat[k][2];
            float s = 0.f;
            for (int p = 0; p < kNPos; ++p) {
                const int r = p / kS, c = p % kS, yy = r + c_feat[k][0], xx = c + c_feat[k][1];
                if (yy < 0 || yy >= kS || xx < 0 || xx >= kS) continue;
                if ((kind == 0) != interior(yy, xx)) continue;
                s += dH[p * kC + co] * (float)x[yy * kS + xx];
            }
            atomicAdd(&gacc[kOffW1 + e], s);
        }
        if (lane < kC) {
            float s = 0.f;
            for (int p = 0; p < kNPos; ++p) s += dH[p * kC + lane];
            atomicAdd(&gacc[kOffB1 + lane], s);
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_down_sync(0xffffffffu, loss_acc, o);
    if (lane == 0) atomicAdd(loss, loss_acc);
    __syncthreads();
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x)
        if (gacc[i] != 0.f) atomicAdd(&grad[i], gacc[i]);
}

// Adam (Kingma & Ba 2015) on the fp32 masters, then refresh the bf16 copy.
__global__ void adam_kernel(float* w, float* m, float* v, const float* g, __nv_bfloat16* wb, float lr,
                            float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
}

__global__ void to_bf16_kernel(const float* w, __nv_bfloat16* wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParams) wb[i] = __float2bfloat16_rn(w[i]);
}

// spin at (x, y) of a packed lattice (layout of include/ising.h)
__device__ __forceinline__ int8_t packed_spin(const uint32_t* base, uint32_t L, uint32_t x, uint32_t y) {
    const uint32_t wn = L >> 6, c = (x + y) & 1u, j = x >> 1;
    const uint32_t w = base[((size_t)c * L + y) * wn + (j >> 5)];
    return ((w >> (j & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
}

// Training windows: window b's snapshot, and the (x, y) of its top-left
// interior site, from Philox (counter (b, step, 0, 6), key = seed).
__global__ void train_windows_kernel(const uint32_t* pool, int n_snap, uint32_t L, int nwin, uint32_t seed_lo,
                                     uint32_t seed_hi, uint32_t step, int8_t* win) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nwin * kNPos; i += gridDim.x * blockDim.x) {
        const int b = i / kNPos, p = i % kNPos;
        const uint4 r = philox((uint32_t)b, step, 0u, 6u, seed_lo, seed_hi);
        const uint32_t snap = r.x % (uint32_t)n_snap, x0 = r.y % L, y0 = r.z % L;
        const uint32_t* base = pool + (size_t)snap * ((size_t)L * L / 32);
        const uint32_t y = (y0 + L - 1 + p / kS) % L, x = (x0 + L - 1 + p % kS) % L;
        win[i] = packed_spin(base, L, x, y);
    }
}

// Patch windows of every lattice of a handle for one round, and their keys.
// The lattice of patch w (the same w in every lane): the last entry with
// patch_begin <= w (entry 0 begins at 0), by a 32-way search -- each round
// the lanes probe 32 evenly spaced entries of the remaining range and a ballot
// keeps the last one at or below w (one round up to 32 lattices, two up to 1024).
__device__ __forceinline__ int patch_lattice_warp(const LearnedLat* ll, int n_lat, int w, int lane) {
    int lo = 0, span = n_lat;
    while (span > 1) {
        const int step = (span + 31) / 32, idx = lo + lane * step;
        const bool le = lane * step < span && (int)ll[idx].patch_begin <= w;
        const int k = 31 - __clz(__ballot_sync(0xffffffffu, le));
        lo += k * step;
        span = min(step, span - k * step);
    }
    return lo;
}

// One warp per patch: its window (the 8 x 8 patch with the ring around it)
// into win and win2, and its key.
__global__ void gather_patches_kernel(DevState st, const LearnedLat* ll, int n_lat, int nwin, uint32_t ox,
                                      uint32_t oy, int8_t* win, int8_t* win2, LearnedKey* keys) {
    const int lane = threadIdx.x & 31;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwin; w += (gridDim.x * blockDim.x) >> 5) {
        const LearnedLat d = ll[patch_lattice_warp(ll, n_lat, w, lane)];
        const uint32_t L = d.L, per_row = L / 16, j = (uint32_t)w - d.patch_begin;
        const uint32_t xs = (16u * (j % per_row) + ox + L - 1) % L, ys = (16u * (j / per_row) + oy + L - 1) % L;
        const uint32_t* base = st.spins + d.word_off;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = lane + 32 * i;
            if (p < kNPos) {
                uint32_t x = xs + (uint32_t)(p % kS), y = ys + (uint32_t)(p / kS);
                if (x >= L) x -= L;
                if (y >= L) y -= L;
                const int8_t sv = packed_spin(base, L, x, y);
                win[(size_t)w * kNPos + p] = sv;
                win2[(size_t)w * kNPos + p] = sv;
            }
        }
        if (lane == 0) keys[w] = LearnedKey{d.key0, d.key1, d.sim, j};
    }
}

// Metropolis-Hastings acceptance (FP64) and write-back of accepted patches.
// A warp takes 32 consecutive patches: their old and new windows are staged
// in shared memory (3200 contiguous bytes each, 16-byte loads); lane k then
// computes patch k's change of the energy of the bonds touching the interior
// and of the interior magnetization (the 100-byte window stride is 25 words,
// so the lanes hit 32 distinct banks) and takes its FP64 decision (all lanes
// at once: the FP64 pipe is narrow); the accepted patches are written back
// one after another by the warp.
constexpr int kMhWarps = 4;
__global__ void __launch_bounds__(kMhWarps * 32) mh_apply_kernel(DevState st, const LearnedLat* ll, int n_lat,
                                                                int nwin, uint32_t ox, uint32_t oy,
                                                                const int8_t* win_old, const int8_t* win_new,
                                                                const float* lq_old, const float* lq_new,
                                                                uint32_t round_t, unsigned long long* accepted) {
    __shared__ __align__(16) int8_t sw[kMhWarps][2][32 * kNPos];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wbase = (blockIdx.x * kMhWarps + warp) * 32;
    if (wbase >= nwin) return;
    const int nw = min(32, nwin - wbase);
    int8_t* xo = sw[warp][0];
    int8_t* xn = sw[warp][1];
    const int8_t* go = win_old + (size_t)wbase * kNPos;
    const int8_t* gn = win_new + (size_t)wbase * kNPos;
    if (nw == 32) {                     // wbase * 100 is a multiple of 3200: 16-byte aligned
        for (int i = lane; i < 32 * kNPos / 16; i += 32) {
            reinterpret_cast<uint4*>(xo)[i] = reinterpret_cast<const uint4*>(go)[i];
            reinterpret_cast<uint4*>(xn)[i] = reinterpret_cast<const uint4*>(gn)[i];
        }
    } else {
        for (int i = lane; i < nw * kNPos; i += 32) { xo[i] = go[i]; xn[i] = gn[i]; }
    }
    __syncwarp();
    // the lattice of each lane's patch: from the first patch's, forward (32
    // consecutive patches span few lattices: a lattice has at least 16)
    int lat = patch_lattice_warp(ll, n_lat, wbase, lane);
    if (lane < nw)
        while (lat + 1 < n_lat && (int)ll[lat + 1].patch_begin <= wbase + lane) ++lat;
    int e = 0, m = 0;
    bool accept = false;
    if (lane < nw) {
        const int8_t* o = xo + lane * kNPos;
        const int8_t* q = xn + lane * kNPos;
        // bonds (r, c)-(r, c + 1), r in 1..8, c in 0..8, and (r, c)-(r + 1, c), c in 1..8, r in 0..8
        for (int r = 1; r <= kP; ++r)
            for (int c = 0; c < kS - 1; ++c) {
                const int p = r * kS + c;
                e -= q[p] * q[p + 1] - o[p] * o[p + 1];
                if (c >= 1) m += q[p] - o[p];
            }
        for (int c = 1; c <= kP; ++c)
            for (int r = 0; r < kS - 1; ++r) {
                const int p = r * kS + c;
                e -= q[p] * q[p + kS] - o[p] * o[p + kS];
            }
        const int w = wbase + lane;
        const LearnedLat d = ll[lat];
        const uint32_t j = (uint32_t)w - d.patch_begin;
        const double log_alpha = -(double)e * d.beta + (double)lq_old[w] - (double)lq_new[w];
        const uint4 r = philox(j, round_t, d.sim, 5u, d.key0, d.key1);
        const double u = ((double)((r.x >> 5) * 67108864ull + (r.y >> 6)) + 0.5) / 9007199254740992.0;
        accept = log(u) < log_alpha;
    }
    for (uint32_t bal = __ballot_sync(0xffffffffu, accept); bal; bal &= bal - 1) {
        const int k = __ffs(bal) - 1, wk = wbase + k;
        const int ek = __shfl_sync(0xffffffffu, e, k), mk = __shfl_sync(0xffffffffu, m, k);
        const LearnedLat d = ll[__shfl_sync(0xffffffffu, lat, k)];
        const uint32_t j = (uint32_t)wk - d.patch_begin;
        const int8_t* o = xo + k * kNPos;
        const int8_t* q = xn + k * kNPos;
        // lane 2 rr + c: the flipped sites of interior row rr in colour c, one xor
        // (x0 is a multiple of 8 -- patch origins 16a + {0, 8} -- and L of 64, so
        // the four sites of one colour in a row share one 32-bit word)
        const uint32_t L = d.L, wn = L >> 6, per_row = L / 16;
        const uint32_t x0 = (16u * (j % per_row) + ox) % L, y0 = (16u * (j / per_row) + oy) % L;
        if (lane < 2 * kP) {
            const int rr = lane >> 1;
            const uint32_t c = (uint32_t)(lane & 1), y = (y0 + rr) % L;
            uint32_t mask = 0u, widx = 0u;
            for (int cc = 0; cc < kP; ++cc) {
                const uint32_t x = (x0 + cc) % L;
                if (((x + y) & 1u) != c) continue;
                const uint32_t jj = x >> 1;
                widx = (c * L + y) * wn + (jj >> 5);
                if (o[(rr + 1) * kS + cc + 1] != q[(rr + 1) * kS + cc + 1]) mask |= 1u << (jj & 31);
            }
            if (mask) atomicXor(&st.spins[d.word_off + widx], mask);
        }
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&st.obs[2 * d.lat]), (unsigned long long)(long long)ek);
            atomicAdd(reinterpret_cast<unsigned long long*>(&st.obs[2 * d.lat + 1]),
                      (unsigned long long)(long long)mk);
            atomicAdd(&accepted[d.lat], 1ull);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launch wrappers (used by the C ABI below)
// ---------------------------------------------------------------------------
static int fwd_blocks(int n) { return (n + kWin * kWarpsFwd - 1) / (kWin * kWarpsFwd); }

cudaError_t configure_learned_kernels() {
    cudaError_t e = cudaFuncSetAttribute(ar_net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kWarpsFwd * kWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ar_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ar_sample_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmpQSmem);
    const int bwd = (((kNParams + 3) / 4) * 4 + kWarpsBwd * 2 * kNPos * kC) * (int)sizeof(float);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(net_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bwd);
    return e;
}

cudaError_t launch_net_forward(const NetState& ns, const int8_t* win, int n, float* lq, float* z, __nv_bfloat16* h,
                               cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    NetPtrs np{ns.wb, ns.w};
    ar_net_kernel<<<fwd_blocks(n), kWarpsFwd * 32, kWarpsFwd * kWarpSmem, stream>>>(np, win, n, lq, z, h);
    return cudaGetLastError();
}

cudaError_t launch_net_sample_fp8(const NetState& ns, int8_t* win, int n, float* lq, const LearnedKey* keys,
                                  uint32_t round_t, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int blocks = std::min((n + kWarpsSmp * kWinT - 1) / (kWarpsSmp * kWinT), device_sm_count() * 4);
    ar_sample_fp8_kernel<<<blocks, kWarpsSmp * 32, kSmpQSmem, stream>>>(ns.wq, ns.wscale, ns.w, win, n, lq, keys,
                                                                       round_t);
    return cudaGetLastError();
}

cudaError_t launch_to_fp8(const NetState& ns, cudaStream_t stream) {
    to_fp8_kernel<<<(kNParams + 255) / 256, 256, 0, stream>>>(ns.w, ns.wscale, ns.wq);
    return cudaGetLastError();
}

cudaError_t launch_net_sample(const NetState& ns, int8_t* win, int n, float* lq, const LearnedKey* keys,
                              uint32_t round_t, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    NetPtrs np{ns.wb, ns.w};
    const int blocks = std::min((n + kWarpsSmp * kWinT - 1) / (kWarpsSmp * kWinT), device_sm_count() * 4);
    ar_sample_kernel<<<blocks, kWarpsSmp * 32, kSmpSmem, stream>>>(np, win, n, lq, keys, round_t);
    return cudaGetLastError();
}

cudaError_t launch_net_backward(const NetState& ns, const int8_t* win, int n, const float* z,
                                const __nv_bfloat16* h, float* grad, float* loss, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    NetPtrs np{ns.wb, ns.w};
    const int bwd = (((kNParams + 3) / 4) * 4 + kWarpsBwd * 2 * kNPos * kC) * (int)sizeof(float);
    int blocks = (n + kWarpsBwd - 1) / kWarpsBwd;
    blocks = std::min(blocks, device_sm_count() * 2);
    net_backward_kernel<<<blocks, kWarpsBwd * 32, bwd, stream>>>(np, win, n, z, h, grad, loss, 1.0f / (float)n);
    return cudaGetLastError();
}

cudaError_t launch_adam(const NetState& ns, float lr, int step, cudaStream_t stream) {
    // bias corrections 1 - beta^step in double on the host: in fp32 from the
    // rounded betas, 1 - 0.999f loses about 1e-5 of its value to cancellation
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)step)), bc2 = (float)(1.0 - std::pow(0.999, (double)step));
    adam_kernel<<<(kNParams + 255) / 256, 256, 0, stream>>>(ns.w, ns.m, ns.v, ns.g, ns.wb, lr, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const NetState& ns, cudaStream_t stream) {
    to_bf16_kernel<<<(kNParams + 255) / 256, 256, 0, stream>>>(ns.w, ns.wb);
    return cudaGetLastError();
}

cudaError_t launch_train_windows(const uint32_t* pool, int n_snap, uint32_t L, int nwin, uint64_t seed,
                                 uint32_t step, int8_t* win, cudaStream_t stream) {
    const int blocks = std::min((nwin * kNPos + 255) / 256, device_sm_count() * 8);
    train_windows_kernel<<<blocks, 256, 0, stream>>>(pool, n_snap, L, nwin, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                    step, win);
    return cudaGetLastError();
}

cudaError_t launch_gather_patches(const DevState& st, const LearnedLat* ll, int n_lat, int nwin, uint32_t ox,
                                  uint32_t oy, int8_t* win, int8_t* win2, LearnedKey* keys, cudaStream_t stream) {
    if (nwin <= 0) return cudaSuccess;
    const int blocks = std::min((nwin + 7) / 8, device_sm_count() * 8);
    gather_patches_kernel<<<blocks, 256, 0, stream>>>(st, ll, n_lat, nwin, ox, oy, win, win2, keys);
    return cudaGetLastError();
}

cudaError_t launch_mh_apply(const DevState& st, const LearnedLat* ll, int n_lat, int nwin, uint32_t ox, uint32_t oy,
                            const int8_t* win_old, const int8_t* win_new, const float* lq_old, const float* lq_new,
                            uint32_t round_t, unsigned long long* accepted, cudaStream_t stream) {
    if (nwin <= 0) return cudaSuccess;
    mh_apply_kernel<<<(nwin + 32 * kMhWarps - 1) / (32 * kMhWarps), kMhWarps * 32, 0, stream>>>(
        st, ll, n_lat, nwin, ox, oy, win_old, win_new, lq_old, lq_new, round_t, accepted);
    return cudaGetLastError();
}

}  // namespace ising
