// ising_learned_tc.cu -- teacher-forced scoring of the learned proposal's
// windows on the fifth-generation tensor cores (tcgen05, accumulators in
// tensor memory), in BF16 or FP8 (E4M3).
//
// The net (include/ising.h, ising_net_*) is four masked 3x3 convolutions over
// a 10 x 10 window.  With the window known, every layer is an implicit GEMM:
// M = positions, K = (tap, input channel), N = 16 output channels (layer 4:
// N = the five taps, whose shifted sum is the logit).  The paper has no
// learned component; it motivates one by the critical slowing down of local
// moves near T_c (Section 1).
//
// Layout.  A CTA scores kTcWin windows at a time, one M = 128 tile per window.
// Row q of a window's tile is position (r, c) with q = 11 (r + 1) + c + 1
// (rows 12 .. 120; q % 11 == 0 and rows outside are zero padding), so tap
// (dy, dx) of row q is row q + 11 dy + dx and every input outside the window
// is a zero row.  Activations are stored K-major without swizzle, as planes of
// 16-byte rows (bf16: channels 0-7 and 8-15 in two planes; e4m3: the 16
// channels in one plane): eight consecutive rows are one core matrix, so the
// shared-memory descriptor of a tap is the plane address shifted by the tap's
// row offset -- the taps cost no copies.  In FP8 one K = 32 instruction takes
// two taps: its second K half is the same plane at another row offset (the
// descriptor's leading-dimension stride is the offset between the taps).
//
// Each layer: one thread issues the layer's MMAs for all windows of the chunk
// (per window BF16: 1 + 5 + 5 + 1, the layer-1 bias riding in W1's unused K
// rows against features that are 1.0 there; E4M3: 1 + 3 + 3 + 1) and commits
// them to an mbarrier; every thread then reads its row (32x32b tcgen05.ld:
// warp w reads lanes 32 (w % 4) ..), adds the bias, applies relu and rounds
// to the layer's activation type in one conversion (pad rows give zeros) and
// writes the row back over the layer's input (all MMAs that read it have
// completed).  With N = 16 an MMA does 16 FLOP per byte of A it reads from
// shared memory, so the MMAs per window, not the tensor pipe, set the pace.
// Same masks, weights, rounding points and fp32 accumulation as the other net
// kernels; only the order of the fp32 sums differs.
#include "../../include/ising.h"
#include "ising_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace ising {
namespace {

constexpr int kS = 10, kNPos = 100, kP = 8, kC = 16, kPW = 11;
constexpr int kOffW1 = 0, kOffB1 = 256, kOffW2 = 272, kOffB2 = 1552, kOffW3 = 1568, kOffB3 = 2848,
              kOffW4 = 2864, kOffB4 = 2944;
constexpr int kTcWarps = 4, kTcThreads = 32 * kTcWarps;   // warp w reads tensor-memory lanes 32 w ..
constexpr int kTcWin = 8;                        // windows (M tiles) per chunk
constexpr int kTcRows = 128;                     // tile rows per window
constexpr int kTcGuard = 16;                     // zero rows before the first window (taps reach 12 back)
constexpr int kTcPlaneRows = kTcGuard + kTcWin * kTcRows;
constexpr int kTcPlane = kTcPlaneRows * 16;      // bytes of one plane
constexpr int kTcCols = kTcWin * 16;             // tensor-memory columns: 16 fp32 per window
constexpr int kTcURows = kTcWin * 5 * kTcRows;   // layer-4 outputs u[window][tap][row] (fp32)
constexpr int kTcSpin = 136;                     // padded spin rows per window (taps reach row + 12)
constexpr int kTcCtasPerSm = 512 / kTcCols;      // tensor memory: 512 columns per SM
constexpr int kTcLdGroup = 4;                    // windows whose accumulators one tensor-memory load fetches
static_assert(kTcWin % kTcLdGroup == 0, "load groups");
constexpr unsigned long long kTcWaitNs = 1000ull * 1000ull * 1000ull;   // bound of an mbarrier wait: 1 s

__host__ __device__ constexpr int tc_tap(int t) { return t < 3 ? -kPW + t - 1 : (t == 3 ? -1 : 0); }

template <bool FP8>
struct TcLayout {
    static constexpr int kPlanes = FP8 ? 1 : 2;
    static constexpr int kAct = kPlanes * kTcPlane > kTcURows * 4 ? kPlanes * kTcPlane : kTcURows * 4;
    // B tiles of 512 bytes.  BF16: W1 (its rows k = 13, 14, 15 hold the layer-1
    // bias as three exact bf16 parts, met by features that are 1.0 there), the
    // five taps of W2 and of W3, W4; E4M3: see the weight set-up below.
    static constexpr int kNTiles = FP8 ? 8 : 12;
    static constexpr int kWts = kNTiles * 512;
    static constexpr int kOffWts = kAct;
    static constexpr int kOffBias = kOffWts + kWts;           // 3 x 16 fp32
    // spins as operand codes (bf16 bits / e4m3 bytes): [window][interior, ring][kTcSpin]
    using SpinT = typename std::conditional<FP8, uint8_t, uint16_t>::type;
    static constexpr int kOffSpin = kOffBias + 3 * 16 * 4;
    static constexpr int kOffBar = kOffSpin + ((kTcWin * 2 * kTcSpin * (int)sizeof(SpinT) + 15) / 16) * 16;
    static constexpr int kBytes = kOffBar + 16;
    static_assert(kOffWts % 128 == 0 && kOffSpin % 16 == 0 && kOffBar % 8 == 0, "alignment");
    static_assert(kBytes < (1 << 18), "descriptor address range");
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // K-major, no swizzle: start, leading (K) stride, stride (8-row) offset, all >> 4; version 1
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptors: fp32 accumulate, both operands K-major, M = 128, N = 16
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescE4m3 = (1u << 4) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

template <bool FP8>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    if constexpr (FP8) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(a), "l"(b), "r"(kIdescE4m3), "r"(accumulate));
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem), "l"(a), "l"(b), "r"(kIdescBf16), "r"(accumulate));
    }
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ unsigned long long tc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with the given parity; false if it did not
// complete within the bound.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    const unsigned long long t0 = tc_now();
    for (;;) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (tc_now() - t0 > kTcWaitNs) return false;
    }
}

// The accumulators of four consecutive windows (64 columns) of this warp's
// lanes in one 32x32b.x64 load, then one wait.
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float (&v)[4][16]) {
    uint32_t r[64];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int j = 0; j < 16; ++j) v[g][j] = __uint_as_float(r[16 * g + j]);
}

__device__ __forceinline__ uint32_t tc_pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ bool tc_pad_row(int q) { return q < kPW + 1 || q >= 121 || q % kPW == 0; }

__device__ __forceinline__ float tc_log_sigmoid(float t) { return -(fmaxf(-t, 0.0f) + log1pf(expf(-fabsf(t)))); }

// relu, then round to e4m3 (satfinite), a in the lowest byte: one conversion per pair
__device__ __forceinline__ uint32_t tc_pack_e4m3_relu(float a, float b, float c, float d) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// The 16 layer-1 features: k < 4 interior spins at the mask-A taps, 4 <= k < 13
// ring spins at the nine taps, then zeros.  feat_kind: 0 interior, 1 ring, 2 zero;
// feat_off: the row offset 11 dy + dx of the tap.
__host__ __device__ constexpr int feat_kind(int k) { return k < 4 ? 0 : (k < 13 ? 1 : 2); }
__host__ __device__ constexpr int feat_off(int k) {
    return k < 4 ? (k < 3 ? -kPW + k - 1 : -1) : (k < 13 ? kPW * ((k - 4) / 3 - 1) + (k - 4) % 3 - 1 : 0);
}

struct TcArgs {
    const __nv_bfloat16* wb;   // bf16 weights (flat parameter order)
    const uint8_t* wq;         // e4m3 weights times their layer scale
    const float* wscale;       // [4] layer scales of the e4m3 copy
    const float* wf;           // fp32 masters (biases)
    const int8_t* win_a;
    float* lq_a;
    float* z_a;
    const int8_t* win_b;
    float* lq_b;
    int n;
    int* err;                  // set nonzero if an mbarrier wait ran out
};

// Windows [0, n) from win_a (log q to lq_a, logits to z_a if given), [n, 2n)
// from win_b if given (log q to lq_b).
template <bool FP8>
__global__ void __launch_bounds__(kTcThreads, 4) ar_score_tc_kernel(const TcArgs args) {
    using Lay = TcLayout<FP8>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
    unsigned char* act = smem;
    float* bias = reinterpret_cast<float*>(smem + Lay::kOffBias);
    using SpinT = typename Lay::SpinT;
    SpinT* spin = reinterpret_cast<SpinT*>(smem + Lay::kOffSpin);
    constexpr uint32_t kPlus = FP8 ? 0x38u : 0x3F80u, kMinus = FP8 ? 0xB8u : 0xBF80u;   // +1, -1
    const uint32_t s_bar = s_base + Lay::kOffBar;

    // ---- one-time set-up: zero the activations (guard and pad rows stay zero),
    // the B tiles (weights, transposed to [n][k]), biases, mbarrier, tensor memory
    for (int i = tid; i < Lay::kAct / 16; i += kTcThreads) reinterpret_cast<uint4*>(act)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < (Lay::kOffBar - Lay::kOffSpin) / 4; i += kTcThreads) reinterpret_cast<uint32_t*>(spin)[i] = 0u;
    unsigned char* wts = smem + Lay::kOffWts;
    if constexpr (!FP8) {
        // tile = [2 chunks][16 n][8 k] bf16: element (n, k) at (k / 8) * 256 + n * 16 + (k % 8) * 2
        __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(wts);
        for (int i = tid; i < Lay::kNTiles * 256; i += kTcThreads) {
            const int tile = i >> 8, n = (i >> 4) & 15, k = i & 15;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (tile == 0) {
                if (k < 13) {
                    v = args.wb[kOffW1 + k * kC + n];
                } else {
                    // layer-1 bias as hi + mid + lo, each exact in bf16, summing to the fp32 bias
                    const float b = args.wf[kOffB1 + n];
                    const float h = __bfloat162float(__float2bfloat16_rn(b));
                    const float m = __bfloat162float(__float2bfloat16_rn(b - h));
                    v = __float2bfloat16_rn(k == 13 ? h : k == 14 ? m : (b - h) - m);
                }
            }
            else if (tile <= 5) v = args.wb[kOffW2 + (tile - 1) * 256 + k * kC + n];
            else if (tile <= 10) v = args.wb[kOffW3 + (tile - 6) * 256 + k * kC + n];
            else if (n < 5) v = args.wb[kOffW4 + n * kC + k];
            wt[tile * 256 + (k >> 3) * 128 + n * 8 + (k & 7)] = v;
        }
    } else {
        // tile = [2 chunks][16 n][16 k] e4m3: element (n, k) at (k / 16) * 256 + n * 16 + k % 16;
        // tiles: L1 (0 | W1), L2 (t0 | t1), (t2 | t3), (0 | t4), L3 the same, L4 (0 | W4)
        for (int i = tid; i < 8 * 512; i += kTcThreads) {
            const int tile = i >> 9, half = (i >> 8) & 1, n = (i >> 4) & 15, k = i & 15;
            uint8_t v = 0;
            if (tile == 0) v = half ? args.wq[kOffW1 + k * kC + n] : 0;
            else if (tile <= 6) {
                const int s = (tile - 1) % 3, base = tile <= 3 ? kOffW2 : kOffW3;
                const int t = s == 2 ? (half ? 4 : -1) : 2 * s + half;
                v = t >= 0 ? args.wq[base + t * 256 + k * kC + n] : 0;
            } else if (half && n < 5) v = args.wq[kOffW4 + n * kC + k];
            wts[i] = v;
        }
    }
    for (int i = tid; i < 48; i += kTcThreads)
        bias[i] = args.wf[(i < 16 ? kOffB1 : i < 32 ? kOffB2 : kOffB3) + (i & 15)];
    const float b4 = args.wf[kOffB4];
    // FP8: the products carry the layer's weight scale (a power of two)
    const float inv_s1 = FP8 ? 1.0f / args.wscale[0] : 1.0f, inv_s2 = FP8 ? 1.0f / args.wscale[1] : 1.0f;
    const float inv_s3 = FP8 ? 1.0f / args.wscale[2] : 1.0f, inv_s4 = FP8 ? 1.0f / args.wscale[3] : 1.0f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(s_bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    const int row = 32 * warp + lane;                   // this thread's tile row (tensor-memory lane)
    const bool pad = tc_pad_row(row);
    const uint32_t s_act = s_base;
    const uint32_t plane_bytes = kTcPlane;
    uint32_t parity = 0;
    bool failed = false;

    const int total = args.win_b ? 2 * args.n : args.n;
    const int chunks = (total + kTcWin - 1) / kTcWin;
    // spins of a chunk: 8 windows x 25 words, two per thread (4-byte loads;
    // windows are 100 bytes), fetched one chunk ahead
    constexpr int kSpinWords = (kTcWin * 25 + kTcThreads - 1) / kTcThreads;
    auto fetch = [&](int chunk, uint32_t (&v)[kSpinWords]) {
#pragma unroll
        for (int j = 0; j < kSpinWords; ++j) {
            const int i = tid + j * kTcThreads, m = i / 25, k = i - m * 25, w = chunk * kTcWin + m;
            v[j] = 0u;
            if (i < kTcWin * 25 && chunk < chunks && w < total) {
                const int8_t* src = w >= args.n ? args.win_b + (size_t)(w - args.n) * kNPos : args.win_a + (size_t)w * kNPos;
                v[j] = *reinterpret_cast<const uint32_t*>(src + 4 * k);
            }
        }
    };
    uint32_t next[kSpinWords];
    fetch(blockIdx.x, next);
    for (int chunk = blockIdx.x; chunk < chunks; chunk += gridDim.x) {
        const int w0 = chunk * kTcWin;
        uint32_t cur[kSpinWords];
#pragma unroll
        for (int j = 0; j < kSpinWords; ++j) cur[j] = next[j];
        fetch(chunk + (int)gridDim.x, next);
        // ---- the chunk's spins into the padded interior / ring arrays
#pragma unroll
        for (int j = 0; j < kSpinWords; ++j) {
            const int i = tid + j * kTcThreads, m = i / 25, k = i - m * 25;
            if (i >= kTcWin * 25) continue;
            const uint32_t v = cur[j];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int p = 4 * k + e, r = p / kS, c = p - r * kS, q = kPW * (r + 1) + c + 1;
                const int8_t x = (int8_t)(v >> (8 * e));
                const SpinT code = (SpinT)(x > 0 ? kPlus : (x < 0 ? kMinus : 0u));
                const bool in = r >= 1 && r <= kP && c >= 1 && c <= kP;
                spin[(m * 2 + 0) * kTcSpin + q] = in ? code : (SpinT)0;
                spin[(m * 2 + 1) * kTcSpin + q] = in ? (SpinT)0 : code;
            }
        }
        __syncthreads();
        // ---- layer-1 input: 16 features of the real rows of every window (pad rows stay zero)
        for (int i = tid; i < kTcWin * 112; i += kTcThreads) {
            const int m = i / 112, q = kPW + 1 + (i - m * 112);
            if (tc_pad_row(q)) continue;
            const SpinT* sp = spin + (m * 2) * kTcSpin + q;
            auto fv = [&](int k) -> uint32_t {          // operand code of feature k (compile-time k)
                // BF16: 1.0 at k >= 13, where W1 holds the bias; E4M3: zero there
                return feat_kind(k) == 2 ? (FP8 ? 0u : kPlus) : (uint32_t)sp[feat_kind(k) * kTcSpin + feat_off(k)];
            };
            const int r = kTcGuard + kTcRows * m + q;
            if constexpr (!FP8) {
                *reinterpret_cast<uint4*>(act + r * 16) =
                    make_uint4(fv(0) | fv(1) << 16, fv(2) | fv(3) << 16, fv(4) | fv(5) << 16, fv(6) | fv(7) << 16);
                *reinterpret_cast<uint4*>(act + plane_bytes + r * 16) =
                    make_uint4(fv(8) | fv(9) << 16, fv(10) | fv(11) << 16, fv(12) | fv(13) << 16, fv(14) | fv(15) << 16);
            } else {
                *reinterpret_cast<uint4*>(act + r * 16) =
                    make_uint4(fv(0) | fv(1) << 8 | fv(2) << 16 | fv(3) << 24, fv(4) | fv(5) << 8 | fv(6) << 16 | fv(7) << 24,
                               fv(8) | fv(9) << 8 | fv(10) << 16 | fv(11) << 24,
                               fv(12) | fv(13) << 8 | fv(14) << 16 | fv(15) << 24);
            }
        }
        // ---- layers 1 .. 4
        for (int layer = 0; layer < 4; ++layer) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors: a row shift of the A operand is an add of (16 * rows) >> 4 = rows to the start field
                const uint32_t wt = s_base + Lay::kOffWts;
                const uint64_t a0 = smem_desc(s_act + 16u * kTcGuard, FP8 ? 0u : plane_bytes, 128);
                auto bt = [&](int tile) { return smem_desc(wt + 512u * (uint32_t)tile, 256, 128); };
                for (int m = 0; m < kTcWin; ++m) {
                    const uint32_t d = tmem + 16u * (uint32_t)m;
                    const uint64_t am = a0 + (uint64_t)(kTcRows * m);
                    if constexpr (!FP8) {
                        if (layer == 0 || layer == 3) {
                            tc_mma<false>(d, am, bt(layer == 0 ? 0 : 11), 0u);
                        } else {
#pragma unroll
                            for (int t = 0; t < 5; ++t)
                                tc_mma<false>(d, am + (uint64_t)(int64_t)tc_tap(t), bt(layer == 1 ? 1 + t : 6 + t),
                                              t > 0 ? 1u : 0u);
                        }
                    } else {
                        // e4m3: K = 32 takes two row offsets of one plane; the leading stride is their distance
                        auto ap = [&](int r0, int r1) {
                            return (am + (uint64_t)(int64_t)r0) + ((uint64_t)(uint32_t)(r1 - r0) << 16);
                        };
                        if (layer == 0 || layer == 3) {
                            // (row - 1 | row): the first K half meets a zero B half
                            tc_mma<true>(d, ap(-1, 0), bt(layer == 0 ? 0 : 7), 0u);
                        } else {
                            const int tb = layer == 1 ? 1 : 4;
                            tc_mma<true>(d, ap(tc_tap(0), tc_tap(1)), bt(tb), 0u);
                            tc_mma<true>(d, ap(tc_tap(2), tc_tap(3)), bt(tb + 1), 1u);
                            tc_mma<true>(d, ap(tc_tap(3), tc_tap(4)), bt(tb + 2), 1u);
                        }
                    }
                }
                tc_commit(s_bar);
            }
            const bool ok = tc_wait(s_bar, parity);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) { failed = true; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // ---- epilogue: this thread's row of every window of the chunk, kTcLdGroup windows per wait
            const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
            // the layer's bias (BF16 layer 1: already in the accumulator) and FP8 scale
            float bl[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) bl[k] = (layer == 3 || (!FP8 && layer == 0)) ? 0.0f : bias[16 * layer + k];
            const float sc = layer == 0 ? inv_s1 : layer == 1 ? inv_s2 : inv_s3;
            for (int m = 0; m < kTcWin; m += kTcLdGroup) {
                float v[kTcLdGroup][16];
                tc_ld64(tl + 16u * (uint32_t)m, v);
#pragma unroll
                for (int h = 0; h < kTcLdGroup; ++h) {
                    const int r = kTcGuard + kTcRows * (m + h) + row;
                    if (layer < 3) {
                        if (pad) continue;       // pad rows are never written: they stay zero
                        float x[16];
                        if constexpr (!FP8) {
                            // bias add, then relu and bf16 rounding in one conversion
#pragma unroll
                            for (int k = 0; k < 16; ++k) x[k] = v[h][k] + bl[k];
                            *reinterpret_cast<uint4*>(act + r * 16) =
                                make_uint4(tc_pack_bf16_relu(x[0], x[1]), tc_pack_bf16_relu(x[2], x[3]),
                                           tc_pack_bf16_relu(x[4], x[5]), tc_pack_bf16_relu(x[6], x[7]));
                            *reinterpret_cast<uint4*>(act + plane_bytes + r * 16) =
                                make_uint4(tc_pack_bf16_relu(x[8], x[9]), tc_pack_bf16_relu(x[10], x[11]),
                                           tc_pack_bf16_relu(x[12], x[13]), tc_pack_bf16_relu(x[14], x[15]));
                        } else {
                            // scale and bias, then relu and e4m3 rounding in one conversion
#pragma unroll
                            for (int k = 0; k < 16; ++k) x[k] = v[h][k] * sc + bl[k];
                            *reinterpret_cast<uint4*>(act + r * 16) =
                                make_uint4(tc_pack_e4m3_relu(x[0], x[1], x[2], x[3]), tc_pack_e4m3_relu(x[4], x[5], x[6], x[7]),
                                           tc_pack_e4m3_relu(x[8], x[9], x[10], x[11]),
                                           tc_pack_e4m3_relu(x[12], x[13], x[14], x[15]));
                        }
                    } else {
                        // u[m][t][row] = H3[row] . W4[t] over the activations (no longer read)
                        float* u = reinterpret_cast<float*>(act);
#pragma unroll
                        for (int t = 0; t < 5; ++t) u[((m + h) * 5 + t) * kTcRows + row] = v[h][t];
                    }
                }
            }
        }
        if (failed) break;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // ---- logits and log q: warp w scores windows w0 + w and w0 + w + 4
        for (int m = warp; m < kTcWin; m += kTcWarps) {
            const int w = w0 + m;
            const float* u = reinterpret_cast<const float*>(act) + m * 5 * kTcRows;
            auto logit = [&](int q) -> float {
                float s = 0.0f;
#pragma unroll
                for (int t = 0; t < 5; ++t) s += u[t * kTcRows + q + tc_tap(t)];
                return s * inv_s4 + b4;
            };
            if (w < total) {
                const bool second = w >= args.n;
                const int wi = second ? w - args.n : w;
                float lq = 0.0f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = lane + 32 * h, q = kPW * (2 + j / kP) + 2 + j % kP;
                    const float x = spin[(m * 2) * kTcSpin + q] == (SpinT)kPlus ? 1.0f : -1.0f;
                    lq += tc_log_sigmoid(x * logit(q));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lq += __shfl_down_sync(0xffffffffu, lq, o);
                if (lane == 0) (second ? args.lq_b : args.lq_a)[wi] = lq;
                if (!second && args.z_a)
                    for (int p = lane; p < kNPos; p += 32)
                        args.z_a[(size_t)wi * kNPos + p] = logit(kPW * (p / kS + 1) + p % kS + 1);
            }
        }
        // the u rows overlay the activations: rows that must stay zero (guard
        // and pad rows) are cleared again before the next chunk
        __syncthreads();
        for (int i = tid; i < kTcURows / 4; i += kTcThreads) reinterpret_cast<uint4*>(act)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    if (failed && tid == 0) atomicExch(args.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

// Dynamic shared memory of a CTA: at least its layout, and enough that no
// more than kTcCtasPerSm CTAs fit on an SM (their tensor memory fills the
// SM's 512 columns; a further CTA would wait in tcgen05.alloc).
template <bool FP8>
int tc_smem_bytes() {
    using Lay = TcLayout<FP8>;
    int dev = 0, per_sm = 0, per_block = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // per CTA the SM also holds 1 KB of driver-reserved and 1 KB of static shared memory
    int bytes = per_sm / (kTcCtasPerSm + 1) + 1;
    bytes = std::max(bytes, Lay::kBytes);
    return std::min(bytes, per_block);
}

template <bool FP8>
cudaError_t launch_tc(const TcArgs& a, cudaStream_t stream) {
    static int smem = 0, grid_max = 0;
    if (smem == 0) {
        const int bytes = tc_smem_bytes<FP8>();
        cudaError_t e = cudaFuncSetAttribute(ar_score_tc_kernel<FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ar_score_tc_kernel<FP8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // the shared-memory size admits kTcCtasPerSm CTAs per SM; the grid is
        // persistent over chunks (the occupancy query reported one CTA per SM
        // for this kernel, while the SM holds four)
        grid_max = device_sm_count() * kTcCtasPerSm;
        smem = bytes;
    }
    const int total = a.win_b ? 2 * a.n : a.n;
    const int chunks = (total + kTcWin - 1) / kTcWin;
    ar_score_tc_kernel<FP8><<<std::min(chunks, grid_max), kTcThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_net_score_tc(const NetState& ns, bool fp8, const int8_t* win, int n, float* lq, float* z,
                                const int8_t* win_b, float* lq_b, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    TcArgs a{ns.wb, ns.wq, ns.wscale, ns.w, win, lq, z, win_b, lq_b, n, ns.err};
    return fp8 ? launch_tc<true>(a, stream) : launch_tc<false>(a, stream);
}

}  // namespace ising
