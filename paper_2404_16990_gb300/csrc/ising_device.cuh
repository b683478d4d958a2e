// ising_device.cuh -- device helpers shared by the sweep kernels, the
// cluster kernels and the learned-proposal kernels: the Philox4x32-10
// counter-based generator and the per-sweep observable record.
#pragma once

#include <cstdint>

#include "ising_internal.h"

namespace ising {

constexpr uint32_t kMulA = 0xD2511F53u;   // Philox4x32 round multipliers
constexpr uint32_t kMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;  // Philox4x32 key increments
constexpr uint32_t kWeylB = 0xBB67AE85u;

// One Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// two 32x32->64 products of counter words 0 and 2 with the multipliers, the
// new counter being (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1,
// lo(A c0)), with the key advanced by the increments between rounds.  Counter
// words 1..3 and the key are usually the same for all sites of a thread, so the
// compiler hoists their products and the round keys out of per-site loops.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t ka = k0 + (uint32_t)r * kWeylA;
        const uint32_t kb = k1 + (uint32_t)r * kWeylB;
        // one 32x32->64 product each (a single wide multiply-add instruction)
        const uint64_t pa = (uint64_t)kMulA * c0, pb = (uint64_t)kMulB * c2;
        const uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
        const uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
        c0 = hi_b ^ c1 ^ ka;
        c1 = lo_b;
        c2 = hi_a ^ c3 ^ kb;
        c3 = lo_a;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Store E and M of lattice `lat` after sweep t: current values, the trace
// ring slot t % cap, and (if measuring) the FP64 moments of m = M/N, e = E/N.
__device__ __forceinline__ void record_em(const DevState& st, uint32_t lat, uint32_t L, long long E,
                                          long long M, unsigned long long t) {
    st.obs[2 * lat + 0] = E;
    st.obs[2 * lat + 1] = M;
    const long long cap = st.ctl->trace_cap;
    if (cap > 0) {
        const long long slot = (long long)(t % (unsigned long long)cap);
        st.trace[((long long)lat * cap + slot) * 2 + 0] = E;
        st.trace[((long long)lat * cap + slot) * 2 + 1] = M;
    }
    if (st.ctl->measure) {
        const double inv = 1.0 / ((double)L * (double)L);
        const double m = (double)M * inv, e = (double)E * inv;
        const double m2 = m * m;
        double* mo = st.mom + 6 * (size_t)lat;
        mo[0] += 1.0;
        mo[1] += fabs(m);
        mo[2] += m2;
        mo[3] += m2 * m2;
        mo[4] += e;
        mo[5] += e * e;
    }
}

}  // namespace ising
