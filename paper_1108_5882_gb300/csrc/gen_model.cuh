// Candidate generation shared by the toy generators: Philox4x32-10 (Salmon, Moraes, Dror,
// Shaw, SC'11) from its published definition, the flat phase-space point and accept uniform of
// candidate j, and the FP32 intensity I(Omega) = |sum_a V_a A_a(Omega)|^2 (Eq. 1).
#pragma once

#include "amp_model.cuh"

namespace pwa {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0];
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ float u01(uint32_t x) { return __fmul_rn((float)(x >> 8), 5.9604644775390625e-08f); }

struct Candidate {
    float m, ct, ph, u;
};

__device__ __forceinline__ Candidate candidate(uint64_t seed, uint32_t stream, int64_t j) {
    uint32_t c[4] = {(uint32_t)(uint64_t)j, (uint32_t)((uint64_t)j >> 32), stream, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    Candidate cd;
    cd.m = __fadd_rn(0.99f, __fmul_rn(2.01f, u01(c[0])));
    cd.ct = __fsub_rn(__fmul_rn(2.0f, u01(c[1])), 1.0f);
    cd.ph = __fmul_rn(6.2831855f, u01(c[2]));
    cd.u = u01(c[3]);
    return cd;
}

__device__ __forceinline__ float intensity(const WaveTable& wt, const float2* sV, const Candidate& cd) {
    EventAngles t;
    event_angles(cd.ct, cd.ph, t);
    float ur = 0.f, ui = 0.f;
    for (int a = 0; a < wt.K; ++a) {
        float dr;
        const float2 id = bw_inv_den(wt, a, cd.m, &dr);
        const float2 amp = cmul(make_float2(wt.MW[a] * id.x, wt.MW[a] * id.y), wave_angle(wt, a, t));
        const float2 p = cmul(sV[a], amp);
        ur += p.x;
        ui += p.y;
    }
    return ur * ur + ui * ui;
}

}  // namespace pwa
