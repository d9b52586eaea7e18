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

// I(Omega) = |sum_g Y_g(Omega) sum_{a in g} V_a BW_a(m)|^2: the waves of a group share the
// angular factor Y_g = P_J(cos theta) exp(i lambda phi), selected once per group; the
// Breit-Wigner denominator uses the fast reciprocal (relative error of a few ulp).
__device__ __forceinline__ float intensity(const WaveTable& wt, const float2* sV, const Candidate& cd) {
    EventAngles t;
    event_angles(cd.ct, cd.ph, t);
    float ur = 0.f, ui = 0.f;
    int s = 0;
    for (int g = 0; g < wt.ng; ++g) {
        const int end = wt.gend[g];
        float wr = 0.f, wi = 0.f;
        for (; s < end; ++s) {
            const int a = wt.gord[s];
            const float Mh = wt.Mhi[a], Ml = wt.Mlo[a], MW = wt.MW[a];
            const float dr = ((Mh - cd.m) + Ml) * ((Mh + cd.m) + Ml);  // M^2 - m^2
            const float inv = __fdividef(MW, dr * dr + MW * MW);        // MW / |D|^2
            const float br = dr * inv, bi = MW * inv;                   // BW = MW / D
            const float2 v = sV[a];
            cmac(wr, wi, v.x, v.y, br, bi);
        }
        const float2 y = wave_angle(wt, wt.gord[end - 1], t);
        cmac(ur, ui, y.x, y.y, wr, wi);
    }
    return fmaf(ur, ur, ui * ui);
}

}  // namespace pwa
