// Per-event amplitude model shared by the amplitude kernel and the toy generator:
// A_a = BW_a(m) * P_J(cos theta) * exp(i lambda phi), BW(m) = M G / (M^2 - m^2 - i M G)
// (fixed width, unit modulus at the peak).  FP32 throughout; the mass enters as a two-float
// split (M_hi + M_lo) so that M - m keeps the resonance position exact to FP32 rounding of m.
#pragma once

#include "pwa_internal.cuh"

namespace pwa {

constexpr int AMP_JMAX = 8;

// Angular tables of one event: Legendre P_0..P_8(cos theta), and z^0..z^8, z = exp(i phi).
struct EventAngles {
    float P[AMP_JMAX + 1];
    float zr[AMP_JMAX + 1], zi[AMP_JMAX + 1];
};

__device__ __forceinline__ void event_angles(float ct, float ph, EventAngles& t) {
    t.P[0] = 1.f;
    t.P[1] = ct;
#pragma unroll
    for (int j = 1; j < AMP_JMAX; ++j)  // Bonnet: (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}
        t.P[j + 1] = ((2.f * j + 1.f) * ct * t.P[j] - (float)j * t.P[j - 1]) * (1.f / (float)(j + 1));
    float s1, c1;
    sincosf(ph, &s1, &c1);
    t.zr[0] = 1.f;
    t.zi[0] = 0.f;
#pragma unroll
    for (int k = 1; k <= AMP_JMAX; ++k) {
        t.zr[k] = t.zr[k - 1] * c1 - t.zi[k - 1] * s1;
        t.zi[k] = t.zr[k - 1] * s1 + t.zi[k - 1] * c1;
    }
}

// Angular factor P_J(cos theta) exp(i lambda phi) of wave a.  J and lambda are the same for
// every thread of the launch, so the branches below are uniform (no divergence).
__device__ __forceinline__ float2 wave_angle(const WaveTable& wt, int a, const EventAngles& t) {
    const int J = wt.J[a];
    const int lam = wt.lam[a];
    const int al = lam < 0 ? -lam : lam;
    float pj = t.P[0];
#pragma unroll
    for (int j = 1; j <= AMP_JMAX; ++j)
        if (J == j) pj = t.P[j];
    float er = t.zr[0], ei = t.zi[0];
#pragma unroll
    for (int j = 1; j <= AMP_JMAX; ++j)
        if (al == j) {
            er = t.zr[j];
            ei = t.zi[j];
        }
    if (lam < 0) ei = -ei;
    return make_float2(pj * er, pj * ei);
}

// 1/D for D = M^2 - m^2 - i M G (returned as (Re, Im)), plus M^2 - m^2.
__device__ __forceinline__ float2 bw_inv_den(const WaveTable& wt, int a, float m, float* dr_out) {
    const float Mh = wt.Mhi[a], Ml = wt.Mlo[a], MW = wt.MW[a];
    const float dm = (Mh - m) + Ml;  // M - m
    const float sm = (Mh + m) + Ml;  // M + m
    const float dr = dm * sm;        // M^2 - m^2
    const float inv = __frcp_rn(dr * dr + MW * MW);
    *dr_out = dr;
    return make_float2(dr * inv, MW * inv);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

}  // namespace pwa
