// Amplitudes with mass-dependent widths and Blatt-Weisskopf barrier factors: the constants of
// one decay channel X -> 1 + 2 (two spinless daughters, orbital angular momentum L = J of the
// wave) and the launcher.  The per-wave constants are formed on the host in double precision.
#pragma once

#include "pwa_internal.cuh"

namespace pwa {

constexpr int BARRIER_LMAX = 4;

struct BarrierTable {
    float msum_hi, msum_lo;  // m1 + m2 as a two-float sum
    float mdif_hi, mdif_lo;  // |m1 - m2| as a two-float sum
    float R, R2;             // R (GeV^-1) and R^2
    float num[PWA_MAX_WAVES];  // M Gamma_0 / B_J(q0 R)
    float cw[PWA_MAX_WAVES];   // M^2 Gamma_0 / (q0 B_J^2(q0 R)), so that M Gamma(m) = cw q B_J^2(q R) / m
};

// Squared barrier factor B_L^2(z), z = x^2, from the recurrence of the outgoing spherical Hankel
// functions: with g_L(x) = x^(L+1) h_L(x) exp(-ix), g_0 = -i, g_1 = -(x + i) and
// g_(l+1) = (2l + 1) g_l - x^2 g_(l-1), B_L^2 = x^(2L) / |g_L|^2 (normalised to 1 at large x).
__host__ __device__ inline double barrier2_host(int L, double z) {
    const double x = sqrt(z);
    double pr = 0.0, pi = -1.0;  // g_0
    if (L == 0) return 1.0;
    double cr = -x, ci = -1.0;   // g_1
    double zl = z;
    for (int l = 1; l < L; ++l) {
        const double nr = (2.0 * l + 1.0) * cr - z * pr, ni = (2.0 * l + 1.0) * ci - z * pi;
        pr = cr;
        pi = ci;
        cr = nr;
        ci = ni;
        zl *= z;
    }
    return zl / (cr * cr + ci * ci);
}

cudaError_t launch_amp_barrier(const WaveTable& wt, const BarrierTable& bt, const float* kin, int64_t n,
                               int64_t ld, float2* A, int sm_count, cudaStream_t st);

}  // namespace pwa
