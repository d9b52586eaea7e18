// Decay amplitudes A_a(Omega_i) = BW_a(m_i) * P_J(cos theta_i) * exp(i lambda phi_i).
//
// Paper: Sec. 2, Eq. 1 (A_a is the complex decay amplitude at phase-space point Omega) and
// Sec. 3 ("facilities for amplitude calculation").  The paper prints no amplitude formula;
// the model is the fixed-width relativistic Breit-Wigner with unit modulus at the peak,
// BW(m) = M G / (M^2 - m^2 - i M G), times the ordinary Legendre polynomial P_J and the
// phase factor exp(i lambda phi).  When masses and widths float (Sec. 2: then nothing can be
// precomputed) the kernel also writes
//   dBW/dM = -G (M^2 + m^2) / D^2,   dBW/dG = M (M^2 - m^2) / D^2,   D = M^2 - m^2 - i M G,
// each times the same angular factor.
//
// One thread per event, all K waves: the kinematics are read once (12 B/event) and every
// wave row is written with one coalesced 8-byte store per thread, so the kernel is bound by
// the HBM write stream of 8K (or 24K with derivatives) bytes per event.
//
// Precision: everything in FP32 (see amp_model.cuh for the two-float mass split).
#include "amp_model.cuh"

namespace pwa {

namespace {

template <bool DERIV>
__global__ void __launch_bounds__(PWA_THREADS) k_amplitudes(WaveTable wt, const float* __restrict__ kin,
                                                            int64_t n, int64_t ld, float2* __restrict__ A,
                                                            float2* __restrict__ dAdM, float2* __restrict__ dAdW) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += stride) {
        if (i >= n) {  // zero padding columns
            for (int a = 0; a < wt.K; ++a) {
                A[a * ld + i] = make_float2(0.f, 0.f);
                if (DERIV) {
                    dAdM[a * ld + i] = make_float2(0.f, 0.f);
                    dAdW[a * ld + i] = make_float2(0.f, 0.f);
                }
            }
            continue;
        }
        const float m = __ldg(kin + i);
        const float ct = __ldg(kin + ld + i);
        const float ph = __ldg(kin + 2 * ld + i);
        EventAngles t;
        event_angles(ct, ph, t);
        const float m2 = m * m;
        for (int a = 0; a < wt.K; ++a) {
            const float2 ang = wave_angle(wt, a, t);
            float dr;
            const float2 id = bw_inv_den(wt, a, m, &dr);  // 1/D
            const float MW = wt.MW[a];
            const float2 bw = make_float2(MW * id.x, MW * id.y);
            A[a * ld + i] = cmul(bw, ang);
            if (DERIV) {
                const float2 id2 = cmul(id, id);                    // 1/D^2
                const float cm = -wt.W[a] * (wt.Mhi[a] * wt.Mhi[a] + m2);  // -G (M^2 + m^2)
                const float cw = (wt.Mhi[a] + wt.Mlo[a]) * dr;      // M (M^2 - m^2)
                dAdM[a * ld + i] = cmul(make_float2(cm * id2.x, cm * id2.y), ang);
                dAdW[a * ld + i] = cmul(make_float2(cw * id2.x, cw * id2.y), ang);
            }
        }
    }
}

}  // namespace

cudaError_t launch_amplitudes(const WaveTable& wt, const float* kin, int64_t n, int64_t ld,
                              float2* A, float2* dAdM, float2* dAdW, int sm_count,
                              cudaStream_t st) {
    if (ld == 0) return cudaSuccess;
    int64_t blocks = (ld + PWA_THREADS - 1) / PWA_THREADS;
    int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (dAdM)
        k_amplitudes<true><<<(unsigned)blocks, PWA_THREADS, 0, st>>>(wt, kin, n, ld, A, dAdM, dAdW);
    else
        k_amplitudes<false><<<(unsigned)blocks, PWA_THREADS, 0, st>>>(wt, kin, n, ld, A, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace pwa
