// Decay amplitudes A_a(Omega_i) = BW_a(m_i) * P_J(cos theta_i) * exp(i lambda phi_i).
//
// Paper: Sec. 2, Eq. 1 (A_a: wave a's complex amplitude at the phase-space point Omega) and
// Sec. 3 ("facilities for amplitude calculation").  The paper prints no amplitude formula;
// the model is the fixed-width relativistic Breit-Wigner with unit modulus at the peak,
// BW(m) = M G / (M^2 - m^2 - i M G), times the ordinary Legendre polynomial P_J and the
// phase factor exp(i lambda phi).  When masses and widths float (Sec. 2: then nothing can be
// precomputed) the kernel also writes
//   dBW/dM = -G (M^2 + m^2) / D^2,   dBW/dG = M (M^2 - m^2) / D^2,   D = M^2 - m^2 - i M G,
// each times the same angular factor.
//
// Each thread takes four consecutive events and loops over the K waves: the kinematics are
// read once (12 B/event), the per-wave parameters are uniform across the launch, and every
// wave row is written with two coalesced 16-byte stores per thread, so the kernel is bound by
// the HBM write stream of 8K (or 24K with derivatives) bytes per event.
//
// Precision: everything in FP32 (see amp_model.cuh for the two-float mass split).
#include "amp_model.cuh"

namespace pwa {

namespace {

constexpr int AMP_EV = 4;  // events per thread (consecutive: two 16-byte stores per wave)

__constant__ float c_inv_int[AMP_JMAX + 1] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};

__device__ __forceinline__ void store4(float2* row, int64_t i0, int64_t ld, bool full, const float2 (&v)[AMP_EV]) {
    if (full) {
        reinterpret_cast<float4*>(row)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4*>(row)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else {
#pragma unroll
        for (int k = 0; k < AMP_EV; ++k)
            if (i0 + k < ld) row[k] = v[k];
    }
}

// Waves are visited group by group (groups of equal (J, lambda) in ascending J, see WaveTable):
// the Legendre recurrence (Bonnet, (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}) advances from one
// group's J to the next, exp(i lambda phi) is formed once per group, and each wave of the group
// only adds its Breit-Wigner factor.
template <bool DERIV>
__global__ void __launch_bounds__(PWA_THREADS) k_amplitudes(WaveTable wt, const float* __restrict__ kin,
                                                            int64_t n, int64_t ld, float2* __restrict__ A,
                                                            float2* __restrict__ dAdM, float2* __restrict__ dAdW) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * AMP_EV;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * AMP_EV; i0 < ld; i0 += stride) {
        float m[AMP_EV], ct[AMP_EV], c1[AMP_EV], s1[AMP_EV];
#pragma unroll
        for (int k = 0; k < AMP_EV; ++k) {
            const int64_t i = i0 + k;
            const bool in = i < n;
            m[k] = in ? __ldg(kin + i) : 2.f;
            ct[k] = in ? __ldg(kin + ld + i) : 0.f;
            const float ph = in ? __ldg(kin + 2 * ld + i) : 0.f;
            sincosf(ph, &s1[k], &c1[k]);
        }
        const bool full = i0 + AMP_EV <= ld;  // ld is even: pairs never straddle it
        float pcur[AMP_EV], pprev[AMP_EV];     // P_jc, P_{jc-1}
#pragma unroll
        for (int k = 0; k < AMP_EV; ++k) {
            pcur[k] = 1.f;
            pprev[k] = 0.f;
        }
        int jc = 0, s = 0;
        for (int g = 0; g < wt.ng; ++g) {
            const int end = wt.gend[g];
            const int a0 = wt.gord[s];
            const int J = wt.J[a0], lam = wt.lam[a0];
            const int al = lam < 0 ? -lam : lam;
            for (; jc < J; ++jc) {
                const float c2 = 2.f * jc + 1.f, cj = (float)jc, rj = c_inv_int[jc];
#pragma unroll
                for (int k = 0; k < AMP_EV; ++k) {
                    const float pn = (c2 * ct[k] * pcur[k] - cj * pprev[k]) * rj;
                    pprev[k] = pcur[k];
                    pcur[k] = pn;
                }
            }
            float2 ang[AMP_EV];  // P_J(cos theta) exp(i lambda phi)
#pragma unroll
            for (int k = 0; k < AMP_EV; ++k) {
                float er = 1.f, ei = 0.f;
                for (int j = 0; j < al; ++j) {
                    const float tr = er * c1[k] - ei * s1[k];
                    ei = er * s1[k] + ei * c1[k];
                    er = tr;
                }
                if (lam < 0) ei = -ei;
                ang[k] = make_float2(pcur[k] * er, pcur[k] * ei);
            }
            for (; s < end; ++s) {
                const int a = wt.gord[s];
                const float Mh = wt.Mhi[a], Ml = wt.Mlo[a], MW = wt.MW[a], G = wt.W[a];
                float2 out[AMP_EV], oM[AMP_EV], oW[AMP_EV];
#pragma unroll
                for (int k = 0; k < AMP_EV; ++k) {
                    // 1/D, D = M^2 - m^2 - i M G, with M - m from the two-float mass
                    const float dr = ((Mh - m[k]) + Ml) * ((Mh + m[k]) + Ml);
                    const float inv = __fdividef(1.f, fmaf(dr, dr, MW * MW));
                    const float2 id = make_float2(dr * inv, MW * inv);
                    const bool in = i0 + k < n;
                    const float2 bw = make_float2(MW * id.x, MW * id.y);
                    out[k] = in ? cmul(bw, ang[k]) : make_float2(0.f, 0.f);
                    if (DERIV) {
                        const float2 id2 = cmul(id, id);                // 1/D^2
                        const float cm = -G * (Mh * Mh + m[k] * m[k]);  // -G (M^2 + m^2)
                        const float cw = (Mh + Ml) * dr;                // M (M^2 - m^2)
                        oM[k] = in ? cmul(make_float2(cm * id2.x, cm * id2.y), ang[k]) : make_float2(0.f, 0.f);
                        oW[k] = in ? cmul(make_float2(cw * id2.x, cw * id2.y), ang[k]) : make_float2(0.f, 0.f);
                    }
                }
                store4(A + a * ld + i0, i0, ld, full, out);
                if (DERIV) {
                    store4(dAdM + a * ld + i0, i0, ld, full, oM);
                    store4(dAdW + a * ld + i0, i0, ld, full, oW);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_amplitudes(const WaveTable& wt, const float* kin, int64_t n, int64_t ld,
                              float2* A, float2* dAdM, float2* dAdW, int sm_count,
                              cudaStream_t st) {
    if (ld == 0) return cudaSuccess;
    int64_t blocks = (ld + PWA_THREADS * AMP_EV - 1) / (PWA_THREADS * AMP_EV);
    int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (dAdM)
        k_amplitudes<true><<<(unsigned)blocks, PWA_THREADS, 0, st>>>(wt, kin, n, ld, A, dAdM, dAdW);
    else
        k_amplitudes<false><<<(unsigned)blocks, PWA_THREADS, 0, st>>>(wt, kin, n, ld, A, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace pwa
