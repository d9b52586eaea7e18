// Decay amplitudes with a mass-dependent width and Blatt-Weisskopf barrier factors,
//   A_a(Omega) = BW_a(m) P_J(cos theta) exp(i lambda phi),
//   BW_a(m) = M Gamma_0 [B_J(q R) / B_J(q0 R)] / (M^2 - m^2 - i M Gamma(m)),
//   Gamma(m) = Gamma_0 (M / m) (q / q0) B_J^2(q R) / B_J^2(q0 R),
// for a resonance decaying into two spinless daughters (m1, m2) with orbital angular momentum
// L = J, breakup momentum q(m) (q0 = q(M)) and interaction radius R.  The paper gives no
// amplitude formula (Sec. 2, Eq. 1 only names A_a); this is the standard refinement of its
// fixed-width model, and keeps the unit modulus at the peak, BW(M) = i.
//
// Layout and threading as the fixed-width kernel: four consecutive events per thread, waves
// visited group by group in ascending J, so that the Legendre recurrence and the Hankel-function
// recurrence of the barrier factor each advance once per event from one group's J to the next;
// each wave then adds its own Breit-Wigner.  Every wave row is written with two 16-byte stores
// per thread: the kernel is bound by the HBM write stream of 8K bytes per event.
//
// Precision: FP32; the resonance mass and the daughter-mass sums enter as two-float values so
// that M - m and m - (m1 + m2) are exact to the rounding of m.  Divisions use __fdividef (within
// 2 ulp for denominators in the normal range, which m, |g_J|^2 >= 1 and the Breit-Wigner
// denominator are).
#include "amp_model.cuh"
#include "barrier.cuh"

namespace pwa {

namespace {

constexpr int BEV = 4;  // events per thread

__constant__ float c_b_inv_int[AMP_JMAX + 1] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};  // 1/(j+1)

__device__ __forceinline__ void store_ev(float2* row, int64_t i0, int64_t ld, bool full, const float2 (&v)[BEV]) {
    if (full) {
        reinterpret_cast<float4*>(row)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4*>(row)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    } else {
#pragma unroll
        for (int k = 0; k < BEV; ++k)
            if (i0 + k < ld) row[k] = v[k];
    }
}

__global__ void __launch_bounds__(PWA_THREADS) k_amp_barrier(WaveTable wt, BarrierTable bt, const float* __restrict__ kin,
                                                             int64_t n, int64_t ld, float2* __restrict__ A) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * BEV;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * BEV; i0 < ld; i0 += stride) {
        float m[BEV], ct[BEV], c1[BEV], s1[BEV], q[BEV], z[BEV], x[BEV], rm[BEV];
#pragma unroll
        for (int k = 0; k < BEV; ++k) {
            const int64_t i = i0 + k;
            const bool in = i < n;
            m[k] = in ? __ldg(kin + i) : 2.f;
            ct[k] = in ? __ldg(kin + ld + i) : 0.f;
            const float ph = in ? __ldg(kin + 2 * ld + i) : 0.f;
            sincosf(ph, &s1[k], &c1[k]);
            // q^2 = (m - (m1+m2)) (m + (m1+m2)) (m - |m1-m2|) (m + |m1-m2|) / (4 m^2), 0 below threshold
            const float a = (m[k] - bt.msum_hi) - bt.msum_lo, b = (m[k] + bt.msum_hi) + bt.msum_lo;
            const float c = (m[k] - bt.mdif_hi) - bt.mdif_lo, d = (m[k] + bt.mdif_hi) + bt.mdif_lo;
            rm[k] = __fdividef(1.f, m[k]);
            const float q2 = a > 0.f ? (a * b) * (c * d) * (0.25f * rm[k] * rm[k]) : 0.f;
            q[k] = sqrtf(q2);
            z[k] = q2 * bt.R2;
            x[k] = q[k] * bt.R;
        }
        const bool full = i0 + BEV <= ld;  // ld is even: pairs never straddle it
        float pcur[BEV], pprev[BEV];       // P_jc, P_(jc-1)
        float gcr[BEV], gci[BEV], gpr[BEV], gpi[BEV], zj[BEV];  // g_jc, g_(jc-1), z^jc
#pragma unroll
        for (int k = 0; k < BEV; ++k) {
            pcur[k] = 1.f;
            pprev[k] = 0.f;
            gcr[k] = 0.f;
            gci[k] = -1.f;
            gpr[k] = gpi[k] = 0.f;
            zj[k] = 1.f;
        }
        int jc = 0, s = 0;
        for (int g = 0; g < wt.ng; ++g) {
            const int end = wt.gend[g];
            const int a0 = wt.gord[s];
            const int J = wt.J[a0], lam = wt.lam[a0];
            const int al = lam < 0 ? -lam : lam;
            for (; jc < J; ++jc) {
                const float c2 = 2.f * jc + 1.f, cj = (float)jc, rj = c_b_inv_int[jc];
#pragma unroll
                for (int k = 0; k < BEV; ++k) {
                    const float pn = (c2 * ct[k] * pcur[k] - cj * pprev[k]) * rj;
                    pprev[k] = pcur[k];
                    pcur[k] = pn;
                    // Hankel recurrence: g_1 = -(x + i); g_(l+1) = (2l+1) g_l - z g_(l-1) for l >= 1
                    const float nr = jc == 0 ? -x[k] : fmaf(c2, gcr[k], -z[k] * gpr[k]);
                    const float ni = jc == 0 ? -1.f : fmaf(c2, gci[k], -z[k] * gpi[k]);
                    gpr[k] = gcr[k];
                    gpi[k] = gci[k];
                    gcr[k] = nr;
                    gci[k] = ni;
                    zj[k] *= z[k];
                }
            }
            float2 ang[BEV];  // P_J(cos theta) exp(i lambda phi)
            float b[BEV], t[BEV];  // B_J(q R) and q B_J^2(q R) / m
#pragma unroll
            for (int k = 0; k < BEV; ++k) {
                float er = 1.f, ei = 0.f;
                for (int j = 0; j < al; ++j) {
                    const float tr = er * c1[k] - ei * s1[k];
                    ei = er * s1[k] + ei * c1[k];
                    er = tr;
                }
                if (lam < 0) ei = -ei;
                ang[k] = make_float2(pcur[k] * er, pcur[k] * ei);
                const float b2 = __fdividef(zj[k], fmaf(gcr[k], gcr[k], gci[k] * gci[k]));  // |g_J|^2 >= 1
                b[k] = sqrtf(b2);
                t[k] = q[k] * b2 * rm[k];
            }
            for (; s < end; ++s) {
                const int a = wt.gord[s];
                const float Mh = wt.Mhi[a], Ml = wt.Mlo[a], nu = bt.num[a], cw = bt.cw[a];
                float2 out[BEV];
#pragma unroll
                for (int k = 0; k < BEV; ++k) {
                    // BW = nu b / (dr - i MG),  dr = M^2 - m^2 from the two-float mass, MG = cw t
                    const float dr = ((Mh - m[k]) + Ml) * ((Mh + m[k]) + Ml);
                    const float mg = cw * t[k];
                    const float sc = nu * b[k] * __fdividef(1.f, fmaf(dr, dr, mg * mg));  // <= 2 ulp
                    const float2 bw = make_float2(dr * sc, mg * sc);
                    out[k] = i0 + k < n ? cmul(bw, ang[k]) : make_float2(0.f, 0.f);
                }
                store_ev(A + a * ld + i0, i0, ld, full, out);
            }
        }
    }
}

}  // namespace

cudaError_t launch_amp_barrier(const WaveTable& wt, const BarrierTable& bt, const float* kin, int64_t n,
                               int64_t ld, float2* A, int sm_count, cudaStream_t st) {
    if (ld == 0) return cudaSuccess;
    int64_t blocks = (ld + PWA_THREADS * BEV - 1) / (PWA_THREADS * BEV);
    const int64_t cap = (int64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    k_amp_barrier<<<(unsigned)blocks, PWA_THREADS, 0, st>>>(wt, bt, kin, n, ld, A);
    return cudaGetLastError();
}

}  // namespace pwa
