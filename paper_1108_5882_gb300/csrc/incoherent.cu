// -lnL and its gradient with the intensity summed incoherently over H unobserved states (the
// photon helicity of J/psi -> gamma X, the paper's example channel): Eq. 1 summed over h,
//   I_i = sum_h |u_ih|^2,  u_ih = sum_a V_a A_{a,h}(i),
//   f = -sum_i ln I_i + n_f sum_ab V_a conj(V_b) Psi_ab   (Psi summed over h),
//   g_c = -2 sum_i sum_h conj(A_{c,h}(i)) u_ih / I_i + 2 n_f sum_a Psi_ac V_a.
// One parameter set per launch: the single-set streaming kernel with an h loop, one thread per
// event, or per pair of events with 16-byte loads for K <= 16 (a warp reads 256 or 512
// contiguous bytes per (wave, state) row); the gradient pass reloads the event's amplitudes (L1
// hits), and the same exact fixed-point grid reduction and last-block finalisation
// (normalisation term included) as the coherent single-set kernel.  P sets are P
// launches in stream order (each launch's last block clears the control words).
#include "nll_common.cuh"

namespace pwa {

namespace {

template <int KMAX, bool GRAD>
__global__ void __launch_bounds__(PWA_THREADS, KMAX <= 16 ? 2 : 1) k_nll_incoherent(
    const float2* __restrict__ A, int K, int H, int64_t n, int64_t ld, const float2* __restrict__ V,
    const double2* __restrict__ Psi, double nfac, float2* __restrict__ part, unsigned* __restrict__ counter,
    int* __restrict__ badw, int* __restrict__ status, double* __restrict__ nll, double* __restrict__ grad) {
    constexpr int NG = 2 * KMAX;
    constexpr bool EV2 = KMAX <= 16;  // two events per thread and iteration (16-byte loads)
    __shared__ float2 sV[KMAX];
    __shared__ StreamReduceSmem<KMAX, PWA_THREADS> red;
    const int tid = threadIdx.x;
    if (tid < KMAX) sV[tid] = tid < K ? V[tid] : make_float2(0.f, 0.f);
    stream_reduce_init<KMAX, PWA_THREADS>(red, Psi, K);
    __syncthreads();

    float g[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) g[v] = 0.f;
    ff lacc = ff_zero();
    bool bad = false;
    const int64_t hld = (int64_t)H * ld;  // between waves; states of a wave are ld apart
    const int64_t stride = (int64_t)gridDim.x * PWA_THREADS;
    if (EV2) {
        // two events per thread: 16-byte loads of (event 2q, event 2q + 1) per (wave, state)
        const float4* A4 = reinterpret_cast<const float4*>(A);
        const int64_t hld2 = hld >> 1, ld2 = ld >> 1;
        const int64_t npairs = (n + 1) >> 1;
        for (int64_t q = (int64_t)blockIdx.x * PWA_THREADS + tid; q < npairs; q += stride) {
            const bool has1 = 2 * q + 1 < n;
            float u[PWA_MAX_STATES][4];
            float I0 = 0.f, I1 = 0.f;
#pragma unroll
            for (int h = 0; h < PWA_MAX_STATES; ++h) {
                u[h][0] = u[h][1] = u[h][2] = u[h][3] = 0.f;
                if (h < H) {
#pragma unroll
                    for (int c = 0; c < KMAX; ++c) {
                        float4 x = (c < K) ? __ldg(A4 + c * hld2 + h * ld2 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (!has1) x.z = x.w = 0.f;  // odd n: the pair's second slot is padding
                        const float2 v = sV[c];
                        cmac(u[h][0], u[h][1], v.x, v.y, x.x, x.y);
                        cmac(u[h][2], u[h][3], v.x, v.y, x.z, x.w);
                    }
                    I0 = fmaf(u[h][0], u[h][0], fmaf(u[h][1], u[h][1], I0));
                    I1 = fmaf(u[h][2], u[h][2], fmaf(u[h][3], u[h][3], I1));
                }
            }
            float r0 = 0.f, r1 = 0.f;
            if (intensity_ok(I0)) {
                lacc = ff_add_f(lacc, __logf(I0));
                r0 = __frcp_rn(I0);
            } else {
                bad = true;
            }
            if (has1) {
                if (intensity_ok(I1)) {
                    lacc = ff_add_f(lacc, __logf(I1));
                    r1 = __frcp_rn(I1);
                } else {
                    bad = true;
                }
            }
            if (GRAD) {
#pragma unroll
                for (int h = 0; h < PWA_MAX_STATES; ++h) {
                    if (h < H) {
                        const float w0r = u[h][0] * r0, w0i = u[h][1] * r0, w1r = u[h][2] * r1, w1i = u[h][3] * r1;
#pragma unroll
                        for (int c = 0; c < KMAX; ++c) {
                            float4 x = (c < K) ? __ldg(A4 + c * hld2 + h * ld2 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                            if (!has1) x.z = x.w = 0.f;
                            cmac_conj(g[2 * c], g[2 * c + 1], x.x, x.y, w0r, w0i);
                            cmac_conj(g[2 * c], g[2 * c + 1], x.z, x.w, w1r, w1i);
                        }
                    }
                }
            }
        }
    } else
    for (int64_t i = (int64_t)blockIdx.x * PWA_THREADS + tid; i < n; i += stride) {
        float ur[PWA_MAX_STATES], ui[PWA_MAX_STATES];
        float I = 0.f;
#pragma unroll
        for (int h = 0; h < PWA_MAX_STATES; ++h) {
            ur[h] = ui[h] = 0.f;
            if (h < H) {
#pragma unroll
                for (int c = 0; c < KMAX; ++c) {
                    const float2 x = (c < K) ? __ldg(A + c * hld + h * ld + i) : make_float2(0.f, 0.f);
                    const float2 v = sV[c];
                    cmac(ur[h], ui[h], v.x, v.y, x.x, x.y);
                }
                I = fmaf(ur[h], ur[h], fmaf(ui[h], ui[h], I));
            }
        }
        float r = 0.f;
        if (intensity_ok(I)) {
            lacc = ff_add_f(lacc, __logf(I));
            r = __frcp_rn(I);
        } else {
            bad = true;
        }
        if (GRAD) {
#pragma unroll
            for (int h = 0; h < PWA_MAX_STATES; ++h) {
                if (h < H) {
                    const float wr = ur[h] * r, wi = ui[h] * r;
#pragma unroll
                    for (int c = 0; c < KMAX; ++c) {
                        const float2 x = (c < K) ? __ldg(A + c * hld + h * ld + i) : make_float2(0.f, 0.f);
                        cmac_conj(g[2 * c], g[2 * c + 1], x.x, x.y, wr, wi);
                    }
                }
            }
        }
    }
    stream_reduce_finalize<KMAX, GRAD, true, PWA_THREADS>(g, lacc, bad, sV, red, K, Psi, nfac, part, counter, badw,
                                                          status, nll, grad);
}

template <int KMAX, bool GRAD>
cudaError_t inc_launch(const float2* A, int K, int H, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                       double nfac, double* nll, double* grad, void* ws, unsigned* counter, int* status, int sm_count,
                       cudaStream_t st) {
    auto kern = k_nll_incoherent<KMAX, GRAD>;
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, PWA_THREADS, 0);
        occ = o > 0 ? o : 1;
    }
    int64_t g = (n + PWA_THREADS - 1) / PWA_THREADS;
    if (g > (int64_t)sm_count * occ) g = (int64_t)sm_count * occ;
    if (g < 1) g = 1;
    int* badw = reinterpret_cast<int*>(counter + 1);
    kern<<<(unsigned)g, PWA_THREADS, 0, st>>>(A, K, H, n, ld, V, Psi, nfac, (float2*)ws, counter, badw, status, nll,
                                              grad);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t inc_dispatch(const float2* A, int K, int H, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                         double nfac, double* nll, double* grad, void* ws, unsigned* counter, int* status,
                         int sm_count, cudaStream_t st) {
    if (grad) return inc_launch<KMAX, true>(A, K, H, n, ld, V, Psi, nfac, nll, grad, ws, counter, status, sm_count, st);
    return inc_launch<KMAX, false>(A, K, H, n, ld, V, Psi, nfac, nll, nullptr, ws, counter, status, sm_count, st);
}

}  // namespace

cudaError_t launch_nll_incoherent(const float2* A, int K, int H, int64_t n, int64_t ld, const float2* V, int P,
                                  const double2* Psi, double nfac, double* nll, double* grad, void* ws,
                                  unsigned* counter, int* status, int sm_count, cudaStream_t st) {
    for (int p = 0; p < P; ++p) {
        const float2* Vp = V + (int64_t)p * K;
        double* np = nll + p;
        double* gp = grad ? grad + (int64_t)p * 2 * K : nullptr;
        cudaError_t e;
        if (K <= 4) e = inc_dispatch<4>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        else if (K <= 8) e = inc_dispatch<8>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        else if (K <= 16) e = inc_dispatch<16>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        else if (K <= 32) e = inc_dispatch<32>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        else if (K <= 48) e = inc_dispatch<48>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        else e = inc_dispatch<64>(A, K, H, n, ld, Vp, Psi, nfac, np, gp, ws, counter, status, sm_count, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pwa
