// -lnL and its gradient when resonance masses and widths float (Sec. 2: with floating shape
// parameters the MC bracket of Eq. 3 and the per-event products cannot be precomputed, so the
// amplitudes of the floating waves are recomputed every iteration and the normalisation is the
// MC sum itself):
//
//   f(V, theta) = -sum_i ln|u_i|^2 + (n_f / N_gen) sum_j w_j |u_j|^2,     u = sum_a V_a A_a,
//   g_c         = 2 df/dconj(V_c) = -2 sum_i conj(A_ic) u_i/I_i + 2 (n_f/N_gen) sum_j w_j conj(A_jc) u_j,
//   df/dtheta_q = -2 sum_i Re(conj(u_i) V_r dA_iq)/I_i + 2 (n_f/N_gen) sum_j w_j Re(conj(u_j) V_r dA_jq),
//
// with dA_q = dA_r/dtheta_q the derivative row of floating parameter q (wave r = fwave[q]).
//
// One launch covers both samples: the first Gd blocks stream the data events, the others the
// MC events (blocks split in proportion to the bytes), each block writes double-single partials
// of (scalar, 2K gradient sums, F shape sums), and the last block sums the data partials and the
// MC partials separately, in block order, and combines them in FP64.
//
// (The multi-channel fitter does not use this kernel: its evaluation, in uneven.cu, recomputes
// the amplitudes from the kinematics at the device trial point.)
#include "amp_model.cuh"
#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int SH_FMAX = 8;

struct ShapeArgs {
    const float2* A;
    const float2* dA;
    int64_t n, ld;
    const float2* Am;
    const float2* dAm;
    const float* wm;
    int64_t nm, ldm;
    int K, F;
    int fwave[SH_FMAX];
    int Gd;  // blocks on data
};

template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS) k_nll_shape(ShapeArgs s, const float2* __restrict__ V, double scale,
                                                           float2* __restrict__ part, unsigned* __restrict__ counter,
                                                           int* __restrict__ badw, int* __restrict__ status,
                                                           double* __restrict__ nll, double* __restrict__ grad) {
    constexpr bool HOLD = KMAX <= 32;
    constexpr int NG = 2 * KMAX + SH_FMAX;
    constexpr int ROUNDS = (NG + 31) / 32;
    constexpr int NW = PWA_THREADS / 32;
    __shared__ float2 sV[KMAX];
    __shared__ float2 sVr[SH_FMAX];
    __shared__ float sred[NW][ROUNDS * 32];
    __shared__ ff slred[NW];
    __shared__ int sLast;
    __shared__ ff sfin[2][PWA_THREADS];
    __shared__ double sval[2][1 + NG];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = s.K, F = s.F;
    if (tid < KMAX) sV[tid] = tid < K ? V[tid] : make_float2(0.f, 0.f);
    if (tid < SH_FMAX) sVr[tid] = tid < F ? V[s.fwave[tid]] : make_float2(0.f, 0.f);
    __syncthreads();

    const bool is_data = (int)blockIdx.x < s.Gd;
    const float2* A = is_data ? s.A : s.Am;
    const float2* dA = is_data ? s.dA : s.dAm;
    const int64_t n = is_data ? s.n : s.nm;
    const int64_t ld = is_data ? s.ld : s.ldm;
    const int64_t b0 = is_data ? blockIdx.x : blockIdx.x - s.Gd;
    const int64_t nb = is_data ? s.Gd : gridDim.x - s.Gd;

    float g[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) g[v] = 0.f;
    ff acc = ff_zero();
    bool bad = false;
    for (int64_t i = b0 * PWA_THREADS + tid; i < n; i += nb * PWA_THREADS) {
        float2 a[HOLD ? KMAX : 1];
        float ur = 0.f, ui = 0.f;
#pragma unroll
        for (int c = 0; c < KMAX; ++c) {
            const float2 x = (c < K) ? __ldg(A + c * ld + i) : make_float2(0.f, 0.f);
            if (HOLD) a[c] = x;
            cmac(ur, ui, sV[c].x, sV[c].y, x.x, x.y);
        }
        const float I0 = fmaf(ur, ur, ui * ui);  // one contraction, the same in every variant
        float wr, wi;
        if (is_data) {
            if (!intensity_ok(I0)) {
                bad = true;
                continue;
            }
            acc = ff_add_f(acc, __logf(I0));
            const float r = __frcp_rn(I0);
            wr = ur * r;
            wi = ui * r;
        } else {
            const float wt = s.wm ? __ldg(s.wm + i) : 1.f;
            acc = ff_add_f(acc, wt * I0);
            wr = wt * ur;
            wi = wt * ui;
        }
#pragma unroll
        for (int c = 0; c < KMAX; ++c) {
            float2 x;
            if (HOLD) x = a[c];
            else x = (c < K) ? __ldg(A + c * ld + i) : make_float2(0.f, 0.f);
            cmac_conj(g[2 * c], g[2 * c + 1], x.x, x.y, wr, wi);
        }
#pragma unroll
        for (int q = 0; q < SH_FMAX; ++q) {
            if (q < F) {
                const float2 d = __ldg(dA + q * ld + i);
                // Re(conj(w) * V_r * dA)
                const float2 vd = make_float2(sVr[q].x * d.x - sVr[q].y * d.y, sVr[q].x * d.y + sVr[q].y * d.x);
                g[2 * KMAX + q] = fmaf(wr, vd.x, g[2 * KMAX + q]);
                g[2 * KMAX + q] = fmaf(wi, vd.y, g[2 * KMAX + q]);
            }
        }
    }
    // warp reduce-scatter, block sum over warps -> block partial [1 + 2K + F]
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        float x[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (32 * r + j < NG) x[j] = g[32 * r + j];
            else x[j] = 0.f;
        }
        warp_transpose_reduce32(x);
        sred[warp][32 * r + lane] = x[0];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, m));
    if (lane == 0) slred[warp] = acc;
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    const int NV = 1 + 2 * K + F;
    float2* bp = part + (int64_t)blockIdx.x * NV;
    for (int v = tid; v < NV; v += PWA_THREADS) {
        ff t = ff_zero();
        if (v == 0) {
            for (int w = 0; w < NW; ++w) t = ff_add(t, slred[w]);
        } else {
            const int gi = v <= 2 * K ? v - 1 : 2 * KMAX + (v - 1 - 2 * K);
            for (int w = 0; w < NW; ++w) t = ff_add_f(t, sred[w][gi]);
        }
        bp[v] = make_float2(t.hi, t.lo);
    }
    if (any_bad && tid == 0) atomicOr(badw, 1);
    __threadfence();
    __syncthreads();
    if (tid == 0) sLast = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    // data partials (blocks 0..Gd-1) and MC partials (Gd..G-1), each in block order
    const int nch = PWA_THREADS / NV > 0 ? PWA_THREADS / NV : 1;
    for (int set = 0; set < 2; ++set) {
        const int first = set == 0 ? 0 : s.Gd;
        const int count = set == 0 ? s.Gd : (int)gridDim.x - s.Gd;
        for (int vv = tid; vv < nch * NV; vv += PWA_THREADS) {
            const int v = vv % NV, ch = vv / NV;
            const int cnt = count > ch ? (count - ch + nch - 1) / nch : 0;
            sfin[set][vv] = ff_sum_strided(part, (int64_t)(first + ch) * NV + v, (int64_t)nch * NV, cnt);
        }
    }
    __syncthreads();
    for (int v = tid; v < NV; v += PWA_THREADS)
        for (int set = 0; set < 2; ++set) {
            ff t = ff_zero();
            for (int ch = 0; ch < nch; ++ch) t = ff_add(t, sfin[set][ch * NV + v]);
            sval[set][v] = ff_to_double(t);
        }
    if (tid == 0) sLast = __ldcg(badw) != 0;
    __syncthreads();
    const bool isbad = sLast != 0;
    if (tid == 0) {
        nll[0] = isbad ? INFINITY : (-sval[0][0] + scale * sval[1][0]);
        if (isbad) atomicOr(status, 1);
        *badw = 0;
        *counter = 0u;
    }
    for (int v = 1 + tid; v < NV; v += PWA_THREADS)
        grad[v - 1] = isbad ? 0.0 : (-2.0 * sval[0][v] + 2.0 * scale * sval[1][v]);
}

int kmax_shape(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64; }

template <int KMAX>
int shape_occupancy() {
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nll_shape<KMAX>, PWA_THREADS, 0);
        occ = o > 0 ? o : 1;
    }
    return occ;
}

template <int KMAX>
cudaError_t shape_launch(ShapeArgs a, const float2* V, double scale, void* ws, size_t ws_bytes, unsigned* counter,
                         int* badw, int* status, double* nll, double* grad, int sm_count, cudaStream_t st) {
    // blocks in proportion to the bytes each sample streams, at least one per non-empty sample
    int64_t G = (int64_t)sm_count * shape_occupancy<KMAX>();
    const int64_t need = (a.n + a.nm + PWA_THREADS - 1) / PWA_THREADS;
    if (G > need) G = need;
    if (G < 2) G = 2;
    int64_t Gd = (int64_t)((double)G * (double)a.n / (double)(a.n + a.nm > 0 ? a.n + a.nm : 1) + 0.5);
    if (Gd < 1) Gd = 1;
    if (Gd > G - 1) Gd = G - 1;
    a.Gd = (int)Gd;
    const int NV = 1 + 2 * a.K + a.F;
    if ((size_t)G * NV * sizeof(float2) > ws_bytes) return cudaErrorInvalidValue;
    k_nll_shape<KMAX><<<(unsigned)G, PWA_THREADS, 0, st>>>(a, V, scale, (float2*)ws, counter, badw, status, nll, grad);
    return cudaGetLastError();
}

}  // namespace

size_t shape_workspace(int K, int F, int sm_count) {
    return sizeof(float2) * (size_t)(1 + 2 * K + F) * (size_t)sm_count * 8;
}

cudaError_t launch_nll_shape(const float2* A, const float2* dA, int K, int64_t n, int64_t ld, const float2* Am,
                             const float2* dAm, int64_t nm, int64_t ldm, const float* wm, double n_gen,
                             const int* fwave, int F, const float2* V, double nfac, double* nll, double* grad,
                             void* ws, size_t ws_bytes, unsigned* counter, int* badw, int* status, int sm_count,
                             cudaStream_t st) {
    ShapeArgs a;
    a.A = A;
    a.dA = dA;
    a.n = n;
    a.ld = ld;
    a.Am = Am;
    a.dAm = dAm;
    a.wm = wm;
    a.nm = nm;
    a.ldm = ldm;
    a.K = K;
    a.F = F;
    for (int q = 0; q < SH_FMAX; ++q) a.fwave[q] = q < F ? fwave[q] : 0;
    a.Gd = 1;
    const double scale = nfac / n_gen;
    switch (kmax_shape(K)) {
        case 4: return shape_launch<4>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
        case 8: return shape_launch<8>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
        case 16: return shape_launch<16>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
        case 32: return shape_launch<32>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
        case 48: return shape_launch<48>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
        default: return shape_launch<64>(a, V, scale, ws, ws_bytes, counter, badw, status, nll, grad, sm_count, st);
    }
}

}  // namespace pwa
