// Extended negative log-likelihood and its gradient in V (Sec. 2, Eq. 3 and footnote 2):
//
//   f(V)  = -sum_i ln I_i + n_f * S(V),     I_i = |u_i|^2,  u_i = sum_a V_a A_a(i),
//   S(V)  = sum_ab V_a conj(V_b) Psi_ab,
//   g_c   = dF/dRe V_c + i dF/dIm V_c = -2 sum_i conj(A_c(i)) u_i / I_i + 2 n_f sum_a Psi_ac V_a.
//
// The per-event K x K table of Sec. 2 (A_a conj(A_a') precomputed per event) is not built:
// the double sum over (a, a') of Eq. 3 equals |u_i|^2 of Eq. 1, which costs 2K reals and
// 8K flops per event instead of K^2 of each, so the data sum streams A once per evaluation.
//
// Two kernels:
//  * k_nll_stream  (one parameter set): HBM-bound stream over A (8K bytes per event).  Each
//    thread takes two events per 16-byte load per wave, holds V in shared memory, and keeps
//    FP32 gradient partials in registers.  Warp partials are combined by a reduce-scatter
//    (31 shuffles for 32 values) and then summed exactly in fixed point; the last block of the
//    grid adds the normalisation term (nll_common.cuh): one launch per evaluation,
//    deterministic.
//  * k_nll_batched (P > 1 parameter sets, multi-start): the event x wave x start complex
//    contraction U = A V^T, W = U / |U|^2, G = A^H W on FP32 FMA pipes, tiled through shared
//    memory (an A tile of E events feeds both contractions), with per-start compensated
//    sums of ln I.  k_nll_finalize then sums the chunk partials per start in order and adds
//    the normalisation term in FP64.
//
// Sec. 2 precision remark: FP32 amplitudes and per-event arithmetic, FP64 for the last sum,
// added in a tree-like order.  Here the per-thread sums are FP32 (gradient) or
// double-single (ln I) over a bounded number of events, warp sums a fixed tree; across warps
// and blocks the single-set kernels sum exactly (integer fixed point) and the batched kernel
// carries double-single pairs in a fixed order.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "nll_common.cuh"
#include "tma.cuh"

namespace pwa {

namespace {

// ======================================================================= one parameter set
template <int KMAX, bool GRAD, bool HOLD, bool FUSED>
__global__ void __launch_bounds__(PWA_THREADS) k_nll_stream(
    const float2* __restrict__ A, int K, int64_t n, int64_t ld, const float2* __restrict__ V,
    const double2* __restrict__ Psi, double nfac, float2* __restrict__ part, unsigned* __restrict__ counter,
    int* __restrict__ badw, int* __restrict__ status, double* __restrict__ nll, double* __restrict__ grad) {
    constexpr bool EV2 = KMAX <= 16;   // two events per thread and iteration (16-byte loads)
    // HOLD: keep the event's amplitudes in registers for the gradient pass; otherwise reload
    // them (L1 hits: the same lines were just read) to free registers for more warps
    constexpr int NG = 2 * KMAX;
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
    const int64_t stride = (int64_t)gridDim.x * PWA_THREADS;

    if (EV2) {
        const float4* A4 = reinterpret_cast<const float4*>(A);
        const int64_t ld2 = ld >> 1;
        const int64_t npairs = (n + 1) >> 1;
        for (int64_t q = (int64_t)blockIdx.x * PWA_THREADS + tid; q < npairs; q += stride) {
            float4 a[KMAX];
#pragma unroll
            for (int c = 0; c < KMAX; ++c) a[c] = (c < K) ? __ldg(A4 + c * ld2 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool has1 = 2 * q + 1 < n;
            if (!has1) {  // odd n: the pair's second slot is padding, whatever it holds
#pragma unroll
                for (int c = 0; c < KMAX; ++c) a[c].z = a[c].w = 0.f;
            }
            float u0r = 0.f, u0i = 0.f, u1r = 0.f, u1i = 0.f;
#pragma unroll
            for (int c = 0; c < KMAX; ++c) {
                const float2 v = sV[c];
                cmac(u0r, u0i, v.x, v.y, a[c].x, a[c].y);
                cmac(u1r, u1i, v.x, v.y, a[c].z, a[c].w);
            }
            const float I0 = fmaf(u0r, u0r, u0i * u0i);  // one contraction, the same in every variant
            const float I1 = fmaf(u1r, u1r, u1i * u1i);  // one contraction, the same in every variant
            float w0r = 0.f, w0i = 0.f, w1r = 0.f, w1i = 0.f;
            if (intensity_ok(I0)) {
                lacc = ff_add_f(lacc, __logf(I0));
                const float r = __frcp_rn(I0);
                w0r = u0r * r;
                w0i = u0i * r;
            } else {
                bad = true;
            }
            if (has1) {
                if (intensity_ok(I1)) {
                    lacc = ff_add_f(lacc, __logf(I1));
                    const float r = __frcp_rn(I1);
                    w1r = u1r * r;
                    w1i = u1i * r;
                } else {
                    bad = true;
                }
            }
            if (GRAD) {
#pragma unroll
                for (int c = 0; c < KMAX; ++c) {
                    float4 x = a[c];
                    if (!HOLD) {
                        x = (c < K) ? __ldg(A4 + c * ld2 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (!has1) x.z = x.w = 0.f;
                    }
                    cmac_conj(g[2 * c], g[2 * c + 1], x.x, x.y, w0r, w0i);
                    cmac_conj(g[2 * c], g[2 * c + 1], x.z, x.w, w1r, w1i);
                }
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * PWA_THREADS + tid; i < n; i += stride) {
            float2 a[HOLD ? KMAX : 1];
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int c = 0; c < KMAX; ++c) {
                const float2 x = (c < K) ? __ldg(A + c * ld + i) : make_float2(0.f, 0.f);
                if (HOLD) a[c] = x;
                const float2 v = sV[c];
                cmac(ur, ui, v.x, v.y, x.x, x.y);
            }
            const float I0 = fmaf(ur, ur, ui * ui);  // one contraction, the same in every variant
            float wr = 0.f, wi = 0.f;
            if (intensity_ok(I0)) {
                lacc = ff_add_f(lacc, __logf(I0));
                const float r = __frcp_rn(I0);
                wr = ur * r;
                wi = ui * r;
            } else {
                bad = true;
            }
            if (GRAD) {
#pragma unroll
                for (int c = 0; c < KMAX; ++c) {
                    float2 x;
                    if (HOLD) x = a[c];
                    else x = (c < K) ? __ldg(A + c * ld + i) : make_float2(0.f, 0.f);
                    cmac_conj(g[2 * c], g[2 * c + 1], x.x, x.y, wr, wi);
                }
            }
        }
    }

    stream_reduce_finalize<KMAX, GRAD, FUSED, PWA_THREADS>(g, lacc, bad, sV, red, K, Psi, nfac, part, counter, badw,
                                                           status, nll, grad);
}

// ----------------------------------------------------------------------- TMA-pipelined variant
// The same arithmetic with the amplitude stream staged through shared memory by bulk copies:
// thread 0 keeps S stages of E events x K waves in flight (one 1-D cp.async.bulk per wave row,
// completion counted on the stage's mbarrier), so the bytes in flight no longer depend on how
// many registers the consumers use.  One thread per event of the tile; persistent grid.
template <int KMAX>
struct TmaCfg {
    static constexpr int E = 128;  // events per tile == threads per block
    static constexpr int S0 = 98304 / (KMAX * E * 8);
    static constexpr int S = S0 < 2 ? 2 : (S0 > 4 ? 4 : S0);
    static constexpr size_t SMEM = sizeof(float2) * (size_t)S * KMAX * E + 64;
};

template <int KMAX, bool GRAD>
__global__ void __launch_bounds__(TmaCfg<KMAX>::E) k_nll_tma(
    const float2* __restrict__ A, int K, int64_t n, int64_t ld, const float2* __restrict__ V,
    const double2* __restrict__ Psi, double nfac, float2* __restrict__ part, unsigned* __restrict__ counter,
    int* __restrict__ badw, int* __restrict__ status, double* __restrict__ nll, double* __restrict__ grad) {
    using C = TmaCfg<KMAX>;
    constexpr int E = C::E, S = C::S, NG = 2 * KMAX;
    extern __shared__ __align__(128) unsigned char tsm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(tsm);               // [S] (64 bytes reserved)
    float2* buf = reinterpret_cast<float2*>(tsm + 64);                // [S][KMAX][E]
    __shared__ float2 sV[KMAX];
    __shared__ StreamReduceSmem<KMAX, E> red;
    const int tid = threadIdx.x;
    if (tid < KMAX) sV[tid] = tid < K ? V[tid] : make_float2(0.f, 0.f);
    const int64_t ntile = (n + E - 1) / E;
    const int64_t my_tiles = blockIdx.x < ntile ? (ntile - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int st = 0; st < S; ++st) mbar_init(&full[st], 1);
        fence_mbar_init();
    }
    stream_reduce_init<KMAX, E>(red, Psi, K);
    __syncthreads();
    auto issue = [&](int64_t j) {  // tile index j of this block -> stage j % S
        const int st = (int)(j % S);
        const int64_t e0 = ((int64_t)blockIdx.x + j * gridDim.x) * E;
        int64_t ev = n - e0;
        if (ev > E) ev = E;
        ev = (ev + 1) & ~(int64_t)1;  // even: 16-byte multiple (ld is even, so still inside the row)
        const uint32_t row_bytes = (uint32_t)(ev * sizeof(float2));
        mbar_arrive_expect_tx(&full[st], row_bytes * (uint32_t)K);
        for (int a = 0; a < K; ++a)
            bulk_copy_g2s(buf + ((size_t)st * KMAX + a) * E, A + a * ld + e0, row_bytes, &full[st]);
    };
    if (tid == 0)
        for (int64_t j = 0; j < my_tiles && j < S; ++j) issue(j);

    float g[NG];
#pragma unroll
    for (int v = 0; v < NG; ++v) g[v] = 0.f;
    ff lacc = ff_zero();
    bool bad = false;
    __shared__ int s_timeout_at;
    if (tid == 0) s_timeout_at = -1;
    __syncthreads();
    int64_t timeout_at = -1;
    for (int64_t j = 0; j < my_tiles; ++j) {
        const int st = (int)(j % S);
        const uint32_t parity = (uint32_t)((j / S) & 1);
        if (!mbar_wait_bounded(&full[st], parity, 2000000000ull)) timeout_at = j;
        if (__syncthreads_or(timeout_at >= 0 ? 1 : 0)) {
            if (timeout_at >= 0) atomicCAS(&s_timeout_at, -1, (int)timeout_at);
            break;
        }
        const int64_t e = ((int64_t)blockIdx.x + j * gridDim.x) * E + tid;
        if (e < n) {
            const float2* col = buf + (size_t)st * KMAX * E + tid;
            float2 a[KMAX];
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int c = 0; c < KMAX; ++c) {
                a[c] = (c < K) ? col[c * E] : make_float2(0.f, 0.f);
                const float2 v = sV[c];
                cmac(ur, ui, v.x, v.y, a[c].x, a[c].y);
            }
            const float I0 = fmaf(ur, ur, ui * ui);  // one contraction, the same in every variant
            if (intensity_ok(I0)) {
                lacc = ff_add_f(lacc, __logf(I0));
                if (GRAD) {
                    const float r = __frcp_rn(I0);
                    const float wr = ur * r, wi = ui * r;
#pragma unroll
                    for (int c = 0; c < KMAX; ++c) {
                        cmac_conj(g[2 * c], g[2 * c + 1], a[c].x, a[c].y, wr, wi);
                    }
                }
            } else {
                bad = true;
            }
        }
        __syncthreads();  // every thread is done with stage st
        if (tid == 0 && j + S < my_tiles) {
            fence_proxy_async_smem();
            issue(j + S);
        }
    }
    __syncthreads();
    if (s_timeout_at >= 0) {
        // a stage never completed: flag the error, then wait (bounded) for the copies of the
        // stages still in flight so that none lands after the block has exited
        if (tid == 0) {
            atomicOr(status, 2);
            atomicOr(badw, 1);
            const int64_t j0 = s_timeout_at;
            for (int64_t jj = j0; jj < my_tiles && jj < j0 + S; ++jj)
                mbar_wait_bounded(&full[jj % S], (uint32_t)((jj / S) & 1), 100000000ull);
        }
        bad = true;
    }
    stream_reduce_finalize<KMAX, GRAD, true, E>(g, lacc, bad, sV, red, K, Psi, nfac, part, counter, badw, status, nll,
                                                grad);
}

// Second half of the unfused variant: one block sums the G block partials in block order and
// adds the FP64 normalisation term.
template <int KMAX, bool GRAD>
__global__ void __launch_bounds__(PWA_THREADS) k_nll_stream_final(
    const float2* __restrict__ part, int G, int K, const float2* __restrict__ V, const double2* __restrict__ Psi,
    double nfac, int* __restrict__ badw, int* __restrict__ status, double* __restrict__ nll,
    double* __restrict__ grad) {
    constexpr int NG = 2 * KMAX;
    __shared__ ff sfin[PWA_THREADS];
    __shared__ double sval[1 + NG];
    __shared__ double2 sT[KMAX];
    __shared__ float2 sV[KMAX];
    __shared__ int sBad;
    __shared__ double2 scratch[PWA_THREADS];
    __shared__ double sS;
    const int tid = threadIdx.x;
    if (tid < KMAX) sV[tid] = tid < K ? V[tid] : make_float2(0.f, 0.f);
    const int NV = 1 + 2 * K;
    const int NVu = GRAD ? NV : 1;
    const int nch = PWA_THREADS / NVu;
    if (tid < nch * NVu) {
        const int v = tid % NVu, ch = tid / NVu;
        const int cnt = (G - ch + nch - 1) / nch;
        sfin[tid] = ff_sum_strided(part, (int64_t)ch * NV + v, (int64_t)nch * NV, cnt);
    }
    if (tid == 0) sBad = *badw;
    __syncthreads();
    if (tid < NVu) {
        ff s = ff_zero();
        for (int ch = 0; ch < nch; ++ch) s = ff_add(s, sfin[ch * NVu + tid]);
        sval[tid] = ff_to_double(s);
    }
    const double S = psi_times_v<PWA_THREADS>(Psi, sV, K, sT, scratch, &sS);
    const bool isbad = sBad != 0;
    if (tid == 0) {
        nll[0] = isbad ? INFINITY : (-sval[0] + nfac * S);
        if (isbad) atomicOr(status, 1);
        *badw = 0;
    }
    if (GRAD && tid < K) {
        grad[2 * tid] = isbad ? 0.0 : (-2.0 * sval[1 + 2 * tid] + 2.0 * nfac * sT[tid].x);
        grad[2 * tid + 1] = isbad ? 0.0 : (-2.0 * sval[2 + 2 * tid] + 2.0 * nfac * sT[tid].y);
    }
}

// ======================================================================= P parameter sets
template <int KMAX, int E, int PB>
struct BatchedCfg {
    static constexpr int EA = E + 2;             // padded row stride of sA (float2, even -> 16-B rows)
    static constexpr int EW = E + 2;             // padded row stride of sW ([PB][EW])
    static constexpr int TE = E / 16;            // GEMM1 events per thread (pairs of 2)
    static constexpr int TP = PB / 16;           // GEMM1 starts per thread (pairs of 2)
    static constexpr int TA = KMAX < 16 ? KMAX : 16;
    static constexpr int TPG = PWA_THREADS / TA;
    static constexpr int KA = KMAX / TA;         // GEMM2 waves per thread
    static constexpr int PP = PB / TPG;          // GEMM2 starts per thread
    static constexpr int LD4 = KMAX * E / 2 / PWA_THREADS;  // float4 tile loads per thread
    static constexpr int FLUSH = (128 + E - 1) / E;          // tiles between flushes of G
    static constexpr size_t SMEM = sizeof(float2) * (KMAX * PB + KMAX * EA + PB * EW) +
                                   sizeof(float4) * KMAX * PB + sizeof(ff) * PB + sizeof(int) * PB;
    static_assert(TE >= 2 && TP >= 2 && PP >= 1 && KA >= 1, "tile shape");
    static_assert(KMAX * E / 2 % PWA_THREADS == 0, "tile loader");
};

template <int KMAX, int E, int PB>
__global__ void __launch_bounds__(PWA_THREADS, 2) k_nll_batched(
    const float2* __restrict__ A, int K, int64_t n, int64_t ld, const float2* __restrict__ V, int P,
    int64_t ev_per_chunk, float2* __restrict__ part, int* __restrict__ bad, int with_grad) {
    using C = BatchedCfg<KMAX, E, PB>;
    extern __shared__ float4 smem[];
    float2* sV = reinterpret_cast<float2*>(smem);  // [KMAX][PB]
    float2* sA = sV + KMAX * PB;                    // [KMAX][EA]
    float2* sW = sA + KMAX * C::EA;                 // [PB][EW]
    float4* sG = reinterpret_cast<float4*>(sW + PB * C::EW);  // [PB][KMAX] complex double-single
    ff* sL = reinterpret_cast<ff*>(sG + KMAX * PB);            // [PB]
    int* sBad = reinterpret_cast<int*>(sL + PB);               // [PB]

    const int tid = threadIdx.x;
    const int chunk = blockIdx.x;
    const int p0 = blockIdx.y * PB;
    const int NV = 1 + 2 * K;
    const int K4 = (K + 3) & ~3;  // <= KMAX (KMAX is a multiple of 8)

    for (int idx = tid; idx < KMAX * PB; idx += PWA_THREADS) {
        const int a = idx / PB, p = idx % PB;
        sV[idx] = (a < K && p0 + p < P) ? V[(int64_t)(p0 + p) * K + a] : make_float2(0.f, 0.f);
        sG[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int p = tid; p < PB; p += PWA_THREADS) {
        sL[p] = ff_zero();
        sBad[p] = 0;
    }

    const int64_t e_begin = (int64_t)chunk * ev_per_chunk;
    int64_t e_end = e_begin + ev_per_chunk;
    if (e_end > n) e_end = n;

    // GEMM1 coordinates: events 2*te + {0,1} + 32*r, starts 2*tp + {0,1} + 32*s
    const int te = tid % 16, tp = tid / 16;
    // GEMM2 coordinates: waves ta + TA*k, starts tg + TPG*s
    const int ta = tid % C::TA, tg = tid / C::TA;

    float4 pre[C::LD4];
    auto load_tile = [&](int64_t e0) {
#pragma unroll
        for (int j = 0; j < C::LD4; ++j) {
            const int idx = tid + PWA_THREADS * j;
            const int a = idx / (E / 2), c4 = idx % (E / 2);
            const int64_t e = e0 + 2 * c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a < K && e < e_end) {
                v = __ldg(reinterpret_cast<const float4*>(A + a * ld + e));
                if (e + 1 >= e_end) { v.z = 0.f; v.w = 0.f; }
            }
            pre[j] = v;
        }
    };

    ff lsum[C::TP];
#pragma unroll
    for (int s = 0; s < C::TP; ++s) lsum[s] = ff_zero();
    float gacc[C::KA][C::PP][2];
#pragma unroll
    for (int k = 0; k < C::KA; ++k)
#pragma unroll
        for (int s = 0; s < C::PP; ++s) gacc[k][s][0] = gacc[k][s][1] = 0.f;
    int since_flush = 0;

    auto flush_g = [&]() {
#pragma unroll
        for (int k = 0; k < C::KA; ++k)
#pragma unroll
            for (int s = 0; s < C::PP; ++s) {
                float4* dst = sG + (tg + C::TPG * s) * KMAX + (ta + C::TA * k);
                float4 cur = *dst;
                ff re = ff_add_f(ff{cur.x, cur.y}, gacc[k][s][0]);
                ff im = ff_add_f(ff{cur.z, cur.w}, gacc[k][s][1]);
                *dst = make_float4(re.hi, re.lo, im.hi, im.lo);
                gacc[k][s][0] = gacc[k][s][1] = 0.f;
            }
    };

    if (e_begin < e_end) load_tile(e_begin);
    for (int64_t e0 = e_begin; e0 < e_end; e0 += E) {
        __syncthreads();  // previous GEMM2 done with sA / sW
#pragma unroll
        for (int j = 0; j < C::LD4; ++j) {
            const int idx = tid + PWA_THREADS * j;
            const int a = idx / (E / 2), c4 = idx % (E / 2);
            *reinterpret_cast<float4*>(sA + a * C::EA + 2 * c4) = pre[j];
        }
        __syncthreads();
        if (e0 + E < e_end) load_tile(e0 + E);  // prefetch next tile into registers

        // ---- GEMM1: U[e][p] = sum_a A[a][e] V[p][a]
        float u[C::TE][C::TP][2];
#pragma unroll
        for (int r = 0; r < C::TE; ++r)
#pragma unroll
            for (int s = 0; s < C::TP; ++s) u[r][s][0] = u[r][s][1] = 0.f;
        // rows K..K4-1 of sA and sV are zero, so the wave loop runs in steps of 4 with
        // compile-time offsets inside each step
        const float2* pA = sA + 2 * te;
        const float2* pV = sV + 2 * tp;
        for (int a0 = 0; a0 < K4; a0 += 4)
#pragma unroll
        for (int da = 0; da < 4; ++da) {
            const int a = a0 + da;
            float4 av[C::TE / 2], vv[C::TP / 2];
#pragma unroll
            for (int r = 0; r < C::TE / 2; ++r) av[r] = *reinterpret_cast<const float4*>(pA + a * C::EA + 32 * r);
#pragma unroll
            for (int s = 0; s < C::TP / 2; ++s) vv[s] = *reinterpret_cast<const float4*>(pV + a * PB + 32 * s);
#pragma unroll
            for (int r = 0; r < C::TE / 2; ++r)
#pragma unroll
                for (int s = 0; s < C::TP / 2; ++s) {
                    // events (2r: av.x,av.y) (2r+1: av.z,av.w); starts (2s: vv.x,vv.y) (2s+1: vv.z,vv.w)
                    cmac(u[2 * r][2 * s][0], u[2 * r][2 * s][1], av[r].x, av[r].y, vv[s].x, vv[s].y);
                    cmac(u[2 * r][2 * s + 1][0], u[2 * r][2 * s + 1][1], av[r].x, av[r].y, vv[s].z, vv[s].w);
                    cmac(u[2 * r + 1][2 * s][0], u[2 * r + 1][2 * s][1], av[r].z, av[r].w, vv[s].x, vv[s].y);
                    cmac(u[2 * r + 1][2 * s + 1][0], u[2 * r + 1][2 * s + 1][1], av[r].z, av[r].w, vv[s].z, vv[s].w);
                }
        }
        // ---- epilogue: I = |U|^2, ln I, W = U / I  -> sW[p][e]
#pragma unroll
        for (int s = 0; s < C::TP; ++s) {
            const int p = 2 * tp + (s & 1) + 32 * (s >> 1);
            const bool pv = p0 + p < P;
            float lpart = 0.f;
#pragma unroll
            for (int r = 0; r < C::TE; r += 2) {
                const int e = 2 * te + 32 * (r >> 1);
                float w[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float ur = u[r + h][s][0], ui = u[r + h][s][1];
                    const float I = fmaf(ur, ur, ui * ui);  // one contraction, the same in every variant
                    float wr = 0.f, wi = 0.f;
                    if (pv && e0 + e + h < e_end) {
                        if (intensity_ok(I)) {
                            lpart += __logf(I);
                            const float rc = __fdividef(1.f, I);
                            wr = ur * rc;
                            wi = ui * rc;
                        } else {
                            sBad[p] = 1;
                        }
                    }
                    w[2 * h] = wr;
                    w[2 * h + 1] = wi;
                }
                *reinterpret_cast<float4*>(sW + p * C::EW + e) = make_float4(w[0], w[1], w[2], w[3]);
            }
            lsum[s] = ff_add_f(lsum[s], lpart);
        }
        __syncthreads();
        // ---- GEMM2: G[a][p] += sum_e conj(A[a][e]) W[p][e]
        if (with_grad) {
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                float4 av[C::KA], wv[C::PP];
#pragma unroll
                for (int k = 0; k < C::KA; ++k) av[k] = *reinterpret_cast<const float4*>(sA + (ta + C::TA * k) * C::EA + e);
#pragma unroll
                for (int s = 0; s < C::PP; ++s) wv[s] = *reinterpret_cast<const float4*>(sW + (tg + C::TPG * s) * C::EW + e);
#pragma unroll
                for (int k = 0; k < C::KA; ++k)
#pragma unroll
                    for (int s = 0; s < C::PP; ++s) {
                        cmac_conj(gacc[k][s][0], gacc[k][s][1], av[k].x, av[k].y, wv[s].x, wv[s].y);
                        cmac_conj(gacc[k][s][0], gacc[k][s][1], av[k].z, av[k].w, wv[s].z, wv[s].w);
                    }
            }
            if (++since_flush == C::FLUSH) {
                since_flush = 0;
                flush_g();
            }
        }
    }
    if (with_grad) flush_g();
    // ln I: reduce the 16 GEMM1 event groups (lanes te = 0..15 of a half warp) per start
#pragma unroll
    for (int s = 0; s < C::TP; ++s) {
        ff v = lsum[s];
#pragma unroll
        for (int m = 8; m > 0; m >>= 1) v = ff_add(v, ff_shfl_xor(v, m));
        if (te == 0) sL[2 * tp + (s & 1) + 32 * (s >> 1)] = v;
    }
    __syncthreads();
    // ---- block result -> part[chunk][p][v]  (v = 0: sum ln I; 1+2a, 2+2a: Re, Im of G[a])
    const int np = (P - p0) < PB ? (P - p0) : PB;
    const int NVu = with_grad ? NV : 1;
    for (int idx = tid; idx < np * NVu; idx += PWA_THREADS) {
        const int p = idx / NVu, v = idx % NVu;
        float2 out;
        if (v == 0) {
            out = make_float2(sL[p].hi, sL[p].lo);
        } else {
            const float4 gv = sG[p * KMAX + ((v - 1) >> 1)];
            out = ((v - 1) & 1) ? make_float2(gv.z, gv.w) : make_float2(gv.x, gv.y);
        }
        part[((int64_t)chunk * P + p0 + p) * NV + v] = out;
    }
    for (int p = tid; p < np; p += PWA_THREADS)
        if (sBad[p]) bad[p0 + p] = 1;
}

// ----------------------------------------------------------------------- P sets, pipelined
// The same contraction with larger register tiles and the amplitude tile staged by bulk copies
// (K <= 32): tiles of E = 128 events x PB = 64 starts per block, one block per SM.
//  * U = A V^T: thread (te, tp) holds 8 events x 4 starts (events 2 te + {0,1} + 32 r, starts
//    2 tp + {0,1} + 32 s): per wave 6 shared 16-byte loads feed 128 FMAs.
//  * G = A^H W: the four event quarters of the tile are summed by four groups of 64 threads;
//    thread (q, ta, tg) holds waves ta + 8 k (k < K/8) x starts tg + 8 s (s < 8) over its
//    quarter's events: per event pair 4 + 8 loads feed 256 FMAs (K = 32).  The groups' FP32
//    partials are added to the block's double-single G in four phases every FLUSH tiles.
//  * Rows of the shared tiles are padded to E + 2 (a stride of 4 banks), so the eight wave
//    rows (or the four start rows) that a warp reads hit distinct banks.
//  * Thread 0 keeps two stages of K row copies in flight (cp.async.bulk, completion counted
//    on each stage's mbarrier); every wait is bounded (a timeout flags the error and leaves).
template <int KMAX>
struct Batched2Cfg {
    static constexpr int E = 128, PB = 64, NT = PWA_THREADS;
    static constexpr int EA = E + 2;  // float2 row stride of sA and sW
    static constexpr int S = 2;       // amplitude stages
    static constexpr int GW = KMAX / 8;  // G waves per thread
    static constexpr int FLUSH = 4;   // tiles between flushes of G
    static constexpr size_t OFF_A = 64;  // after the stage mbarriers
    static constexpr size_t OFF_V = OFF_A + sizeof(float2) * S * KMAX * EA;
    static constexpr size_t OFF_W = OFF_V + sizeof(float2) * KMAX * PB;
    static constexpr size_t OFF_G = OFF_W + sizeof(float2) * PB * EA;
    static constexpr size_t OFF_L = OFF_G + sizeof(float4) * KMAX * PB;
    static constexpr size_t OFF_B = OFF_L + sizeof(ff) * PB;
    static constexpr size_t SMEM = OFF_B + sizeof(int) * (PB + 4);
    static_assert(KMAX % 8 == 0 && KMAX <= 32, "pipelined batched kernel: K <= 32");
};

template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS, 1) k_nll_batched2(
    const float2* __restrict__ A, int K, int64_t n, int64_t ld, const float2* __restrict__ V, int P,
    int64_t ev_per_chunk, float2* __restrict__ part, int* __restrict__ bad, int with_grad, int* __restrict__ status) {
    using C = Batched2Cfg<KMAX>;
    constexpr int E = C::E, PB = C::PB, EA = C::EA, S = C::S, GW = C::GW;
    extern __shared__ __align__(128) unsigned char bsm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(bsm);
    float2* sA = reinterpret_cast<float2*>(bsm + C::OFF_A);  // [S][KMAX][EA]
    float2* sV = reinterpret_cast<float2*>(bsm + C::OFF_V);  // [KMAX][PB]
    float2* sW = reinterpret_cast<float2*>(bsm + C::OFF_W);  // [PB][EA]
    float4* sG = reinterpret_cast<float4*>(bsm + C::OFF_G);  // [PB][KMAX] complex double-single
    ff* sL = reinterpret_cast<ff*>(bsm + C::OFF_L);          // [PB]
    int* sBad = reinterpret_cast<int*>(bsm + C::OFF_B);      // [PB], then the timeout word

    const int tid = threadIdx.x;
    const int p0 = blockIdx.y * PB;
    const int NV = 1 + 2 * K;
    const int K4 = (K + 3) & ~3;
    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_chunk;
    int64_t e_end = e_begin + ev_per_chunk;
    if (e_end > n) e_end = n;
    const int64_t ntile = e_begin < e_end ? (e_end - e_begin + E - 1) / E : 0;

    for (int i = tid; i < S * KMAX * EA; i += PWA_THREADS) sA[i] = make_float2(0.f, 0.f);
    for (int idx = tid; idx < KMAX * PB; idx += PWA_THREADS) {
        const int a = idx / PB, p = idx % PB;
        sV[idx] = (a < K && p0 + p < P) ? V[(int64_t)(p0 + p) * K + a] : make_float2(0.f, 0.f);
        sG[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int p = tid; p < PB; p += PWA_THREADS) {
        sL[p] = ff_zero();
        sBad[p] = 0;
    }
    if (tid == 0) {
        sBad[PB] = 0;
        for (int st = 0; st < S; ++st) mbar_init(&mbar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // tile j -> stage j % S: K row copies of its (even) event count
    auto issue = [&](int64_t j) {
        const int st = (int)(j % S);
        const int64_t e0 = e_begin + j * E;
        int64_t ev = e_end - e0;
        if (ev > E) ev = E;
        ev = (ev + 1) & ~(int64_t)1;  // ld is even: the extra column is padding inside the row
        const uint32_t row_bytes = (uint32_t)(ev * sizeof(float2));
        mbar_arrive_expect_tx(&mbar[st], row_bytes * (uint32_t)K);
        for (int a = 0; a < K; ++a)
            bulk_copy_g2s(sA + ((size_t)st * KMAX + a) * EA, A + a * ld + e0, row_bytes, &mbar[st]);
    };
    if (tid == 0) {
        fence_proxy_async_smem();  // the zero fill above precedes the copies into the stages
        for (int64_t j = 0; j < ntile && j < S; ++j) issue(j);
    }

    // GEMM1 coordinates
    const int te = tid & 15, tp = tid >> 4;
    // GEMM2 coordinates
    const int q = tid >> 6, ta = tid & 7, tg = (tid >> 3) & 7;

    ff lsum[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) lsum[s] = ff_zero();
    float gacc[GW][8][2];
#pragma unroll
    for (int k = 0; k < GW; ++k)
#pragma unroll
        for (int s = 0; s < 8; ++s) gacc[k][s][0] = gacc[k][s][1] = 0.f;

    auto flush_g = [&]() {
        for (int ph = 0; ph < 4; ++ph) {
            if (q == ph) {
#pragma unroll
                for (int k = 0; k < GW; ++k)
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        float4* dst = sG + (tg + 8 * s) * KMAX + (ta + 8 * k);
                        const float4 cur = *dst;
                        const ff re = ff_add_f(ff{cur.x, cur.y}, gacc[k][s][0]);
                        const ff im = ff_add_f(ff{cur.z, cur.w}, gacc[k][s][1]);
                        *dst = make_float4(re.hi, re.lo, im.hi, im.lo);
                        gacc[k][s][0] = gacc[k][s][1] = 0.f;
                    }
            }
            __syncthreads();
        }
    };

    int64_t timeout_at = -1;
    for (int64_t j = 0; j < ntile; ++j) {
        const int st = (int)(j % S);
        const uint32_t parity = (uint32_t)((j / S) & 1);
        const bool ok = mbar_wait_bounded(&mbar[st], parity, 2000000000ull);
        if (__syncthreads_or(ok ? 0 : 1)) {
            timeout_at = j;
            break;
        }
        const int64_t e0 = e_begin + j * E;
        const int nvalid = (int)((e_end - e0) < E ? (e_end - e0) : E);
        const float2* sAs = sA + (size_t)st * KMAX * EA;
        // an odd event count copies one padding column: clear it before use (NaN-safe)
        if ((nvalid & 1) && tid < K) sA[((size_t)st * KMAX + tid) * EA + nvalid] = make_float2(0.f, 0.f);
        if (nvalid & 1) __syncthreads();

        // ---- GEMM1: U[e][p] = sum_a A[a][e] V[p][a]
        float u[8][4][2];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int s = 0; s < 4; ++s) u[i][s][0] = u[i][s][1] = 0.f;
        const float2* pA = sAs + 2 * te;
        const float2* pV = sV + 2 * tp;
        for (int a0 = 0; a0 < K4; a0 += 4)
#pragma unroll
            for (int da = 0; da < 4; ++da) {
                const int a = a0 + da;
                float4 av[4], vv[2];
#pragma unroll
                for (int r = 0; r < 4; ++r) av[r] = *reinterpret_cast<const float4*>(pA + a * EA + 32 * r);
#pragma unroll
                for (int s = 0; s < 2; ++s) vv[s] = *reinterpret_cast<const float4*>(pV + a * PB + 32 * s);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        // events (2r: av.x,av.y) (2r+1: av.z,av.w); starts (2s: vv.x,vv.y) (2s+1: vv.z,vv.w)
                        cmac(u[2 * r][2 * s][0], u[2 * r][2 * s][1], av[r].x, av[r].y, vv[s].x, vv[s].y);
                        cmac(u[2 * r][2 * s + 1][0], u[2 * r][2 * s + 1][1], av[r].x, av[r].y, vv[s].z, vv[s].w);
                        cmac(u[2 * r + 1][2 * s][0], u[2 * r + 1][2 * s][1], av[r].z, av[r].w, vv[s].x, vv[s].y);
                        cmac(u[2 * r + 1][2 * s + 1][0], u[2 * r + 1][2 * s + 1][1], av[r].z, av[r].w, vv[s].z, vv[s].w);
                    }
            }
        // ---- epilogue: I = |U|^2, ln I, W = U / I -> sW[p][e]
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int p = 2 * tp + (s & 1) + 32 * (s >> 1);
            const bool pv = p0 + p < P;
            float lpart = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = 2 * te + 32 * r;
                float w[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float ur = u[2 * r + h][s][0], ui = u[2 * r + h][s][1];
                    const float I = fmaf(ur, ur, ui * ui);  // one contraction, the same in every variant
                    float wr = 0.f, wi = 0.f;
                    if (pv && e + h < nvalid) {
                        if (intensity_ok(I)) {
                            lpart += __logf(I);
                            const float rc = __fdividef(1.f, I);
                            wr = ur * rc;
                            wi = ui * rc;
                        } else {
                            sBad[p] = 1;
                        }
                    }
                    w[2 * h] = wr;
                    w[2 * h + 1] = wi;
                }
                *reinterpret_cast<float4*>(sW + p * EA + e) = make_float4(w[0], w[1], w[2], w[3]);
            }
            lsum[s] = ff_add_f(lsum[s], lpart);
        }
        __syncthreads();
        // ---- GEMM2: G[a][p] += sum_e conj(A[a][e]) W[p][e] over this thread's event quarter
        if (with_grad) {
            const float2* qA = sAs + ta * EA + 32 * q;
            const float2* qW = sW + tg * EA + 32 * q;
#pragma unroll 2
            for (int e = 0; e < 32; e += 2) {
                float4 av[GW], wv[8];
#pragma unroll
                for (int k = 0; k < GW; ++k) av[k] = *reinterpret_cast<const float4*>(qA + 8 * k * EA + e);
#pragma unroll
                for (int s = 0; s < 8; ++s) wv[s] = *reinterpret_cast<const float4*>(qW + 8 * s * EA + e);
#pragma unroll
                for (int k = 0; k < GW; ++k)
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        cmac_conj(gacc[k][s][0], gacc[k][s][1], av[k].x, av[k].y, wv[s].x, wv[s].y);
                        cmac_conj(gacc[k][s][0], gacc[k][s][1], av[k].z, av[k].w, wv[s].z, wv[s].w);
                    }
            }
        }
        __syncthreads();  // every thread is done with stage st and sW
        if (tid == 0 && j + S < ntile) {
            fence_proxy_async_smem();
            issue(j + S);
        }
        if (with_grad && (j % C::FLUSH) == C::FLUSH - 1) flush_g();
    }
    if (timeout_at >= 0) {
        // a stage never completed: flag the error, then wait (bounded) for the copies still in
        // flight (tiles timeout_at .. timeout_at + S - 1) so that none lands after the block exits
        if (tid == 0) {
            atomicOr(status, 2);
            sBad[PB] = 1;
            for (int64_t jj = timeout_at; jj < ntile && jj < timeout_at + S; ++jj)
                mbar_wait_bounded(&mbar[jj % S], (uint32_t)((jj / S) & 1), 100000000ull);
        }
        __syncthreads();
    }
    if (with_grad) flush_g();
    // ln I: reduce the 16 GEMM1 event groups (lanes te = 0..15 of a half warp) per start
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        ff v = lsum[s];
#pragma unroll
        for (int m = 8; m > 0; m >>= 1) v = ff_add(v, ff_shfl_xor(v, m));
        if (te == 0) sL[2 * tp + (s & 1) + 32 * (s >> 1)] = v;
    }
    __syncthreads();
    const int np = (P - p0) < PB ? (P - p0) : PB;
    const int NVu = with_grad ? NV : 1;
    for (int idx = tid; idx < np * NVu; idx += PWA_THREADS) {
        const int p = idx / NVu, v = idx % NVu;
        float2 out;
        if (v == 0) {
            out = make_float2(sL[p].hi, sL[p].lo);
        } else {
            const float4 gv = sG[p * KMAX + ((v - 1) >> 1)];
            out = ((v - 1) & 1) ? make_float2(gv.z, gv.w) : make_float2(gv.x, gv.y);
        }
        part[((int64_t)blockIdx.x * P + p0 + p) * NV + v] = out;
    }
    for (int p = tid; p < np; p += PWA_THREADS)
        if (sBad[p] || sBad[PB]) bad[p0 + p] = 1;
}

// Per parameter set: sum the chunk partials in chunk order, add the FP64 normalisation term.
__global__ void __launch_bounds__(PWA_THREADS) k_nll_finalize(
    const float2* __restrict__ part, int nchunk, int K, int P, const float2* __restrict__ V,
    const double2* __restrict__ Psi, double nfac, int* __restrict__ bad, int* __restrict__ status,
    double* __restrict__ nll, double* __restrict__ grad, int with_grad) {
    __shared__ double sval[1 + 2 * PWA_MAX_WAVES];
    __shared__ double2 sT[PWA_MAX_WAVES];
    __shared__ float2 sVf[PWA_MAX_WAVES];
    __shared__ double2 scratch[PWA_THREADS];
    __shared__ double sS;
    const int p = blockIdx.x, tid = threadIdx.x;
    const int NV = 1 + 2 * K;
    const int NVu = with_grad ? NV : 1;
    if (tid < K) sVf[tid] = V[(int64_t)p * K + tid];
    if (tid < NVu) sval[tid] = ff_to_double(ff_sum_strided(part, (int64_t)p * NV + tid, (int64_t)P * NV, nchunk));
    __syncthreads();
    const double S = psi_times_v<PWA_THREADS>(Psi, sVf, K, sT, scratch, &sS);
    const bool isbad = bad[p] != 0;
    if (tid == 0) {
        nll[p] = isbad ? INFINITY : (-sval[0] + nfac * S);
        if (isbad) atomicOr(status, 1);
    }
    if (with_grad && tid < K) {
        grad[(int64_t)p * 2 * K + 2 * tid] = isbad ? 0.0 : (-2.0 * sval[1 + 2 * tid] + 2.0 * nfac * sT[tid].x);
        grad[(int64_t)p * 2 * K + 2 * tid + 1] = isbad ? 0.0 : (-2.0 * sval[2 + 2 * tid] + 2.0 * nfac * sT[tid].y);
    }
    __syncthreads();
    if (tid == 0) bad[p] = 0;
}

// ----------------------------------------------------------------------- launch helpers
int kmax_stream(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64; }
int kmax_batched(int K) { return K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64; }

template <int KMAX, bool GRAD, bool HOLD, bool FUSED>
int stream_occupancy() {
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_nll_stream<KMAX, GRAD, HOLD, FUSED>, PWA_THREADS, 0);
        occ = o > 0 ? o : 1;
    }
    return occ;
}

int64_t stream_grid(int64_t n, int sm_count, int occ) {
    const int64_t npairs = (n + 1) / 2;
    int64_t g = (npairs + PWA_THREADS - 1) / PWA_THREADS;
    int64_t cap = (int64_t)sm_count * occ;
    // PWA_STREAM_GRID: blocks per launch (tuning), at most the workspace bound of 8 per SM
    const char* e = getenv("PWA_STREAM_GRID");
    if (e && atoi(e) > 0) cap = atoi(e) < 8 * sm_count ? atoi(e) : 8 * sm_count;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return g;
}

// Register-holding variant by default for K <= 32; PWA_STREAM_HOLD=0/1 overrides (tuning).
inline int stream_hold_override() {
    const char* e = getenv("PWA_STREAM_HOLD");
    return e ? atoi(e) : -1;
}

// Fused (last block finalises, one launch) or split (streaming kernel + one-block finalise);
// PWA_STREAM_FUSED=0/1 overrides the default (tuning).
inline int stream_fused_override() {
    const char* e = getenv("PWA_STREAM_FUSED");
    return e ? atoi(e) : -1;
}

template <int KMAX, bool GRAD, bool HOLD, bool FUSED>
cudaError_t stream_launch_v(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                            double nfac, double* nll, double* grad, void* ws, size_t ws_bytes, unsigned* counter,
                            int* badw, int* status, int sm_count, cudaStream_t st) {
    const int64_t g = stream_grid(KMAX <= 16 ? n : 2 * n, sm_count, stream_occupancy<KMAX, GRAD, HOLD, FUSED>());
    if ((size_t)g * (1 + 2 * (size_t)K) * sizeof(float2) > ws_bytes) return cudaErrorInvalidValue;
    k_nll_stream<KMAX, GRAD, HOLD, FUSED><<<(unsigned)g, PWA_THREADS, 0, st>>>(A, K, n, ld, V, Psi, nfac, (float2*)ws,
                                                                              counter, badw, status, nll, grad);
    if (FUSED) return cudaGetLastError();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nll_stream_final<KMAX, GRAD><<<1, PWA_THREADS, 0, st>>>((const float2*)ws, (int)g, K, V, Psi, nfac, badw, status,
                                                               nll, grad);
    return cudaGetLastError();
}

inline int stream_tma_override() {
    const char* e = getenv("PWA_STREAM_TMA");
    return e ? atoi(e) : -1;
}

template <int KMAX, bool GRAD>
cudaError_t tma_launch(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                       double nfac, double* nll, double* grad, void* ws, size_t ws_bytes, unsigned* counter,
                       int* badw, int* status, int sm_count, cudaStream_t st) {
    using C = TmaCfg<KMAX>;
    auto kern = k_nll_tma<KMAX, GRAD>;
    static int occ = -1;
    if (occ < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, C::E, C::SMEM);
        occ = o > 0 ? o : 1;
    }
    const int64_t ntile = (n + C::E - 1) / C::E;
    int64_t g = (int64_t)sm_count * occ;
    if (g > (int64_t)sm_count * 8) g = (int64_t)sm_count * 8;  // workspace bound
    const char* e = getenv("PWA_STREAM_GRID");
    if (e && atoi(e) > 0 && atoi(e) < g) g = atoi(e);
    if (g > ntile) g = ntile;
    if (g < 1) g = 1;
    if ((size_t)g * (1 + 2 * (size_t)K) * sizeof(float2) > ws_bytes) return cudaErrorInvalidValue;
    kern<<<(unsigned)g, C::E, C::SMEM, st>>>(A, K, n, ld, V, Psi, nfac, (float2*)ws, counter, badw, status, nll, grad);
    return cudaGetLastError();
}

template <int KMAX, bool GRAD>
cudaError_t stream_launch(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                          double nfac, double* nll, double* grad, void* ws, size_t ws_bytes, unsigned* counter,
                          int* badw, int* status, int sm_count, cudaStream_t st) {
    // The bulk-copy variant is the default for 16 < K <= 32 (measured: K=32, 1e6 events 59.9
    // against 79.8 us; slower for K <= 16, where two events per 16-byte load keep enough bytes in
    // flight); PWA_STREAM_TMA=0/1 overrides, and an explicit HOLD or FUSED override selects the
    // register kernel.
    const int to = stream_tma_override();
    const bool tma = to == 1 || (to < 0 && KMAX == 32 && stream_hold_override() < 0 && stream_fused_override() < 0);
    if (tma)
        return tma_launch<KMAX, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status,
                                      sm_count, st);
    const int ov = stream_hold_override();
    const bool hold = ov >= 0 ? ov != 0 : KMAX <= 32;
    const int fo = stream_fused_override();
    const bool fused = fo >= 0 ? fo != 0 : true;
#define PWA_SL(H, F) stream_launch_v<KMAX, GRAD, H, F>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, \
                                                       badw, status, sm_count, st)
    if (hold) return fused ? PWA_SL(true, true) : PWA_SL(true, false);
    return fused ? PWA_SL(false, true) : PWA_SL(false, false);
#undef PWA_SL
}

template <bool GRAD>
cudaError_t stream_dispatch(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                            double nfac, double* nll, double* grad, void* ws, size_t ws_bytes, unsigned* counter,
                            int* badw, int* status, int sm_count, cudaStream_t st) {
    switch (kmax_stream(K)) {
        case 4: return stream_launch<4, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        case 8: return stream_launch<8, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        case 16: return stream_launch<16, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        case 32: return stream_launch<32, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        case 48: return stream_launch<48, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        default: return stream_launch<64, GRAD>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
    }
}

// batched tile shapes (E events x PB starts per block tile)
struct Shape {
    int E, PB;
};
// shapes 0-2: k_nll_batched<KMAX, E, PB>; shape 3: the pipelined k_nll_batched2 (K <= 32);
// shape 4: the tensor-core kernel k_nll_tc (3xTF32, K <= 32)
const Shape kShapes[] = {{64, 64}, {64, 32}, {128, 32}, {128, 64}, {64, 128}};
constexpr int kNumShapes = 5;
constexpr int kTensorShape = 4;

template <int KMAX, int E, int PB>
bool shape_feasible() {
    return BatchedCfg<KMAX, E, PB>::SMEM <= 113 * 1024;
}


template <int KMAX, int E, int PB>
cudaError_t batched_launch_shape(const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                                 size_t ws_bytes, int* bad, int with_grad, int sm_count, cudaStream_t st, int* nchunk_out) {
    using C = BatchedCfg<KMAX, E, PB>;
    auto kern = k_nll_batched<KMAX, E, PB>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        attr = true;
    }
    int nchunk;
    int64_t epc;
    batched_geometry(n, P, PB, E, sm_count, &nchunk, &epc);
    if ((size_t)nchunk * (size_t)P * (1 + 2 * (size_t)K) * sizeof(float2) > ws_bytes) return cudaErrorInvalidValue;
    dim3 grid(nchunk, (P + PB - 1) / PB);
    kern<<<grid, PWA_THREADS, C::SMEM, st>>>(A, K, n, ld, V, P, epc, (float2*)ws, bad, with_grad);
    *nchunk_out = nchunk;
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t batched2_launch(const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                            size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count, cudaStream_t st,
                            int* nchunk_out) {
    if constexpr (KMAX <= 32 && KMAX % 8 == 0) {
        using C = Batched2Cfg<KMAX>;
        auto kern = k_nll_batched2<KMAX>;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            attr = true;
        }
        int nchunk;
        int64_t epc;
        batched_geometry(n, P, C::PB, C::E, sm_count, &nchunk, &epc, 1);
        if ((size_t)nchunk * (size_t)P * (1 + 2 * (size_t)K) * sizeof(float2) > ws_bytes) return cudaErrorInvalidValue;
        dim3 grid(nchunk, (P + C::PB - 1) / C::PB);
        kern<<<grid, PWA_THREADS, C::SMEM, st>>>(A, K, n, ld, V, P, epc, (float2*)ws, bad, with_grad, status);
        *nchunk_out = nchunk;
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int KMAX>
cudaError_t batched_launch(int shape, const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                           size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count, cudaStream_t st,
                           int* nchunk) {
    switch (shape) {
        case 0: return batched_launch_shape<KMAX, 64, 64>(A, K, n, ld, V, P, ws, ws_bytes, bad, with_grad, sm_count, st, nchunk);
        case 1: return batched_launch_shape<KMAX, 64, 32>(A, K, n, ld, V, P, ws, ws_bytes, bad, with_grad, sm_count, st, nchunk);
        case 2: return batched_launch_shape<KMAX, 128, 32>(A, K, n, ld, V, P, ws, ws_bytes, bad, with_grad, sm_count, st, nchunk);
        case 3: return batched2_launch<KMAX>(A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk);
        default: return tc_batched_launch(KMAX, A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk);
    }
}

template <int KMAX>
bool batched_shape_ok(int shape) {
    switch (shape) {
        case 0: return shape_feasible<KMAX, 64, 64>();
        case 1: return shape_feasible<KMAX, 64, 32>();
        case 2: return shape_feasible<KMAX, 128, 32>();
        case 3: return KMAX <= 32 && KMAX % 8 == 0;
        default: return tc_batched_ok(KMAX);
    }
}

bool shape_ok(int kmax, int shape) {
    switch (kmax) {
        case 8: return batched_shape_ok<8>(shape);
        case 16: return batched_shape_ok<16>(shape);
        case 32: return batched_shape_ok<32>(shape);
        case 48: return batched_shape_ok<48>(shape);
        default: return batched_shape_ok<64>(shape);
    }
}

cudaError_t batched_dispatch(int shape, const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P,
                             void* ws, size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count,
                             cudaStream_t st, int* nchunk) {
#define PWA_BD(KM) batched_launch<KM>(shape, A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk)
    switch (kmax_batched(K)) {
        case 8: return PWA_BD(8);
        case 16: return PWA_BD(16);
        case 32: return PWA_BD(32);
        case 48: return PWA_BD(48);
        default: return PWA_BD(64);
    }
#undef PWA_BD
}

// ---- autotuner: per (KMAX, P bucket, n bucket) time every feasible shape once, keep the fastest
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;

int bucket_log2(int64_t x) {
    int b = 0;
    while (x > 1) { x >>= 1; ++b; }
    return b;
}

int tuned_shape(int K, int64_t n, int P) {
    const int kmax = kmax_batched(K);
    const char* env = getenv("PWA_BATCHED_SHAPE");
    if (env) {
        int s = atoi(env);
        if (s >= 0 && s < kNumShapes && shape_ok(kmax, s)) return s;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(kmax, bucket_log2(P), bucket_log2(n), 0));
    return it != g_tuned.end() ? it->second : -1;
}

// precise: the fastest of the FP32 SIMT shapes (0-3), whose gradient error at a minimum is ~20x
// below the tensor-core shape's; the fitter resumes starts whose line search stalled on the
// tensor-core shape's rounding with it.
int choose_shape(int K, int64_t n, int P, const float2* A, int64_t ld, const float2* V, void* ws, size_t ws_bytes, int* bad,
                 int* status, int with_grad, int sm_count, cudaStream_t st, bool precise) {
    const int kmax = kmax_batched(K);
    const char* env = getenv("PWA_BATCHED_SHAPE");
    if (env) {
        int s = atoi(env);
        if (s >= 0 && s < kNumShapes && shape_ok(kmax, s) && !(precise && s == kTensorShape)) return s;
    }
    const auto key = std::make_tuple(kmax, bucket_log2(P), bucket_log2(n), precise ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    int fallback = shape_ok(kmax, 0) ? 0 : 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    const char* tune = getenv("PWA_TUNE");
    if (cs != cudaStreamCaptureStatusNone || (tune && tune[0] == '0') || n < 4096) return fallback;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = fallback, best_p = fallback;
    float best_ms = 1e30f, best_p_ms = 1e30f;
    for (int s = 0; s < kNumShapes; ++s) {
        if (!shape_ok(kmax, s)) continue;
        int nc;
        float tot = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, st);
            ok = batched_dispatch(s, A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, &nc) ==
                 cudaSuccess;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;  // first launch is a warm-up
        }
        if (ok && tot < best_ms) {
            best_ms = tot;
            best = s;
        }
        if (ok && s != kTensorShape && tot < best_p_ms) {
            best_p_ms = tot;
            best_p = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // clear the non-finite flags the trial launches may have set
    cudaMemsetAsync(bad, 0, sizeof(int) * (size_t)P, st);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(kmax, bucket_log2(P), bucket_log2(n), 0)] = best;
    g_tuned[std::make_tuple(kmax, bucket_log2(P), bucket_log2(n), 1)] = best_p;
    return precise ? best_p : best;
}

// One parameter set with caller-provided scratch and a cap on the number of blocks (used by
// the allocation-free entry point): the fused streaming kernel, register-holding variant.
template <int KMAX>
cudaError_t stream_launch_capped(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                                 double nfac, double* nll, double* grad, float2* part, size_t part_bytes,
                                 unsigned* counter, int* badw, int* status, int max_blocks, int sm_count,
                                 cudaStream_t st) {
    constexpr bool HOLD = KMAX <= 32;
    int64_t g = stream_grid(KMAX <= 16 ? n : 2 * n, sm_count, stream_occupancy<KMAX, true, HOLD, true>());
    if (g > max_blocks) g = max_blocks;
    if ((size_t)g * (1 + 2 * (size_t)K) * sizeof(float2) > part_bytes) return cudaErrorInvalidValue;
    k_nll_stream<KMAX, true, HOLD, true><<<(unsigned)g, PWA_THREADS, 0, st>>>(A, K, n, ld, V, Psi, nfac, part, counter,
                                                                             badw, status, nll, grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_nll_grad_scratch(const float2* A, int K, int64_t n, int64_t ld, const float2* V,
                                    const double2* Psi, double nfac, double* nll, double* grad, float2* part,
                                    size_t part_bytes, unsigned* counter, int* badw, int* status, int max_blocks,
                                    int sm_count, cudaStream_t st) {
#define PWA_SC(KM) stream_launch_capped<KM>(A, K, n, ld, V, Psi, nfac, nll, grad, part, part_bytes, counter, badw, \
                                            status, max_blocks, sm_count, st)
    switch (kmax_stream(K)) {
        case 4: return PWA_SC(4);
        case 8: return PWA_SC(8);
        case 16: return PWA_SC(16);
        case 32: return PWA_SC(32);
        case 48: return PWA_SC(48);
        default: return PWA_SC(64);
    }
#undef PWA_SC
}

int batched_shape(int K, int64_t n, int P) { return tuned_shape(K, n, P); }

size_t nll_workspace(int K, int64_t n, int P, int sm_count) {
    const size_t NV = 1 + 2 * (size_t)K;
    if (P == 1) return sizeof(float2) * NV * (size_t)sm_count * 8;
    // batched: the most chunks of all shapes, the SIMT ones (at most those of (E = 64, PB = 64),
    // two blocks per SM) and the tensor-core one (E = 48, PB = 128, one block per SM)
    int nchunk, nchunk_tc;
    int64_t epc;
    batched_geometry(n, P, 64, 64, sm_count, &nchunk, &epc);
    batched_geometry(n, P, 128, 48, sm_count, &nchunk_tc, &epc, 1);
    if (nchunk_tc > nchunk) nchunk = nchunk_tc;
    return sizeof(float2) * NV * (size_t)P * (size_t)nchunk;
}

cudaError_t launch_nll(const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P,
                       const double2* Psi, double nfac, double* nll, double* grad, void* ws, size_t ws_bytes,
                       unsigned* counter, int* bad, int* status, int sm_count, cudaStream_t st, bool precise) {
    if (P == 1) {
        // counter[0]: completion ticket, counter[1]: non-finite flag of this evaluation
        int* badw = reinterpret_cast<int*>(counter + 1);
        if (grad)
            return stream_dispatch<true>(A, K, n, ld, V, Psi, nfac, nll, grad, ws, ws_bytes, counter, badw, status, sm_count, st);
        return stream_dispatch<false>(A, K, n, ld, V, Psi, nfac, nll, nullptr, ws, ws_bytes, counter, badw, status, sm_count, st);
    }
    const int with_grad = grad != nullptr;
    const int shape = choose_shape(K, n, P, A, ld, V, ws, ws_bytes, bad, status, with_grad, sm_count, st, precise);
    int nchunk = 1;
    cudaError_t e = batched_dispatch(shape, A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st,
                                     &nchunk);
    if (e != cudaSuccess) return e;
    k_nll_finalize<<<P, PWA_THREADS, 0, st>>>((const float2*)ws, nchunk, K, P, V, Psi, nfac, bad, status, nll, grad,
                                              with_grad);
    return cudaGetLastError();
}

}  // namespace pwa
