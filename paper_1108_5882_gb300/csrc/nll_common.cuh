// Block and grid reduction + finalisation shared by the one-parameter-set likelihood kernels.
//
// Each thread brings FP32 gradient partials g[2K] (sum_i conj(A_c(i)) u_i / I_i, re/im) and a
// double-single partial of sum_i ln I_i.  The warp combines the gradient partials by a
// reduce-scatter (31 shuffles for 32 values), the block sums its warps in a fixed order into a
// double-single partial per value, and the last block to arrive (completion counter) sums the
// block partials in block order and adds the FP64 normalisation term of Eq. 3 (extended form):
//   f = -sum ln I + n_f S,  S = sum_ab V_a conj(V_b) Psi_ab,
//   g_c = -2 sum_i conj(A_c(i)) u_i / I_i + 2 n_f sum_a Psi_ac V_a.
#pragma once

#include "pwa_internal.cuh"

namespace pwa {

template <int KMAX, int NTHR>
struct StreamReduceSmem {
    static constexpr int NG = 2 * KMAX;
    static constexpr int ROUNDS = (NG + 31) / 32;
    static constexpr int NW = NTHR / 32;
    float sred[NW][ROUNDS * 32];
    ff slred[NW];
    int sLast;
    ff sfin[NTHR > 1 + NG ? NTHR : 1 + NG];
    double sval[1 + NG];
    double2 sT[KMAX];
    double2 scratch[NTHR];
    double S;
};

// t_c = sum_a Psi_ac V_a for c < K and S = sum_c conj(V_c) t_c (FP64).  Every thread of the
// block loads its share of Psi at once (one memory round trip), and both sums are fixed-order
// pairwise trees: GB300 executes FP64 with a long latency, so a sequential chain of K dependent
// additions would dominate the whole finalisation.  scratch must hold NTHR double2 (and the
// tree over c uses scratch again).  Call with the whole block; returns S in all threads.
template <int NTHR>
__device__ __forceinline__ double psi_times_v(const double2* __restrict__ Psi, const float2* sV, int K,
                                              double2* sT, double2* scratch, double* sS) {
    const int tid = threadIdx.x;
    int nparts = NTHR / K > 0 ? NTHR / K : 1;
    int np2 = 1;  // parts rounded down to a power of two for the tree
    while (np2 * 2 <= nparts) np2 *= 2;
    nparts = np2;
    if (tid < nparts * K) {
        const int c = tid % K, part = tid / K;
        double tr = 0.0, ti = 0.0;
#pragma unroll 4
        for (int a = part; a < K; a += nparts) {
            const double2 p = Psi[a * K + c];
            const double vr = sV[a].x, vi = sV[a].y;
            tr += p.x * vr - p.y * vi;
            ti += p.x * vi + p.y * vr;
        }
        scratch[tid] = make_double2(tr, ti);
    }
    __syncthreads();
    // pairwise tree over the parts: level h adds part p + h into part p (p < h)
    for (int hlf = nparts / 2; hlf > 0; hlf /= 2) {
        if (tid < hlf * K) {
            const double2 a = scratch[tid], b = scratch[tid + hlf * K];
            scratch[tid] = make_double2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
    }
    for (int c = tid; c < K; c += NTHR) sT[c] = scratch[c];
    __syncthreads();
    // S: products per c, then a pairwise tree over c (padded with zeros to a power of two)
    int kp = 1;
    while (kp < K) kp *= 2;
    for (int c = tid; c < kp; c += NTHR)
        scratch[c].x = c < K ? (double)sV[c].x * sT[c].x + (double)sV[c].y * sT[c].y : 0.0;
    __syncthreads();
    for (int hlf = kp / 2; hlf > 0; hlf /= 2) {
        for (int c = tid; c < hlf; c += NTHR) scratch[c].x += scratch[c + hlf].x;
        __syncthreads();
    }
    if (tid == 0) *sS = scratch[0].x;
    __syncthreads();
    return *sS;
}

// Returns after the block's partial is written; the last block also writes nll (and grad).
template <int KMAX, bool GRAD, bool FUSED, int NTHR>
__device__ __forceinline__ void stream_reduce_finalize(float (&g)[2 * KMAX], ff lacc, bool bad, const float2* sV,
                                                       StreamReduceSmem<KMAX, NTHR>& sm, int K,
                                                       const double2* __restrict__ Psi, double nfac,
                                                       float2* __restrict__ part, unsigned* __restrict__ counter,
                                                       int* __restrict__ badw, int* __restrict__ status,
                                                       double* __restrict__ nll, double* __restrict__ grad) {
    constexpr int NG = 2 * KMAX;
    constexpr int ROUNDS = (NG + 31) / 32;
    constexpr int NW = NTHR / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (GRAD) {
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (32 * r + j < NG) x[j] = g[32 * r + j];
                else x[j] = 0.f;
            }
            warp_transpose_reduce32(x);
            sm.sred[warp][32 * r + lane] = x[0];
        }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) lacc = ff_add(lacc, ff_shfl_xor(lacc, m));
    if (lane == 0) sm.slred[warp] = lacc;
    const int any_bad = __syncthreads_or(bad ? 1 : 0);

    const int NV = 1 + 2 * K;
    float2* bp = part + (int64_t)blockIdx.x * NV;
    if (tid == 0) {
        ff s = ff_zero();
        for (int w = 0; w < NW; ++w) s = ff_add(s, sm.slred[w]);
        bp[0] = make_float2(s.hi, s.lo);
    }
    if (GRAD && tid < 2 * K) {
        ff s = ff_zero();
        for (int w = 0; w < NW; ++w) s = ff_add_f(s, sm.sred[w][tid]);
        bp[1 + tid] = make_float2(s.hi, s.lo);
    }
    if (any_bad && tid == 0) atomicOr(badw, 1);
    if (!FUSED) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) sm.sLast = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!sm.sLast) return;

    __threadfence();
    const int NVu = GRAD ? NV : 1;
    const int nch = NTHR / NVu > 0 ? NTHR / NVu : 1;
    for (int vv = tid; vv < nch * NVu; vv += NTHR) {
        const int v = vv % NVu, ch = vv / NVu;
        const int cnt = ((int)gridDim.x - ch + nch - 1) / nch;
        sm.sfin[vv] = ff_sum_strided<32>(part, (int64_t)ch * NV + v, (int64_t)nch * NV, cnt);
    }
    __syncthreads();
    for (int v = tid; v < NVu; v += NTHR) {
        ff s = ff_zero();
        for (int ch = 0; ch < nch; ++ch) s = ff_add(s, sm.sfin[ch * NVu + v]);
        sm.sval[v] = ff_to_double(s);
    }
    if (tid == 0) sm.sLast = __ldcg(badw) != 0;
    const double S = psi_times_v<NTHR>(Psi, sV, K, sm.sT, sm.scratch, &sm.S);
    const bool isbad = sm.sLast != 0;
    if (tid == 0) {
        nll[0] = isbad ? INFINITY : (-sm.sval[0] + nfac * S);
        if (isbad) atomicOr(status, 1);
        *badw = 0;
        *counter = 0u;
    }
    if (GRAD)
        for (int c = tid; c < K; c += NTHR) {
            grad[2 * c] = isbad ? 0.0 : (-2.0 * sm.sval[1 + 2 * c] + 2.0 * nfac * sm.sT[c].x);
            grad[2 * c + 1] = isbad ? 0.0 : (-2.0 * sm.sval[2 + 2 * c] + 2.0 * nfac * sm.sT[c].y);
        }
}

}  // namespace pwa
