// Block and grid reduction + finalisation shared by the one-parameter-set likelihood kernels.
//
// Each thread brings FP32 gradient partials g[2K] (sum_i conj(A_c(i)) u_i / I_i, re/im) and a
// double-single partial of sum_i ln I_i.  The warp combines the gradient partials by a
// reduce-scatter (31 shuffles for 32 values).  From there on every sum is exact: each value is
// converted to fixed point (two tiers of three signed 42-bit limbs, below) and the limbs are
// added as 64-bit integers.  Integer addition is exact and associative, so the result does not
// depend on the order in which warps and blocks arrive.
//
// The warps park their sums in shared memory; after one block barrier thread v adds the warps'
// limbs of value v in registers and adds them to the grid words (global integer atomics); the
// grid's last block (completion counter) reads 6 (2K + 2) words and writes the results of
// Eq. 3 (extended form):
//   f = -sum ln I + n_f S,  S = sum_ab V_a conj(V_b) Psi_ab,
//   g_c = -2 sum_i conj(A_c(i)) u_i / I_i + 2 n_f t_c,  t_c = sum_a Psi_ac V_a.
// t_c and Re(conj(V_c) t_c) are computed by warp 0 of the K blocks with the fewest events (Psi
// prefetched to L2 at their start), one column each; the products go into S's fixed-point
// words, so the last block does no FP64 reduction (GB300 runs FP64 with a latency of ~64
// cycles per dependent operation and ~2 operations per cycle per SM).
#pragma once

#include "pwa_internal.cuh"

namespace pwa {

// ---------------------------------------------------------------- fixed-point grid sums ----
// A finite float x is m 2^(e - 150) (m a 24-bit integer, e the biased exponent; subnormals
// m 2^-149).  Tier 0 holds X0 = trunc(|x| 2^64) for |x| < 2^61 (bits below 2^-64 dropped);
// tier 1 holds X1 = |x| 2^-37 for |x| >= 2^61, an integer since such floats are multiples of
// 2^38.  Each tier is three limbs, X = L0 + L1 2^42 + L2 2^84 (X < 2^125), so every limb of a
// single float is below 2^42 and 2^21 of them add up without overflow.  The value of the
// words is sum(X0) 2^-64 + sum(X1) 2^37.
constexpr int FIX_LIMB_BITS = 42;
constexpr unsigned long long FIX_LIMB_MASK = (1ull << FIX_LIMB_BITS) - 1ull;

// Adds the limbs of f to L[0..5] (L[3 t + k] = limb k of tier t).  False (nothing added) if f
// is not finite.
__device__ __forceinline__ bool fix_add(float f, long long (&L)[FIX_WORDS]) {
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 255) return false;
    unsigned long long m = u & 0x7fffffu;
    int sh;
    if (e == 0) {
        sh = -85;
    } else {
        m |= 0x800000u;
        sh = e - 86;
    }
    const int tier = sh > 101 ? 1 : 0;
    if (tier) sh = e - 187;
    const bool neg = (u >> 31) != 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = sh - FIX_LIMB_BITS * k;
        unsigned long long p = 0ull;
        if (s >= 0) {
            if (s < 64) p = (m << s) & FIX_LIMB_MASK;
        } else if (-s < 64) {
            p = (m >> -s) & FIX_LIMB_MASK;
        }
        const long long v = neg ? -(long long)p : (long long)p;
        if (tier) L[3 + k] += v;
        else L[k] += v;
    }
    return true;
}

// The same limbs for a double x = m 2^(e - 1075) (53-bit m): tier 0 for |x| < 2^61, else tier 1
// (trunc(|x| 2^-37): doubles of that size may have bits below 2^37, which are dropped).
// False (nothing added) if x is not finite or |x| >= 2^125.
__device__ __forceinline__ bool fix_add_double(double x, long long (&L)[FIX_WORDS]) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ffull);
    if (e == 2047) return false;
    unsigned long long m = u & ((1ull << 52) - 1ull);
    int sh;
    if (e == 0) {
        sh = 1 - 1011;
    } else {
        m |= 1ull << 52;
        sh = e - 1011;
    }
    int tier = 0;
    if (sh + 53 > 125) {
        tier = 1;
        sh = e - 1112;
        if (sh + 53 > 125) return false;
    }
    const bool neg = (u >> 63) != 0ull;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = sh - FIX_LIMB_BITS * k;
        unsigned long long p = 0ull;
        if (s >= 0) {
            if (s < 64) p = (m << s) & FIX_LIMB_MASK;
        } else if (-s < 64) {
            p = (m >> -s) & FIX_LIMB_MASK;
        }
        const long long v = neg ? -(long long)p : (long long)p;
        if (tier) L[3 + k] += v;
        else L[k] += v;
    }
    return true;
}

// X 2^-64 for X = T0 + T1 2^42 + T2 2^84.  Carries are normalised in integers (r0, r1 in
// [0, 2^42)); then X = (T2 2^20 + m) 2^64 + l with m = r1 >> 22 and l = (r1 mod 2^22) 2^42 + r0
// a 64-bit word, so X 2^-64 = (T2 2^20 + m) + l 2^-64: three conversions and two FMAs.
__device__ __forceinline__ double fix_tier_value(long long T0, long long T1, long long T2) {
    const long long r0 = T0 & (long long)FIX_LIMB_MASK;
    T1 += (T0 - r0) >> FIX_LIMB_BITS;  // exact: T0 - r0 is a multiple of 2^42
    const long long r1 = T1 & (long long)FIX_LIMB_MASK;
    T2 += (T1 - r1) >> FIX_LIMB_BITS;
    const unsigned long long l = ((unsigned long long)(r1 & ((1ll << 22) - 1)) << FIX_LIMB_BITS) |
                                 (unsigned long long)r0;
    const double top = fma((double)T2, 1048576.0, (double)(int)(r1 >> 22));
    return fma((double)l, 0x1p-64, top);
}

__device__ __forceinline__ double fix_to_double(const long long (&T)[FIX_WORDS]) {
    double v = fix_tier_value(T[0], T[1], T[2]);
    if ((T[3] | T[4] | T[5]) != 0) v += fix_tier_value(T[3], T[4], T[5]) * 0x1p101;
    return v;
}

template <int KMAX, int NTHR>
struct StreamReduceSmem {
    static constexpr int NG = 2 * KMAX;
    static constexpr int ROUNDS = (NG + 31) / 32;
    static constexpr int NW = NTHR / 32;
    float sred[NW][ROUNDS * 32];  // warp sums of the gradient partials
    ff slred[NW];                 // unfused variant: warp sums of ln I
    long long slw[NW][3];         // fused variant: warp sums of ln I as tier-0 limbs
    int sLast;
    int sFlags;
    double sval[2 + NG];
};

// Called by every thread of the block before the event loop: on the blocks that will compute
// normalisation-term columns, prefetches Psi into L2.
template <int KMAX, int NTHR>
__device__ __forceinline__ void stream_reduce_init(StreamReduceSmem<KMAX, NTHR>& sm, const double2* __restrict__ Psi,
                                                   int K) {
    const int c0 = (int)gridDim.x - 1 - (int)blockIdx.x;
    if (c0 < K) {
        const char* base = reinterpret_cast<const char*>(Psi);
        const int lines = (K * K * 16 + 127) / 128;
        for (int l = threadIdx.x; l < lines; l += NTHR) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + 128 * l));
    }
}

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

// Normalisation-term columns for the fused kernels, by one warp: t_c = sum_a Psi_ac V_a (lane l
// sums a = l and a = l + 32, then an xor-shuffle tree) for the columns c = c0, c0 + G, ... < K
// (c0 = G - 1 - block: in both stream kernels the highest-index blocks have the fewest events),
// written to the control words; Re(conj(V_c) t_c) is added to S's fixed-point words.  Returns
// false if a product was not finite.
__device__ __forceinline__ bool psi_columns_warp(const double2* __restrict__ Psi, const float2* sV, int K,
                                                 unsigned* __restrict__ counter) {
    const int G = (int)gridDim.x, lane = threadIdx.x & 31;
    bool ok = true;
    double2* tout = stream_psi_t(counter);
    long long* sw = stream_limbs(counter) + STREAM_NV_MAX * FIX_WORDS;
    for (int c = G - 1 - (int)blockIdx.x; c < K; c += G) {
        double tr = 0.0, ti = 0.0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int a = lane + 32 * h;
            if (a < K) {
                const double2 p = __ldg(Psi + a * K + c);
                const double vr = sV[a].x, vi = sV[a].y;
                tr += p.x * vr - p.y * vi;
                ti += p.x * vi + p.y * vr;
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            tr += __shfl_xor_sync(0xffffffffu, tr, m);
            ti += __shfl_xor_sync(0xffffffffu, ti, m);
        }
        if (lane == 0) {
            tout[c] = make_double2(tr, ti);
            long long L[FIX_WORDS] = {0, 0, 0, 0, 0, 0};
            ok = fix_add_double((double)sV[c].x * tr + (double)sV[c].y * ti, L) && ok;
#pragma unroll
            for (int k = 0; k < FIX_WORDS; ++k)
                if (L[k] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(sw + k), (unsigned long long)L[k]);
        }
    }
    return ok;
}

// Returns after the block's contribution is added; the grid's last block also writes nll (and
// grad).  FUSED: exact fixed-point sums (stream_reduce_init must have run; counter points at
// the launch's control words, badw at its flag word).  Unfused: the block writes double-single
// partials part[block][1 + 2K] for the one-block finalise kernel.
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
    const int NV = 1 + 2 * K;
    const int NVu = GRAD ? NV : 1;
    if (!FUSED) {
        if (GRAD) {
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                float x[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) x[j] = (32 * r + j < NG) ? g[32 * r + j] : 0.f;
                warp_transpose_reduce32(x);
                sm.sred[warp][32 * r + lane] = x[0];
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) lacc = ff_add(lacc, ff_shfl_xor(lacc, m));
        if (lane == 0) sm.slred[warp] = lacc;
        const int any_bad = __syncthreads_or(bad ? 1 : 0);
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
        if (any_bad && tid == 0) atomicOr(badw, STREAM_FLAG_NONFINITE);
        return;
    }

    // ---- warp: ln I as tier-0 limbs (|ln I| < 104 for any positive finite float I, so a
    // thread partial never reaches 2^61; a tier-1 word is flagged), an exact integer shuffle
    // reduction; the gradient by a reduce-scatter.  Both parked in shared memory.
    {
        long long L[FIX_WORDS] = {0, 0, 0, 0, 0, 0};
        const bool ok = fix_add(lacc.hi, L) && fix_add(lacc.lo, L);
        if (!ok || (L[3] | L[4] | L[5]) != 0) bad = true;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) L[k] += __shfl_xor_sync(0xffffffffu, L[k], m);
        if (lane == 0) {
            sm.slw[warp][0] = L[0];
            sm.slw[warp][1] = L[1];
            sm.slw[warp][2] = L[2];
        }
    }
    if (GRAD) {
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            float x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = (32 * r + j < NG) ? g[32 * r + j] : 0.f;
            warp_transpose_reduce32(x);
            sm.sred[warp][32 * r + lane] = x[0];
        }
    }
    if (warp == 0 && !psi_columns_warp(Psi, sV, K, counter)) bad = true;
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    // ---- block words of value v (0: ln I, 1 + j: gradient component j) by thread v: the
    // warps' limbs added in registers, then to the grid words
    long long* limbs = stream_limbs(counter);
    for (int v = tid; v < NVu; v += NTHR) {
        long long T[FIX_WORDS] = {0, 0, 0, 0, 0, 0};
        bool ok = true;
        if (v == 0) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                T[0] += sm.slw[w][0];
                T[1] += sm.slw[w][1];
                T[2] += sm.slw[w][2];
            }
        } else {
#pragma unroll
            for (int w = 0; w < NW; ++w) ok = fix_add(sm.sred[w][v - 1], T) && ok;
        }
        if (!ok) atomicOr(badw, STREAM_FLAG_NONFINITE);
#pragma unroll
        for (int k = 0; k < FIX_WORDS; ++k)
            if (T[k] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(limbs + v * FIX_WORDS + k), (unsigned long long)T[k]);
    }
    if (any_bad && tid == 0) atomicOr(badw, STREAM_FLAG_NONFINITE);
    __syncthreads();
    // release: the barrier orders every thread's atomics before thread 0's fence and ticket
    if (tid == 0) {
        __threadfence();
        const bool last = atomicAdd(counter, 1u) == gridDim.x - 1;
        if (last) {
            __threadfence();  // acquire: every block's words and the Psi columns
            sm.sFlags = __ldcg(badw);
        }
        sm.sLast = last;
    }
    __syncthreads();
    if (!sm.sLast) return;

    // ---- last block: read (and clear) the words of every value and of S (value NVu here)
    for (int v = tid; v <= NVu; v += NTHR) {
        long long* wv = limbs + (v < NVu ? v : STREAM_NV_MAX) * FIX_WORDS;
        long long T[FIX_WORDS];
#pragma unroll
        for (int k = 0; k < FIX_WORDS; ++k) T[k] = __ldcg(wv + k);
#pragma unroll
        for (int k = 0; k < FIX_WORDS; ++k) wv[k] = 0;
        sm.sval[v] = fix_to_double(T);
    }
    __syncthreads();
    const bool isbad = (sm.sFlags & STREAM_FLAG_NONFINITE) != 0;
    if (tid == 0) {
        nll[0] = isbad ? INFINITY : fma(nfac, sm.sval[NVu], -sm.sval[0]);
        if (isbad) atomicOr(status, 1);
        *badw = 0;
        *counter = 0u;
    }
    if (GRAD) {
        const double2* tin = stream_psi_t(counter);
        for (int c = tid; c < K; c += NTHR) {
            const double2 t = __ldcg(tin + c);
            grad[2 * c] = isbad ? 0.0 : 2.0 * fma(nfac, t.x, -sm.sval[1 + 2 * c]);
            grad[2 * c + 1] = isbad ? 0.0 : 2.0 * fma(nfac, t.y, -sm.sval[2 + 2 * c]);
        }
    }
}

}  // namespace pwa
