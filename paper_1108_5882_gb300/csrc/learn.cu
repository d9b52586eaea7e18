// Features of the learned start proposer: per mass bin, the event averages of the 25 real
// spherical harmonics Y_LM(theta, phi), L <= 4 (40 bins x 25 = 1000 features), of a data
// sample, and the same for toy samples drawn on the fly from many production-amplitude sets.
//
// Moments are accumulated as fixed-point integers (Y * 2^36 rounded to int64): integer addition
// is associative, so the sums do not depend on the order in which events, warps and blocks are
// added (the result is deterministic), and |Y| < 1 keeps 1e7 events far from int64 overflow.
// Each warp owns a private accumulator [n_bins][25] in shared memory.  The events a warp takes
// in one step are added one after the other: the event's lane broadcasts its 25 values by
// shuffles, lane k adds value k, so no two lanes touch the same word and no atomics are needed
// in the event loop (shared-memory 64-bit atomics serialise badly when lanes share a bin).  The
// block sums its warps' accumulators and adds them to the grid's with integer atomics.  Toy
// events are generated, tested and accumulated without ever being stored: each block owns a
// range of one toy's candidates.
//
// Per toy t, the number of candidates is chosen so that about N_target events are accepted:
// n_cand = N_target * C_t / S_t, with C_t the accept-reject envelope (the per-mass-interval bound
// of pwa_envelope, in FP64 on the device) and S_t = V_t^T Psi V_t* the mean intensity over the
// flat phase space (Psi from flat MC: the acceptance probability is S_t / C_t).
#include "gen_model.cuh"

namespace pwa {

namespace {

constexpr int LM = 25;                 // real Y_LM with L <= 4
constexpr float FIX_SCALE = 68719476736.f;  // 2^36
constexpr double FIX_INV = 1.0 / 68719476736.0;

// normalisation constants N_LM (sqrt(2) N_L|M| for M != 0) in shared memory, index L^2 + L + M
__device__ void ylm_norms(float* sN) {
    const int t = threadIdx.x;
    if (t < LM) {
        int L = 0;
        while ((L + 1) * (L + 1) <= t) ++L;
        const int M = t - L * L - L;
        const int am = M < 0 ? -M : M;
        double fr = 1.0;  // (L - |M|)! / (L + |M|)!
        for (int i = L - am + 1; i <= L + am; ++i) fr /= (double)i;
        double N = sqrt((2.0 * L + 1.0) / (4.0 * 3.14159265358979323846) * fr);
        if (M != 0) N *= sqrt(2.0);
        sN[t] = (float)N;
    }
}

// y[L^2 + L + M] = real Y_LM(theta, phi) for L <= 4 (associated Legendre functions with the
// Condon-Shortley phase, by the standard recurrences in L at fixed M)
__device__ __forceinline__ void ylm25(float ct, float ph, const float* sN, float (&y)[LM]) {
    const float s = sqrtf(fmaxf((1.f - ct) * (1.f + ct), 0.f));
    float P[5][5];  // P[L][M]
#pragma unroll
    for (int M = 0; M <= 4; ++M) {
        float pmm = 1.f;
#pragma unroll
        for (int i = 1; i <= M; ++i) pmm *= -(2.f * i - 1.f) * s;
        P[M][M] = pmm;
        if (M + 1 <= 4) P[M + 1][M] = ct * (2.f * M + 1.f) * pmm;
#pragma unroll
        for (int L = M + 2; L <= 4; ++L)
            P[L][M] = (ct * (2.f * L - 1.f) * P[L - 1][M] - (L + M - 1.f) * P[L - 2][M]) / (float)(L - M);
    }
    float s1, c1;
    sincosf(ph, &s1, &c1);
    float cm[5], sm[5];
    cm[0] = 1.f;
    sm[0] = 0.f;
#pragma unroll
    for (int M = 1; M <= 4; ++M) {
        cm[M] = cm[M - 1] * c1 - sm[M - 1] * s1;
        sm[M] = sm[M - 1] * c1 + cm[M - 1] * s1;
    }
#pragma unroll
    for (int L = 0; L <= 4; ++L) {
        y[L * L + L] = sN[L * L + L] * P[L][0];
#pragma unroll
        for (int M = 1; M <= L; ++M) {
            y[L * L + L + M] = sN[L * L + L + M] * P[L][M] * cm[M];
            y[L * L + L - M] = sN[L * L + L - M] * P[L][M] * sm[M];
        }
    }
}

__device__ __forceinline__ int mass_bin(float m, int n_bins, float m_lo, float inv_w) {
    const float dm = __fsub_rn(m, m_lo);
    int b = (int)floorf(__fmul_rn(dm, inv_w));
    return b < 0 ? 0 : (b >= n_bins ? n_bins - 1 : b);
}

// Adds the events of the lanes in `mask` to the warp's accumulator wacc [n_bins][25]: per event
// (in lane order) 25 shuffles from its lane, lane k adding component k.  Call with the whole warp.
__device__ __forceinline__ void warp_add_events(long long* wacc, unsigned mask, int b, const float (&y)[LM]) {
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int e = __ffs(mask) - 1;
        mask &= mask - 1;
        const int be = __shfl_sync(0xffffffffu, b, e);
        float mine = 0.f;
#pragma unroll
        for (int k = 0; k < LM; ++k) {
            const float v = __shfl_sync(0xffffffffu, y[k], e);
            if (lane == k) mine = v;
        }
        // one float -> int64 conversion per lane (GB300 runs 64-bit conversions on its narrow
        // FP64 pipe, so converting inside the loop above would cost 25 of them per event)
        if (lane < LM) wacc[be * LM + lane] += __float2ll_rn(mine * FIX_SCALE);
    }
}

// The warps' accumulators of the block summed and added to acc (integer atomics).
__device__ __forceinline__ void block_flush(const long long* swacc, int nf, unsigned long long* __restrict__ acc) {
    constexpr int NW = PWA_THREADS / 32;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += swacc[w * nf + i];
        if (t) atomicAdd(acc + i, (unsigned long long)t);
    }
}

// moments of given events: per-warp accumulators, flushed into acc [n_bins][25] (int64)
__global__ void __launch_bounds__(PWA_THREADS) k_moments(const float* __restrict__ kin, int64_t n, int64_t ld,
                                                         int n_bins, float m_lo, float inv_w,
                                                         unsigned long long* __restrict__ acc) {
    extern __shared__ long long swacc[];  // [PWA_THREADS / 32][n_bins * 25]
    __shared__ float sN[LM];
    const int nf = n_bins * LM, lane = threadIdx.x & 31;
    ylm_norms(sN);
    for (int i = threadIdx.x; i < (PWA_THREADS / 32) * nf; i += blockDim.x) swacc[i] = 0;
    __syncthreads();
    long long* wacc = swacc + (threadIdx.x >> 5) * nf;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop: the warp's first event decides, lanes past n idle
    for (int64_t iw = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); iw < n; iw += stride) {
        const int64_t i = iw + lane;
        const bool has = i < n;
        float y[LM];
        int b = 0;
        if (has) {
            ylm25(__ldg(kin + ld + i), __ldg(kin + 2 * ld + i), sN, y);
            b = mass_bin(__ldg(kin + i), n_bins, m_lo, inv_w);
        } else {
#pragma unroll
            for (int k = 0; k < LM; ++k) y[k] = 0.f;
        }
        warp_add_events(wacc, __ballot_sync(0xffffffffu, has), b, y);
    }
    __syncthreads();
    block_flush(swacc, nf, acc);
}

// feat = acc * 2^-36 / count (count from a device counter, or the given n)
__global__ void k_moments_final(const unsigned long long* __restrict__ acc, int nf, const long long* __restrict__ cnt,
                                long long n_fixed, double* __restrict__ feat, int T) {
    const int64_t total = (int64_t)T * nf;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / nf);
        const long long c = cnt ? cnt[t] : n_fixed;
        feat[i] = c > 0 ? (double)(long long)acc[i] * FIX_INV / (double)c : 0.0;
    }
}

struct ToyWaves {
    WaveTable wt;
    double M[PWA_MAX_WAVES], W[PWA_MAX_WAVES];
};

// per toy: envelope C_t (FP64, per-mass-interval bound) and candidates for ~N_target events
__global__ void k_toy_setup(ToyWaves tw, const float2* __restrict__ V, const double2* __restrict__ Psi, int T,
                            double n_target, double* __restrict__ C, long long* __restrict__ n_cand) {
    const int t = blockIdx.x;
    if (t >= T) return;
    const int K = tw.wt.K;
    const float2* Vt = V + (int64_t)t * K;
    __shared__ double red[PWA_THREADS];
    // envelope over 4096 equal intervals of [0.99, 3.0]: thread-strided intervals, max-reduce
    double best = 0.0;
    for (int k = threadIdx.x; k < 4096; k += blockDim.x) {
        const double a0 = 0.99 + 2.01 * k / 4096.0, a1 = 0.99 + 2.01 * (k + 1) / 4096.0;
        double s = 0.0;
        for (int a = 0; a < K; ++a) {
            const double M = tw.M[a], Wd = tw.W[a];
            const double mm = M < a0 ? a0 : (M > a1 ? a1 : M);
            const double d = M * M - mm * mm;
            s += hypot((double)Vt[a].x, (double)Vt[a].y) * (M * Wd / sqrt(d * d + M * M * Wd * Wd));
        }
        best = fmax(best, s * s);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double Ct = red[0];
        double S = 0.0;  // V^T Psi V* (real)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                const double2 p = Psi[a * K + b];
                const double vr = Vt[a].x * (double)Vt[b].x + Vt[a].y * (double)Vt[b].y;  // Re(V_a conj V_b)
                const double vi = Vt[a].y * (double)Vt[b].x - Vt[a].x * (double)Vt[b].y;  // Im(V_a conj V_b)
                S += vr * p.x - vi * p.y;
            }
        C[t] = Ct;
        n_cand[t] = (S > 0.0 && Ct > 0.0) ? (long long)ceil(n_target * Ct / S) : 0;
    }
}

// fused accept-reject + moments: grid (T, BPT); block b of toy t covers candidates
// [b * chunk, (b + 1) * chunk) of that toy's sequence (stream = stream_base + t)
__global__ void __launch_bounds__(PWA_THREADS) k_toy_moments(ToyWaves tw, const float2* __restrict__ V,
                                                             const double* __restrict__ C,
                                                             const long long* __restrict__ n_cand, uint64_t seed,
                                                             uint32_t stream_base, int n_bins,
                                                             unsigned long long* __restrict__ acc,
                                                             long long* __restrict__ n_acc) {
    extern __shared__ long long swacc[];  // [PWA_THREADS / 32][n_bins * 25]
    __shared__ float sN[LM];
    __shared__ float2 sV[PWA_MAX_WAVES];
    __shared__ int scount[PWA_THREADS / 32];
    const int t = blockIdx.x;
    const int K = tw.wt.K;
    const int nf = n_bins * LM, lane = threadIdx.x & 31;
    ylm_norms(sN);
    if (threadIdx.x < K) sV[threadIdx.x] = V[(int64_t)t * K + threadIdx.x];
    for (int i = threadIdx.x; i < (PWA_THREADS / 32) * nf; i += blockDim.x) swacc[i] = 0;
    __syncthreads();
    long long* wacc = swacc + (threadIdx.x >> 5) * nf;
    const long long nc = n_cand[t];
    const float Cf = (float)C[t];
    const long long chunk = (nc + gridDim.y - 1) / gridDim.y;
    const long long j0 = (long long)blockIdx.y * chunk;
    long long j1 = j0 + chunk;
    if (j1 > nc) j1 = nc;
    const float inv_w = (float)((double)n_bins / (3.0 - 0.99));
    int cnt = 0;
    // warp-uniform loop: the warp's first candidate decides, lanes past j1 idle
    for (long long jw = j0 + (threadIdx.x & ~31); jw < j1; jw += blockDim.x) {
        const long long j = jw + lane;
        bool take = false;
        Candidate cd;
        if (j < j1) {
            cd = candidate(seed, stream_base + (uint32_t)t, j);
            take = cd.u * Cf < intensity(tw.wt, sV, cd);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, take);
        if (mask) {
            float y[LM];
            int b = 0;
            if (take) {
                ylm25(cd.ct, cd.ph, sN, y);
                b = mass_bin(cd.m, n_bins, 0.99f, inv_w);
            } else {
#pragma unroll
                for (int k = 0; k < LM; ++k) y[k] = 0.f;
            }
            warp_add_events(wacc, mask, b, y);
            cnt += take ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) scount[threadIdx.x >> 5] = cnt;
    __syncthreads();
    block_flush(swacc, nf, acc + (int64_t)t * nf);
    if (threadIdx.x == 0) {
        long long c = 0;
        for (int w = 0; w < PWA_THREADS / 32; ++w) c += scount[w];
        atomicAdd(reinterpret_cast<unsigned long long*>(n_acc + t), (unsigned long long)c);
    }
}

// per-warp accumulators of the moments kernels (n_bins <= 64: at most 102,400 bytes)
size_t moments_smem(int n_bins) { return sizeof(long long) * (PWA_THREADS / 32) * (size_t)n_bins * LM; }

}  // namespace

size_t moments_workspace(int n_bins, int T) { return sizeof(unsigned long long) * (size_t)n_bins * LM * (size_t)T; }

cudaError_t launch_moments(const float* kin, int64_t n, int64_t ld, int n_bins, double m_lo, double m_hi, double* feat,
                           void* ws, int sm_count, cudaStream_t st) {
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(ws);
    cudaError_t e = cudaMemsetAsync(acc, 0, moments_workspace(n_bins, 1), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + PWA_THREADS - 1) / PWA_THREADS;
    if (blocks > (int64_t)sm_count * 4) blocks = (int64_t)sm_count * 4;
    if (blocks < 1) blocks = 1;
    const size_t smem = moments_smem(n_bins);
    cudaFuncSetAttribute(k_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_moments<<<(unsigned)blocks, PWA_THREADS, smem, st>>>(kin, n, ld, n_bins, (float)m_lo,
                                                           (float)(n_bins / (m_hi - m_lo)), acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_moments_final<<<(n_bins * LM + 255) / 256, 256, 0, st>>>(acc, n_bins * LM, nullptr, n, feat, 1);
    return cudaGetLastError();
}

cudaError_t launch_toy_moments(const WaveTable& wt, const double* Md, const double* Wd, const float2* V, int T,
                               const double2* Psi_flat, double n_target, uint64_t seed, uint32_t stream_base,
                               int n_bins, double* feat, long long* n_acc, void* ws, cudaStream_t st) {
    ToyWaves tw;
    tw.wt = wt;
    for (int a = 0; a < PWA_MAX_WAVES; ++a) {
        tw.M[a] = a < wt.K ? Md[a] : 1.0;
        tw.W[a] = a < wt.K ? Wd[a] : 1.0;
    }
    char* c = reinterpret_cast<char*>(ws);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(c);
    c += (moments_workspace(n_bins, T) + 255) & ~size_t(255);
    double* C = reinterpret_cast<double*>(c);
    c += (sizeof(double) * T + 255) & ~size_t(255);
    long long* nc = reinterpret_cast<long long*>(c);
    cudaError_t e = cudaMemsetAsync(acc, 0, moments_workspace(n_bins, T), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_acc, 0, sizeof(long long) * T, st);
    if (e != cudaSuccess) return e;
    k_toy_setup<<<T, PWA_THREADS, 0, st>>>(tw, V, Psi_flat, T, n_target, C, nc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int bpt = 16;  // blocks per toy
    const size_t smem = moments_smem(n_bins);
    cudaFuncSetAttribute(k_toy_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_toy_moments<<<dim3(T, bpt), PWA_THREADS, smem, st>>>(tw, V, C, nc, seed, stream_base, n_bins, acc, n_acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)T * n_bins * LM;
    k_moments_final<<<(unsigned)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535), 256, 0, st>>>(
        acc, n_bins * LM, n_acc, 0, feat, T);
    return cudaGetLastError();
}

size_t toy_moments_workspace(int n_bins, int T) {
    return ((moments_workspace(n_bins, T) + 255) & ~size_t(255)) + ((sizeof(double) * T + 255) & ~size_t(255)) +
           sizeof(long long) * T + 256;
}

}  // namespace pwa
