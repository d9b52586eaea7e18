// Toy events by accept-reject from the intensity I(Omega) = |sum_a V_a A_a(Omega)|^2 (Eq. 1).
//
// The paper's workflow draws data from a model with known production amplitudes to study
// fits (repeated fits from many starts, Sec. 2 and Sec. 4 "Fits with large numbers of
// parameters"); the data samples of every workload here are made this way.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: counter (j_lo, j_hi, stream, 0) for candidate j, key (seed_lo,
// seed_hi).  The four output words give m_KK = 0.99 + 2.01 u0, cos(theta) = 2 u1 - 1,
// phi = 2 pi u2 (flat phase space) and the accept uniform u3, each u = (word >> 8) 2^-24, in
// round-to-nearest single precision without contraction, so any other implementation of the
// same definition reproduces the candidates bit for bit.
//
// Candidate j is accepted iff u3 * C < I(Omega_j) with I evaluated in FP32 by the same model
// code as the amplitude kernel; C is a bound on I (pwa_envelope).  Accepted events are written
// in candidate order: a counting pass, a scan of the per-block counts, and a writing pass that
// re-evaluates the accept decision, so the output is deterministic and independent of the
// launch geometry.
#include "gen_model.cuh"

namespace pwa {

namespace {

constexpr int GEN_CPT = 16;                       // candidates per thread
constexpr int GEN_CPB = GEN_CPT * PWA_THREADS;   // candidates per block


__device__ __forceinline__ unsigned accept_mask(const WaveTable& wt, const float2* sV, uint64_t seed, uint32_t stream,
                                                int64_t first, int64_t end, float C) {
    unsigned mask = 0;
    for (int k = 0; k < GEN_CPT; ++k) {
        const int64_t j = first + k;
        if (j >= end) break;
        const Candidate cd = candidate(seed, stream, j);
        if (cd.u * C < intensity(wt, sV, cd)) mask |= 1u << k;
    }
    return mask;
}

__global__ void __launch_bounds__(PWA_THREADS) k_gen_count(WaveTable wt, const float2* __restrict__ V, uint64_t seed,
                                                           uint32_t stream, int64_t cand0, int64_t n_cand, float C,
                                                           long long* __restrict__ counts) {
    __shared__ float2 sV[PWA_MAX_WAVES];
    __shared__ int swarp[PWA_THREADS / 32];
    if (threadIdx.x < wt.K) sV[threadIdx.x] = V[threadIdx.x];
    __syncthreads();
    const int64_t first = cand0 + (int64_t)blockIdx.x * GEN_CPB + (int64_t)threadIdx.x * GEN_CPT;
    const unsigned m = accept_mask(wt, sV, seed, stream, first, cand0 + n_cand, C);
    int c = __popc(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < PWA_THREADS / 32; ++w) s += swarp[w];
        counts[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts (one block, sequential chunks of 1024), total -> n_acc.
__global__ void __launch_bounds__(1024) k_gen_scan(long long* __restrict__ counts, int nb,
                                                   long long* __restrict__ n_acc) {
    __shared__ long long s[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < nb ? counts[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) counts[i] = carry + s[threadIdx.x] - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_acc = carry;
}

__global__ void __launch_bounds__(PWA_THREADS) k_gen_write(WaveTable wt, const float2* __restrict__ V, uint64_t seed,
                                                           uint32_t stream, int64_t cand0, int64_t n_cand, float C,
                                                           const long long* __restrict__ offsets,
                                                           float* __restrict__ kin, int64_t ld_out,
                                                           int64_t max_out) {
    __shared__ float2 sV[PWA_MAX_WAVES];
    __shared__ int swarp[PWA_THREADS / 32];
    if (threadIdx.x < wt.K) sV[threadIdx.x] = V[threadIdx.x];
    __syncthreads();
    const int64_t first = cand0 + (int64_t)blockIdx.x * GEN_CPB + (int64_t)threadIdx.x * GEN_CPT;
    const unsigned m = accept_mask(wt, sV, seed, stream, first, cand0 + n_cand, C);
    // block-wide exclusive scan of the per-thread counts (thread order == candidate order)
    const int c = __popc(m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) swarp[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += swarp[w];
    int64_t pos = offsets[blockIdx.x] + wbase + incl - c;
    for (int k = 0; k < GEN_CPT; ++k) {
        if (!((m >> k) & 1u)) continue;
        if (pos < max_out) {
            const Candidate cd = candidate(seed, stream, first + k);
            kin[pos] = cd.m;
            kin[ld_out + pos] = cd.ct;
            kin[2 * ld_out + pos] = cd.ph;
        }
        ++pos;
    }
}

}  // namespace

size_t generate_workspace(int64_t n_cand) {
    const int64_t nb = (n_cand + GEN_CPB - 1) / GEN_CPB;
    return sizeof(long long) * (size_t)(nb > 0 ? nb : 1);
}

cudaError_t launch_generate(const WaveTable& wt, const float2* V, uint64_t seed, uint32_t stream, int64_t cand0,
                            int64_t n_cand, double envelope, float* kin, int64_t ld_out, int64_t max_out,
                            long long* n_acc, void* ws, cudaStream_t st) {
    const int64_t nb = (n_cand + GEN_CPB - 1) / GEN_CPB;
    long long* counts = reinterpret_cast<long long*>(ws);
    const float C = (float)envelope;
    if (nb > 0) {
        k_gen_count<<<(unsigned)nb, PWA_THREADS, 0, st>>>(wt, V, seed, stream, cand0, n_cand, C, counts);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_gen_scan<<<1, 1024, 0, st>>>(counts, (int)nb, n_acc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nb == 0) return e;
    k_gen_write<<<(unsigned)nb, PWA_THREADS, 0, st>>>(wt, V, seed, stream, cand0, n_cand, C, counts, kin, ld_out,
                                                     max_out);
    return cudaGetLastError();
}

}  // namespace pwa
