// Kernels of the learned start proposer's MLP (1000 -> 256 -> 256 -> 256 -> 32 x 2K):
// BF16 weights and activations, FP32 accumulation, trained with the project's own forward,
// backward, loss and optimiser kernels.
//
//  * k_gemm: C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]) (ReLU), with arbitrary element strides
//    for A and B, so one kernel serves the forward product (X W^T), the data gradient (dY W)
//    and the weight gradient (dY^T X).  64 x 64 (or 32 x 32) output tiles, 16-deep k tiles
//    staged through shared memory as FP32 along the operand's contiguous dimension, 4 x 4
//    outputs per thread; sequential k order per output, so the result is deterministic.
//  * k_wta_loss: winner-takes-all over C candidate V vectors per sample (one warp per sample,
//    one lane per candidate): d_c = |V_c|^2 + |T|^2 - 2 |sum_a conj(V_ca) T_a| is the distance
//    after the optimal global phase (the likelihood does not see a global phase, Eq. 1);
//    loss = (1 - eps) d_winner + eps mean_c d_c, gradient 2 (V_c - exp(-i arg z_c) T) per
//    candidate, weighted.
//  * k_adam: Adam (Kingma and Ba) on FP32 master weights, writing the BF16 copy.
#include <cuda_bf16.h>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

__device__ __forceinline__ float ld_elem(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_elem(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

constexpr int GK = 16;

// Output tiles of TM x TN (TM = TN = 64 with 256 threads, or 32 with 64 threads for grids too
// small to fill the GPU), 4 x 4 outputs per thread, 16-deep k tiles staged through shared
// memory as FP32.  The staging loads run along whichever of (m, k) -- and (n, k) -- is
// contiguous in memory, so every operand layout is read with coalesced loads.
template <int TM, typename TA, typename TB>
__global__ void __launch_bounds__(TM * TM / 16) k_gemm(int M, int N, int Kc, const TA* __restrict__ A, int64_t sam,
                                                       int64_t sak, const TB* __restrict__ B, int64_t sbn, int64_t sbk,
                                                       const float* __restrict__ bias, int relu, int accumulate,
                                                       float* __restrict__ C, __nv_bfloat16* __restrict__ Cb,
                                                       int64_t ldc) {
    constexpr int NT = TM * TM / 16;     // threads
    constexpr int TS = TM / 4;           // threads along m (and along n)
    constexpr int LOADS = TM * GK / NT;  // staged elements per thread and operand
    __shared__ float sA[GK][TM + 4];
    __shared__ float sB[GK][TM + 4];
    const int tid = threadIdx.x;
    const int tm = tid % TS, tn = tid / TS;  // outputs m = m0 + tm + TS i, n = n0 + tn + TS j
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TM;
    const bool a_mfast = sam == 1 && sak != 1;  // A contiguous along m
    const bool b_nfast = sbn == 1 && sbk != 1;  // B contiguous along n
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < Kc; k0 += GK) {
#pragma unroll
        for (int r = 0; r < LOADS; ++r) {
            const int idx = tid + NT * r;
            {
                const int mm = a_mfast ? idx % TM : idx / GK, kk = a_mfast ? idx / TM : idx % GK;
                const int gm = m0 + mm, gk = k0 + kk;
                sA[kk][mm] = (gm < M && gk < Kc) ? ld_elem(A, (int64_t)gm * sam + (int64_t)gk * sak) : 0.f;
            }
            {
                const int nn = b_nfast ? idx % TM : idx / GK, kk = b_nfast ? idx / TM : idx % GK;
                const int gn = n0 + nn, gk = k0 + kk;
                sB[kk][nn] = (gn < N && gk < Kc) ? ld_elem(B, (int64_t)gn * sbn + (int64_t)gk * sbk) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][tm + TS * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tn + TS * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tm + TS * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tn + TS * j;
            if (gn >= N) continue;
            float v = acc[i][j];
            if (bias) v += bias[gn];
            const int64_t o = (int64_t)gm * ldc + gn;
            if (accumulate && C) v += C[o];
            if (relu) v = fmaxf(v, 0.f);
            if (C) C[o] = v;
            if (Cb) Cb[o] = __float2bfloat16_rn(v);
        }
    }
}

__global__ void k_relu_bwd(const __nv_bfloat16* __restrict__ Y, float* __restrict__ dY, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(Y[i]) > 0.f)) dY[i] = 0.f;
}

// db[n] = sum_b dY[b][n]: a block takes 32 columns; warp w sums rows w, w + 8, ... of them (lanes
// along n, coalesced), then lane n of warp 0 adds the 8 warp sums in warp order (fixed order).
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ dY, int B, int N, float* __restrict__ db) {
    __shared__ float part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nidx = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (nidx < N) {
#pragma unroll 8
        for (int b = w; b < B; b += 8) s += dY[(int64_t)b * N + nidx];
    }
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && nidx < N) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        db[nidx] = t;
    }
}

// one warp per sample; lane c = candidate c (C <= 32)
__global__ void k_wta_loss(const float* __restrict__ out, const float* __restrict__ target, int B, int C, int K,
                           float eps, float* __restrict__ loss, float* __restrict__ dout, int* __restrict__ winner) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const int D = 2 * K;
    const float* tb = target + (int64_t)warp * D;
    const float* ob = out + (int64_t)warp * C * D;
    float d = INFINITY, zr = 0.f, zi = 0.f, vv = 0.f, tt = 0.f;
    if (lane < C) {
        const float* v = ob + (int64_t)lane * D;
        for (int a = 0; a < K; ++a) {
            const float vr = v[2 * a], vi = v[2 * a + 1], tr = tb[2 * a], ti = tb[2 * a + 1];
            zr += vr * tr + vi * ti;  // conj(v) t
            zi += vr * ti - vi * tr;
            vv += vr * vr + vi * vi;
            tt += tr * tr + ti * ti;
        }
        d = vv + tt - 2.f * sqrtf(zr * zr + zi * zi);
    }
    // argmin over lanes (smallest index on ties)
    float best = d;
    int bi = lane < C ? lane : 1 << 30;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob2 < best || (ob2 == best && oi < bi)) {
            best = ob2;
            bi = oi;
        }
    }
    float dsum = lane < C ? d : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0) {
        loss[warp] = (1.f - eps) * best + eps * dsum / (float)C;
        if (winner) winner[warp] = bi;
    }
    if (lane < C && dout) {
        const float w = ((lane == bi) ? (1.f - eps) : 0.f) + eps / (float)C;
        const float zn = sqrtf(zr * zr + zi * zi);
        // exp(-i arg z)
        const float er = zn > 0.f ? zr / zn : 1.f, ei = zn > 0.f ? -zi / zn : 0.f;
        const float* v = ob + (int64_t)lane * D;
        float* g = dout + ((int64_t)warp * C + lane) * D;
        const float sc = 2.f * w / (float)B;
        for (int a = 0; a < K; ++a) {
            const float tr = tb[2 * a], ti = tb[2 * a + 1];
            g[2 * a] = sc * (v[2 * a] - (er * tr - ei * ti));
            g[2 * a + 1] = sc * (v[2 * a + 1] - (er * ti + ei * tr));
        }
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const double* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n, float scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn((float)(x[i] * (double)scale));
}

unsigned grid1d(int64_t n, int sm_count) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)sm_count * 16) b = (int64_t)sm_count * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <int TM>
cudaError_t mlp_gemm_tiles(int M, int N, int Kc, const void* A, int a_bf16, int64_t sam, int64_t sak, const void* B,
                           int b_bf16, int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate, float* C,
                           __nv_bfloat16* cb, int64_t ldc, cudaStream_t st) {
    dim3 grid((M + TM - 1) / TM, (N + TM - 1) / TM);
    constexpr int NT = TM * TM / 16;
    if (a_bf16 && b_bf16)
        k_gemm<TM, __nv_bfloat16, __nv_bfloat16><<<grid, NT, 0, st>>>(
            M, N, Kc, (const __nv_bfloat16*)A, sam, sak, (const __nv_bfloat16*)B, sbn, sbk, bias, relu, accumulate, C, cb, ldc);
    else if (a_bf16)
        k_gemm<TM, __nv_bfloat16, float><<<grid, NT, 0, st>>>(M, N, Kc, (const __nv_bfloat16*)A, sam, sak,
                                                              (const float*)B, sbn, sbk, bias, relu, accumulate, C, cb, ldc);
    else if (b_bf16)
        k_gemm<TM, float, __nv_bfloat16><<<grid, NT, 0, st>>>(M, N, Kc, (const float*)A, sam, sak,
                                                              (const __nv_bfloat16*)B, sbn, sbk, bias, relu, accumulate, C,
                                                              cb, ldc);
    else
        k_gemm<TM, float, float><<<grid, NT, 0, st>>>(M, N, Kc, (const float*)A, sam, sak, (const float*)B, sbn, sbk,
                                                      bias, relu, accumulate, C, cb, ldc);
    return cudaGetLastError();
}

cudaError_t launch_mlp_gemm(int M, int N, int Kc, const void* A, int a_bf16, int64_t sam, int64_t sak, const void* B,
                            int b_bf16, int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate, float* C,
                            uint16_t* Cb, int64_t ldc, int sm_count, cudaStream_t st) {
    __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(Cb);
    const int64_t tiles64 = (int64_t)((M + 63) / 64) * ((N + 63) / 64);
    if (tiles64 < 2 * (int64_t)sm_count)  // too few 64 x 64 tiles to fill the GPU
        return mlp_gemm_tiles<32>(M, N, Kc, A, a_bf16, sam, sak, B, b_bf16, sbn, sbk, bias, relu, accumulate, C, cb, ldc, st);
    return mlp_gemm_tiles<64>(M, N, Kc, A, a_bf16, sam, sak, B, b_bf16, sbn, sbk, bias, relu, accumulate, C, cb, ldc, st);
}

cudaError_t launch_mlp_relu_bwd(const uint16_t* Y, float* dY, int64_t n, int sm_count, cudaStream_t st) {
    k_relu_bwd<<<grid1d(n, sm_count), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Y), dY, n);
    return cudaGetLastError();
}

cudaError_t launch_mlp_bias_grad(const float* dY, int B, int N, float* db, cudaStream_t st) {
    k_bias_grad<<<(N + 31) / 32, 256, 0, st>>>(dY, B, N, db);
    return cudaGetLastError();
}

cudaError_t launch_mlp_wta(const float* out, const float* target, int B, int C, int K, float eps, float* loss,
                           float* dout, int* winner, cudaStream_t st) {
    const int warps_per_block = 8;
    k_wta_loss<<<(B + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(out, target, B, C, K, eps,
                                                                                            loss, dout, winner);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* p, const float* g, float* m, float* v, uint16_t* pb, int64_t n, float lr, float b1,
                            float b2, float eps, int step, int sm_count, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid1d(n, sm_count), 256, 0, st>>>(p, g, m, v, reinterpret_cast<__nv_bfloat16*>(pb), n, lr, b1, b2, eps, c1,
                                                c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_to_bf16(const double* x, uint16_t* y, int64_t n, float scale, int sm_count, cudaStream_t st) {
    k_to_bf16<<<grid1d(n, sm_count), 256, 0, st>>>(x, reinterpret_cast<__nv_bfloat16*>(y), n, scale);
    return cudaGetLastError();
}

}  // namespace pwa
