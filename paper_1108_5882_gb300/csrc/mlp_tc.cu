// The MLP's GEMM on the fifth-generation tensor cores (tcgen05.mma kind::f16, BF16 operands,
// FP32 accumulation in tensor memory):
//
//   C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]) (+ C, ReLU), A(m, k) = A[m sam + k sak],
//   B(n, k) = B[n sbn + k sbk], B in BF16, A in BF16 or FP32.
//
// An FP32 operand (the back-propagated gradients) is split into three BF16 parts, x = hi + mid +
// lo with hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid) (24 significant bits in all),
// and each part is multiplied by the BF16 operand exactly (8 x 8 bit products), so the products
// are those of FP32 arithmetic; BF16 x BF16 (the forward pass) is one product.
//
// Block: a 128 x 64 output tile (one tensor-memory lane per row, 64 FP32 columns), 256 threads.
// The contraction runs in chunks of 64: the threads stage the chunk of A (each part) and B into
// shared memory as K-major core matrices (8 rows x 16 bytes, no swizzle), one thread issues 4 k-steps x (1 or 3) MMAs, and
// after they complete every thread adds its row's 64 columns to FP32 registers (rounded to
// nearest).  Keeping the tensor-memory accumulation to one chunk bounds the error of its
// unrounded FP32 additions to ~12 steps.  The smaller parts go first.
#include <cuda_bf16.h>

#include "pwa_internal.cuh"
#include "tc.cuh"

namespace pwa {

namespace {

constexpr int MT_NT = 256, MT_BM = 128, MT_BN = 64, MT_BK = 64;
constexpr int MT_IA = MT_BM * MT_BK / 8 / MT_NT, MT_IB = MT_BN * MT_BK / 8 / MT_NT;  // staging items per thread
constexpr uint32_t MT_SBO = 8u * MT_BK * 2u;  // bytes between 8-row groups (rows of 64 BF16)
constexpr uint32_t MT_A_BYTES = MT_BM * MT_BK * 2u, MT_B_BYTES = MT_BN * MT_BK * 2u;
constexpr uint64_t MT_WAIT_NS = 1000000000ull;

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, dense, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// byte offset of BF16 element (row, k) in a K-major tile of rows of MT_BK elements
__device__ __forceinline__ uint32_t bf_off(int row, int k) {
    return (uint32_t)(row >> 3) * MT_SBO + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ float ld_val(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

// 256 threads: warps w and w + 4 share tensor-memory lanes 32 (w % 4) + 0..31 (the tile's rows)
// and take columns 0..31 and 32..63 of them.  Per chunk each thread loads its 32 elements of A
// and 16 of B into registers (the loads of chunk c + 1 are issued while the MMAs of chunk c
// run), then converts and stores them as 16-byte rows of core matrices.
template <typename TA>
__global__ void __launch_bounds__(MT_NT) k_mlp_tc(int M, int N, int Kc, const TA* __restrict__ A, int64_t sam,
                                                  int64_t sak, const __nv_bfloat16* __restrict__ B, int64_t sbn,
                                                  int64_t sbk, const float* __restrict__ bias, int relu,
                                                  int accumulate, float* __restrict__ C, __nv_bfloat16* __restrict__ Cb,
                                                  int64_t ldc, int* __restrict__ status) {
    constexpr bool SPLIT = sizeof(TA) == 4;  // FP32 A: three BF16 parts
    constexpr int NPA = SPLIT ? 3 : 1;
    extern __shared__ __align__(1024) unsigned char msm[];
    // [part][A tile] then [B tile], then the mbarrier and the tensor-memory address
    unsigned char* sA = msm;
    unsigned char* sB = msm + NPA * MT_A_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sB + MT_B_BYTES);
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(sB + MT_B_BYTES + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int lq = warp & 3, hh = warp >> 2;
    const int m0 = blockIdx.x * MT_BM, n0 = blockIdx.y * MT_BN;

    if (warp == 0) tmem_alloc(taddr_s, 64);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *taddr_s;
    const uint32_t lane_t = tmem + ((uint32_t)(32 * lq) << 16);
    const uint32_t sbase = smem_u32(msm);
    constexpr uint32_t idesc = umma_idesc_bf16(MT_BM, MT_BN);

    // staging items: (row, 8 consecutive k) -> one 16-byte store per part into the K-major
    // tile; the lanes of a warp take consecutive rows, so the 8 lanes of a store phase write 8
    // rows of one core matrix (no bank conflict)
    float xa[MT_IA][8];
    __nv_bfloat16 xb[MT_IB][8];
    auto load_chunk = [&](int k0) {
#pragma unroll
        for (int r = 0; r < MT_IA; ++r) {
            const int idx = tid + MT_NT * r;
            const int mm = idx % MT_BM, ko = idx / MT_BM;
            const int gm = m0 + mm;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int gk = k0 + 8 * ko + j;
                xa[r][j] = (gm < M && gk < Kc) ? ld_val(A, (int64_t)gm * sam + (int64_t)gk * sak) : 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < MT_IB; ++r) {
            const int idx = tid + MT_NT * r;
            const int nn = idx % MT_BN, ko = idx / MT_BN;
            const int gn = n0 + nn;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int gk = k0 + 8 * ko + j;
                xb[r][j] = (gn < N && gk < Kc) ? B[(int64_t)gn * sbn + (int64_t)gk * sbk] : __float2bfloat16_rn(0.f);
            }
        }
    };
    auto pack8 = [](const __nv_bfloat16 (&v)[8]) {
        uint4 u;
        u.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
        u.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
        u.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
        u.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
        return u;
    };
    auto store_chunk = [&]() {
#pragma unroll
        for (int r = 0; r < MT_IA; ++r) {
            const int idx = tid + MT_NT * r;
            const int mm = idx % MT_BM, ko = idx / MT_BM;
            const uint32_t o = bf_off(mm, 8 * ko);
            __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                hi[j] = __float2bfloat16_rn(xa[r][j]);
                if (SPLIT) {
                    const float rr = xa[r][j] - __bfloat162float(hi[j]);
                    mid[j] = __float2bfloat16_rn(rr);
                    lo[j] = __float2bfloat16_rn(rr - __bfloat162float(mid[j]));
                }
            }
            *reinterpret_cast<uint4*>(sA + o) = pack8(hi);
            if (SPLIT) {
                *reinterpret_cast<uint4*>(sA + MT_A_BYTES + o) = pack8(mid);
                *reinterpret_cast<uint4*>(sA + 2 * MT_A_BYTES + o) = pack8(lo);
            }
        }
#pragma unroll
        for (int r = 0; r < MT_IB; ++r) {
            const int idx = tid + MT_NT * r;
            const int nn = idx % MT_BN, ko = idx / MT_BN;
            *reinterpret_cast<uint4*>(sB + bf_off(nn, 8 * ko)) = pack8(xb[r]);
        }
    };

    float acc[32];  // columns 32 hh + 0..31 of row 32 lq + lane
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    bool ok = true;
    uint32_t phase = 0;
    if (Kc > 0) load_chunk(0);
    for (int k0 = 0; k0 < Kc && ok; k0 += MT_BK) {
        store_chunk();
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint64_t dB = umma_desc(sbase + NPA * MT_A_BYTES, 128u, MT_SBO);
            uint32_t first = 1;
#pragma unroll
            for (int part = NPA - 1; part >= 0; --part) {  // smallest part first
                const uint64_t dA = umma_desc(sbase + part * MT_A_BYTES, 128u, MT_SBO);
#pragma unroll
                for (int s = 0; s < MT_BK / 16; ++s) {
                    mma_bf16_ss(tmem, dA + 16u * s, dB + 16u * s, idesc, first ? 0u : 1u);
                    first = 0;
                }
            }
            umma_commit(bar);
        }
        if (k0 + MT_BK < Kc) load_chunk(k0 + MT_BK);  // overlaps the MMAs
        ok = mbar_wait_bounded(bar, phase, MT_WAIT_NS);
        ok = __syncthreads_and(ok);
        if (ok) phase ^= 1u;
        tc_fence_after();
        if (ok) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float d[16];
                tmem_ld16(lane_t + 32 * hh + 16 * q, d);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[16 * q + j] += d[j];
            }
        }
        tc_fence_before();
        __syncthreads();  // the chunk's tiles and the accumulator may be overwritten
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, 2);
        mbar_wait_bounded(bar, phase, MT_WAIT_NS / 10);  // the group in flight, before tmem is freed
    }
    // ---- epilogue: row 32 lq + lane, columns 32 hh + 0..31
    const int gm = m0 + 32 * lq + (tid & 31);
    if (ok && gm < M) {
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const int gn = n0 + 32 * hh + j;
            if (gn >= N) break;
            float v = acc[j];
            if (bias) v += bias[gn];
            const int64_t o = (int64_t)gm * ldc + gn;
            if (accumulate && C) v += C[o];
            if (relu) v = fmaxf(v, 0.f);
            if (C) C[o] = v;
            if (Cb) Cb[o] = __float2bfloat16_rn(v);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
}

template <typename TA>
cudaError_t mlp_tc_launch(int M, int N, int Kc, const TA* A, int64_t sam, int64_t sak, const __nv_bfloat16* B,
                          int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate, float* C,
                          __nv_bfloat16* Cb, int64_t ldc, int* status, cudaStream_t st) {
    constexpr int NPA = sizeof(TA) == 4 ? 3 : 1;
    const size_t smem = (size_t)NPA * MT_A_BYTES + MT_B_BYTES + 64;
    auto kern = k_mlp_tc<TA>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    dim3 grid((M + MT_BM - 1) / MT_BM, (N + MT_BN - 1) / MT_BN);
    kern<<<grid, MT_NT, smem, st>>>(M, N, Kc, A, sam, sak, B, sbn, sbk, bias, relu, accumulate, C, Cb, ldc, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_gemm_tc(int M, int N, int Kc, const void* A, int a_bf16, int64_t sam, int64_t sak,
                               const void* B, int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate,
                               float* C, uint16_t* Cb, int64_t ldc, int* status, cudaStream_t st) {
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(B);
    __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(Cb);
    if (a_bf16)
        return mlp_tc_launch<__nv_bfloat16>(M, N, Kc, reinterpret_cast<const __nv_bfloat16*>(A), sam, sak, b, sbn, sbk,
                                            bias, relu, accumulate, C, cb, ldc, status, st);
    return mlp_tc_launch<float>(M, N, Kc, reinterpret_cast<const float*>(A), sam, sak, b, sbn, sbk, bias, relu,
                                accumulate, C, cb, ldc, status, st);
}

}  // namespace pwa
