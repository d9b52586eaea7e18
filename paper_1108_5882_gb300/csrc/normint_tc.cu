// Monte-Carlo normalisation integral on the fifth-generation tensor cores (Sec. 2, Eq. 3, inner
// bracket of the second term, with unit weights): Psi_ab = (1/N_gen) sum_j A_a(j) conj(A_b(j)),
// K <= 32, from stored amplitudes or straight from the MC kinematics.
//
// With X = [Re A; Im A] (2K real rows over the events) the real Gram matrix G = X X^T holds Psi:
//   Re Psi_ab = G[a][b] + G[K+a][K+b],   Im Psi_ab = G[K+a][b] - G[a][K+b].
// FP32 products of FP32 operands are three TF32 products, each operand split as x = hi + lo (both
// the nearest TF32 values: x - hi - lo within 2^-22 |x|, unbiased).  Because G is symmetric,
// X X^T ~ Xh Xh^T + Xl Xh^T + (Xl Xh^T)^T, so ONE real GEMM per tile gives all three products:
//   D = [Xh; Xl] Xh^T   (M = 128 rows: Xh then Xl, padded with zero rows; N = 2 KMAX columns;
//                        contraction over the 128 events of the tile)
//   G = D[0:2K] + D[2K:4K] + D[2K:4K]^T.
// The A operand is the tile itself and the B operand its first 2 KMAX rows (one shared-memory
// tile, read twice by the tensor cores).
//
// Pipeline (one block per SM, 16 compute warps + 1 MMA warp): two shared-memory stages of 128
// events and two tensor-memory accumulators.  For tile s the compute warps fill stage s % 2 (the
// amplitudes, computed from the kinematics or loaded, split into TF32 hi / lo), the MMA warp
// issues the 16 MMAs of the tile into accumulator s % 2 (a fresh sum each tile), and the compute
// warps add the accumulator of tile s - 1 into FP32 registers (round to nearest; warps w, w + 4,
// w + 8 and w + 12 share lane quarter w % 4 and take a quarter of the columns each, at least 8),
// which enter double-single sums in shared memory every 8 tiles.  The fill, not the MMAs, bounds
// a tile (an MMA of N = 2K <= 64 costs ~60 cycles; computing and splitting 128 x K amplitudes
// costs several thousand), hence the 16 warps.  The tensor memory's FP32 accumulation does not round to
// nearest and the diagonal of G is a sum of squares (coherent), so the sums leave tensor memory
// every tile: their error stays ~1e-6 of the entry.  Every wait is bounded; a timeout sets status bit 1,
// skips the remaining waits and MMAs, and the tensor memory is freed only after the MMAs issued
// have completed (bounded).
//
// Work split of a fill: thread (warp w, lane l) takes the 4 consecutive events 4 q .. 4 q + 3,
// q = 2 w + l / 16, and the waves s = 16 m + (l % 16); the 8 threads of a quarter-warp store the
// 8 rows of one 16-byte column of core matrices, so every shared-memory store is conflict-free.
// From kinematics, each thread first computes the angular factor P_J(cos theta) exp(i lambda phi)
// of every fourth (J, lambda) group for one event of its half-warp into a per-tile table.
#include "amp_model.cuh"
#include "tc.cuh"

namespace pwa {

namespace {

constexpr int NT_E = 128;                  // events per tile (16 k-steps of 8)
constexpr int NT_CW = 16;                  // compute warps
constexpr int NT_THREADS = 32 * NT_CW + 32;  // + 1 MMA warp
constexpr int NT_NG = 16;                  // (J, lambda) groups, at most (from kinematics)
constexpr int NT_YS = NT_NG + 1;           // row stride of the angular table (float2)
constexpr uint32_t NT_SBO = 32u * NT_E;    // bytes between groups of 8 rows of a K-major tile
constexpr uint32_t NT_STAGE = 16u * NT_SBO;  // 128 rows
constexpr uint64_t NT_WAIT_NS = 1000000000ull;
constexpr int NT_FF = 8;                   // tiles per double-single update of the sums

__constant__ float c_nt_inv_int[9] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};

template <int KMAX>
struct NtCfg {
    static constexpr int N = 2 * KMAX;                         // GEMM columns
    static constexpr uint32_t TCOLS = 2 * N < 32 ? 32 : 2 * N;  // two accumulators (power of 2 >= 32)
    static constexpr uint32_t OFF_ST0 = 0, OFF_ST1 = NT_STAGE;
    static constexpr uint32_t OFF_ACC = 2 * NT_STAGE;                       // ff sums [N][128 lanes] hi, then lo
    // angular table float2 [NT_E][NT_YS]: event-major with an odd row stride, so that the 16 lanes
    // of a half-warp (one event, the groups of 16 waves) read distinct banks or broadcast
    static constexpr uint32_t OFF_Y = OFF_ACC + 2u * N * 128u * 4u;
    static constexpr uint32_t OFF_BAR = OFF_Y + (uint32_t)NT_YS * NT_E * 8u;
    static constexpr uint32_t SMEM = OFF_BAR + 128;
    static constexpr int MW = (KMAX + 15) / 16;                // waves per thread
    static constexpr int NH = N / 4 > 8 ? N / 4 : 8;           // drained columns per thread
    static_assert(KMAX % 8 == 0 && KMAX <= 32, "tensor-core normalisation integral: K <= 32");
    static_assert(N % 16 == 0 && N <= 256, "MMA shape");
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// the 4 (events) x (hi, lo) of one real row value into rows r (hi) and r + 2 KMAX (lo)
template <int KMAX>
__device__ __forceinline__ void store_row4(uint32_t st, int r, int q, const float (&x)[4]) {
    float h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) tf32_split(x[k], h[k], l[k]);
    st_shared_v4(st + kmaj_off(r, 4 * q, NT_SBO), h[0], h[1], h[2], h[3]);
    st_shared_v4(st + kmaj_off(r + 2 * KMAX, 4 * q, NT_SBO), l[0], l[1], l[2], l[3]);
}

template <int KMAX, bool FROM_KIN>
__global__ void __launch_bounds__(NT_THREADS, 1) k_normint_tc(const float2* __restrict__ A, int K, int64_t n,
                                                              int64_t ld, const float* __restrict__ kin, WaveTable wt,
                                                              int64_t ev_per_block, float4* __restrict__ part,
                                                              int* __restrict__ status) {
    using C = NtCfg<KMAX>;
    constexpr int N = C::N;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == NT_CW;
    const uint32_t sbase = smem_u32(sm);
    float* acc_hi = reinterpret_cast<float*>(sm + C::OFF_ACC);
    float* acc_lo = acc_hi + N * 128;
    float2* sY = reinterpret_cast<float2*>(sm + C::OFF_Y);
    uint64_t* bar_fill = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);  // [2]
    uint64_t* bar_mma = bar_fill + 2;                                     // [2]
    uint64_t* bar_drain = bar_fill + 4;                                   // [2]
    uint64_t* bar_fin = bar_fill + 6;
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(sm + C::OFF_BAR + 64);
    volatile int* abort_s = reinterpret_cast<volatile int*>(sm + C::OFF_BAR + 68);
    // wave tables (from kinematics): per wave its Breit-Wigner parameters and group
    __shared__ float4 s_prm[KMAX];
    __shared__ int s_grp[KMAX];
    __shared__ int s_gJ[NT_NG], s_glam[NT_NG];

    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_block;
    int64_t e_end = e_begin + ev_per_block;
    if (e_end > n) e_end = n;
    const int ntile = e_begin < e_end ? (int)((e_end - e_begin + NT_E - 1) / NT_E) : 0;

    // zero both stages (rows 4 KMAX .. 127 stay zero) and the sums
    for (int i = tid; i < (int)(2 * NT_STAGE / 16); i += NT_THREADS)
        reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = tid; i < 2 * N * 128; i += NT_THREADS) acc_hi[i] = 0.f;
    if (FROM_KIN) {
        if (tid < KMAX) {
            float4 p = make_float4(0.f, 0.f, 1.f, 1.f);
            int g = 0;
            if (tid < K) {
                p = make_float4(wt.Mhi[tid], wt.Mlo[tid], wt.MW[tid], wt.MW[tid] * wt.MW[tid]);
                int s = 0;
                while (wt.gord[s] != tid) ++s;
                while (wt.gend[g] <= s) ++g;
            }
            s_prm[tid] = p;
            s_grp[tid] = g;
        }
        if (tid < wt.ng && tid < NT_NG) {
            const int a0 = wt.gord[tid == 0 ? 0 : wt.gend[tid - 1]];
            s_gJ[tid] = wt.J[a0];
            s_glam[tid] = wt.lam[a0];
        }
    }
    if (warp == 0) tmem_alloc(taddr_s, C::TCOLS);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_fill + b, NT_CW);
            mbar_init(bar_mma + b, 1);
            mbar_init(bar_drain + b, NT_CW);
        }
        mbar_init(bar_fin, 1);
        *abort_s = 0;
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *taddr_s;

    if (mma_warp) {
        // ================================================================ MMA warp
        constexpr uint32_t idesc = umma_idesc_tf32(128, N);
        for (int s = 0; s < ntile; ++s) {
            const int b = s & 1;
            const uint32_t par = (uint32_t)(s >> 1) & 1u;
            bool ab = *abort_s != 0;
            if (!ab && !mbar_wait_bounded(bar_fill + b, par, NT_WAIT_NS)) ab = true;
            if (!ab && s >= 2 && !mbar_wait_bounded(bar_drain + b, par ^ 1u, NT_WAIT_NS)) ab = true;
            if (ab) {
                *abort_s = 1;
                continue;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t st = sbase + (b ? C::OFF_ST1 : C::OFF_ST0);
                const uint64_t da = umma_desc(st, 128u, NT_SBO);
#pragma unroll
                for (int k = 0; k < NT_E / 8; ++k)
                    mma_tf32_ss(tmem + (uint32_t)(b * N), da + 16u * k, da + 16u * k, idesc, k > 0 ? 1u : 0u);
                umma_commit(bar_mma + b);
            }
            __syncwarp();
        }
        if (lane == 0) umma_commit(bar_fin);
        __syncwarp();
        if (!mbar_wait_bounded(bar_fin, 0, NT_WAIT_NS)) *abort_s = 1;
    } else {
        // ================================================================ compute warps
        const int q = 2 * warp + (lane >> 4);  // event quad of the tile
        const int j = lane & 15;               // wave residue
        const uint32_t lane_t = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        // Drain of the accumulator of tile s: warps w, w + 4, w + 8, w + 12 share lane quarter
        // w % 4 and take NH columns each (the warps past N columns take none); the tile's values
        // are added in FP32 (round to nearest) into registers, and every NT_FF tiles into the
        // double-single sums in shared memory.
        constexpr int NH = C::NH;
        float racc[NH];
#pragma unroll
        for (int v = 0; v < NH; ++v) racc[v] = 0.f;
        const int c_half = (warp >> 2) * NH;
        const bool drains = c_half < N;
        const int row = 32 * (warp & 3) + lane;
        auto flush = [&]() {
            if (!drains) return;
#pragma unroll
            for (int v = 0; v < NH; ++v) {
                const int idx = (c_half + v) * 128 + row;
                const ff r = ff_add_f(ff{acc_hi[idx], acc_lo[idx]}, racc[v]);
                acc_hi[idx] = r.hi;
                acc_lo[idx] = r.lo;
                racc[v] = 0.f;
            }
        };
        int since_ff = 0;
        auto drain = [&](int s) {
            const int b = s & 1;
            const uint32_t par = (uint32_t)(s >> 1) & 1u;
            if (*abort_s != 0 || !mbar_wait_bounded(bar_mma + b, par, NT_WAIT_NS)) {
                *abort_s = 1;
                return;
            }
            tc_fence_after();
            if (drains) {
                if constexpr (NH % 16 == 0) {
#pragma unroll
                    for (int c0 = 0; c0 < NH; c0 += 16) {
                        float d[16];
                        tmem_ld16(lane_t + (uint32_t)(b * N + c_half + c0), d);
                        tmem_wait_ld();
#pragma unroll
                        for (int k = 0; k < 16; ++k) racc[c0 + k] += d[k];
                    }
                } else {
#pragma unroll
                    for (int c0 = 0; c0 < NH; c0 += 8) {
                        float d[8];
                        tmem_ld8(lane_t + (uint32_t)(b * N + c_half + c0), d);
                        tmem_wait_ld();
#pragma unroll
                        for (int k = 0; k < 8; ++k) racc[c0 + k] += d[k];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive_one(bar_drain + b);
            if (++since_ff == NT_FF) {
                flush();
                since_ff = 0;
            }
        };
        // registers of the next tile, loaded one tile ahead so that the global-memory latency
        // overlaps the drain and the wait for the free stage
        float2 pa[C::MW][4];                                 // stored amplitudes
        float pm[4], pct = 0.f, pph = 0.f;                   // kinematics
        auto prefetch = [&](int s) {
            const int64_t e0 = e_begin + (int64_t)s * NT_E + 4 * q;
            if (FROM_KIN) {
#pragma unroll
                for (int k = 0; k < 4; ++k) pm[k] = (s < ntile && e0 + k < e_end) ? __ldg(kin + e0 + k) : 2.f;
                const int64_t ie = e0 + (j & 3);
                const bool in = s < ntile && ie < e_end;
                pct = in ? __ldg(kin + ld + ie) : 0.f;
                pph = in ? __ldg(kin + 2 * ld + ie) : 0.f;
            } else {
#pragma unroll
                for (int mm = 0; mm < C::MW; ++mm) {
                    const int a = 16 * mm + j;
                    if (s < ntile && a < K && e0 + 3 < e_end) {
                        const float4* src = reinterpret_cast<const float4*>(A + (int64_t)a * ld + e0);
                        const float4 v0 = __ldg(src), v1 = __ldg(src + 1);
                        pa[mm][0] = make_float2(v0.x, v0.y);
                        pa[mm][1] = make_float2(v0.z, v0.w);
                        pa[mm][2] = make_float2(v1.x, v1.y);
                        pa[mm][3] = make_float2(v1.z, v1.w);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            pa[mm][k] = (s < ntile && a < K && e0 + k < e_end) ? __ldg(A + (int64_t)a * ld + e0 + k)
                                                                              : make_float2(0.f, 0.f);
                    }
                }
            }
        };
        prefetch(0);
        for (int s = 0; s < ntile; ++s) {
            const int b = s & 1;
            const uint32_t par = (uint32_t)(s >> 1) & 1u;
            // stage b is free once the MMAs of tile s - 2 have completed
            if (s >= 2 && *abort_s == 0 && !mbar_wait_bounded(bar_mma + b, par ^ 1u, NT_WAIT_NS)) *abort_s = 1;
            const uint32_t st = sbase + (b ? C::OFF_ST1 : C::OFF_ST0);
            const int64_t e0 = e_begin + (int64_t)s * NT_E + 4 * q;
            if (FROM_KIN) {
                // angular factors of the groups for event e0 + (j % 4) (groups j / 4, j / 4 + 4, ...)
                {
                    // sin and cos of the event's phi once per event (the four lanes j = e, e + 4,
                    // e + 8, e + 12 of a half-warp share event e), passed by shuffle
                    float s1 = 0.f, c1 = 1.f;
                    if ((j >> 2) == 0) sincosf(pph, &s1, &c1);
                    s1 = __shfl_sync(0xffffffffu, s1, lane & ~12);
                    c1 = __shfl_sync(0xffffffffu, c1, lane & ~12);
                    const float ct = pct;
                    float pcur = 1.f, pprev = 0.f;
                    int jc = 0;
                    for (int g = (j >> 2); g < wt.ng; g += 4) {
                        const int J = s_gJ[g], lam = s_glam[g];
                        for (; jc < J; ++jc) {
                            const float pn = ((2.f * jc + 1.f) * ct * pcur - (float)jc * pprev) * c_nt_inv_int[jc];
                            pprev = pcur;
                            pcur = pn;
                        }
                        const int al = lam < 0 ? -lam : lam;
                        float er = 1.f, ei = 0.f;
                        for (int t = 0; t < al; ++t) {
                            const float tr = er * c1 - ei * s1;
                            ei = er * s1 + ei * c1;
                            er = tr;
                        }
                        if (lam < 0) ei = -ei;
                        sY[(4 * q + (j & 3)) * NT_YS + g] = make_float2(pcur * er, pcur * ei);
                    }
                }
                float m4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) m4[k] = pm[k];
                prefetch(s + 1);
                __syncwarp();
#pragma unroll
                for (int mm = 0; mm < C::MW; ++mm) {
                    const int a = 16 * mm + j;
                    if (a >= KMAX) continue;  // KMAX = 8: half of the residues have no wave
                    const float4 p = s_prm[a];
                    const int g = s_grp[a];
                    float re[4], im[4];
                    // whole quads of events of a wave that exists need no per-event selects
                    const bool full = a < K && e0 + 3 < e_end;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float dr = ((p.x - m4[k]) + p.y) * ((p.x + m4[k]) + p.y);
                        const float inv = __fdividef(1.f, fmaf(dr, dr, p.w));
                        const float t1 = p.z * inv;
                        const float br = dr * t1, bi = p.z * t1;
                        const float2 y = sY[(4 * q + k) * NT_YS + g];
                        re[k] = br * y.x - bi * y.y;
                        im[k] = br * y.y + bi * y.x;
                    }
                    if (!full) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const bool in = a < K && e0 + k < e_end;
                            re[k] = in ? re[k] : 0.f;
                            im[k] = in ? im[k] : 0.f;
                        }
                    }
                    store_row4<KMAX>(st, a, q, re);
                    store_row4<KMAX>(st, KMAX + a, q, im);
                }
                __syncwarp();  // the angular table is rewritten by the next tile
            } else {
#pragma unroll
                for (int mm = 0; mm < C::MW; ++mm) {
                    const int a = 16 * mm + j;
                    if (a >= KMAX) continue;
                    float re[4], im[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        re[k] = pa[mm][k].x;
                        im[k] = pa[mm][k].y;
                    }
                    store_row4<KMAX>(st, a, q, re);
                    store_row4<KMAX>(st, KMAX + a, q, im);
                }
                prefetch(s + 1);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbarrier_arrive_one(bar_fill + b);
            if (s >= 1) drain(s - 1);
        }
        if (ntile >= 1) drain(ntile - 1);
        flush();
    }
    tc_fence_before();
    __syncthreads();
    const bool timeout = *abort_s != 0;
    if (timeout && tid == 0) atomicOr(status, 2);
    // ---- block partial: G = S[0:2K] + S[2K:4K] + S[2K:4K]^T, then Psi (upper triangle)
    float4* bp = part + (int64_t)blockIdx.x * KMAX * KMAX;
    auto S = [&](int r, int c) { const int idx = c * 128 + r; return ff{acc_hi[idx], acc_lo[idx]}; };
    auto G = [&](int r, int c) { return ff_add(ff_add(S(r, c), S(2 * KMAX + r, c)), S(2 * KMAX + c, r)); };
    for (int o = tid; o < K * K; o += NT_THREADS) {
        const int a = o / K, b = o % K;
        if (a > b) continue;
        ff re = ff_add(G(a, b), G(KMAX + a, KMAX + b));
        const ff g2 = G(a, KMAX + b);
        ff im = ff_add(G(KMAX + a, b), ff{-g2.hi, -g2.lo});
        if (timeout || ntile == 0) re = im = ff_zero();
        bp[a * KMAX + b] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TCOLS);
    }
}

template <int KMAX, bool FROM_KIN>
cudaError_t nt_launch(const float2* A, int K, int64_t n, int64_t ld, const float* kin, const WaveTable& wt,
                      float4* part, int* status, int sm_count, cudaStream_t st, int* nblocks) {
    using C = NtCfg<KMAX>;
    auto kern = k_normint_tc<KMAX, FROM_KIN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t tiles = (n + NT_E - 1) / NT_E;
    int64_t nb = sm_count;
    if (nb > tiles) nb = tiles;
    if (nb < 1) nb = 1;
    const int64_t ev_per_block = (tiles + nb - 1) / nb * NT_E;
    nb = (n + ev_per_block - 1) / ev_per_block;
    if (nb < 1) nb = 1;
    kern<<<(unsigned)nb, NT_THREADS, C::SMEM, st>>>(A, K, n, ld, kin, wt, ev_per_block, part, status);
    *nblocks = (int)nb;
    return cudaGetLastError();
}

}  // namespace

bool normint_tc_ok(int K, const float* w, const WaveTable* wt) {
    if (K > 32 || w) return false;
    if (wt && wt->ng > NT_NG) return false;
    return true;
}

cudaError_t launch_normint_tc(const float2* A, int K, int64_t n, int64_t ld, const float* kin, const WaveTable* wt,
                              float4* part, int* status, int sm_count, cudaStream_t st, int* nblocks) {
    const WaveTable w0 = wt ? *wt : WaveTable{};
#define PWA_NT(KM) (kin ? nt_launch<KM, true>(A, K, n, ld, kin, w0, part, status, sm_count, st, nblocks) \
                        : nt_launch<KM, false>(A, K, n, ld, kin, w0, part, status, sm_count, st, nblocks))
    if (K <= 8) return PWA_NT(8);
    if (K <= 16) return PWA_NT(16);
    return PWA_NT(32);
#undef PWA_NT
}

}  // namespace pwa
