// Batched -lnL and gradient for P parameter sets on the tensor cores (one tile shape of the
// batched evaluation, chosen by the autotuner when it is the fastest): the event x wave x start
// contraction of Eq. 3 as two real GEMMs per tile of E = 64 events, in FP32-accurate
// arithmetic emulated with three TF32 products, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (each operand split as x = hi + lo: hi the nearest TF32 value, lo = x - hi exactly, of which the
// tensor cores use the leading 11 bits; the dropped a_lo b_lo and the truncation of lo leave a
// relative error below 2^-20 per product, and the products accumulate in FP32 in tensor memory).
//
// Block: PB = 128 parameter sets (one per tensor-memory lane and per thread) x one chunk of
// events, one block per SM.  Complex numbers are expanded into real rows and columns so that
// each GEMM is a plain real product with both operands K-major:
//
//   GEMM1 (U = A V^T, M = 128 sets, N = 2E, contraction 2 KMAX):
//     D1[p][e + E h] = sum_c V'[p][c] A'[e + E h][c],  V'[p] = (Re V_p | Im V_p),
//     A'[e, h=0] = (Re A_e | -Im A_e),  A'[e, h=1] = (Im A_e | Re A_e)
//     so D1[p][e] = Re u_ep and D1[p][E + e] = Im u_ep.
//   epilogue (thread p, its own lane): I = |u|^2, ln I, w = u / I, split w into TF32 hi / lo and
//     store it into tensor memory as Y[p][c] (c = e: Re w, c = E + e: Im w).
//   GEMM2 (G += W^H-weighted A, M = 128 sets, N = 2 KMAX, contraction 2E, A operand Y from tensor
//     memory):
//     D2[p][a + KMAX g] = sum_c Y[p][c] X[a + KMAX g][c],  X[a, g=0] = (Re A_a | Im A_a) over events,
//     X[a, g=1] = (-Im A_a | Re A_a), so D2[p][a] = sum_e Re(conj(A_ea) w_ep) and
//     D2[p][KMAX + a] = sum_e Im(conj(A_ea) w_ep).
//
// Shared memory holds V' (hi, lo), A' and X (hi, lo; both layouts are written from registers,
// since a transposed TF32 operand is not available) and the low words of the G accumulators;
// tensor memory holds D1 (Y hi overwrites it), Y lo, D2 and the high words of the G
// accumulators.  D2 has two column blocks: hi.hi alone, and the small hi.lo + lo.hi.  They
// accumulate in FP32 in tensor memory over WINDOW tiles (64 events), are added in FP32 (rounded
// to nearest) into registers, and every FF_EVERY windows into the double-single G
// accumulators.  The tensor cores' FP32 accumulation does not round to nearest; at a minimum the
// data sum of the gradient is coherent (about n Psi^T V), so that error adds up over a window
// instead of averaging out: draining every tile keeps it ~1e-8 of the gradient scale, 10x below
// the minimiser's convergence threshold at 2e6 events.  At the end they are written to the
// block's [chunk][P][1 + 2K] partials, the layout of the other tile shapes, so one finalisation
// serves all.  Sum ln I: FP32 per tile and thread, double-single across tiles.  Every wait on the
// tensor cores is bounded; a timeout sets status bit 1 and the block's sets' bad flags, waits
// (bounded) for the MMAs in flight and frees the tensor memory.
#include "nll_common.cuh"
#include "tc.cuh"

#ifndef PWA_TC_WINDOW
#define PWA_TC_WINDOW 1
#endif

namespace pwa {

namespace {

template <int KMAX>
struct TcCfg {
    static constexpr int NC = 256, NT = NC + 32, E = 64, PB = 128;  // 8 compute warps + 1 MMA warp
    static constexpr int C1 = 2 * KMAX;  // GEMM1 contraction
    static constexpr int C2 = 2 * E;     // GEMM2 contraction
    static constexpr int N2 = 2 * KMAX;  // GEMM2 columns
    static constexpr uint32_t SBO1 = 32u * C1, SBO2 = 32u * C2;
    static constexpr uint32_t V_BYTES = (uint32_t)PB * C1 * 4u;
    static constexpr uint32_t A1_BYTES = (uint32_t)(2 * E) * C1 * 4u;
    static constexpr uint32_t X_BYTES = (uint32_t)N2 * C2 * 4u;
    static constexpr uint32_t ACC_BYTES = (uint32_t)N2 * PB * 4u;  // low words of the G accumulators
    static constexpr uint32_t OFF_VH = 0, OFF_VL = V_BYTES, OFF_AH = 2 * V_BYTES, OFF_AL = OFF_AH + A1_BYTES,
                              OFF_XH = OFF_AL + A1_BYTES, OFF_XL = OFF_XH + X_BYTES, OFF_ACC = OFF_XL + X_BYTES,
                              OFF_BAR = OFF_ACC + ACC_BYTES;
    static constexpr uint32_t SMEM_USED = OFF_BAR + 64;
    // at least half of an SM's shared memory, so that one block holds the SM (and its tensor memory)
    static constexpr uint32_t SMEM = SMEM_USED > 118784u ? SMEM_USED : 118784u;
    // tensor-memory columns: D1 (U, then Y hi in place), Y lo, D2 (two column blocks: hi.hi, and
    // hi.lo + lo.hi), the high words of the G accumulators
    static constexpr uint32_t T_D1 = 0, T_YL = 2 * E, T_D2 = 4 * E, T_ACC = T_D2 + 2 * N2, TMEM_COLS = 512;
    // tiles per FP32 accumulation window of G in tensor memory before it is added to the
    // double-single accumulators (the tensor cores' accumulation is not rounded to nearest, so
    // its error grows with the window)
    static constexpr int WINDOW = PWA_TC_WINDOW;
    // windows per double-single update of the G accumulators (FP32 round-to-nearest in between)
    static constexpr int FF_EVERY = 4;
    static constexpr int ITEMS_TOT = E * KMAX / 4;                // load items per tile and layout
    static constexpr int ITEMS = (ITEMS_TOT + NC - 1) / NC;       // per compute thread
    static_assert(KMAX % 8 == 0 && KMAX <= 32, "tensor-core batched kernel: K <= 32");
    static_assert(T_ACC + N2 <= TMEM_COLS, "tensor memory");
    static_assert(OFF_XL == OFF_XH + X_BYTES, "X hi and lo form one operand of 2 N2 rows");
    static_assert(N2 % 16 == 0 && 2 * E <= 256 && 2 * N2 <= 256, "MMA shape");
    static_assert(A1_BYTES >= 2 * PB * sizeof(float4), "end-of-kernel exchange area");
};

constexpr uint64_t TC_WAIT_NS = 1000000000ull;

// named barriers (id 0 is __syncthreads) between the compute warps and the MMA warp; both
// sides wait (bar.sync), so neither can run a barrier instance ahead of the other
constexpr int NB_A = 1;   // A' (and for the first tile X) of the next tile stored
constexpr int NB_Y0 = 2;  // Y of the first half of the tile's events in tensor memory
constexpr int NB_Y1 = 3;  // Y of the second half
constexpr int NB_C = 4;   // compute warps only

__device__ __forceinline__ void nb_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ bool nb_or(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// Warp roles: warps 0-7 (two threads per set: lane quarter warp % 4, event half warp / 4) load
// and store the operand tiles and run the epilogue; warp 8 issues every MMA (one lane).
// Per tile t:
//   MMA warp:     [A'(t) stored] wait GEMM2(t-1) -> GEMM1(t) -> commit g1
//                 [Y of events half 0 stored] GEMM2 k-steps of half 0
//                 [Y of half 1 stored] GEMM2 k-steps of half 1 -> commit g2
//   compute warps: wait g1 -> epilogue half 0 -> (arrive) -> epilogue half 1 -> (arrive)
//                 -> store A'(t+1) -> (arrive) -> wait g2 -> store X(t+1), load tile t+2, drain G
// so GEMM2 of half 0 runs during the epilogue of half 1, and GEMM1(t+1) during the X copy,
// the loads and the drain.  The epilogue writes Y hi over D1 in place; GEMM1(t+1), which
// overwrites D1, waits for GEMM2(t), which reads Y hi.  GEMM2 takes X hi and X lo as one
// operand of 2 N2 rows (hi.hi and hi.lo in one MMA per k-step), then adds lo.hi into the second
// column block.  Every WINDOW tiles the two column blocks are added to the G accumulators (high
// words in tensor memory, low words in shared memory).  A wait that times out sets a block flag;
// from then on no MMA is issued and no mbarrier wait is made, but every named barrier is still
// passed in the same order by both roles, so neither waits on a barrier that the other skips.
template <int KMAX>
__global__ void __launch_bounds__(288, 1) k_nll_tc(const float2* __restrict__ A, int K, int64_t n, int64_t ld,
                                                   const float2* __restrict__ V, int P, int64_t ev_per_chunk,
                                                   float2* __restrict__ part, int* __restrict__ bad, int with_grad,
                                                   int* __restrict__ status) {
    using C = TcCfg<KMAX>;
    constexpr int E = C::E;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 8;
    const int lq = warp & 3, hh = (warp >> 2) & 1;  // tensor-memory lane quarter; event / column half
    const int pl = 32 * lq + lane;                  // this thread's set within the block (its lane)
    const int p0 = blockIdx.y * C::PB;
    const int p = p0 + pl;
    const bool pvalid = !mma_warp && p < P;
    const int NV = 1 + 2 * K;
    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_chunk;
    int64_t e_end = e_begin + ev_per_chunk;
    if (e_end > n) e_end = n;
    const int64_t ntile = e_begin < e_end ? (e_end - e_begin + E - 1) / E : 0;
    uint64_t* bar_g1 = reinterpret_cast<uint64_t*>(tsm + C::OFF_BAR);
    uint64_t* bar_g2 = bar_g1 + 1;
    uint64_t* bar_fin = bar_g1 + 2;
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(tsm + C::OFF_BAR + 24);
    volatile int* abort_s = reinterpret_cast<volatile int*>(tsm + C::OFF_BAR + 28);

    // V' = (Re V | Im V) per set, split into TF32 hi / lo
    for (int idx = tid; idx < C::PB * KMAX; idx += C::NT) {
        const int pp = idx / KMAX, a = idx % KMAX;
        float2 v = make_float2(0.f, 0.f);
        if (a < K && p0 + pp < P) v = V[(int64_t)(p0 + pp) * K + a];
        float h, l;
        tf32_split(v.x, h, l);
        *reinterpret_cast<float*>(tsm + C::OFF_VH + kmaj_off(pp, a, C::SBO1)) = h;
        *reinterpret_cast<float*>(tsm + C::OFF_VL + kmaj_off(pp, a, C::SBO1)) = l;
        tf32_split(v.y, h, l);
        *reinterpret_cast<float*>(tsm + C::OFF_VH + kmaj_off(pp, KMAX + a, C::SBO1)) = h;
        *reinterpret_cast<float*>(tsm + C::OFF_VL + kmaj_off(pp, KMAX + a, C::SBO1)) = l;
    }
    if (warp == 0) tmem_alloc(taddr_s, C::TMEM_COLS);
    if (tid == 0) {
        mbar_init(bar_g1, 1);
        mbar_init(bar_g2, 1);
        mbar_init(bar_fin, 1);
        *abort_s = 0;
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *taddr_s;
    const uint32_t lane_t = tmem + ((uint32_t)(32 * lq) << 16);  // this warp's 32 lanes
    const uint32_t sbase = smem_u32(tsm);
    const bool grad = with_grad != 0;

    ff lsum = ff_zero();
    bool mybad = false, drained = false;
    int since_ff = 0;

    if (mma_warp) {
        // ================================================================ MMA warp
        const uint64_t dVh = umma_desc(sbase + C::OFF_VH, 128u, C::SBO1), dVl = umma_desc(sbase + C::OFF_VL, 128u, C::SBO1);
        const uint64_t dAh = umma_desc(sbase + C::OFF_AH, 128u, C::SBO1), dAl = umma_desc(sbase + C::OFF_AL, 128u, C::SBO1);
        const uint64_t dXh = umma_desc(sbase + C::OFF_XH, 128u, C::SBO2);
        constexpr uint32_t id1 = umma_idesc_tf32(128, 2 * E);
        constexpr uint32_t idw = umma_idesc_tf32(128, 2 * C::N2), idn = umma_idesc_tf32(128, C::N2);
        int win = 0;
        for (int64_t t = 0; t < ntile; ++t) {
            nb_sync(NB_A, C::NT);
            bool ab = *abort_s != 0;
            if (!ab && grad && t > 0 && !mbar_wait_bounded(bar_g2, (uint32_t)((t - 1) & 1), TC_WAIT_NS)) {
                ab = true;
                *abort_s = 1;
            }
            tc_fence_after();
            if (!ab && lane == 0) {
                // U = V' A'^T: the small products (hi, lo) and (lo, hi) first, then (hi, hi), so
                // that most accumulation steps add to a small running sum (the tensor cores'
                // FP32 accumulation does not round to nearest)
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s)
                    mma_tf32_ss(tmem + C::T_D1, dVh + 16u * s, dAl + 16u * s, id1, s > 0 ? 1u : 0u);
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s) mma_tf32_ss(tmem + C::T_D1, dVl + 16u * s, dAh + 16u * s, id1, 1u);
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s) mma_tf32_ss(tmem + C::T_D1, dVh + 16u * s, dAh + 16u * s, id1, 1u);
                umma_commit(bar_g1);
            }
            __syncwarp();
            if (grad) {
                const bool fresh = win == 0;
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    nb_sync(hf == 0 ? NB_Y0 : NB_Y1, C::NT);
                    ab = ab || *abort_s != 0;
                    tc_fence_after();
                    if (!ab && lane == 0) {
                        // contraction c = (Re | Im) x 64 events; this half's events are 16 hf + 0..15
                        // and 32 + 16 hf + 0..15, i.e. k-steps 4 j + 2 hf + {0, 1}
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int d = 0; d < 2; ++d) {
                                const uint32_t s = 4 * j + 2 * hf + d;
                                mma_tf32_ts(tmem + C::T_D2, tmem + C::T_D1 + 8u * s, dXh + 16u * s, idw,
                                            (fresh && hf == 0 && j == 0 && d == 0) ? 0u : 1u);
                            }
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int d = 0; d < 2; ++d) {
                                const uint32_t s = 4 * j + 2 * hf + d;
                                mma_tf32_ts(tmem + C::T_D2 + C::N2, tmem + C::T_YL + 8u * s, dXh + 16u * s, idn, 1u);
                            }
                        if (hf == 1) umma_commit(bar_g2);
                    }
                    __syncwarp();
                }
                if (++win == C::WINDOW || t + 1 == ntile) win = 0;
            }
        }
        // every MMA of this warp has completed (bounded) before the tensor memory is released
        if (lane == 0) umma_commit(bar_fin);
        __syncwarp();
        if (!mbar_wait_bounded(bar_fin, 0, TC_WAIT_NS)) *abort_s = 1;
    } else {
        // ================================================================ compute warps
        float2 ra[C::ITEMS][4];
        float4 rx[C::ITEMS][2];
        // two register images of the same K x E tile:
        //  ra: item (event e, waves 4 aq .. 4 aq + 3) for A'  (a warp reads 32 events of one wave row)
        //  rx: item (wave a, events 4 eq .. 4 eq + 3) for X   (8 waves x 4 quads per warp)
        auto load_tile = [&](int64_t e0) {
#pragma unroll
            for (int i = 0; i < C::ITEMS; ++i) {
                const int j = tid + C::NC * i;
                if (j < C::ITEMS_TOT) {
                    const int e = j % E, aq = j / E;
                    const int64_t ge = e0 + e;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int a = 4 * aq + q;
                        ra[i][q] = (a < K && ge < e_end) ? __ldg(A + a * ld + ge) : make_float2(0.f, 0.f);
                    }
                }
                if (grad && j < C::ITEMS_TOT) {
                    const int blk = j >> 5, ln = j & 31;
                    const int a = (blk % (KMAX / 8)) * 8 + (ln & 7);
                    const int eq = (blk / (KMAX / 8)) * 4 + (ln >> 3);
                    const int64_t ge = e0 + 4 * eq;
                    float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
                    if (a < K) {
                        const float2* src = A + a * ld + ge;
                        if (ge + 3 < e_end) {
                            x0 = __ldg(reinterpret_cast<const float4*>(src));
                            x1 = __ldg(reinterpret_cast<const float4*>(src + 2));
                        } else {
                            float2 tq[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) tq[k] = ge + k < e_end ? __ldg(src + k) : make_float2(0.f, 0.f);
                            x0 = make_float4(tq[0].x, tq[0].y, tq[1].x, tq[1].y);
                            x1 = make_float4(tq[2].x, tq[2].y, tq[3].x, tq[3].y);
                        }
                    }
                    rx[i][0] = x0;
                    rx[i][1] = x1;
                }
            }
        };
        auto st4 = [&](uint32_t off, float a, float b, float c, float d) {
            *reinterpret_cast<float4*>(tsm + off) = make_float4(a, b, c, d);
        };
        // registers -> A' or X (hi and lo).  Each 16-byte store of a warp phase (8 lanes) hits 8
        // different rows of one core-matrix column: A' rows e = 8 consecutive events, X rows a =
        // 8 consecutive waves.
        auto store_a1 = [&]() {
#pragma unroll
            for (int i = 0; i < C::ITEMS; ++i) {
                const int j = tid + C::NC * i;
                if (j < C::ITEMS_TOT) {
                    const int e = j % E, aq = j / E;
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        tf32_split(ra[i][q].x, rh[q], rl[q]);
                        tf32_split(ra[i][q].y, ih[q], il[q]);
                    }
                    const uint32_t re0 = kmaj_off(e, 4 * aq, C::SBO1), im0 = kmaj_off(e, KMAX + 4 * aq, C::SBO1);
                    const uint32_t re1 = kmaj_off(E + e, 4 * aq, C::SBO1), im1 = kmaj_off(E + e, KMAX + 4 * aq, C::SBO1);
                    st4(C::OFF_AH + re0, rh[0], rh[1], rh[2], rh[3]);
                    st4(C::OFF_AH + im0, -ih[0], -ih[1], -ih[2], -ih[3]);
                    st4(C::OFF_AH + re1, ih[0], ih[1], ih[2], ih[3]);
                    st4(C::OFF_AH + im1, rh[0], rh[1], rh[2], rh[3]);
                    st4(C::OFF_AL + re0, rl[0], rl[1], rl[2], rl[3]);
                    st4(C::OFF_AL + im0, -il[0], -il[1], -il[2], -il[3]);
                    st4(C::OFF_AL + re1, il[0], il[1], il[2], il[3]);
                    st4(C::OFF_AL + im1, rl[0], rl[1], rl[2], rl[3]);
                }
            }
        };
        auto store_x = [&]() {
#pragma unroll
            for (int i = 0; i < C::ITEMS; ++i) {
                const int j = tid + C::NC * i;
                if (j < C::ITEMS_TOT) {
                    const int blk = j >> 5, ln = j & 31;
                    const int a = (blk % (KMAX / 8)) * 8 + (ln & 7);
                    const int eq = (blk / (KMAX / 8)) * 4 + (ln >> 3);
                    const float xr[4] = {rx[i][0].x, rx[i][0].z, rx[i][1].x, rx[i][1].z};
                    const float xi[4] = {rx[i][0].y, rx[i][0].w, rx[i][1].y, rx[i][1].w};
                    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        tf32_split(xr[q], rh[q], rl[q]);
                        tf32_split(xi[q], ih[q], il[q]);
                    }
                    const uint32_t g0r = kmaj_off(a, 4 * eq, C::SBO2), g0i = kmaj_off(a, E + 4 * eq, C::SBO2);
                    const uint32_t g1r = kmaj_off(KMAX + a, 4 * eq, C::SBO2), g1i = kmaj_off(KMAX + a, E + 4 * eq, C::SBO2);
                    st4(C::OFF_XH + g0r, rh[0], rh[1], rh[2], rh[3]);
                    st4(C::OFF_XH + g0i, ih[0], ih[1], ih[2], ih[3]);
                    st4(C::OFF_XH + g1r, -ih[0], -ih[1], -ih[2], -ih[3]);
                    st4(C::OFF_XH + g1i, rh[0], rh[1], rh[2], rh[3]);
                    st4(C::OFF_XL + g0r, rl[0], rl[1], rl[2], rl[3]);
                    st4(C::OFF_XL + g0i, il[0], il[1], il[2], il[3]);
                    st4(C::OFF_XL + g1r, -il[0], -il[1], -il[2], -il[3]);
                    st4(C::OFF_XL + g1i, rl[0], rl[1], rl[2], rl[3]);
                }
            }
        };
        float* acc_lo = reinterpret_cast<float*>(tsm + C::OFF_ACC) + pl;  // [column][PB]
        // Every tile the two column blocks of D2 are added in FP32 (round to nearest, on the CUDA
        // cores) into racc; every FF_EVERY tiles racc enters the double-single G accumulators (hi
        // in tensor memory, lo in shared memory).  The two threads of a lane take alternate groups
        // of 16 columns (racc[16 i + k]: group hh + 2 i).
        constexpr int NGRP = (C::N2 / 16 + 1) / 2;  // column groups per thread
        float racc[16 * NGRP];
#pragma unroll
        for (int v = 0; v < 16 * NGRP; ++v) racc[v] = 0.f;
        auto drain_tile = [&]() {
#pragma unroll
            for (int i = 0; i < NGRP; ++i) {
                const int q = hh + 2 * i;
                if (q < C::N2 / 16) {
                    float d0[16], d1[16];
                    tmem_ld16(lane_t + C::T_D2 + 16 * q, d0);
                    tmem_ld16(lane_t + C::T_D2 + C::N2 + 16 * q, d1);
                    tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; ++k) racc[16 * i + k] += d0[k] + d1[k];
                }
            }
        };
        auto flush = [&](bool first) {
#pragma unroll
            for (int i = 0; i < NGRP; ++i) {
                const int q = hh + 2 * i;
                if (q < C::N2 / 16) {
                    float ah[16];
                    tmem_ld16(lane_t + C::T_ACC + 16 * q, ah);
                    tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        float* lo = acc_lo + (16 * q + k) * C::PB;
                        const ff r = ff_add_f(first ? ff_zero() : ff{ah[k], *lo}, racc[16 * i + k]);
                        ah[k] = r.hi;
                        *lo = r.lo;
                        racc[16 * i + k] = 0.f;
                    }
                    tmem_st16(lane_t + C::T_ACC + 16 * q, ah);
                }
            }
            tmem_wait_st();
        };
        // I, ln I, W = U / I for the 16 events of column group q -> Y (hi over U, lo)
        auto epilogue = [&](int q, int64_t nvalid, float& lt) {
            float ur[16], ui[16];
            tmem_ld16(lane_t + C::T_D1 + 16 * q, ur);
            tmem_ld16(lane_t + C::T_D1 + E + 16 * q, ui);
            tmem_wait_ld();
            float yrh[16], yrl[16], yih[16], yil[16];
            if (nvalid >= 16 * q + 16) {
                // all 16 events inside the chunk: no per-event selects.  A zero or non-finite
                // intensity makes ln I, and so the group's sum, non-finite: one test per group
                // flags the set (its Y, and so only its own row of G, may then hold NaN; a
                // flagged set's results are not used)
                float lg16 = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float I = fmaf(ur[k], ur[k], ui[k] * ui[k]);
                    lg16 += __logf(I);
                    const float rc = __fdividef(1.f, I);
                    tf32_split(ur[k] * rc, yrh[k], yrl[k]);
                    tf32_split(ui[k] * rc, yih[k], yil[k]);
                }
                mybad |= !(fabsf(lg16) < INFINITY);
                lt += lg16;
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    // branch-free, so that the 16 events interleave: events past the end or sets past
                    // P contribute nothing; a zero or non-finite intensity flags the set
                    const float I = fmaf(ur[k], ur[k], ui[k] * ui[k]);
                    const bool valid = 16 * q + k < nvalid;
                    const bool ok = intensity_ok(I);
                    mybad |= valid && !ok;
                    const bool use = valid && ok;
                    const float Iu = use ? I : 1.f;
                    // both functions evaluated unconditionally (a select, not a branch, picks the result)
                    const float lgu = __logf(Iu);
                    const float rcu = __fdividef(1.f, Iu);
                    lt += use ? lgu : 0.f;
                    const float rc = use ? rcu : 0.f;
                    tf32_split(use ? ur[k] * rc : 0.f, yrh[k], yrl[k]);
                    tf32_split(use ? ui[k] * rc : 0.f, yih[k], yil[k]);
                }
            }
            if (grad) {
                tmem_st16(lane_t + C::T_D1 + 16 * q, yrh);  // Y hi over U, in place
                tmem_st16(lane_t + C::T_D1 + E + 16 * q, yih);
                tmem_st16(lane_t + C::T_YL + 16 * q, yrl);
                tmem_st16(lane_t + C::T_YL + E + 16 * q, yil);
                tmem_wait_st();
            }
        };
        bool ab = false;
        // block-uniform (compute warps) wait on an MMA group; a timeout sets the abort flag
        auto wait_mma = [&](uint64_t* b, uint32_t parity) {
            const bool ok = ab || mbar_wait_bounded(b, parity, TC_WAIT_NS);
            if (nb_or(NB_C, C::NC, !ok || *abort_s != 0)) {
                ab = true;
                if (tid == 0) *abort_s = 1;
            }
            tc_fence_after();
        };
        int win = 0;
        if (ntile > 0) {
            load_tile(e_begin);
            store_a1();
            if (grad) store_x();
            fence_proxy_async_smem();
            nb_sync(NB_A, C::NT);
            if (ntile > 1) load_tile(e_begin + E);
        }
        for (int64_t t = 0; t < ntile; ++t) {
            const int64_t e0 = e_begin + t * E;
            wait_mma(bar_g1, (uint32_t)(t & 1));  // GEMM1(t)
            const int64_t nvalid = (pvalid && !ab) ? (e_end - e0) : 0;
            float lt = 0.f;
#pragma unroll 1
            for (int hf = 0; hf < 2; ++hf) {
                if (!ab) epilogue(2 * hh + hf, nvalid, lt);
                tc_fence_before();
                if (grad) nb_sync(hf == 0 ? NB_Y0 : NB_Y1, C::NT);
            }
            lsum = ff_add_f(lsum, lt);
            if (t + 1 < ntile) {
                if (!ab) store_a1();  // A'(t + 1): GEMM1(t) has completed
                fence_proxy_async_smem();
                nb_sync(NB_A, C::NT);
            }
            if (grad) wait_mma(bar_g2, (uint32_t)(t & 1));  // GEMM2(t)
            if (t + 1 < ntile) {
                if (grad && !ab) store_x();  // X(t + 1): GEMM2(t) has completed
                if (t + 2 < ntile) load_tile(e0 + 2 * E);
                fence_proxy_async_smem();
            }
            if (grad && (++win == C::WINDOW || t + 1 == ntile)) {
                if (!ab) {
                    drain_tile();
                    if (++since_ff == C::FF_EVERY || t + 1 == ntile) {
                        flush(!drained);
                        drained = true;
                        since_ff = 0;
                    }
                }
                win = 0;
            }
        }
    }
    // ---- results: combine the two threads of each set (the A' area is free now)
    tc_fence_before();
    __syncthreads();
    const bool timeout = *abort_s != 0;
    if (timeout && tid == 0) atomicOr(status, 2);
    float4* xch = reinterpret_cast<float4*>(tsm + C::OFF_AH);
    if (!mma_warp && hh == 1) xch[pl] = make_float4(lsum.hi, lsum.lo, mybad ? 1.f : 0.f, 0.f);
    __syncthreads();
    float2* prow = part + ((int64_t)blockIdx.x * P + p) * NV;  // this set's partials (valid if pvalid)
    if (!mma_warp && hh == 0 && pvalid) {
        const float4 o = xch[pl];
        lsum = ff_add(lsum, ff{o.x, o.y});
        prow[0] = make_float2(lsum.hi, lsum.lo);
        if (mybad || o.z != 0.f || timeout) bad[p] = 1;
    }
    // G: both threads of a set write their column groups
    if (!mma_warp && grad) {
        const float* acc_lo = reinterpret_cast<const float*>(tsm + C::OFF_ACC) + pl;
#pragma unroll 1
        for (int q = hh; q < C::N2 / 16; q += 2) {
            float ah[16];
            tmem_ld16(lane_t + C::T_ACC + 16 * q, ah);
            tmem_wait_ld();
            if (pvalid) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int col = 16 * q + k;
                    const int a = col % KMAX, g = col / KMAX;
                    if (a < K)
                        prow[1 + 2 * a + g] =
                            (drained && !timeout) ? make_float2(ah[k], acc_lo[col * C::PB]) : make_float2(0.f, 0.f);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int KMAX>
cudaError_t tc_launch_k(const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                        size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count, cudaStream_t st,
                        int* nchunk_out) {
    using C = TcCfg<KMAX>;
    auto kern = k_nll_tc<KMAX>;
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
    kern<<<grid, C::NT, C::SMEM, st>>>(A, K, n, ld, V, P, epc, (float2*)ws, bad, with_grad, status);
    *nchunk_out = nchunk;
    return cudaGetLastError();
}

}  // namespace

bool tc_batched_ok(int kmax) { return kmax == 8 || kmax == 16 || kmax == 32; }

cudaError_t tc_batched_launch(int kmax, const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                              size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count, cudaStream_t st,
                              int* nchunk) {
    switch (kmax) {
        case 8: return tc_launch_k<8>(A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk);
        case 16: return tc_launch_k<16>(A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk);
        case 32: return tc_launch_k<32>(A, K, n, ld, V, P, ws, ws_bytes, bad, status, with_grad, sm_count, st, nchunk);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pwa
