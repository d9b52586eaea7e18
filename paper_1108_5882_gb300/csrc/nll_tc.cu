// Batched -lnL and gradient for P parameter sets on the tensor cores (one tile shape of the
// batched evaluation, chosen by the autotuner when it is the fastest): the event x wave x start
// contraction of Eq. 3 as two real GEMMs per tile of E = 48 events, in FP32-accurate
// arithmetic emulated with three TF32 products, a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (each operand split as x = hi + lo, hi the nearest TF32 value and lo the nearest TF32 value of
// x - hi; the dropped a_lo b_lo and the rounding of lo leave a relative error near 2^-21 per
// product, and the products accumulate in FP32 in tensor memory).
//
// Block: PB = 128 parameter sets (one per tensor-memory lane, two threads per set) x one chunk
// of events, one block per SM.  Complex numbers are expanded into real rows and columns so
// that each GEMM is a plain real product with both operands K-major:
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
// GEMM2's MMAs have N = 2 N2 >= 128 (the hi and lo parts of X stacked as one operand) where K
// allows it; GEMM1's have N = 2E = 96, a compromise: an MMA instruction costs at least ~60
// cycles whatever its N (N = 128 is the smallest at the tensor cores' arithmetic rate), but
// 48-event tiles let tensor memory hold four regions of 2E columns beside D2.  Shared memory
// holds V', A' and X (hi, lo; both layouts are written from registers, since a transposed TF32
// operand is not available).  The four regions rotate over the tiles (tile t: U in region
// 2t mod 4, Y hi written over it in place, Y lo in region 2t + 1 mod 4), so GEMM1(t + 1) writes
// the regions of tile t - 1 while the epilogue of tile t runs, and the epilogue writes Y lo(t)
// into a region whose last reader, GEMM2(t - 2), has completed: it waits for GEMM2(t - 1) only
// to drain D2.  D2 has two column blocks: hi.hi alone, and the small hi.lo + lo.hi.  They
// accumulate in FP32 in tensor memory over one tile, are added in FP32 (rounded to nearest)
// into registers, and every FF_EVERY tiles into the double-single G accumulators (high words in
// registers, low words in shared memory).  The tensor cores' FP32 accumulation does not round
// to nearest; at a minimum the data sum of the gradient is coherent (about n Psi^T V), so that
// error adds up over the accumulation instead of averaging out: draining every tile keeps it
// ~1e-8 of the gradient scale, 10x below the minimiser's convergence threshold at 2e6 events.
// At the end the sums are written to the block's [chunk][P][1 + 2K] partials, the layout of the
// other tile shapes, so one finalisation serves all.  Sum ln I: FP32 per tile and thread,
// double-single across tiles.
//
// The compute warps signal the MMA warp by mbarrier arrivals (they never wait for it to issue,
// which blocks while the tensor cores' queue is full), the MMA warp signals them by
// tcgen05.commit.  Every wait is bounded; a timeout sets an abort flag, after which no MMA is
// issued, no tensor memory is touched and no wait is made, but every arrival and commit is still
// made, so neither side waits for a phase the other skips.  A timeout sets status bit 1 and the
// block's sets' bad flags; the tensor memory is freed after a bounded wait for the MMAs in flight.
#include "nll_common.cuh"
#include "tc.cuh"

namespace pwa {

namespace {

template <int KMAX>
struct TcCfg {
    // 8 epilogue warps, 1 MMA warp, 3 operand warps
    static constexpr int NC = 256, NL = 96, NT = NC + 32 + NL, E = 48, PB = 128;
    static constexpr int NCW = NC / 32, NLW = NL / 32;  // arrivals per phase
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
    // tensor-memory columns: four rotating regions of 2E (U, then Y hi in place; Y lo), D2 (two
    // column blocks: hi.hi, and hi.lo + lo.hi)
    static constexpr uint32_t NREG = 4, T_REG = 2 * E, T_D2 = NREG * T_REG, TMEM_COLS = 512;
    static constexpr int NQ = E / 16;  // epilogue quarters of 8 events per thread
    // tiles per double-single update of the G accumulators (FP32 round-to-nearest in between)
    static constexpr int FF_EVERY = 8;
    static constexpr int ITEMS_TOT = E * KMAX / 4;                // load items per tile and layout
    static constexpr int ITEMS = (ITEMS_TOT + NL - 1) / NL;       // per operand thread
    static constexpr int NGRP = (N2 / 16 + 1) / 2;               // 16-column groups of G per thread
    static_assert(KMAX % 8 == 0 && KMAX <= 32, "tensor-core batched kernel: K <= 32");
    static_assert(T_D2 + 2 * N2 <= TMEM_COLS, "tensor memory");
    static_assert(SMEM_USED <= 232448u, "shared memory");
    static_assert(OFF_XL == OFF_XH + X_BYTES, "X hi and lo form one operand of 2 N2 rows");
    static_assert(N2 % 16 == 0 && (2 * E) % 16 == 0 && 2 * E <= 256 && 2 * N2 <= 256, "MMA shape");
    static_assert(E % 16 == 0 && (E * KMAX / 4) % 32 == 0, "whole 8-event quarters; whole warps of load items");
    static_assert(A1_BYTES >= 2 * PB * sizeof(float4), "end-of-kernel exchange area");
};

constexpr uint64_t TC_WAIT_NS = 1000000000ull;

// Warp roles: warps 0-7 (two threads per set: lane quarter warp % 4, event half warp / 4) run
// the epilogue; warp 8 issues every MMA (one lane); warps 9-11 load the amplitude tiles and store
// the operands A' and X (hi, lo) into shared memory.
// Per tile t (u_t = region 2t mod 4 holds U(t), then Y hi(t); l_t = region 2t + 1 mod 4 holds
// Y lo(t); u_{t+2} = u_t, l_{t+2} = l_t):
//   MMA warp:      wait a_ready(t + 1), wait g2(t - 1) [u_{t+1} = u_{t-1} free]
//                  -> GEMM1(t + 1) into u_{t+1} -> commit g1
//                  wait y_ready(t) [Y(t), X(t) stored, D2 drained] -> GEMM2(t) -> commit g2
//   operand warps: wait g1(t) -> store A'(t + 1) (GEMM1(t) has read A'(t)) -> arrive a_ready
//                  -> wait g2(t - 1) (GEMM2(t - 1) has read X(t - 1)) -> store X(t) -> arrive
//                  y_ready -> load the registers of tiles t + 2 (A') and t + 1 (X)
//   epilogue warps: wait g1(t) -> arrive a_ready -> epilogue and Y of the tile in three quarters
//                  of 8 events (l_t = l_{t-2}: GEMM1(t) was issued after GEMM2(t - 2) completed)
//                  -> wait g2(t - 1) (D2 complete) -> drain D2 -> arrive y_ready
// Tensor-core order: ... GEMM2(t - 1), GEMM1(t + 1), GEMM2(t), GEMM1(t + 2) ...; the epilogue of
// tile t overlaps GEMM2(t - 1) and GEMM1(t + 1).  Phase discipline: every mbarrier completes once per tile, and
// each waiter waits for the oldest phase it has not seen, which cannot be overtaken: the next
// completion needs an arrival or an issue that comes after this wait (every warp that waits on
// g1 arrives on a_ready afterwards, every warp that waits on g2 arrives on y_ready afterwards).
template <int KMAX>
__global__ void __launch_bounds__(384, 1) k_nll_tc(const float2* __restrict__ A, int K, int64_t n, int64_t ld,
                                                   const float2* __restrict__ V, int P, int64_t ev_per_chunk,
                                                   float2* __restrict__ part, int* __restrict__ bad, int with_grad,
                                                   int* __restrict__ status) {
    using C = TcCfg<KMAX>;
    constexpr int E = C::E;
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool compute = warp < 8, mma_warp = warp == 8;  // warps 9 to 11 stage the operands
    const int lq = warp & 3, hh = (warp >> 2) & 1;  // tensor-memory lane quarter; event / column half
    const int pl = 32 * lq + lane;                  // this thread's set within the block (its lane)
    const int p0 = blockIdx.y * C::PB;
    const int p = p0 + pl;
    const bool pvalid = compute && p < P;
    const int NV = 1 + 2 * K;
    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_chunk;
    int64_t e_end = e_begin + ev_per_chunk;
    if (e_end > n) e_end = n;
    const int64_t ntile = e_begin < e_end ? (e_end - e_begin + E - 1) / E : 0;
    uint64_t* bar_g1 = reinterpret_cast<uint64_t*>(tsm + C::OFF_BAR);
    uint64_t* bar_g2 = bar_g1 + 1;
    // A' of the next tile stored (operand warps), the epilogue warps past their wait for the
    // current GEMM1 (one arrival per warp)
    uint64_t* bar_a = bar_g1 + 2;
    uint64_t* bar_y = bar_g1 + 3;  // Y and X of the tile stored, D2 drained (one arrival per epilogue and operand warp)
    uint64_t* bar_fin = bar_g1 + 4;
    uint32_t* taddr_s = reinterpret_cast<uint32_t*>(tsm + C::OFF_BAR + 40);
    volatile int* abort_s = reinterpret_cast<volatile int*>(tsm + C::OFF_BAR + 44);

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
    for (int idx = tid; idx < C::N2 * C::PB; idx += C::NT) reinterpret_cast<float*>(tsm + C::OFF_ACC)[idx] = 0.f;
    if (warp == 0) tmem_alloc(taddr_s, C::TMEM_COLS);
    if (tid == 0) {
        mbar_init(bar_g1, 1);
        mbar_init(bar_g2, 1);
        mbar_init(bar_a, C::NCW + C::NLW);
        mbar_init(bar_y, C::NCW + C::NLW);
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
    // bounded wait; after a timeout (here or on the other side) no further wait is made
    auto wait_or_abort = [&](uint64_t* b, uint32_t parity) {
        if (*abort_s != 0) return false;
        if (!mbar_wait_bounded(b, parity, TC_WAIT_NS)) {
            *abort_s = 1;
            return false;
        }
        tc_fence_after();
        return true;
    };
    auto region = [&](int64_t t, int which) {  // which 0: u_t, 1: l_t
        return (uint32_t)((2 * t + which) % C::NREG) * C::T_REG;
    };

    ff lsum = ff_zero();
    bool mybad = false;
    // double-single G accumulators of this thread's column groups: high words in registers, low
    // words in shared memory ([column][PB])
    float ghi[16 * C::NGRP];
#pragma unroll
    for (int v = 0; v < 16 * C::NGRP; ++v) ghi[v] = 0.f;
    float* acc_lo = reinterpret_cast<float*>(tsm + C::OFF_ACC) + pl;
    auto glo = [&](int i, int k) -> float& { return acc_lo[(16 * (hh + 2 * i) + k) * C::PB]; };

    if (mma_warp) {
        // ================================================================ MMA warp
        const uint64_t dVh = umma_desc(sbase + C::OFF_VH, 128u, C::SBO1), dVl = umma_desc(sbase + C::OFF_VL, 128u, C::SBO1);
        const uint64_t dAh = umma_desc(sbase + C::OFF_AH, 128u, C::SBO1), dAl = umma_desc(sbase + C::OFF_AL, 128u, C::SBO1);
        const uint64_t dXh = umma_desc(sbase + C::OFF_XH, 128u, C::SBO2);
        constexpr uint32_t id1 = umma_idesc_tf32(128, 2 * E);
        constexpr uint32_t idw = umma_idesc_tf32(128, 2 * C::N2), idn = umma_idesc_tf32(128, C::N2);
        // U = V' A'^T into region d: the small products (hi, lo) and (lo, hi) first, then (hi, hi),
        // so that most accumulation steps add to a small running sum (the tensor cores' FP32
        // accumulation does not round to nearest)
        auto gemm1 = [&](uint32_t d) {
            if (*abort_s == 0 && lane == 0) {
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s) mma_tf32_ss(d, dVh + 16u * s, dAl + 16u * s, id1, s > 0 ? 1u : 0u);
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s) mma_tf32_ss(d, dVl + 16u * s, dAh + 16u * s, id1, 1u);
#pragma unroll
                for (int s = 0; s < C::C1 / 8; ++s) mma_tf32_ss(d, dVh + 16u * s, dAh + 16u * s, id1, 1u);
            }
            if (lane == 0) umma_commit(bar_g1);
            __syncwarp();
        };
        if (ntile > 0) {
            wait_or_abort(bar_a, 0);  // A'(0)
            gemm1(tmem + region(0, 0));
        }
        for (int64_t t = 0; t < ntile; ++t) {
            if (t + 1 < ntile) {
                wait_or_abort(bar_a, (uint32_t)((t + 1) & 1));                // A'(t + 1)
                if (grad && t >= 1) wait_or_abort(bar_g2, (uint32_t)((t - 1) & 1));  // region u_{t+1} = u_{t-1} read
                gemm1(tmem + region(t + 1, 0));
            }
            if (grad) {
                wait_or_abort(bar_y, (uint32_t)(t & 1));  // Y(t), X(t), D2 drained
                if (*abort_s == 0 && lane == 0) {
                    // G = Y X^T over the contraction c = (Re | Im) x E events: hi.hi and hi.lo in
                    // one MMA per k-step (X hi and lo as one operand of 2 N2 rows), then lo.hi
                    // into the second column block; the first k-step overwrites D2
                    const uint32_t yh = tmem + region(t, 0), yl = tmem + region(t, 1);
#pragma unroll
                    for (int s = 0; s < C::C2 / 8; ++s)
                        mma_tf32_ts(tmem + C::T_D2, yh + 8u * s, dXh + 16u * s, idw, s > 0 ? 1u : 0u);
#pragma unroll
                    for (int s = 0; s < C::C2 / 8; ++s)
                        mma_tf32_ts(tmem + C::T_D2 + C::N2, yl + 8u * s, dXh + 16u * s, idn, 1u);
                }
                if (lane == 0) umma_commit(bar_g2);
                __syncwarp();
            }
        }
        // every MMA of this warp has completed (bounded) before the tensor memory is released
        if (lane == 0) umma_commit(bar_fin);
        __syncwarp();
        if (!mbar_wait_bounded(bar_fin, 0, TC_WAIT_NS)) *abort_s = 1;
    } else if (compute) {
        // ================================================================ epilogue warps
        // Every tile the two column blocks of D2 are added in FP32 (round to nearest, on the CUDA
        // cores) into racc; every FF_EVERY tiles racc enters the double-single G accumulators.
        // The two threads of a lane take alternate groups of 16 columns (racc[16 i + k]: group
        // hh + 2 i).
        float racc[16 * C::NGRP];
#pragma unroll
        for (int v = 0; v < 16 * C::NGRP; ++v) racc[v] = 0.f;
        int since_ff = 0;
        auto flush = [&]() {
#pragma unroll
            for (int i = 0; i < C::NGRP; ++i) {
                if (hh + 2 * i < C::N2 / 16) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const ff r = ff_add_f(ff{ghi[16 * i + k], glo(i, k)}, racc[16 * i + k]);
                        ghi[16 * i + k] = r.hi;
                        glo(i, k) = r.lo;
                        racc[16 * i + k] = 0.f;
                    }
                }
            }
        };
        auto drain = [&]() {
#pragma unroll
            for (int i = 0; i < C::NGRP; ++i) {
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
            if (++since_ff == C::FF_EVERY) {
                flush();
                since_ff = 0;
            }
        };
        // I, ln I, W = U / I for the 8 events (E/2) hh + 8 qq + 0..7 of the tile (U in region u) ->
        // registers yr / yi (hi, lo); events past the end of the chunk or sets past P give 0
        auto epi_math = [&](uint32_t u, int qq, int64_t nvalid, float& lt, float (&yrh)[8], float (&yrl)[8],
                            float (&yih)[8], float (&yil)[8]) {
            const int c0 = (E / 2) * hh + 8 * qq;
            float ur[8], ui[8];
            tmem_ld8(lane_t + u + c0, ur);
            tmem_ld8(lane_t + u + E + c0, ui);
            tmem_wait_ld();
            if (nvalid >= c0 + 8) {
                // all 8 events inside the chunk: no per-event selects.  A zero or non-finite
                // intensity makes ln I, and so the group's sum, non-finite: one test per group
                // flags the set (its Y, and so only its own row of G, may then hold NaN; a
                // flagged set's results are not used)
                float lg = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float I = fmaf(ur[k], ur[k], ui[k] * ui[k]);
                    lg += __logf(I);
                    const float rc = __fdividef(1.f, I);
                    tf32_split(ur[k] * rc, yrh[k], yrl[k]);
                    tf32_split(ui[k] * rc, yih[k], yil[k]);
                }
                mybad |= !(fabsf(lg) < INFINITY);
                lt += lg;
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    // branch-free: a select, not a branch, picks each result
                    const float I = fmaf(ur[k], ur[k], ui[k] * ui[k]);
                    const bool valid = c0 + k < nvalid;
                    const bool ok = intensity_ok(I);
                    mybad |= valid && !ok;
                    const bool use = valid && ok;
                    const float Iu = use ? I : 1.f;
                    const float lgu = __logf(Iu);
                    const float rcu = __fdividef(1.f, Iu);
                    lt += use ? lgu : 0.f;
                    const float rc = use ? rcu : 0.f;
                    tf32_split(use ? ur[k] * rc : 0.f, yrh[k], yrl[k]);
                    tf32_split(use ? ui[k] * rc : 0.f, yih[k], yil[k]);
                }
            }
        };
        auto epi_store = [&](uint32_t u, uint32_t l, int qq, const float (&yrh)[8], const float (&yrl)[8],
                             const float (&yih)[8], const float (&yil)[8]) {
            const int c0 = (E / 2) * hh + 8 * qq;
            tmem_st8(lane_t + u + c0, yrh);  // Y hi over U, in place
            tmem_st8(lane_t + u + E + c0, yih);
            tmem_st8(lane_t + l + c0, yrl);
            tmem_st8(lane_t + l + E + c0, yil);
        };
        auto arrive = [&](uint64_t* b) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbarrier_arrive_one(b);
        };
        // The epilogue warps also arrive on a_ready, once before the first tile and once after
        // each wait for GEMM1(t), so that GEMM1(t + 1) cannot complete before every epilogue warp
        // has seen GEMM1(t) complete (a parity wait must not fall two phases behind)
        if (ntile > 0) arrive(bar_a);
        for (int64_t t = 0; t < ntile; ++t) {
            const int64_t e0 = e_begin + t * E;
            const uint32_t u = region(t, 0), l = region(t, 1);
            const bool ok1 = wait_or_abort(bar_g1, (uint32_t)(t & 1));  // GEMM1(t): U(t) in u
            if (t + 1 < ntile) arrive(bar_a);
            const int64_t nvalid = (pvalid && ok1) ? (e_end - e0) : 0;
            float lt = 0.f;
            float yrh[8], yrl[8], yih[8], yil[8];
            if (grad) {
                // region l = l_{t-2} is free: GEMM1(t), which has completed, was issued after
                // GEMM2(t - 2), its last reader
                if (ok1) {
#pragma unroll 1
                    for (int qq = 0; qq < C::NQ; ++qq) {
                        epi_math(u, qq, nvalid, lt, yrh, yrl, yih, yil);
                        epi_store(u, l, qq, yrh, yrl, yih, yil);
                    }
                }
                // GEMM2(t - 1) complete: its sums in D2, drained before GEMM2(t) overwrites them
                const bool ok2 = t == 0 || wait_or_abort(bar_g2, (uint32_t)((t - 1) & 1));
                if (ok2 && t > 0) drain();
                if (ok1) tmem_wait_st();
                arrive(bar_y);
            } else if (ok1) {
#pragma unroll 1
                for (int qq = 0; qq < C::NQ; ++qq) epi_math(u, qq, nvalid, lt, yrh, yrl, yih, yil);
            }
            lsum = ff_add_f(lsum, lt);
        }
        if (grad && ntile > 0 && wait_or_abort(bar_g2, (uint32_t)((ntile - 1) & 1))) {  // the last GEMM2
            drain();
            flush();
        }
    } else {
        // ================================================================ operand warps
        const int lt = tid - (C::NC + 32);
        auto arrive = [&](uint64_t* b) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbarrier_arrive_one(b);
        };
        float2 ra[C::ITEMS][4];
        float4 rx[C::ITEMS][2];
        // two register images of K x E tiles: ra for A' (item: event e, waves 4 aq .. 4 aq + 3; a
        // warp reads 32 events of one wave row), rx for X (item: wave a, events 4 eq .. 4 eq + 3;
        // 8 waves x 4 quads per warp).  ra holds the tile after the current one, rx the current one.
        auto load_a = [&](int64_t e0) {
#pragma unroll
            for (int i = 0; i < C::ITEMS; ++i) {
                const int j = lt + C::NL * i;
                if (j < C::ITEMS_TOT) {
                    const int e = j % E, aq = j / E;
                    const int64_t ge = e0 + e;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int a = 4 * aq + q;
                        ra[i][q] = (a < K && ge < e_end) ? __ldg(A + a * ld + ge) : make_float2(0.f, 0.f);
                    }
                }
            }
        };
        auto load_x = [&](int64_t e0) {
#pragma unroll
            for (int i = 0; i < C::ITEMS; ++i) {
                const int j = lt + C::NL * i;
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
                const int j = lt + C::NL * i;
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
                const int j = lt + C::NL * i;
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
        if (ntile > 0) {
            load_a(e_begin);
            load_x(e_begin);
            store_a1();
            arrive(bar_a);  // A'(0)
            if (ntile > 1) load_a(e_begin + E);
        }
        for (int64_t t = 0; t < ntile; ++t) {
            const int64_t e0 = e_begin + t * E;
            const bool ok1 = wait_or_abort(bar_g1, (uint32_t)(t & 1));  // GEMM1(t) has read A'(t)
            if (t + 1 < ntile) {
                if (ok1) store_a1();  // A'(t + 1)
                arrive(bar_a);
            }
            if (grad) {
                // GEMM2(t - 1) has read X(t - 1)
                const bool ok2 = t == 0 || wait_or_abort(bar_g2, (uint32_t)((t - 1) & 1));
                if (ok2) store_x();  // X(t)
                arrive(bar_y);
            }
            if (t + 2 < ntile) load_a(e0 + 2 * E);
            if (grad && t + 1 < ntile) load_x(e0 + E);
        }
    }
    // ---- results: combine the two threads of each set (the A' area is free now: every MMA has
    // completed)
    tc_fence_before();
    __syncthreads();
    const bool timeout = *abort_s != 0;
    if (timeout && tid == 0) atomicOr(status, 2);
    float4* xch = reinterpret_cast<float4*>(tsm + C::OFF_AH);
    if (compute && hh == 1) xch[pl] = make_float4(lsum.hi, lsum.lo, mybad ? 1.f : 0.f, 0.f);
    __syncthreads();
    if (compute) {
        float2* prow = part + ((int64_t)blockIdx.x * P + p) * NV;  // this set's partials (valid if pvalid)
        if (hh == 0 && pvalid) {
            const float4 o = xch[pl];
            lsum = ff_add(lsum, ff{o.x, o.y});
            prow[0] = make_float2(lsum.hi, lsum.lo);
            if (mybad || o.z != 0.f || timeout) bad[p] = 1;
        }
        // G: both threads of a set write their column groups
        if (grad && pvalid) {
#pragma unroll
            for (int i = 0; i < C::NGRP; ++i) {
                const int q = hh + 2 * i;
                if (q < C::N2 / 16) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int col = 16 * q + k;
                        const int a = col % KMAX, g = col / KMAX;
                        if (a < K)
                            prow[1 + 2 * a + g] =
                                (ntile > 0 && !timeout) ? make_float2(ghi[16 * i + k], glo(i, k)) : make_float2(0.f, 0.f);
                    }
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
