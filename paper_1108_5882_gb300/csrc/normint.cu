// Monte-Carlo normalisation integral Psi_ab = (1/N_gen) sum_j w_j A_a(j) conj(A_b(j)).
//
// Paper: Sec. 2, Eq. 3 (inner bracket of the second term: sum over accepted MC events divided
// by the number generated; footnote 1 for weighted, non-uniform MC).  With masses and widths
// fixed the bracket is computed once per fit (Sec. 2).
//
// This is a Hermitian rank-N update Psi = A diag(w) A^H / N_gen with K <= 64 and N ~ 1e7,
// so the work is a reduction over events, not a GEMM with reuse in the output: the kernel
// streams event tiles of E = 256 events through shared memory (the next tile is prefetched
// into registers while the current one is consumed) and gives each thread a 4 x 4 block of
// the upper triangle of Psi and an event phase.  The tile is stored event-major, so per event
// a thread issues 4 shared 16-byte loads for 16 complex multiply-adds (64 FFMA).
//
// Accumulation: FP32 per thread over a window of about 64 events, then folded into a
// per-thread double-single accumulator held in shared memory (v-major, conflict-free); the
// phases and then the blocks are combined in a fixed order, and the final division and the
// Hermitian completion are done in FP64.
#include "amp_model.cuh"

namespace pwa {

namespace {

constexpr int NI_E = 256;  // events per tile
// the tile is held event-major, sA[e][a] with a row stride of KMAX + 2 float2 (even, so that a
// thread's four consecutive waves of one event are two 16-byte loads)
template <int KMAX>
__host__ __device__ constexpr int ni_rs() { return KMAX + 2; }

__constant__ float c_ni_inv_int[AMP_JMAX + 1] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};

// The amplitudes of one event, A_a = BW_a(m) P_J(cos theta) exp(i lambda phi) for a < K, into
// row[a]: the arithmetic of the amplitude kernel (waves visited group by group, the Legendre
// recurrence carried across groups), for one event per thread.
__device__ __forceinline__ void event_amplitudes(const WaveTable& wt, float m, float ct, float ph, bool in,
                                                 float2* row) {
    float s1, c1;
    sincosf(ph, &s1, &c1);
    float pcur = 1.f, pprev = 0.f;  // P_jc, P_{jc-1}
    int jc = 0, s = 0;
    for (int g = 0; g < wt.ng; ++g) {
        const int end = wt.gend[g];
        const int a0 = wt.gord[s];
        const int J = wt.J[a0], lam = wt.lam[a0];
        const int al = lam < 0 ? -lam : lam;
        for (; jc < J; ++jc) {
            const float c2 = 2.f * jc + 1.f, cj = (float)jc, rj = c_ni_inv_int[jc];
            const float pn = (c2 * ct * pcur - cj * pprev) * rj;
            pprev = pcur;
            pcur = pn;
        }
        float er = 1.f, ei = 0.f;
        for (int j = 0; j < al; ++j) {
            const float tr = er * c1 - ei * s1;
            ei = er * s1 + ei * c1;
            er = tr;
        }
        if (lam < 0) ei = -ei;
        const float2 ang = make_float2(pcur * er, pcur * ei);
        for (; s < end; ++s) {
            const int a = wt.gord[s];
            const float Mh = wt.Mhi[a], Ml = wt.Mlo[a], MW = wt.MW[a];
            const float dr = ((Mh - m) + Ml) * ((Mh + m) + Ml);
            const float inv = __fdividef(1.f, fmaf(dr, dr, MW * MW));
            const float2 id = make_float2(dr * inv, MW * inv);
            const float2 bw = make_float2(MW * id.x, MW * id.y);
            row[a] = in ? cmul(bw, ang) : make_float2(0.f, 0.f);
        }
    }
}

// block partial layout: part[block][KMAX*KMAX] of complex ff = 4 floats (re.hi, re.lo, im.hi, im.lo)
// FROM_KIN: the tile's amplitudes are computed from the kinematics kin [3][ld] (thread t: event
// e0 + t, all waves) instead of read from A: Psi straight from the MC events, with no amplitude
// array written or read.
template <int KMAX, bool WEIGHTED, bool FROM_KIN = false>
__global__ void __launch_bounds__(PWA_THREADS) k_normint(const float2* __restrict__ A, int K, int64_t n,
                                                         int64_t ld, const float* __restrict__ w,
                                                         int64_t ev_per_block, float4* __restrict__ part,
                                                         const float* __restrict__ kin = nullptr,
                                                         WaveTable wt = WaveTable{}) {
    constexpr int KB = KMAX / 4;                 // 4x4 tile rows
    constexpr int NT = KB * (KB + 1) / 2;        // upper-triangle tiles
    constexpr int NPH = PWA_THREADS / NT > 0 ? PWA_THREADS / NT : 1;  // event phases
    constexpr int EPT = (NI_E + NPH - 1) / NPH;  // events per thread and tile
    constexpr int FLUSH = (64 + EPT - 1) / EPT;  // tiles per FP32 accumulation window (~64 events)
    constexpr int LD2 = KMAX * NI_E / PWA_THREADS;  // float2 tile loads per thread
    constexpr int RS = ni_rs<KMAX>();
    extern __shared__ float4 smem4[];
    float2* sA = reinterpret_cast<float2*>(smem4);              // [NI_E][RS], event-major
    float* sw = reinterpret_cast<float*>(sA + NI_E * RS);       // [NI_E]
    float* sacc = sw + NI_E;  // [64][PWA_THREADS]: 16 complex ff per thread, v-major

    const int tid = threadIdx.x;
    const bool active = tid < NT * NPH;
    const int t = tid % NT;
    const int ph = tid / NT;
    // tile t -> (ti, tj) with ti <= tj, row-major over the upper triangle
    int ti = 0, tj = 0;
    {
        int r = t, row = 0, len = KB;
        while (r >= len) { r -= len; ++row; --len; }
        ti = row;
        tj = row + r;
    }
    for (int v = 0; v < 64; ++v) sacc[v * PWA_THREADS + tid] = 0.f;
    if (FROM_KIN)  // the padding waves K..KMAX-1 of the computed tiles
        for (int a = K; a < KMAX; ++a) sA[tid * RS + a] = make_float2(0.f, 0.f);

    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_block;
    int64_t e_end = e_begin + ev_per_block;
    if (e_end > n) e_end = n;

    // register prefetch of the next tile: element idx = tid + 256 j -> row idx / NI_E, event idx % NI_E
    float2 pre[LD2];
    float prew = 0.f;
    float km = 2.f, kct = 0.f, kph = 0.f;  // FROM_KIN: the kinematics of event e0 + tid
    auto load_tile = [&](int64_t e0) {
        if (FROM_KIN) {
            const bool in = e0 + tid < e_end;
            km = in ? __ldg(kin + e0 + tid) : 2.f;
            kct = in ? __ldg(kin + ld + e0 + tid) : 0.f;
            kph = in ? __ldg(kin + 2 * ld + e0 + tid) : 0.f;
        } else {
#pragma unroll
            for (int j = 0; j < LD2; ++j) {
                const int idx = tid + PWA_THREADS * j;
                const int a = idx / NI_E, e = idx % NI_E;
                pre[j] = (a < K && e0 + e < e_end) ? __ldg(A + a * ld + e0 + e) : make_float2(0.f, 0.f);
            }
        }
        if (WEIGHTED) prew = (e0 + tid < e_end) ? __ldg(w + e0 + tid) : 0.f;  // NI_E == PWA_THREADS
    };

    float acc[32];
#pragma unroll
    for (int v = 0; v < 32; ++v) acc[v] = 0.f;
    int since_flush = 0;

    if (e_begin < e_end) load_tile(e_begin);
    for (int64_t e0 = e_begin; e0 < e_end; e0 += NI_E) {
        __syncthreads();  // previous tile consumed
        if (FROM_KIN) {
            event_amplitudes(wt, km, kct, kph, e0 + tid < e_end, sA + tid * RS);  // waves K.. stay zero
        } else {
#pragma unroll
            for (int j = 0; j < LD2; ++j) {
                const int idx = tid + PWA_THREADS * j;
                sA[(idx % NI_E) * RS + idx / NI_E] = pre[j];
            }
        }
        if (WEIGHTED) sw[tid] = prew;
        __syncthreads();
        if (e0 + NI_E < e_end) load_tile(e0 + NI_E);
        if (active) {
#pragma unroll 2
            for (int e = ph; e < NI_E; e += NPH) {
                float2 xa[4], xb[4];
                {
                    const float4* ra = reinterpret_cast<const float4*>(sA + e * RS + 4 * ti);
                    const float4* rb = reinterpret_cast<const float4*>(sA + e * RS + 4 * tj);
                    const float4 a01 = ra[0], a23 = ra[1], b01 = rb[0], b23 = rb[1];
                    xa[0] = make_float2(a01.x, a01.y);
                    xa[1] = make_float2(a01.z, a01.w);
                    xa[2] = make_float2(a23.x, a23.y);
                    xa[3] = make_float2(a23.z, a23.w);
                    xb[0] = make_float2(b01.x, b01.y);
                    xb[1] = make_float2(b01.z, b01.w);
                    xb[2] = make_float2(b23.x, b23.y);
                    xb[3] = make_float2(b23.z, b23.w);
                }
                if (WEIGHTED) {
                    const float we = sw[e];
#pragma unroll
                    for (int r = 0; r < 4; ++r) { xa[r].x *= we; xa[r].y *= we; }
                }
                // acc[(r*4+c)*2 + {0,1}] += xa[r] * conj(xb[c])
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cmac_conj(acc[(r * 4 + c) * 2], acc[(r * 4 + c) * 2 + 1], xb[c].x, xb[c].y, xa[r].x, xa[r].y);
                    }
            }
        }
        if (++since_flush == FLUSH) {
            since_flush = 0;
#pragma unroll
            for (int v = 0; v < 32; ++v) {
                ff a = {sacc[(2 * v) * PWA_THREADS + tid], sacc[(2 * v + 1) * PWA_THREADS + tid]};
                a = ff_add_f(a, acc[v]);
                sacc[(2 * v) * PWA_THREADS + tid] = a.hi;
                sacc[(2 * v + 1) * PWA_THREADS + tid] = a.lo;
                acc[v] = 0.f;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 32; ++v) {
        ff a = {sacc[(2 * v) * PWA_THREADS + tid], sacc[(2 * v + 1) * PWA_THREADS + tid]};
        a = ff_add_f(a, acc[v]);
        sacc[(2 * v) * PWA_THREADS + tid] = a.hi;
        sacc[(2 * v + 1) * PWA_THREADS + tid] = a.lo;
    }
    __syncthreads();
    // combine the phases of each tile in order and write the block partial (upper tiles only;
    // lower tiles of the KMAX x KMAX partial are left unwritten and never read)
    float4* bp = part + (int64_t)blockIdx.x * KMAX * KMAX;
    for (int o = tid; o < NT * 16; o += PWA_THREADS) {
        const int tt = o / 16, q = o % 16;
        ff re = ff_zero(), im = ff_zero();
        for (int p = 0; p < NPH; ++p) {
            const int th = p * NT + tt;
            re = ff_add(re, ff{sacc[(4 * q) * PWA_THREADS + th], sacc[(4 * q + 1) * PWA_THREADS + th]});
            im = ff_add(im, ff{sacc[(4 * q + 2) * PWA_THREADS + th], sacc[(4 * q + 3) * PWA_THREADS + th]});
        }
        int r2 = tt, row = 0, len = KB;
        while (r2 >= len) { r2 -= len; ++row; --len; }
        const int a = 4 * row + q / 4, b = 4 * (row + r2) + q % 4;
        bp[a * KMAX + b] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

// Sum the block partials and finalise Psi in FP64 (full Hermitian matrix).  One warp per upper
// entry (a <= b): lane l sums the partials of blocks l, l + 32, ... in order (all of its loads
// in flight at once), then the lanes are combined by a fixed xor-shuffle tree, so the order of
// every addition is fixed and the result deterministic.
template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS) k_normint_final(const float4* __restrict__ part, int nblocks,
                                                               int K, double inv_ngen, double2* __restrict__ Psi) {
    constexpr int PER_LANE = 16;  // loads in flight per lane and batch
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < K * K; o += nwarps) {
        const int a = o / K, b = o % K;
        if (a > b) continue;  // warp-uniform
        ff re = ff_zero(), im = ff_zero();
        for (int b0 = lane; b0 < nblocks; b0 += 32 * PER_LANE) {
            float4 v[PER_LANE];
#pragma unroll
            for (int j = 0; j < PER_LANE; ++j) {
                const int blk = b0 + 32 * j;
                v[j] = blk < nblocks ? __ldg(part + (int64_t)blk * KMAX * KMAX + a * KMAX + b)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < PER_LANE; ++j) {
                re = ff_add(re, ff{v[j].x, v[j].y});
                im = ff_add(im, ff{v[j].z, v[j].w});
            }
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            re = ff_add(re, ff_shfl_xor(re, m));
            im = ff_add(im, ff_shfl_xor(im, m));
        }
        if (lane == 0) {
            const double r = ff_to_double(re) * inv_ngen, i = ff_to_double(im) * inv_ngen;
            Psi[a * K + b] = make_double2(r, a == b ? 0.0 : i);
            if (a != b) Psi[b * K + a] = make_double2(r, -i);
        }
    }
}

template <int KMAX>
size_t ni_smem() {
    return sizeof(float2) * NI_E * ni_rs<KMAX>() + sizeof(float) * NI_E + sizeof(float) * 64 * PWA_THREADS;
}

// the tensor-core kernel (normint_tc.cu) and the same fixed-order finalisation
template <int KMAX>
cudaError_t ni_launch_tc(const float2* A, int K, int64_t n, const int64_t ld, double n_gen, double2* Psi, void* ws,
                         int* status, int sm_count, cudaStream_t st, const float* kin, const WaveTable* wt) {
    float4* part = reinterpret_cast<float4*>(ws);
    int nb = 1;
    cudaError_t e = launch_normint_tc(A, K, n, ld, kin, wt, part, status, sm_count, st, &nb);
    if (e != cudaSuccess) return e;
    const int fin_blocks = (K * K * 32 + PWA_THREADS - 1) / PWA_THREADS;  // one warp per entry
    k_normint_final<KMAX><<<fin_blocks, PWA_THREADS, 0, st>>>(part, nb, K, 1.0 / n_gen, Psi);
    return cudaGetLastError();
}

// The tensor-core kernel by default for 16 < K <= 32 with unit weights (measured on GB300: at
// K = 32 and 1e7 events from the kinematics 1.31 ms against 2.15 ms on SIMT; at K = 16 its
// two-stage pipeline is latency-bound and the SIMT kernel is faster).  PWA_NORMINT_TC=1 takes it
// for every K <= 32, PWA_NORMINT_TC=0 never.
bool use_normint_tc(int K, const float* w, const WaveTable* wt, const int* status) {
    if (!status || !normint_tc_ok(K, w, wt)) return false;
    const char* e = getenv("PWA_NORMINT_TC");
    if (e && e[0] == '0') return false;
    if (e && e[0] == '1') return true;
    return K > 16;
}

template <int KMAX>
cudaError_t ni_launch(const float2* A, int K, int64_t n, int64_t ld, const float* w, double n_gen,
                      double2* Psi, void* ws, int sm_count, cudaStream_t st, const float* kin = nullptr,
                      const WaveTable* wt = nullptr) {
    const size_t smem = ni_smem<KMAX>();
    auto kw = kin ? k_normint<KMAX, true, true> : k_normint<KMAX, true, false>;
    auto ku = kin ? k_normint<KMAX, false, true> : k_normint<KMAX, false, false>;
    cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const WaveTable wt0 = wt ? *wt : WaveTable{};
    int64_t tiles = (n + NI_E - 1) / NI_E;
    int64_t nb = (int64_t)sm_count * 2;
    if (nb > tiles) nb = tiles;
    if (nb < 1) nb = 1;
    const int64_t tiles_per_block = (tiles + nb - 1) / nb;
    const int64_t ev_per_block = tiles_per_block * NI_E;
    nb = ev_per_block > 0 ? (n + ev_per_block - 1) / ev_per_block : 1;
    if (nb < 1) nb = 1;
    float4* part = reinterpret_cast<float4*>(ws);
    if (w)
        kw<<<(unsigned)nb, PWA_THREADS, smem, st>>>(A, K, n, ld, w, ev_per_block, part, kin, wt0);
    else
        ku<<<(unsigned)nb, PWA_THREADS, smem, st>>>(A, K, n, ld, nullptr, ev_per_block, part, kin, wt0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int fin_blocks = (K * K * 32 + PWA_THREADS - 1) / PWA_THREADS;  // one warp per entry
    k_normint_final<KMAX><<<fin_blocks, PWA_THREADS, 0, st>>>(part, (int)nb, K, 1.0 / n_gen, Psi);
    return cudaGetLastError();
}

}  // namespace

size_t normint_workspace(int K, int sm_count) {
    // block partials of the SIMT kernel (2 blocks per SM) or of the tensor-core one (1 per SM, KMAX >= 8)
    int KMAX = K <= 8 ? 8 : K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64;
    return sizeof(float4) * (size_t)KMAX * KMAX * (size_t)sm_count * 2;
}

cudaError_t launch_normint_kin(const WaveTable& wt, const float* kin, int K, int64_t n, int64_t ld, const float* w,
                               double n_gen, double2* Psi, void* ws, int sm_count, cudaStream_t st, int* status) {
    if (use_normint_tc(K, w, &wt, status)) {
        if (K <= 8) return ni_launch_tc<8>(nullptr, K, n, ld, n_gen, Psi, ws, status, sm_count, st, kin, &wt);
        if (K <= 16) return ni_launch_tc<16>(nullptr, K, n, ld, n_gen, Psi, ws, status, sm_count, st, kin, &wt);
        return ni_launch_tc<32>(nullptr, K, n, ld, n_gen, Psi, ws, status, sm_count, st, kin, &wt);
    }
    if (K <= 4) return ni_launch<4>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
    if (K <= 8) return ni_launch<8>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
    if (K <= 16) return ni_launch<16>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
    if (K <= 32) return ni_launch<32>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
    if (K <= 48) return ni_launch<48>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
    return ni_launch<64>(nullptr, K, n, ld, w, n_gen, Psi, ws, sm_count, st, kin, &wt);
}

cudaError_t launch_normint(const float2* A, int K, int64_t n, int64_t ld, const float* w,
                           double n_gen, double2* Psi, void* ws, int sm_count, cudaStream_t st, int* status) {
    if (use_normint_tc(K, w, nullptr, status)) {
        if (K <= 8) return ni_launch_tc<8>(A, K, n, ld, n_gen, Psi, ws, status, sm_count, st, nullptr, nullptr);
        if (K <= 16) return ni_launch_tc<16>(A, K, n, ld, n_gen, Psi, ws, status, sm_count, st, nullptr, nullptr);
        return ni_launch_tc<32>(A, K, n, ld, n_gen, Psi, ws, status, sm_count, st, nullptr, nullptr);
    }
    if (K <= 4) return ni_launch<4>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
    if (K <= 8) return ni_launch<8>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
    if (K <= 16) return ni_launch<16>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
    if (K <= 32) return ni_launch<32>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
    if (K <= 48) return ni_launch<48>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
    return ni_launch<64>(A, K, n, ld, w, n_gen, Psi, ws, sm_count, st);
}

}  // namespace pwa
