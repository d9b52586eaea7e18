// Second derivatives of f = -sum_i ln I_i + n_f S in the real coordinates theta = (Re V_0,
// Im V_0, Re V_1, ...) of one parameter set: the curvature the Fumili / Newton-type fitters of
// the paper's frameworks use (Sec. 4), and the parameter errors (its inverse).
//   r_i = grad_theta ln I_i:  r_i[2c] = 2 Re(conj(A_c) u_i) / I_i,  r_i[2c+1] = 2 Im(conj(A_c) u_i) / I_i
//   Fumili (outer-product) form:  H = sum_i r_i r_i^T
//   exact form:                   H = sum_i r_i r_i^T - E(sum_i A_i A_i^H / I_i) + n_f E(Psi)
// with E(C)[2a][2b] = E(C)[2a+1][2b+1] = 2 Re C_ab, E(C)[2a][2b+1] = 2 Im C_ab,
// E(C)[2a+1][2b] = -2 Im C_ab (the real matrix of the quadratic form sum_ab V_a conj(V_b) C_ab).
//
// The event sums are Gram sums.  sum_i r_i r_i^T (2K x 2K, real symmetric) is formed by one
// fused kernel that runs two blocks per SM (at most 128 registers, at most 110 KB of shared
// memory each) over whole event tiles:
//  * the amplitudes of the next tile are copied global -> shared (cp.async, one 8-byte copy per
//    event and wave) while the current tile is accumulated, so the HBM reads overlap the FMAs;
//  * r_i of each event is computed from the staged amplitudes in two passes (u = sum V A, then
//    r from the reloaded amplitudes) into an event-major shared tile;
//  * each thread accumulates an 8 x 8 block of the upper triangle over a phase of the tile's
//    events (64 FMA per four 16-byte shared loads) in FP32 over windows of about 64 events;
//  * at the end of a window the phases' FP32 sums go through shared scratch (the consumed r
//    tile) and one owner thread per matrix entry adds them, in phase order, to one double-single
//    sum for the entry.
// r_i never goes to HBM: the kernel reads A once (8K bytes per event).  For the exact form the
// kernel also writes 1/I_i, and the normalisation-integral kernel forms sum_i A_i A_i^H / I_i
// with those weights.  2K <= PWA_MAX_WAVES, so K <= 32.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int KMAX>
struct GnCfg {
    static constexpr int E = KMAX <= 16 ? 256 : 128;            // events per tile
    static constexpr int TPE = PWA_THREADS / E;                 // threads per event in the r step
    static constexpr int D = 2 * KMAX;                          // real rows (padded)
    static constexpr int DB = D / 8;                            // 8 x 8 tile rows
    static constexpr int NT = DB * (DB + 1) / 2;                // upper-triangle tiles
    static constexpr int NPH = PWA_THREADS / NT;                // event phases
    static constexpr int EPT = (E + NPH - 1) / NPH;             // events per thread and tile
    static constexpr int FLUSH = (64 + EPT - 1) / EPT;          // tiles per FP32 window
    static constexpr int RS = D + 4;                            // r tile row stride (floats)
    static constexpr int NE = NT * 64;                          // matrix entries held
    static constexpr int STAGE = KMAX * E * 2;                  // staged amplitudes (floats)
    static constexpr int SFF = 2 * NE;                          // double-single entry sums (floats)
    // phases per scratch batch: as many as fit beside the stage and the sums in 110 KB
    static constexpr int XCAP = (110 * 1024 / 4 - STAGE - SFF);
    static constexpr int PBMAX = XCAP / NE < NPH ? XCAP / NE : NPH;
    static constexpr int NBATCH = (NPH + PBMAX - 1) / PBMAX;
    static constexpr int PB = (NPH + NBATCH - 1) / NBATCH;
    static constexpr int X = E * RS > PB * NE ? E * RS : PB * NE;  // r tile / window scratch
    static constexpr size_t SMEM = sizeof(float) * ((size_t)X + STAGE + SFF);
    static_assert(PBMAX >= 1, "shared-memory budget");
    static_assert(SMEM <= 110 * 1024, "two blocks per SM");
    static_assert(E % TPE == 0 && KMAX % TPE == 0, "r step split");
};

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// stage the amplitudes of events [e0, e0 + E) (zero beyond e_end) as [wave][event]
template <int KMAX>
__device__ __forceinline__ void gn_prefetch(float2* stage, const float2* __restrict__ A, int K, int64_t ld,
                                            int64_t e0, int64_t e_end) {
    using C = GnCfg<KMAX>;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(stage);
    for (int idx = threadIdx.x; idx < K * C::E; idx += PWA_THREADS) {
        const int c = idx / C::E, ev = idx % C::E;
        const int64_t e = e0 + ev;
        const bool in = e < e_end;
        cp_async8(base + 8u * (uint32_t)idx, in ? (const void*)(A + c * ld + e) : (const void*)A, in ? 8u : 0u);
    }
    cp_async_commit();
}

// Block partials part[block][D][D] (float2 = hi, lo of a double-single sum; entries a <= b of
// the 8 x 8 tiles on and above the diagonal written).  wI: 1/I_i for i < n when non-NULL.
template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS, 2) k_gn_gram(const float2* __restrict__ A, int K, int64_t n,
                                                            int64_t ld, const float2* __restrict__ V,
                                                            int64_t ev_per_block, float2* __restrict__ part,
                                                            float* __restrict__ wI, int* __restrict__ badw) {
    using C = GnCfg<KMAX>;
    extern __shared__ float4 smem4[];
    float* sR = reinterpret_cast<float*>(smem4);             // [E][RS] event-major r tile, or scratch
    float2* stage = reinterpret_cast<float2*>(sR + C::X);    // [KMAX][E] staged amplitudes
    float* sff = sR + C::X + C::STAGE;                       // [2][NE] hi, lo of the entry sums
    __shared__ float2 sV[KMAX];

    const int tid = threadIdx.x;
    const bool active = tid < C::NT * C::NPH;
    const int t = tid % C::NT;
    const int ph = tid / C::NT;
    int ti = 0, tj = 0;  // tile t -> (ti, tj), ti <= tj, row-major over the upper triangle
    {
        int r = t, row = 0, len = C::DB;
        while (r >= len) { r -= len; ++row; --len; }
        ti = row;
        tj = row + r;
    }
    if (tid < KMAX) sV[tid] = tid < K ? V[tid] : make_float2(0.f, 0.f);
    for (int v = tid; v < C::SFF; v += PWA_THREADS) sff[v] = 0.f;

    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_block;
    int64_t e_end = e_begin + ev_per_block;
    if (e_end > n) e_end = n;
    if (e_begin < e_end) gn_prefetch<KMAX>(stage, A, K, ld, e_begin, e_end);

    float acc[64];
#pragma unroll
    for (int v = 0; v < 64; ++v) acc[v] = 0.f;
    int since_flush = 0;
    bool bad = false;
    const int ev = tid / C::TPE, part_id = tid % C::TPE;

    for (int64_t e0 = e_begin; e0 < e_end; e0 += C::E) {
        cp_async_wait_all();
        __syncthreads();  // this tile staged for every thread; the previous r tile / scratch consumed
        {
            // r of event e0 + ev: r[2c] + i r[2c+1] = 2 conj(A_c) u / I; this thread's waves
            // c = part_id, part_id + TPE, ... (zero when the event is not used)
            const int64_t e = e0 + ev;
            const bool in = e < e_end;
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int j = 0; j < KMAX / C::TPE; ++j) {
                const int c = part_id + j * C::TPE;
                if (c < K) {
                    const float2 a = stage[c * C::E + ev];
                    cmac(ur, ui, sV[c].x, sV[c].y, a.x, a.y);
                }
            }
            if (C::TPE == 2) {
                ur += __shfl_xor_sync(0xffffffffu, ur, 1);
                ui += __shfl_xor_sync(0xffffffffu, ui, 1);
            }
            const float I = fmaf(ur, ur, ui * ui);
            const bool use = in && intensity_ok(I);
            if (in && !use) bad = true;
            const float rc = use ? __frcp_rn(I) : 0.f;
            const float r2 = 2.f * rc;
            float2* row = reinterpret_cast<float2*>(sR + ev * C::RS);
#pragma unroll
            for (int j = 0; j < KMAX / C::TPE; ++j) {
                const int c = part_id + j * C::TPE;
                const float2 a = c < K ? stage[c * C::E + ev] : make_float2(0.f, 0.f);
                const float zr = fmaf(a.x, ur, a.y * ui), zi = fmaf(a.x, ui, -a.y * ur);
                row[c] = make_float2(zr * r2, zi * r2);
            }
            if (wI && in && part_id == 0) wI[e] = rc;
        }
        __syncthreads();  // r tile complete; the stage is free for the next tile
        if (e0 + C::E < e_end) gn_prefetch<KMAX>(stage, A, K, ld, e0 + C::E, e_end);
        if (active) {
#pragma unroll 2
            for (int e = ph; e < C::E; e += C::NPH) {
                const float4* ra = reinterpret_cast<const float4*>(sR + e * C::RS + 8 * ti);
                const float4* rb = reinterpret_cast<const float4*>(sR + e * C::RS + 8 * tj);
                const float4 a0 = ra[0], a1 = ra[1], b0 = rb[0], b1 = rb[1];
                const float xa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float xb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r * 8 + c] = fmaf(xa[r], xb[c], acc[r * 8 + c]);
            }
        }
        if (++since_flush == C::FLUSH || e0 + C::E >= e_end) {
            // window end: scratch[v][slot] <- acc[v] of phase batch [p0, p0 + PB); the owner of
            // entry o = v * NT + tile adds the batch's phases in order to its double-single sum
            since_flush = 0;
            for (int p0 = 0; p0 < C::NPH; p0 += C::PB) {
                __syncthreads();  // r tile (or the previous batch) consumed
                if (active && ph >= p0 && ph < p0 + C::PB) {
                    const int slot = (ph - p0) * C::NT + t;
#pragma unroll
                    for (int v = 0; v < 64; ++v) sR[v * (C::PB * C::NT) + slot] = acc[v];
                }
                __syncthreads();
                const int pe = p0 + C::PB < C::NPH ? p0 + C::PB : C::NPH;
                for (int o = tid; o < C::NE; o += PWA_THREADS) {
                    const int v = o / C::NT, tt = o % C::NT;
                    ff s2 = {sff[o], sff[C::NE + o]};
                    for (int p = p0; p < pe; ++p) s2 = ff_add_f(s2, sR[v * (C::PB * C::NT) + (p - p0) * C::NT + tt]);
                    sff[o] = s2.hi;
                    sff[C::NE + o] = s2.lo;
                }
            }
#pragma unroll
            for (int v = 0; v < 64; ++v) acc[v] = 0.f;
        }
    }
    if (bad) atomicOr(badw, 1);
    __syncthreads();
    // write the block partial: entry o = v * NT + tile holds element (8 row + v / 8, 8 col + v % 8)
    float2* bp = part + (int64_t)blockIdx.x * C::D * C::D;
    for (int o = tid; o < C::NE; o += PWA_THREADS) {
        const int v = o / C::NT, tt = o % C::NT;
        int r2 = tt, row = 0, len = C::DB;
        while (r2 >= len) { r2 -= len; ++row; --len; }
        const int a = 8 * row + v / 8, b = 8 * (row + r2) + v % 8;
        bp[a * C::D + b] = make_float2(sff[o], sff[C::NE + o]);
    }
}

// H from the block partials: one warp per entry x <= y < D2 = 2K sums the blocks' partials of
// sum_i r_i r_i^T in a fixed order (lane-strided over the blocks, then an xor tree), adds the
// exact form's terms and writes H[x][y] and H[y][x]; NaN everywhere if some intensity was not
// positive and finite.
template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS) k_gn_final(const float2* __restrict__ part, int nblocks, int K,
                                                          const double2* __restrict__ Cw,
                                                          const double2* __restrict__ Psi, double nfac, int exact,
                                                          const int* __restrict__ badw, int* __restrict__ status,
                                                          double* __restrict__ H) {
    constexpr int D = 2 * KMAX;
    const int D2 = 2 * K;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool bad = *badw != 0;
    for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < D2 * D2; o += nwarps) {
        const int x = o / D2, y = o % D2;
        if (x > y) continue;  // warp-uniform
        ff s2 = ff_zero();
        for (int blk = lane; blk < nblocks; blk += 32) {
            const float2 v = __ldg(part + (int64_t)blk * D * D + x * D + y);
            s2 = ff_add(s2, ff{v.x, v.y});
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) s2 = ff_add(s2, ff_shfl_xor(s2, m));
        if (lane < 2) {
            // lane 0 writes H[x][y], lane 1 H[y][x]
            const int r = lane == 0 ? x : y, c = lane == 0 ? y : x;
            double v = ff_to_double(s2);
            if (exact) {
                const int a = r >> 1, b2 = c >> 1, pr = r & 1, pc = c & 1;
                const double2 cw = Cw[a * K + b2], ps = Psi[a * K + b2];
                // E(M)[2a+pr][2b+pc] = 2 Re M_ab (pr == pc), 2 Im M_ab (0, 1), -2 Im M_ab (1, 0)
                const double ec = pr == pc ? 2.0 * cw.x : (pr == 0 ? 2.0 * cw.y : -2.0 * cw.y);
                const double ep = pr == pc ? 2.0 * ps.x : (pr == 0 ? 2.0 * ps.y : -2.0 * ps.y);
                v = v - ec + nfac * ep;
            }
            if (lane == 0 || x != y) H[r * D2 + c] = bad ? NAN : v;
        }
    }
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1);
}

// blocks of the fused Gram kernel: one wave of two per SM, each over whole tiles of E events
inline int64_t gn_blocks(int64_t n, int E, int sm_count, int64_t* ev_per_block) {
    const int64_t tiles = (n + E - 1) / E;
    int64_t nb = (int64_t)sm_count * 2;
    if (nb > tiles) nb = tiles;
    if (nb < 1) nb = 1;
    const int64_t tpb = (tiles + nb - 1) / nb;
    *ev_per_block = tpb > 0 ? tpb * E : E;
    nb = (n + *ev_per_block - 1) / *ev_per_block;
    return nb < 1 ? 1 : nb;
}

template <int KMAX>
cudaError_t gn_gram(const float2* A, int K, int64_t n, int64_t ld, const float2* V, float2* part, float* wI,
                    int* badw, int* nblocks, int sm_count, cudaStream_t st) {
    using C = GnCfg<KMAX>;
    auto kern = k_gn_gram<KMAX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int64_t epb = C::E;
    const int64_t nb = gn_blocks(n, C::E, sm_count, &epb);
    kern<<<(unsigned)nb, PWA_THREADS, C::SMEM, st>>>(A, K, n, ld, V, epb, part, wI, badw);
    *nblocks = (int)nb;
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t gn_final(const float2* part, int nblocks, int K, const double2* Cw, const double2* Psi, double nfac,
                     int exact, const int* badw, int* status, double* H, cudaStream_t st) {
    const int D2 = 2 * K;
    const int fin_blocks = (D2 * D2 * 32 + PWA_THREADS - 1) / PWA_THREADS;  // one warp per entry
    k_gn_final<KMAX><<<fin_blocks, PWA_THREADS, 0, st>>>(part, nblocks, K, Cw, Psi, nfac, exact, badw, status, H);
    return cudaGetLastError();
}

inline int gn_kmax(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32; }

}  // namespace

size_t hessian_workspace(int K, int64_t ld, int sm_count) {
    const size_t DM = 2 * (size_t)gn_kmax(K);
    return al256(sizeof(float) * (size_t)ld) + al256(sizeof(double2) * (size_t)K * K) + 256 +
           al256(sizeof(float2) * DM * DM * 2 * (size_t)sm_count) + normint_workspace(K, sm_count);
}

cudaError_t launch_hessian(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                           double nfac, int exact, double* H, void* ws, int* status, int sm_count, cudaStream_t st) {
    const size_t DM = 2 * (size_t)gn_kmax(K);
    char* p = static_cast<char*>(ws);
    float* wI = reinterpret_cast<float*>(p);
    p += al256(sizeof(float) * (size_t)ld);
    double2* Cw = reinterpret_cast<double2*>(p);
    p += al256(sizeof(double2) * (size_t)K * K);
    int* badw = reinterpret_cast<int*>(p);
    p += 256;
    float2* part = reinterpret_cast<float2*>(p);
    p += al256(sizeof(float2) * DM * DM * 2 * (size_t)sm_count);
    void* nws = p;
    cudaError_t e = cudaMemsetAsync(badw, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    float* w = exact ? wI : nullptr;
    int nb = 0;
    // sum_i r_i r_i^T (and 1/I_i for the exact form) in one pass over A
    if (K <= 4) e = gn_gram<4>(A, K, n, ld, V, part, w, badw, &nb, sm_count, st);
    else if (K <= 8) e = gn_gram<8>(A, K, n, ld, V, part, w, badw, &nb, sm_count, st);
    else if (K <= 16) e = gn_gram<16>(A, K, n, ld, V, part, w, badw, &nb, sm_count, st);
    else e = gn_gram<32>(A, K, n, ld, V, part, w, badw, &nb, sm_count, st);
    if (e != cudaSuccess) return e;
    if (exact) {
        e = launch_normint(A, K, n, ld, wI, 1.0, Cw, nws, sm_count, st);  // sum_i A_i A_i^H / I_i
        if (e != cudaSuccess) return e;
    }
    if (K <= 4) return gn_final<4>(part, nb, K, Cw, Psi, nfac, exact, badw, status, H, st);
    if (K <= 8) return gn_final<8>(part, nb, K, Cw, Psi, nfac, exact, badw, status, H, st);
    if (K <= 16) return gn_final<16>(part, nb, K, Cw, Psi, nfac, exact, badw, status, H, st);
    return gn_final<32>(part, nb, K, Cw, Psi, nfac, exact, badw, status, H, st);
}

}  // namespace pwa
