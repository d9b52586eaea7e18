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
// fused kernel: each thread computes r_i of one event of a 256-event tile into shared memory
// (event-major), then each thread accumulates an 8 x 8 block of the upper triangle over a
// phase of the tile's events (64 FMA per four 16-byte shared loads), in FP32 over windows of
// about 64 events folded into double-single, with the phases and then the blocks combined in a
// fixed order.  r_i never goes to HBM: the kernel reads A once (8K bytes per event).  For the
// exact form the kernel also writes 1/I_i, and the normalisation-integral kernel forms
// sum_i A_i A_i^H / I_i with those weights.  2K <= PWA_MAX_WAVES, so K <= 32.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int GN_E = 256;  // events per tile: one per thread in the production step

template <int KMAX>
struct GnCfg {
    static constexpr int D = 2 * KMAX;                          // real rows (padded)
    static constexpr int DB = D / 8;                            // 8 x 8 tile rows
    static constexpr int NT = DB * (DB + 1) / 2;                // upper-triangle tiles
    static constexpr int NPH = PWA_THREADS / NT;                // event phases
    static constexpr int EPT = (GN_E + NPH - 1) / NPH;          // events per thread and tile
    static constexpr int FLUSH = (64 + EPT - 1) / EPT;          // tiles per FP32 window
    static constexpr int RS = D + 4;                            // tile row stride (floats)
    static constexpr size_t SMEM = sizeof(float) * ((size_t)GN_E * RS + 128 * PWA_THREADS);
};

// Block partials part[block][D][D] (float2 = hi, lo of a double-single sum; entries a <= b of
// the 8 x 8 tiles on and above the diagonal written).  wI: 1/I_i for i < n when non-NULL.
template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS, 1) k_gn_gram(const float2* __restrict__ A, int K, int64_t n,
                                                            int64_t ld, const float2* __restrict__ V,
                                                            int64_t ev_per_block, float2* __restrict__ part,
                                                            float* __restrict__ wI, int* __restrict__ badw) {
    using C = GnCfg<KMAX>;
    extern __shared__ float4 smem4[];
    float* sR = reinterpret_cast<float*>(smem4);     // [GN_E][RS], event-major
    float* sacc = sR + GN_E * C::RS;                  // [128][PWA_THREADS]: 64 double-single sums
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
    for (int v = 0; v < 128; ++v) sacc[v * PWA_THREADS + tid] = 0.f;
    for (int c = C::D; c < C::RS; ++c) sR[tid * C::RS + c] = 0.f;  // row padding (never read)
    __syncthreads();

    const int64_t e_begin = (int64_t)blockIdx.x * ev_per_block;
    int64_t e_end = e_begin + ev_per_block;
    if (e_end > n) e_end = n;

    float acc[64];
#pragma unroll
    for (int v = 0; v < 64; ++v) acc[v] = 0.f;
    int since_flush = 0;
    bool bad = false;

    for (int64_t e0 = e_begin; e0 < e_end; e0 += GN_E) {
        __syncthreads();  // previous tile consumed
        {
            // r of event e0 + tid: r[2c] + i r[2c+1] = 2 conj(A_c) u / I (zero when not used)
            const int64_t e = e0 + tid;
            const bool in = e < e_end;
            float2 a[KMAX];
            float ur = 0.f, ui = 0.f;
#pragma unroll
            for (int c = 0; c < KMAX; ++c) {
                a[c] = (c < K && in) ? __ldg(A + c * ld + e) : make_float2(0.f, 0.f);
                cmac(ur, ui, sV[c].x, sV[c].y, a[c].x, a[c].y);
            }
            const float I = fmaf(ur, ur, ui * ui);
            const bool use = in && intensity_ok(I);
            if (in && !use) bad = true;
            const float rc = use ? __frcp_rn(I) : 0.f;
            const float r2 = 2.f * rc;
            float* row = sR + tid * C::RS;
#pragma unroll
            for (int c = 0; c < KMAX; ++c) {
                const float zr = fmaf(a[c].x, ur, a[c].y * ui), zi = fmaf(a[c].x, ui, -a[c].y * ur);
                row[2 * c] = zr * r2;
                row[2 * c + 1] = zi * r2;
            }
            if (wI && in) wI[e] = rc;
        }
        __syncthreads();
        if (active) {
#pragma unroll 2
            for (int e = ph; e < GN_E; e += C::NPH) {
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
        if (++since_flush == C::FLUSH) {
            since_flush = 0;
#pragma unroll
            for (int v = 0; v < 64; ++v) {
                ff s2 = {sacc[(2 * v) * PWA_THREADS + tid], sacc[(2 * v + 1) * PWA_THREADS + tid]};
                s2 = ff_add_f(s2, acc[v]);
                sacc[(2 * v) * PWA_THREADS + tid] = s2.hi;
                sacc[(2 * v + 1) * PWA_THREADS + tid] = s2.lo;
                acc[v] = 0.f;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 64; ++v) {
        ff s2 = {sacc[(2 * v) * PWA_THREADS + tid], sacc[(2 * v + 1) * PWA_THREADS + tid]};
        s2 = ff_add_f(s2, acc[v]);
        sacc[(2 * v) * PWA_THREADS + tid] = s2.hi;
        sacc[(2 * v + 1) * PWA_THREADS + tid] = s2.lo;
    }
    if (bad) atomicOr(badw, 1);
    __syncthreads();
    // combine the phases of each tile in order and write the block partial
    float2* bp = part + (int64_t)blockIdx.x * C::D * C::D;
    for (int o = tid; o < C::NT * 64; o += PWA_THREADS) {
        const int tt = o / 64, q = o % 64;
        ff s2 = ff_zero();
        for (int p = 0; p < C::NPH; ++p) {
            const int th = p * C::NT + tt;
            s2 = ff_add(s2, ff{sacc[(2 * q) * PWA_THREADS + th], sacc[(2 * q + 1) * PWA_THREADS + th]});
        }
        int r2 = tt, row = 0, len = C::DB;
        while (r2 >= len) { r2 -= len; ++row; --len; }
        const int a = 8 * row + q / 8, b = 8 * (row + r2) + q % 8;
        bp[a * C::D + b] = make_float2(s2.hi, s2.lo);
    }
}

// Sum the block partials of each entry a <= b < D2 = 2K in a fixed order (one warp per entry:
// lane-strided over the blocks, then an xor tree) and write the symmetric D2 x D2 matrix, as
// complex values with zero imaginary part (the layout the assembly kernel reads).
template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS) k_gn_final(const float2* __restrict__ part, int nblocks, int D2,
                                                          double2* __restrict__ P) {
    constexpr int D = 2 * KMAX;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < D2 * D2; o += nwarps) {
        const int a = o / D2, b = o % D2;
        if (a > b) continue;  // warp-uniform
        ff s2 = ff_zero();
        for (int blk = lane; blk < nblocks; blk += 32) {
            const float2 v = __ldg(part + (int64_t)blk * D * D + a * D + b);
            s2 = ff_add(s2, ff{v.x, v.y});
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) s2 = ff_add(s2, ff_shfl_xor(s2, m));
        if (lane == 0) {
            const double v = ff_to_double(s2);
            P[a * D2 + b] = make_double2(v, 0.0);
            P[b * D2 + a] = make_double2(v, 0.0);
        }
    }
}

// H[x][y] from the Gram sums; NaN everywhere if some intensity was not positive and finite
__global__ void k_hessian_final(const double2* __restrict__ Prr, const double2* __restrict__ Cw,
                                const double2* __restrict__ Psi, int K, double nfac, int exact,
                                const int* __restrict__ badw, int* __restrict__ status, double* __restrict__ H) {
    const int D = 2 * K;
    const bool bad = *badw != 0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * D; idx += gridDim.x * blockDim.x) {
        const int x = idx / D, y = idx % D;
        double v = Prr[idx].x;
        if (exact) {
            const int a = x >> 1, b = y >> 1, px = x & 1, py = y & 1;
            const double2 c = Cw[a * K + b], p = Psi[a * K + b];
            // E(M)[2a+px][2b+py] = 2 Re M_ab (px == py), 2 Im M_ab (0, 1), -2 Im M_ab (1, 0)
            const double ec = px == py ? 2.0 * c.x : (px == 0 ? 2.0 * c.y : -2.0 * c.y);
            const double ep = px == py ? 2.0 * p.x : (px == 0 ? 2.0 * p.y : -2.0 * p.y);
            v = v - ec + nfac * ep;
        }
        H[idx] = bad ? NAN : v;
    }
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1);
}

// blocks of the fused Gram kernel: at most two per SM, each over whole 256-event tiles
inline int64_t gn_blocks(int64_t n, int sm_count, int64_t* ev_per_block) {
    const int64_t tiles = (n + GN_E - 1) / GN_E;
    int64_t nb = (int64_t)sm_count * 2;
    if (nb > tiles) nb = tiles;
    if (nb < 1) nb = 1;
    const int64_t tpb = (tiles + nb - 1) / nb;
    *ev_per_block = tpb > 0 ? tpb * GN_E : GN_E;
    nb = (n + *ev_per_block - 1) / *ev_per_block;
    return nb < 1 ? 1 : nb;
}

template <int KMAX>
cudaError_t gn_gram(const float2* A, int K, int64_t n, int64_t ld, const float2* V, float2* part, float* wI,
                    int* badw, double2* Prr, int sm_count, cudaStream_t st) {
    using C = GnCfg<KMAX>;
    auto kern = k_gn_gram<KMAX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int64_t epb = GN_E;
    const int64_t nb = gn_blocks(n, sm_count, &epb);
    kern<<<(unsigned)nb, PWA_THREADS, C::SMEM, st>>>(A, K, n, ld, V, epb, part, wI, badw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int D2 = 2 * K;
    const int fin_blocks = (D2 * D2 * 32 + PWA_THREADS - 1) / PWA_THREADS;  // one warp per entry
    k_gn_final<KMAX><<<fin_blocks, PWA_THREADS, 0, st>>>(part, (int)nb, D2, Prr);
    return cudaGetLastError();
}

inline int gn_kmax(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32; }

}  // namespace

size_t hessian_workspace(int K, int64_t ld, int sm_count) {
    const size_t D = 2 * (size_t)K, DM = 2 * (size_t)gn_kmax(K);
    return al256(sizeof(float) * (size_t)ld) + al256(sizeof(double2) * D * D) + al256(sizeof(double2) * (size_t)K * K) +
           256 + al256(sizeof(float2) * DM * DM * 2 * (size_t)sm_count) + normint_workspace(K, sm_count);
}

cudaError_t launch_hessian(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                           double nfac, int exact, double* H, void* ws, int* status, int sm_count, cudaStream_t st) {
    const size_t D = 2 * (size_t)K, DM = 2 * (size_t)gn_kmax(K);
    char* p = static_cast<char*>(ws);
    float* wI = reinterpret_cast<float*>(p);
    p += al256(sizeof(float) * (size_t)ld);
    double2* Prr = reinterpret_cast<double2*>(p);
    p += al256(sizeof(double2) * D * D);
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
    // sum_i r_i r_i^T (and 1/I_i for the exact form) in one pass over A
    if (K <= 4) e = gn_gram<4>(A, K, n, ld, V, part, w, badw, Prr, sm_count, st);
    else if (K <= 8) e = gn_gram<8>(A, K, n, ld, V, part, w, badw, Prr, sm_count, st);
    else if (K <= 16) e = gn_gram<16>(A, K, n, ld, V, part, w, badw, Prr, sm_count, st);
    else e = gn_gram<32>(A, K, n, ld, V, part, w, badw, Prr, sm_count, st);
    if (e != cudaSuccess) return e;
    if (exact) {
        e = launch_normint(A, K, n, ld, wI, 1.0, Cw, nws, sm_count, st);  // sum_i A_i A_i^H / I_i
        if (e != cudaSuccess) return e;
    }
    const int nt = (int)(D * D);
    k_hessian_final<<<(nt + PWA_THREADS - 1) / PWA_THREADS, PWA_THREADS, 0, st>>>(Prr, Cw, Psi, K, nfac, exact, badw,
                                                                                  status, H);
    return cudaGetLastError();
}

}  // namespace pwa
