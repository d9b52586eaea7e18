// Second derivatives of f = -sum_i ln I_i + n_f S in the real coordinates theta = (Re V_0,
// Im V_0, Re V_1, ...) of one parameter set: the curvature the Fumili / Newton-type fitters of
// the paper's frameworks use (Sec. 4), and the parameter errors (its inverse).
//   r_i = grad_theta ln I_i:  r_i[2c] = 2 Re(conj(A_c) u_i) / I_i,  r_i[2c+1] = 2 Im(conj(A_c) u_i) / I_i
//   Fumili (outer-product) form:  H = sum_i r_i r_i^T
//   exact form:                   H = sum_i r_i r_i^T - E(sum_i A_i A_i^H / I_i) + n_f E(Psi)
// with E(C)[2a][2b] = E(C)[2a+1][2b+1] = 2 Re C_ab, E(C)[2a][2b+1] = 2 Im C_ab,
// E(C)[2a+1][2b] = -2 Im C_ab (the real matrix of the quadratic form sum_ab V_a conj(V_b) C_ab).
//
// Both sums over events are Hermitian rank-N updates, which is what the normalisation-integral
// kernel computes: one pass writes r_i (as 2K complex rows with zero imaginary part) and 1/I_i,
// then k_normint forms sum_i r_i r_i^T (2K x 2K) and sum_i A_i A_i^H / I_i (K x K, the weights
// 1/I_i) with its double-single accumulation and fixed-order final sum, and a last kernel
// assembles H.  2K <= PWA_MAX_WAVES, so K <= 32.
#include "pwa_internal.cuh"

namespace pwa {

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int KMAX>
__global__ void __launch_bounds__(PWA_THREADS) k_gn_vectors(const float2* __restrict__ A, int K, int64_t n, int64_t ld,
                                                            const float2* __restrict__ V, float2* __restrict__ Z,
                                                            float* __restrict__ wI, int* __restrict__ badw) {
    __shared__ float2 sV[KMAX];
    if (threadIdx.x < KMAX) sV[threadIdx.x] = (int)threadIdx.x < K ? V[threadIdx.x] : make_float2(0.f, 0.f);
    __syncthreads();
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += stride) {
        float2 a[KMAX];
        float ur = 0.f, ui = 0.f;
#pragma unroll
        for (int c = 0; c < KMAX; ++c) {
            a[c] = (c < K && i < n) ? __ldg(A + c * ld + i) : make_float2(0.f, 0.f);
            cmac(ur, ui, sV[c].x, sV[c].y, a[c].x, a[c].y);
        }
        const float I = fmaf(ur, ur, ui * ui);
        const bool use = i < n && intensity_ok(I);
        if (i < n && !use) bad = true;
        const float rc = use ? __frcp_rn(I) : 0.f;
        const float r2 = 2.f * rc;
#pragma unroll
        for (int c = 0; c < KMAX; ++c) {
            if (c < K) {
                // conj(A_c) u
                const float zr = fmaf(a[c].x, ur, a[c].y * ui), zi = fmaf(a[c].x, ui, -a[c].y * ur);
                Z[(int64_t)(2 * c) * ld + i] = make_float2(zr * r2, 0.f);
                Z[(int64_t)(2 * c + 1) * ld + i] = make_float2(zi * r2, 0.f);
            }
        }
        wI[i] = rc;
    }
    if (bad) atomicOr(badw, 1);
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

template <int KMAX>
cudaError_t gn_vectors(const float2* A, int K, int64_t n, int64_t ld, const float2* V, float2* Z, float* wI, int* badw,
                       int sm_count, cudaStream_t st) {
    int64_t g = (ld + PWA_THREADS - 1) / PWA_THREADS;
    if (g > (int64_t)sm_count * 8) g = (int64_t)sm_count * 8;
    if (g < 1) g = 1;
    k_gn_vectors<KMAX><<<(unsigned)g, PWA_THREADS, 0, st>>>(A, K, n, ld, V, Z, wI, badw);
    return cudaGetLastError();
}

}  // namespace

size_t hessian_workspace(int K, int64_t ld, int sm_count) {
    const size_t D = 2 * (size_t)K;
    return al256(sizeof(float2) * D * (size_t)ld) + al256(sizeof(float) * (size_t)ld) + al256(sizeof(double2) * D * D) +
           al256(sizeof(double2) * (size_t)K * K) + 256 + normint_workspace((int)D, sm_count);
}

cudaError_t launch_hessian(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                           double nfac, int exact, double* H, void* ws, int* status, int sm_count, cudaStream_t st) {
    const size_t D = 2 * (size_t)K;
    char* p = static_cast<char*>(ws);
    float2* Z = reinterpret_cast<float2*>(p);
    p += al256(sizeof(float2) * D * (size_t)ld);
    float* wI = reinterpret_cast<float*>(p);
    p += al256(sizeof(float) * (size_t)ld);
    double2* Prr = reinterpret_cast<double2*>(p);
    p += al256(sizeof(double2) * D * D);
    double2* Cw = reinterpret_cast<double2*>(p);
    p += al256(sizeof(double2) * (size_t)K * K);
    int* badw = reinterpret_cast<int*>(p);
    p += 256;
    void* nws = p;
    cudaError_t e = cudaMemsetAsync(badw, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (K <= 4) e = gn_vectors<4>(A, K, n, ld, V, Z, wI, badw, sm_count, st);
    else if (K <= 8) e = gn_vectors<8>(A, K, n, ld, V, Z, wI, badw, sm_count, st);
    else if (K <= 16) e = gn_vectors<16>(A, K, n, ld, V, Z, wI, badw, sm_count, st);
    else e = gn_vectors<32>(A, K, n, ld, V, Z, wI, badw, sm_count, st);
    if (e != cudaSuccess) return e;
    // sum_i r_i r_i^T over the 2K real rows (stored as complex rows with zero imaginary part)
    e = launch_normint(Z, (int)D, n, ld, nullptr, 1.0, Prr, nws, sm_count, st);
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
