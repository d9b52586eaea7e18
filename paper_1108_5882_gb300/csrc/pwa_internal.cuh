// Internal declarations shared by the translation units of libpwa.so (not installed).
//
// Numerics used throughout: per-event arithmetic in FP32 (the paper's Sec. 2 precision
// remark: single precision suffices for the individual amplitude), per-thread FP32
// accumulation over a bounded window of events, and every longer sum carried as a
// double-single ("ff") pair (hi + lo, Knuth's TwoSum and Dekker's Fast2Sum), combined across
// warps and blocks in a fixed order so results are bitwise reproducible.  FP64 is used only
// for the O(K^2) normalisation term: GB300 runs FP64 at a small fraction of its FP32 rate.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/pwa.h"

#define PWA_THREADS 256

struct pwa_handle {
    int device = 0;
    int sm_count = 0;
    std::string err;
    void* ws = nullptr;          // workspace: block partials
    size_t ws_bytes = 0;
    unsigned* counters = nullptr;  // completion counters (zero between calls)
    int* status = nullptr;         // sticky device status word (bit 0: non-finite intensity)
    int* bad = nullptr;            // per-parameter-set non-finite flags [bad_cap]
    int bad_cap = 0;
    void* fitws = nullptr;         // batched-fit state and evaluation buffers
    size_t fitws_bytes = 0;
    cudaStream_t fit_stream = nullptr;  // capturable stream the fitter runs on
    cudaEvent_t fit_event = nullptr;
    void* uws = nullptr;                 // multi-channel evaluation: descriptors, work list, item sums
    size_t uws_bytes = 0;
    std::vector<unsigned char> uws_key;  // host image of the descriptors and work list last uploaded
};

namespace pwa {

// ---------------------------------------------------------------- double-single sums ----
struct ff {
    float hi, lo;
};

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    return {s, e};
}
// Fast2Sum (Dekker), valid for |a| >= |b|.
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ ff ff_shfl_xor(ff a, int m) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

// ---------------------------------------------------------------- warp reductions -------
// Reduce-scatter of 32 per-lane values across the warp: on return x[0] of lane l holds the
// warp-wide sum of value l.  31 shuffles instead of 32 x 5 for a butterfly per value.  Each
// level halves the live values: lanes with bit LVL set keep the upper half and send the lower.
template <int LVL>
__device__ __forceinline__ void transpose_reduce_level(float (&x)[32], int lane) {
    constexpr int HALF = 1 << LVL;
    const bool upper = (lane >> LVL) & 1;
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const float lo = x[j], hi = x[j + HALF];
        const float send = upper ? lo : hi;
        const float keep = upper ? hi : lo;
        x[j] = keep + __shfl_xor_sync(0xffffffffu, send, HALF);
    }
    if constexpr (LVL > 0) transpose_reduce_level<LVL - 1>(x, lane);
}
__device__ __forceinline__ void warp_transpose_reduce32(float (&x)[32]) {
    transpose_reduce_level<4>(x, threadIdx.x & 31);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Fixed-order double-single sum of x[first], x[first + step], ... (count terms) with UNR
// independent loads in flight per batch (the partials live in L2: a dependent load chain
// would cost one L2 round trip per term).  Loads bypass L1 (written by other blocks).
template <int UNR = 16>
__device__ __forceinline__ ff ff_sum_strided(const float2* __restrict__ x, int64_t first, int64_t step, int count) {
    ff s = ff_zero();
    for (int j0 = 0; j0 < count; j0 += UNR) {
        float2 v[UNR];
#pragma unroll
        for (int j = 0; j < UNR; ++j) v[j] = (j0 + j < count) ? __ldcg(x + first + (int64_t)(j0 + j) * step) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < UNR; ++j) s = ff_add(s, ff{v[j].x, v[j].y});
    }
    return s;
}

// Complex multiply-accumulate into an (re, im) float pair as chains of FMAs into the
// accumulator: acc += a b (cmac) and acc += conj(a) b (cmac_conj).  Written this way each real
// part costs two FMAs; the expression acc += x y - z w would round x y - z w first and cost
// an extra multiply and add (no reassociation without fast-math).
__device__ __forceinline__ void cmac(float& re, float& im, float ar, float ai, float br, float bi) {
    re = fmaf(ar, br, re);
    re = fmaf(-ai, bi, re);
    im = fmaf(ar, bi, im);
    im = fmaf(ai, br, im);
}
__device__ __forceinline__ void cmac_conj(float& re, float& im, float ar, float ai, float br, float bi) {
    re = fmaf(ar, br, re);
    re = fmaf(ai, bi, re);
    im = fmaf(ar, bi, im);
    im = fmaf(-ai, br, im);
}

// Non-finite or non-positive intensity test (the likelihood needs ln I_i).
__device__ __forceinline__ bool intensity_ok(float I) { return I > 0.f && I < INFINITY; }

// Control words of a one-parameter-set likelihood launch (device memory; the words marked
// "zero" are zero between launches: the launch's last block clears them):
//   byte 0                   completion ticket (zero)
//   byte 4                   flag word, STREAM_FLAG_* (zero)
//   STREAM_CTRL_LIMB_OFFSET  fixed-point words [STREAM_NV_MAX + 1][FIX_WORDS] (int64, zero) of the
//                            grid sums of ln I (value 0), of the 2K gradient components (values
//                            1..2K) and of S = sum_c Re(conj(V_c) t_c) (value STREAM_NV_MAX)
//   STREAM_CTRL_T_OFFSET     t_c = sum_a Psi_ac V_a, double2 [PWA_MAX_WAVES] (written each launch)
constexpr int STREAM_FLAG_NONFINITE = 1;  // some intensity was <= 0 or not finite
constexpr int STREAM_NV_MAX = 1 + 2 * PWA_MAX_WAVES;
constexpr int FIX_WORDS = 6;              // two tiers of three 42-bit limbs per value
constexpr size_t STREAM_CTRL_LIMB_OFFSET = 256;
constexpr size_t STREAM_CTRL_T_OFFSET = 6656;
constexpr size_t STREAM_CTRL_BYTES = 8192;
constexpr size_t HANDLE_COUNTER_BYTES = 8192;  // the handle's control words
static_assert(STREAM_CTRL_LIMB_OFFSET + 8 * FIX_WORDS * (STREAM_NV_MAX + 1) <= STREAM_CTRL_T_OFFSET, "control words");
static_assert(STREAM_CTRL_T_OFFSET + 16 * PWA_MAX_WAVES <= STREAM_CTRL_BYTES, "control words");
static_assert(STREAM_CTRL_BYTES <= HANDLE_COUNTER_BYTES, "control words");
__host__ __device__ inline long long* stream_limbs(unsigned* counter) {
    return reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(counter) + STREAM_CTRL_LIMB_OFFSET);
}
__host__ __device__ inline double2* stream_psi_t(unsigned* counter) {
    return reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(counter) + STREAM_CTRL_T_OFFSET);
}

// ---------------------------------------------------------------- launchers --------------
// All launchers validate nothing: the C ABI layer has done it.  They return the CUDA launch
// error (cudaSuccess on success).
struct WaveTable {
    int K;
    int J[PWA_MAX_WAVES];
    int lam[PWA_MAX_WAVES];
    float Mhi[PWA_MAX_WAVES], Mlo[PWA_MAX_WAVES];
    float W[PWA_MAX_WAVES];
    float MW[PWA_MAX_WAVES];
    // waves grouped by (J, lambda) (same angular factor): group g is gord[gend[g-1] .. gend[g]-1]
    int ng;
    int gend[PWA_MAX_WAVES];
    int gord[PWA_MAX_WAVES];
};

cudaError_t launch_amplitudes(const WaveTable& wt, const float* kin, int64_t n, int64_t ld,
                              float2* A, float2* dAdM, float2* dAdW, int sm_count,
                              cudaStream_t st);

size_t normint_workspace(int K, int sm_count);
// With status given, unit weights and 16 < K <= 32 the tensor-core kernel runs (normint_tc.cu; a
// timeout of its bounded waits sets status bit 1); otherwise FP32 SIMT.  PWA_NORMINT_TC=1 / 0
// forces the tensor-core kernel for K <= 32 / the SIMT one.
cudaError_t launch_normint(const float2* A, int K, int64_t n, int64_t ld, const float* w,
                           double n_gen, double2* Psi, void* ws, int sm_count, cudaStream_t st,
                           int* status = nullptr);

size_t nll_workspace(int K, int64_t n, int P, int sm_count);
cudaError_t launch_nll_grad_scratch(const float2* A, int K, int64_t n, int64_t ld, const float2* V,
                                    const double2* Psi, double nfac, double* nll, double* grad, float2* part,
                                    size_t part_bytes, unsigned* counter, int* badw, int* status, int max_blocks,
                                    int sm_count, cudaStream_t st);
// P > 1: the autotuned tile shape (precise: the fastest shape other than the tensor-core one)
cudaError_t launch_nll(const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P,
                       const double2* Psi, double nfac, double* nll, double* grad, void* ws, size_t ws_bytes,
                       unsigned* counter, int* bad, int* status, int sm_count, cudaStream_t st, bool precise = false);

// record a message for pwa_last_error(NULL) (calls without a handle)
void record_global_error(const char* msg);

// mode bits of the fit kernels: FIT_GAUGE rotates each start so that V_0 is real >= 0 and
// freezes the phase component of V_0; FIT_POLAR makes the minimiser's coordinates of wave a
// (rho_a, phi_a) with V_a = rho_a exp(i phi_a) instead of (Re V_a, Im V_a); FIT_PAUSE pauses a
// start (status FIT_PAUSED) whose line search has backtracked FIT_PAUSE_BACKTRACKS times in a
// row, a sign that the evaluation's rounding hides the decrease it looks for, so that the
// caller can resume it (fit_resume_paused) on a more precise evaluation
constexpr int FIT_GAUGE = 1, FIT_POLAR = 2, FIT_PAUSE = 4;
constexpr int FIT_PAUSED = 4, FIT_PAUSE_BACKTRACKS = 10;
// the pause limit travels in bits 8..15 of the mode (0: FIT_PAUSE_BACKTRACKS)
constexpr int FIT_PAUSE_SHIFT = 8;
__host__ __device__ __forceinline__ int fit_pause_backtracks(int mode) {
    const int b = (mode >> FIT_PAUSE_SHIFT) & 255;
    return b > 0 ? b : FIT_PAUSE_BACKTRACKS;
}

size_t fit_workspace(int P_tot, int m);
size_t fit_eval_bytes(int P, int K);
cudaError_t fit_launch_init(void* fitws, int P_tot, int m, const float2* V0, int K, int P, int p_off, int mode,
                            float2* Vt, cudaStream_t s, int F = 0, const double* theta0 = nullptr,
                            double* theta_t = nullptr);
cudaError_t fit_launch_step(void* fitws, int P_tot, int m, const double* ft, const double* gt, float2* Vt, int K,
                            int P, int p_off, double gtol, int mode, int max_iter, cudaStream_t s, int F = 0,
                            double* theta_t = nullptr, const double* lb = nullptr);
cudaError_t fit_export_x(void* fitws, int P_tot, int m, int K, int D, int p, int mode, double* xout, cudaStream_t s);
cudaError_t fit_launch_count(void* fitws, int P_tot, int m, int* host_out, cudaStream_t s);
// paused starts -> running, their next evaluation at their accepted point; *host_count = how
// many (the stream is synchronised)
cudaError_t fit_resume_paused(void* fitws, int P_tot, int m, int* host_count, cudaStream_t s);
// the starts whose status is running, in increasing order (the stream is synchronised)
cudaError_t fit_running_list(void* fitws, int P_tot, int m, std::vector<int>& idx, cudaStream_t s);
// a subset of the parameter sets of one fit as a dense batch: Vc[i] = Vt[idx[i]] (K waves each),
// and the results of that batch back into the fit's rows: nll[idx[i]] = nll_c[i], grad[idx[i]]
// = grad_c[i] (D components each)
cudaError_t fit_gather_sets(const float2* Vt, const int* idx, int n, int K, float2* Vc, cudaStream_t s);
cudaError_t fit_scatter_sets(const double* nll_c, const double* grad_c, const int* idx, int n, int D, double* nll,
                             double* grad, cudaStream_t s);
cudaError_t fit_read_results(void* fitws, int P_tot, int m, std::vector<double>& f, std::vector<double>& gmax,
                             std::vector<int>& iter, std::vector<int>& evals, std::vector<int>& status, int D_of_p[],
                             cudaStream_t s);
cudaError_t fit_export(void* fitws, int P_tot, int m, int K, int P, int p_off, int mode, double* Vout,
                       cudaStream_t s);

// Per-start arguments of the L-BFGS step over fits of different sizes: wave count, shape
// parameters, offsets of the start's gradient row, trial V and trial theta in their packed
// arrays, convergence threshold and the shape parameters' lower bounds.
struct StepArgs {
    int K, F, goff, voff, toff;
    double gtol;
    double lb[PWA_MAX_FLOAT];
};
cudaError_t fit_launch_step_multi(void* fitws, int P_tot, int m, const StepArgs* args, const double* ft,
                                  const double* gt, float2* Vt, double* theta_t, int mode, int max_iter,
                                  cudaStream_t s);

// Many channels of floating-shape likelihoods in one persistent launch (uneven.cu).  Device
// descriptor of one channel; waves in (J, lambda)-sorted order s, ord[s] the caller's index.
struct UnevenChannel {
    const float* kin;
    const float* kin_mc;
    const float* w_mc;
    int64_t n, ld, n_mc, ld_mc;
    double scale;  // n_factor / n_gen
    int K, F, ng;
    int epi;       // events per work item
    int items_d, items_m;
    int voff, toff, goff;
    int64_t poff;  // first item-sum slot (float2 units)
    int ord[PWA_MAX_WAVES];
    double Md[PWA_MAX_WAVES], Wd[PWA_MAX_WAVES];
    signed char qM[PWA_MAX_WAVES], qW[PWA_MAX_WAVES];  // floating parameter of the mass / width, -1 fixed
    int gend[PWA_MAX_WAVES], gJ[PWA_MAX_WAVES], glam[PWA_MAX_WAVES];
};
struct UnevenPlan {
    int n_ch = 0;
    std::vector<UnevenChannel> chans;
    std::vector<int2> items;  // (channel, item within the channel: data items, then MC items)
    int64_t part_f2 = 0;      // item-sum slots (float2)
    int n_v = 0, n_theta = 0, n_grad = 0;  // lengths of the packed V, theta and gradient arrays
};
// builds the plan from validated descriptors; returns 0, or -1 with a message in err
int uneven_build_plan(const pwa_uneven_channel* ch, int n_ch, UnevenPlan* plan, char* err, size_t err_len);
size_t uneven_workspace(const UnevenPlan& p);
cudaError_t uneven_upload(const UnevenPlan& p, void* ws, cudaStream_t st);
cudaError_t uneven_launch(const UnevenPlan& p, void* ws, const float2* V, const double* theta, double* nll,
                          double* grad, int* status, int sm_count, cudaStream_t st);

size_t shape_workspace(int K, int F, int sm_count);
cudaError_t launch_nll_shape(const float2* A, const float2* dA, int K, int64_t n, int64_t ld, const float2* Am,
                             const float2* dAm, int64_t nm, int64_t ldm, const float* wm, double n_gen,
                             const int* fwave, int F, const float2* V, double nfac, double* nll, double* grad,
                             void* ws, size_t ws_bytes, unsigned* counter, int* badw, int* status, int sm_count,
                             cudaStream_t st);

size_t moments_workspace(int n_bins, int T);
size_t toy_moments_workspace(int n_bins, int T);
cudaError_t launch_moments(const float* kin, int64_t n, int64_t ld, int n_bins, double m_lo, double m_hi, double* feat,
                           void* ws, int sm_count, cudaStream_t st);
cudaError_t launch_toy_moments(const WaveTable& wt, const double* Md, const double* Wd, const float2* V, int T,
                               const double2* Psi_flat, double n_target, uint64_t seed, uint32_t stream_base,
                               int n_bins, double* feat, long long* n_acc, void* ws, cudaStream_t st);

cudaError_t launch_mlp_gemm(int M, int N, int Kc, const void* A, int a_bf16, int64_t sam, int64_t sak, const void* B,
                            int b_bf16, int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate, float* C,
                            uint16_t* Cb, int64_t ldc, int sm_count, cudaStream_t st);
// Hessian of -lnL in the real coordinates of one set V (K <= 32): the Fumili outer-product form,
// or (exact) the full second derivatives; H double [2K][2K].
size_t hessian_workspace(int K, int64_t ld, int sm_count);
cudaError_t launch_hessian(const float2* A, int K, int64_t n, int64_t ld, const float2* V, const double2* Psi,
                           double nfac, int exact, double* H, void* ws, int* status, int sm_count, cudaStream_t st);

// Psi straight from MC kinematics kin [3][ld]: the amplitudes of each tile of events are computed
// in shared memory (with the arithmetic of pwa_amplitudes) and consumed there.
cudaError_t launch_normint_kin(const WaveTable& wt, const float* kin, int K, int64_t n, int64_t ld, const float* w,
                               double n_gen, double2* Psi, void* ws, int sm_count, cudaStream_t st,
                               int* status = nullptr);
bool normint_tc_ok(int K, const float* w, const WaveTable* wt);
cudaError_t launch_normint_tc(const float2* A, int K, int64_t n, int64_t ld, const float* kin, const WaveTable* wt,
                              float4* part, int* status, int sm_count, cudaStream_t st, int* nblocks);

// The same product on the tensor cores (tcgen05 kind::f16) for a BF16 B; an FP32 A is split into
// three BF16 parts.  A timeout of its bounded wait sets status bit 1.
cudaError_t launch_mlp_gemm_tc(int M, int N, int Kc, const void* A, int a_bf16, int64_t sam, int64_t sak,
                               const void* B, int64_t sbn, int64_t sbk, const float* bias, int relu, int accumulate,
                               float* C, uint16_t* Cb, int64_t ldc, int* status, cudaStream_t st);
cudaError_t launch_mlp_relu_bwd(const uint16_t* Y, float* dY, int64_t n, int sm_count, cudaStream_t st);
cudaError_t launch_mlp_bias_grad(const float* dY, int B, int N, float* db, cudaStream_t st);
cudaError_t launch_mlp_wta(const float* out, const float* target, int B, int C, int K, float eps, float* loss,
                           float* dout, int* winner, cudaStream_t st);
cudaError_t launch_mlp_adam(float* p, const float* g, float* m, float* v, uint16_t* pb, int64_t n, float lr, float b1,
                            float b2, float eps, int step, int sm_count, cudaStream_t st);
cudaError_t launch_mlp_to_bf16(const double* x, uint16_t* y, int64_t n, float scale, int sm_count, cudaStream_t st);

size_t generate_workspace(int64_t n_cand);
cudaError_t launch_generate(const WaveTable& wt, const float2* V, uint64_t seed, uint32_t stream, int64_t cand0,
                            int64_t n_cand, double envelope, float* kin, int64_t ld_out, int64_t max_out,
                            long long* n_acc, void* ws, cudaStream_t st);

// Batched evaluation geometry: the events are cut into nchunk chunks of ev_per_chunk events (a
// multiple of the tile E) so that chunks x ceil(P / PB) blocks fill blocks_per_sm blocks per SM.
inline void batched_geometry(int64_t n, int P, int PB, int E, int sm_count, int* nchunk, int64_t* ev_per_chunk,
                             int blocks_per_sm = 2) {
    const int ntp = (P + PB - 1) / PB;
    int64_t target = ((int64_t)sm_count * blocks_per_sm) / ntp;
    if (target < 1) target = 1;
    int64_t tiles = (n + E - 1) / E;
    if (tiles < 1) tiles = 1;
    if (target > tiles) target = tiles;
    const int64_t tpc = (tiles + target - 1) / target;
    *ev_per_chunk = tpc * E;
    int64_t nc = (n + *ev_per_chunk - 1) / *ev_per_chunk;
    *nchunk = (int)(nc < 1 ? 1 : nc);
}

// -lnL (+ gradient if grad) with the intensity summed incoherently over H states, A [K][H][ld];
// one fused single-set launch per parameter set.
cudaError_t launch_nll_incoherent(const float2* A, int K, int H, int64_t n, int64_t ld, const float2* V, int P,
                                  const double2* Psi, double nfac, double* nll, double* grad, void* ws,
                                  unsigned* counter, int* status, int sm_count, cudaStream_t st);

// The autotuned batched tile shape for (K, n, P), or -1 before the first evaluation of that size.
int batched_shape(int K, int64_t n, int P);

// The tensor-core tile shape of the batched evaluation (3xTF32 emulated FP32, K <= 32).
bool tc_batched_ok(int kmax);
cudaError_t tc_batched_launch(int kmax, const float2* A, int K, int64_t n, int64_t ld, const float2* V, int P, void* ws,
                              size_t ws_bytes, int* bad, int* status, int with_grad, int sm_count, cudaStream_t st,
                              int* nchunk);

}  // namespace pwa
