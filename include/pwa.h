/*
 * pwa.h -- C ABI of the GB300 partial-wave-analysis library (libpwa.so).
 *
 * The library evaluates the unbinned extended negative log-likelihood of a coherent
 * partial-wave model (Berger, "Partial Wave Analysis using Graphics Cards", arXiv:1108.5882,
 * Sec. 2, Eqs. 1-3) and its analytic gradient in the complex production amplitudes V, the
 * per-event decay amplitudes A_a(Omega), and the Monte-Carlo normalisation integral Psi.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Complex numbers are stored as interleaved (re, im) pairs: "complex float" = 2 floats
 *    (8 bytes), "complex double" = 2 doubles (16 bytes).
 *  - Amplitude arrays are wave-major structure-of-arrays: A[a][i] for wave a < K and event
 *    i < n lives at complex offset a*ld + i, i.e. float offset 2*(a*ld + i).  ld (the leading
 *    dimension, in complex elements) must be even and >= n, and the array must be 16-byte
 *    aligned: the kernels stream two events per 16-byte load.
 *  - Kinematics arrays are float SoA [3][ld]: m_KK (GeV), cos(theta), phi (rad).
 *  - Every array argument is DEVICE memory owned by the caller unless marked "host".  The
 *    library only borrows it for the duration of the stream-ordered call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *    asynchronous on that stream: outputs are valid once the stream reaches the call.
 *  - Arguments are validated on the host before anything is launched; a rejected call returns
 *    PWA_ERR_INVALID_ARG, launches nothing, leaves the outputs untouched and records a message
 *    retrievable with pwa_last_error().
 *  - Problems found on the device (an event with intensity <= 0 or not finite) cannot be
 *    returned synchronously: the affected parameter set gets nll = +inf, and a sticky status
 *    word in the handle is set; pwa_sync_status() reads and clears it.
 *  - A handle owns a device workspace (block partial sums, completion counters).  Calls that
 *    share a handle must be ordered on one stream; use one handle per concurrent stream.
 *  - There is no CPU fallback: without a CUDA device pwa_create() fails with
 *    PWA_ERR_NO_DEVICE.
 */
#ifndef PWA_H
#define PWA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PWA_API __attribute__((visibility("default")))
#else
#define PWA_API
#endif

#define PWA_ABI_VERSION 1
#define PWA_MAX_WAVES 64
#define PWA_MAX_STATES 4   /* incoherently summed states (pwa_nll_grad_incoherent) */
#define PWA_MAX_FLOAT 8   /* floating shape parameters per likelihood (pwa_nll_grad_shape) */

typedef enum pwa_status {
    PWA_OK = 0,
    PWA_ERR_INVALID_ARG = -1,
    PWA_ERR_NO_DEVICE = -2,
    PWA_ERR_CUDA = -3,
    PWA_ERR_NONFINITE = -4,   /* some event had I_i <= 0 or a non-finite intensity */
    PWA_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    PWA_ERR_WORKSPACE = -6,   /* workspace allocation failed */
    PWA_NOT_CONVERGED = 1     /* warning from the fitters */
} pwa_status;

typedef struct pwa_handle pwa_handle;

/* One partial wave: A_a(Omega) = BW(m; mass, width) * P_J(cos theta) * exp(i lambda phi).
 * The paper leaves the amplitude model to the analysis (Sec. 2 names only "the complex decay
 * amplitude"); this library uses the fixed-width relativistic Breit-Wigner normalised to unit
 * modulus at the peak, BW(m) = M G / (M^2 - m^2 - i M G), and the ordinary Legendre
 * polynomial P_J.  Constraints: 0 <= J <= 8, |lambda| <= 8, mass > 0, width > 0. */
typedef struct pwa_wave {
    int J;
    int lambda;
    double mass;
    double width;
} pwa_wave;

/* ABI version of the loaded library (PWA_ABI_VERSION at build time). */
PWA_API int pwa_abi_version(void);

/* Human-readable name of a pwa_status value.  Never NULL. */
PWA_API const char* pwa_status_string(int status);

/* Create a handle bound to CUDA device `device`.  Fails with PWA_ERR_NO_DEVICE when no
 * device is visible and PWA_ERR_INVALID_ARG for a bad index.  *h is NULL on failure. */
PWA_API pwa_status pwa_create(pwa_handle** h, int device);

/* Release the handle and its workspace (synchronises the device first).  NULL is a no-op. */
PWA_API void pwa_destroy(pwa_handle* h);

/* Message describing the last failed call on this handle ("" if none).  Owned by the handle;
 * valid until the next call on it. h may be NULL (returns the last create() error). */
PWA_API const char* pwa_last_error(const pwa_handle* h);

/* Bytes of device workspace a pwa_nll / pwa_nll_grad call with these sizes uses. */
PWA_API size_t pwa_workspace_size(const pwa_handle* h, int K, int64_t n, int P);

/* Grow the workspace to fit calls up to (K, n, P) now, so that later calls allocate nothing
 * (required before capturing those calls into a CUDA graph). */
PWA_API pwa_status pwa_reserve(pwa_handle* h, int K, int64_t n, int P);

/* Tile shape of the batched (P > 1) evaluation chosen for calls of this size: the autotuner
 * times every feasible shape once per (K bucket, P bucket, n bucket) on the first call and keeps
 * the fastest.  0-3: FP32 SIMT kernels (0-2: E x PB tiles of 64x64, 64x32, 128x32 events x sets,
 * 3: 128x64 with bulk-copy staging); 4: the tensor-core kernel (tcgen05, FP32 products emulated
 * with three TF32 products, K <= 32).  Returns -1 before the first call of that size (or the
 * value forced by the PWA_BATCHED_SHAPE environment variable, if set and valid).  Host only. */
PWA_API int pwa_batched_shape(int K, int64_t n, int P);

/* Synchronise `stream`, then read and clear the device status word: PWA_OK, or
 * PWA_ERR_NONFINITE if any evaluation since the last check met I_i <= 0 / non-finite. */
PWA_API pwa_status pwa_sync_status(pwa_handle* h, void* stream);

/* Decay amplitudes A_a(Omega_i) (Sec. 2, Eq. 1; "facilities for amplitude calculation",
 * Sec. 3) for K waves over n events, computed in single precision (Sec. 2 precision remark).
 *   waves  host array [K]
 *   kin    float [3][ld]            m_KK, cos(theta), phi
 *   A      complex float [K][ld]    output; columns n..ld-1 are set to zero
 *   dA_dM, dA_dW   complex float [K][ld] or NULL: derivatives of A_a in the mass and width
 *                  of wave a (for fits in which masses and widths float, Sec. 2)
 * 1 <= K <= PWA_MAX_WAVES, n >= 0, ld >= n, ld even, kin and outputs 16-byte aligned. */
PWA_API pwa_status pwa_amplitudes(pwa_handle* h, const pwa_wave* waves, int K, const float* kin,
                          int64_t n, int64_t ld, float* A, float* dA_dM, float* dA_dW,
                          void* stream);

/* Decay amplitudes as pwa_amplitudes, with a mass-dependent width and Blatt-Weisskopf barrier
 * factors for a resonance decaying into two spinless daughters of masses m1, m2 (GeV) with
 * orbital angular momentum L = J of the wave and interaction radius R (GeV^-1).  The paper names
 * A_a (Sec. 2, Eq. 1) without a formula; this is the usual refinement of the fixed-width form:
 *   q(m)     = breakup momentum of m -> m1 + m2 (0 at and below threshold), q0 = q(M)
 *   B_L(z)   = Blatt-Weisskopf factor at z = (q R)^2, normalised to 1 as z -> infinity
 *   Gamma(m) = Gamma_0 (M / m) (q / q0) B_J^2(q R) / B_J^2(q0 R)
 *   BW(m)    = M Gamma_0 [B_J(q R) / B_J(q0 R)] / (M^2 - m^2 - i M Gamma(m))   (BW(M) = i)
 * A_a = BW_a(m) P_J(cos theta) exp(i lambda phi).  Single precision.
 *   waves  host array [K] with J <= 4 and mass > m1 + m2
 *   m1, m2 finite, >= 0;  R in (0, 100]
 *   kin, A, layout and alignment as pwa_amplitudes (columns n..ld-1 of A set to zero)
 * No intermediate overflows for m up to 100 GeV. */
PWA_API pwa_status pwa_amplitudes_barrier(pwa_handle* h, const pwa_wave* waves, int K, double m1, double m2,
                                          double R, const float* kin, int64_t n, int64_t ld, float* A,
                                          void* stream);

/* Monte-Carlo normalisation integral (Sec. 2, Eq. 3, inner bracket of the second term):
 *   Psi_ab = (1/n_gen) * sum_{j < n_mc} w_j A_a(j) conj(A_b(j))
 * summed in single precision per thread with compensated (double-single) carries, and
 * finalised in double precision.
 *   A_mc   complex float [K][ld]
 *   w      float [n_mc] or NULL: 1/0 acceptance flags or event weights (non-uniform MC,
 *          Sec. 2 footnote 1); NULL means w_j = 1 for every event
 *   n_gen  number of generated MC events (> 0, finite), may exceed n_mc (acceptance)
 *   Psi    complex double [K][K] output (full Hermitian matrix) */
PWA_API pwa_status pwa_normint(pwa_handle* h, const float* A_mc, int K, int64_t n_mc, int64_t ld,
                       const float* w, double n_gen, double* Psi, void* stream);

/* The same integral straight from the MC kinematics, with the amplitudes never stored: each
 * tile of events has its amplitudes computed in on-chip memory with the arithmetic of
 * pwa_amplitudes (equal to within FP32 rounding), then accumulated as pwa_normint accumulates
 * them: pwa_amplitudes followed by pwa_normint, without the K x n_mc amplitude array in HBM.
 *   waves  host array [K]; kin float [3][ld] (m_KK, cos theta, phi), 16-byte aligned
 *   w, n_gen, Psi as in pwa_normint. */
PWA_API pwa_status pwa_normint_from_kinematics(pwa_handle* h, const pwa_wave* waves, int K, const float* kin,
                                               int64_t n_mc, int64_t ld, const float* w, double n_gen,
                                               double* Psi, void* stream);

/* Extended negative log-likelihood (Sec. 2, Eq. 3 and footnote 2) for P parameter sets:
 *   nll[p] = -sum_{i<n} ln |sum_a V[p][a] A_a(i)|^2 + n_factor * sum_ab V[p][a] conj(V[p][b]) Psi_ab
 *   A      complex float [K][ld]    data amplitudes
 *   V      complex float [P][K]     production amplitudes
 *   Psi    complex double [K][K]    normalisation integral (pwa_normint)
 *   n_factor  the factor on the normalisation term (the number of data events for the
 *             extended likelihood; 1.0 gives Eq. 3 exactly as printed)
 *   nll    double [P] output (+inf for a set that met I_i <= 0 or a non-finite intensity)
 * Event sums run in single precision per thread (ln I in double-single); across threads and
 * blocks they are combined exactly in 64-bit integer fixed point for P = 1, and in double-single
 * along a fixed-order tree for P > 1.  Either way identical inputs give identical bits.
 * For P > 1 the autotuner may pick the tensor-core shape (pwa_batched_shape() == 4): FP32
 * products emulated by three TF32 products (both parts rounded to TF32), accumulated in FP32 in
 * tensor memory over 64 events, then in double-single.  It meets the same tolerances (1e-5 of the
 * -lnL scale, 1e-4 of the gradient scale); at a minimum, where the gradient cancels to ~1e-6 of
 * its terms, its error is ~4e-8 of the gradient scale (about 30x that of the SIMT shapes, 10x
 * below pwa_fit_batch's convergence threshold at 2e6 events).  PWA_BATCHED_SHAPE=0..4 forces a
 * shape. */
PWA_API pwa_status pwa_nll(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V,
                   int P, const double* Psi, double n_factor, double* nll, void* stream);

/* As pwa_nll, plus the gradient in the real coordinates of V:
 *   grad[p][2c] = d nll[p] / d Re V[p][c],  grad[p][2c+1] = d nll[p] / d Im V[p][c]
 * i.e. (Re, Im) of g_c = 2 d nll / d conj(V_c)
 *                      = -2 sum_i conj(A_c(i)) u_i / |u_i|^2 + 2 n_factor sum_a Psi_ac V_a,
 * u_i = sum_a V_a A_a(i).   grad: double [P][2K] output (zero for a non-finite set). */
PWA_API pwa_status pwa_nll_grad(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld,
                        const float* V, int P, const double* Psi, double n_factor, double* nll,
                        double* grad, void* stream);

/* Second derivatives of nll (pwa_nll) for ONE parameter set in theta = (Re V_0, Im V_0, Re V_1, ...),
 * the curvature the Fumili / Newton-type fitters use and whose inverse gives the parameter errors
 * (Sec. 4, "More control over the fitters"):
 *   r_i = grad_theta ln I_i,  r_i[2c] = 2 Re(conj(A_c) u_i) / I_i,  r_i[2c+1] = 2 Im(conj(A_c) u_i) / I_i
 *   exact = 0 (Fumili, outer-product form):  H = sum_i r_i r_i^T
 *   exact = 1:  H = sum_i r_i r_i^T - E(sum_i A_i A_i^H / I_i) + n_factor E(Psi),
 * E(C)[2a][2b] = E(C)[2a+1][2b+1] = 2 Re C_ab, E(C)[2a][2b+1] = 2 Im C_ab, E(C)[2a+1][2b] = -2 Im C_ab.
 *   A    complex float [K][ld] (ld even, 16-byte aligned), 1 <= K <= 32
 *   V    complex float [K]; Psi complex double [K][K]
 *   H    double [2K][2K] output, row-major; all NaN (and the status word set) if some I_i <= 0 or
 *        not finite.  The event sums are accumulated in double-single in a fixed order. */
PWA_API pwa_status pwa_hessian(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V,
                               const double* Psi, double n_factor, int exact, double* H, void* stream);

/* -lnL (and its gradient) with the intensity summed incoherently over H unobserved states, e.g.
 * the helicity of the radiated photon in J/psi -> gamma X (the paper's example, Sec. 2): Eq. 1
 * summed over h with the production amplitudes shared by all states,
 *   I_i = sum_h |sum_a V[p][a] A_{a,h}(i)|^2,
 *   nll[p] = -sum_i ln I_i + n_factor sum_ab V[p][a] conj(V[p][b]) Psi_ab,
 *   g_c = -2 sum_i sum_h conj(A_{c,h}(i)) u_ih / I_i + 2 n_factor sum_a Psi_ac V[p][a].
 *   A    complex float [K][H][ld]: A_{a,h}(i) at element (a H + h) ld + i; ld even, 16-byte aligned
 *   H    1 <= H <= PWA_MAX_STATES
 *   Psi  the normalisation integral summed over the states: pwa_normint over the MC amplitudes
 *        viewed as [K][H ld] with n = H ld (the (event, state) pairs are the terms of one MC
 *        sum; padding columns must be zero, as pwa_amplitudes writes them)
 *   grad double [P][2K] output, or NULL for -lnL only.
 * One parameter set per launch (the single-set kernel with a loop over h, exact fixed-point
 * grid sums, deterministic); P sets are P launches on `stream`. */
PWA_API pwa_status pwa_nll_grad_incoherent(pwa_handle* h, const float* A, int K, int H, int64_t n, int64_t ld,
                                           const float* V, int P, const double* Psi, double n_factor,
                                           double* nll, double* grad, void* stream);

/* Bound C >= max over the flat phase space of I(Omega) = |sum_a V_a A_a(Omega)|^2 (Eq. 1)
 * for m in [m_lo, m_hi], used as the accept-reject envelope of pwa_generate.  HOST function
 * (no device work): V is a HOST complex float [K] array.  On each of n_intervals equal
 * m-intervals |BW_a| is maximal at m = M_a when M_a lies inside, else at the interval end
 * nearer M_a, and |P_J| <= 1, |exp(i lambda phi)| = 1; C is the largest interval value of
 * (sum_a |V_a| max|BW_a|)^2.  Returns a negative value for invalid arguments. */
PWA_API double pwa_envelope(const pwa_wave* waves, int K, const float* V, double m_lo, double m_hi,
                    int n_intervals);

/* Toy events drawn by accept-reject from I(Omega) (Eq. 1) on the flat phase space
 * m_KK in [0.99, 3.0), cos(theta) in [-1, 1), phi in [0, 2 pi).
 * Candidate j (cand0 <= j < cand0 + n_cand) takes its phase-space point and accept uniform
 * from Philox4x32-10 (Salmon et al., SC'11) with counter (j_lo, j_hi, stream_id, 0) and key
 * (seed_lo, seed_hi); it is accepted iff u * envelope < I(Omega_j) (I in single precision).
 *   V           complex float [K] (device)
 *   kin         float [3][ld_out] output: accepted events in candidate order (first max_out)
 *   n_accepted  int64 (device) output: number accepted in the range (may exceed max_out)
 * The result is deterministic: independent of the launch geometry. */
PWA_API pwa_status pwa_generate(pwa_handle* h, const pwa_wave* waves, int K, const float* V, uint64_t seed,
                        uint32_t stream_id, int64_t cand0, int64_t n_cand, double envelope,
                        float* kin, int64_t ld_out, int64_t max_out, int64_t* n_accepted,
                        void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched fits: minimise -lnL (Sec. 2, footnote 2) over V for many starts of many fits at
 * once (repeated fits from random starts, Sec. 2 and Sec. 4).  Every start is an independent
 * L-BFGS run with Armijo backtracking whose state lives on the device; each iteration is one
 * batched -lnL + gradient evaluation (pwa_nll_grad) and one L-BFGS step kernel, replayed as a
 * captured CUDA graph between host convergence checks.  Blocks until all starts stop. */
typedef struct pwa_fit_desc {
    const float* A;       /* complex float [K][ld] data amplitudes (device) */
    int K;
    int64_t n;
    int64_t ld;
    const double* Psi;    /* complex double [K][K] normalisation integral (device) */
    double n_factor;      /* factor on the normalisation term (N_data for the extended form) */
    int P;                /* number of starts */
    const float* V0;      /* complex float [P][K] starting values (device) */
    double* V_out;        /* complex double [P][K] results (device), may be NULL */
} pwa_fit_desc;

typedef struct pwa_fit_opts {
    int max_iter;         /* accepted L-BFGS steps per start (default 1000) */
    int history;          /* L-BFGS memory, 1..20 (default 10) */
    double gtol;          /* converged when max_c |grad_c| < gtol * n_factor (default 1e-6) */
    int check_every;      /* iterations per graph replay between host checks (default 20) */
    int gauge_fix;        /* 1: rotate each start so that V_0 is real >= 0 and freeze Im V_0 */
    int use_graph;        /* 1: replay iterations as a captured CUDA graph (default 1) */
    int polar;            /* 1: minimise over (rho_a, phi_a), V_a = rho_a exp(i phi_a), instead of
                           * (Re V_a, Im V_a) (Sec. 4, "Fits with complex parameters"); the
                           * magnitude is signed and the phase unwrapped, so neither is bounded;
                           * with gauge_fix, phi_0 is frozen at 0.  grad_max and gtol then refer
                           * to these coordinates; V_out and x_out hold V either way (default 0) */
} pwa_fit_opts;

typedef struct pwa_fit_result {
    double nll;           /* -lnL at the result */
    double grad_max;      /* max_c |grad_c| at the result (frozen gauge component excluded) */
    int iterations;       /* accepted steps */
    int evaluations;      /* -lnL + gradient evaluations */
    int status;           /* 0 converged, 1 max_iter, 2 line search failed, 3 non-finite start */
} pwa_fit_result;

/* Fill *opts with the defaults above. */
PWA_API void pwa_fit_default_opts(pwa_fit_opts* opts);

/* Run n_fits fits (fits[f].P starts each).  results: HOST array of sum_f fits[f].P entries in
 * (fit, start) order.  opts may be NULL (defaults).  The workspace grows as needed (outside
 * any stream capture).  Returns PWA_OK once every start has stopped (see result.status).
 * Evaluation: the autotuned tile shape of each fit; a start whose line search backtracks 10
 * times in a row pauses, and once no start is running the paused ones resume from their
 * accepted points with the fastest FP32 SIMT shape (the tensor-core shape's rounding can hide
 * the decrease the line search looks for near a minimum); only the resumed starts are then
 * evaluated, gathered into one dense batch per fit.  PWA_FIT_PAUSE_BACKTRACKS=b (1..255)
 * overrides the 10. */
PWA_API pwa_status pwa_fit_batch(pwa_handle* h, const pwa_fit_desc* fits, int n_fits,
                                 const pwa_fit_opts* opts, pwa_fit_result* results, void* stream);

/* -lnL and its gradient when resonance masses and widths float.  Sec. 2: then neither the MC
 * bracket of Eq. 3 nor the per-event products can be precomputed, so the normalisation is the
 * MC sum itself (streamed) and the amplitudes of the floating waves are recomputed by the caller
 * (pwa_amplitudes with derivatives) at every new (M, Gamma):
 *   f = -sum_i ln|u_i|^2 + (n_factor / n_gen) sum_j w_j |u_j|^2,   u = sum_a V_a A_a,
 *   grad[2c], grad[2c+1] = d f / d Re V_c, d f / d Im V_c,
 *   grad[2K + q] = d f / d theta_q = -2 sum_i Re(conj(u_i) V_r dA_iq)/I_i
 *                                    + 2 (n_factor/n_gen) sum_j w_j Re(conj(u_j) V_r dA_jq),
 * for floating parameter q of wave r = float_wave[q] with derivative row dA_q = dA_r/dtheta_q.
 *   A, A_mc   complex float [K][ld], [K][ld_mc]   current amplitudes of data and MC events
 *   dA, dA_mc complex float [F][ld], [F][ld_mc]   derivative rows (NULL if F = 0)
 *   w_mc      float [n_mc] or NULL (acceptance flags / weights), n_gen as pwa_normint
 *   float_wave HOST int [F], 0 <= F <= PWA_MAX_FLOAT
 *   V complex float [K]; nll double [1]; grad double [2K + F] (outputs, device)
 * One parameter set.  Deterministic (fixed-order double-single sums, FP64 combination). */
PWA_API pwa_status pwa_nll_grad_shape(pwa_handle* h, const float* A, const float* dA, int K,
                                      int64_t n, int64_t ld, const float* A_mc, const float* dA_mc,
                                      int64_t n_mc, int64_t ld_mc, const float* w_mc, double n_gen,
                                      const int* float_wave, int F, const float* V,
                                      double n_factor, double* nll, double* grad, void* stream);

/* Fits with floating resonance masses and widths, many channels (independent fits of uneven
 * wave and event counts) at once.  Sec. 2: with floating shape parameters the amplitudes are
 * recomputed every iteration and the MC normalisation is summed anew; Sec. 4: at least three or
 * four free parameters per resonance.  One start per channel: x = (Re V, Im V, theta), theta the
 * floating masses/widths.  One iteration is two launches for all channels together: the
 * persistent multi-channel evaluation of pwa_nll_grad_uneven (every amplitude recomputed from the
 * kinematics at the device trial point) and one L-BFGS step per channel; the minimiser works in
 * log(mass) and log(width) (widths and masses also kept above 1e-3 GeV by a fraction-to-the-
 * boundary step limit), so result.grad_max and gtol refer to d f / d log(theta) for those;
 * check_every iterations are replayed as one captured CUDA graph between host convergence
 * checks.  A start whose shape parameter sits on its bound with the gradient pushing below it
 * stops with status 2. */
typedef struct pwa_shape_fit_desc {
    const pwa_wave* waves;      /* HOST [K]: J, lambda and the starting mass/width of each wave */
    int K;
    const float* kin;           /* data kinematics float [3][ld] (device) */
    int64_t n;
    int64_t ld;
    const float* kin_mc;        /* MC kinematics float [3][ld_mc] (device) */
    int64_t n_mc;
    int64_t ld_mc;
    const float* w_mc;          /* float [n_mc] or NULL */
    double n_gen;               /* generated MC events */
    double n_factor;            /* N_data for the extended likelihood */
    int F;                      /* floating parameters, 0..PWA_MAX_FLOAT, 2K + F <= 128 */
    const int* float_wave;      /* HOST [F]: wave index of each floating parameter */
    const int* float_kind;      /* HOST [F]: 0 = mass, 1 = width */
    float* A;                   /* unused (may be NULL): the amplitudes are recomputed on chip */
    float* A_mc;                /* unused (may be NULL) */
    float* dA;                  /* unused (may be NULL) */
    float* dA_mc;               /* unused (may be NULL) */
    const float* V0;            /* complex float [K] starting V (device) */
    double* x_out;              /* double [2K + F] result (Re V_0, Im V_0, ..., theta) or NULL */
} pwa_shape_fit_desc;

PWA_API pwa_status pwa_fit_shape_batch(pwa_handle* h, const pwa_shape_fit_desc* fits, int n_fits,
                                       const pwa_fit_opts* opts, pwa_fit_result* results,
                                       void* stream);

/* ---------------------------------------------------------------------------------------
 * Many independent channels (fits of uneven wave and event counts) with floating resonance
 * masses and widths, evaluated together in ONE persistent kernel launch (Sec. 2: repeated fits,
 * and shape parameters that float, so that neither the MC bracket of Eq. 3 nor the per-event
 * products can be precomputed; Sec. 4: fits with many free parameters).  For each channel the
 * objective and gradient are those of pwa_nll_grad_shape,
 *   f = -sum_i ln|u_i|^2 + (n_factor / n_gen) sum_j w_j |u_j|^2,  u = sum_a V_a A_a,
 * with every amplitude A_a recomputed inside the kernel from the kinematics (the model of
 * pwa_amplitudes), the floating masses and widths taken from theta.  Nothing is stored per
 * event besides the caller's kinematics. */
typedef struct pwa_uneven_channel {
    const pwa_wave* waves;      /* HOST [K]: J, lambda, mass, width (floating ones: see theta) */
    int K;                      /* 1..PWA_MAX_WAVES */
    const float* kin;           /* data kinematics float [3][ld] (device, 16-byte aligned) */
    int64_t n;
    int64_t ld;                 /* even, >= n */
    const float* kin_mc;        /* MC kinematics float [3][ld_mc] (device, 16-byte aligned) */
    int64_t n_mc;
    int64_t ld_mc;
    const float* w_mc;          /* float [n_mc] acceptance flags / weights, or NULL */
    double n_gen;               /* generated MC events (> 0) */
    double n_factor;            /* factor on the normalisation term (N_data for the extended form) */
    int F;                      /* floating shape parameters, 0..PWA_MAX_FLOAT */
    const int* float_wave;      /* HOST [F]: wave of each floating parameter */
    const int* float_kind;      /* HOST [F]: 0 = mass, 1 = width (each (wave, kind) at most once) */
} pwa_uneven_channel;

/* f and the gradient in (V, theta) of n_ch channels in one launch.  Packed device arrays, channel c
 * at the running offset of the channels before it:
 *   V      complex float [sum_c K_c]           production amplitudes
 *   theta  double [sum_c F_c]                  current values of the floating masses / widths
 *                                              (> 0; may be NULL when no channel has F > 0)
 *   nll    double [n_ch]                       output (+inf for a channel that met I_i <= 0)
 *   grad   double [sum_c (2 K_c + F_c)]        output: (Re, Im) pairs of 2 df/dconj(V_a) for the
 *                                              K_c waves in the caller's order, then df/dtheta_q
 * The kernel walks a device work list of (channel, event range) items; each item's double-single
 * sums go to a slot of their own and the block that finishes a channel's last item sums its slots
 * in a fixed order, so results are deterministic.  The work list is uploaded when the channel
 * descriptors differ from the previous call's (then the call is not capturable). */
PWA_API pwa_status pwa_nll_grad_uneven(pwa_handle* h, const pwa_uneven_channel* channels, int n_ch,
                                       const float* V, const double* theta, double* nll, double* grad,
                                       void* stream);

/* ---------------------------------------------------------------------------------------
 * Learned start proposer (no counterpart in the paper; its Sec. 2 and Sec. 4 describe the
 * expense of repeating fits from many random starts, which the proposer targets).
 * Features: per mass bin (n_bins equal bins of [m_lo, m_hi)) the event averages of the 25 real
 * spherical harmonics Y_LM(theta, phi), L <= 4, index L^2 + L + M (orthonormal, associated
 * Legendre functions with the Condon-Shortley phase).  Accumulated as exact fixed-point
 * integers (2^-36 resolution): deterministic. */

/* feat double [n_bins][25] (device) of n events kin float [3][ld]; 1 <= n_bins <= 64. */
PWA_API pwa_status pwa_moments(pwa_handle* h, const float* kin, int64_t n, int64_t ld, int n_bins,
                               double m_lo, double m_hi, double* feat, void* stream);

/* Toy samples drawn by accept-reject from I(Omega) (Eq. 1) under T production-amplitude sets
 * V [T][K] (device), reduced to features on the fly (events are never stored) on the flat
 * phase space m in [0.99, 3.0).  Toy t uses the pwa_generate candidates of (seed,
 * stream_base + t), its own envelope (the pwa_envelope bound, FP64 on the device, 4096
 * intervals) and n_cand_t = ceil(n_target * C_t / S_t) candidates, S_t = V_t^T Psi_flat V_t*
 * the mean intensity over the flat phase space (Psi_flat: pwa_normint of flat MC), so about
 * n_target events are accepted.  Outputs feat double [T][n_bins][25] and n_acc int64 [T]. */
PWA_API pwa_status pwa_toy_moments(pwa_handle* h, const pwa_wave* waves, int K, const float* V, int T,
                                   const double* Psi_flat, double n_target, uint64_t seed,
                                   uint32_t stream_base, int n_bins, double* feat, int64_t* n_acc,
                                   void* stream);

/* MLP building blocks of the proposer (BF16 = bfloat16 bit patterns in uint16_t; FP32 accumulate).
 * pwa_mlp_gemm: C[m][n] = sum_{k<Kc} A(m,k) B(n,k) (+ bias[n]) (ReLU if relu), over m < M, n < N,
 *   with A(m,k) = A[m*sam + k*sak], B(n,k) = B[n*sbn + k*sbk] (element strides; a_type/b_type
 *   0 = float32, 1 = bfloat16); writes C (float, row stride ldc) and/or C_bf16; accumulate adds
 *   the previous C.  Forward: A = X[B][in], B = W[out][in].  Data gradient: A = dY, B = W with
 *   (sbn, sbk) = (1, in).  Weight gradient: A = dY with (sam, sak) = (1, out), B = X with (1, in).
 *   With B in BF16 the product runs on the tensor cores (BF16 MMA, FP32 accumulation in tensor
 *   memory over chunks of 64, then FP32 in registers); an FP32 A is split into three BF16 parts
 *   (24 significant bits), so its products are exact as in FP32.  With B in FP32: SIMT FP32. */
PWA_API pwa_status pwa_mlp_gemm(pwa_handle* h, int M, int N, int Kc, const void* A, int a_type,
                                int64_t sam, int64_t sak, const void* B, int b_type, int64_t sbn,
                                int64_t sbk, const float* bias, int relu, int accumulate, float* C,
                                uint16_t* C_bf16, int64_t ldc, void* stream);
/* dY[i] = 0 where the layer's (post-ReLU) output Y_bf16[i] <= 0. */
PWA_API pwa_status pwa_mlp_relu_backward(pwa_handle* h, const uint16_t* Y_bf16, float* dY, int64_t n,
                                         void* stream);
/* db[n] = sum_b dY[b][n] (fixed order). */
PWA_API pwa_status pwa_mlp_bias_grad(pwa_handle* h, const float* dY, int B, int N, float* db,
                                     void* stream);
/* Winner-takes-all loss over C <= 32 candidate V (out [B][C][2K], (re, im) pairs) against the
 * target V (target [B][2K]): d_c = |V_c|^2 + |T|^2 - 2|sum_a conj(V_ca) T_a| (distance after the
 * optimal global phase), loss[b] = (1 - eps) min_c d_c + eps mean_c d_c; dout = d(mean_b loss)
 * / d out (may be NULL); winner[b] (may be NULL). */
PWA_API pwa_status pwa_mlp_wta_loss(pwa_handle* h, const float* out, const float* target, int B, int C,
                                    int K, float eps, float* loss, float* dout, int* winner,
                                    void* stream);
/* One Adam step (Kingma and Ba, bias-corrected, step >= 1) on FP32 parameters p with gradient g
 * and moments m, v; writes the BF16 copy p_bf16 if given. */
PWA_API pwa_status pwa_mlp_adam(pwa_handle* h, float* p, const float* g, float* m, float* v,
                                uint16_t* p_bf16, int64_t n, float lr, float b1, float b2, float eps,
                                int step, void* stream);
/* y = bfloat16(scale * x) (round to nearest even). */
PWA_API pwa_status pwa_mlp_to_bf16(pwa_handle* h, const double* x, uint16_t* y, int64_t n, float scale,
                                   void* stream);

/* -lnL and its gradient for ONE parameter set (P = 1) with no device allocation at all: no
 * handle, no workspace, no cudaMalloc / cudaFree, for callers that cannot allocate device
 * memory (under a memory manager that forbids allocation after start-up, as a plug-in of a
 * program that owns all device memory, or in a latency-critical loop that must not take the
 * allocator's locks and implicit synchronisation).  The paper has no counterpart; this is an
 * interface convenience.
 *   Arguments, layouts and results as pwa_nll_grad with P = 1, on the CURRENT device.
 *   Scratch: a static device array of 1,056,768 + 8,448 bytes compiled into the library (held
 *   by every GPU that loads it until exit) supports K <= PWA_MAX_WAVES and at most 1024 blocks
 *   per launch; larger K is rejected with PWA_ERR_INVALID_ARG (message via pwa_last_error(NULL)).
 *   The first call in each CUDA context looks up the scratch's device address in that context
 *   (cudaGetSymbolAddress; keyed by the driver's context id, so a context made after
 *   cudaDeviceReset, or another context current on the device, gets its own lookup); make that
 *   first call before any stream capture.
 *   Every call shares the scratch: calls ordered on one stream are safe (each call clears the
 *   scratch's counter and flag words on its stream), calls that overlap on the GPU race.
 *   A set that meets I_i <= 0 or a non-finite intensity gets nll = +inf and a zero gradient. */
PWA_API pwa_status pwa_nll_grad_noalloc(const float* A, int K, int64_t n, int64_t ld, const float* V,
                                        const double* Psi, double n_factor, double* nll,
                                        double* grad, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PWA_H */
