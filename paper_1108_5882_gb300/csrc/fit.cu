// Batched minimisation of -lnL (Sec. 2, footnote 2: -lnL is fed to the minimiser) over the
// production amplitudes V, many parameter sets at once.
//
// The paper's fits run sequentially through Minuit/Fumili (Sec. 4, "More control over the
// fitters") and are rerun from many random starts so that the lowest minimum found can be
// trusted as global (Sec. 2 and Sec. 4, "Fits with large numbers of parameters").  Here every
// start of every fit is an independent L-BFGS run whose state lives on the device:
//
//   one iteration = one batched evaluation of f and g at the trial points of all starts
//                 + k_lbfgs_step: per start, an Armijo test of the trial point; on acceptance
//                   the (s, y) pair enters the limited-memory history and the two-loop
//                   recursion gives the next direction; on rejection the step is shortened
//                   by safeguarded quadratic interpolation; the next trial point is written
//                   as single-precision V for the next evaluation.
//
// The host replays check_every iterations as one captured CUDA graph and reads back a single
// counter of running starts between replays.  No lean-fitter extras (no Hessian or error
// analysis) are done (Sec. 4 asks for exactly this control).
//
// Gauge: f is invariant under a global phase of V (Eq. 1), so the Hessian is singular along
// i V.  With gauge_fix each start is rotated so that V_0 is real and non-negative and the
// Im V_0 component of the gradient is frozen at zero.
//
// Coordinates (Sec. 4, "Fits with complex parameters": the minimiser sees real numbers, and
// either real coordinate pair for a complex parameter has drawbacks).
// Cartesian: x_2a = Re V_a, x_2a+1 = Im V_a.  Polar: x_2a = rho_a, x_2a+1 = phi_a with
// V_a = rho_a exp(i phi_a); the gradient of pwa_nll_grad is carried over by the chain rule,
//   d f / d rho = g_re cos phi + g_im sin phi,   d f / d phi = rho (g_im cos phi - g_re sin phi).
// The magnitude is signed (rho < 0 is the point (|rho|, phi + pi)), so there is no lower bound
// to enforce, and the phase is left unwrapped.  With the gauge fixed, phi_0 is the frozen
// component.  The results are reported as V in both cases.
//
// Floating shape parameters (resonance masses and widths, all positive) enter the minimiser as
// log(theta): the gradient becomes theta d f / d theta, on the scale of the V components
// instead of ~ n / Gamma, and no step can take a parameter to or below zero; a lower bound
// (1e-3 GeV) is still kept by a fraction-to-the-boundary step limit in these coordinates.
#include <cmath>
#include <vector>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int FIT_RUNNING = -1;

struct FitState {
    // per start (P_tot starts over all fits), D = 2K <= 2*PWA_MAX_WAVES
    double* x;      // [P][DM] accepted point
    double* g;      // [P][DM] gradient at x
    double* d;      // [P][DM] search direction
    double* S;      // [P][m][DM]
    double* Y;      // [P][m][DM]
    double* rho;    // [P][m]
    double* f;      // [P]
    double* alpha;  // [P]
    double* gtd;    // [P]
    int* iter;      // [P]
    int* nhist;     // [P]
    int* head;      // [P]
    int* status;    // [P]
    int* evals;     // [P]
    int* nfail;     // [P] line-search backtracks in a row
    int* running;   // [1]
};

constexpr int DM = 2 * PWA_MAX_WAVES;

// V_a of its two coordinates: Cartesian (Re, Im) or polar (rho, phi)
__device__ __forceinline__ double2 coords_to_v(double x0, double x1, bool polar) {
    if (!polar) return make_double2(x0, x1);
    double s, c;
    sincos(x1, &s, &c);
    return make_double2(x0 * c, x0 * s);
}

__device__ __forceinline__ double block_dot(const double* a, const double* b, int D, double* red) {
    // fixed-order dot product over D <= 128 components: per-thread products, shared tree
    const int t = threadIdx.x;
    red[t] = t < D ? a[t] * b[t] : 0.0;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max_abs(const double* a, int D, double* red) {
    const int t = threadIdx.x;
    red[t] = t < D ? fabs(a[t]) : 0.0;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) red[t] = fmax(red[t], red[t + o]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// init: x <- gauge-fixed V0 (double), trial <- x, status running
struct Theta0 {
    double v[PWA_MAX_FLOAT];
    double lb[PWA_MAX_FLOAT];
};

__global__ void k_fit_init(FitState st, const float2* __restrict__ V0, int K, int p_off, int mode,
                           float2* __restrict__ Vt, int F, Theta0 th, double* __restrict__ theta_t) {
    const int p = p_off + blockIdx.x, t = threadIdx.x;
    const bool gauge = mode & FIT_GAUGE, polar = mode & FIT_POLAR;
    // phase of V_0
    const float2 v0 = V0[(int64_t)blockIdx.x * K];
    double c = 1.0, s = 0.0;
    if (gauge) {
        const double r = hypot((double)v0.x, (double)v0.y);
        if (r > 0.0) {
            c = v0.x / r;
            s = -v0.y / r;  // multiply by exp(-i arg V_0)
        }
    }
    if (t < K) {
        const float2 v = V0[(int64_t)blockIdx.x * K + t];
        const double re = c * v.x - s * v.y, im = (gauge && t == 0) ? 0.0 : c * v.y + s * v.x;
        // polar: rho = |V_a|, phi = arg V_a (phi_0 = 0 exactly when the gauge is fixed)
        const double x0 = polar ? hypot(re, im) : re, x1 = polar ? atan2(im, re) : im;
        st.x[(int64_t)p * DM + 2 * t] = x0;
        st.x[(int64_t)p * DM + 2 * t + 1] = x1;
        const double2 vt = coords_to_v(x0, x1, polar);
        Vt[(int64_t)blockIdx.x * K + t] = make_float2((float)vt.x, (float)vt.y);
    }
    if (t < F) {
        st.x[(int64_t)p * DM + 2 * K + t] = log(th.v[t]);  // shape parameters: log coordinates
        theta_t[(int64_t)blockIdx.x * F + t] = th.v[t];
    }
    if (t == 0) {
        st.iter[p] = 0;
        st.nhist[p] = 0;
        st.head[p] = 0;
        st.status[p] = FIT_RUNNING;
        st.evals[p] = 0;
        st.nfail[p] = 0;
        st.alpha[p] = 0.0;  // 0: the first evaluation defines the starting point
        st.f[p] = INFINITY;
        st.gtd[p] = 0.0;
    }
}

// One L-BFGS step per start.  ft/gt: f and g at the trial point just evaluated (layout of
// pwa_nll_grad).  Writes the next trial point as single-precision V.
// Writes the trial V (and, for F > 0 floating shape parameters, the trial theta) of the next
// evaluation; x = (Re V_0, Im V_0, ..., Re V_K-1, Im V_K-1, theta_0..theta_F-1).
// Vrow: the start's trial V [K]; th_row: its trial theta [F] (unused when F = 0)
__device__ __forceinline__ void write_trial(const double* x, const double* d, double a, int K, int F, float2* Vrow,
                                            double* th_row, bool polar) {
    const int t = threadIdx.x;
    if (t < K) {
        const double2 v = coords_to_v(x[2 * t] + a * d[2 * t], x[2 * t + 1] + a * d[2 * t + 1], polar);
        Vrow[t] = make_float2((float)v.x, (float)v.y);
    }
    if (t < F) th_row[t] = exp(x[2 * K + t] + a * d[2 * K + t]);
}

// The step of start p (one block of 128 threads): fnew and gp = f and g [2K + F] at the trial point
// just evaluated; lb the lower bounds of the F shape parameters.
__device__ __forceinline__ void lbfgs_step_body(FitState& st, int p, double fnew, const double* __restrict__ gp,
                                                float2* Vrow, double* th_row, int K, int F, int m, double gtol,
                                                int mode, int max_iter, const double* lb) {
    __shared__ double red[128];
    __shared__ double q[DM], xt[DM];
    __shared__ double a_hist[32];
    __shared__ int s_action;  // 0: keep, 1: accepted, 2: rejected
    const int t = threadIdx.x;
    const int D = 2 * K + F;
    const bool gauge = mode & FIT_GAUGE, polar = mode & FIT_POLAR;
    double* x = st.x + (int64_t)p * DM;
    double* g = st.g + (int64_t)p * DM;
    double* d = st.d + (int64_t)p * DM;
    double* S = st.S + (int64_t)p * m * DM;
    double* Y = st.Y + (int64_t)p * m * DM;
    double* rho = st.rho + (int64_t)p * m;
    const int status = st.status[p];
    if (status != FIT_RUNNING) {
        write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
        return;
    }
    if (t == 0) st.evals[p] += 1;
    // trial point that was evaluated = x + alpha d (or x itself for the first evaluation)
    const double alpha = st.alpha[p];
    if (t < D) xt[t] = (alpha == 0.0) ? x[t] : x[t] + alpha * d[t];
    __syncthreads();
    if (t < D) {
        double gv = gp[t];
        if (polar && t < 2 * K) {  // chain rule from (Re V_a, Im V_a) to (rho_a, phi_a)
            const int a = t >> 1;
            double sn, cs;
            sincos(xt[2 * a + 1], &sn, &cs);
            gv = (t & 1) ? xt[2 * a] * (gp[2 * a + 1] * cs - gp[2 * a] * sn) : gp[2 * a] * cs + gp[2 * a + 1] * sn;
        }
        if (t >= 2 * K) gv *= exp(xt[t]);  // d f / d log(theta) = theta d f / d theta
        if (gauge && t == 1) gv = 0.0;
        q[t] = gv;  // gradient at the trial point (frozen gauge component)
    }
    __syncthreads();
    // directional derivative at the trial point, phi'(alpha) = g(x + alpha d) . d
    const double dphi = (alpha == 0.0) ? 0.0 : block_dot(q, d, D, red);
    if (t == 0) {
        const bool finite = isfinite(fnew);
        if (alpha == 0.0) {
            s_action = finite ? 1 : 3;
        } else {
            // Armijo, or the approximate Wolfe conditions of Hager and Zhang (2005), which
            // test the step by phi' when f differences fall below the rounding of f itself:
            // sigma phi'(0) <= phi'(alpha) <= (2 delta - 1) phi'(0), f(alpha) <= f(0) + eps |f(0)|
            const double f0 = st.f[p], g0 = st.gtd[p];
            const bool armijo = fnew <= f0 + 1e-4 * alpha * g0;
            const bool awolfe = fnew <= f0 + 1e-6 * fabs(f0) && dphi >= 0.9 * g0 && dphi <= -0.8 * g0;
            s_action = (finite && (armijo || awolfe)) ? 1 : 2;
        }
    }
    __syncthreads();
    const int action = s_action;
    if (action == 3) {  // non-finite at the start point
        if (t == 0) st.status[p] = 3;
        write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
        return;
    }
    if (action == 2) {
        // shorten the step: minimiser of the quadratic through f0, f0' and f(alpha), clamped
        if (t == 0) {
            const double f0 = st.f[p], g0 = st.gtd[p];
            double an = alpha * 0.5;
            if (isfinite(fnew) && isfinite(dphi) && dphi > 0.0) {
                an = alpha * (-g0) / (dphi - g0);  // secant zero of phi' between 0 and alpha
            } else if (isfinite(fnew)) {
                const double den = 2.0 * (fnew - f0 - g0 * alpha);
                if (den > 0.0) an = -g0 * alpha * alpha / den;  // quadratic interpolation of phi
            }
            an = fmin(fmax(an, 0.1 * alpha), 0.5 * alpha);
            st.alpha[p] = an;
            const int nf = st.nfail[p] + 1;
            st.nfail[p] = nf;
            if (an < 1e-20) st.status[p] = 2;
            else if ((mode & FIT_PAUSE) && nf >= fit_pause_backtracks(mode)) st.status[p] = FIT_PAUSED;
        }
        __syncthreads();
        if (st.status[p] == FIT_PAUSED) write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
        else write_trial(x, d, st.alpha[p], K, F, Vrow, th_row, polar);
        return;
    }
    // ---- accepted: history update with s = xt - x, y = gt - g
    const int nh = st.nhist[p];
    int head = st.head[p];
    if (alpha != 0.0) {
        double* sN = S + (int64_t)head * DM;
        double* yN = Y + (int64_t)head * DM;
        if (t < D) {
            sN[t] = xt[t] - x[t];
            yN[t] = q[t] - g[t];
        }
        __syncthreads();
        const double sy = block_dot(sN, yN, D, red);
        const double yy = block_dot(yN, yN, D, red);
        if (t == 0) {
            if (sy > 1e-12 * yy && sy > 0.0) {
                rho[head] = 1.0 / sy;
                st.head[p] = (head + 1) % m;
                st.nhist[p] = nh < m ? nh + 1 : m;
            }
        }
        __syncthreads();
    }
    if (t < D) {
        x[t] = xt[t];
        g[t] = q[t];
    }
    if (t == 0) {
        st.f[p] = fnew;
        st.nfail[p] = 0;
        if (alpha != 0.0) st.iter[p] += 1;
    }
    __syncthreads();
    const double gmax = block_max_abs(g, D, red);
    if (gmax < gtol) {
        if (t == 0) st.status[p] = 0;
        write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
        return;
    }
    if (st.iter[p] >= max_iter) {
        if (t == 0) st.status[p] = 1;
        write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
        return;
    }
    // ---- two-loop recursion: q = g; newest to oldest
    const int n_h = st.nhist[p];
    head = st.head[p];
    for (int j = 0; j < n_h; ++j) {
        const int k = (head - 1 - j + 2 * m) % m;
        const double a = rho[k] * block_dot(S + (int64_t)k * DM, q, D, red);
        if (t == 0) a_hist[k] = a;
        if (t < D) q[t] -= a * Y[(int64_t)k * DM + t];
        __syncthreads();
    }
    double gamma = 1.0;
    if (n_h > 0) {
        const int k = (head - 1 + m) % m;
        const double yy = block_dot(Y + (int64_t)k * DM, Y + (int64_t)k * DM, D, red);
        gamma = 1.0 / (rho[k] * yy);  // s.y / y.y
    }
    if (t < D) q[t] *= gamma;
    __syncthreads();
    for (int j = n_h - 1; j >= 0; --j) {
        const int k = (head - 1 - j + 2 * m) % m;
        const double b = rho[k] * block_dot(Y + (int64_t)k * DM, q, D, red);
        if (t < D) q[t] += (a_hist[k] - b) * S[(int64_t)k * DM + t];
        __syncthreads();
    }
    // d = -H g
    if (t < D) d[t] = (gauge && t == 1) ? 0.0 : -q[t];
    __syncthreads();
    double gtd = block_dot(g, d, D, red);
    double a0 = 1.0;
    if (!(gtd < 0.0) || n_h == 0) {
        // no curvature information yet (or not a descent direction): steepest descent with a
        // step that moves the largest component by 1% of the largest |x| (or 1e-3)
        if (t < D) d[t] = (gauge && t == 1) ? 0.0 : -g[t];
        __syncthreads();
        gtd = block_dot(g, d, D, red);
        const double xm = block_max_abs(x, D, red);
        a0 = 0.01 * fmax(xm, 0.1) / gmax;
        if (!(gtd < 0.0) && t == 0) st.nhist[p] = 0;
    }
    // fraction to the boundary: shape parameters stay above their lower bounds
    if (F > 0) {
        if (t == 0) {
            double amax = a0;
            for (int q = 0; q < F; ++q) {
                const double dq = d[2 * K + q];
                if (dq < 0.0) amax = fmin(amax, 0.9 * (x[2 * K + q] - log(lb[q])) / (-dq));
            }
            red[0] = amax;
        }
        __syncthreads();
        a0 = red[0];
        __syncthreads();
        if (!(a0 > 0.0)) {
            // a shape parameter sits on its lower bound and the direction points below it: no
            // feasible step is left, so the start stops (line search failed) instead of
            // evaluating zero-length steps until the iteration bound
            if (t == 0) st.status[p] = 2;
            write_trial(x, x, 0.0, K, F, Vrow, th_row, polar);
            return;
        }
    }
    if (t == 0) {
        st.gtd[p] = gtd;
        st.alpha[p] = a0;
    }
    write_trial(x, d, a0, K, F, Vrow, th_row, polar);
}

__global__ void __launch_bounds__(128) k_lbfgs_step(FitState st, const double* __restrict__ ft,
                                                    const double* __restrict__ gt, float2* __restrict__ Vt, int K,
                                                    int p_off, int m, double gtol, int mode, int max_iter, int F,
                                                    double* __restrict__ theta_t, Theta0 th) {
    const int pl = blockIdx.x;
    lbfgs_step_body(st, p_off + pl, ft[pl], gt + (int64_t)pl * (2 * K + F), Vt + (int64_t)pl * K,
                    theta_t + (int64_t)pl * F, K, F, m, gtol, mode, max_iter, th.lb);
}

// One step for every start p of fits of different sizes: start p's K, F, gradient row, trial V
// and theta offsets, tolerance and bounds from args[p]; f of start p is ft[p].
__global__ void __launch_bounds__(128) k_lbfgs_step_multi(FitState st, const StepArgs* __restrict__ args,
                                                          const double* __restrict__ ft, const double* __restrict__ gt,
                                                          float2* __restrict__ Vt, double* __restrict__ theta_t, int m,
                                                          int mode, int max_iter) {
    const int p = blockIdx.x;
    const StepArgs a = args[p];
    lbfgs_step_body(st, p, ft[p], gt + a.goff, Vt + a.voff, theta_t + a.toff, a.K, a.F, m, a.gtol, mode, max_iter,
                    a.lb);
}

// paused -> running with alpha = 0: the next evaluation (at the trial point x, written when the
// start paused) replaces f and g at x and the line search starts afresh; the count to out
__global__ void k_fit_resume(FitState st, int P, int* __restrict__ out) {
    __shared__ int s[256];
    int c = 0;
    for (int i = threadIdx.x; i < P; i += 256) {
        if (st.status[i] == FIT_PAUSED) {
            st.status[i] = FIT_RUNNING;
            st.alpha[i] = 0.0;
            st.nfail[i] = 0;
            ++c;
        }
    }
    s[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_count_running(const int* __restrict__ status, int P, int* __restrict__ out) {
    __shared__ int s[256];
    int c = 0;
    for (int i = threadIdx.x; i < P; i += 256) c += status[i] == FIT_RUNNING;
    s[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// V_a of start p from its coordinates.  With the gauge fixed, a start whose V_0 ended on the
// negative real axis is reported as -V, the same point of f, so that V_0 >= 0 as documented.
__device__ __forceinline__ double2 export_v(const FitState& st, int p, int a, int mode) {
    const double* x = st.x + (int64_t)p * DM;
    double2 v = coords_to_v(x[2 * a], x[2 * a + 1], mode & FIT_POLAR);
    if ((mode & FIT_GAUGE) && coords_to_v(x[0], x[1], mode & FIT_POLAR).x < 0.0) v = make_double2(-v.x, -v.y);
    return v;
}

__global__ void k_fit_export(FitState st, int K, int p_off, int mode, double2* __restrict__ Vout) {
    const int pl = blockIdx.x, p = p_off + pl, t = threadIdx.x;
    if (t < K && Vout) Vout[(int64_t)pl * K + t] = export_v(st, p, t, mode);
}

// (Re V_0, Im V_0, ..., theta) of start p
__global__ void k_fit_export_x(FitState st, int K, int D, int p, int mode, double* __restrict__ xout) {
    const int t = threadIdx.x;
    if (t < K) {
        const double2 v = export_v(st, p, t, mode);
        xout[2 * t] = v.x;
        xout[2 * t + 1] = v.y;
    } else if (t >= 2 * K && t < D) {
        xout[t] = exp(st.x[(int64_t)p * DM + t]);
    }
}

}  // namespace

size_t fit_state_bytes(int P_tot, int m) {
    const size_t p = (size_t)P_tot;
    return sizeof(double) * p * DM * (3 + 2 * (size_t)m) + sizeof(double) * p * ((size_t)m + 3) +
           sizeof(int) * (p * 5 + 16) + 1024;
}

struct FitLayout {
    FitState st;
};

static FitState carve(void* base, int P_tot, int m) {
    char* c = reinterpret_cast<char*>(base);
    auto take = [&](size_t bytes) {
        void* r = c;
        c += (bytes + 255) & ~size_t(255);
        return r;
    };
    FitState s;
    const size_t p = (size_t)P_tot;
    s.x = (double*)take(sizeof(double) * p * DM);
    s.g = (double*)take(sizeof(double) * p * DM);
    s.d = (double*)take(sizeof(double) * p * DM);
    s.S = (double*)take(sizeof(double) * p * m * DM);
    s.Y = (double*)take(sizeof(double) * p * m * DM);
    s.rho = (double*)take(sizeof(double) * p * m);
    s.f = (double*)take(sizeof(double) * p);
    s.alpha = (double*)take(sizeof(double) * p);
    s.gtd = (double*)take(sizeof(double) * p);
    s.iter = (int*)take(sizeof(int) * p);
    s.nhist = (int*)take(sizeof(int) * p);
    s.head = (int*)take(sizeof(int) * p);
    s.status = (int*)take(sizeof(int) * p);
    s.evals = (int*)take(sizeof(int) * p);
    s.nfail = (int*)take(sizeof(int) * p);
    s.running = (int*)take(sizeof(int) * 16);
    return s;
}

size_t fit_workspace(int P_tot, int m) {
    // carve() rounds every array to 256 bytes
    const size_t p = (size_t)P_tot;
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    return 3 * r(sizeof(double) * p * DM) + 2 * r(sizeof(double) * p * m * DM) + r(sizeof(double) * p * m) +
           3 * r(sizeof(double) * p) + 6 * r(sizeof(int) * p) + r(sizeof(int) * 16);
}

// Per-fit device buffers for the evaluation (V trial, nll, grad) live in `evalbuf`.
size_t fit_eval_bytes(int P, int K) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    return r(sizeof(float2) * (size_t)P * K) + r(sizeof(double) * P) + r(sizeof(double) * (size_t)P * 2 * K);
}

static Theta0 make_theta0(int F, const double* theta0, const double* lb) {
    Theta0 th;
    for (int q = 0; q < PWA_MAX_FLOAT; ++q) {
        th.v[q] = q < F && theta0 ? theta0[q] : 0.0;
        th.lb[q] = q < F && lb ? lb[q] : 0.0;
    }
    return th;
}

cudaError_t fit_launch_init(void* fitws, int P_tot, int m, const float2* V0, int K, int P, int p_off, int mode,
                            float2* Vt, cudaStream_t s, int F, const double* theta0, double* theta_t) {
    FitState st = carve(fitws, P_tot, m);
    k_fit_init<<<P, 128, 0, s>>>(st, V0, K, p_off, mode, Vt, F, make_theta0(F, theta0, nullptr), theta_t);
    return cudaGetLastError();
}

cudaError_t fit_launch_step(void* fitws, int P_tot, int m, const double* ft, const double* gt, float2* Vt, int K,
                            int P, int p_off, double gtol, int mode, int max_iter, cudaStream_t s, int F,
                            double* theta_t, const double* lb) {
    FitState st = carve(fitws, P_tot, m);
    k_lbfgs_step<<<P, 128, 0, s>>>(st, ft, gt, Vt, K, p_off, m, gtol, mode, max_iter, F, theta_t,
                                   make_theta0(F, nullptr, lb));
    return cudaGetLastError();
}

cudaError_t fit_launch_step_multi(void* fitws, int P_tot, int m, const StepArgs* args, const double* ft,
                                  const double* gt, float2* Vt, double* theta_t, int mode, int max_iter,
                                  cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    k_lbfgs_step_multi<<<P_tot, 128, 0, s>>>(st, args, ft, gt, Vt, theta_t, m, mode, max_iter);
    return cudaGetLastError();
}

cudaError_t fit_launch_count(void* fitws, int P_tot, int m, int* host_out, cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    k_count_running<<<1, 256, 0, s>>>(st.status, P_tot, st.running);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(host_out, st.running, sizeof(int), cudaMemcpyDeviceToHost, s);
}

cudaError_t fit_resume_paused(void* fitws, int P_tot, int m, int* host_count, cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    k_fit_resume<<<1, 256, 0, s>>>(st, P_tot, st.running);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_count, st.running, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t fit_running_list(void* fitws, int P_tot, int m, std::vector<int>& idx, cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    std::vector<int> status(P_tot);
    cudaError_t e = cudaMemcpyAsync(status.data(), st.status, sizeof(int) * P_tot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    idx.clear();
    for (int p = 0; p < P_tot; ++p)
        if (status[p] == FIT_RUNNING) idx.push_back(p);
    return e;
}

__global__ void k_gather_sets(const float2* __restrict__ Vt, const int* __restrict__ idx, int n, int K,
                              float2* __restrict__ Vc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * K; i += gridDim.x * blockDim.x)
        Vc[i] = Vt[(int64_t)idx[i / K] * K + i % K];
}

__global__ void k_scatter_sets(const double* __restrict__ nll_c, const double* __restrict__ grad_c,
                               const int* __restrict__ idx, int n, int D, double* __restrict__ nll,
                               double* __restrict__ grad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * D; i += gridDim.x * blockDim.x) {
        const int r = i / D, c = i % D;
        grad[(int64_t)idx[r] * D + c] = grad_c[i];
        if (c == 0) nll[idx[r]] = nll_c[r];
    }
}

cudaError_t fit_gather_sets(const float2* Vt, const int* idx, int n, int K, float2* Vc, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n * K + 255) / 256;
    k_gather_sets<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(Vt, idx, n, K, Vc);
    return cudaGetLastError();
}

cudaError_t fit_scatter_sets(const double* nll_c, const double* grad_c, const int* idx, int n, int D, double* nll,
                             double* grad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n * D + 255) / 256;
    k_scatter_sets<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(nll_c, grad_c, idx, n, D, nll, grad);
    return cudaGetLastError();
}

cudaError_t fit_read_results(void* fitws, int P_tot, int m, std::vector<double>& f, std::vector<double>& gmax,
                             std::vector<int>& iter, std::vector<int>& evals, std::vector<int>& status, int D_of_p[],
                             cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    f.resize(P_tot);
    iter.resize(P_tot);
    evals.resize(P_tot);
    status.resize(P_tot);
    gmax.resize(P_tot);
    std::vector<double> g((size_t)P_tot * DM);
    cudaError_t e = cudaMemcpyAsync(f.data(), st.f, sizeof(double) * P_tot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(iter.data(), st.iter, sizeof(int) * P_tot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(evals.data(), st.evals, sizeof(int) * P_tot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), st.status, sizeof(int) * P_tot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.data(), st.g, sizeof(double) * P_tot * DM, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int p = 0; p < P_tot; ++p) {
        double mx = 0.0;
        for (int c = 0; c < D_of_p[p]; ++c) mx = fmax(mx, fabs(g[(size_t)p * DM + c]));
        gmax[p] = mx;
    }
    return cudaSuccess;
}

cudaError_t fit_export_x(void* fitws, int P_tot, int m, int K, int D, int p, int mode, double* xout, cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    k_fit_export_x<<<1, 128, 0, s>>>(st, K, D, p, mode, xout);
    return cudaGetLastError();
}

cudaError_t fit_export(void* fitws, int P_tot, int m, int K, int P, int p_off, int mode, double* Vout,
                       cudaStream_t s) {
    FitState st = carve(fitws, P_tot, m);
    k_fit_export<<<P, 128, 0, s>>>(st, K, p_off, mode, reinterpret_cast<double2*>(Vout));
    return cudaGetLastError();
}

}  // namespace pwa
