/*
 * pwa_oracle.c -- plain, single-threaded FP64 CPU oracle for the partial-wave-analysis
 * likelihood of Berger, "Partial Wave Analysis using Graphics Cards" (arXiv:1108.5882).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file;
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.  It shares
 * no header, helper, table or constant with the CUDA library.
 *
 * What is computed, and where the paper defines it:
 *   - coherent intensity I(Omega) = |sum_a V_a A_a(Omega)|^2                     (Sec. 2, Eq. 1)
 *   - MC normalisation Psi_ab = (1/N_gen) sum_{j in acc} w_j A_a(j) conj(A_b(j)) (Sec. 2, Eq. 3,
 *     inner bracket of the second term; acceptance/weights from the text around Eq. 2)
 *   - -lnL fed to the minimiser (Sec. 2, footnote 2), extended form
 *       f(V) = -sum_i ln I_i + n_factor * sum_ab V_a conj(V_b) Psi_ab
 *     and its gradient g_c = dF/dRe V_c + i dF/dIm V_c = 2 dF/dconj(V_c)
 *   - the same with the intensity summed incoherently over unobserved states h,
 *     I = sum_h |sum_a V_a A_{a,h}|^2 (Eq. 1 summed over h; the paper's own example, J/psi ->
 *     gamma X, has such a state: the photon helicity)
 *   - the Hessian of -lnL in the real coordinates of V: the Fumili outer-product form and the
 *     exact form (Sec. 4, the fitters)
 *   - the double-sum form of Eq. 3 in long double (used only to pin the O(K) form above)
 *   - the amplitude model A_a = BW_a(m) P_J(cos th) exp(i lambda phi) and its derivatives
 *     in the resonance mass and width (the paper gives no amplitude formula; the reading is
 *     the fixed-width, unit-peak relativistic Breit-Wigner with ordinary Legendre P_J).
 *   - the same model with a mass-dependent width and Blatt-Weisskopf barrier factors for a
 *     two-body decay X -> 1 + 2 into spinless daughters (orbital angular momentum L = J).
 *
 * Everything is the textbook definition evaluated in double precision, in the order the
 * definition states, with Neumaier-compensated accumulation of the long event sums.
 *
 * Parity pins: every function here is pinned by tests against closed forms, identities,
 * library routines or brute force (see tests/test_oracle_*.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------- compensated summation (Neumaier) ---------------------------------------- */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

/* ---------- amplitude model ----------------------------------------------------------- */

/* Fixed-width relativistic Breit-Wigner, normalised to unit modulus at the peak:
 * BW(m) = M*Gamma / (M^2 - m^2 - i M Gamma).  At m = M it equals i, and |BW| <= 1. */
cplx orc_bw(double m, double M, double W) {
    cplx den = (M * M - m * m) - I * (M * W);
    return (M * W) / den;
}

/* d BW / d M and d BW / d Gamma by the quotient rule, written out unsimplified. */
void orc_bw_deriv(double m, double M, double W, cplx* dM, cplx* dW) {
    cplx num = M * W;
    cplx den = (M * M - m * m) - I * (M * W);
    cplx dnum_dM = W, dden_dM = 2.0 * M - I * W;
    cplx dnum_dW = M, dden_dW = -I * M;
    *dM = (dnum_dM * den - num * dden_dM) / (den * den);
    *dW = (dnum_dW * den - num * dden_dW) / (den * den);
}

/* Ordinary Legendre polynomial P_J(x) by Bonnet's recurrence
 * (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
double orc_legendre(int J, double x) {
    if (J == 0) return 1.0;
    double pm = 1.0, p = x;
    for (int n = 1; n < J; ++n) {
        double pn = ((2.0 * n + 1.0) * x * p - n * pm) / (n + 1.0);
        pm = p;
        p = pn;
    }
    return p;
}

/* A_a(Omega_i) for K waves over n events.  kin is float32 SoA [3][ld]: m, cos(theta), phi.
 * A, dAdM, dAdW are complex double [K][n] (dAdM/dAdW may be NULL). */
void orc_amplitudes(int K, const int* J, const int* lam, const double* M, const double* W,
                    int64_t n, const float* kin, int64_t ld,
                    double* A, double* dAdM, double* dAdW) {
    cplx* Ac = (cplx*)A;
    cplx* dM = (cplx*)dAdM;
    cplx* dW = (cplx*)dAdW;
    for (int a = 0; a < K; ++a) {
        for (int64_t i = 0; i < n; ++i) {
            double m = kin[i], ct = kin[ld + i], ph = kin[2 * ld + i];
            cplx ang = orc_legendre(J[a], ct) * cexp(I * (lam[a] * ph));
            Ac[(int64_t)a * n + i] = orc_bw(m, M[a], W[a]) * ang;
            if (dM || dW) {
                cplx bm, bw;
                orc_bw_deriv(m, M[a], W[a], &bm, &bw);
                if (dM) dM[(int64_t)a * n + i] = bm * ang;
                if (dW) dW[(int64_t)a * n + i] = bw * ang;
            }
        }
    }
}

/* ---------- mass-dependent width and barrier factors ---------------------------------- */

/* Breakup momentum of a state of mass m decaying into masses m1, m2, in its rest frame:
 * q^2 = lambda(m^2, m1^2, m2^2) / (4 m^2) with the Kallen function
 * lambda(x, y, w) = x^2 + y^2 + w^2 - 2xy - 2xw - 2yw.  Zero at and below threshold. */
double orc_breakup_q(double m, double m1, double m2) {
    if (!(m > m1 + m2)) return 0.0;
    double x = m * m, y = m1 * m1, w = m2 * m2;
    double lam = x * x + y * y + w * w - 2.0 * x * y - 2.0 * x * w - 2.0 * y * w;
    return lam > 0.0 ? sqrt(lam) / (2.0 * m) : 0.0;
}

/* Squared Blatt-Weisskopf barrier factor of orbital angular momentum L <= 4 at z = (q R)^2,
 * normalised to 1 as z -> infinity: B_L^2(z) = z^L / P_L(z) with the textbook polynomials
 *   P_0 = 1, P_1 = 1 + z, P_2 = 9 + 3z + z^2, P_3 = 225 + 45z + 6z^2 + z^3,
 *   P_4 = 11025 + 1575z + 135z^2 + 10z^3 + z^4
 * (P_L(z) = |x^(L+1) h_L(x)|^2, h_L the outgoing spherical Hankel function, x^2 = z). */
double orc_barrier2(int L, double z) {
    switch (L) {
        case 0: return 1.0;
        case 1: return z / (1.0 + z);
        case 2: return z * z / (9.0 + 3.0 * z + z * z);
        case 3: return z * z * z / (225.0 + 45.0 * z + 6.0 * z * z + z * z * z);
        case 4: return z * z * z * z / (11025.0 + 1575.0 * z + 135.0 * z * z + 10.0 * z * z * z + z * z * z * z);
        default: return NAN;
    }
}

/* Breit-Wigner of a resonance (M, Gamma_0) decaying to m1 + m2 with L = J and radius R:
 *   Gamma(m) = Gamma_0 (M / m) (q / q0) B_L^2(q^2 R^2) / B_L^2(q0^2 R^2),   q0 = q(M),
 *   BW(m)    = M Gamma_0 [B_L(q R) / B_L(q0 R)] / (M^2 - m^2 - i M Gamma(m)),
 * which keeps the unit modulus at the peak, BW(M) = i, of the fixed-width form. */
cplx orc_bw_barrier(double m, double M, double W, int L, double m1, double m2, double R) {
    double q = orc_breakup_q(m, m1, m2), q0 = orc_breakup_q(M, m1, m2);
    double b2 = orc_barrier2(L, q * q * R * R), b20 = orc_barrier2(L, q0 * q0 * R * R);
    double Gm = W * (M / m) * (q / q0) * (b2 / b20);
    cplx den = (M * M - m * m) - I * (M * Gm);
    return (M * W * sqrt(b2 / b20)) / den;
}

/* A_a(Omega_i) with the barrier Breit-Wigner above, L_a = J_a; layout as orc_amplitudes. */
void orc_amplitudes_barrier(int K, const int* J, const int* lam, const double* M, const double* W,
                            double m1, double m2, double R, int64_t n, const float* kin, int64_t ld,
                            double* A) {
    cplx* Ac = (cplx*)A;
    for (int a = 0; a < K; ++a)
        for (int64_t i = 0; i < n; ++i) {
            double m = kin[i], ct = kin[ld + i], ph = kin[2 * ld + i];
            cplx ang = orc_legendre(J[a], ct) * cexp(I * (lam[a] * ph));
            Ac[(int64_t)a * n + i] = orc_bw_barrier(m, M[a], W[a], J[a], m1, m2, R) * ang;
        }
}

/* ---------- MC normalisation integral -------------------------------------------------- */

/* Psi_ab = (1/n_gen) sum_j w_j A_a(j) conj(A_b(j)); A is complex64 interleaved [K][ld]
 * (the same array the GPU consumes, promoted to double).  w may be NULL (all ones).
 * Psi is complex double [K][K], full matrix. */
void orc_normint(int K, int64_t n, const float* A, int64_t ld, const float* w, double n_gen,
                 double* Psi) {
    cplx* out = (cplx*)Psi;
    for (int a = 0; a < K; ++a) {
        for (int b = 0; b < K; ++b) {
            nsum re = {0, 0}, im = {0, 0};
            for (int64_t j = 0; j < n; ++j) {
                cplx Aa = A[2 * ((int64_t)a * ld + j)] + I * A[2 * ((int64_t)a * ld + j) + 1];
                cplx Ab = A[2 * ((int64_t)b * ld + j)] + I * A[2 * ((int64_t)b * ld + j) + 1];
                double wj = w ? (double)w[j] : 1.0;
                cplx t = wj * Aa * conj(Ab);
                nsum_add(&re, creal(t));
                nsum_add(&im, cimag(t));
            }
            out[a * K + b] = (nsum_get(&re) + I * nsum_get(&im)) / n_gen;
        }
    }
}

/* ---------- negative log-likelihood and gradient --------------------------------------- */

/* f(V) and g(V) for P parameter sets.  A: complex64 interleaved [K][ld]; V: complex double
 * [P][K]; Psi: complex double [K][K].  Outputs nll[P], grad[P][2K] = (Re g_c, Im g_c).
 * cond_f[P] = max(|f|, sum_i |ln I_i|, n_factor*|S|) and cond_g[P][K] =
 * 2 sum_i |A_ic| s_i / I_i + 2 n_factor sum_a |Psi_ac||V_a|, s_i = sum_a |V_a||A_ia| >= |u_i|,
 * are the scales the parity tolerances are taken relative to (either may be NULL).  s_i is the
 * forward-error scale of the sum u_i: a single-precision evaluation of u_i (Sec. 2 precision
 * remark) is off by about eps * s_i, which moves the term conj(A_ic)/conj(u_i) by about
 * |A_ic| eps s_i / I_i, large where u_i nearly cancels (s_i >> |u_i|).
 * Returns the number of parameter sets with a non-positive or non-finite intensity at some
 * event; those get nll = +inf and a zero gradient. */
int orc_nll_grad(int K, int64_t n, const float* A, int64_t ld, int P, const double* Vd,
                 const double* Psid, double n_factor, double* nll, double* grad,
                 double* cond_f, double* cond_g) {
    const cplx* V = (const cplx*)Vd;
    const cplx* Psi = (const cplx*)Psid;
    int bad_sets = 0;
    cplx* Ai = (cplx*)malloc(sizeof(cplx) * (size_t)K);
    nsum* gre = (nsum*)malloc(sizeof(nsum) * (size_t)K);
    nsum* gim = (nsum*)malloc(sizeof(nsum) * (size_t)K);
    double* gsc = (double*)malloc(sizeof(double) * (size_t)K);
    for (int p = 0; p < P; ++p) {
        const cplx* Vp = V + (int64_t)p * K;
        nsum lnsum = {0, 0};
        double lnabs = 0.0;
        int bad = 0;
        for (int c = 0; c < K; ++c) { gre[c].s = gre[c].c = gim[c].s = gim[c].c = 0.0; gsc[c] = 0.0; }
        for (int64_t i = 0; i < n; ++i) {
            cplx u = 0.0;
            double su = 0.0;
            for (int a = 0; a < K; ++a) {
                Ai[a] = A[2 * ((int64_t)a * ld + i)] + I * A[2 * ((int64_t)a * ld + i) + 1];
                u += Vp[a] * Ai[a];
                su += cabs(Vp[a]) * cabs(Ai[a]);
            }
            double Ii = creal(u) * creal(u) + cimag(u) * cimag(u);
            if (!(Ii > 0.0) || !isfinite(Ii)) { bad = 1; continue; }
            double l = log(Ii);
            nsum_add(&lnsum, l);
            lnabs += fabs(l);
            /* d(-ln I_i)/d conj(V_c) = -conj(A_ic) u_i / I_i; g = 2 * that */
            for (int c = 0; c < K; ++c) {
                cplx t = conj(Ai[c]) * u / Ii;
                nsum_add(&gre[c], -2.0 * creal(t));
                nsum_add(&gim[c], -2.0 * cimag(t));
                gsc[c] += 2.0 * cabs(Ai[c]) * su / Ii;
            }
        }
        /* normalisation term S = sum_ab V_a conj(V_b) Psi_ab and its gradient 2 n sum_a Psi_ac V_a */
        cplx S = 0.0;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) S += Vp[a] * conj(Vp[b]) * Psi[a * K + b];
        double f = -nsum_get(&lnsum) + n_factor * creal(S);
        for (int c = 0; c < K; ++c) {
            cplx nt = 0.0;
            double nts = 0.0;
            for (int a = 0; a < K; ++a) {
                nt += Psi[a * K + c] * Vp[a];
                nts += cabs(Psi[a * K + c]) * cabs(Vp[a]);
            }
            double gr = nsum_get(&gre[c]) + 2.0 * n_factor * creal(nt);
            double gi = nsum_get(&gim[c]) + 2.0 * n_factor * cimag(nt);
            grad[(int64_t)p * 2 * K + 2 * c] = bad ? 0.0 : gr;
            grad[(int64_t)p * 2 * K + 2 * c + 1] = bad ? 0.0 : gi;
            if (cond_g) cond_g[(int64_t)p * K + c] = gsc[c] + 2.0 * fabs(n_factor) * nts;
        }
        nll[p] = bad ? INFINITY : f;
        if (cond_f) {
            double cf = fabs(f);
            if (lnabs > cf) cf = lnabs;
            if (fabs(n_factor * creal(S)) > cf) cf = fabs(n_factor * creal(S));
            cond_f[p] = cf;
        }
        bad_sets += bad;
    }
    free(Ai); free(gre); free(gim); free(gsc);
    return bad_sets;
}

/* Incoherent sum over H unobserved states (e.g. the radiated photon's helicity in J/psi ->
 * gamma X): the amplitudes carry a state index h, A_{a,h}(i) at A[2 ((a H + h) ld + i)], the
 * production amplitudes V_a are shared by all h, and the intensity adds the states
 * incoherently (a sum of Eq. 1 over h):
 *   I_i = sum_h |u_ih|^2,  u_ih = sum_a V_a A_{a,h}(i).
 * The extended -lnL keeps the form of Eq. 3 with the normalisation integral summed over h,
 * Psi_ab = (1/N_gen) sum_j sum_h A_{a,h}(j) conj(A_{b,h}(j)) (the caller passes that Psi):
 *   f = -sum_i ln I_i + n_factor sum_ab V_a conj(V_b) Psi_ab,
 *   g_c = 2 df/dconj(V_c) = -2 sum_i sum_h conj(A_{c,h}(i)) u_ih / I_i + 2 n_factor sum_a Psi_ac V_a.
 * cond_f / cond_g as in orc_nll_grad, with s_ih = sum_a |V_a| |A_{a,h}(i)| per state. */
int orc_nll_grad_incoherent(int K, int H, int64_t n, const float* A, int64_t ld, int P, const double* Vd,
                            const double* Psid, double n_factor, double* nll, double* grad,
                            double* cond_f, double* cond_g) {
    const cplx* V = (const cplx*)Vd;
    const cplx* Psi = (const cplx*)Psid;
    int bad_sets = 0;
    cplx* Ai = (cplx*)malloc(sizeof(cplx) * (size_t)K * (size_t)H);
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)H);
    double* su = (double*)malloc(sizeof(double) * (size_t)H);
    nsum* gre = (nsum*)malloc(sizeof(nsum) * (size_t)K);
    nsum* gim = (nsum*)malloc(sizeof(nsum) * (size_t)K);
    double* gsc = (double*)malloc(sizeof(double) * (size_t)K);
    for (int p = 0; p < P; ++p) {
        const cplx* Vp = V + (int64_t)p * K;
        nsum lnsum = {0, 0};
        double lnabs = 0.0;
        int bad = 0;
        for (int c = 0; c < K; ++c) { gre[c].s = gre[c].c = gim[c].s = gim[c].c = 0.0; gsc[c] = 0.0; }
        for (int64_t i = 0; i < n; ++i) {
            double Ii = 0.0;
            for (int h = 0; h < H; ++h) {
                u[h] = 0.0;
                su[h] = 0.0;
                for (int a = 0; a < K; ++a) {
                    const int64_t o = 2 * (((int64_t)a * H + h) * ld + i);
                    Ai[a * H + h] = A[o] + I * A[o + 1];
                    u[h] += Vp[a] * Ai[a * H + h];
                    su[h] += cabs(Vp[a]) * cabs(Ai[a * H + h]);
                }
                Ii += creal(u[h]) * creal(u[h]) + cimag(u[h]) * cimag(u[h]);
            }
            if (!(Ii > 0.0) || !isfinite(Ii)) { bad = 1; continue; }
            double l = log(Ii);
            nsum_add(&lnsum, l);
            lnabs += fabs(l);
            for (int c = 0; c < K; ++c) {
                cplx t = 0.0;
                double ts = 0.0;
                for (int h = 0; h < H; ++h) {
                    t += conj(Ai[c * H + h]) * u[h];
                    ts += cabs(Ai[c * H + h]) * su[h];
                }
                t /= Ii;
                nsum_add(&gre[c], -2.0 * creal(t));
                nsum_add(&gim[c], -2.0 * cimag(t));
                gsc[c] += 2.0 * ts / Ii;
            }
        }
        cplx S = 0.0;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) S += Vp[a] * conj(Vp[b]) * Psi[a * K + b];
        double f = -nsum_get(&lnsum) + n_factor * creal(S);
        for (int c = 0; c < K; ++c) {
            cplx nt = 0.0;
            double nts = 0.0;
            for (int a = 0; a < K; ++a) {
                nt += Psi[a * K + c] * Vp[a];
                nts += cabs(Psi[a * K + c]) * cabs(Vp[a]);
            }
            double gr = nsum_get(&gre[c]) + 2.0 * n_factor * creal(nt);
            double gi = nsum_get(&gim[c]) + 2.0 * n_factor * cimag(nt);
            grad[(int64_t)p * 2 * K + 2 * c] = bad ? 0.0 : gr;
            grad[(int64_t)p * 2 * K + 2 * c + 1] = bad ? 0.0 : gi;
            if (cond_g) cond_g[(int64_t)p * K + c] = gsc[c] + 2.0 * fabs(n_factor) * nts;
        }
        nll[p] = bad ? INFINITY : f;
        if (cond_f) {
            double cf = fabs(f);
            if (lnabs > cf) cf = lnabs;
            if (fabs(n_factor * creal(S)) > cf) cf = fabs(n_factor * creal(S));
            cond_f[p] = cf;
        }
        bad_sets += bad;
    }
    free(Ai); free(u); free(su); free(gre); free(gim); free(gsc);
    return bad_sets;
}

/* Second derivatives of f = -sum_i ln I_i + n_factor S in the real coordinates
 * theta = (Re V_0, Im V_0, Re V_1, ...) of one parameter set, for the Fumili / Gauss-Newton
 * step the paper's fitters take (Sec. 4: Minuit and Fumili):
 *   r_i = grad_theta ln I_i, r_i[2c] = 2 Re(conj(A_c) u_i) / I_i, r_i[2c+1] = 2 Im(conj(A_c) u_i) / I_i
 *   mode 0 (Fumili, the outer-product form):  H = sum_i r_i r_i^T
 *   mode 1 (exact):  H = sum_i (r_i r_i^T - E(A_i A_i^H) / I_i) + n_factor E(Psi)
 * where E(C) embeds a Hermitian K x K matrix as the 2K x 2K real matrix of the quadratic form
 * theta -> sum_ab V_a conj(V_b) C_ab: E[2a][2b] = E[2a+1][2b+1] = 2 Re C_ab, E[2a][2b+1] =
 * 2 Im C_ab, E[2a+1][2b] = -2 Im C_ab (so that d2 I_i = E(A_i A_i^H) and d2 S = E(Psi)).
 * H is row-major [2K][2K].  cond [2K][2K] (may be NULL): sum_i (|r_ix| |r_iy| (+ |E(A_i A_i^H)| / I_i
 * for mode 1)) s_i / |u_i| (+ n |E(Psi)|), with s_i = sum_a |V_a| |A_a(i)|: the scale the parity
 * tolerance is taken against.  As for the gradient, s_i is the forward-error scale of u_i in
 * single precision: an FP32 evaluation moves u_i by about eps s_i, so each event's terms move
 * by about their size times eps s_i / |u_i|.  Returns 1 if some I_i is not positive and finite
 * (H is then left zero), else 0. */
int orc_hessian(int K, int64_t n, const float* A, int64_t ld, const double* Vd, const double* Psid,
                double n_factor, int mode, double* H, double* cond) {
    const cplx* V = (const cplx*)Vd;
    const cplx* Psi = (const cplx*)Psid;
    const int D = 2 * K;
    nsum* acc = (nsum*)calloc((size_t)D * D, sizeof(nsum));
    double* sc = (double*)calloc((size_t)D * D, sizeof(double));
    cplx* Ai = (cplx*)malloc(sizeof(cplx) * (size_t)K);
    double* r = (double*)malloc(sizeof(double) * (size_t)D);
    int bad = 0;
    for (int64_t i = 0; i < n && !bad; ++i) {
        cplx u = 0.0;
        double su = 0.0;
        for (int a = 0; a < K; ++a) {
            Ai[a] = A[2 * ((int64_t)a * ld + i)] + I * A[2 * ((int64_t)a * ld + i) + 1];
            u += V[a] * Ai[a];
            su += cabs(V[a]) * cabs(Ai[a]);
        }
        const double Ii = creal(u) * creal(u) + cimag(u) * cimag(u);
        if (!(Ii > 0.0) || !isfinite(Ii)) { bad = 1; break; }
        const double amp = su / sqrt(Ii);  /* s_i / |u_i| >= 1 */
        for (int c = 0; c < K; ++c) {
            const cplx z = conj(Ai[c]) * u;
            r[2 * c] = 2.0 * creal(z) / Ii;
            r[2 * c + 1] = 2.0 * cimag(z) / Ii;
        }
        for (int x = 0; x < D; ++x)
            for (int y = 0; y < D; ++y) {
                nsum_add(&acc[x * D + y], r[x] * r[y]);
                sc[x * D + y] += fabs(r[x] * r[y]) * amp;
            }
        if (mode == 1) {
            for (int a = 0; a < K; ++a)
                for (int b = 0; b < K; ++b) {
                    const cplx cab = Ai[a] * conj(Ai[b]) / Ii;
                    const double re = 2.0 * creal(cab), im = 2.0 * cimag(cab);
                    nsum_add(&acc[(2 * a) * D + 2 * b], -re);
                    nsum_add(&acc[(2 * a + 1) * D + 2 * b + 1], -re);
                    nsum_add(&acc[(2 * a) * D + 2 * b + 1], -im);
                    nsum_add(&acc[(2 * a + 1) * D + 2 * b], im);
                    sc[(2 * a) * D + 2 * b] += fabs(re) * amp;
                    sc[(2 * a + 1) * D + 2 * b + 1] += fabs(re) * amp;
                    sc[(2 * a) * D + 2 * b + 1] += fabs(im) * amp;
                    sc[(2 * a + 1) * D + 2 * b] += fabs(im) * amp;
                }
        }
    }
    for (int x = 0; x < D * D; ++x) H[x] = 0.0;
    if (!bad) {
        for (int x = 0; x < D * D; ++x) H[x] = nsum_get(&acc[x]);
        if (mode == 1) {
            for (int a = 0; a < K; ++a)
                for (int b = 0; b < K; ++b) {
                    const double re = 2.0 * n_factor * creal(Psi[a * K + b]);
                    const double im = 2.0 * n_factor * cimag(Psi[a * K + b]);
                    H[(2 * a) * D + 2 * b] += re;
                    H[(2 * a + 1) * D + 2 * b + 1] += re;
                    H[(2 * a) * D + 2 * b + 1] += im;
                    H[(2 * a + 1) * D + 2 * b] -= im;
                    sc[(2 * a) * D + 2 * b] += fabs(re);
                    sc[(2 * a + 1) * D + 2 * b + 1] += fabs(re);
                    sc[(2 * a) * D + 2 * b + 1] += fabs(im);
                    sc[(2 * a + 1) * D + 2 * b] += fabs(im);
                }
        }
    }
    if (cond)
        for (int x = 0; x < D * D; ++x) cond[x] = sc[x];
    free(acc); free(sc); free(Ai); free(r);
    return bad;
}

/* Eq. 3 exactly as printed: ln L = sum_i ln( sum_a sum_a' V_a conj(V_a') A_a conj(A_a') )
 *   - sum_a sum_a' V_a conj(V_a') Psi_aa'.  Returns -ln L * (with n_factor on the second term)
 * accumulated in long double, O(K^2) per event.  Used only on tiny inputs to pin the O(K)
 * form |sum_a V_a A_a|^2 of Eq. 1. */
double orc_nll_double_sum(int K, int64_t n, const float* A, int64_t ld, const double* Vd,
                          const double* Psid, double n_factor) {
    long double lnsum = 0.0L;
    for (int64_t i = 0; i < n; ++i) {
        long double re = 0.0L;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                long double var = Vd[2 * a], vai = Vd[2 * a + 1];
                long double vbr = Vd[2 * b], vbi = -Vd[2 * b + 1];
                long double aar = A[2 * ((int64_t)a * ld + i)], aai = A[2 * ((int64_t)a * ld + i) + 1];
                long double abr = A[2 * ((int64_t)b * ld + i)], abi = -A[2 * ((int64_t)b * ld + i) + 1];
                /* (va * conj vb) * (Aa * conj Ab), real part (the imaginary parts cancel in the sum) */
                long double pr = var * vbr - vai * vbi, pi = var * vbi + vai * vbr;
                long double qr = aar * abr - aai * abi, qi = aar * abi + aai * abr;
                re += pr * qr - pi * qi;
            }
        lnsum += logl(re);
    }
    long double norm = 0.0L;
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            long double var = Vd[2 * a], vai = Vd[2 * a + 1];
            long double vbr = Vd[2 * b], vbi = -Vd[2 * b + 1];
            long double pr = var * vbr - vai * vbi, pi = var * vbi + vai * vbr;
            long double sr = Psid[2 * (a * K + b)], si = Psid[2 * (a * K + b) + 1];
            norm += pr * sr - pi * si;
        }
    return (double)(-lnsum + (long double)n_factor * norm);
}

/* ---------- floating resonance parameters (streamed MC normalisation) -------------------- */

/* When masses and widths float, Psi cannot be precomputed (Sec. 2, the remark after Eq. 3) and
 * the normalisation is the MC sum itself:
 *   f(V, theta) = -sum_i ln|u_i|^2 + (n_factor / n_gen) sum_j w_j |u_j|^2,  u = sum_a V_a A_a.
 * Gradients: g_c = 2 df/dconj(V_c) (re, im) and, for each floating parameter q of wave r_q with
 * derivative rows dA_q = dA_{r_q}/dtheta_q,
 *   df/dtheta_q = -2 sum_i Re(conj(u_i) V_r dA_iq)/I_i + 2 (n_factor/n_gen) sum_j w_j Re(conj(u_j) V_r dA_jq).
 * A, A_mc: complex64 [K][ld]; dA, dA_mc: complex64 [F][ld]; w_mc may be NULL.
 * Outputs: *nll, grad_V [2K], grad_shape [F]; returns 1 if some data event has I <= 0. */
int orc_nll_grad_shape(int K, int64_t n, const float* A, const float* dA, int64_t ld, int64_t n_mc,
                       const float* A_mc, const float* dA_mc, int64_t ld_mc, const float* w_mc,
                       double n_gen, const int* fwave, int F, const double* Vd, double n_factor,
                       double* nll, double* grad_V, double* grad_shape) {
    const cplx* V = (const cplx*)Vd;
    nsum lsum = {0, 0}, ssum = {0, 0};
    nsum* gd = (nsum*)calloc((size_t)(2 * K + F), sizeof(nsum));  /* data sums */
    nsum* gm = (nsum*)calloc((size_t)(2 * K + F), sizeof(nsum));  /* MC sums */
    cplx* Ai = (cplx*)malloc(sizeof(cplx) * (size_t)K);
    int bad = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t cnt = pass == 0 ? n : n_mc;
        const float* AA = pass == 0 ? A : A_mc;
        const float* DD = pass == 0 ? dA : dA_mc;
        const int64_t L = pass == 0 ? ld : ld_mc;
        nsum* acc = pass == 0 ? gd : gm;
        for (int64_t i = 0; i < cnt; ++i) {
            cplx u = 0.0;
            for (int a = 0; a < K; ++a) {
                Ai[a] = AA[2 * ((int64_t)a * L + i)] + I * AA[2 * ((int64_t)a * L + i) + 1];
                u += V[a] * Ai[a];
            }
            double Ii = creal(u) * creal(u) + cimag(u) * cimag(u);
            cplx wgt;
            if (pass == 0) {
                if (!(Ii > 0.0) || !isfinite(Ii)) { bad = 1; continue; }
                nsum_add(&lsum, log(Ii));
                wgt = u / Ii;
            } else {
                double wj = w_mc ? (double)w_mc[i] : 1.0;
                nsum_add(&ssum, wj * Ii);
                wgt = wj * u;
            }
            for (int c = 0; c < K; ++c) {
                cplx t = conj(Ai[c]) * wgt;
                nsum_add(&acc[2 * c], creal(t));
                nsum_add(&acc[2 * c + 1], cimag(t));
            }
            for (int q = 0; q < F; ++q) {
                cplx d = DD[2 * ((int64_t)q * L + i)] + I * DD[2 * ((int64_t)q * L + i) + 1];
                nsum_add(&acc[2 * K + q], creal(conj(wgt) * V[fwave[q]] * d));
            }
        }
    }
    const double sc = n_factor / n_gen;
    *nll = bad ? INFINITY : (-nsum_get(&lsum) + sc * nsum_get(&ssum));
    for (int v = 0; v < 2 * K; ++v) grad_V[v] = bad ? 0.0 : (-2.0 * nsum_get(&gd[v]) + 2.0 * sc * nsum_get(&gm[v]));
    for (int q = 0; q < F; ++q)
        grad_shape[q] = bad ? 0.0 : (-2.0 * nsum_get(&gd[2 * K + q]) + 2.0 * sc * nsum_get(&gm[2 * K + q]));
    free(gd); free(gm); free(Ai);
    return bad;
}

/* The same objective evaluated in FP64 directly from the kinematics (amplitudes recomputed
 * in double precision for the given masses and widths); used by the finite-difference pins. */
double orc_nll_shape_from_kin(int K, const int* J, const int* lam, const double* M, const double* W,
                              int64_t n, const float* kin, int64_t n_mc, const float* kin_mc,
                              double n_gen, const double* Vd, double n_factor) {
    const cplx* V = (const cplx*)Vd;
    nsum lsum = {0, 0}, ssum = {0, 0};
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t cnt = pass == 0 ? n : n_mc;
        const float* kk = pass == 0 ? kin : kin_mc;
        for (int64_t i = 0; i < cnt; ++i) {
            double m = kk[i], ct = kk[cnt + i], ph = kk[2 * cnt + i];
            cplx u = 0.0;
            for (int a = 0; a < K; ++a)
                u += V[a] * orc_bw(m, M[a], W[a]) * orc_legendre(J[a], ct) * cexp(I * (lam[a] * ph));
            double Ii = creal(u) * creal(u) + cimag(u) * cimag(u);
            if (pass == 0) nsum_add(&lsum, log(Ii));
            else nsum_add(&ssum, Ii);
        }
    }
    return -nsum_get(&lsum) + n_factor / n_gen * nsum_get(&ssum);
}
