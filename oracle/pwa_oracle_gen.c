/*
 * pwa_oracle_gen.c -- oracle toy generator (accept-reject from the intensity of Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY (see pwa_oracle.c).  Shares nothing with the CUDA library.
 *
 *   - Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written from its definition:
 *     ten rounds of two 32x32->64 multiplications (constants 0xD2511F53, 0xCD9E8D57) whose
 *     high halves are xored with the other two words and the round key; the key is bumped
 *     by the Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.
 *   - candidate j of a (seed, stream) sequence uses counter (j_lo, j_hi, stream, 0) and key
 *     (seed_lo, seed_hi); its four words give m, cos(theta), phi on the flat phase space and
 *     the accept-reject uniform, each as (word >> 8) * 2^-24 in single precision.
 *   - candidate accepted iff u * C < I(Omega) = |sum_a V_a A_a(Omega)|^2 (Eq. 1), C a bound
 *     on I over the phase space; accepted events are returned in candidate order.
 *   - envelope: on each of n_int equal m-intervals, |BW_a| is maximal at m = M_a if M_a lies
 *     inside, else at the interval end nearer M_a (|BW|^2 rises below M and falls above), and
 *     |P_J| <= 1, |exp(i lambda phi)| = 1; so (sum_a |V_a| max|BW_a|)^2 bounds I on the
 *     interval, and C is the largest interval bound.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>

typedef double complex cplx;

cplx orc_bw(double m, double M, double W);
double orc_legendre(int J, double x);

static uint32_t mulhilo(uint32_t a, uint32_t b, uint32_t* hi) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

void orc_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, hi1;
        uint32_t lo0 = mulhilo(0xD2511F53u, c0, &hi0);
        uint32_t lo1 = mulhilo(0xCD9E8D57u, c2, &hi1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

/* the flat phase-space point and accept uniform of candidate j */
void orc_candidate(uint64_t seed, uint32_t stream, int64_t j, float* m, float* ct, float* ph, float* u) {
    uint32_t ctr[4] = {(uint32_t)(uint64_t)j, (uint32_t)((uint64_t)j >> 32), stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32(ctr, key, r);
    float f0 = u01(r[0]), f1 = u01(r[1]), f2 = u01(r[2]);
    float t = 2.01f * f0;
    *m = 0.99f + t;
    float s = 2.0f * f1;
    *ct = s - 1.0f;
    *ph = 6.2831855f * f2;
    *u = u01(r[3]);
}

static double intensity(int K, const int* J, const int* lam, const double* M, const double* W,
                        const double* Vd, double m, double ct, double ph) {
    const cplx* V = (const cplx*)Vd;
    cplx u = 0.0;
    for (int a = 0; a < K; ++a)
        u += V[a] * orc_bw(m, M[a], W[a]) * orc_legendre(J[a], ct) * cexp(I * (lam[a] * ph));
    return creal(u) * creal(u) + cimag(u) * cimag(u);
}

double orc_envelope(int K, const double* M, const double* W, const double* Vd, double m_lo,
                    double m_hi, int n_int) {
    const cplx* V = (const cplx*)Vd;
    double best = 0.0;
    for (int k = 0; k < n_int; ++k) {
        double a0 = m_lo + (m_hi - m_lo) * k / n_int;
        double a1 = m_lo + (m_hi - m_lo) * (k + 1) / n_int;
        double s = 0.0;
        for (int a = 0; a < K; ++a) {
            double mm = M[a] < a0 ? a0 : (M[a] > a1 ? a1 : M[a]);
            s += cabs(V[a]) * cabs(orc_bw(mm, M[a], W[a]));
        }
        if (s * s > best) best = s * s;
    }
    return best;
}

/* Accept-reject over candidates [cand0, cand0 + n_cand).  Writes up to max_out accepted
 * events as float SoA [3][ld_out] in candidate order; returns the number accepted (which
 * may exceed max_out).  *max_ratio receives max I/C over the candidates (<= 1 for a valid
 * envelope). */
int64_t orc_generate(int K, const int* J, const int* lam, const double* M, const double* W,
                     const double* V, uint64_t seed, uint32_t stream, int64_t cand0,
                     int64_t n_cand, double C, float* kin, int64_t ld_out, int64_t max_out,
                     double* max_ratio) {
    int64_t na = 0;
    double mr = 0.0;
    for (int64_t j = cand0; j < cand0 + n_cand; ++j) {
        float m, ct, ph, u;
        orc_candidate(seed, stream, j, &m, &ct, &ph, &u);
        double Ii = intensity(K, J, lam, M, W, V, m, ct, ph);
        if (Ii / C > mr) mr = Ii / C;
        if ((double)u * C < Ii) {
            if (na < max_out) {
                kin[na] = m;
                kin[ld_out + na] = ct;
                kin[2 * ld_out + na] = ph;
            }
            ++na;
        }
    }
    if (max_ratio) *max_ratio = mr;
    return na;
}

/* Per-candidate view of the same accept-reject step, for judging a single-precision generator
 * decision by decision: for candidates [cand0, cand0 + n_cand) the phase-space point (float SoA
 * [3][n_cand]), the accept uniform u, the FP64 intensity I(Omega) of Eq. 1 and the magnitude
 * sum s = sum_a |V_a| |A_a(Omega)| (>= |u|, the scale of the rounding error of the sum u). */
void orc_candidates(int K, const int* J, const int* lam, const double* M, const double* W,
                    const double* Vd, uint64_t seed, uint32_t stream, int64_t cand0, int64_t n_cand,
                    float* kin, float* u_out, double* I_out, double* s_out) {
    const cplx* V = (const cplx*)Vd;
    for (int64_t k = 0; k < n_cand; ++k) {
        float m, ct, ph, u;
        orc_candidate(seed, stream, cand0 + k, &m, &ct, &ph, &u);
        kin[k] = m;
        kin[n_cand + k] = ct;
        kin[2 * n_cand + k] = ph;
        u_out[k] = u;
        I_out[k] = intensity(K, J, lam, M, W, Vd, m, ct, ph);
        double s = 0.0;
        for (int a = 0; a < K; ++a)
            s += cabs(V[a]) * cabs(orc_bw(m, M[a], W[a])) * fabs(orc_legendre(J[a], ct));
        s_out[k] = s;
    }
}

/* ---------- angular moments (features of the learned start proposer) ------------------ */

/* Real spherical harmonics Y_LM(theta, phi), L <= 4, index k = L^2 + L + M, orthonormal on the
 * sphere: Y_L0 = N_L0 P_L(x); M > 0: sqrt(2) N_LM P_L^M(x) cos(M phi);
 * M < 0: sqrt(2) N_L|M| P_L^|M|(x) sin(|M| phi);  N_LM = sqrt((2L+1)/(4 pi) (L-M)!/(L+M)!),
 * P_L^M the associated Legendre function with the Condon-Shortley phase (-1)^M. */
static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

static double assoc_legendre(int L, int M, double x) {
    /* P_M^M = (-1)^M (2M-1)!! (1-x^2)^{M/2}; P_{M+1}^M = x (2M+1) P_M^M;
     * (L-M) P_L^M = x (2L-1) P_{L-1}^M - (L+M-1) P_{L-2}^M */
    double pmm = 1.0;
    double s = sqrt((1.0 - x) * (1.0 + x));
    for (int i = 1; i <= M; ++i) pmm *= -(2.0 * i - 1.0) * s;
    if (L == M) return pmm;
    double pm1 = x * (2.0 * M + 1.0) * pmm;
    if (L == M + 1) return pm1;
    double pl = 0.0;
    for (int l = M + 2; l <= L; ++l) {
        pl = (x * (2.0 * l - 1.0) * pm1 - (l + M - 1.0) * pmm) / (l - M);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

double orc_ylm_real(int L, int M, double ct, double phi) {
    int am = M < 0 ? -M : M;
    const double pi = 3.14159265358979323846;
    double N = sqrt((2.0 * L + 1.0) / (4.0 * pi) * factorial(L - am) / factorial(L + am));
    double p = assoc_legendre(L, am, ct);
    if (M == 0) return N * p;
    if (M > 0) return sqrt(2.0) * N * p * cos(am * phi);
    return sqrt(2.0) * N * p * sin(am * phi);
}

/* feat[b][k] = (1/n) sum_{events in mass bin b} Y_k(theta, phi), bins of equal width on
 * [m_lo, m_hi), 25 moments (L <= 4) per bin.  kin is float SoA [3][ld]. */
void orc_moments(int64_t n, const float* kin, int64_t ld, int n_bins, double m_lo, double m_hi,
                 double* feat) {
    for (int i = 0; i < n_bins * 25; ++i) feat[i] = 0.0;
    /* the bin index is an integer decided by floating point: it is taken in single precision,
     * (m - m_lo) * (n_bins / (m_hi - m_lo)) with both factors rounded to float, as the kernel
     * does, so both sides put every event in the same bin */
    const float lo_f = (float)m_lo;
    const float inv_w = (float)((double)n_bins / (m_hi - m_lo));
    for (int64_t i = 0; i < n; ++i) {
        double m = kin[i], ct = kin[ld + i], ph = kin[2 * ld + i];
        float dm = kin[i] - lo_f;
        float xb = dm * inv_w;
        int b = (int)floorf(xb);
        if (b < 0) b = 0;
        if (b >= n_bins) b = n_bins - 1;
        for (int L = 0; L <= 4; ++L)
            for (int M = -L; M <= L; ++M) feat[b * 25 + L * L + L + M] += orc_ylm_real(L, M, ct, ph);
    }
    if (n > 0)
        for (int i = 0; i < n_bins * 25; ++i) feat[i] /= (double)n;
}
