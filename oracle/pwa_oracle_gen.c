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
