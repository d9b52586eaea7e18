// Many independent likelihoods of uneven wave and event counts, with floating resonance masses
// and widths, in ONE persistent launch (Sec. 2: repeated fits, and fits whose shape parameters
// float, so that neither the MC bracket of Eq. 3 nor the per-event products can be
// precomputed; Sec. 4: fits with many free parameters).  For channel c
//
//   f_c(V, theta) = -sum_i ln|u_i|^2 + (n_f / N_gen) sum_j w_j |u_j|^2,    u = sum_a V_a A_a,
//   g_a           = 2 df/dconj(V_a) = -2 sum_i conj(A_ia) u_i/I_i + 2 (n_f/N_gen) sum_j w_j conj(A_ja) u_j,
//   df/dtheta_q   = -2 sum_i Re(conj(u_i) V_r dA_iq)/I_i + 2 (n_f/N_gen) sum_j w_j Re(conj(u_j) V_r dA_jq),
//
// as pwa_nll_grad_shape computes one channel.  Here every amplitude is recomputed from the
// kinematics (12 bytes per event) inside the kernel, the floating waves' masses and widths read
// from the device trial point theta: no amplitude array is stored or streamed.
//
// Work list.  The host cuts each channel's data and MC samples into items of about 2^19
// wave-events (a whole number of 4096-event sub-tiles), ordered channel by channel, largest
// channels first.  Every block of the persistent grid takes the next item from an atomic
// counter until none is left.  An item's sums are written to a slot of its own, so the result
// does not depend on which block took which item; the block that completes a channel's last
// item sums that channel's item slots in a fixed order (data, then MC) and writes f and the
// gradient.  The last block to leave resets the item counter, so consecutive launches (and
// graph replays) need no memset.
//
// An item is processed in tiles of 256 events.  Phase A, one thread per event: the waves are
// walked group by group (groups of equal (J, lambda) share P_J(cos theta) exp(i lambda phi)) to
// form u, then I, ln I (data) or w_j I (MC), and w = u / I or w_j u; the per-group products
// y_g = conj(Y_g) w go to shared memory.  Phase B, one thread per (wave a, subset r of the tile's
// events): g_a += conj(BW_a(m_e)) y_{g(a),e} over the subset, with the wave's parameters held in
// registers, plus the mass and width derivative terms on the threads of floating waves.  Each
// thread's FP32 tile sums enter double-single accumulators; the item's sums combine the subsets
// of each wave in a fixed order.  Small loops and no per-wave register arrays keep the code
// compact (its instruction fetch, not the arithmetic, limited earlier designs).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int UN_EPT = 2;                       // phase A: events per thread
constexpr int UN_TILE = UN_EPT * PWA_THREADS;   // events per tile
constexpr int UN_NG = 12;                       // groups of equal (J, lambda) per channel, at most
constexpr int UN_NFW = PWA_MAX_FLOAT;           // floating waves per channel, at most
constexpr int UN_NW = PWA_THREADS / 32;
constexpr int64_t UN_ITEM_WORK = 1 << 19;       // target wave-events per item
constexpr int64_t UN_ITEM_MIN_EV = 4096;
constexpr int64_t UN_ITEM_MAX_EV = 65536;

__constant__ float c_un_inv_int[9] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};

// Legendre state of one event: P_{jc}(x) and P_{jc-1}(x), advanced by Bonnet's recurrence
// (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1} (the same arithmetic as the amplitude kernel).
struct Leg {
    float pcur, pprev;
    int jc;
};

// Angular factor P_J(cos theta) exp(i lambda phi) of a group; J must not decrease between calls.
__device__ __forceinline__ float2 group_angle(Leg& L, int J, int lam, float ct, float c1, float s1) {
    for (; L.jc < J; ++L.jc) {
        const float c2 = 2.f * L.jc + 1.f, cj = (float)L.jc, rj = c_un_inv_int[L.jc];
        const float pn = (c2 * ct * L.pcur - cj * L.pprev) * rj;
        L.pprev = L.pcur;
        L.pcur = pn;
    }
    const int al = lam < 0 ? -lam : lam;
    float er = 1.f, ei = 0.f;
    for (int j = 0; j < al; ++j) {
        const float tr = er * c1 - ei * s1;
        ei = er * s1 + ei * c1;
        er = tr;
    }
    if (lam < 0) ei = -ei;
    return make_float2(L.pcur * er, L.pcur * ei);
}

// Breit-Wigner BW = M G / (M^2 - m^2 - i M G) of one wave at m, and M^2 - m^2, from its
// parameters (M_hi, M_lo, M G, (M G)^2); the reciprocal of |D|^2 by __fdividef (2 ulp).
__device__ __forceinline__ float2 bw_of(float4 p, float m, float* dr_out) {
    const float dr = ((p.x - m) + p.y) * ((p.x + m) + p.y);
    const float inv = __fdividef(1.f, fmaf(dr, dr, p.w));
    const float t1 = p.z * inv;
    *dr_out = dr;
    return make_float2(dr * t1, p.z * t1);
}

struct UnevenSmem {
    float4 prm[PWA_MAX_WAVES];  // per sorted wave: M_hi, M_lo, M G, (M G)^2
    float2 V[PWA_MAX_WAVES];    // production amplitude of sorted wave s
    int gend[UN_NG], gJ[UN_NG], glam[UN_NG];
    // floating waves: sorted index, group, width, 1 / (M G), and their mass / width parameter
    int fs[UN_NFW], fg[UN_NFW], fqM[UN_NFW], fqW[UN_NFW];
    float fW[UN_NFW], frMW[UN_NFW];
    float2 y[UN_NG][UN_TILE + 1];  // per group and event of the tile: conj(Y_g) w (Y_g during phase A)
    float m[UN_TILE];
    ff gre[PWA_THREADS], gim[PWA_THREADS];  // item sums per (wave, subset) thread
    float2 sh[UN_NW][2 * UN_NFW];           // per warp: the floating waves' mass and width sums
    ff lred[UN_NW];
    int nfw, item, last, bad;
};

__global__ void __launch_bounds__(PWA_THREADS, 3) k_uneven(const UnevenChannel* __restrict__ chans, int n_ch,
                                                           const int2* __restrict__ items, int n_items,
                                                           const float2* __restrict__ V,
                                                           const double* __restrict__ theta, double* __restrict__ nll,
                                                           double* __restrict__ grad, float2* __restrict__ part,
                                                           unsigned* __restrict__ ctrl, int* __restrict__ status) {
    __shared__ UnevenSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned* tickets = ctrl + 1;
    unsigned* bad_ch = ctrl + 1 + n_ch;
    unsigned* exit_count = ctrl + 1 + 2 * n_ch;

    for (;;) {
        if (tid == 0) sm.item = (int)atomicAdd(ctrl, 1u);
        __syncthreads();
        const int it = sm.item;
        if (it >= n_items) break;
        const int2 wi = items[it];
        const UnevenChannel& C = chans[wi.x];
        const int K = C.K, F = C.F, ng = C.ng;
        // ---- per item: the channel's wave table at the trial point
        if (tid < K) {
            double M = C.Md[tid], G = C.Wd[tid];
            if (C.qM[tid] >= 0) M = theta[C.toff + C.qM[tid]];
            if (C.qW[tid] >= 0) G = theta[C.toff + C.qW[tid]];
            const float Mh = (float)M;
            const float MW = (float)(M * G);
            sm.prm[tid] = make_float4(Mh, (float)(M - (double)Mh), MW, MW * MW);
            sm.V[tid] = V[C.voff + C.ord[tid]];
        }
        if (tid < ng) {
            sm.gend[tid] = C.gend[tid];
            sm.gJ[tid] = C.gJ[tid];
            sm.glam[tid] = C.glam[tid];
        }
        if (tid == 0) {
            // the floating waves in sorted order, with their parameters' indices
            int nf = 0, g = 0;
            for (int s = 0; s < K; ++s) {
                while (C.gend[g] <= s) ++g;
                if (C.qM[s] >= 0 || C.qW[s] >= 0) {
                    sm.fs[nf] = s;
                    sm.fg[nf] = g;
                    sm.fqM[nf] = C.qM[s];
                    sm.fqW[nf] = C.qW[s];
                    const double Mf = C.qM[s] >= 0 ? theta[C.toff + C.qM[s]] : C.Md[s];
                    const double Gf = C.qW[s] >= 0 ? theta[C.toff + C.qW[s]] : C.Wd[s];
                    sm.fW[nf] = (float)Gf;
                    sm.frMW[nf] = 1.f / (float)(Mf * Gf);
                    ++nf;
                }
            }
            sm.nfw = nf;
            sm.bad = 0;
        }
        const bool is_mc = wi.y >= C.items_d;
        const int li = is_mc ? wi.y - C.items_d : wi.y;
        const float* kin = is_mc ? C.kin_mc : C.kin;
        const int64_t ns = is_mc ? C.n_mc : C.n;
        const int64_t ld = is_mc ? C.ld_mc : C.ld;
        const float* wm = is_mc ? C.w_mc : nullptr;
        const int64_t begin = (int64_t)li * C.epi;
        const int64_t end = min(begin + (int64_t)C.epi, ns);
        // phase-B role of this thread: wave a (sorted), event subset r of R
        const int R = PWA_THREADS / K;
        const int a = tid % K, r = tid / K;
        const bool active = r < R;
        __syncthreads();
        float4 pa = make_float4(0.f, 0.f, 1.f, 1.f);
        int ga = 0;
        if (active) {
            pa = sm.prm[a];
            while (sm.gend[ga] <= a) ++ga;
        }
        const int nfw = sm.nfw;
        ff gre = ff_zero(), gim = ff_zero(), lacc = ff_zero();
        float shM[UN_NFW], shW[UN_NFW];  // floating waves' d/dM and d/dG sums of the item (phase A)
#pragma unroll
        for (int j = 0; j < UN_NFW; ++j) shM[j] = shW[j] = 0.f;
        bool bad = false;

        for (int64_t t0 = begin; t0 < end; t0 += UN_TILE) {
            const int ntile = (int)min((int64_t)UN_TILE, end - t0);
            // ---- phase A: UN_EPT events per thread; u, I, w; conj(Y_g) w per group into shared
            // memory; the floating waves' mass and width derivative terms
            {
                float m[UN_EPT], ct[UN_EPT], c1[UN_EPT], s1[UN_EPT], ur[UN_EPT], ui[UN_EPT];
                Leg L[UN_EPT];
#pragma unroll
                for (int k = 0; k < UN_EPT; ++k) {
                    const int e = k * PWA_THREADS + tid;
                    const int64_t i = t0 + e;
                    const bool valid = e < ntile;
                    m[k] = valid ? __ldg(kin + i) : 2.f;
                    ct[k] = valid ? __ldg(kin + ld + i) : 0.f;
                    const float ph = valid ? __ldg(kin + 2 * ld + i) : 0.f;
                    sincosf(ph, &s1[k], &c1[k]);
                    L[k] = Leg{1.f, 0.f, 0};
                    ur[k] = ui[k] = 0.f;
                }
                int s = 0;
                for (int g = 0; g < ng; ++g) {
                    float2 Y[UN_EPT];
                    float zr[UN_EPT], zi[UN_EPT];
#pragma unroll
                    for (int k = 0; k < UN_EPT; ++k) {
                        Y[k] = group_angle(L[k], sm.gJ[g], sm.glam[g], ct[k], c1[k], s1[k]);
                        sm.y[g][k * PWA_THREADS + tid] = Y[k];
                        zr[k] = zi[k] = 0.f;
                    }
                    const int ge = sm.gend[g];
                    for (; s < ge; ++s) {
                        const float4 p = sm.prm[s];
                        const float2 v = sm.V[s];
#pragma unroll
                        for (int k = 0; k < UN_EPT; ++k) {
                            float dr;
                            const float2 bw = bw_of(p, m[k], &dr);
                            cmac(zr[k], zi[k], v.x, v.y, bw.x, bw.y);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < UN_EPT; ++k) cmac(ur[k], ui[k], Y[k].x, Y[k].y, zr[k], zi[k]);
                }
#pragma unroll
                for (int k = 0; k < UN_EPT; ++k) {
                    const int e = k * PWA_THREADS + tid;
                    const float I0 = fmaf(ur[k], ur[k], ui[k] * ui[k]);
                    float wr = 0.f, wi = 0.f;
                    if (e < ntile) {
                        if (!is_mc) {
                            if (intensity_ok(I0)) {
                                lacc = ff_add_f(lacc, __logf(I0));
                                const float rI = __frcp_rn(I0);
                                wr = ur[k] * rI;
                                wi = ui[k] * rI;
                            } else {
                                bad = true;
                            }
                        } else {
                            const float wt = wm ? __ldg(wm + t0 + e) : 1.f;
                            lacc = ff_add_f(lacc, wt * I0);
                            wr = wt * ur[k];
                            wi = wt * ui[k];
                        }
                    }
                    for (int g = 0; g < ng; ++g) {
                        const float2 Y = sm.y[g][e];
                        sm.y[g][e] = make_float2(Y.x * wr + Y.y * wi, Y.x * wi - Y.y * wr);  // conj(Y) w
                    }
                    sm.m[e] = m[k];
                    // floating wave j (sorted index fs, group fg): d/dM and d/dG of Re(conj(w) V A):
                    // dA/dM = -G (M^2 + m^2) Y / D^2, dA/dG = M (M^2 - m^2) Y / D^2, 1/D = BW / (M G),
                    // so each is its coefficient times Re(V (1/D)^2 conj(y)), y = conj(Y) w
#pragma unroll
                    for (int j = 0; j < UN_NFW; ++j) {
                        if (j < nfw) {
                            const int sj = sm.fs[j];
                            const float4 p = sm.prm[sj];
                            const float2 v = sm.V[sj];
                            const float2 y = sm.y[sm.fg[j]][e];
                            float dr;
                            const float2 bw = bw_of(p, m[k], &dr);
                            const float rMW = sm.frMW[j];
                            const float idr = bw.x * rMW, idi = bw.y * rMW;
                            const float i2r = idr * idr - idi * idi, i2i = 2.f * idr * idi;
                            const float qr = v.x * i2r - v.y * i2i, qi = v.x * i2i + v.y * i2r;
                            const float Rr = qr * y.x + qi * y.y;
                            shM[j] = fmaf(-sm.fW[j] * (p.x * p.x + m[k] * m[k]), Rr, shM[j]);
                            shW[j] = fmaf((p.x + p.y) * dr, Rr, shW[j]);
                        }
                    }
                }
            }
            __syncthreads();
            // ---- phase B: thread = (wave a, subset r); g_a += conj(BW_a(m_e)) y_e over the tile
            if (active) {
                float ar = 0.f, ai = 0.f;
                const float2* yg = sm.y[ga];
#pragma unroll 4
                for (int e = r; e < ntile; e += R) {
                    float dr;
                    const float2 bw = bw_of(pa, sm.m[e], &dr);
                    const float2 y = yg[e];
                    cmac_conj(ar, ai, bw.x, bw.y, y.x, y.y);
                }
                gre = ff_add_f(gre, ar);
                gim = ff_add_f(gim, ai);
            }
            __syncthreads();
        }
        // ---- item sums: per wave over the subsets r in order; ln I (or w I) and the floating
        // waves' sums over the warps in order
        sm.gre[tid] = gre;
        sm.gim[tid] = gim;
#pragma unroll
        for (int mm = 16; mm > 0; mm >>= 1) lacc = ff_add(lacc, ff_shfl_xor(lacc, mm));
#pragma unroll
        for (int j = 0; j < UN_NFW; ++j) {
            shM[j] = warp_sum(shM[j]);
            shW[j] = warp_sum(shW[j]);
        }
        if (lane == 0) {
            sm.lred[warp] = lacc;
#pragma unroll
            for (int j = 0; j < UN_NFW; ++j) sm.sh[warp][2 * j] = make_float2(shM[j], shW[j]);
        }
        const int any_bad = __syncthreads_or(bad ? 1 : 0);
        const int NV = 1 + 2 * K + F;
        float2* slot = part + C.poff + (int64_t)wi.y * NV;
        if (tid < K) {
            ff tr = ff_zero(), ti = ff_zero();
            for (int rr = 0; rr < R; ++rr) {
                const int t = rr * K + tid;
                tr = ff_add(tr, sm.gre[t]);
                ti = ff_add(ti, sm.gim[t]);
            }
            const int o = C.ord[tid];
            slot[1 + 2 * o] = make_float2(tr.hi, tr.lo);
            slot[2 + 2 * o] = make_float2(ti.hi, ti.lo);
        } else if (tid >= PWA_THREADS - 2 * UN_NFW) {
            const int jj = tid - (PWA_THREADS - 2 * UN_NFW), j = jj >> 1, kind = jj & 1;
            if (j < nfw) {
                ff t = ff_zero();
                for (int w = 0; w < UN_NW; ++w) t = ff_add_f(t, kind ? sm.sh[w][2 * j].y : sm.sh[w][2 * j].x);
                const int q = kind ? sm.fqW[j] : sm.fqM[j];
                if (q >= 0) slot[1 + 2 * K + q] = make_float2(t.hi, t.lo);
            }
        } else if (tid == PWA_THREADS - 2 * UN_NFW - 1) {
            ff t = ff_zero();
            for (int w = 0; w < UN_NW; ++w) t = ff_add(t, sm.lred[w]);
            slot[0] = make_float2(t.hi, t.lo);
        }
        if (any_bad && tid == 0) atomicOr(bad_ch + wi.x, 1u);
        __threadfence();
        __syncthreads();
        if (tid == 0) sm.last = atomicAdd(tickets + wi.x, 1u) == (unsigned)(C.items_d + C.items_m - 1);
        __syncthreads();
        if (sm.last) {
            // ---- the channel's last item: fixed-order sums of its slots, data then MC
            __threadfence();
            const float2* cp = part + C.poff;
            const int nd = C.items_d, nm = C.items_m;
            const int nch = PWA_THREADS / NV > 0 ? PWA_THREADS / NV : 1;
            float2* sfin = reinterpret_cast<float2*>(&sm.y[0][0]);  // the tile buffers are free now
            for (int set = 0; set < 2; ++set) {
                const int first = set == 0 ? 0 : nd;
                const int count = set == 0 ? nd : nm;
                for (int vv = tid; vv < nch * NV; vv += PWA_THREADS) {
                    const int v = vv % NV, chn = vv / NV;
                    const int cnt = count > chn ? (count - chn + nch - 1) / nch : 0;
                    const ff t = ff_sum_strided(cp, (int64_t)(first + chn) * NV + v, (int64_t)nch * NV, cnt);
                    sfin[set * nch * NV + vv] = make_float2(t.hi, t.lo);
                }
            }
            __syncthreads();
            if (tid == 0) sm.bad = (int)__ldcg(bad_ch + wi.x);
            __syncthreads();
            const bool isbad = sm.bad != 0;
            for (int v = tid; v < NV; v += PWA_THREADS) {
                double val[2];
                for (int set = 0; set < 2; ++set) {
                    ff t = ff_zero();
                    for (int chn = 0; chn < nch; ++chn) {
                        const float2 x = sfin[set * nch * NV + chn * NV + v];
                        t = ff_add(t, ff{x.x, x.y});
                    }
                    val[set] = ff_to_double(t);
                }
                if (v == 0) {
                    nll[wi.x] = isbad ? INFINITY : (-val[0] + C.scale * val[1]);
                } else {
                    grad[C.goff + v - 1] = isbad ? 0.0 : (-2.0 * val[0] + 2.0 * C.scale * val[1]);
                }
            }
            if (tid == 0) {
                if (isbad) atomicOr(status, 1);
                bad_ch[wi.x] = 0u;
                tickets[wi.x] = 0u;
            }
        }
        __syncthreads();
    }
    // the last block to leave resets the item counter for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(exit_count, 1u) == gridDim.x - 1) {
            ctrl[0] = 0u;
            *exit_count = 0u;
            __threadfence();
        }
    }
}

int g_uneven_occ = -1;

}  // namespace

int uneven_build_plan(const pwa_uneven_channel* ch, int n_ch, UnevenPlan* plan, char* err, size_t err_len) {
    plan->chans.assign(n_ch, UnevenChannel{});
    plan->n_ch = n_ch;
    int voff = 0, toff = 0, goff = 0;
    int64_t poff = 0;
    struct Tmp {
        int c;
        int64_t work;
    };
    std::vector<Tmp> order(n_ch);
    for (int c = 0; c < n_ch; ++c) {
        const pwa_uneven_channel& d = ch[c];
        UnevenChannel& u = plan->chans[c];
        u.kin = d.kin;
        u.kin_mc = d.kin_mc;
        u.w_mc = d.w_mc;
        u.n = d.n;
        u.ld = d.ld;
        u.n_mc = d.n_mc;
        u.ld_mc = d.ld_mc;
        u.scale = d.n_factor / d.n_gen;
        u.K = d.K;
        u.F = d.F;
        // waves sorted by (J, lambda), stable: the groups share their angular factor
        std::vector<int> idx(d.K);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return d.waves[a].J != d.waves[b].J ? d.waves[a].J < d.waves[b].J : d.waves[a].lambda < d.waves[b].lambda;
        });
        u.ng = 0;
        for (int s = 0; s < d.K; ++s) {
            const pwa_wave& w = d.waves[idx[s]];
            u.ord[s] = idx[s];
            u.Md[s] = w.mass;
            u.Wd[s] = w.width;
            u.qM[s] = -1;
            u.qW[s] = -1;
            if (s == 0 || w.J != d.waves[idx[s - 1]].J || w.lambda != d.waves[idx[s - 1]].lambda) {
                u.gJ[u.ng] = w.J;
                u.glam[u.ng] = w.lambda;
                ++u.ng;
            }
            u.gend[u.ng - 1] = s + 1;
        }
        for (int q = 0; q < d.F; ++q) {
            int s = 0;
            while (u.ord[s] != d.float_wave[q]) ++s;
            (d.float_kind[q] == 0 ? u.qM[s] : u.qW[s]) = (signed char)q;
        }
        if (u.ng > UN_NG) {
            snprintf(err, err_len, "channel %d: %d groups of equal (J, lambda), at most %d", c, u.ng, UN_NG);
            return -1;
        }
        int64_t epi = (UN_ITEM_WORK / d.K + 1023) / 1024 * 1024;
        epi = std::min<int64_t>(std::max<int64_t>(epi, UN_ITEM_MIN_EV), UN_ITEM_MAX_EV);
        u.epi = (int)epi;
        u.items_d = (int)std::max<int64_t>(1, (d.n + epi - 1) / epi);
        u.items_m = (int)((d.n_mc + epi - 1) / epi);
        u.voff = voff;
        u.toff = toff;
        u.goff = goff;
        u.poff = poff;
        voff += d.K;
        toff += d.F;
        goff += 2 * d.K + d.F;
        poff += (int64_t)(u.items_d + u.items_m) * (1 + 2 * d.K + d.F);
        order[c] = {c, (d.n + d.n_mc) * (int64_t)d.K};
    }
    // channels with the most work first: their final sums overlap the remaining items
    std::stable_sort(order.begin(), order.end(), [](const Tmp& a, const Tmp& b) { return a.work > b.work; });
    plan->items.clear();
    for (const Tmp& o : order) {
        const UnevenChannel& u = plan->chans[o.c];
        for (int li = 0; li < u.items_d + u.items_m; ++li) plan->items.push_back(make_int2(o.c, li));
    }
    if (plan->items.size() > (size_t)INT32_MAX) {
        snprintf(err, err_len, "too many work items");
        return -1;
    }
    plan->part_f2 = poff;
    plan->n_v = voff;
    plan->n_theta = toff;
    plan->n_grad = goff;
    return 0;
}

size_t uneven_workspace(const UnevenPlan& p) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    return r(sizeof(unsigned) * (2 * (size_t)p.n_ch + 2)) + r(sizeof(UnevenChannel) * p.chans.size()) +
           r(sizeof(int2) * p.items.size()) + r(sizeof(float2) * (size_t)p.part_f2);
}

namespace {
struct UnevenLayout {
    unsigned* ctrl;
    UnevenChannel* chans;
    int2* items;
    float2* part;
};
UnevenLayout uneven_layout(const UnevenPlan& p, void* ws) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* c = reinterpret_cast<char*>(ws);
    UnevenLayout L;
    L.ctrl = reinterpret_cast<unsigned*>(c);
    c += r(sizeof(unsigned) * (2 * (size_t)p.n_ch + 2));
    L.chans = reinterpret_cast<UnevenChannel*>(c);
    c += r(sizeof(UnevenChannel) * p.chans.size());
    L.items = reinterpret_cast<int2*>(c);
    c += r(sizeof(int2) * p.items.size());
    L.part = reinterpret_cast<float2*>(c);
    return L;
}
}  // namespace

cudaError_t uneven_upload(const UnevenPlan& p, void* ws, cudaStream_t st) {
    UnevenLayout L = uneven_layout(p, ws);
    cudaError_t e = cudaMemsetAsync(L.ctrl, 0, sizeof(unsigned) * (2 * (size_t)p.n_ch + 2), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.chans, p.chans.data(), sizeof(UnevenChannel) * p.chans.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.items, p.items.data(), sizeof(int2) * p.items.size(), cudaMemcpyHostToDevice, st);
    return e;
}

cudaError_t uneven_launch(const UnevenPlan& p, void* ws, const float2* V, const double* theta, double* nll,
                          double* grad, int* status, int sm_count, cudaStream_t st) {
    UnevenLayout L = uneven_layout(p, ws);
    const size_t smem = 0;
    if (g_uneven_occ < 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_uneven, PWA_THREADS, smem);
        if (e != cudaSuccess) return e;
        g_uneven_occ = o > 0 ? o : 1;
    }
    int64_t grid = (int64_t)sm_count * g_uneven_occ;
    if (grid > (int64_t)p.items.size()) grid = (int64_t)p.items.size();
    if (grid < 1) grid = 1;
    k_uneven<<<(unsigned)grid, PWA_THREADS, smem, st>>>(L.chans, p.n_ch, L.items, (int)p.items.size(), V, theta, nll,
                                                        grad, L.part, L.ctrl, status);
    return cudaGetLastError();
}

}  // namespace pwa
