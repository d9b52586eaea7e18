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
// Per 4096-event sub-tile, phase A walks the waves group by group (groups of equal (J, lambda)
// share P_J(cos theta) exp(i lambda phi)) to form u, then I, ln I and w = u / I (data) or
// w = w_j u (MC), kept in shared memory with cos(phi), sin(phi).  Phase B runs over chunks of 16
// waves: per event y = conj(Y_g) w for the current group and, per wave, g_a += conj(BW_a) y with
// BW_a recomputed, plus the mass and width derivative terms of floating waves.  Each thread
// accumulates in FP32 over its 16 events of the sub-tile; the block combines in double-single.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "pwa_internal.cuh"

namespace pwa {

namespace {

constexpr int UN_KPT = 16;                      // waves per phase-B chunk (32 accumulators)
constexpr int UN_NCH_MAX = PWA_MAX_WAVES / UN_KPT;
constexpr int UN_SUB = 4096;                    // events per sub-tile (cached in shared memory)
constexpr int UN_EPT = UN_SUB / PWA_THREADS;    // events per thread per sub-tile
constexpr int UN_NW = PWA_THREADS / 32;
constexpr int64_t UN_ITEM_WORK = 1 << 19;       // target wave-events per item
constexpr int64_t UN_ITEM_MAX_EV = 65536;

__constant__ float c_un_inv_int[9] = {1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7, 1.f / 8, 1.f / 9};

// Legendre state of one event: P_{jc}(x) and P_{jc-1}(x), advanced by Bonnet's recurrence
// (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1} (the same arithmetic as the amplitude kernel).
struct Leg {
    float pcur, pprev;
    int jc;
};

__device__ __forceinline__ void leg_reset(Leg& L) {
    L.pcur = 1.f;
    L.pprev = 0.f;
    L.jc = 0;
}

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

struct UnevenItemSmem {
    float4 prm[PWA_MAX_WAVES];  // per sorted wave: M_hi, M_lo, M G, (M G)^2
    float2 V[PWA_MAX_WAVES];    // production amplitude of sorted wave s
    float W[PWA_MAX_WAVES];     // width (floating waves' derivative terms)
    int ord[PWA_MAX_WAVES];     // original index of sorted wave s
    int gend[PWA_MAX_WAVES];
    int gJ[PWA_MAX_WAVES], glam[PWA_MAX_WAVES];
    signed char qM[PWA_MAX_WAVES], qW[PWA_MAX_WAVES];
    int cgrp[UN_NCH_MAX];
    ff acc[1 + 2 * PWA_MAX_WAVES + PWA_MAX_FLOAT];  // item sums (original wave order)
    float red[UN_NW][32];
    ff lred[UN_NW];
    float sred[UN_NW][PWA_MAX_FLOAT];
    int item, last, bad;
};

__device__ __forceinline__ void item_setup(UnevenItemSmem& sm, const UnevenChannel& C, const float2* __restrict__ V,
                                           const double* __restrict__ theta) {
    const int t = threadIdx.x;
    const int K = C.K;
    if (t < K) {
        const int a = C.ord[t];
        double M = C.Md[t], G = C.Wd[t];
        if (C.qM[t] >= 0) M = theta[C.toff + C.qM[t]];
        if (C.qW[t] >= 0) G = theta[C.toff + C.qW[t]];
        const float Mh = (float)M;
        const float Ml = (float)(M - (double)Mh);
        const float MW = (float)(M * G);
        sm.prm[t] = make_float4(Mh, Ml, MW, MW * MW);
        sm.W[t] = (float)G;
        sm.V[t] = V[C.voff + a];
        sm.ord[t] = a;
        sm.qM[t] = C.qM[t];
        sm.qW[t] = C.qW[t];
    }
    if (t < C.ng) {
        sm.gend[t] = C.gend[t];
        sm.gJ[t] = C.gJ[t];
        sm.glam[t] = C.glam[t];
    }
    if (t < UN_NCH_MAX) sm.cgrp[t] = C.cgrp[t];
    for (int v = t; v < 1 + 2 * K + C.F; v += PWA_THREADS) sm.acc[v] = ff_zero();
    if (t == 0) sm.bad = 0;
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

// Block sum of one value per lane l < 32 (value l of every thread) into sm.acc[dst(l)].
template <class Dst>
__device__ __forceinline__ void block_add_32(UnevenItemSmem& sm, float (&x)[32], Dst dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_transpose_reduce32(x);
    sm.red[warp][lane] = x[0];
    __syncthreads();
    if (threadIdx.x < 32) {
        const int d = dst(lane);
        if (d >= 0) {
            ff s = sm.acc[d];
            for (int w = 0; w < UN_NW; ++w) s = ff_add_f(s, sm.red[w][lane]);
            sm.acc[d] = s;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PWA_THREADS, 3) k_uneven(const UnevenChannel* __restrict__ chans, int n_ch,
                                                           const int2* __restrict__ items, int n_items,
                                                           const float2* __restrict__ V,
                                                           const double* __restrict__ theta, double* __restrict__ nll,
                                                           double* __restrict__ grad, float2* __restrict__ part,
                                                           unsigned* __restrict__ ctrl, int* __restrict__ status) {
    extern __shared__ float4 s_ev[];  // [UN_SUB]: (Re w, Im w, cos phi, sin phi) of the sub-tile
    __shared__ UnevenItemSmem sm;
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
        item_setup(sm, C, V, theta);
        const bool is_mc = wi.y >= C.items_d;
        const int li = is_mc ? wi.y - C.items_d : wi.y;
        const float* kin = is_mc ? C.kin_mc : C.kin;
        const int64_t ns = is_mc ? C.n_mc : C.n;
        const int64_t ld = is_mc ? C.ld_mc : C.ld;
        const float* wm = is_mc ? C.w_mc : nullptr;
        const int64_t begin = (int64_t)li * C.epi;
        const int64_t end = min(begin + (int64_t)C.epi, ns);
        const int K = C.K, F = C.F, ng = C.ng, nchunk = C.nchunk;
        __syncthreads();

        ff lacc = ff_zero();
        bool bad = false;
        float gsh[PWA_MAX_FLOAT];
#pragma unroll
        for (int q = 0; q < PWA_MAX_FLOAT; ++q) gsh[q] = 0.f;

        for (int64_t s0 = begin; s0 < end; s0 += UN_SUB) {
            // ---- phase A: u, I, ln I (or w_j I), w per event; cache w and (cos, sin) phi
            for (int k = 0; k < UN_EPT; ++k) {
                const int e = k * PWA_THREADS + tid;
                const int64_t i = s0 + e;
                const bool valid = i < end;
                const float m = valid ? __ldg(kin + i) : 2.f;
                const float ct = valid ? __ldg(kin + ld + i) : 0.f;
                const float ph = valid ? __ldg(kin + 2 * ld + i) : 0.f;
                float s1, c1;
                sincosf(ph, &s1, &c1);
                Leg L;
                leg_reset(L);
                float ur = 0.f, ui = 0.f;
                int s = 0;
                for (int g = 0; g < ng; ++g) {
                    const float2 Y = group_angle(L, sm.gJ[g], sm.glam[g], ct, c1, s1);
                    float zr = 0.f, zi = 0.f;
                    const int ge = sm.gend[g];
                    for (; s < ge; ++s) {
                        float dr;
                        const float2 bw = bw_of(sm.prm[s], m, &dr);
                        const float2 v = sm.V[s];
                        cmac(zr, zi, v.x, v.y, bw.x, bw.y);
                    }
                    cmac(ur, ui, Y.x, Y.y, zr, zi);
                }
                const float I0 = fmaf(ur, ur, ui * ui);
                float wr = 0.f, wi = 0.f;
                if (valid) {
                    if (!is_mc) {
                        if (intensity_ok(I0)) {
                            lacc = ff_add_f(lacc, __logf(I0));
                            const float r = __frcp_rn(I0);
                            wr = ur * r;
                            wi = ui * r;
                        } else {
                            bad = true;
                        }
                    } else {
                        const float wt = wm ? __ldg(wm + i) : 1.f;
                        lacc = ff_add_f(lacc, wt * I0);
                        wr = wt * ur;
                        wi = wt * ui;
                    }
                }
                s_ev[e] = make_float4(wr, wi, c1, s1);
            }
            __syncthreads();
            // ---- phase B: gradient sums over chunks of UN_KPT waves
            for (int c = 0; c < nchunk; ++c) {
                float acc[32];
#pragma unroll
                for (int v = 0; v < 32; ++v) acc[v] = 0.f;
                const int sb = c * UN_KPT;
                for (int k = 0; k < UN_EPT; ++k) {
                    const int e = k * PWA_THREADS + tid;
                    const int64_t i = s0 + e;
                    const bool valid = i < end;
                    const float m = valid ? __ldg(kin + i) : 2.f;
                    const float ct = valid ? __ldg(kin + ld + i) : 0.f;
                    const float4 ev = s_ev[e];
                    Leg L;
                    leg_reset(L);
                    int g = sm.cgrp[c];
                    float2 Y = group_angle(L, sm.gJ[g], sm.glam[g], ct, ev.z, ev.w);
                    // y = conj(Y) w
                    float yr = Y.x * ev.x + Y.y * ev.y, yi = Y.x * ev.y - Y.y * ev.x;
                    int gnext = sm.gend[g];
#pragma unroll
                    for (int j = 0; j < UN_KPT; ++j) {
                        const int s = sb + j;
                        if (s < K) {
                            if (s == gnext) {
                                ++g;
                                Y = group_angle(L, sm.gJ[g], sm.glam[g], ct, ev.z, ev.w);
                                yr = Y.x * ev.x + Y.y * ev.y;
                                yi = Y.x * ev.y - Y.y * ev.x;
                                gnext = sm.gend[g];
                            }
                            const float4 p = sm.prm[s];
                            float dr;
                            const float2 bw = bw_of(p, m, &dr);
                            cmac_conj(acc[2 * j], acc[2 * j + 1], bw.x, bw.y, yr, yi);
                            const int qm = sm.qM[s], qw = sm.qW[s];
                            if (qm >= 0 || qw >= 0) {
                                // dA/dM = -G (M^2 + m^2) Y / D^2, dA/dG = M (M^2 - m^2) Y / D^2; with
                                // 1/D = BW / (M G): R = Re(V (1/D)^2 conj(y))
                                const float rinv = __fdividef(1.f, p.z);
                                const float idr = bw.x * rinv, idi = bw.y * rinv;
                                const float i2r = idr * idr - idi * idi, i2i = 2.f * idr * idi;
                                const float2 v = sm.V[s];
                                const float qr = v.x * i2r - v.y * i2i, qi = v.x * i2i + v.y * i2r;
                                const float R = qr * yr + qi * yi;
                                const float cm = -sm.W[s] * (p.x * p.x + m * m);
                                const float cw = (p.x + p.y) * dr;
#pragma unroll
                                for (int q = 0; q < PWA_MAX_FLOAT; ++q) {
                                    if (q == qm) gsh[q] = fmaf(cm, R, gsh[q]);
                                    if (q == qw) gsh[q] = fmaf(cw, R, gsh[q]);
                                }
                            }
                        }
                    }
                }
                const int Kc = K - sb;
                block_add_32(sm, acc, [&](int l) { return (l >> 1) < Kc ? 1 + 2 * sm.ord[sb + (l >> 1)] + (l & 1) : -1; });
            }
        }
        // ---- item sums of the scalar and the shape terms
#pragma unroll
        for (int mm = 16; mm > 0; mm >>= 1) lacc = ff_add(lacc, ff_shfl_xor(lacc, mm));
#pragma unroll
        for (int q = 0; q < PWA_MAX_FLOAT; ++q) gsh[q] = warp_sum(gsh[q]);
        if (lane == 0) {
            sm.lred[warp] = lacc;
#pragma unroll
            for (int q = 0; q < PWA_MAX_FLOAT; ++q) sm.sred[warp][q] = gsh[q];
        }
        const int any_bad = __syncthreads_or(bad ? 1 : 0);
        const int NV = 1 + 2 * K + F;
        float2* slot = part + C.poff + (int64_t)wi.y * NV;
        for (int v = tid; v < NV; v += PWA_THREADS) {
            ff t;
            if (v == 0) {
                t = ff_zero();
                for (int w = 0; w < UN_NW; ++w) t = ff_add(t, sm.lred[w]);
            } else if (v <= 2 * K) {
                t = sm.acc[v];
            } else {
                t = ff_zero();
                for (int w = 0; w < UN_NW; ++w) t = ff_add_f(t, sm.sred[w][v - 1 - 2 * K]);
            }
            slot[v] = make_float2(t.hi, t.lo);
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
            // sm.red / sm.acc are free now: combine chunk sums in registers via shared ff
            for (int set = 0; set < 2; ++set) {
                const int first = set == 0 ? 0 : nd;
                const int count = set == 0 ? nd : nm;
                for (int vv = tid; vv < nch * NV; vv += PWA_THREADS) {
                    const int v = vv % NV, chn = vv / NV;
                    const int cnt = count > chn ? (count - chn + nch - 1) / nch : 0;
                    const ff t = ff_sum_strided(cp, (int64_t)(first + chn) * NV + v, (int64_t)nch * NV, cnt);
                    s_ev[set * nch * NV + vv] = make_float4(t.hi, t.lo, 0.f, 0.f);
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
                        const float4 x = s_ev[set * nch * NV + chn * NV + v];
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

size_t uneven_smem_bytes() { return sizeof(float4) * (size_t)UN_SUB; }

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
        u.nchunk = (d.K + UN_KPT - 1) / UN_KPT;
        for (int cc = 0; cc < UN_NCH_MAX; ++cc) {
            int g = 0;
            const int s0 = cc * UN_KPT;
            while (g < u.ng && u.gend[g] <= s0) ++g;
            u.cgrp[cc] = g < u.ng ? g : u.ng - 1;
        }
        int64_t epi = (UN_ITEM_WORK / d.K + UN_SUB - 1) / UN_SUB * UN_SUB;
        epi = std::min<int64_t>(std::max<int64_t>(epi, UN_SUB), UN_ITEM_MAX_EV);
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
    const size_t smem = uneven_smem_bytes();
    if (g_uneven_occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(k_uneven, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_uneven, PWA_THREADS, smem);
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
