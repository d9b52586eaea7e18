// C ABI of libpwa.so: handle lifetime, argument validation, workspace management and
// dispatch to the kernels.  Every entry point validates its arguments on the host before
// launching anything; there is no CPU fallback path.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "barrier.cuh"
#include "pwa_internal.cuh"

namespace {

std::mutex g_err_mu;
std::string g_create_err;

pwa_status fail(pwa_handle* h, pwa_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_err = buf;
    }
    return st;
}

pwa_status cuda_fail(pwa_handle* h, cudaError_t e, const char* what) {
    return fail(h, PWA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

pwa_status ensure_workspace(pwa_handle* h, size_t bytes, int P) {
    if (bytes > h->ws_bytes) {
        if (h->ws) {
            cudaDeviceSynchronize();
            cudaFree(h->ws);
            h->ws = nullptr;
            h->ws_bytes = 0;
        }
        size_t want = bytes + bytes / 4;
        cudaError_t e = cudaMalloc(&h->ws, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, PWA_ERR_WORKSPACE, "workspace allocation of %zu bytes failed: %s", want,
                        cudaGetErrorString(e));
        }
        h->ws_bytes = want;
    }
    if (P > h->bad_cap) {
        if (h->bad) {
            cudaDeviceSynchronize();
            cudaFree(h->bad);
            h->bad = nullptr;
            h->bad_cap = 0;
        }
        int cap = P < 1024 ? 1024 : P;
        cudaError_t e = cudaMalloc(&h->bad, sizeof(int) * (size_t)cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, PWA_ERR_WORKSPACE, "flag allocation failed: %s", cudaGetErrorString(e));
        }
        e = cudaMemset(h->bad, 0, sizeof(int) * (size_t)cap);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset");
        h->bad_cap = cap;
    }
    return PWA_OK;
}

pwa_status check_amp_layout(pwa_handle* h, int K, int64_t n, int64_t ld) {
    if (K < 1 || K > PWA_MAX_WAVES)
        return fail(h, PWA_ERR_INVALID_ARG, "K = %d outside [1, %d]", K, PWA_MAX_WAVES);
    if (n < 0) return fail(h, PWA_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (ld < n) return fail(h, PWA_ERR_INVALID_ARG, "ld = %lld < n = %lld", (long long)ld, (long long)n);
    if (ld & 1) return fail(h, PWA_ERR_INVALID_ARG, "ld = %lld must be even", (long long)ld);
    if ((int64_t)K * ld > ((int64_t)1 << 40))
        return fail(h, PWA_ERR_INVALID_ARG, "K * ld = %lld too large", (long long)((int64_t)K * ld));
    return PWA_OK;
}

pwa_status fill_waves(pwa_handle* h, const pwa_wave* waves, int K, pwa::WaveTable* wt) {
    wt->K = K;
    for (int a = 0; a < K; ++a) {
        const pwa_wave& w = waves[a];
        if (w.J < 0 || w.J > 8 || w.lambda < -8 || w.lambda > 8)
            return fail(h, PWA_ERR_INVALID_ARG, "wave %d: J = %d or lambda = %d out of range", a, w.J, w.lambda);
        if (!(w.mass > 0.0) || !(w.width > 0.0) || !std::isfinite(w.mass) || !std::isfinite(w.width))
            return fail(h, PWA_ERR_INVALID_ARG, "wave %d: mass and width must be finite and > 0", a);
        wt->J[a] = w.J;
        wt->lam[a] = w.lambda;
        wt->Mhi[a] = (float)w.mass;
        wt->Mlo[a] = (float)(w.mass - (double)wt->Mhi[a]);
        wt->W[a] = (float)w.width;
        wt->MW[a] = (float)(w.mass * w.width);
    }
    // group the waves by (J, lambda): groups in ascending (J, lambda), waves of a group in the
    // given order (the amplitude kernel advances its Legendre recurrence from group to group)
    int n = 0;
    wt->ng = 0;
    for (int J = 0; J <= 8; ++J)
        for (int lam = -8; lam <= 8; ++lam) {
            const int n0 = n;
            for (int a = 0; a < K; ++a)
                if (wt->J[a] == J && wt->lam[a] == lam) wt->gord[n++] = a;
            if (n > n0) wt->gend[wt->ng++] = n;
        }
    return PWA_OK;
}

pwa_status nll_common(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V, int P,
                      const double* Psi, double n_factor, double* nll, double* grad, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    if (P < 1 || P > (1 << 24)) return fail(h, PWA_ERR_INVALID_ARG, "P = %d outside [1, 2^24]", P);
    if ((n > 0 && !A) || !V || !Psi || !nll)
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array argument (A, V, Psi and nll are required)");
    if (n > 0 && !aligned16(A)) return fail(h, PWA_ERR_INVALID_ARG, "A is not 16-byte aligned");
    if (!aligned16(Psi)) return fail(h, PWA_ERR_INVALID_ARG, "Psi is not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) != 0) return fail(h, PWA_ERR_INVALID_ARG, "V is not 8-byte aligned");
    if (!std::isfinite(n_factor)) return fail(h, PWA_ERR_INVALID_ARG, "n_factor is not finite");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::nll_workspace(K, n, P, h->sm_count), P);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_nll(reinterpret_cast<const float2*>(A), K, n, ld, reinterpret_cast<const float2*>(V),
                                    P, reinterpret_cast<const double2*>(Psi), n_factor, nll, grad, h->ws, h->ws_bytes,
                                    h->counters, h->bad, h->status, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "nll launch");
    h->err.clear();
    return PWA_OK;
}


// The fitter runs on a handle-owned non-blocking (capturable) stream ordered after the
// caller's stream; the fit calls return after that stream has drained.
pwa_status fit_stream_begin(pwa_handle* h, void* stream, cudaStream_t* out) {
    if (!h->fit_stream) {
        cudaError_t ce = cudaStreamCreateWithFlags(&h->fit_stream, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->fit_event, cudaEventDisableTiming);
        if (ce != cudaSuccess) return cuda_fail(h, ce, "fit stream");
    }
    cudaError_t ce = cudaEventRecord(h->fit_event, (cudaStream_t)stream);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(h->fit_stream, h->fit_event, 0);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "fit stream ordering");
    *out = h->fit_stream;
    return PWA_OK;
}

// One eager iteration (tile-shape selection happens outside any capture), then check_every
// iterations per captured graph replay until no start is running.  Bounded: every iteration
// evaluates once and a start stops after max_iter accepted steps.
template <class Iter>
cudaError_t run_fit_loop(pwa_handle* h, cudaStream_t s, const pwa_fit_opts& o, int P_tot, int m, Iter iteration) {
    cudaError_t e = iteration();
    if (e != cudaSuccess) return e;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    bool graph_ok = false;
    if (o.use_graph) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs == cudaStreamCaptureStatusNone &&
            cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t ce = cudaSuccess;
            for (int it = 0; it < o.check_every && ce == cudaSuccess; ++it) ce = iteration();
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            if (ce == cudaSuccess && ee == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
                graph_ok = true;
            cudaGetLastError();
        }
    }
    int* running_h = nullptr;
    if (cudaMallocHost(&running_h, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        running_h = nullptr;
    }
    int running_local = 1;
    int* running = running_h ? running_h : &running_local;
    const long long max_loops = 60LL * (long long)o.max_iter + 100;
    long long loops = 1;
    while (e == cudaSuccess) {
        e = pwa::fit_launch_count(h->fitws, P_tot, m, running, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || *running == 0 || loops >= max_loops) break;
        if (graph_ok) {
            e = cudaGraphLaunch(exec, s);
        } else {
            for (int it = 0; it < o.check_every && e == cudaSuccess; ++it) e = iteration();
        }
        loops += o.check_every;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (running_h) cudaFreeHost(running_h);
    return e;
}

pwa_status grow_fitws(pwa_handle* h, size_t need) {
    if (need > h->fitws_bytes) {
        if (h->fitws) {
            cudaDeviceSynchronize();
            cudaFree(h->fitws);
            h->fitws = nullptr;
            h->fitws_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&h->fitws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, PWA_ERR_WORKSPACE, "fit workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        }
        h->fitws_bytes = need;
    }
    return PWA_OK;
}

// Arguments of one channel of the multi-channel (uneven) evaluation.
pwa_status check_uneven_channel(pwa_handle* h, const pwa_uneven_channel& d, int c) {
    pwa_status st = check_amp_layout(h, d.K, d.n, d.ld);
    if (st == PWA_OK) st = check_amp_layout(h, d.K, d.n_mc, d.ld_mc);
    if (st != PWA_OK) return fail(h, st, "channel %d: %s", c, h->err.c_str());
    if (!d.waves) return fail(h, PWA_ERR_INVALID_ARG, "channel %d: waves NULL", c);
    pwa::WaveTable wt;
    st = fill_waves(h, d.waves, d.K, &wt);
    if (st != PWA_OK) return fail(h, st, "channel %d: %s", c, h->err.c_str());
    if (d.F < 0 || d.F > PWA_MAX_FLOAT || (d.F > 0 && (!d.float_wave || !d.float_kind)))
        return fail(h, PWA_ERR_INVALID_ARG, "channel %d: F out of range or NULL float_wave/float_kind", c);
    for (int q = 0; q < d.F; ++q) {
        if (d.float_wave[q] < 0 || d.float_wave[q] >= d.K || (d.float_kind[q] != 0 && d.float_kind[q] != 1))
            return fail(h, PWA_ERR_INVALID_ARG, "channel %d: bad floating parameter %d", c, q);
        for (int r = 0; r < q; ++r)
            if (d.float_wave[r] == d.float_wave[q] && d.float_kind[r] == d.float_kind[q])
                return fail(h, PWA_ERR_INVALID_ARG, "channel %d: floating parameter %d repeated", c, q);
    }
    if ((d.n > 0 && !d.kin) || (d.n_mc > 0 && !d.kin_mc))
        return fail(h, PWA_ERR_INVALID_ARG, "channel %d: NULL kinematics", c);
    if ((d.kin && !aligned16(d.kin)) || (d.kin_mc && !aligned16(d.kin_mc)) ||
        (d.w_mc && (reinterpret_cast<uintptr_t>(d.w_mc) & 3u)))
        return fail(h, PWA_ERR_INVALID_ARG, "channel %d: misaligned array", c);
    if (!(d.n_gen > 0.0) || !std::isfinite(d.n_gen) || !std::isfinite(d.n_factor))
        return fail(h, PWA_ERR_INVALID_ARG, "channel %d: bad n_gen or n_factor", c);
    return PWA_OK;
}

// Plan of a multi-channel evaluation, and its descriptors and work list on the device (uploaded
// only when they differ from the last upload; not capturable then).
pwa_status uneven_prepare(pwa_handle* h, const pwa_uneven_channel* ch, int n_ch, pwa::UnevenPlan* plan,
                          cudaStream_t s) {
    char msg[256] = {0};
    if (pwa::uneven_build_plan(ch, n_ch, plan, msg, sizeof msg) != 0) return fail(h, PWA_ERR_INVALID_ARG, "%s", msg);
    const size_t need = pwa::uneven_workspace(*plan);
    std::vector<unsigned char> key(sizeof(pwa::UnevenChannel) * plan->chans.size() + sizeof(int2) * plan->items.size());
    memcpy(key.data(), plan->chans.data(), sizeof(pwa::UnevenChannel) * plan->chans.size());
    memcpy(key.data() + sizeof(pwa::UnevenChannel) * plan->chans.size(), plan->items.data(),
           sizeof(int2) * plan->items.size());
    if (need > h->uws_bytes) {
        if (h->uws) {
            cudaDeviceSynchronize();
            cudaFree(h->uws);
            h->uws = nullptr;
            h->uws_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&h->uws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, PWA_ERR_WORKSPACE, "multi-channel workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        }
        h->uws_bytes = need;
        h->uws_key.clear();
    }
    if (key != h->uws_key) {
        cudaError_t e = pwa::uneven_upload(*plan, h->uws, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "multi-channel work list upload");
        h->uws_key.swap(key);
    }
    return PWA_OK;
}

}  // namespace

namespace pwa {
void record_global_error(const char* msg) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
}
}  // namespace pwa

extern "C" {

int pwa_abi_version(void) { return PWA_ABI_VERSION; }

const char* pwa_status_string(int s) {
    switch (s) {
        case PWA_OK: return "PWA_OK";
        case PWA_ERR_INVALID_ARG: return "PWA_ERR_INVALID_ARG";
        case PWA_ERR_NO_DEVICE: return "PWA_ERR_NO_DEVICE";
        case PWA_ERR_CUDA: return "PWA_ERR_CUDA";
        case PWA_ERR_NONFINITE: return "PWA_ERR_NONFINITE";
        case PWA_ERR_TIMEOUT: return "PWA_ERR_TIMEOUT";
        case PWA_ERR_WORKSPACE: return "PWA_ERR_WORKSPACE";
        case PWA_NOT_CONVERGED: return "PWA_NOT_CONVERGED";
        default: return "PWA_UNKNOWN_STATUS";
    }
}

pwa_status pwa_create(pwa_handle** out, int device) {
    if (!out) return PWA_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(nullptr, PWA_ERR_NO_DEVICE, "no CUDA device: %s",
                    e != cudaSuccess ? cudaGetErrorString(e) : "device count is 0");
    }
    if (device < 0 || device >= count)
        return fail(nullptr, PWA_ERR_INVALID_ARG, "device %d outside [0, %d)", device, count);
    DeviceGuard dg(device);
    if (!dg.ok) return fail(nullptr, PWA_ERR_CUDA, "cannot select device %d", device);
    pwa_handle* h = new pwa_handle();
    h->device = device;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (h->sm_count <= 0) h->sm_count = 1;
    e = cudaMalloc(&h->counters, pwa::HANDLE_COUNTER_BYTES);
    if (e == cudaSuccess) e = cudaMemset(h->counters, 0, pwa::HANDLE_COUNTER_BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        pwa_status st = fail(nullptr, PWA_ERR_CUDA, "handle allocation: %s", cudaGetErrorString(e));
        pwa_destroy(h);
        return st;
    }
    *out = h;
    return PWA_OK;
}

void pwa_destroy(pwa_handle* h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    if (h->counters) cudaFree(h->counters);
    if (h->status) cudaFree(h->status);
    if (h->bad) cudaFree(h->bad);
    if (h->fitws) cudaFree(h->fitws);
    if (h->fit_event) cudaEventDestroy(h->fit_event);
    if (h->fit_stream) cudaStreamDestroy(h->fit_stream);
    if (h->uws) cudaFree(h->uws);
    delete h;
}

const char* pwa_last_error(const pwa_handle* h) {
    if (h) return h->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_err.c_str();
}

int pwa_batched_shape(int K, int64_t n, int P) {
    if (K < 1 || K > PWA_MAX_WAVES || n < 0 || P < 2) return -1;
    return pwa::batched_shape(K, n, P);
}

size_t pwa_workspace_size(const pwa_handle* h, int K, int64_t n, int P) {
    if (!h || K < 1 || K > PWA_MAX_WAVES || n < 0 || P < 1) return 0;
    size_t a = pwa::nll_workspace(K, n, P, h->sm_count);
    size_t b = pwa::normint_workspace(K, h->sm_count);
    return a > b ? a : b;
}

pwa_status pwa_reserve(pwa_handle* h, int K, int64_t n, int P) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (K < 1 || K > PWA_MAX_WAVES || n < 0 || P < 1)
        return fail(h, PWA_ERR_INVALID_ARG, "bad sizes K=%d n=%lld P=%d", K, (long long)n, P);
    DeviceGuard dg(h->device);
    return ensure_workspace(h, pwa_workspace_size(h, K, n, P), P);
}

pwa_status pwa_sync_status(pwa_handle* h, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    int s = 0;
    e = cudaMemcpy(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (s) {
        e = cudaMemset(h->status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(h, e, "status clear");
        if (s & 2) return fail(h, PWA_ERR_TIMEOUT, "a bounded device-side wait gave up (results of that call are flagged)");
        return fail(h, PWA_ERR_NONFINITE, "an evaluation met an event with intensity <= 0 or not finite");
    }
    return PWA_OK;
}

pwa_status pwa_amplitudes(pwa_handle* h, const pwa_wave* waves, int K, const float* kin, int64_t n,
                          int64_t ld, float* A, float* dA_dM, float* dA_dW, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    if (!waves) return fail(h, PWA_ERR_INVALID_ARG, "waves is NULL");
    if (ld > 0 && (!A || (n > 0 && !kin)))
        return fail(h, PWA_ERR_INVALID_ARG, "NULL kinematics or amplitude array");
    if ((dA_dM == nullptr) != (dA_dW == nullptr))
        return fail(h, PWA_ERR_INVALID_ARG, "dA_dM and dA_dW must be both given or both NULL");
    if ((A && !aligned16(A)) || (kin && !aligned16(kin)) || (dA_dM && !aligned16(dA_dM)) ||
        (dA_dW && !aligned16(dA_dW)))
        return fail(h, PWA_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    pwa::WaveTable wt;
    st = fill_waves(h, waves, K, &wt);
    if (st != PWA_OK) return st;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = pwa::launch_amplitudes(wt, kin, n, ld, reinterpret_cast<float2*>(A),
                                           reinterpret_cast<float2*>(dA_dM), reinterpret_cast<float2*>(dA_dW),
                                           h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "amplitude launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_amplitudes_barrier(pwa_handle* h, const pwa_wave* waves, int K, double m1, double m2, double R,
                                  const float* kin, int64_t n, int64_t ld, float* A, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    if (!waves) return fail(h, PWA_ERR_INVALID_ARG, "waves is NULL");
    if (ld > 0 && (!A || (n > 0 && !kin))) return fail(h, PWA_ERR_INVALID_ARG, "NULL kinematics or amplitude array");
    if ((A && !aligned16(A)) || (kin && !aligned16(kin)))
        return fail(h, PWA_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    if (!(m1 >= 0.0) || !(m2 >= 0.0) || !std::isfinite(m1) || !std::isfinite(m2))
        return fail(h, PWA_ERR_INVALID_ARG, "daughter masses must be finite and >= 0");
    if (!(R > 0.0) || !(R <= 100.0)) return fail(h, PWA_ERR_INVALID_ARG, "radius R must be in (0, 100] GeV^-1");
    pwa::WaveTable wt;
    st = fill_waves(h, waves, K, &wt);
    if (st != PWA_OK) return st;
    pwa::BarrierTable bt;
    const double msum = m1 + m2, mdif = std::fabs(m1 - m2);
    bt.msum_hi = (float)msum;
    bt.msum_lo = (float)(msum - (double)bt.msum_hi);
    bt.mdif_hi = (float)mdif;
    bt.mdif_lo = (float)(mdif - (double)bt.mdif_hi);
    bt.R = (float)R;
    bt.R2 = (float)(R * R);
    for (int a = 0; a < K; ++a) {
        const pwa_wave& w = waves[a];
        if (w.J > pwa::BARRIER_LMAX)
            return fail(h, PWA_ERR_INVALID_ARG, "wave %d: J = %d above %d for barrier factors", a, w.J, pwa::BARRIER_LMAX);
        if (!(w.mass > msum)) return fail(h, PWA_ERR_INVALID_ARG, "wave %d: mass at or below the decay threshold", a);
        // q0 = q(M) from the factorised Kallen function; B_J^2(q0^2 R^2) > 0 since q0 > 0
        const double M = w.mass;
        const double q0 = std::sqrt((M - msum) * (M + msum) * (M - mdif) * (M + mdif)) / (2.0 * M);
        const double b20 = pwa::barrier2_host(w.J, q0 * q0 * R * R);
        bt.num[a] = (float)(M * w.width / std::sqrt(b20));
        bt.cw[a] = (float)(M * M * w.width / (q0 * b20));
    }
    for (int a = K; a < PWA_MAX_WAVES; ++a) bt.num[a] = bt.cw[a] = 0.f;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    cudaError_t e = pwa::launch_amp_barrier(wt, bt, kin, n, ld, reinterpret_cast<float2*>(A), h->sm_count,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "barrier amplitude launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_normint(pwa_handle* h, const float* A_mc, int K, int64_t n_mc, int64_t ld, const float* w,
                       double n_gen, double* Psi, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n_mc, ld);
    if (st != PWA_OK) return st;
    if ((n_mc > 0 && !A_mc) || !Psi) return fail(h, PWA_ERR_INVALID_ARG, "NULL A_mc or Psi");
    if (n_mc > 0 && !aligned16(A_mc)) return fail(h, PWA_ERR_INVALID_ARG, "A_mc is not 16-byte aligned");
    if (!aligned16(Psi)) return fail(h, PWA_ERR_INVALID_ARG, "Psi is not 16-byte aligned");
    if (w && (reinterpret_cast<uintptr_t>(w) & 3u)) return fail(h, PWA_ERR_INVALID_ARG, "w is not 4-byte aligned");
    if (!(n_gen > 0.0) || !std::isfinite(n_gen))
        return fail(h, PWA_ERR_INVALID_ARG, "n_gen must be finite and > 0");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::normint_workspace(K, h->sm_count), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_normint(reinterpret_cast<const float2*>(A_mc), K, n_mc, ld, w, n_gen,
                                        reinterpret_cast<double2*>(Psi), h->ws, h->sm_count, (cudaStream_t)stream,
                                        h->status);
    if (e != cudaSuccess) return cuda_fail(h, e, "normint launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_normint_from_kinematics(pwa_handle* h, const pwa_wave* waves, int K, const float* kin, int64_t n_mc,
                                       int64_t ld, const float* w, double n_gen, double* Psi, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n_mc, ld);
    if (st != PWA_OK) return st;
    if (!waves) return fail(h, PWA_ERR_INVALID_ARG, "waves is NULL");
    if ((n_mc > 0 && !kin) || !Psi) return fail(h, PWA_ERR_INVALID_ARG, "NULL kin or Psi");
    if (kin && !aligned16(kin)) return fail(h, PWA_ERR_INVALID_ARG, "kin is not 16-byte aligned");
    if (!aligned16(Psi)) return fail(h, PWA_ERR_INVALID_ARG, "Psi is not 16-byte aligned");
    if (w && (reinterpret_cast<uintptr_t>(w) & 3u)) return fail(h, PWA_ERR_INVALID_ARG, "w is not 4-byte aligned");
    if (!(n_gen > 0.0) || !std::isfinite(n_gen))
        return fail(h, PWA_ERR_INVALID_ARG, "n_gen must be finite and > 0");
    pwa::WaveTable wt;
    st = fill_waves(h, waves, K, &wt);
    if (st != PWA_OK) return st;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::normint_workspace(K, h->sm_count), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_normint_kin(wt, kin, K, n_mc, ld, w, n_gen, reinterpret_cast<double2*>(Psi), h->ws,
                                            h->sm_count, (cudaStream_t)stream, h->status);
    if (e != cudaSuccess) return cuda_fail(h, e, "normint (kinematics) launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_nll(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V, int P,
                   const double* Psi, double n_factor, double* nll, void* stream) {
    return nll_common(h, A, K, n, ld, V, P, Psi, n_factor, nll, nullptr, stream);
}

pwa_status pwa_nll_grad(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V, int P,
                        const double* Psi, double n_factor, double* nll, double* grad, void* stream) {
    if (h && !grad) return fail(h, PWA_ERR_INVALID_ARG, "grad is NULL");
    return nll_common(h, A, K, n, ld, V, P, Psi, n_factor, nll, grad, stream);
}

pwa_status pwa_hessian(pwa_handle* h, const float* A, int K, int64_t n, int64_t ld, const float* V, const double* Psi,
                       double n_factor, int exact, double* H, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    if (K > PWA_MAX_WAVES / 2) return fail(h, PWA_ERR_INVALID_ARG, "pwa_hessian: K = %d > %d", K, PWA_MAX_WAVES / 2);
    if ((n > 0 && !A) || !V || !Psi || !H)
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array argument (A, V, Psi and H are required)");
    if (n > 0 && !aligned16(A)) return fail(h, PWA_ERR_INVALID_ARG, "A is not 16-byte aligned");
    if (!aligned16(Psi)) return fail(h, PWA_ERR_INVALID_ARG, "Psi is not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) != 0) return fail(h, PWA_ERR_INVALID_ARG, "V is not 8-byte aligned");
    if (!std::isfinite(n_factor)) return fail(h, PWA_ERR_INVALID_ARG, "n_factor is not finite");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::hessian_workspace(K, ld, h->sm_count), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_hessian(reinterpret_cast<const float2*>(A), K, n, ld, reinterpret_cast<const float2*>(V),
                                        reinterpret_cast<const double2*>(Psi), n_factor, exact ? 1 : 0, H, h->ws,
                                        h->status, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "hessian launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_nll_grad_incoherent(pwa_handle* h, const float* A, int K, int H, int64_t n, int64_t ld,
                                   const float* V, int P, const double* Psi, double n_factor, double* nll,
                                   double* grad, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (H < 1 || H > PWA_MAX_STATES) return fail(h, PWA_ERR_INVALID_ARG, "H = %d outside [1, %d]", H, PWA_MAX_STATES);
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    if (P < 1 || P > (1 << 24)) return fail(h, PWA_ERR_INVALID_ARG, "P = %d outside [1, 2^24]", P);
    if ((n > 0 && !A) || !V || !Psi || !nll)
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array argument (A, V, Psi and nll are required)");
    if (n > 0 && !aligned16(A)) return fail(h, PWA_ERR_INVALID_ARG, "A is not 16-byte aligned");
    if (!aligned16(Psi)) return fail(h, PWA_ERR_INVALID_ARG, "Psi is not 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) != 0) return fail(h, PWA_ERR_INVALID_ARG, "V is not 8-byte aligned");
    if (!std::isfinite(n_factor)) return fail(h, PWA_ERR_INVALID_ARG, "n_factor is not finite");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::nll_workspace(K, n, 1, h->sm_count), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_nll_incoherent(reinterpret_cast<const float2*>(A), K, H, n, ld,
                                               reinterpret_cast<const float2*>(V), P,
                                               reinterpret_cast<const double2*>(Psi), n_factor, nll, grad, h->ws,
                                               h->counters, h->status, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "incoherent nll launch");
    h->err.clear();
    return PWA_OK;
}

double pwa_envelope(const pwa_wave* waves, int K, const float* V, double m_lo, double m_hi, int n_intervals) {
    if (!waves || !V || K < 1 || K > PWA_MAX_WAVES || !(m_hi > m_lo) || n_intervals < 1) return -1.0;
    double best = 0.0;
    for (int k = 0; k < n_intervals; ++k) {
        const double a0 = m_lo + (m_hi - m_lo) * k / n_intervals;
        const double a1 = m_lo + (m_hi - m_lo) * (k + 1) / n_intervals;
        double s = 0.0;
        for (int a = 0; a < K; ++a) {
            const double M = waves[a].mass, W = waves[a].width;
            if (!(M > 0.0) || !(W > 0.0)) return -1.0;
            // |BW|^2 = (M W)^2 / ((M^2 - m^2)^2 + (M W)^2) rises below M and falls above it
            const double mm = M < a0 ? a0 : (M > a1 ? a1 : M);
            const double d = M * M - mm * mm;
            s += std::hypot((double)V[2 * a], (double)V[2 * a + 1]) * (M * W / std::sqrt(d * d + M * M * W * W));
        }
        if (s * s > best) best = s * s;
    }
    return best;
}

pwa_status pwa_generate(pwa_handle* h, const pwa_wave* waves, int K, const float* V, uint64_t seed,
                        uint32_t stream_id, int64_t cand0, int64_t n_cand, double envelope, float* kin,
                        int64_t ld_out, int64_t max_out, int64_t* n_accepted, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (!waves || !V || !n_accepted || (max_out > 0 && !kin))
        return fail(h, PWA_ERR_INVALID_ARG, "NULL argument (waves, V, n_accepted, kin)");
    if (K < 1 || K > PWA_MAX_WAVES) return fail(h, PWA_ERR_INVALID_ARG, "K = %d outside [1, %d]", K, PWA_MAX_WAVES);
    if (cand0 < 0 || n_cand < 0 || max_out < 0 || ld_out < max_out)
        return fail(h, PWA_ERR_INVALID_ARG, "bad sizes: cand0, n_cand, max_out >= 0 and ld_out >= max_out required");
    if (n_cand > ((int64_t)1 << 40)) return fail(h, PWA_ERR_INVALID_ARG, "n_cand too large");
    if (!(envelope > 0.0) || !std::isfinite(envelope) || envelope > 3.0e38)
        return fail(h, PWA_ERR_INVALID_ARG, "envelope must be finite and > 0");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) || (reinterpret_cast<uintptr_t>(n_accepted) & 7u))
        return fail(h, PWA_ERR_INVALID_ARG, "V must be 8-byte aligned, n_accepted 8-byte aligned");
    pwa::WaveTable wt;
    pwa_status st = fill_waves(h, waves, K, &wt);
    if (st != PWA_OK) return st;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::generate_workspace(n_cand), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_generate(wt, reinterpret_cast<const float2*>(V), seed, stream_id, cand0, n_cand,
                                         envelope, kin, ld_out, max_out, reinterpret_cast<long long*>(n_accepted),
                                         h->ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "generate launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_nll_grad_shape(pwa_handle* h, const float* A, const float* dA, int K, int64_t n, int64_t ld,
                              const float* A_mc, const float* dA_mc, int64_t n_mc, int64_t ld_mc, const float* w_mc,
                              double n_gen, const int* float_wave, int F, const float* V, double n_factor,
                              double* nll, double* grad, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    pwa_status st = check_amp_layout(h, K, n, ld);
    if (st != PWA_OK) return st;
    st = check_amp_layout(h, K, n_mc, ld_mc);
    if (st != PWA_OK) return st;
    if (F < 0 || F > PWA_MAX_FLOAT) return fail(h, PWA_ERR_INVALID_ARG, "F = %d outside [0, %d]", F, PWA_MAX_FLOAT);
    if (F > 0 && !float_wave) return fail(h, PWA_ERR_INVALID_ARG, "float_wave is NULL");
    for (int q = 0; q < F; ++q)
        if (float_wave[q] < 0 || float_wave[q] >= K)
            return fail(h, PWA_ERR_INVALID_ARG, "float_wave[%d] = %d outside [0, K)", q, float_wave[q]);
    if ((n > 0 && (!A || (F > 0 && !dA))) || (n_mc > 0 && (!A_mc || (F > 0 && !dA_mc))) || !V || !nll || !grad)
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array argument");
    if ((A && !aligned16(A)) || (dA && !aligned16(dA)) || (A_mc && !aligned16(A_mc)) || (dA_mc && !aligned16(dA_mc)))
        return fail(h, PWA_ERR_INVALID_ARG, "amplitude arrays must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) || (w_mc && (reinterpret_cast<uintptr_t>(w_mc) & 3u)))
        return fail(h, PWA_ERR_INVALID_ARG, "misaligned V or w_mc");
    if (!(n_gen > 0.0) || !std::isfinite(n_gen) || !std::isfinite(n_factor))
        return fail(h, PWA_ERR_INVALID_ARG, "n_gen must be finite and > 0, n_factor finite");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::shape_workspace(K, F, h->sm_count), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_nll_shape(reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(dA), K,
                                          n, ld, reinterpret_cast<const float2*>(A_mc),
                                          reinterpret_cast<const float2*>(dA_mc), n_mc, ld_mc, w_mc, n_gen,
                                          float_wave, F, reinterpret_cast<const float2*>(V), n_factor, nll, grad,
                                          h->ws, h->ws_bytes, h->counters, reinterpret_cast<int*>(h->counters + 1),
                                          h->status, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "shape launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_moments(pwa_handle* h, const float* kin, int64_t n, int64_t ld, int n_bins, double m_lo, double m_hi,
                       double* feat, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (n < 0 || ld < n || (n > 0 && !kin) || !feat) return fail(h, PWA_ERR_INVALID_ARG, "bad sizes or NULL array");
    if (n_bins < 1 || n_bins > 64 || !(m_hi > m_lo))
        return fail(h, PWA_ERR_INVALID_ARG, "n_bins must be 1..64 and m_hi > m_lo");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    pwa_status st = ensure_workspace(h, pwa::moments_workspace(n_bins, 1), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_moments(kin, n, ld, n_bins, m_lo, m_hi, feat, h->ws, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_toy_moments(pwa_handle* h, const pwa_wave* waves, int K, const float* V, int T, const double* Psi_flat,
                           double n_target, uint64_t seed, uint32_t stream_base, int n_bins, double* feat,
                           int64_t* n_acc, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (!waves || !V || !Psi_flat || !feat || !n_acc || T < 1 || T > (1 << 24))
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array or T out of range");
    if (K < 1 || K > PWA_MAX_WAVES) return fail(h, PWA_ERR_INVALID_ARG, "K = %d outside [1, %d]", K, PWA_MAX_WAVES);
    if (n_bins < 1 || n_bins > 64) return fail(h, PWA_ERR_INVALID_ARG, "n_bins must be 1..64");
    if (!(n_target >= 1.0) || !(n_target <= 1e9)) return fail(h, PWA_ERR_INVALID_ARG, "n_target out of range");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) || !aligned16(Psi_flat) || (reinterpret_cast<uintptr_t>(n_acc) & 7u))
        return fail(h, PWA_ERR_INVALID_ARG, "misaligned array");
    pwa::WaveTable wt;
    pwa_status st = fill_waves(h, waves, K, &wt);
    if (st != PWA_OK) return st;
    double Md[PWA_MAX_WAVES], Wd[PWA_MAX_WAVES];
    for (int a = 0; a < K; ++a) {
        Md[a] = waves[a].mass;
        Wd[a] = waves[a].width;
    }
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    st = ensure_workspace(h, pwa::toy_moments_workspace(n_bins, T), 1);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::launch_toy_moments(wt, Md, Wd, reinterpret_cast<const float2*>(V), T,
                                            reinterpret_cast<const double2*>(Psi_flat), n_target, seed, stream_base,
                                            n_bins, feat, reinterpret_cast<long long*>(n_acc), h->ws,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "toy moments launch");
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_mlp_gemm(pwa_handle* h, int M, int N, int Kc, const void* A, int a_type, int64_t sam, int64_t sak,
                        const void* B, int b_type, int64_t sbn, int64_t sbk, const float* bias, int relu,
                        int accumulate, float* C, uint16_t* C_bf16, int64_t ldc, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (M < 1 || N < 1 || Kc < 1 || !A || !B || (!C && !C_bf16) || ldc < N || (accumulate && !C))
        return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_gemm: bad sizes or NULL arrays");
    if ((a_type != 0 && a_type != 1) || (b_type != 0 && b_type != 1))
        return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_gemm: element type must be 0 (float32) or 1 (bfloat16)");
    if (sam < 0 || sak < 0 || sbn < 0 || sbk < 0) return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_gemm: negative stride");
    DeviceGuard dg(h->device);
    // B in BF16 (every product of the proposer's network): tensor cores; B in FP32: SIMT kernel
    cudaError_t e = b_type == 1
                        ? pwa::launch_mlp_gemm_tc(M, N, Kc, A, a_type, sam, sak, B, sbn, sbk, bias, relu, accumulate,
                                                  C, C_bf16, ldc, h->status, (cudaStream_t)stream)
                        : pwa::launch_mlp_gemm(M, N, Kc, A, a_type, sam, sak, B, b_type, sbn, sbk, bias, relu,
                                               accumulate, C, C_bf16, ldc, h->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp gemm");
    return PWA_OK;
}

pwa_status pwa_mlp_relu_backward(pwa_handle* h, const uint16_t* Y_bf16, float* dY, int64_t n, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!Y_bf16 || !dY))) return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_relu_backward: bad args");
    DeviceGuard dg(h->device);
    cudaError_t e = pwa::launch_mlp_relu_bwd(Y_bf16, dY, n, h->sm_count, (cudaStream_t)stream);
    return e == cudaSuccess ? PWA_OK : cuda_fail(h, e, "relu backward");
}

pwa_status pwa_mlp_bias_grad(pwa_handle* h, const float* dY, int B, int N, float* db, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (B < 1 || N < 1 || !dY || !db) return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_bias_grad: bad args");
    DeviceGuard dg(h->device);
    cudaError_t e = pwa::launch_mlp_bias_grad(dY, B, N, db, (cudaStream_t)stream);
    return e == cudaSuccess ? PWA_OK : cuda_fail(h, e, "bias grad");
}

pwa_status pwa_mlp_wta_loss(pwa_handle* h, const float* out, const float* target, int B, int C, int K, float eps,
                            float* loss, float* dout, int* winner, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (B < 1 || C < 1 || C > 32 || K < 1 || K > PWA_MAX_WAVES || !out || !target || !loss || !(eps >= 0.f && eps <= 1.f))
        return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_wta_loss: bad args (1 <= C <= 32, 0 <= eps <= 1)");
    DeviceGuard dg(h->device);
    cudaError_t e = pwa::launch_mlp_wta(out, target, B, C, K, eps, loss, dout, winner, (cudaStream_t)stream);
    return e == cudaSuccess ? PWA_OK : cuda_fail(h, e, "wta loss");
}

pwa_status pwa_mlp_adam(pwa_handle* h, float* p, const float* g, float* m, float* v, uint16_t* p_bf16, int64_t n,
                        float lr, float b1, float b2, float eps, int step, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!p || !g || !m || !v)) || step < 1 || !(lr > 0.f) || !(b1 >= 0.f && b1 < 1.f) ||
        !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_adam: bad args");
    DeviceGuard dg(h->device);
    cudaError_t e = pwa::launch_mlp_adam(p, g, m, v, p_bf16, n, lr, b1, b2, eps, step, h->sm_count, (cudaStream_t)stream);
    return e == cudaSuccess ? PWA_OK : cuda_fail(h, e, "adam");
}

pwa_status pwa_mlp_to_bf16(pwa_handle* h, const double* x, uint16_t* y, int64_t n, float scale, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!x || !y))) return fail(h, PWA_ERR_INVALID_ARG, "pwa_mlp_to_bf16: bad args");
    DeviceGuard dg(h->device);
    cudaError_t e = pwa::launch_mlp_to_bf16(x, y, n, scale, h->sm_count, (cudaStream_t)stream);
    return e == cudaSuccess ? PWA_OK : cuda_fail(h, e, "to bf16");
}

pwa_status pwa_nll_grad_uneven(pwa_handle* h, const pwa_uneven_channel* channels, int n_ch, const float* V,
                               const double* theta, double* nll, double* grad, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (!channels || n_ch < 1 || n_ch > (1 << 20)) return fail(h, PWA_ERR_INVALID_ARG, "channels NULL or n_ch < 1");
    int nF = 0;
    for (int c = 0; c < n_ch; ++c) {
        pwa_status st = check_uneven_channel(h, channels[c], c);
        if (st != PWA_OK) return st;
        nF += channels[c].F;
    }
    if (!V || !nll || !grad || (nF > 0 && !theta))
        return fail(h, PWA_ERR_INVALID_ARG, "NULL array argument (V, nll, grad, and theta when F > 0)");
    if ((reinterpret_cast<uintptr_t>(V) & 7u) || (reinterpret_cast<uintptr_t>(nll) & 7u) ||
        (reinterpret_cast<uintptr_t>(grad) & 7u) || (theta && (reinterpret_cast<uintptr_t>(theta) & 7u)))
        return fail(h, PWA_ERR_INVALID_ARG, "misaligned V, theta, nll or grad");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t s = (cudaStream_t)stream;
    pwa::UnevenPlan plan;
    pwa_status st = uneven_prepare(h, channels, n_ch, &plan, s);
    if (st != PWA_OK) return st;
    cudaError_t e = pwa::uneven_launch(plan, h->uws, reinterpret_cast<const float2*>(V), theta, nll, grad, h->status,
                                       h->sm_count, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "multi-channel launch");
    h->err.clear();
    return PWA_OK;
}

void pwa_fit_default_opts(pwa_fit_opts* o) {
    if (!o) return;
    o->max_iter = 1000;
    o->history = 10;
    o->gtol = 1e-6;
    o->check_every = 20;
    o->gauge_fix = 1;
    o->use_graph = 1;
    o->polar = 0;
}

// the fit kernels' mode bits of a set of options
static int fit_mode(const pwa_fit_opts& o) {
    return (o.gauge_fix ? pwa::FIT_GAUGE : 0) | (o.polar ? pwa::FIT_POLAR : 0);
}

pwa_status pwa_fit_batch(pwa_handle* h, const pwa_fit_desc* fits, int n_fits, const pwa_fit_opts* opts_in,
                         pwa_fit_result* results, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (!fits || n_fits < 1 || !results) return fail(h, PWA_ERR_INVALID_ARG, "fits/results NULL or n_fits < 1");
    pwa_fit_opts o;
    pwa_fit_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.max_iter < 1 || o.history < 1 || o.history > 20 || !(o.gtol > 0.0) || o.check_every < 1 ||
        (o.polar != 0 && o.polar != 1))
        return fail(h, PWA_ERR_INVALID_ARG,
                    "bad options (max_iter >= 1, 1 <= history <= 20, gtol > 0, check_every >= 1, polar 0 or 1)");
    int P_tot = 0;
    size_t ws_need = 0;
    for (int f = 0; f < n_fits; ++f) {
        const pwa_fit_desc& d = fits[f];
        pwa_status st = check_amp_layout(h, d.K, d.n, d.ld);
        if (st != PWA_OK) return st;
        if (d.P < 1 || d.P > (1 << 20)) return fail(h, PWA_ERR_INVALID_ARG, "fit %d: P = %d out of range", f, d.P);
        if ((d.n > 0 && !d.A) || !d.Psi || !d.V0) return fail(h, PWA_ERR_INVALID_ARG, "fit %d: NULL A, Psi or V0", f);
        if ((d.n > 0 && !aligned16(d.A)) || !aligned16(d.Psi) || (reinterpret_cast<uintptr_t>(d.V0) & 7u))
            return fail(h, PWA_ERR_INVALID_ARG, "fit %d: misaligned array", f);
        if (d.V_out && (reinterpret_cast<uintptr_t>(d.V_out) & 15u))
            return fail(h, PWA_ERR_INVALID_ARG, "fit %d: V_out not 16-byte aligned", f);
        if (!std::isfinite(d.n_factor)) return fail(h, PWA_ERR_INVALID_ARG, "fit %d: n_factor not finite", f);
        P_tot += d.P;
        size_t w = pwa::nll_workspace(d.K, d.n, d.P, h->sm_count);
        if (w > ws_need) ws_need = w;
    }
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t s;
    {
        pwa_status fs = fit_stream_begin(h, stream, &s);
        if (fs != PWA_OK) return fs;
    }
    const int m = o.history;
    pwa_status st = ensure_workspace(h, ws_need, P_tot);
    if (st != PWA_OK) return st;
    // fit state + per-fit evaluation buffers (V trial, nll, grad; twice: the second set holds the
    // dense batch of the starts resumed in the precise phase, with their indices)
    size_t state_b = pwa::fit_workspace(P_tot, m);
    size_t need = state_b;
    for (int f = 0; f < n_fits; ++f) need += 2 * pwa::fit_eval_bytes(fits[f].P, fits[f].K) + 256 + sizeof(int) * fits[f].P;
    st = grow_fitws(h, need);
    if (st != PWA_OK) return st;
    struct EvalBuf {
        float2* Vt;
        double* nll;
        double* grad;
        float2* Vc;  // the resumed starts' V, their results and indices into the fit
        double* nll_c;
        double* grad_c;
        int* idx;
        int n_c;
    };
    std::vector<EvalBuf> eb(n_fits);
    std::vector<int> K_of_p(P_tot);
    {
        char* c = reinterpret_cast<char*>(h->fitws) + state_b;
        auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
        int q = 0;
        for (int f = 0; f < n_fits; ++f) {
            const int P = fits[f].P, K = fits[f].K;
            eb[f].Vt = reinterpret_cast<float2*>(c);
            c += r(sizeof(float2) * (size_t)P * K);
            eb[f].nll = reinterpret_cast<double*>(c);
            c += r(sizeof(double) * P);
            eb[f].grad = reinterpret_cast<double*>(c);
            c += r(sizeof(double) * (size_t)P * 2 * K);
            eb[f].Vc = reinterpret_cast<float2*>(c);
            c += r(sizeof(float2) * (size_t)P * K);
            eb[f].nll_c = reinterpret_cast<double*>(c);
            c += r(sizeof(double) * P);
            eb[f].grad_c = reinterpret_cast<double*>(c);
            c += r(sizeof(double) * (size_t)P * 2 * K);
            eb[f].idx = reinterpret_cast<int*>(c);
            c += r(sizeof(int) * (size_t)P);
            eb[f].n_c = 0;
            for (int p = 0; p < P; ++p) K_of_p[q++] = 2 * K;  // components per start
        }
    }
    cudaError_t e = cudaSuccess;
    int off = 0;
    for (int f = 0; f < n_fits && e == cudaSuccess; ++f) {
        e = pwa::fit_launch_init(h->fitws, P_tot, m, reinterpret_cast<const float2*>(fits[f].V0), fits[f].K, fits[f].P,
                                 off, fit_mode(o), eb[f].Vt, s);
        off += fits[f].P;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "fit init");
    // Two phases.  First every fit evaluates with its autotuned tile shape; a start whose line
    // search keeps backtracking (the tensor-core shape's rounding, ~1e-8 of the gradient scale,
    // can hide the decrease near a minimum) pauses.  Then the paused starts resume from their
    // accepted points with the fastest FP32 SIMT shape, without pausing, until they stop; only
    // they are evaluated, as one dense batch per fit (the step skips every other start).
    bool precise = false;
    // PWA_FIT_PAUSE_BACKTRACKS=b (1..255) overrides the pause limit (a test takes it to 1 so that
    // many starts pause and resume)
    int pause_mode = pwa::FIT_PAUSE;
    if (const char* pb = getenv("PWA_FIT_PAUSE_BACKTRACKS")) {
        const int b = atoi(pb);
        if (b >= 1 && b <= 255) pause_mode |= b << pwa::FIT_PAUSE_SHIFT;
    }
    auto iteration = [&]() -> cudaError_t {
        int p_off = 0;
        for (int f = 0; f < n_fits; ++f) {
            const pwa_fit_desc& d = fits[f];
            cudaError_t ee = cudaSuccess;
            if (!precise) {
                ee = pwa::launch_nll(reinterpret_cast<const float2*>(d.A), d.K, d.n, d.ld, eb[f].Vt, d.P,
                                     reinterpret_cast<const double2*>(d.Psi), d.n_factor, eb[f].nll, eb[f].grad,
                                     h->ws, h->ws_bytes, h->counters, h->bad, h->status, h->sm_count, s, false);
            } else if (eb[f].n_c > 0) {
                ee = pwa::fit_gather_sets(eb[f].Vt, eb[f].idx, eb[f].n_c, d.K, eb[f].Vc, s);
                if (ee == cudaSuccess)
                    ee = pwa::launch_nll(reinterpret_cast<const float2*>(d.A), d.K, d.n, d.ld, eb[f].Vc, eb[f].n_c,
                                         reinterpret_cast<const double2*>(d.Psi), d.n_factor, eb[f].nll_c,
                                         eb[f].grad_c, h->ws, h->ws_bytes, h->counters, h->bad, h->status,
                                         h->sm_count, s, true);
                if (ee == cudaSuccess)
                    ee = pwa::fit_scatter_sets(eb[f].nll_c, eb[f].grad_c, eb[f].idx, eb[f].n_c, 2 * d.K, eb[f].nll,
                                               eb[f].grad, s);
            }
            if (ee != cudaSuccess) return ee;
            ee = pwa::fit_launch_step(h->fitws, P_tot, m, eb[f].nll, eb[f].grad, eb[f].Vt, d.K, d.P, p_off,
                                      o.gtol * std::fabs(d.n_factor), fit_mode(o) | (precise ? 0 : pause_mode),
                                      o.max_iter, s);
            if (ee != cudaSuccess) return ee;
            p_off += d.P;
        }
        return cudaSuccess;
    };
    e = run_fit_loop(h, s, o, P_tot, m, iteration);
    if (e != cudaSuccess) return cuda_fail(h, e, "fit loop");
    int n_paused = 0;
    e = pwa::fit_resume_paused(h->fitws, P_tot, m, &n_paused, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "fit resume");
    if (n_paused > 0) {
        std::vector<int> run;
        e = pwa::fit_running_list(h->fitws, P_tot, m, run, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "fit resume");
        std::vector<int> loc;
        int p_off = 0;
        size_t r = 0;
        for (int f = 0; f < n_fits && e == cudaSuccess; ++f) {
            loc.clear();
            for (; r < run.size() && run[r] < p_off + fits[f].P; ++r) loc.push_back(run[r] - p_off);
            eb[f].n_c = (int)loc.size();
            if (!loc.empty())
                e = cudaMemcpyAsync(eb[f].idx, loc.data(), sizeof(int) * loc.size(), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            p_off += fits[f].P;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "fit resume");
        // a smaller batch may take more event chunks per set than the full one
        size_t ws_c = 0;
        for (int f = 0; f < n_fits; ++f)
            if (eb[f].n_c > 0) {
                const size_t w = pwa::nll_workspace(fits[f].K, fits[f].n, eb[f].n_c, h->sm_count);
                if (w > ws_c) ws_c = w;
            }
        st = ensure_workspace(h, ws_c, P_tot);
        if (st != PWA_OK) return st;
        precise = true;
        e = run_fit_loop(h, s, o, P_tot, m, iteration);
        if (e != cudaSuccess) return cuda_fail(h, e, "fit loop (precise evaluation)");
    }
    off = 0;
    for (int f = 0; f < n_fits && e == cudaSuccess; ++f) {
        if (fits[f].V_out)
            e = pwa::fit_export(h->fitws, P_tot, m, fits[f].K, fits[f].P, off, fit_mode(o), fits[f].V_out, s);
        off += fits[f].P;
    }
    std::vector<double> fv, gm;
    std::vector<int> it, ev, stv;
    if (e == cudaSuccess) e = pwa::fit_read_results(h->fitws, P_tot, m, fv, gm, it, ev, stv, K_of_p.data(), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "fit results");
    for (int p = 0; p < P_tot; ++p) {
        results[p].nll = fv[p];
        results[p].grad_max = gm[p];
        results[p].iterations = it[p];
        results[p].evaluations = ev[p];
        results[p].status = stv[p] < 0 ? 1 : stv[p];  // still running at the loop bound: max_iter
    }
    h->err.clear();
    return PWA_OK;
}

pwa_status pwa_fit_shape_batch(pwa_handle* h, const pwa_shape_fit_desc* fits, int n_fits, const pwa_fit_opts* opts_in,
                               pwa_fit_result* results, void* stream) {
    if (!h) return PWA_ERR_INVALID_ARG;
    if (!fits || n_fits < 1 || !results) return fail(h, PWA_ERR_INVALID_ARG, "fits/results NULL or n_fits < 1");
    pwa_fit_opts o;
    pwa_fit_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.max_iter < 1 || o.history < 1 || o.history > 20 || !(o.gtol > 0.0) || o.check_every < 1 ||
        (o.polar != 0 && o.polar != 1))
        return fail(h, PWA_ERR_INVALID_ARG, "bad options");
    std::vector<pwa_uneven_channel> chs(n_fits);
    for (int f = 0; f < n_fits; ++f) {
        const pwa_shape_fit_desc& d = fits[f];
        pwa_uneven_channel& c = chs[f];
        c.waves = d.waves;
        c.K = d.K;
        c.kin = d.kin;
        c.n = d.n;
        c.ld = d.ld;
        c.kin_mc = d.kin_mc;
        c.n_mc = d.n_mc;
        c.ld_mc = d.ld_mc;
        c.w_mc = d.w_mc;
        c.n_gen = d.n_gen;
        c.n_factor = d.n_factor;
        c.F = d.F;
        c.float_wave = d.float_wave;
        c.float_kind = d.float_kind;
        pwa_status st = check_uneven_channel(h, c, f);
        if (st != PWA_OK) return st;
        if (2 * d.K + d.F > 128) return fail(h, PWA_ERR_INVALID_ARG, "fit %d: 2K + F > 128", f);
        if (!d.V0 || !d.kin || !d.kin_mc) return fail(h, PWA_ERR_INVALID_ARG, "fit %d: NULL array", f);
        if ((reinterpret_cast<uintptr_t>(d.V0) & 7u) || (d.x_out && (reinterpret_cast<uintptr_t>(d.x_out) & 7u)))
            return fail(h, PWA_ERR_INVALID_ARG, "fit %d: misaligned array", f);
    }
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(h, PWA_ERR_CUDA, "cannot select device %d", h->device);
    cudaStream_t s;
    pwa_status pst = fit_stream_begin(h, stream, &s);
    if (pst != PWA_OK) return pst;
    pwa::UnevenPlan plan;
    pst = uneven_prepare(h, chs.data(), n_fits, &plan, s);
    if (pst != PWA_OK) return pst;
    const int m = o.history;
    const int P_tot = n_fits;
    // workspace: fit state, then the packed trial V and theta, f, gradient and per-start step arguments
    auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t state_b = pwa::fit_workspace(P_tot, m);
    const size_t vt_b = r256(sizeof(float2) * plan.n_v), th_b = r256(sizeof(double) * (plan.n_theta + 1)),
                 f_b = r256(sizeof(double) * n_fits), g_b = r256(sizeof(double) * plan.n_grad),
                 a_b = r256(sizeof(pwa::StepArgs) * n_fits);
    pst = grow_fitws(h, state_b + vt_b + th_b + f_b + g_b + a_b);
    if (pst != PWA_OK) return pst;
    char* c0 = reinterpret_cast<char*>(h->fitws) + state_b;
    float2* Vt = reinterpret_cast<float2*>(c0);
    double* tht = reinterpret_cast<double*>(c0 + vt_b);
    double* fv_d = reinterpret_cast<double*>(c0 + vt_b + th_b);
    double* gv_d = reinterpret_cast<double*>(c0 + vt_b + th_b + f_b);
    pwa::StepArgs* args_d = reinterpret_cast<pwa::StepArgs*>(c0 + vt_b + th_b + f_b + g_b);
    std::vector<pwa::StepArgs> args(n_fits);
    std::vector<std::vector<double>> th0(n_fits);
    for (int f = 0; f < n_fits; ++f) {
        const pwa_shape_fit_desc& d = fits[f];
        const pwa::UnevenChannel& u = plan.chans[f];
        pwa::StepArgs& a = args[f];
        a.K = d.K;
        a.F = d.F;
        a.goff = u.goff;
        a.voff = u.voff;
        a.toff = u.toff;
        a.gtol = o.gtol * std::fabs(d.n_factor);
        th0[f].resize(d.F);
        for (int q = 0; q < PWA_MAX_FLOAT; ++q) a.lb[q] = 1e-3;  // masses and widths stay above 1 MeV
        for (int q = 0; q < d.F; ++q)
            th0[f][q] = d.float_kind[q] == 0 ? d.waves[d.float_wave[q]].mass : d.waves[d.float_wave[q]].width;
    }
    cudaError_t e = cudaMemcpyAsync(args_d, args.data(), sizeof(pwa::StepArgs) * n_fits, cudaMemcpyHostToDevice, s);
    for (int f = 0; f < n_fits && e == cudaSuccess; ++f) {
        const pwa_shape_fit_desc& d = fits[f];
        e = pwa::fit_launch_init(h->fitws, P_tot, m, reinterpret_cast<const float2*>(d.V0), d.K, 1, f, fit_mode(o),
                                 Vt + args[f].voff, s, d.F, th0[f].data(), tht + args[f].toff);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors above must outlive the copies
    if (e != cudaSuccess) return cuda_fail(h, e, "shape fit init");
    // one iteration: every channel's f and gradient in one persistent launch, then one L-BFGS step
    // launch over all channels
    auto iteration = [&]() -> cudaError_t {
        cudaError_t ee = pwa::uneven_launch(plan, h->uws, Vt, tht, fv_d, gv_d, h->status, h->sm_count, s);
        if (ee != cudaSuccess) return ee;
        return pwa::fit_launch_step_multi(h->fitws, P_tot, m, args_d, fv_d, gv_d, Vt, tht, fit_mode(o), o.max_iter, s);
    };
    e = run_fit_loop(h, s, o, P_tot, m, iteration);
    if (e != cudaSuccess) return cuda_fail(h, e, "shape fit loop");
    std::vector<int> D_of_p(P_tot);
    for (int f = 0; f < n_fits && e == cudaSuccess; ++f) {
        D_of_p[f] = 2 * fits[f].K + fits[f].F;
        if (fits[f].x_out)
            e = pwa::fit_export_x(h->fitws, P_tot, m, fits[f].K, D_of_p[f], f, fit_mode(o), fits[f].x_out, s);
    }
    std::vector<double> fv, gm;
    std::vector<int> it, ev, stv;
    if (e == cudaSuccess) e = pwa::fit_read_results(h->fitws, P_tot, m, fv, gm, it, ev, stv, D_of_p.data(), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "shape fit results");
    for (int p = 0; p < P_tot; ++p) {
        results[p].nll = fv[p];
        results[p].grad_max = gm[p];
        results[p].iterations = it[p];
        results[p].evaluations = ev[p];
        results[p].status = stv[p] < 0 ? 1 : stv[p];
    }
    h->err.clear();
    return PWA_OK;
}

}  // extern "C"
