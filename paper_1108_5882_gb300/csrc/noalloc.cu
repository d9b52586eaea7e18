// -lnL and its gradient for one parameter set without any device allocation.
//
// Some callers cannot call cudaMalloc: host code under a memory manager that forbids
// allocations after start-up, plug-ins of a larger program that owns all device memory, and
// latency-critical loops that must not take the allocator's locks or its implicit
// synchronisation.  pwa_nll_grad needs a handle, and both the handle and its workspace are
// allocated with cudaMalloc.  pwa_nll_grad_noalloc needs neither: its scratch (block partial
// sums, the completion counter, flags and fixed-point sums) lives in the file-scope device array
// below, which every GPU that loads the library holds until exit.
//
// Limits: K <= PWA_MAX_WAVES and at most NOALLOC_MAX_BLOCKS blocks per launch (the launch is
// capped there; any n is accepted).  The scratch is shared by every call on a device and keeps
// the last call's contents: each call clears the control words on its stream before
// its kernel runs, so calls ordered on one stream are safe, while calls that overlap on the
// GPU (different streams, different host threads) race on the scratch and give wrong results.
//
// The scratch's device address belongs to the CUDA context in which it was looked up.  It is
// looked up on the first call in each context (keyed by the driver's unique context id, so a
// context created after cudaDeviceReset, or another context made current on the same device,
// gets a fresh lookup instead of a stale address).
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "pwa_internal.cuh"

namespace {

constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr size_t NOALLOC_HEADER = 8448;  // control words of the launch, then the status word
constexpr size_t NOALLOC_STATUS_OFFSET = pwa::STREAM_CTRL_BYTES;
static_assert(NOALLOC_STATUS_OFFSET + sizeof(int) <= NOALLOC_HEADER, "noalloc header");
constexpr size_t NOALLOC_PART_BYTES = sizeof(float2) * (size_t)NOALLOC_MAX_BLOCKS * (1 + 2 * PWA_MAX_WAVES);
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + NOALLOC_PART_BYTES;  // 1,056,768 + 8448 bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
struct NoallocSlot {
    unsigned long long ctx_id;  // unique id of the context the address was looked up in
    void* ptr;
    int sms;
    bool valid;
};
NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES] = {};

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime (no link-time
// dependency on libcuda).
using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

bool current_context_id(int dev, unsigned long long* id) {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return false;
        get_current = reinterpret_cast<PfnCtxGetCurrent>(f0);
        get_id = reinterpret_cast<PfnCtxGetId>(f1);
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS) return false;
    if (!c) {
        // no context is current yet: cudaSetDevice makes the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess || get_current(&c) != CUDA_SUCCESS || !c) return false;
    }
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array and the SM count of the current device, looked up once
// per context (with that device current).  In host code the symbol g_noalloc_scratch is only a
// host-side stand-in: its device address has to come from cudaGetSymbolAddress.
cudaError_t noalloc_setup(int dev, void** ptr, int* sms) {
    unsigned long long id = 0;
    if (!current_context_id(dev, &id)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocSlot& s = g_noalloc_slot[dev];
    if (!s.valid || s.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        s.ptr = p;
        s.sms = n > 0 ? n : 1;
        s.ctx_id = id;
        s.valid = true;
    }
    *ptr = s.ptr;
    *sms = s.sms;
    return cudaSuccess;
}

pwa_status noalloc_fail(pwa_status st, const char* msg) {
    pwa::record_global_error(msg);
    return st;
}

}  // namespace

extern "C" PWA_API pwa_status pwa_nll_grad_noalloc(const float* A, int K, int64_t n, int64_t ld, const float* V,
                                                   const double* Psi, double n_factor, double* nll, double* grad,
                                                   void* stream) {
    if (K < 1 || K > PWA_MAX_WAVES) return noalloc_fail(PWA_ERR_INVALID_ARG, "pwa_nll_grad_noalloc: K outside [1, 64]");
    if (n < 0 || ld < n || (ld & 1) || (int64_t)K * ld > ((int64_t)1 << 40))
        return noalloc_fail(PWA_ERR_INVALID_ARG, "pwa_nll_grad_noalloc: need 0 <= n <= ld, ld even");
    if ((n > 0 && !A) || !V || !Psi || !nll || !grad)
        return noalloc_fail(PWA_ERR_INVALID_ARG, "pwa_nll_grad_noalloc: NULL array argument");
    if ((n > 0 && (reinterpret_cast<uintptr_t>(A) & 15u)) || (reinterpret_cast<uintptr_t>(Psi) & 15u) ||
        (reinterpret_cast<uintptr_t>(V) & 7u))
        return noalloc_fail(PWA_ERR_INVALID_ARG, "pwa_nll_grad_noalloc: misaligned array");
    if (!(n_factor == n_factor) || n_factor > 1e300 || n_factor < -1e300)
        return noalloc_fail(PWA_ERR_INVALID_ARG, "pwa_nll_grad_noalloc: n_factor not finite");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return noalloc_fail(PWA_ERR_NO_DEVICE, "pwa_nll_grad_noalloc: no usable current device");
    }
    void* base = nullptr;
    int sms = 1;
    cudaError_t e = noalloc_setup(dev, &base, &sms);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(PWA_ERR_CUDA, "pwa_nll_grad_noalloc: no current context, or cudaGetSymbolAddress of the "
                                          "scratch failed");
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* b = reinterpret_cast<unsigned char*>(base);
    unsigned* counter = reinterpret_cast<unsigned*>(b);
    int* badw = reinterpret_cast<int*>(b + 4);
    int* status = reinterpret_cast<int*>(b + NOALLOC_STATUS_OFFSET);
    float2* part = reinterpret_cast<float2*>(b + NOALLOC_HEADER);
    // the previous call's words may be left set (e.g. the status bit of a non-finite set)
    e = cudaMemsetAsync(b, 0, NOALLOC_STATUS_OFFSET + sizeof(int), st);
    if (e == cudaSuccess)
        e = pwa::launch_nll_grad_scratch(reinterpret_cast<const float2*>(A), K, n, ld,
                                         reinterpret_cast<const float2*>(V), reinterpret_cast<const double2*>(Psi),
                                         n_factor, nll, grad, part, NOALLOC_PART_BYTES, counter, badw, status,
                                         NOALLOC_MAX_BLOCKS, sms, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(PWA_ERR_CUDA, "pwa_nll_grad_noalloc: launch failed");
    }
    return PWA_OK;
}
