// Allocation-free variant of the plain per-model FP64 value iteration.
//
// Its scratch (the second value buffer, the state-action values, the
// recorded actions and the residual word) lives in one file-scope static
// device array, so the call itself never allocates device or pinned host
// memory.  It runs the same kernels as morap_solve_plain, including the
// scheduler's anchoring rounds (its one extra scratch word is the round
// counter next to the residual word).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace morap {
namespace {

constexpr int64_t kNoallocMaxStates = 131072;  // product states, done slot included
constexpr int64_t kNoallocMaxSA = 655360;      // state-action rows

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffY = 0;
constexpr size_t kOffQ = kOffY + align256(sizeof(double) * kNoallocMaxStates);
constexpr size_t kOffRec = kOffQ + align256(sizeof(double) * kNoallocMaxSA);
constexpr size_t kOffRes = kOffRec + align256(sizeof(int32_t) * kNoallocMaxStates);
constexpr size_t kScratchBytes = kOffRes + 256;  // about 6.3 MB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// symbol itself is only a host-side stand-in, so the address is looked up
// once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MORAP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(MORAP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(MORAP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return MORAP_OK;
}

}  // namespace
}  // namespace morap

using namespace morap;

extern "C" int morap_plain_vi_noalloc(int32_t n_states, int32_t n_sa, const uint32_t *state_sa, const uint32_t *sa_tr,
                                      const int32_t *col, const double *prob, const double *cost, int32_t pre_begin,
                                      int32_t init_state, double w_cost, double w_prob, double eps, double tau,
                                      int32_t max_sweeps, void *stream, double *values, int32_t *policy,
                                      double *c_out, int32_t *sweeps_out) {
    if (n_states < 0 || n_sa < 0 || !state_sa || !sa_tr || !col || !prob || !cost || !values || !policy)
        return fail(MORAP_EINVAL, "noalloc: null pointer or negative size");
    if ((int64_t)n_states + 1 > kNoallocMaxStates || (int64_t)n_sa > kNoallocMaxSA)
        return fail(MORAP_EINVAL, "noalloc: at most " + std::to_string(kNoallocMaxStates - 1) + " states and " +
                                      std::to_string(kNoallocMaxSA) + " state-action rows (got " +
                                      std::to_string(n_states) + ", " + std::to_string(n_sa) + ")");
    if (init_state < 0 || init_state > n_states || pre_begin < 0 || pre_begin > n_states)
        return fail(MORAP_EINVAL, "noalloc: init_state / pre_begin out of range");
    if (!(eps > 0) || !(tau >= 0) || max_sweeps < 1 || !(w_cost >= 0) || !(w_prob >= 0))
        return fail(MORAP_EINVAL, "noalloc: eps > 0, tau >= 0, max_sweeps >= 1, weights >= 0 required");
    cudaStream_t s = (cudaStream_t)stream;
    // The call waits on the stream after every sweep, so it cannot be part of
    // a stream capture: refuse one before touching the stream.
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &capturing);
    if (ce != cudaSuccess) return fail(MORAP_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (capturing != cudaStreamCaptureStatusNone)
        return fail(MORAP_EINVAL, "noalloc: the stream is being captured (the call is synchronous)");
    // The scratch is the current device's copy of the array: the stream and
    // every buffer must belong to that device too.
    int dev = -1;
    if ((ce = cudaGetDevice(&dev)) != cudaSuccess)
        return fail(MORAP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (s) {
        int sdev = -1;
        if ((ce = cudaStreamGetDevice(s, &sdev)) != cudaSuccess)
            return fail(MORAP_ECUDA, std::string("cudaStreamGetDevice: ") + cudaGetErrorString(ce));
        if (sdev != dev)
            return fail(MORAP_EINVAL, "noalloc: the stream belongs to device " + std::to_string(sdev) +
                                          ", the current device is " + std::to_string(dev));
    }
    const void *bufs[] = {state_sa, sa_tr, col, prob, cost, values, policy};
    const char *names[] = {"state_sa", "sa_tr", "col", "prob", "cost", "values", "policy"};
    for (int i = 0; i < 7; ++i) {
        cudaPointerAttributes at{};
        if ((ce = cudaPointerGetAttributes(&at, bufs[i])) != cudaSuccess) {
            cudaGetLastError();
            return fail(MORAP_EINVAL, std::string("noalloc: ") + names[i] + " is not a device address");
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return fail(MORAP_EINVAL, std::string("noalloc: ") + names[i] + " is not memory of the current device (" +
                                          std::to_string(dev) + ")");
    }
    unsigned char *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != MORAP_OK) return rc;
    double *y = reinterpret_cast<double *>(scratch + kOffY);
    double *q = reinterpret_cast<double *>(scratch + kOffQ);
    int32_t *a_rec = reinterpret_cast<int32_t *>(scratch + kOffRec);
    unsigned long long *dres = reinterpret_cast<unsigned long long *>(scratch + kOffRes);
    const uint32_t n = (uint32_t)n_states;
    // the scratch keeps the previous call's contents: clear what must start at 0
#define NA_CK(call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail(MORAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define NA_CKL(expr)                                                                                  \
    do {                                                                                              \
        int e_ = (expr);                                                                              \
        if (e_ != 0) return fail(MORAP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString((cudaError_t)e_)); \
    } while (0)
    NA_CK(cudaMemsetAsync(values, 0, sizeof(double) * (n + 1), s));
    NA_CK(cudaMemsetAsync(y, 0, sizeof(double) * (n + 1), s));
    NA_CK(cudaMemsetAsync(a_rec, 0, sizeof(int32_t) * (n + 1), s));
    // the first state-action row of the pre-sink states (read from the device)
    uint32_t pre_sa_begin = (uint32_t)n_sa;
    if ((uint32_t)pre_begin < n)
        NA_CK(cudaMemcpyAsync(&pre_sa_begin, state_sa + pre_begin, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    double *xc = values, *yc = y;
    int sweeps = 0;
    bool converged = false;
    while (sweeps < max_sweeps) {
        NA_CK(cudaMemsetAsync(dres, 0, sizeof(unsigned long long), s));
        NA_CKL(launch_plain_spmv(sa_tr, col, prob, cost, 0u, (uint32_t)n_sa, w_cost, w_prob, pre_sa_begin, 0u, xc, q,
                                 s));
        NA_CKL(launch_plain_reduce(state_sa, 0u, n, 0u, q, xc, yc, a_rec, eps, dres, s));
        unsigned long long rbits = 0;
        NA_CK(cudaMemcpyAsync(&rbits, dres, sizeof(rbits), cudaMemcpyDeviceToHost, s));
        NA_CK(cudaStreamSynchronize(s));
        std::swap(xc, yc);
        ++sweeps;
        double r;
        std::memcpy(&r, &rbits, sizeof(r));
        if (r <= eps) {
            converged = true;
            break;
        }
    }
    if (xc != values) NA_CK(cudaMemcpyAsync(values, xc, sizeof(double) * (n + 1), cudaMemcpyDeviceToDevice, s));
    NA_CKL(launch_plain_spmv(sa_tr, col, prob, cost, 0u, (uint32_t)n_sa, w_cost, w_prob, pre_sa_begin, 0u, values, q,
                             s));
    NA_CKL(plain_finalize(state_sa, sa_tr, col, prob, 0u, n, 0u, q, a_rec, tau, policy, dres + 1, s));
    double c = 0.0;
    if ((uint32_t)init_state < n) NA_CK(cudaMemcpyAsync(&c, values + init_state, sizeof(c), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
#undef NA_CKL
    if (c_out) *c_out = c;
    if (sweeps_out) *sweeps_out = sweeps;
    if (!converged) return fail(MORAP_ENOTCONV, "noalloc: sweep cap reached");
    return MORAP_OK;
}
