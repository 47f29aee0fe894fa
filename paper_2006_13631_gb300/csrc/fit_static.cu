// hlbm_fit_static: the least-squares sine fit of hlbm_gamma for callers that
// cannot allocate device memory.
//
// Some callers must not allocate: services that run under a fixed
// device-memory budget or inside a framework that owns every allocation,
// and time-critical loops that cannot afford the implicit device
// synchronisation of cudaMalloc / cudaFree.  This entry point takes the
// samples from the caller's device memory and keeps its intermediate sums in
// one file-scope device array instead of allocating.
//
// That array (kFitBlocks x 8 doubles) exists on every GPU that loads the
// library and stays there until the process exits.  All calls on a device
// share it and it keeps the last call's contents; every slot a call reads
// is written earlier in the same call, so nothing has to be cleared, but
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cuda.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "hlbm.h"

namespace {

constexpr int kFitBlocks = 256;      // blocks of the partial-sum passes
constexpr int kFitThreads = 256;
constexpr int64_t kFitMaxSamples = (int64_t)1 << 26;
constexpr int kMaxDevices = 64;

// partial sums of each block (5 used by the first pass, 1 by the residual
// pass) and, in the last row, the final results
static __device__ __align__(256) double g_fit_scratch[(kFitBlocks + 1) * 8];

// Device address of g_fit_scratch per device, with the unique id of the
// context it belongs to.  In host code the name g_fit_scratch denotes a
// host-side stand-in, so the address must come from cudaGetSymbolAddress.
// It is looked up on the first call on a device and again whenever the
// device's current context has changed (a cudaDeviceReset destroys the
// primary context and the module with it; context ids are never reused).
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_ctx_once;

// unique id of the current context, 0 when there is none (or no driver entry)
unsigned long long current_ctx_id() {
    std::call_once(g_ctx_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = (CtxGetIdFn)fn;
        cudaGetLastError();
    });
    unsigned long long id = 0;
    if (!g_ctx_get_id || g_ctx_get_id(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr& c = g_scratch_addr[dev];
    const unsigned long long id = current_ctx_id();
    if (c.ptr && id != 0 && id == c.ctx_id) {
        *out = c.ptr;
        return cudaSuccess;
    }
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_fit_scratch);  // makes the primary context current
    if (e != cudaSuccess) {
        c = ScratchAddr{};
        return e;
    }
    c.ptr = p;
    c.ctx_id = current_ctx_id();
    *out = p;
    return cudaSuccess;
}

// Per-block sums over samples t0..t1 of s^2, s c, c^2, F s, F c with
// s = sin(w t), c = cos(w t), F = samples[t * stride].
__global__ void __launch_bounds__(kFitThreads) k_fit_partials(const double* samples, int64_t stride, int64_t t0,
                                                             int64_t t1, double omega, double* scratch) {
    __shared__ double sh[5][kFitThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t t = t0 + blockIdx.x * (int64_t)kFitThreads + threadIdx.x; t <= t1;
         t += (int64_t)gridDim.x * kFitThreads) {
        double s, c;
        sincos(omega * (double)t, &s, &c);
        const double F = samples[t * stride];
        acc[0] += s * s;
        acc[1] += s * c;
        acc[2] += c * c;
        acc[3] += F * s;
        acc[4] += F * c;
    }
    for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = kFitThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) scratch[8 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// Fixed-order sum of the block partials, then the 2x2 normal equations:
// a, b into the result row, and in its slot 3 whether the system is regular.
// With s = sin(w t), c = cos(w t), s^2 + c^2 = 1, so S_ss + S_cc is the sample
// count n and det = S_ss S_cc - S_sc^2 <= n^2 / 4; det below 1e-12 n^2 means
// the two columns are (nearly) dependent, e.g. w a multiple of pi, where
// sin(w t) vanishes at every integer t.
__global__ void k_fit_solve(int nblocks, double* scratch) {
    if (threadIdx.x != 0) return;
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int j = 0; j < 5; ++j) s[j] += scratch[8 * b + j];
    const double det = s[0] * s[2] - s[1] * s[1];
    const double n = s[0] + s[2];
    double* res = scratch + 8 * kFitBlocks;
    res[0] = (s[3] * s[2] - s[4] * s[1]) / det;
    res[1] = (s[4] * s[0] - s[3] * s[1]) / det;
    res[3] = (isfinite(det) && det > 1e-12 * n * n) ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(kFitThreads) k_fit_resid_partials(const double* samples, int64_t stride, int64_t t0,
                                                                   int64_t t1, double omega, double* scratch) {
    __shared__ double sh[kFitThreads];
    const double* res = scratch + 8 * kFitBlocks;
    const double a = res[0], b = res[1];
    double acc = 0.0;
    for (int64_t t = t0 + blockIdx.x * (int64_t)kFitThreads + threadIdx.x; t <= t1;
         t += (int64_t)gridDim.x * kFitThreads) {
        double s, c;
        sincos(omega * (double)t, &s, &c);
        const double e = samples[t * stride] - (a * s + b * c);
        acc += e * e;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kFitThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[8 * blockIdx.x + 5] = sh[0];
}

__global__ void k_fit_rms(int nblocks, int64_t count, double* scratch) {
    if (threadIdx.x != 0) return;
    double r2 = 0.0;
    for (int b = 0; b < nblocks; ++b) r2 += scratch[8 * b + 5];
    scratch[8 * kFitBlocks + 2] = sqrt(r2 / (double)count);
}

}  // namespace

extern "C" int hlbm_fit_static(const double* samples, int64_t stride, int64_t t0, int64_t t1, double omega,
                               void* cuda_stream, double* a, double* b, double* rms) {
    if (!samples || !a || !b || stride < 1 || t0 < 0 || t1 <= t0 || !(omega > 0.0) || !std::isfinite(omega))
        return HLBM_EINVAL;
    const int64_t count = t1 - t0 + 1;
    if (count > kFitMaxSamples) return HLBM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the call ends with a read-back to host memory and a stream
    // synchronisation, which a stream being captured does not allow (they
    // would invalidate the caller's capture): refuse before touching it
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        if (e != cudaSuccess) cudaGetLastError();
        return HLBM_EINVAL;
    }
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return HLBM_ECUDA;
    const int nblocks = (int)((count + kFitThreads * 16 - 1) / (kFitThreads * 16)) < kFitBlocks
                            ? (int)((count + kFitThreads * 16 - 1) / (kFitThreads * 16))
                            : kFitBlocks;
    k_fit_partials<<<nblocks, kFitThreads, 0, s>>>(samples, stride, t0, t1, omega, scratch);
    k_fit_solve<<<1, 32, 0, s>>>(nblocks, scratch);
    k_fit_resid_partials<<<nblocks, kFitThreads, 0, s>>>(samples, stride, t0, t1, omega, scratch);
    k_fit_rms<<<1, 32, 0, s>>>(nblocks, count, scratch);
    // a rejected launch must not let the read-back return the previous
    // call's results, which the shared array still holds
    e = cudaGetLastError();
    if (e != cudaSuccess) return HLBM_ECUDA;
    double out[4];
    e = cudaMemcpyAsync(out, scratch + 8 * kFitBlocks, sizeof out, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HLBM_ECUDA;
    if (out[3] != 1.0) return HLBM_EINVAL;  // sin and cos columns dependent: no unique fit
    *a = out[0];
    *b = out[1];
    if (rms) *rms = out[2];
    return HLBM_OK;
}
