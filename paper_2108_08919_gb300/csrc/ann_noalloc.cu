// Velocity moments of a device velocity field with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a host framework that owns a fixed device memory pool or a
// hard memory budget and forbids allocations after start-up, or a real-time loop that cannot take
// the implicit device synchronisation cudaMalloc may perform.  This entry point serves them: its
// only scratch (one FP64 partial sum per block of 256 particles, and a completion ticket) is the
// file-scope array below, which every GPU that loads this library holds until the process exits.
#include "../../include/ann.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int kQ = 4;                                       // moments per block partial
constexpr int kMaxBlocks = ANN_NOALLOC_MAX_N / kThreads;     // 8192
constexpr size_t kPartialBytes = sizeof(double) * kQ * kMaxBlocks;
constexpr size_t kScratchBytes = kPartialBytes + 256;        // partials, then the ticket
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a host-side stand-in for the device array: host
// code must use the address obtained from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// One pass: each block reduces its 256 particles in a fixed order and stores a partial; the block
// that takes the last ticket reduces the partials in block order and writes out[0..3].  The result
// does not depend on which block finishes last.
__global__ void __launch_bounds__(kThreads) k_moments_noalloc(const float *ux, const float *uy, const float *mass,
                                                              double m0, int n, unsigned char *scratch,
                                                              double *out)
{
    __shared__ double red[kQ][kThreads];
    __shared__ bool last;
    double *part = reinterpret_cast<double *>(scratch);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + kPartialBytes);
    int t = threadIdx.x;
    int i = blockIdx.x * kThreads + t;
    double v[kQ] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        double x = ux[i], y = uy[i];
        double m = mass ? (double)mass[i] : m0;
        v[0] = m * x;
        v[1] = m * y;
        v[2] = 0.5 * (x * x + y * y);
        v[3] = sqrt(x * x + y * y);
    }
    for (int q = 0; q < kQ; q++) red[q][t] = v[q];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (t < s) {
            for (int q = 0; q < 3; q++) red[q][t] += red[q][t + s];
            red[3][t] = fmax(red[3][t], red[3][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        for (int q = 0; q < kQ; q++) part[blockIdx.x * kQ + q] = red[q][0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int q = 0; q < kQ; q++) {
        double acc = 0.0;   // sums, and the max of non-negative speeds
        for (int k = t; k < (int)gridDim.x; k += kThreads) {
            double a = __ldcg(&part[k * kQ + q]);
            acc = (q == 3) ? fmax(acc, a) : acc + a;
        }
        red[q][t] = acc;
    }
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (t < s) {
            for (int q = 0; q < 3; q++) red[q][t] += red[q][t + s];
            red[3][t] = fmax(red[3][t], red[3][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
        out[2] = red[2][0] / (double)n;
        out[3] = red[3][0];
        *ticket = 0u;
    }
}

// True when p is device (or managed) memory of device dev: the kernel runs on dev and must not be
// handed host memory or another GPU's memory.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int ann_velocity_moments_noalloc(const float *ux, const float *uy, const float *mass, double m0,
                                            int64_t n, double *out, void *stream)
{
    if (!ux || !uy || !out || n < 1) return ANN_ERR_INVALID_ARG;
    if (n > ANN_NOALLOC_MAX_N) return ANN_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return ANN_ERR_CUDA;
    }
    if (!on_device(ux, dev) || !on_device(uy, dev) || !on_device(out, dev) || (mass && !on_device(mass, dev)))
        return ANN_ERR_INVALID_ARG;
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            // set-up, once per device, with that device current
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return ANN_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<unsigned char *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the completion ticket must start at zero
    if (cudaMemsetAsync(scratch + kPartialBytes, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return ANN_ERR_CUDA;
    }
    int blocks = (int)((n + kThreads - 1) / kThreads);
    k_moments_noalloc<<<blocks, kThreads, 0, s>>>(ux, uy, mass, m0, (int)n, scratch, out);
    if (cudaGetLastError() != cudaSuccess) return ANN_ERR_CUDA;
    return ANN_OK;
}
