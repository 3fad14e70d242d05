// osscir_dtpl_counts_static: the transmission-Poisson data discrepancy D_TPL of
// given expected and measured counts, computed without allocating any memory.
//
// Why this exists: some callers of this library must not call cudaMalloc after
// start-up, for example a server whose memory arena claims the device memory
// at launch so later cudaMalloc calls fail, or a latency-bound loop that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree may
// imply.  The other D_TPL entry point (osscir_dtpl) needs a context, whose
// creation allocates.  This variant needs no context: its per-block partial
// sums live in a fixed-size array in the library's own device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (128 KiB) until the process exits.  Host code must not pass
// the variable's name to a kernel (on the host that name is only a stand-in,
// not a device address); the address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

#include "../../include/osscir.h"
#include "osscir_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPartials = 16384;                     // 128 KiB of doubles
constexpr long long kMaxRays = (long long)kThreads * kMaxPartials;   // 4,194,304 rays
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dtpl_partials[kMaxPartials];

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

// c^ - c - c log(c^/c) = c (u - log(1 + u)), u = (c^ - c)/c; a series for small
// |u| avoids the cancellation; a measured count of zero contributes c^.
__device__ __forceinline__ float dtpl_term_static(float chat, float c) {
    if (!(c > 0.0f)) return chat;
    const float u = (chat - c) / c;
    if (fabsf(u) < 0.0625f) {
        const float p = 0.5f - u * (1.0f / 3.0f - u * (0.25f - u * (0.2f - u * (1.0f / 6.0f - u * (1.0f / 7.0f - u * 0.125f)))));
        return c * u * u * p;
    }
    return chat - c - c * logf(chat / c);
}

__device__ __forceinline__ double block_sum_static(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;
}

// One partial per block: the D_TPL terms of its rays (four windows each).
__global__ void __launch_bounds__(kThreads) k_dtpl_terms_static(const float4* chat, const float4* c, int n_rays,
                                                                double* partials) {
    __shared__ double red[kThreads / 32];
    const int l = blockIdx.x * kThreads + threadIdx.x;
    double v = 0.0;
    if (l < n_rays) {
        const float4 a = chat[l], b = c[l];
        v = (double)dtpl_term_static(a.x, b.x) + (double)dtpl_term_static(a.y, b.y) +
            (double)dtpl_term_static(a.z, b.z) + (double)dtpl_term_static(a.w, b.w);
    }
    const double s = block_sum_static(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Fixed-order sum of the partials (deterministic for a given n_rays).
__global__ void __launch_bounds__(kThreads) k_dtpl_sum_static(const double* partials, int n, double* out) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += partials[i];
    const double t = block_sum_static(s, red);
    if (threadIdx.x == 0) *out = t;
}

// Device address of the partials array on the current device (looked up on
// the first call on each device, with that device current).
osscir_status partials_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OSSCIR_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return OSSCIR_E_INVALID;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dtpl_partials) != cudaSuccess || !p) return OSSCIR_E_CUDA;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return OSSCIR_OK;
}

}  // namespace

extern "C" osscir_status osscir_dtpl_counts_static(const float* chat, const float* c, int n_rays, double* out,
                                                   void* stream) {
    if (!chat || !c || !out || n_rays < 1) return OSSCIR_E_INVALID;
    if ((long long)n_rays > kMaxRays) return OSSCIR_E_INVALID;
    double* partials = nullptr;
    const osscir_status s = partials_address(&partials);
    if (s != OSSCIR_OK) return s;
    const int blocks = (n_rays + kThreads - 1) / kThreads;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_dtpl_terms_static<<<blocks, kThreads, 0, st>>>(reinterpret_cast<const float4*>(chat),
                                                     reinterpret_cast<const float4*>(c), n_rays, partials);
    if (cudaGetLastError() != cudaSuccess) return OSSCIR_E_CUDA;
    k_dtpl_sum_static<<<1, kThreads, 0, st>>>(partials, blocks, out);
    if (cudaGetLastError() != cudaSuccess) return OSSCIR_E_CUDA;
    return OSSCIR_OK;
}
