// Seeded Poisson noise for simulated counts (include/osscir.h,
// osscir_poisson_noise): c ~ Poisson(c^) elementwise, the way the paper's
// simulated data are made noisy (Sec. 3), on the device.
//
// Uniform numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011): per round the two
// 32x32-bit products of words 0 and 2 with 0xD2511F53 and 0xCD9E8D57 are mixed
// with words 1 and 3 and the key, and the key advances by 0x9E3779B9 and
// 0xBB67AE85.  Sample i takes its t-th draw from counter (i, t, 0, 0) under key
// (seed mod 2^32, seed / 2^32), two output words making one uniform with 53
// random bits.  Means below 10 are sampled by inverting the distribution
// function; larger ones by the transformed rejection with squeeze of Hormann
// (1993).  The arithmetic that decides a count is FP64 with every operation
// spelled as an _rn intrinsic, so no FMA contraction changes it.
#include <cstdint>

#include "../../include/osscir.h"

namespace {

__device__ __forceinline__ uint4 philox10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * x.x, hi0 = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo1 = 0xCD9E8D57u * x.z, hi1 = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

// [0, 1) from the top 27 + 26 bits of two words
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
    return __dmul_rn(__dadd_rn(__dmul_rn((double)(hi >> 5), 67108864.0), (double)(lo >> 6)),
                     1.0 / 9007199254740992.0);
}

// log k! : the log of the exact product up to 18! (< 2^53), else the Stirling
// series of log Gamma(k + 1) to its x^-7 term.
__device__ double log_kfact(double k) {
    if (k <= 18.0) {
        double p = 1.0;
        for (double i = 2.0; i <= k; i = __dadd_rn(i, 1.0)) p = __dmul_rn(p, i);
        return log(p);
    }
    const double x = __dadd_rn(k, 1.0), ix = __ddiv_rn(1.0, x), ix2 = __dmul_rn(ix, ix);
    double t = __dsub_rn(1.0 / 1260.0, __dmul_rn(ix2, 1.0 / 1680.0));
    t = __dsub_rn(1.0 / 360.0, __dmul_rn(ix2, t));
    t = __dsub_rn(1.0 / 12.0, __dmul_rn(ix2, t));
    const double series = __dmul_rn(ix, t);
    const double main = __dsub_rn(__dmul_rn(__dsub_rn(x, 0.5), log(x)), x);
    return __dadd_rn(__dadd_rn(main, 0.91893853320467274178), series);
}

__device__ double poisson_draw(double lam, uint32_t i, uint32_t k0, uint32_t k1) {
    if (!(lam > 0.0)) return 0.0;
    if (lam < 10.0) {
        const uint4 r = philox10(make_uint4(i, 0u, 0u, 0u), k0, k1);
        const double u = uniform53(r.x, r.y);
        double p = exp(-lam), F = p, k = 0.0;
        while (u > F && k < 1000.0) {
            k = __dadd_rn(k, 1.0);
            p = __ddiv_rn(__dmul_rn(p, lam), k);
            F = __dadd_rn(F, p);
        }
        return k;
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
    const double invalpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(b, 3.4)));
    const double vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(b, 2.0)));
    for (uint32_t t = 0; t < 64u; ++t) {   // a trial is accepted with probability > 0.9
        const uint4 r = philox10(make_uint4(i, t, 0u, 0u), k0, k1);
        const double U = __dsub_rn(uniform53(r.x, r.y), 0.5), V = uniform53(r.z, r.w);
        const double us = __dsub_rn(0.5, fabs(U));
        const double slope = __dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b);
        const double k = floor(__dadd_rn(__dadd_rn(__dmul_rn(slope, U), lam), 0.43));
        if (us >= 0.07 && V <= vr) return k;
        if (k < 0.0 || (us < 0.013 && V > us)) continue;
        const double lhs =
            __dsub_rn(__dadd_rn(log(V), log(invalpha)), log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
        const double rhs = __dsub_rn(__dadd_rn(-lam, __dmul_rn(k, loglam)), log_kfact(k));
        if (lhs <= rhs) return k;
    }
    return floor(lam);
}

__global__ void k_poisson_noise(const float* __restrict__ chat, int n, uint32_t k0, uint32_t k1,
                                float* __restrict__ c) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        c[i] = (float)poisson_draw((double)chat[i], (uint32_t)i, k0, k1);
}

}  // namespace

extern "C" osscir_status osscir_poisson_noise(const float* chat, int n, uint64_t seed, float* c, void* stream) {
    if (n < 0 || (n > 0 && (!chat || !c))) return OSSCIR_E_INVALID;
    if (n == 0) return OSSCIR_OK;
    // a grid-stride loop over at most 64 blocks per SM of the current device
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return OSSCIR_E_CUDA;
    const int threads = 256, need = (n + threads - 1) / threads, blocks = need < sms * 64 ? need : sms * 64;
    k_poisson_noise<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        chat, n, (uint32_t)seed, (uint32_t)(seed >> 32), c);
    return cudaGetLastError() == cudaSuccess ? OSSCIR_OK : OSSCIR_E_CUDA;
}
