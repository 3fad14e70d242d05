/* FP64 oracle of the seeded Poisson noise of simulated counts (the step before
 * the reconstruction: c ~ Poisson(c^(f_true)), Sec. 3 simulates noisy data this
 * way).  TEST INFRASTRUCTURE ONLY, like mocca_oracle.c; the GPU library has its
 * own implementation of the same definitions and shares no code with this one.
 *
 * Uniform numbers: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten
 * rounds of two 32x32 -> 64-bit multiplications (multipliers 0xD2511F53 and
 * 0xCD9E8D57) with the key bumped by the Weyl constants 0x9E3779B9 and
 * 0xBB67AE85 between rounds.  Sample s (s = 4 l + w for ray l and window w) takes
 * its t-th draw from counter (s, t, 0, 0) under key (seed mod 2^32, seed / 2^32);
 * two 32-bit words give one uniform in [0, 1) with 53 random bits.
 *
 * Poisson(lam): 0 for lam = 0; for lam < 10 inversion of the distribution
 * function with one uniform; for lam >= 10 the transformed rejection with squeeze
 * (PTRS) of Hormann ("The transformed rejection method for generating Poisson
 * random variables", 1993), two uniforms per trial, log k! from an exact
 * product for k <= 18 and the Stirling series of log Gamma beyond.  Every
 * decision is taken in FP64 with the operations in the order written here. */
#include <math.h>
#include <stdint.h>

static void philox_round(uint32_t x[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x[1] ^ k[0], y2 = hi0 ^ x[3] ^ k[1];
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(x, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = x[i];
}

static double u53(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* log k! */
static double log_factorial(double k) {
    if (k <= 18.0) {
        double p = 1.0;
        for (double i = 2.0; i <= k; i += 1.0) p = p * i;   /* exact: 18! < 2^53 */
        return log(p);
    }
    const double x = k + 1.0, ix = 1.0 / x, ix2 = ix * ix;
    const double series = ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0 - ix2 * (1.0 / 1680.0))));
    return (x - 0.5) * log(x) - x + 0.91893853320467274178 + series;   /* 0.5 log(2 pi) */
}

double orc_poisson_draw(double lam, uint32_t sample, const uint32_t key[2]) {
    if (!(lam > 0.0)) return 0.0;
    uint32_t ctr[4] = {sample, 0u, 0u, 0u}, r[4];
    if (lam < 10.0) {
        orc_philox4x32_10(ctr, key, r);
        const double u = u53(r[0], r[1]);
        double p = exp(-lam), F = p, k = 0.0;
        while (u > F && k < 1000.0) {
            k = k + 1.0;
            p = (p * lam) / k;
            F = F + p;
        }
        return k;
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t t = 0; t < 64u; ++t) {   /* a trial is accepted with probability > 0.9 */
        ctr[1] = t;
        orc_philox4x32_10(ctr, key, r);
        const double U = u53(r[0], r[1]) - 0.5, V = u53(r[2], r[3]);
        const double us = 0.5 - fabs(U);
        const double k = floor(((2.0 * a) / us + b) * U + lam + 0.43);
        if (us >= 0.07 && V <= vr) return k;
        if (k < 0.0 || (us < 0.013 && V > us)) continue;
        const double lhs = log(V) + log(invalpha) - log(a / (us * us) + b);
        const double rhs = -lam + k * loglam - log_factorial(k);
        if (lhs <= rhs) return k;
    }
    return floor(lam);
}

/* c[i] ~ Poisson(chat[i]) for i < n, sample i drawn with key (seed low, seed high). */
void orc_poisson_noise(int n, const double *chat, uint64_t seed, double *c) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) c[i] = orc_poisson_draw(chat[i], (uint32_t)i, key);
}
