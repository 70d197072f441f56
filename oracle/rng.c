/*
 * rng.c -- oracle random numbers, Halton jitter and step counts.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11, Sec. 4.  Each round takes the two 32x32->64 products of
 * the even counter words with the round multipliers, and builds the new counter
 * from the high halves xor'ed with the odd counter words and the round key,
 * and the low halves.  The key is bumped by the two Weyl constants (golden
 * ratio and sqrt(3)-1 in 32-bit fixed point) between rounds.
 * Pins: uniformity and independence statistics (tests/test_oracle_rng.py),
 * bijectivity in the counter for a fixed key on a sampled set.
 */
#include "oracle.h"
#include <math.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double oracle_u01(uint32_t w0, uint32_t w1) {
    /* 26 high bits of each word -> 52-bit integer k; (k + 0.5) 2^-52 is exact. */
    uint64_t k = ((uint64_t)(w0 >> 6) << 26) | (uint64_t)(w1 >> 6);
    return ((double)k + 0.5) * ldexp(1.0, -52);
}

void oracle_normals(uint64_t seed, uint32_t tag, uint32_t k, uint32_t j, int64_t D, double* out) {
    /* Box-Muller (Box & Muller 1958): r = sqrt(-2 log u1), angle 2 pi u2;
     * one Philox block gives u1, u2 and two normals, dims 2i and 2i+1. */
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; 2 * i < D; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, j, k, tag}, w[4];
        oracle_philox4x32_10(ctr, seed, w);
        double u1 = oracle_u01(w[0], w[1]);
        double u2 = oracle_u01(w[2], w[3]);
        double r = sqrt(-2.0 * log(u1));
        out[2 * i] = r * cos(two_pi * u2);
        if (2 * i + 1 < D) out[2 * i + 1] = r * sin(two_pi * u2);
    }
}

uint64_t oracle_resample_r64(uint64_t seed, uint32_t k) {
    uint32_t ctr[4] = {0u, 0u, k, (uint32_t)ORACLE_TAG_RESAMPLE}, w[4];
    oracle_philox4x32_10(ctr, seed, w);
    return ((uint64_t)w[0] << 32) | (uint64_t)w[1];
}

uint64_t oracle_multinomial_u64(uint64_t seed, uint32_t k, uint32_t i) {
    uint32_t ctr[4] = {1u, i, k, (uint32_t)ORACLE_TAG_RESAMPLE}, w[4];
    oracle_philox4x32_10(ctr, seed, w);
    return ((uint64_t)w[0] << 32) | (uint64_t)w[1];
}

double oracle_halton2(uint32_t n) {
    /* Radical inverse in base 2 (Halton 1960), digit by digit: the d-th binary
     * digit of n (least significant first) contributes digit * 2^-(d+1). */
    double h = 0.0, scale = 0.5;
    while (n != 0u) {
        if (n & 1u) h += scale;
        n >>= 1;
        scale *= 0.5;
    }
    return h;
}

int32_t oracle_step_count(double h, double L, double eps, int32_t max_steps) {
    /* Algorithm 2: leapfrog(theta, p, eps, ceil(l_m / eps)) with l_m = h_m L. */
    double l = h * L;
    double s = ceil(l / eps);
    if (!(s >= 1.0)) return 1;             /* also catches NaN */
    if (s >= (double)max_steps) return max_steps;
    return (int32_t)s;
}

/* ---------------------------------------------------------------- jitter */
#define ORACLE_MAX_PRIME_INDEX 65536
#define ORACLE_SIEVE_TOP 821642   /* the 65536th prime is 821641 */

int64_t oracle_nth_prime(int64_t m) {
    static int32_t* table = 0;
    if (m < 1 || m > ORACLE_MAX_PRIME_INDEX) return 0;
    /* the table is built once, on first use (under a lock when OpenMP threads
     * may call in together) */
#pragma omp critical(oracle_prime_table)
    if (!table) {
        /* sieve of Eratosthenes up to ORACLE_SIEVE_TOP */
        unsigned char* comp = (unsigned char*)calloc(ORACLE_SIEVE_TOP + 1, 1);
        int32_t* t = (int32_t*)malloc(sizeof(int32_t) * ORACLE_MAX_PRIME_INDEX);
        int64_t cnt = 0;
        for (int64_t p = 2; p <= ORACLE_SIEVE_TOP && cnt < ORACLE_MAX_PRIME_INDEX; ++p) {
            if (comp[p]) continue;
            t[cnt++] = (int32_t)p;
            for (int64_t q = p * p; q <= ORACLE_SIEVE_TOP; q += p) comp[q] = 1;
        }
        free(comp);
        table = t;
    }
    return table[m - 1];
}

double oracle_radical_inverse(uint64_t n, uint64_t b) {
    uint64_t num = 0, den = 1;
    while (n != 0) {
        num = num * b + n % b;   /* next digit, least significant first */
        den *= b;
        n /= b;
    }
    return (double)num / (double)den;
}

uint32_t oracle_shuffle_index(uint64_t seed, uint32_t k, uint32_t j, uint32_t J) {
    int m = 2;
    while ((1ull << m) < (uint64_t)J) m += 2;
    const int half = m / 2;
    const uint32_t mask = (1u << half) - 1u;
    uint32_t v = j;
    for (;;) {
        uint32_t L = v >> half, R = v & mask;
        for (uint32_t r = 0; r < 4; ++r) {
            uint32_t ctr[4] = {R, r, k, (uint32_t)ORACLE_TAG_SHUFFLE}, w[4];
            oracle_philox4x32_10(ctr, seed, w);
            const uint32_t t = L ^ (w[0] & mask);
            L = R;
            R = t;
        }
        v = (L << half) | R;
        if (v < J) return v;
    }
}

static double frac_pos(double x) { return x - floor(x); }

double oracle_jitter(int32_t scheme, uint64_t seed, int64_t j, int64_t k, int64_t J, int64_t K) {
    if (scheme >= 3 && scheme <= 6) k = (k - 1) % K + 1;   /* dimensions reused past K */
    switch (scheme) {
        case 0: return 1.0;
        case 1: return oracle_halton2((uint32_t)(j * K + k));
        case 2: {
            uint32_t ctr[4] = {0u, (uint32_t)j, (uint32_t)k, (uint32_t)ORACLE_TAG_JITTER}, w[4];
            oracle_philox4x32_10(ctr, seed, w);
            return oracle_u01(w[0], w[1]);
        }
        case 3: return oracle_radical_inverse((uint64_t)(j + 1), (uint64_t)oracle_nth_prime(k));
        case 4: return oracle_radical_inverse((uint64_t)(j + 1), (uint64_t)oracle_nth_prime(K + 1 - k));
        case 5: return frac_pos((double)(j + 1) * sqrt((double)oracle_nth_prime(k)));
        case 6: return frac_pos((double)(j + 1) * sqrt((double)oracle_nth_prime(K + 1 - k)));
        case 7: {
            const double g = (sqrt(5.0) - 1.0) * 0.5;
            return frac_pos((double)(j * K + k) * g);
        }
        case 8:
        case 9: {
            double h = (double)(oracle_shuffle_index(seed, (uint32_t)k, (uint32_t)j, (uint32_t)J) + 1) / (double)J;
            if (scheme == 9) {
                uint32_t ctr[4] = {1u, (uint32_t)j, (uint32_t)k, (uint32_t)ORACLE_TAG_JITTER}, w[4];
                oracle_philox4x32_10(ctr, seed, w);
                h += 0.1 * oracle_u01(w[0], w[1]);
            }
            return h;
        }
        case 10: {
            const uint32_t n = (uint32_t)(j * K + k);
            return oracle_halton2(n ^ (n >> 1));
        }
        /* 1-d Halton with the J x K matrix read iteration-major: iteration k
         * takes the J consecutive indices (k - 1) J + 1 .. k J (Sec. 3.2) */
        case 11: return oracle_halton2((uint32_t)((k - 1) * J + j + 1));
        default: return 1.0;
    }
}
