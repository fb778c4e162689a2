/*
 * Counter-based RNG for the oracle (test infrastructure; see oracle.h):
 * Philox4x32 with 10 rounds, written from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11), and the Box-Muller transform (Box & Muller 1958).
 */
#include <math.h>
#include "oracle_internal.h"

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

void box_muller(double u1, double u2, double* z0, double* z1) {
    double rad = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    *z0 = rad * cos(th);
    *z1 = rad * sin(th);
}
