// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11) and the
// Box-Muller transform, on the device.  Counter layout used by the library:
//   MV charges:  (site, (nucleus*Ns + sheet)*2 + j, 1, 0),  j = 0, 1
//   kinematics:  (index in species, species, 2, 0)
//   Haar draws:  (index in species, species, 3, j),  j = 0..4
// key = (seed low word, seed high word).
#pragma once
#include <stdint.h>

namespace gl {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

__device__ __forceinline__ double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

__device__ __forceinline__ void box_muller(double u1, double u2, double& z0, double& z1) {
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(2.0 * 3.14159265358979323846 * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

}  // namespace gl
