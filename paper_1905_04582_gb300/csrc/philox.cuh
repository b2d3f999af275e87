// Counter-based random numbers of the device samplers: Philox4x32-10
// (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
// 3", SC'11) and the Box-Muller transform.  Shared by the HMC kernels
// (reduce_kernel.cu) and the random-walk sampler (rwmh.cu).
#pragma once

#include <cmath>
#include <cstdint>

namespace mds {
namespace {

__device__ __forceinline__ void philox_round(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key schedule.
__device__ __forceinline__ void philox10(uint32_t (&c)[4], uint64_t key) {
    uint32_t k0 = static_cast<uint32_t>(key), k1 = static_cast<uint32_t>(key >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
}

__device__ __forceinline__ double open_unit(uint32_t b) { return (static_cast<double>(b) + 0.5) * (1.0 / 4294967296.0); }

// Box-Muller pair from two 32-bit words, u = (b + 1/2) / 2^32.
__device__ __forceinline__ void box_muller(uint32_t b1, uint32_t b2, double &z0, double &z1) {
    const double u1 = open_unit(b1), u2 = open_unit(b2);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    z0 = rad * cs;
    z1 = rad * sn;
}

// FP32 version: -log(u1) through log1p for u1 >= 1/2 (1 - u1 exact from the
// integer), so the radius keeps full relative precision near u1 = 1.
__device__ __forceinline__ void box_muller(uint32_t b1, uint32_t b2, float &z0, float &z1) {
    float nl;
    if (b1 < 0x80000000u)
        nl = -logf((static_cast<float>(b1) + 0.5f) * 2.3283064365386963e-10f);
    else
        nl = -log1pf(-(static_cast<float>(0xFFFFFFFFu - b1) + 0.5f) * 2.3283064365386963e-10f);
    const float rad = sqrtf(2.0f * nl);
    float sn, cs;
    sincospif(2.0f * ((static_cast<float>(b2) + 0.5f) * 2.3283064365386963e-10f), &sn, &cs);
    z0 = rad * cs;
    z1 = rad * sn;
}

}  // namespace
}  // namespace mds
