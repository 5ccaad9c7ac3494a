// Device helpers shared by the step kernels: the counter-based thermal normals and the
// time-dependent drivers (laser temperature, write-field polarity).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hamr_internal.h"

namespace hamr {

// Philox4x32-10, from the generator's published definition (Salmon, Moraes, Dror, Shaw,
// SC'11): per round, 32x32->64-bit products of counter words 0 and 2 with 0xD2511F53 and
// 0xCD9E8D57; the new words are (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key advances
// by (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 philox_site(unsigned k0, unsigned k1, unsigned long long site,
                                             unsigned long long step) {
    return philox10(make_uint4((unsigned)site, (unsigned)(site >> 32), (unsigned)step,
                               (unsigned)(step >> 32)),
                    k0, k1);
}

// Box-Muller on u_k = (x_k + 1/2) 2^-32: (r1 cos 2pi u1, r1 sin 2pi u1, r2 cos 2pi u3),
// r1 = sqrt(-2 ln u0), r2 = sqrt(-2 ln u2).
__device__ __forceinline__ void normals3(uint4 x, double &n0, double &n1, double &n2) {
    const double s = 2.3283064365386963e-10;  // 2^-32
    const double u0 = ((double)x.x + 0.5) * s, u1 = ((double)x.y + 0.5) * s;
    const double u2 = ((double)x.z + 0.5) * s, u3 = ((double)x.w + 0.5) * s;
    const double r1 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    n0 = r1 * cs;
    n1 = r1 * sn;
    n2 = r2 * cospi(2.0 * u3);
}

__device__ __forceinline__ void normals3(uint4 x, float &n0, float &n1, float &n2) {
    const float s = 2.3283064365386963e-10f;  // 2^-32
    const float u0 = fmaf((float)x.x, s, 0.5f * s), u1 = fmaf((float)x.y, s, 0.5f * s);
    const float u2 = fmaf((float)x.z, s, 0.5f * s), u3 = fmaf((float)x.w, s, 0.5f * s);
    const float r1 = sqrtf(-2.0f * logf(u0)), r2 = sqrtf(-2.0f * logf(u2));
    float sn, cs;
    sincospif(2.0f * u1, &sn, &cs);
    n0 = r1 * cs;
    n1 = r1 * sn;
    n2 = r2 * cospif(2.0f * u3);
}

// Write-field polarity s(t): linear ramp from bit b-1 to bit b over the first ramp_len of
// bit b, end bits held outside the pattern; 1 when there is no pattern.
template <typename Real>
__device__ __forceinline__ Real bit_pol(const uint8_t *bits, int n, long long b) {
    b = b < 0 ? 0 : (b > n - 1 ? n - 1 : b);
    return bits[b] ? Real(-1) : Real(1);
}

__device__ __forceinline__ double field_polarity(const ReplicaDev &R, const uint8_t *bits, double t) {
    if (R.n_bits <= 0) return 1.0;
    const uint8_t *b = bits + R.bits_off;
    const double xh = R.head_x0 + R.head_v * t;
    const double fb = floor(xh / R.bit_len);
    const long long bi = (long long)fb;
    const double into = xh - fb * R.bit_len;
    const double prev = bit_pol<double>(b, R.n_bits, bi - 1), cur = bit_pol<double>(b, R.n_bits, bi);
    double w = R.ramp_len > 0.0 ? into / R.ramp_len : 1.0;
    w = fmin(fmax(w, 0.0), 1.0);
    return prev + (cur - prev) * w;
}

__device__ __forceinline__ float field_polarity_f(const ReplicaDev &R, const uint8_t *bits, float t) {
    if (R.n_bits <= 0) return 1.0f;
    const uint8_t *b = bits + R.bits_off;
    const float xh = fmaf(R.fhead_v, t, R.fhead_x0);
    const float fb = floorf(xh / R.fbit_len);
    const long long bi = (long long)fb;
    const float into = xh - fb * R.fbit_len;
    const float prev = bit_pol<float>(b, R.n_bits, bi - 1), cur = bit_pol<float>(b, R.n_bits, bi);
    float w = R.framp_len > 0.0f ? into / R.framp_len : 1.0f;
    w = fminf(fmaxf(w, 0.0f), 1.0f);
    return prev + (cur - prev) * w;
}

__device__ __forceinline__ double temperature(const ReplicaDev &R, double x, double y, double t) {
    if (R.c_fwhm == 0.0) return R.T_amb;
    const double dx = x - R.x0 - R.vx * t, dy = y - R.y0 - R.vy * t;
    return R.T_amb + R.dT * exp(R.c_fwhm * (dx * dx + dy * dy));
}

__device__ __forceinline__ float temperature_f(const ReplicaDev &R, float x, float y, float t) {
    if (R.fc_fwhm == 0.0f) return R.fT_amb;
    const float dx = x - fmaf(R.fvx, t, R.fx0), dy = y - fmaf(R.fvy, t, R.fy0);
    return fmaf(R.fdT, __expf(R.fc_fwhm * (dx * dx + dy * dy)), R.fT_amb);
}

// Sum of (x, y, z) over the lanes of a warp that all hold the same grain, else per lane;
// then one FP64 atomic per component.
__device__ __forceinline__ void grain_accumulate(double *acc, int g, double sx, double sy, double sz,
                                                 bool active) {
    const unsigned full = 0xffffffffu;
    const int key = active ? g : -1;
    const int k0 = __shfl_sync(full, key, 0);
    if (__all_sync(full, key == k0)) {
        if (k0 < 0) return;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(full, sx, o);
            sy += __shfl_xor_sync(full, sy, o);
            sz += __shfl_xor_sync(full, sz, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(acc + 3 * k0 + 0, sx);
            atomicAdd(acc + 3 * k0 + 1, sy);
            atomicAdd(acc + 3 * k0 + 2, sz);
        }
    } else if (key >= 0) {
        atomicAdd(acc + 3 * key + 0, sx);
        atomicAdd(acc + 3 * key + 1, sy);
        atomicAdd(acc + 3 * key + 2, sz);
    }
}

}  // namespace hamr
