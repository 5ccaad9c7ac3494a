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
__device__ __forceinline__ uint4 philox_round(uint4 c, unsigned k0, unsigned k1) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    return make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k0, (unsigned)p1, (unsigned)(p0 >> 32) ^ c.w ^ k1, (unsigned)p0);
}

__device__ __forceinline__ uint4 philox10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        c = philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the ten round keys precomputed: rk[r] = (k0_r, k1_r, k0_r+1, k1_r+1)
// for r = 0, 2, 4, 6, 8 (kept in shared memory by the fused kernel and read by broadcast).
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint4 *rk) {
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const uint4 k = rk[r];
        c = philox_round(c, k.x, k.y);
        c = philox_round(c, k.z, k.w);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_ctr(unsigned long long site, unsigned long long step) {
    return make_uint4((unsigned)site, (unsigned)(site >> 32), (unsigned)step, (unsigned)(step >> 32));
}

__device__ __forceinline__ uint4 philox_site(unsigned k0, unsigned k1, unsigned long long site,
                                             unsigned long long step) {
    return philox10(philox_ctr(site, step), k0, k1);
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

// The FP32 path evaluates the same formulas in FP32 with the hardware approximations:
// u_k = x_k 2^-32 + 2^-33 (one rounding), -2 ln u = -2 ln2 log2(u) kept above 1e-30 so
// that u rounded up to 1 gives a radius of ~0 rather than a NaN, sqrt(t) = t rsqrt(t), and
// the angles centred on (-pi, pi) where the sine and cosine approximations are accurate:
// cos 2pi u = -cos(2pi (u - 1/2)), sin 2pi u = -sin(2pi (u - 1/2)).
__device__ __forceinline__ void normals3(uint4 x, float &n0, float &n1, float &n2) {
    const float s = 2.3283064365386963e-10f, h = 1.1641532182693481e-10f;  // 2^-32, 2^-33
    const float u0 = fmaf((float)x.x, s, h), u1 = fmaf((float)x.y, s, h);
    const float u2 = fmaf((float)x.z, s, h), u3 = fmaf((float)x.w, s, h);
    const float m2ln2 = -1.3862943611198906f;  // -2 ln 2
    const float t1 = fmaxf(m2ln2 * __log2f(u0), 1e-30f), t2 = fmaxf(m2ln2 * __log2f(u2), 1e-30f);
    const float r1 = t1 * rsqrtf(t1), r2 = t2 * rsqrtf(t2);
    const float twopi = 6.2831853071795865f;
    float sn, cs;
    __sincosf(twopi * (u1 - 0.5f), &sn, &cs);
    n0 = -r1 * cs;
    n1 = -r1 * sn;
    n2 = -r2 * __cosf(twopi * (u3 - 0.5f));
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

// Exact magnetisation sums of the FP32 path: each spin component is rounded to a multiple
// of 2^-24 (FP32 resolution at 1) and summed as 64-bit integers, so the sum does not depend
// on the order in which CTAs add it.  The warp adds lanes that share a grain by shuffles,
// then one 64-bit atomic per component.
constexpr float FX_SCALE = 16777216.0f;  // 2^24

__device__ __forceinline__ void grain_accumulate_fx(unsigned long long *acc, int g, long long sx, long long sy,
                                                    long long sz, bool active) {
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
            atomicAdd(acc + 3 * k0 + 0, (unsigned long long)sx);
            atomicAdd(acc + 3 * k0 + 1, (unsigned long long)sy);
            atomicAdd(acc + 3 * k0 + 2, (unsigned long long)sz);
        }
    } else if (key >= 0) {
        atomicAdd(acc + 3 * key + 0, (unsigned long long)sx);
        atomicAdd(acc + 3 * key + 1, (unsigned long long)sy);
        atomicAdd(acc + 3 * key + 2, (unsigned long long)sz);
    }
}

}  // namespace hamr
