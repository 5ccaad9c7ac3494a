// The multiscale write window (Sec. II, Fig. 1): a simple-cubic atomistic window embedded in
// a micromagnetic finite-difference track, exchange coupled across the interface and moving
// with the laser spot.  FP64 throughout; one thread per atomistic site or per cell.
//
// Per coupled step n -> n+1 (drivers frozen at t_n):
//   1. k_ms_average   - Eq. 6: every window cell takes the direction of the sum of its sites;
//   2. k_ms_predict,  - the sLLG Heun step of the window (Eq. 1-3); across the window's x
//      k_ms_correct     faces a bond sees the direction of the micromagnetic cell there;
//   3. k_mm_prep,     - one classical RK4 step of the micromagnetic LLG (Eq. 1 without the
//      k_mm_stage x4,   thermal field; Eq. 4 on a 6-point Laplacian, Eq. 5) on the cells
//      k_mm_final       outside the window, with Ms = Ms0 m_e, A = A0 m_e^2, K = K0 m_e^3,
//                       alpha = lambda (1 - T / 3 T_C) and m_e(T) the root of the Langevin
//                       equation (Sec. II); window cells stay at their Eq. 6 directions;
//   4. window moves   - k_ms_average of the trailing column, k_ms_shift of the sites by one
//                       cell column, k_ms_thermalise of the new leading column in the cone
//                       of half-angle theta_max(m_e) (Sec. II).
// Device layout: cell and site arrays are component planes [3][n]; cell q = cx + ncx (cy +
// ncy cz); window site s = i + nxw (j + nyw k) with i along the track.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <utility>
#include <vector>

#include "device_common.cuh"

using namespace hamr;

namespace {

struct MsDev {
    int ncx, ncy, ncz, r, wx;
    int nxw, nyw, nzw;
    long long nc, nw;
    double cell, a;
    double J, mu_s, ku;        // atomistic exchange [J], moment [J/T], anisotropy [J]
    double Ms0, A0, K0;        // micromagnetic constants at 0 K
    double lambda, T_C, gamma, dt;
    double sig0;               // sqrt(2 lambda kB / (gamma mu_s dt)): sigma_i = sig0 sqrt(T_i)
    unsigned key0, key1;       // Philox key = seed (low, high)
};

__device__ __forceinline__ double3 rhs(double gamma, double alpha, double sx, double sy, double sz, double bx,
                                       double by, double bz) {
    // -gamma/(1+alpha^2) [S x B + alpha S x (S x B)]
    const double cx = sy * bz - sz * by, cy = sz * bx - sx * bz, cz = sx * by - sy * bx;
    const double dx = sy * cz - sz * cy, dy = sz * cx - sx * cz, dz = sx * cy - sy * cx;
    const double pref = -gamma / (1.0 + alpha * alpha);
    return make_double3(pref * (cx + alpha * dx), pref * (cy + alpha * dy), pref * (cz + alpha * dz));
}

__device__ __forceinline__ double langevin(double x) {
    if (fabs(x) < 1e-3) return x / 3.0 - x * x * x / 45.0 + 2.0 * x * x * x * x * x / 945.0;
    return 1.0 / tanh(x) - 1.0 / x;
}

__device__ __forceinline__ double langevin_d(double x) {
    if (fabs(x) < 1e-3) return 1.0 / 3.0 - x * x / 15.0 + 2.0 * x * x * x * x / 189.0;
    const double s = sinh(x);
    return 1.0 / (x * x) - 1.0 / (s * s);
}

// m_e(T): the largest root in [0, 1] of m = L(3 T_C m / T + mu_s B / (kB T)).  Newton steps
// from m = 1 kept inside a bracket [lo, hi] with L(.) - m >= 0 at lo and < 0 at hi; a step
// that leaves the bracket is replaced by bisection.
__device__ double me_root(double T_C, double T, double mu_s, double B) {
    if (!(T > 0.0)) return 1.0;
    const double a = 3.0 * T_C / T, b = mu_s * B / (KB * T);
    double lo = 0.0, hi = 1.0, m = 1.0;
    for (int it = 0; it < 200; ++it) {
        const double g = langevin(a * m + b) - m;
        if (g >= 0.0)
            lo = m;
        else
            hi = m;
        const double gp = a * langevin_d(a * m + b) - 1.0;
        double mn = m - g / gp;
        if (!(mn > lo && mn < hi)) mn = 0.5 * (lo + hi);
        if (fabs(mn - m) <= 2e-16 * m || hi - lo <= 2e-16) {
            m = mn;
            break;
        }
        m = mn;
    }
    return m;
}

__device__ __forceinline__ double theta_max(double mr) {
    double x = 1.0 + 6.0 * (mr - 1.0) / 5.0;
    x = fmin(fmax(x, 0.0), 1.0);
    return (5.0 * M_PI / 9.0) * sqrt(1.0 - sqrt(x));
}

__device__ __forceinline__ double3 applied_field(const ReplicaDev &D, const uint8_t *bits, double t) {
    const double s = D.B0 * field_polarity(D, bits, t);
    return make_double3(s * D.dir[0], s * D.dir[1], s * D.dir[2]);
}

__device__ __forceinline__ long long cell_at(const MsDev &P, long long cx, long long cy, long long cz) {
    return cx + (long long)P.ncx * (cy + (long long)P.ncy * cz);
}

// Eq. 6 for the cells of columns [cx0, cx0 + ncol): direction of the sum of their sites.
__global__ void k_ms_average(double *m, const double *S, const int *grain, MsDev P, int ox, int cx0, int ncol) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)ncol * P.ncy * P.ncz;
    if (idx >= n) return;
    const int cx = cx0 + (int)(idx % ncol), cy = (int)((idx / ncol) % P.ncy), cz = (int)(idx / ((long long)ncol * P.ncy));
    const long long q = cell_at(P, cx, cy, cz);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    if (grain[q] >= 0)
        for (int dk = 0; dk < P.r; ++dk)
            for (int dj = 0; dj < P.r; ++dj)
                for (int di = 0; di < P.r; ++di) {
                    const long long i = (long long)(cx - ox) * P.r + di, j = (long long)cy * P.r + dj,
                                    k = (long long)cz * P.r + dk;
                    const long long s = i + P.nxw * (j + (long long)P.nyw * k);
                    sx += S[s];
                    sy += S[P.nw + s];
                    sz += S[2 * P.nw + s];
                }
    const double nn = sqrt(sx * sx + sy * sy + sz * sz);
    m[q] = nn > 0.0 ? sx / nn : 0.0;
    m[P.nc + q] = nn > 0.0 ? sy / nn : 0.0;
    m[2 * P.nc + q] = nn > 0.0 ? sz / nn : 0.0;
}

// Exchange sum sum_j J v_j of window site (i, j, k) of grain g over its same-grain bonds: the
// window spins V inside, the cells m across the window's x faces.
__device__ __forceinline__ double3 exchange(const MsDev &P, const double *V, const double *m, const int *grain,
                                            int ox, int i, int j, int k, int g) {
    double ex = 0.0, ey = 0.0, ez = 0.0;
    const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int ii = i + off[b][0], jj = j + off[b][1], kk = k + off[b][2];
        if (jj < 0 || jj >= P.nyw || kk < 0 || kk >= P.nzw) continue;
        double vx, vy, vz;
        if (ii >= 0 && ii < P.nxw) {
            if (grain[cell_at(P, ox + ii / P.r, jj / P.r, kk / P.r)] != g) continue;
            const long long s = ii + P.nxw * (jj + (long long)P.nyw * kk);
            vx = V[s];
            vy = V[P.nw + s];
            vz = V[2 * P.nw + s];
        } else {
            const long long cx = ox + (ii < 0 ? -1 : P.wx);
            if (cx < 0 || cx >= P.ncx) continue;
            const long long q = cell_at(P, cx, jj / P.r, kk / P.r);
            if (grain[q] != g) continue;
            vx = m[q];
            vy = m[P.nc + q];
            vz = m[2 * P.nc + q];
        }
        ex += P.J * vx;
        ey += P.J * vy;
        ez += P.J * vz;
    }
    return make_double3(ex, ey, ez);
}

__global__ void k_ms_predict(const double *S, double *Sp, double *F1, double *BTH, const double *m, const int *grain,
                             MsDev P, ReplicaDev D, const uint8_t *bits, int ox, long long step) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= P.nw) return;
    const int i = (int)(s % P.nxw), j = (int)((s / P.nxw) % P.nyw), k = (int)(s / ((long long)P.nxw * P.nyw));
    const int g = grain[cell_at(P, ox + i / P.r, j / P.r, k / P.r)];
    if (g < 0) {
        Sp[s] = Sp[P.nw + s] = Sp[2 * P.nw + s] = 0.0;
        return;
    }
    const double t = (double)step * P.dt;
    const double T = temperature(D, ((double)ox * P.r + i + 0.5) * P.a, (j + 0.5) * P.a, t);
    const double sig = P.sig0 * sqrt(T);
    const unsigned long long X = (unsigned long long)ox * P.r + i, NX = (unsigned long long)P.ncx * P.r;
    const unsigned long long site = X + NX * ((unsigned long long)j + (unsigned long long)P.nyw * k);
    double n0, n1, n2;
    normals3(philox_site(P.key0, P.key1, site, (unsigned long long)step), n0, n1, n2);
    const double bthx = sig * n0, bthy = sig * n1, bthz = sig * n2;
    BTH[s] = bthx;
    BTH[P.nw + s] = bthy;
    BTH[2 * P.nw + s] = bthz;
    const double3 ba = applied_field(D, bits, t);
    const double3 ex = exchange(P, S, m, grain, ox, i, j, k, g);
    const double sx = S[s], sy = S[P.nw + s], sz = S[2 * P.nw + s];
    const double3 f = rhs(P.gamma, P.lambda, sx, sy, sz, ex.x / P.mu_s + ba.x + bthx, ex.y / P.mu_s + ba.y + bthy,
                          ex.z / P.mu_s + 2.0 * P.ku / P.mu_s * sz + ba.z + bthz);
    F1[s] = f.x;
    F1[P.nw + s] = f.y;
    F1[2 * P.nw + s] = f.z;
    const double vx = sx + P.dt * f.x, vy = sy + P.dt * f.y, vz = sz + P.dt * f.z;
    const double nv = sqrt(vx * vx + vy * vy + vz * vz);
    Sp[s] = vx / nv;
    Sp[P.nw + s] = vy / nv;
    Sp[2 * P.nw + s] = vz / nv;
}

__global__ void k_ms_correct(double *S, const double *Sp, const double *F1, const double *BTH, const double *m,
                             const int *grain, MsDev P, ReplicaDev D, const uint8_t *bits, int ox, long long step) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= P.nw) return;
    const int i = (int)(s % P.nxw), j = (int)((s / P.nxw) % P.nyw), k = (int)(s / ((long long)P.nxw * P.nyw));
    const int g = grain[cell_at(P, ox + i / P.r, j / P.r, k / P.r)];
    if (g < 0) return;
    const double t = (double)step * P.dt;
    const double3 ba = applied_field(D, bits, t);
    const double3 ex = exchange(P, Sp, m, grain, ox, i, j, k, g);
    const double px = Sp[s], py = Sp[P.nw + s], pz = Sp[2 * P.nw + s];
    const double3 f = rhs(P.gamma, P.lambda, px, py, pz, ex.x / P.mu_s + ba.x + BTH[s],
                          ex.y / P.mu_s + ba.y + BTH[P.nw + s],
                          ex.z / P.mu_s + 2.0 * P.ku / P.mu_s * pz + ba.z + BTH[2 * P.nw + s]);
    const double vx = S[s] + 0.5 * P.dt * (F1[s] + f.x), vy = S[P.nw + s] + 0.5 * P.dt * (F1[P.nw + s] + f.y),
                 vz = S[2 * P.nw + s] + 0.5 * P.dt * (F1[2 * P.nw + s] + f.z);
    const double nv = sqrt(vx * vx + vy * vy + vz * vz);
    S[s] = vx / nv;
    S[P.nw + s] = vy / nv;
    S[2 * P.nw + s] = vz / nv;
}

__device__ __forceinline__ bool evolved(const MsDev &P, const int *grain, long long q, int ox) {
    const int cx = (int)(q % P.ncx);
    return grain[q] >= 0 && (cx < ox || cx >= ox + P.wx);
}

// Per cell at t_n: the laser temperature at the cell centre and m_e(T, |B_app|).
__global__ void k_mm_prep(double *me, double *Tq, MsDev P, ReplicaDev D, double t, double Bm) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= P.nc) return;
    const long long cx = q % P.ncx, cy = (q / P.ncx) % P.ncy;
    const double T = temperature(D, (cx + 0.5) * P.cell, (cy + 0.5) * P.cell, t);
    Tq[q] = T;
    me[q] = me_root(P.T_C, T, P.mu_s, Bm);
}

// One RK4 stage on the evolved cells: K = dm/dt at the stage values Vin, acc += w K and
// Vout = m + c dt K (the next stage's values).  Cells that are not evolved keep m in both
// stage buffers.
__global__ void k_mm_stage(const double *Vin, double *Vout, double *acc, const double *m, const double *me,
                           const double *Tq, const int *grain, MsDev P, int ox, double bx, double by, double bz,
                           double c, double w, int first) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= P.nc || !evolved(P, grain, q, ox)) return;
    const long long cx = q % P.ncx, cy = (q / P.ncx) % P.ncy, cz = q / ((long long)P.ncx * P.ncy);
    const double vx = Vin[q], vy = Vin[P.nc + q], vz = Vin[2 * P.nc + q];
    double lx = 0.0, ly = 0.0, lz = 0.0;
    const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    const double c2 = P.cell * P.cell;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const long long x = cx + off[b][0], y = cy + off[b][1], z = cz + off[b][2];
        if (x < 0 || x >= P.ncx || y < 0 || y >= P.ncy || z < 0 || z >= P.ncz) continue;
        const long long qn = cell_at(P, x, y, z);
        if (grain[qn] != grain[q]) continue;
        lx += (Vin[qn] - vx) / c2;
        ly += (Vin[P.nc + qn] - vy) / c2;
        lz += (Vin[2 * P.nc + qn] - vz) / c2;
    }
    const double e = me[q];
    double cex = 2.0 * P.A0 * e * e / (P.Ms0 * e), cK = 2.0 * P.K0 * e * e * e / (P.Ms0 * e);
    if (!(e > 0.0)) cex = cK = 0.0;
    const double T = fmax(fmin(Tq[q], P.T_C), 0.0);
    const double alpha = P.lambda * (1.0 - T / (3.0 * P.T_C));
    const double3 k = rhs(P.gamma, alpha, vx, vy, vz, cex * lx + bx, cex * ly + by, cex * lz + cK * vz + bz);
    const double a0 = first ? 0.0 : acc[q], a1 = first ? 0.0 : acc[P.nc + q], a2 = first ? 0.0 : acc[2 * P.nc + q];
    acc[q] = a0 + w * k.x;
    acc[P.nc + q] = a1 + w * k.y;
    acc[2 * P.nc + q] = a2 + w * k.z;
    Vout[q] = m[q] + c * P.dt * k.x;
    Vout[P.nc + q] = m[P.nc + q] + c * P.dt * k.y;
    Vout[2 * P.nc + q] = m[2 * P.nc + q] + c * P.dt * k.z;
}

__global__ void k_mm_final(double *m, const double *acc, const int *grain, MsDev P, int ox) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= P.nc || !evolved(P, grain, q, ox)) return;
    const double vx = m[q] + P.dt / 6.0 * acc[q], vy = m[P.nc + q] + P.dt / 6.0 * acc[P.nc + q],
                 vz = m[2 * P.nc + q] + P.dt / 6.0 * acc[2 * P.nc + q];
    const double nv = sqrt(vx * vx + vy * vy + vz * vz);
    m[q] = vx / nv;
    m[P.nc + q] = vy / nv;
    m[2 * P.nc + q] = vz / nv;
}

// Sites move back by one cell column (the last column is thermalised afterwards).
__global__ void k_ms_shift(double *Snew, const double *Sold, MsDev P) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= P.nw) return;
    const int i = (int)(s % P.nxw);
    for (int d = 0; d < 3; ++d) Snew[d * P.nw + s] = i + P.r < P.nxw ? Sold[d * P.nw + s + P.r] : 0.0;
}

// Thermalisation of the sites of cell columns [cx0, cx1): a spin in the cone of half-angle
// theta_max(m_e(T_cell, |B_app|)) around the cell's m, polar angle u0 theta_max and azimuth
// 2 pi u1 from e1 = (z x m)/|z x m| (or (x x m)/|x x m| when |m_z| >= 0.9), e2 = m x e1, with
// u0, u1 from Philox4x32-10 (key = seed, counter = (site low, site high, event low,
// event high | 2^31)).
__global__ void k_ms_thermalise(double *S, const double *m, const int *grain, MsDev P, ReplicaDev D, int ox, int cx0,
                                int cx1, double t, double Bm, unsigned long long event) {
    const long long ncolsites = (long long)(cx1 - cx0) * P.r;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= ncolsites * P.nyw * P.nzw) return;
    const int i = (cx0 - ox) * P.r + (int)(idx % ncolsites);
    const int j = (int)((idx / ncolsites) % P.nyw), k = (int)(idx / (ncolsites * P.nyw));
    const long long s = i + P.nxw * (j + (long long)P.nyw * k);
    const long long q = cell_at(P, ox + i / P.r, j / P.r, k / P.r);
    const double mx = m[q], my = m[P.nc + q], mz = m[2 * P.nc + q];
    if (grain[q] < 0 || (mx == 0.0 && my == 0.0 && mz == 0.0)) {
        S[s] = S[P.nw + s] = S[2 * P.nw + s] = 0.0;
        return;
    }
    const long long cx = q % P.ncx, cy = (q / P.ncx) % P.ncy;
    const double T = temperature(D, (cx + 0.5) * P.cell, (cy + 0.5) * P.cell, t);
    const double thm = theta_max(me_root(P.T_C, T, P.mu_s, Bm));
    const unsigned long long X = (unsigned long long)ox * P.r + i, NX = (unsigned long long)P.ncx * P.r;
    const unsigned long long site = X + NX * ((unsigned long long)j + (unsigned long long)P.nyw * k);
    const uint4 x = philox10(make_uint4((unsigned)site, (unsigned)(site >> 32), (unsigned)event,
                                        (unsigned)(event >> 32) | 0x80000000u),
                             P.key0, P.key1);
    const double u0 = ((double)x.x + 0.5) * 2.3283064365386963e-10, u1 = ((double)x.y + 0.5) * 2.3283064365386963e-10;
    const double th = u0 * thm, ph = 2.0 * M_PI * u1;
    double e1x, e1y, e1z;
    if (fabs(mz) < 0.9) {
        e1x = -my; e1y = mx; e1z = 0.0;
    } else {
        e1x = 0.0; e1y = -mz; e1z = my;
    }
    const double r = sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
    e1x /= r; e1y /= r; e1z /= r;
    const double e2x = my * e1z - mz * e1y, e2y = mz * e1x - mx * e1z, e2z = mx * e1y - my * e1x;
    const double a1 = sin(th) * cos(ph), a2 = sin(th) * sin(ph), a3 = cos(th);
    S[s] = a1 * e1x + a2 * e2x + a3 * mx;
    S[P.nw + s] = a1 * e1y + a2 * e2y + a3 * my;
    S[2 * P.nw + s] = a1 * e1z + a2 * e2z + a3 * mz;
}

// AoS (host layout) <-> component planes
__global__ void k_aos_to_planes(const double *src, double *dst, long long n) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int d = 0; d < 3; ++d) dst[d * n + s] = src[3 * s + d];
}

__global__ void k_planes_to_aos(const double *src, double *dst, long long n) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int d = 0; d < 3; ++d) dst[3 * s + d] = src[d * n + s];
}

// Zero the cells that are non-magnetic.
__global__ void k_zero_void_cells(double *m, const int *grain, long long nc) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nc || grain[q] >= 0) return;
    m[q] = m[nc + q] = m[2 * nc + q] = 0.0;
}

constexpr int BLK = 256;
inline unsigned nblk(long long n) { return (unsigned)((n + BLK - 1) / BLK); }

}  // namespace

struct hamr_ms_ctx {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    MsDev P{};
    ReplicaDev D{};               // laser spot and write field (the atomistic driver fields)
    std::vector<uint8_t> bits_h;
    uint8_t *bits_d = nullptr;
    int *grain_d = nullptr;
    std::vector<int> grain_h;
    double *m = nullptr, *V0 = nullptr, *V1 = nullptr, *acc = nullptr, *me = nullptr, *Tq = nullptr;
    double *S = nullptr, *S2 = nullptr, *Sp = nullptr, *F1 = nullptr, *BTH = nullptr;
    double *stage = nullptr;      // AoS staging for host copies
    int ox = -1;                  // window column (-1: not placed)
    long long step = 0;
    long long events = 0;         // thermalisation events so far
    bool grains_set = false, cells_set = false;
};

namespace {

thread_local std::string g_ms_create_err = "no error";

int msfail(hamr_ms_t h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_ms_create_err = buf;
    return code;
}

#define MSCK(h, call)                                                                                          \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess)                                                                                 \
            return msfail(h, e_ == cudaErrorMemoryAllocation ? HAMR_ERR_OOM : HAMR_ERR_CUDA, "%s: %s (%s:%d)", \
                          #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                  \
    } while (0)

struct MsDeviceGuard {
    int prev = -1;
    explicit MsDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~MsDeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

void ms_free(hamr_ms_t h) {
    double **bufs[] = {&h->m, &h->V0, &h->V1, &h->acc, &h->me, &h->Tq, &h->S, &h->S2, &h->Sp, &h->F1, &h->BTH, &h->stage};
    for (double **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    if (h->grain_d) cudaFree(h->grain_d);
    if (h->bits_d) cudaFree(h->bits_d);
    h->grain_d = nullptr;
    h->bits_d = nullptr;
}

// B_app(t) = B0 s(t) dir, with the polarity s(t) of the bit pattern computed as on the device
void applied_host(const hamr_ms_t h, double t, double B[3]) {
    const ReplicaDev &D = h->D;
    double s = 1.0;
    if (D.n_bits > 0) {
        const double xh = D.head_x0 + D.head_v * t;
        const double fb = floor(xh / D.bit_len);
        const long long b = (long long)fb;
        const double into = xh - fb * D.bit_len;
        auto pol = [&](long long bi) {
            bi = bi < 0 ? 0 : (bi > D.n_bits - 1 ? D.n_bits - 1 : bi);
            return h->bits_h[bi] ? -1.0 : 1.0;
        };
        double w = D.ramp_len > 0.0 ? into / D.ramp_len : 1.0;
        w = fmin(fmax(w, 0.0), 1.0);
        s = pol(b - 1) + (pol(b) - pol(b - 1)) * w;
    }
    for (int d = 0; d < 3; ++d) B[d] = D.B0 * s * D.dir[d];
}

// |B_app(t)|, the field in the Langevin equation for m_e
double field_magnitude_host(const hamr_ms_t h, double t) {
    double B[3];
    applied_host(h, t, B);
    return sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
}

int ms_thermalise(hamr_ms_t h, int cx0, int cx1, double t) {
    const long long n = (long long)(cx1 - cx0) * h->P.r * h->P.nyw * h->P.nzw;
    if (n <= 0) return HAMR_OK;
    k_ms_thermalise<<<nblk(n), BLK, 0, h->stream>>>(h->S, h->m, h->grain_d, h->P, h->D, h->ox, cx0, cx1, t,
                                                    field_magnitude_host(h, t), (unsigned long long)h->events);
    MSCK(h, cudaGetLastError());
    h->events += 1;
    return HAMR_OK;
}

int ms_average(hamr_ms_t h, int cx0, int ncol) {
    const long long n = (long long)ncol * h->P.ncy * h->P.ncz;
    k_ms_average<<<nblk(n), BLK, 0, h->stream>>>(h->m, h->S, h->grain_d, h->P, h->ox, cx0, ncol);
    MSCK(h, cudaGetLastError());
    return HAMR_OK;
}

int ms_target(const hamr_ms_t h, double t) {
    const double xc = h->D.x0 + h->D.vx * t;
    double f = floor(xc / h->P.cell - 0.5 * h->P.wx + 0.5);
    f = fmax(0.0, fmin(f, (double)(h->P.ncx - h->P.wx)));
    return (int)f;
}

// One coupled step n -> n+1 (stages 1-3 of the file header).
int ms_step(hamr_ms_t h) {
    const MsDev &P = h->P;
    cudaStream_t st = h->stream;
    int rc = ms_average(h, h->ox, P.wx);
    if (rc) return rc;
    k_ms_predict<<<nblk(P.nw), BLK, 0, st>>>(h->S, h->Sp, h->F1, h->BTH, h->m, h->grain_d, P, h->D, h->bits_d, h->ox,
                                             h->step);
    k_ms_correct<<<nblk(P.nw), BLK, 0, st>>>(h->S, h->Sp, h->F1, h->BTH, h->m, h->grain_d, P, h->D, h->bits_d, h->ox,
                                             h->step);
    MSCK(h, cudaGetLastError());
    const double t = (double)h->step * P.dt;
    double B[3];
    applied_host(h, t, B);
    k_mm_prep<<<nblk(P.nc), BLK, 0, st>>>(h->me, h->Tq, P, h->D, t, sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
    MSCK(h, cudaMemcpyAsync(h->V0, h->m, sizeof(double) * 3 * P.nc, cudaMemcpyDeviceToDevice, st));
    MSCK(h, cudaMemcpyAsync(h->V1, h->m, sizeof(double) * 3 * P.nc, cudaMemcpyDeviceToDevice, st));
    const double cst[4] = {0.5, 0.5, 1.0, 0.0}, wst[4] = {1.0, 2.0, 2.0, 1.0};
    for (int s = 0; s < 4; ++s) {
        const double *vin = (s & 1) ? h->V1 : h->V0;
        double *vout = (s & 1) ? h->V0 : h->V1;
        k_mm_stage<<<nblk(P.nc), BLK, 0, st>>>(vin, vout, h->acc, h->m, h->me, h->Tq, h->grain_d, P, h->ox, B[0], B[1],
                                               B[2], cst[s], wst[s], s == 0);
    }
    k_mm_final<<<nblk(P.nc), BLK, 0, st>>>(h->m, h->acc, h->grain_d, P, h->ox);
    MSCK(h, cudaGetLastError());
    h->step += 1;
    return HAMR_OK;
}

int ms_shift_forward(hamr_ms_t h, double t) {
    int rc = ms_average(h, h->ox, 1);
    if (rc) return rc;
    k_ms_shift<<<nblk(h->P.nw), BLK, 0, h->stream>>>(h->S2, h->S, h->P);
    MSCK(h, cudaGetLastError());
    std::swap(h->S, h->S2);
    h->ox += 1;
    return ms_thermalise(h, h->ox + h->P.wx - 1, h->ox + h->P.wx, t);
}

}  // namespace

extern "C" {

int hamr_ms_create(hamr_ms_t *out, const hamr_ms_desc *d) {
    if (!out) return msfail(nullptr, HAMR_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return msfail(nullptr, HAMR_ERR_ARG, "desc is NULL");
    if (d->ncx < 1 || d->ncy < 1 || d->ncz < 1 || d->ratio < 1 || d->wx < 1 || d->wx > d->ncx)
        return msfail(nullptr, HAMR_ERR_ARG, "bad mesh: cells >= 1 per axis, ratio >= 1, 1 <= wx <= ncx");
    const long long nc = (long long)d->ncx * d->ncy * d->ncz;
    const long long nw = (long long)d->wx * d->ratio * (long long)d->ncy * d->ratio * (long long)d->ncz * d->ratio;
    if (nc > (1LL << 31) || nw > (1LL << 31)) return msfail(nullptr, HAMR_ERR_ARG, "mesh or window too large");
    const double vals[] = {d->cell, d->mu_s, d->gamma, d->dt, d->T_C, d->Ms0};
    for (double v : vals)
        if (!(v > 0) || !isfinite(v))
            return msfail(nullptr, HAMR_ERR_ARG, "cell, mu_s, gamma, dt, T_C and Ms0 must be positive");
    if (!isfinite(d->J) || !isfinite(d->ku) || !(d->lambda >= 0) || !isfinite(d->A0) || !isfinite(d->K0))
        return msfail(nullptr, HAMR_ERR_ARG, "J, ku, A0, K0 must be finite and lambda >= 0");
    hamr_ms_t h = new (std::nothrow) hamr_ms_ctx();
    if (!h) return msfail(nullptr, HAMR_ERR_OOM, "host allocation failed");
    h->device = d->device;
    MsDeviceGuard dg(h->device);
    MsDev &P = h->P;
    P.ncx = d->ncx; P.ncy = d->ncy; P.ncz = d->ncz; P.r = d->ratio; P.wx = d->wx;
    P.nxw = d->wx * d->ratio; P.nyw = d->ncy * d->ratio; P.nzw = d->ncz * d->ratio;
    P.nc = nc; P.nw = nw;
    P.cell = d->cell; P.a = d->cell / d->ratio;
    P.J = d->J; P.mu_s = d->mu_s; P.ku = d->ku;
    P.Ms0 = d->Ms0; P.A0 = d->A0; P.K0 = d->K0;
    P.lambda = d->lambda; P.T_C = d->T_C; P.gamma = d->gamma; P.dt = d->dt;
    P.sig0 = sqrt(2.0 * d->lambda * KB / (d->gamma * d->mu_s * d->dt));
    P.key0 = (unsigned)d->seed;
    P.key1 = (unsigned)(d->seed >> 32);
    h->D.dir[2] = 1.0;
    if (d->stream) {
        h->stream = (cudaStream_t)d->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return msfail(nullptr, HAMR_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    double **bufs3c[] = {&h->m, &h->V0, &h->V1, &h->acc};
    cudaError_t e = cudaSuccess;
    for (double **b : bufs3c)
        if (e == cudaSuccess) e = cudaMalloc((void **)b, sizeof(double) * 3 * nc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->me, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->Tq, sizeof(double) * nc);
    double **bufs3w[] = {&h->S, &h->S2, &h->Sp, &h->F1, &h->BTH};
    for (double **b : bufs3w)
        if (e == cudaSuccess) e = cudaMalloc((void **)b, sizeof(double) * 3 * nw);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->stage, sizeof(double) * 3 * (nw > nc ? nw : nc));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->grain_d, sizeof(int) * nc);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->m, 0, sizeof(double) * 3 * nc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->S, 0, sizeof(double) * 3 * nw, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->grain_d, 0, sizeof(int) * nc, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        ms_free(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return msfail(nullptr, e == cudaErrorMemoryAllocation ? HAMR_ERR_OOM : HAMR_ERR_CUDA, "device setup: %s",
                      cudaGetErrorString(e));
    }
    h->grain_h.assign(nc, 0);
    *out = h;
    return HAMR_OK;
}

int hamr_ms_set_grain_map(hamr_ms_t h, const int32_t *cell_grain) {
    if (!h || !cell_grain) return h ? msfail(h, HAMR_ERR_ARG, "cell_grain is NULL") : HAMR_ERR_ARG;
    for (long long q = 0; q < h->P.nc; ++q)
        if (cell_grain[q] < -1) return msfail(h, HAMR_ERR_ARG, "grain ids must be >= -1 (cell %lld)", q);
    MsDeviceGuard dg(h->device);
    h->grain_h.assign(cell_grain, cell_grain + h->P.nc);
    MSCK(h, cudaMemcpyAsync(h->grain_d, h->grain_h.data(), sizeof(int) * h->P.nc, cudaMemcpyHostToDevice, h->stream));
    k_zero_void_cells<<<nblk(h->P.nc), BLK, 0, h->stream>>>(h->m, h->grain_d, h->P.nc);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaStreamSynchronize(h->stream));
    h->grains_set = true;
    return HAMR_OK;
}

int hamr_ms_set_temperature_profile(hamr_ms_t h, double T_amb, double T_peak, double fwhm, double x0, double y0,
                                    double vx, double vy) {
    if (!h) return HAMR_ERR_ARG;
    const double v[] = {T_amb, T_peak, fwhm, x0, y0, vx, vy};
    for (double x : v)
        if (!isfinite(x)) return msfail(h, HAMR_ERR_ARG, "temperature profile values must be finite");
    if (T_amb < 0 || (fwhm > 0 && T_peak < 0)) return msfail(h, HAMR_ERR_ARG, "temperatures must be >= 0");
    ReplicaDev &D = h->D;
    D.T_amb = T_amb;
    D.dT = fwhm > 0 ? T_peak - T_amb : 0.0;
    D.c_fwhm = fwhm > 0 ? -4.0 * log(2.0) / (fwhm * fwhm) : 0.0;
    D.x0 = x0; D.y0 = y0; D.vx = vx; D.vy = vy;
    return HAMR_OK;
}

int hamr_ms_set_field_sequence(hamr_ms_t h, double B0, const double dir[3], const uint8_t *bits, int32_t n_bits,
                               double bit_len, double ramp_len, double head_x0, double head_v) {
    if (!h) return HAMR_ERR_ARG;
    if (!dir || !isfinite(B0) || !isfinite(dir[0]) || !isfinite(dir[1]) || !isfinite(dir[2]))
        return msfail(h, HAMR_ERR_ARG, "field amplitude and direction must be finite");
    if (n_bits < 0 || (n_bits > 0 && (!bits || !(bit_len > 0) || !(ramp_len >= 0) || !isfinite(head_x0) ||
                                      !isfinite(head_v))))
        return msfail(h, HAMR_ERR_ARG, "bad bit sequence (bits, bit_len > 0, ramp_len >= 0)");
    MsDeviceGuard dg(h->device);
    ReplicaDev &D = h->D;
    D.B0 = B0;
    for (int k = 0; k < 3; ++k) D.dir[k] = dir[k];
    D.n_bits = n_bits;
    D.bits_off = 0;
    D.bit_len = bit_len; D.ramp_len = ramp_len; D.head_x0 = head_x0; D.head_v = head_v;
    h->bits_h.assign(bits, bits + n_bits);
    if (h->bits_d) cudaFree(h->bits_d);
    h->bits_d = nullptr;
    if (n_bits > 0) {
        MSCK(h, cudaMalloc((void **)&h->bits_d, n_bits));
        MSCK(h, cudaMemcpyAsync(h->bits_d, h->bits_h.data(), n_bits, cudaMemcpyHostToDevice, h->stream));
        MSCK(h, cudaStreamSynchronize(h->stream));
    }
    return HAMR_OK;
}

int hamr_ms_set_cells(hamr_ms_t h, const double *m) {
    if (!h || !m) return h ? msfail(h, HAMR_ERR_ARG, "m is NULL") : HAMR_ERR_ARG;
    for (long long q = 0; q < 3 * h->P.nc; ++q)
        if (!isfinite(m[q])) return msfail(h, HAMR_ERR_ARG, "non-finite cell value at %lld", q / 3);
    MsDeviceGuard dg(h->device);
    MSCK(h, cudaMemcpyAsync(h->stage, m, sizeof(double) * 3 * h->P.nc, cudaMemcpyHostToDevice, h->stream));
    k_aos_to_planes<<<nblk(h->P.nc), BLK, 0, h->stream>>>(h->stage, h->m, h->P.nc);
    k_zero_void_cells<<<nblk(h->P.nc), BLK, 0, h->stream>>>(h->m, h->grain_d, h->P.nc);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaStreamSynchronize(h->stream));
    h->cells_set = true;
    return HAMR_OK;
}

int hamr_ms_set_window(hamr_ms_t h, int32_t x0_cells) {
    if (!h) return HAMR_ERR_ARG;
    if (x0_cells < 0 || x0_cells + h->P.wx > h->P.ncx)
        return msfail(h, HAMR_ERR_ARG, "window [%d, %d) outside the track of %d cells", x0_cells, x0_cells + h->P.wx,
                      h->P.ncx);
    if (!h->cells_set) return msfail(h, HAMR_ERR_STATE, "set the cells (hamr_ms_set_cells) before the window");
    MsDeviceGuard dg(h->device);
    h->ox = x0_cells;
    int rc = ms_thermalise(h, h->ox, h->ox + h->P.wx, (double)h->step * h->P.dt);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_set_moments(hamr_ms_t h, const double *S) {
    if (!h || !S) return h ? msfail(h, HAMR_ERR_ARG, "S is NULL") : HAMR_ERR_ARG;
    if (h->ox < 0) return msfail(h, HAMR_ERR_STATE, "place the window (hamr_ms_set_window) first");
    MsDeviceGuard dg(h->device);
    MSCK(h, cudaMemcpyAsync(h->stage, S, sizeof(double) * 3 * h->P.nw, cudaMemcpyHostToDevice, h->stream));
    k_aos_to_planes<<<nblk(h->P.nw), BLK, 0, h->stream>>>(h->stage, h->S, h->P.nw);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_steps(hamr_ms_t h, int64_t n_steps, int32_t follow) {
    if (!h) return HAMR_ERR_ARG;
    if (n_steps < 0) return msfail(h, HAMR_ERR_ARG, "n_steps must be >= 0");
    if (h->ox < 0) return msfail(h, HAMR_ERR_STATE, "place the window (hamr_ms_set_window) first");
    MsDeviceGuard dg(h->device);
    for (int64_t s = 0; s < n_steps; ++s) {
        int rc = ms_step(h);
        if (rc) return rc;
        if (follow) {
            const double t = (double)h->step * h->P.dt;
            const int target = ms_target(h, t);
            while (h->ox < target)
                if ((rc = ms_shift_forward(h, t))) return rc;
        }
    }
    int rc = ms_average(h, h->ox, h->P.wx);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_read_cells(hamr_ms_t h, double *m_out) {
    if (!h || !m_out) return h ? msfail(h, HAMR_ERR_ARG, "m_out is NULL") : HAMR_ERR_ARG;
    MsDeviceGuard dg(h->device);
    k_planes_to_aos<<<nblk(h->P.nc), BLK, 0, h->stream>>>(h->m, h->stage, h->P.nc);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaMemcpyAsync(m_out, h->stage, sizeof(double) * 3 * h->P.nc, cudaMemcpyDeviceToHost, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_read_moments(hamr_ms_t h, double *S_out) {
    if (!h || !S_out) return h ? msfail(h, HAMR_ERR_ARG, "S_out is NULL") : HAMR_ERR_ARG;
    MsDeviceGuard dg(h->device);
    k_planes_to_aos<<<nblk(h->P.nw), BLK, 0, h->stream>>>(h->S, h->stage, h->P.nw);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaMemcpyAsync(S_out, h->stage, sizeof(double) * 3 * h->P.nw, cudaMemcpyDeviceToHost, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_get_window(hamr_ms_t h, int32_t *x0_cells, int64_t *step) {
    if (!h) return HAMR_ERR_ARG;
    if (x0_cells) *x0_cells = h->ox;
    if (step) *step = h->step;
    return HAMR_OK;
}

const char *hamr_ms_last_error(hamr_ms_t h) { return h ? h->err.c_str() : g_ms_create_err.c_str(); }

void hamr_ms_destroy(hamr_ms_t h) {
    if (!h) return;
    MsDeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    ms_free(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
