// The multiscale write window (Sec. II, Fig. 1): a simple-cubic atomistic window embedded in
// a micromagnetic finite-difference track, exchange coupled across the interface and moving
// with the laser spot.  The state (spins, cells, fields) is FP64 or FP32, the handle's
// precision; m_e(T) and the tensor of Eq. 7 are computed in FP64.
//
// Per coupled step n -> n+1 (drivers frozen at t_n):
//   1. k_ms_average_w - Eq. 6: every window cell takes the direction of the sum of its sites;
//   2. k_mm_prep      - T and m_e(T), the root of the Langevin equation (Sec. II), per cell
//                       column, and the cells' coefficients Ms = Ms0 m_e, A = A0 m_e^2,
//                       K = K0 m_e^3, alpha = lambda (1 - T / 3 T_C);
//   3. with Eq. 7     - k_demag_M, in-plane transforms (cuFFT), k_demag_zmul[_r] (the sum
//                       along z), inverse transforms: B_d of the state at t_n, which the
//                       window step and the RK4 stages read from the transform (BdView);
//   4. k_ms_fused     - the sLLG Heun step of the window (Eq. 1-3), both stages in one pass;
//                       across the window's x faces a bond sees the direction of the
//                       micromagnetic cell there;
//   5. k_mm_stage x4  - one classical RK4 step of the micromagnetic LLG (Eq. 1 without the
//                       thermal field; Eq. 4 on a 6-point Laplacian, Eq. 5) on the cells of
//                       the simulated region outside the window, the last stage applying the
//                       update; window cells stay at their Eq. 6 directions;
//   6. window moves   - k_ms_average_w of the trailing column, k_ms_shift of the sites by one
//                       cell column, k_ms_thermalise of the new leading column in the cone
//                       of half-angle theta_max(m_e) (Sec. II).
// Device layout: cell and site arrays are component planes [3][n]; cell q = cx + ncx (cy +
// ncy cz); window site s = i + nxw (j + nyw k) with i along the track.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cufft.h>

#include <algorithm>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
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
    int profile;               // write field: 0 uniform, 1 tanh profiles following the head
    double pwz, pdz, pBx0, pwx, pdx;  // profile widths, offsets from the head [m], in-plane amplitude [T]
    double cA, cK, mu_kB, i3TC;       // 2 A0 / Ms0, 2 K0 / Ms0, mu_s / kB, 1 / (3 T_C)
    double J_mu, ku2_mu;              // J / mu_s, 2 ku / mu_s
};

// The write field at one step, from the host: B0 s(t) dir, Bx0 s(t) and the head position.
template <typename Real>
struct Field {
    Real bx, by, bz;   // B0 s(t) dir
    Real bxs;          // Bx0 s(t)
    Real xh;           // head position x_h(t)
};

template <typename Real>
struct V3 {
    Real x, y, z;
};

// -gamma/(1+alpha^2) [S x B + alpha S x (S x B)]
template <typename Real>
__device__ __forceinline__ V3<Real> rhs(Real gamma, Real alpha, Real sx, Real sy, Real sz, Real bx, Real by, Real bz) {
    const Real cx = sy * bz - sz * by, cy = sz * bx - sx * bz, cz = sx * by - sy * bx;
    const Real dx = sy * cz - sz * cy, dy = sz * cx - sx * cz, dz = sx * cy - sy * cx;
    const Real pref = -gamma / (Real(1) + alpha * alpha);
    return {pref * (cx + alpha * dx), pref * (cy + alpha * dy), pref * (cz + alpha * dz)};
}

// the laser temperature and the write field in the arithmetic of the state (FP64 or FP32
// driver copies)
__device__ __forceinline__ double temp_at(const ReplicaDev &D, double x, double y, double t) {
    return temperature(D, x, y, t);
}
__device__ __forceinline__ float temp_at(const ReplicaDev &D, float x, float y, float t) {
    return temperature_f(D, x, y, t);
}
// The write field at track position x (Sec. III, Fig. 2): uniform B0 s(t) dir, or with the
// head profile B0 s(t) dir P(x - x_h - dz, wz) + Bx0 s(t) P(x - x_h - dx, wx) x with
// P(u, w) = (1 - tanh(u / w)) / 2.
template <typename Real>
__device__ __forceinline__ V3<Real> field_at(const MsDev &P, const Field<Real> &F, Real x) {
    if (!P.profile) return {F.bx, F.by, F.bz};
    const Real Pz = Real(0.5) * (Real(1) - tanh((x - F.xh - (Real)P.pdz) / (Real)P.pwz));
    const Real Px = Real(0.5) * (Real(1) - tanh((x - F.xh - (Real)P.pdx) / (Real)P.pwx));
    return {F.bx * Pz + F.bxs * Px, F.by * Pz, F.bz * Pz};
}

// The Langevin function L(x) = coth x - 1/x and its derivative L'(x) = 1/x^2 - 1/sinh^2 x
// from one expm1: with u = expm1(-2|x|) in (-1, 0), coth|x| = (2 + u) / (-u) and
// 1/sinh^2 x = 4 (1 + u) / u^2.  Below |x| = 1e-3 both come from their Taylor series.
__device__ __forceinline__ void langevin2(double x, double &L, double &Lp) {
    const double ax = fabs(x);
    if (ax < 1e-3) {
        const double x2 = x * x;
        L = x / 3.0 - x * x2 / 45.0 + 2.0 * x * x2 * x2 / 945.0;
        Lp = 1.0 / 3.0 - x2 / 15.0 + 2.0 * x2 * x2 / 189.0;
        return;
    }
    const double u = expm1(-2.0 * ax);
    const double iu = 1.0 / u, ix = 1.0 / ax;
    const double l = -(2.0 + u) * iu - ix;
    L = x < 0.0 ? -l : l;
    Lp = ix * ix - 4.0 * (1.0 + u) * (iu * iu);
}

// m_e(T): the largest root in [0, 1] of m = L(3 T_C m / T + mu_s B / (kB T)).  Newton steps
// from m0 (extrapolated from the cell's last two solves; 1 when there is none) kept inside a bracket
// [lo, hi] with L(.) - m >= 0 at lo and < 0 at hi; a step that leaves the bracket is
// replaced by bisection.  A Newton step below 1e-13 (1 + m) is taken as converged (the
// iteration is quadratic there; the bound is absolute for small m, where coth x - 1/x loses
// digits to cancellation and the residual is only known to about 1e-14), before the bracket
// test, which a converged step can fail by rounding, but only where the root is stable
// (slope a L' - 1 < 0).  The largest root always is; below T_C without a field, m = 0 is an
// unstable root that a start near 0 (a cell that was above T_C) would otherwise keep.  From
// there the Newton step stays at 0 and leaves the bracket, so bisection takes over.
__device__ double me_root(double T_C, double T, double mu_kB, double B, double m0) {
    if (!(T > 0.0)) return 1.0;
    const double iT = 1.0 / T;
    const double a = 3.0 * T_C * iT, b = mu_kB * B * iT;
    double lo = 0.0, hi = 1.0, m = (m0 > 0.0 && m0 <= 1.0) ? m0 : 1.0;
    for (int it = 0; it < 300; ++it) {
        double L, Lp;
        langevin2(a * m + b, L, Lp);
        const double g = L - m;
        if (g >= 0.0)
            lo = m;
        else
            hi = m;
        const double gp = a * Lp - 1.0;
        const double mn = m - g / gp;
        if (fabs(mn - m) <= 1e-13 * (1.0 + m) && gp < 0.0) return mn;
        m = (mn > lo && mn < hi) ? mn : 0.5 * (lo + hi);
        if (hi - lo <= 1e-16 * hi) return lo;
    }
    return lo;
}

__device__ __forceinline__ double theta_max(double mr) {
    double x = 1.0 + 6.0 * (mr - 1.0) / 5.0;
    x = fmin(fmax(x, 0.0), 1.0);
    return (5.0 * M_PI / 9.0) * sqrt(1.0 - sqrt(x));
}

__device__ __forceinline__ int cell_at(const MsDev &P, int cx, int cy, int cz) {
    return cx + P.ncx * (cy + P.ncy * cz);
}

// v / ratio for v >= 0, with the ratio a compile-time constant when RT != 0 (1, 2 and 4 are
// instantiated; other ratios use the runtime value)
template <int RT>
__device__ __forceinline__ int per_cell(const MsDev &P, int v) {
    return RT ? (int)((unsigned)v / (unsigned)RT) : v / P.r;
}

// 3-D launch over (x, y, z) with blocks of 32 x 4: the thread's coordinates
__device__ __forceinline__ bool coords(int nx, int ny, int &x, int &y, int &z) {
    x = blockIdx.x * 32 + threadIdx.x;
    y = blockIdx.y * 4 + threadIdx.y;
    z = blockIdx.z;
    return x < nx && y < ny;
}

// Eq. 6 for the cells of columns [cx0, cx0 + ncol): direction of the sum of their sites.
template <typename Real>
__global__ void k_ms_average(Real *m, Real *wn, const Real *S, const int *grain, MsDev P, int ox, int cx0, int ncol) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = (long long)ncol * P.ncy * P.ncz;
    if (idx >= n) return;
    const int cx = cx0 + (int)(idx % ncol), cy = (int)((idx / ncol) % P.ncy), cz = (int)(idx / ((long long)ncol * P.ncy));
    const int q = cell_at(P, cx, cy, cz);
    Real sx = 0, sy = 0, sz = 0;
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
    const Real nn = sqrt(sx * sx + sy * sy + sz * sz);
    m[q] = nn > Real(0) ? sx / nn : Real(0);
    m[P.nc + q] = nn > Real(0) ? sy / nn : Real(0);
    m[2 * P.nc + q] = nn > Real(0) ? sz / nn : Real(0);
    wn[q] = nn;
}

// The same for a compile-time ratio RT in {1, 2, 4}: a warp takes 32 / RT consecutive cells
// of one cell row (cy, cz); lane (c, di) sums site column di of cell c over the cell's RT^2
// rows (dj, dk), each row read by the warp as one run of consecutive sites, and the RT lanes
// of a cell add by shuffles.
template <typename Real, int RT>
__global__ void k_ms_average_w(Real *m, Real *wn, const Real *S, const int *grain, MsDev P, int ox, int cx0,
                               int ncol) {
    constexpr int CPW = 32 / RT;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int wpr = (ncol + CPW - 1) / CPW;
    if (w >= (long long)wpr * P.ncy * P.ncz) return;   // uniform over the warp
    const int row = (int)(w / wpr), c = (int)(w % wpr) * CPW + lane / RT, di = lane % RT;
    const int cy = row % P.ncy, cz = row / P.ncy, cx = cx0 + c;
    const bool act = c < ncol;
    const int q = act ? cell_at(P, cx, cy, cz) : 0;
    Real sx = 0, sy = 0, sz = 0;
    if (act && grain[q] >= 0) {
        const long long i = (long long)(cx - ox) * RT + di;
#pragma unroll
        for (int dk = 0; dk < RT; ++dk)
#pragma unroll
            for (int dj = 0; dj < RT; ++dj) {
                const long long s = i + P.nxw * ((long long)cy * RT + dj + (long long)P.nyw * ((long long)cz * RT + dk));
                sx += S[s];
                sy += S[P.nw + s];
                sz += S[2 * P.nw + s];
            }
    }
#pragma unroll
    for (int o = RT / 2; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(full, sx, o);
        sy += __shfl_xor_sync(full, sy, o);
        sz += __shfl_xor_sync(full, sz, o);
    }
    if (act && di == 0) {
        const Real nn = sqrt(sx * sx + sy * sy + sz * sz);
        m[q] = nn > Real(0) ? sx / nn : Real(0);
        m[P.nc + q] = nn > Real(0) ? sy / nn : Real(0);
        m[2 * P.nc + q] = nn > Real(0) ? sz / nn : Real(0);
        wn[q] = nn;
    }
}

__device__ __forceinline__ float inv_norm(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_norm(double x) { return 1.0 / sqrt(x); }

// B_d of Eq. 7 read where it is used: s H + add on the cells of a convolution grid whose
// first column is g0, H the grid's unnormalised inverse transform [3][Ptot] (s = -mu0 / (Px Py))
// and add the frozen cells' part [3][nc] (or null).  H null: no demagnetising field.  A cell
// beyond the grid's columns reads its nearest grid column (only cells that are not evolved,
// whose loads are issued before their tests, ask for one).
template <typename Real>
struct BdView {
    const Real *H = nullptr, *add = nullptr;
    long long Ptot = 0;
    int Px = 0, Py = 0, g0 = 0, ncol = 0;
    Real s = 0;
    __device__ __forceinline__ V3<Real> at(const MsDev &P, int cx, int cy, int cz, int q) const {
        int i = cx - g0;
        i = i < 0 ? 0 : (i >= ncol ? ncol - 1 : i);
        const long long pp = i + (long long)Px * (cy + (long long)Py * cz);
        V3<Real> b = {s * H[pp], s * H[Ptot + pp], s * H[2 * Ptot + pp]};
        if (add) {
            b.x += add[q];
            b.y += add[P.nc + q];
            b.z += add[2 * P.nc + q];
        }
        return b;
    }
};

// ---------------------------------------------------------------- fused window step
// Both Heun stages of the window in one pass over its sites (Sec. II, Eq. 1-3): the predictor
// S' = normalise(S + dt f(S)), the corrector normalise(S + dt/2 f(S) + dt/2 f(S')), both
// with the same thermal field and the drivers at t_n.  A bond within a cell or across a cell
// face between cells of one grain couples; across the window's x faces a site sees the cell
// of the neighbour position, if that cell is of the site's grain.
// A CTA takes a tile of MWX x MWY site columns and a range of MWZ planes.  Each of its threads
// owns one column of the tile or of the two-column ring around it and marches up the planes
// from the one below the range to the one above it: at plane k the tile and the inner ring
// predict S'(k) (the outer ring only stages S for them), then, after the CTA's one barrier of
// the step, the tile's threads correct plane k - 1.  The inner ring's S' is recomputed with
// the same noise as the neighbouring tiles' (the counter is the site's track index), so no
// CTA needs another's S'.  S and S' of the staged columns pass through shared memory as
// (x, y, z, grain code) records; a column beyond the window's x face is the interface: its S
// and S' are the direction m of the cell holding the neighbour position (frozen for the
// window's step), its grain code that cell's.  Columns beyond the track's y edges, beyond the
// track's ends and planes beyond its z faces read 0.
constexpr int MWX = 28, MWY = 8, MWZ = 40;                        // tile columns, planes per item
constexpr int MWSX = MWX + 4, MWSY = MWY + 4, MWPOS = MWSX * MWSY;  // staged columns: a warp per row
constexpr int MWT = MWPOS;                                         // threads

template <typename Real>
struct V4 {
    Real x, y, z, g;  // g: grain code (grain + 1, 0 for a non-magnetic site)
};

template <typename Real, int RT>
__global__ void __launch_bounds__(MWT, sizeof(Real) == 4 ? 2 : 1)
    k_ms_fused(const Real *__restrict__ Sin, Real *__restrict__ Sout, const Real *__restrict__ m,
               const int *__restrict__ grain, MsDev P, ReplicaDev D, Field<Real> F, BdView<Real> V, int ox,
               long long step) {
    extern __shared__ unsigned char ms_smem[];
    V4<Real>(*sS)[MWPOS] = reinterpret_cast<V4<Real>(*)[MWPOS]>(ms_smem);  // [3]: S, plane k in slot k mod 3
    V4<Real>(*sP)[MWPOS] = sS + 3;                                          // [4]: S', plane k in slot k mod 4
    const int tid = threadIdx.x;
    const bool own = tid < MWPOS;
    const int ci = tid % MWSX, cj = tid / MWSX;
    const int i = (int)blockIdx.x * MWX - 2 + ci, j = (int)blockIdx.y * MWY - 2 + cj;
    const int z0 = (int)blockIdx.z * MWZ, z1 = min(P.nzw, z0 + MWZ);
    const bool yin = j >= 0 && j < P.nyw;
    const bool site = own && yin && i >= 0 && i < P.nxw;
    // the interface cell column beyond the window's x face (-1: none)
    int icx = -1;
    if (own && yin && i == -1 && ox > 0) icx = ox - 1;
    if (own && yin && i == P.nxw && ox + P.wx < P.ncx) icx = ox + P.wx;
    const bool pred = ci >= 1 && ci <= MWX + 2 && cj >= 1 && cj <= MWY + 2;  // the tile and the inner ring
    const bool inner = site && ci >= 2 && ci <= MWX + 1 && cj >= 2 && cj <= MWY + 1;
    const int cy = yin ? per_cell<RT>(P, j) : 0;
    const int cxs = site ? ox + per_cell<RT>(P, i) : 0;
    const int lz = P.ncx * P.ncy;
    // S and grain code of this column at plane k (0 off the window and off the track).  Planes
    // are loaded in increasing order, so the grain code (and an interface cell's m) is read
    // once per cell plane (the test on the cell index is the same for the whole CTA).  load()
    // only issues the reads; finish() applies the grain code when the plane is first used, a
    // march step later, so no thread waits on a read it has just issued.
    int lcz = -1, lgq = -1;
    V3<Real> lm = {0, 0, 0};
    // site indices advance by one plane per call (planes are loaded in order, from z0 - 2; the
    // unsigned arithmetic wraps back to the right value once k >= 0); the component planes are
    // addressed from 64-bit bases
    const unsigned pw = (unsigned)P.nxw * (unsigned)P.nyw;
    const unsigned scol = site ? (unsigned)i + (unsigned)P.nxw * (unsigned)j : 0u;
    const Real *Sx = Sin, *Sy = Sin + P.nw, *Sz = Sin + 2 * P.nw;
    unsigned sld = scol + pw * (unsigned)(z0 - 2);
    auto load = [&](int k, V4<Real> &v, bool &in) {
        const unsigned sk_ = sld;
        sld += pw;
        in = k >= 0 && k < P.nzw;
        v.x = v.y = v.z = v.g = Real(0);
        if (in) {
            const int cz = per_cell<RT>(P, k);
            if (cz != lcz) {
                lcz = cz;
                if (site) {
                    lgq = grain[cxs + P.ncx * cy + lz * cz];
                } else if (icx >= 0) {
                    const int q = icx + P.ncx * cy + lz * cz;
                    lgq = grain[q];
                    lm = {m[q], m[P.nc + q], m[2 * P.nc + q]};
                }
            }
        }
        if (site) {  // a valid slot off the window's planes, its value dropped by finish()
            const unsigned ix = in ? sk_ : scol;
            v.x = Sx[ix];
            v.y = Sy[ix];
            v.z = Sz[ix];
        }
    };
    // the plane last loaded, with its cell's grain code (and, for an interface column, m)
    auto finish = [&](V4<Real> &v, bool in) {
        if (!in || lgq < 0) {
            v.x = v.y = v.z = v.g = Real(0);
            return;
        }
        if (!site) {
            v.x = lm.x;
            v.y = lm.y;
            v.z = lm.z;
        }
        v.g = (Real)(lgq + 1);
    };
    // B_d of the predicted plane's cell, read once per cell plane
    int bcz = -1;
    V3<Real> bd = {0, 0, 0};
    // per-column drivers: the laser's thermal-field scale and the applied field along x
    const Real t = (Real)step * (Real)P.dt, a = (Real)P.a;
    const Real xs = ((Real)ox * P.r + i + Real(0.5)) * a;
    Real sig = 0;
    V3<Real> ba0 = {0, 0, 0};
    if (site) {
        sig = (Real)P.sig0 * sqrt(temp_at(D, xs, (j + Real(0.5)) * a, t));
        ba0 = field_at(P, F, xs);
    }
    const unsigned long long X = (unsigned long long)ox * P.r + (unsigned long long)(site ? i : 0),
                             NX = (unsigned long long)P.ncx * P.r;
    const Real Jm = (Real)P.J_mu, Km = (Real)P.ku2_mu, dt = (Real)P.dt, hdt = Real(0.5) * dt;

    // prologue: S of planes z0 - 2 .. z0 in registers, plane z0 - 1 staged
    V4<Real> m1, c0, p1, p2;
    bool in1, in2;
    load(z0 - 2, m1, in1);
    finish(m1, in1);
    load(z0 - 1, c0, in1);
    finish(c0, in1);
    load(z0, p1, in1);
    if (own) sS[(z0 + 2) % 3][tid] = c0;
    __syncthreads();
    // the corrector base S + dt/2 f1 and the S-independent field (applied, thermal) of the
    // plane awaiting correction; the own S' of planes k - 2 and k - 1
    Real amx = 0, amy = 0, amz = 0, hmx = 0, hmy = 0, hmz = 0;
    // running indices of plane k (from z0 - 1): S slot k mod 3, S' slot k mod 4, the site of
    // the plane being corrected (k - 1) and plane k's Philox counter
    int sk = (z0 + 2) % 3, pk = (z0 + 3) & 3;
    unsigned sst = scol + pw * (unsigned)(z0 - 2);
    Real *Ox = Sout, *Oy = Sout + P.nw, *Oz = Sout + 2 * P.nw;
    unsigned long long sidx = X + NX * ((unsigned long long)j + (unsigned long long)P.nyw * (unsigned long long)(z0 - 1));
    const unsigned long long dsid = NX * (unsigned long long)P.nyw;
    for (int k = z0 - 1; k <= z1; ++k) {
        finish(p1, in1);      // plane k + 1, loaded a step ago
        load(k + 2, p2, in2);  // finished next step: its latency overlaps this step
        const int sk1 = sk == 2 ? 0 : sk + 1;
        // ---- predictor on plane k
        V4<Real> sp = {0, 0, 0, 0};
        Real anx = 0, any = 0, anz = 0, hx = 0, hy = 0, hz = 0;
        if (icx >= 0) {
            sp = c0;  // an interface cell: S' = m (frozen for the step)
        } else if (site && pred && k >= 0 && k < P.nzw && c0.g != Real(0)) {
            Real n0, n1, n2;
            normals3(philox_site(P.key0, P.key1, sidx, (unsigned long long)step), n0, n1, n2);
            V3<Real> ba = ba0;
            if (V.H) {  // the demagnetising field of the site's cell (Eq. 7)
                const int cz = per_cell<RT>(P, k);
                if (cz != bcz) {
                    bcz = cz;
                    bd = V.at(P, cxs, cy, cz, cxs + P.ncx * cy + lz * cz);
                }
                ba.x += bd.x;
                ba.y += bd.y;
                ba.z += bd.z;
            }
            hx = ba.x + sig * n0;
            hy = ba.y + sig * n1;
            hz = ba.z + sig * n2;
            const V4<Real> *Q = sS[sk];
            const Real g = c0.g;
            Real ex = 0, ey = 0, ez = 0;
            auto add = [&](const V4<Real> &v) {
                if (v.g == g) {
                    ex += v.x;
                    ey += v.y;
                    ez += v.z;
                }
            };
            add(Q[tid - 1]);
            add(Q[tid + 1]);
            add(Q[tid - MWSX]);
            add(Q[tid + MWSX]);
            add(m1);
            add(p1);
            const V3<Real> f = rhs<Real>((Real)P.gamma, (Real)P.lambda, c0.x, c0.y, c0.z, Jm * ex + hx, Jm * ey + hy,
                                         Jm * ez + Km * c0.z + hz);
            anx = c0.x + hdt * f.x;
            any = c0.y + hdt * f.y;
            anz = c0.z + hdt * f.z;
            const Real vx = c0.x + dt * f.x, vy = c0.y + dt * f.y, vz = c0.z + dt * f.z;
            const Real in = inv_norm(vx * vx + vy * vy + vz * vz);
            sp = {vx * in, vy * in, vz * in, g};
        }
        if (own) {
            sP[pk][tid] = sp;
            sS[sk1][tid] = p1;  // S of plane k + 1, read by the next step's predictor
        }
        __syncthreads();
        // ---- corrector on plane k - 1 (the tile's columns)
        const int kc = k - 1;
        if (inner && kc >= z0 && kc < z1) {
            const V4<Real> *Q = sP[(pk + 3) & 3];
            const V4<Real> v = Q[tid];
            Real ox_ = 0, oy_ = 0, oz_ = 0;
            if (v.g != Real(0)) {
                const Real g = v.g;
                Real ex = 0, ey = 0, ez = 0;
                auto add = [&](const V4<Real> &w) {
                    if (w.g == g) {
                        ex += w.x;
                        ey += w.y;
                        ez += w.z;
                    }
                };
                add(Q[tid - 1]);
                add(Q[tid + 1]);
                add(Q[tid - MWSX]);
                add(Q[tid + MWSX]);
                add(sP[(pk + 2) & 3][tid]);  // S'(k - 2), own
                add(sp);                     // S'(k), own
                const V3<Real> f = rhs<Real>((Real)P.gamma, (Real)P.lambda, v.x, v.y, v.z, Jm * ex + hmx,
                                             Jm * ey + hmy, Jm * ez + Km * v.z + hmz);
                const Real wx = amx + hdt * f.x, wy = amy + hdt * f.y, wz = amz + hdt * f.z;
                const Real in = inv_norm(wx * wx + wy * wy + wz * wz);
                ox_ = wx * in;
                oy_ = wy * in;
                oz_ = wz * in;
            }
            Ox[sst] = ox_;
            Oy[sst] = oy_;
            Oz[sst] = oz_;
        }
        sk = sk1;
        pk = (pk + 1) & 3;
        sst += pw;
        sidx += dsid;
        m1 = c0;
        c0 = p1;
        p1 = p2;
        in1 = in2;
        amx = anx;
        amy = any;
        amz = anz;
        hmx = hx;
        hmy = hy;
        hmz = hz;
    }
}

// Per column (cx, cy) of magnetic cells at time t (FP64): the laser temperature at the column's
// centre and the write field depend on (x, y) only, so every cell of the column has the same
// m_e(T, |B_app|), solved once.  The column keeps its solve state in col [3][ncx ncy]: the
// temperature of its last solve (NaN: none), m_e and the m_e before it (NaN: none).  Newton
// starts from 2 m_e - m_e' (m_e alone when that leaves (0, 1] or there is no m_e'): the changes
// from step to step are smooth, so the first Newton step is usually already below the
// convergence bound.  A column solved last at this temperature and field magnitude
// (Bm == Bm_last, T unchanged) keeps its values: far from the spot T is the ambient
// temperature to the last bit.  Otherwise every magnetic cell of the column (bit z of the
// column's mask; planes from 64 on look up their grain) gets m_e and its field and damping
// coefficients 2 A(T)/Ms(T) = 2 A0 m_e / Ms0, 2 K(T)/Ms(T) = 2 K0 m_e^2 / Ms0,
// alpha = lambda (1 - T/3T_C) with T held in [0, T_C], stored in the arithmetic of the
// state.  The thread's loads are independent of one another and its cell writes are stores
// only: with one thread per column the launch is short of warps, so chains of dependent loads
// would set its duration.
template <typename Real>
__global__ void k_mm_prep(double *me, double *col, Real *coef, const int *grain, const unsigned long long *colmask,
                          MsDev P, ReplicaDev D, double t, Field<double> F, double Bm_last, int cx0, int ncol) {
    int cx, cy, cz;
    if (!coords(ncol, P.ncy, cx, cy, cz)) return;
    cx += cx0;
    const int lz = P.ncx * P.ncy, c = cx + P.ncx * cy;
    const unsigned long long msk = colmask[c];
    const double Tl = col[c], e0 = col[lz + c], ep = col[2 * lz + c];
    const double T = temperature(D, (cx + 0.5) * P.cell, (cy + 0.5) * P.cell, t);
    const V3<double> B = field_at(P, F, (cx + 0.5) * P.cell);
    const double Bm = sqrt(B.x * B.x + B.y * B.y + B.z * B.z);
    bool any = msk != 0;
    for (int z = 64; z < P.ncz && !any; ++z) any = grain[c + z * lz] >= 0;
    if (!any || (!P.profile && Bm == Bm_last && T == Tl)) return;
    double m0 = 2.0 * e0 - ep;
    if (!(m0 > 0.0 && m0 <= 1.0)) m0 = e0;
    const double e = me_root(P.T_C, T, P.mu_kB, Bm, m0);
    col[c] = T;
    col[lz + c] = e;
    col[2 * lz + c] = e0;
    double cex = P.cA * e, cK = P.cK * e * e;
    if (!(e > 0.0)) cex = cK = 0.0;
    const double Tc = fmax(fmin(T, P.T_C), 0.0);
    const Real rex = (Real)cex, rK = (Real)cK, ral = (Real)(P.lambda * (1.0 - Tc * P.i3TC));
    for (int z = 0; z < P.ncz; ++z) {
        const int q = c + z * lz;
        if (z < 64 ? !((msk >> z) & 1ull) : grain[q] < 0) continue;
        me[q] = e;
        coef[q] = rex;
        coef[P.nc + q] = rK;
        coef[2 * P.nc + q] = ral;
    }
}

// One RK4 stage on the evolved cells, the magnetic cells of columns [c0, c1) outside the
// window: K = dm/dt at the stage values Vin, acc += w K and Vout = m + c dt K (the next
// stage's values).  A window cell, and a frozen cell next to the simulated region, writes its
// m to Vout, so that every stage buffer holds m there (stage 0 reads m itself); the launch
// covers [e0, e1), one column beyond the region on each side.  The last stage (last != 0)
// instead replaces m of each evolved cell by the renormalised RK4 update m + dt/6 (acc + K):
// a stage reads no other cell's m, so the update can be made in place.  The values of
// non-magnetic cells are never used (they may be unset).  The threads are short and bound by
// memory latency, so every value a thread may need is loaded before any test.
template <typename Real>
__global__ void k_mm_stage(const Real *Vin, Real *Vout, Real *acc, Real *m, const Real *coef, const int *grain,
                           MsDev P, int ox, Field<Real> F, BdView<Real> V, Real c, Real w, int first, int last, int e0,
                           int ne, int c0, int c1) {
    int cx, cy, cz;
    if (!coords(ne, P.ncy, cx, cy, cz)) return;
    cx += e0;
    const int q = cell_at(P, cx, cy, cz), lz = P.ncx * P.ncy;
    // neighbours -x, +x, -y, +y, -z, +z (an absent one reads the cell itself and is masked).
    // Every load below is of a valid address and none waits on a test: one round trip.
    const bool has[6] = {cx > 0, cx + 1 < P.ncx, cy > 0, cy + 1 < P.ncy, cz > 0, cz + 1 < P.ncz};
    const int qn[6] = {has[0] ? q - 1 : q, has[1] ? q + 1 : q, has[2] ? q - P.ncx : q,
                       has[3] ? q + P.ncx : q, has[4] ? q - lz : q, has[5] ? q + lz : q};
    const int g = grain[q];
    int gn[6];
    Real nx[6], ny[6], nz[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        gn[b] = grain[qn[b]];
        nx[b] = Vin[qn[b]];
        ny[b] = Vin[P.nc + qn[b]];
        nz[b] = Vin[2 * P.nc + qn[b]];
    }
    const Real vx = Vin[q], vy = Vin[P.nc + q], vz = Vin[2 * P.nc + q];
    const Real mx = m[q], my = m[P.nc + q], mz = m[2 * P.nc + q];
    const Real cex = coef[q], cK = coef[P.nc + q], alpha = coef[2 * P.nc + q];
    const Real a0 = first ? Real(0) : acc[q], a1 = first ? Real(0) : acc[P.nc + q],
               a2 = first ? Real(0) : acc[2 * P.nc + q];
    Real bx = 0, by = 0, bz = 0;
    if (V.H) {
        const V3<Real> b = V.at(P, cx, cy, cz, q);
        bx = b.x;
        by = b.y;
        bz = b.z;
    }
    if (g < 0) return;
    if ((cx >= ox && cx < ox + P.wx) || cx < c0 || cx >= c1) {  // a window or frozen cell: not evolved here
        if (last) return;
        Vout[q] = mx;
        Vout[P.nc + q] = my;
        Vout[2 * P.nc + q] = mz;
        return;
    }
    Real lx = 0, ly = 0, lz2 = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const bool on = has[b] && gn[b] == g;  // a select: a non-magnetic neighbour's values are never used
        lx += on ? nx[b] - vx : Real(0);
        ly += on ? ny[b] - vy : Real(0);
        lz2 += on ? nz[b] - vz : Real(0);
    }
    const Real ic2 = (Real)(1.0 / (P.cell * P.cell));
    lx *= ic2;
    ly *= ic2;
    lz2 *= ic2;
    const V3<Real> ba = field_at(P, F, (Real)((cx + 0.5) * P.cell));
    bx += ba.x;
    by += ba.y;
    bz += ba.z;
    const V3<Real> k = rhs<Real>((Real)P.gamma, alpha, vx, vy, vz, cex * lx + bx, cex * ly + by, cex * lz2 + cK * vz + bz);
    const Real s0 = a0 + w * k.x, s1 = a1 + w * k.y, s2 = a2 + w * k.z;
    if (last) {  // the RK4 update m + dt/6 (K1 + 2 K2 + 2 K3 + K4), renormalised; only this cell reads its m
        const Real h6 = (Real)P.dt / Real(6);
        const Real ux = mx + h6 * s0, uy = my + h6 * s1, uz = mz + h6 * s2;
        const Real nv = sqrt(ux * ux + uy * uy + uz * uz);
        m[q] = ux / nv;
        m[P.nc + q] = uy / nv;
        m[2 * P.nc + q] = uz / nv;
        return;
    }
    acc[q] = s0;
    acc[P.nc + q] = s1;
    acc[2 * P.nc + q] = s2;
    const Real dt = (Real)P.dt;
    Vout[q] = mx + c * dt * k.x;
    Vout[P.nc + q] = my + c * dt * k.y;
    Vout[2 * P.nc + q] = mz + c * dt * k.z;
}

// Sites move back by one cell column (the last column is thermalised afterwards).
template <typename Real>
__global__ void k_ms_shift(Real *Snew, const Real *Sold, MsDev P) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= P.nw) return;
    const int i = (int)(s % P.nxw);
    for (int d = 0; d < 3; ++d) Snew[d * P.nw + s] = i + P.r < P.nxw ? Sold[d * P.nw + s + P.r] : Real(0);
}

// Thermalisation of the sites of cell columns [cx0, cx1) (FP64 arithmetic): a spin in the cone
// of half-angle theta_max(m_e) around the cell's m, polar angle u0 theta_max and azimuth
// 2 pi u1 from e1 = (z x m)/|z x m| (or (x x m)/|x x m| when |m_z| >= 0.9), e2 = m x e1, with
// u0, u1 from Philox4x32-10 (key = seed, counter = (site low, site high, event low,
// event high | 2^31)).
template <typename Real>
__global__ void k_ms_thermalise(Real *S, const Real *m, const double *me, const int *grain, MsDev P, int ox, int cx0,
                                int cx1, unsigned long long event) {
    const long long ncolsites = (long long)(cx1 - cx0) * P.r;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= ncolsites * P.nyw * P.nzw) return;
    const int i = (cx0 - ox) * P.r + (int)(idx % ncolsites);
    const int j = (int)((idx / ncolsites) % P.nyw), k = (int)(idx / (ncolsites * P.nyw));
    const long long s = i + P.nxw * (j + (long long)P.nyw * k);
    const int q = cell_at(P, ox + i / P.r, j / P.r, k / P.r);
    const double mx = m[q], my = m[P.nc + q], mz = m[2 * P.nc + q];
    if (grain[q] < 0 || (mx == 0.0 && my == 0.0 && mz == 0.0)) {
        S[s] = S[P.nw + s] = S[2 * P.nw + s] = Real(0);
        return;
    }
    const double thm = theta_max(me[q]);
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
    S[s] = (Real)(a1 * e1x + a2 * e2x + a3 * mx);
    S[P.nw + s] = (Real)(a1 * e1y + a2 * e2y + a3 * my);
    S[2 * P.nw + s] = (Real)(a1 * e1z + a2 * e2z + a3 * mz);
}

// AoS FP64 (host layout) <-> component planes in the state's arithmetic
template <typename Real>
__global__ void k_aos_to_planes(const double *src, Real *dst, long long n) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int d = 0; d < 3; ++d) dst[d * n + s] = (Real)src[3 * s + d];
}

template <typename Real>
__global__ void k_planes_to_aos(const Real *src, double *dst, long long n) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int d = 0; d < 3; ++d) dst[3 * s + d] = (double)src[d * n + s];
}

__global__ void k_fill(double *v, double x, long long n) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < n) v[q] = x;
}

// Zero the cells that are non-magnetic.
template <typename Real>
__global__ void k_zero_void_cells(Real *m, const int *grain, long long nc) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nc || grain[q] >= 0) return;
    m[q] = m[nc + q] = m[2 * nc + q] = Real(0);
}

// Read-back: block b sums m_z over the magnetic cells whose centre x lies in
// [x_start + b L, x_start + (b + 1) L) and whose row lies in [cy0, cy1); each thread takes a
// fixed stride of the band and the block adds the partial sums in a fixed tree, so the result
// does not depend on scheduling.  signal[b] = mean m_z (0 without magnetic cells).
template <typename Real>
__global__ void k_ms_read_track(const Real *m, const int *grain, MsDev P, double x_start, double bit_len, int cy0,
                                int cy1, double *signal) {
    __shared__ double ssum[256];
    __shared__ long long scnt[256];
    const int b = blockIdx.x;
    const double lo = x_start + b * bit_len, hi = x_start + (b + 1) * bit_len;
    const long long nband = (long long)P.ncx * (cy1 - cy0) * P.ncz;
    double sum = 0.0;
    long long cnt = 0;
    for (long long idx = threadIdx.x; idx < nband; idx += blockDim.x) {
        const int cx = (int)(idx % P.ncx);
        const double x = (cx + 0.5) * P.cell;
        if (!(x >= lo && x < hi)) continue;
        const int cy = cy0 + (int)((idx / P.ncx) % (cy1 - cy0)), cz = (int)(idx / ((long long)P.ncx * (cy1 - cy0)));
        const int q = cell_at(P, cx, cy, cz);
        if (grain[q] < 0) continue;
        sum += (double)m[2 * P.nc + q];
        cnt += 1;
    }
    ssum[threadIdx.x] = sum;
    scnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ssum[threadIdx.x] += ssum[threadIdx.x + w];
            scnt[threadIdx.x] += scnt[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) signal[b] = scnt[0] > 0 ? ssum[0] / (double)scnt[0] : 0.0;
}

// ---- demagnetising field (Eq. 7): in x and y an FFT convolution on a zero-padded grid
// Px x Py, along z (a few cells) the direct sum over the planes: for every in-plane frequency
// (kx, ky), H^(t) = sum over planes z' of N^(t - z') M^(z'), N^(d) the in-plane transform of
// the tensor at z offset d.  The same convolution as a 3-D transform padded along z, with
// half the transformed points and no transform along z.
struct Pad {
    int Px, Py, Pz;       // padded x, y; Pz = the track's planes (not padded)
    long long Ptot, Pc;   // real points, complex points (Px / 2 + 1 along x), all planes
    long long Pc2;        // complex points of one plane
};

// The cells' magnetisation in the padded layout of a grid whose first column is g0 (ncol
// columns): window cells M = (mu_s / V) sum of their spins (Eq. 6; wn holds the sum's length
// and m its direction, from the window average of the same state), other magnetic cells
// M = Ms0 m_e m (a frozen cell's m_e is the stored one), non-magnetic cells and columns beyond
// the track 0.  mode selects the sources: 0 every cell, 1 the columns [s0, s1) only, 2 all
// but those, 3 the magnetisation Mg [3][nc] given for every cell.
template <typename Real>
__global__ void k_demag_M(Real *Mpad, const Real *wn, const Real *m, const double *me, const int *grain, MsDev P,
                          Pad pd, int ox, int g0, int ncol, int s0, int s1, int mode, const Real *Mg) {
    int i, cy, cz;
    if (!coords(ncol, P.ncy, i, cy, cz)) return;
    const int cx = g0 + i;
    const long long pp = i + (long long)pd.Px * (cy + (long long)pd.Py * cz);
    Real Mx = 0, My = 0, Mz = 0;
    const int q = cx < P.ncx ? cell_at(P, cx, cy, cz) : 0;
    if (mode == 3) {
        if (cx < P.ncx) {
            Mx = Mg[q];
            My = Mg[P.nc + q];
            Mz = Mg[2 * P.nc + q];
        }
    } else if (cx < P.ncx && grain[q] >= 0 && (mode == 0 || (mode == 1) == (cx >= s0 && cx < s1))) {
        // a window cell: (mu_s / V) |sum of its sites| times their direction, both from Eq. 6
        // of this step; a cell outside: Ms0 m_e(T) m
        const Real a = (cx >= ox && cx < ox + P.wx) ? (Real)(P.mu_s / (P.cell * P.cell * P.cell)) * wn[q]
                                                    : (Real)(P.Ms0 * me[q]);
        Mx = a * m[q];
        My = a * m[P.nc + q];
        Mz = a * m[2 * P.nc + q];
    }
    Mpad[pp] = Mx;
    Mpad[pd.Ptot + pp] = My;
    Mpad[2 * pd.Ptot + pp] = Mz;
}

// The in-plane transform of each tensor component is real or imaginary: on the padded grid
// xx, yy, zz are even in x and in y, xy odd in both (real transforms), xz odd in x and even in
// y, yz the reverse (imaginary).  N^ is kept as one real per component: the real part of xx,
// yy, zz, xy, the imaginary part of xz, yz.
// h += N m for the tensor r at z offset +d (neg = false) or -d (neg = true: N is even in z
// but for xz and yz, which are odd)
template <typename C, typename R>
__device__ __forceinline__ void tmac(C h[3], const R r[6], const C m[3], bool neg) {
    auto re = [](C &a, R c, const C &b) {  // a += c b
        a.x += c * b.x;
        a.y += c * b.y;
    };
    auto im = [](C &a, R c, const C &b) {  // a += (i c) b
        a.x -= c * b.y;
        a.y += c * b.x;
    };
    const R xz = neg ? -r[4] : r[4], yz = neg ? -r[5] : r[5];
    re(h[0], r[0], m[0]);
    re(h[0], r[3], m[1]);
    im(h[0], xz, m[2]);
    re(h[1], r[3], m[0]);
    re(h[1], r[1], m[1]);
    im(h[1], yz, m[2]);
    im(h[2], xz, m[0]);
    im(h[2], yz, m[1]);
    re(h[2], r[2], m[2]);
}

// The compressed tensor [6][Pz][Pc2] from its full in-plane transforms Nc [6][Pz][Pc2].
template <typename C, typename R>
__global__ void k_demag_tensor_compress(R *Nr, const C *Nc, long long Pc) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= 6 * Pc) return;
    Nr[k] = k < 4 * Pc ? Nc[k].x : Nc[k].y;
}

// H^ [3][Pz][Pc2] from M^ [3][Pz][Pc2] and N^ [6][Pz][Pc2] (offsets 0 .. Pz - 1): one thread
// per in-plane frequency and target plane t, summing over the source planes.
template <typename C, typename R>
__global__ void k_demag_zmul(C *Hh, const C *Mh, const R *Nr, long long Pc2, int Pz) {
    const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (f >= Pc2) return;
    const long long Pc = Pc2 * Pz;
    C h[3];
    for (int c = 0; c < 3; ++c) h[c].x = h[c].y = 0;
    for (int z = 0; z < Pz; ++z) {
        const int d = t - z, ad = d < 0 ? -d : d;
        R n[6];
        C m[3];
        for (int c = 0; c < 6; ++c) n[c] = Nr[c * Pc + ad * Pc2 + f];
        for (int c = 0; c < 3; ++c) m[c] = Mh[c * Pc + z * Pc2 + f];
        tmac(h, n, m, d < 0);
    }
    for (int c = 0; c < 3; ++c) Hh[c * Pc + t * Pc2 + f] = h[c];
}

// global -> shared copies that hold no register while in flight, and the wait for all of the
// calling thread's copies
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The same in FP32 for NZ planes (a compile-time count).  A block takes 32 frequencies; its
// NP = min(NZ, 4) parts split the target planes (part p: t = p, p + NP, ...), so that a small
// grid still has several warps per scheduler.  The block stages M^ and N^ of its
// frequencies in shared memory (copies all in flight at once, one barrier); each thread holds
// the NZ source vectors in registers and reads each tensor value where a pair needs it.
template <int NZ>
__global__ void __launch_bounds__(32 * (NZ < 4 ? NZ : 4))
    k_demag_zmul_r(float2 *Hh, const float2 *Mh, const float *Nr, long long Pc2) {
    constexpr int NP = NZ < 4 ? NZ : 4;
    __shared__ float2 sM[3 * NZ][32];
    __shared__ float sN[6 * NZ][32];
    const int tx = threadIdx.x, p = threadIdx.y;
    const long long f = blockIdx.x * 32LL + tx;
    const bool act = f < Pc2;
    const long long Pc = Pc2 * NZ;
    if (act) {
        for (int k = p; k < 3 * NZ; k += NP) cp_async8(&sM[k][tx], &Mh[k * Pc2 + f]);
        for (int k = p; k < 6 * NZ; k += NP) cp_async4(&sN[k][tx], &Nr[k * Pc2 + f]);
    }
    cp_async_wait_all();
    __syncthreads();
    if (!act) return;
    float2 m[NZ][3];
#pragma unroll
    for (int z = 0; z < NZ; ++z)
#pragma unroll
        for (int c = 0; c < 3; ++c) m[z][c] = sM[c * NZ + z][tx];
#pragma unroll
    for (int t0 = 0; t0 < NZ; t0 += NP) {
        const int t = t0 + p;
        if (t >= NZ) break;
        float2 h[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c].x = h[c].y = 0.f;
#pragma unroll
        for (int z = 0; z < NZ; ++z) {
            const int d = t - z, ad = d < 0 ? -d : d;
            float r[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) r[c] = sN[c * NZ + ad][tx];
            tmac(h, r, m[z], d < 0);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) Hh[c * Pc + t * Pc2 + f] = h[c];
    }
}

// B_d = -mu0 H on the cells of the target columns [t0, t1) of a grid whose first column is g0
// (the inverse in-plane transform is unnormalised: divide by Px Py), plus `add` where given.
template <typename Real>
__global__ void k_demag_extract(Real *Bd, const Real *Hpad, MsDev P, Pad pd, int g0, int ncol, int t0, int t1,
                                const Real *add) {
    int i, cy, cz;
    if (!coords(ncol, P.ncy, i, cy, cz)) return;
    const int cx = g0 + i;
    if (cx < t0 || cx >= t1 || cx >= P.ncx) return;
    const int q = cell_at(P, cx, cy, cz);
    const long long pp = i + (long long)pd.Px * (cy + (long long)pd.Py * cz);
    const Real s = (Real)(-1.25663706212e-6 / ((double)pd.Px * pd.Py));
    Real bx = s * Hpad[pp], by = s * Hpad[pd.Ptot + pp], bz = s * Hpad[2 * pd.Ptot + pp];
    if (add) {
        bx += add[q];
        by += add[P.nc + q];
        bz += add[2 * P.nc + q];
    }
    Bd[q] = bx;
    Bd[P.nc + q] = by;
    Bd[2 * P.nc + q] = bz;
}

// One convolution grid of Eq. 7 over ncol cell columns (all of y and z): the tensor's in-plane
// spectra [6][Pz][Pc2] (one real each), the padded M | H buffer [6][Ptot], the transformed
// M | H [6][Pc] and the cuFFT plans (3 Pz in-plane transforms per call).
struct DemagGrid {
    int ncol = 0;
    Pad pd{};
    void *Nh = nullptr, *Mpad = nullptr, *Mh = nullptr;
    cufftHandle plan_f = 0, plan_b = 0;
    bool plans = false;
};

void demag_grid_free(DemagGrid &g) {
    void **b[] = {&g.Nh, &g.Mpad, &g.Mh};
    for (void **p : b)
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    if (g.plans) {
        cufftDestroy(g.plan_f);
        cufftDestroy(g.plan_b);
        g.plans = false;
    }
    g.ncol = 0;
}


constexpr int BLK = 256;
inline unsigned nblk(long long n) { return (unsigned)((n + BLK - 1) / BLK); }
inline dim3 grid3(int nx, int ny, int nz) { return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + 3) / 4), (unsigned)nz); }
const dim3 BLK3(32, 4, 1);

}  // namespace

struct hamr_ms_ctx {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // a second stream for the parts of a step that do not depend on one another, and the
    // events that fork it from the handle's stream and join it back
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    MsDev P{};
    ReplicaDev D{};               // laser spot and write field (the atomistic driver fields)
    std::vector<uint8_t> bits_h;
    uint8_t *bits_d = nullptr;
    int *grain_d = nullptr;
    std::vector<int> grain_h;
    std::vector<unsigned long long> colmask_h;
    int prec = HAMR_FP64;         // arithmetic of the state and the field (HAMR_FP32 / HAMR_FP64)
    // state-precision planes: cells m, V0, V1, acc, coef [3][nc]; window S, S2 [3][nw]
    void *m = nullptr, *V0 = nullptr, *V1 = nullptr, *acc = nullptr, *coef = nullptr;
    void *S = nullptr, *S2 = nullptr;
    void *wn = nullptr;           // |sum of the sites| of each window cell (Eq. 6), state precision
    double *me = nullptr;         // m_e per cell (FP64)
    double *col = nullptr;        // per cell column [3][ncx ncy]: T of the last m_e solve, m_e, the m_e before (NaN: none)
    unsigned long long *colmask = nullptr;  // per cell column: bit z set for a magnetic cell (z < 64)
    double Bm_last = NAN;         // field magnitude of the last m_e solve
    double *stage = nullptr;      // AoS FP64 staging for host copies
    int ox = -1;                  // window column (-1: not placed)
    int margin = -1;              // simulated region: the window and `margin` columns on each side (< 0: the track)
    long long step = 0;
    long long events = 0;         // thermalisation events so far
    bool grains_set = false, cells_set = false;
    bool window_live = false;     // the window's sites are newer than its cells (placed, cells not replaced since)
    // demagnetising field (Eq. 7): the track's padded grid and, with a simulated region, the
    // region's (B_d is read from the grid's inverse transform where it is used); the frozen
    // cells' part of B_d on the region's cells [3][nc], valid for the region [fz_c0, fz_c1)
    // until the frozen cells change
    bool demag = false;
    DemagGrid gtrack, gregion;
    void *Bfz = nullptr;
    int fz_c0 = -1, fz_c1 = -1;
    bool fz_dirty = true;
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
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
        h->side = nullptr;
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->ev_fork = h->ev_join = nullptr;
    void **bufs[] = {&h->m, &h->V0, &h->V1, &h->acc, &h->coef, &h->S, &h->S2};
    for (void **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    void **dbufs[] = {&h->Bfz};
    for (void **b : dbufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    demag_grid_free(h->gtrack);
    demag_grid_free(h->gregion);
    if (h->wn) cudaFree(h->wn);
    if (h->me) cudaFree(h->me);
    if (h->col) cudaFree(h->col);
    if (h->colmask) cudaFree(h->colmask);
    if (h->stage) cudaFree(h->stage);
    h->wn = nullptr;
    h->me = nullptr;
    h->col = nullptr;
    h->colmask = nullptr;
    h->stage = nullptr;
    if (h->grain_d) cudaFree(h->grain_d);
    if (h->bits_d) cudaFree(h->bits_d);
    h->grain_d = nullptr;
    h->bits_d = nullptr;
}

// FP32 copies of the driver parameters (read by the FP32 kernels)
void set_driver_floats(ReplicaDev &D) {
    D.fT_amb = (float)D.T_amb;
    D.fdT = (float)D.dT;
    D.fc_fwhm = (float)D.c_fwhm;
    D.fx0 = (float)D.x0;
    D.fy0 = (float)D.y0;
    D.fvx = (float)D.vx;
    D.fvy = (float)D.vy;
    D.fB0 = (float)D.B0;
    for (int k = 0; k < 3; ++k) D.fdir[k] = (float)D.dir[k];
    D.fbit_len = (float)D.bit_len;
    D.framp_len = (float)D.ramp_len;
    D.fhead_x0 = (float)D.head_x0;
    D.fhead_v = (float)D.head_v;
}

// The polarity s(t) of the bit pattern, computed as on the device: linear ramp from bit b-1's
// polarity to bit b's over the first ramp_len of bit b, 1 without a pattern.
double polarity_host(const hamr_ms_t h, double t) {
    const ReplicaDev &D = h->D;
    if (D.n_bits <= 0) return 1.0;
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
    return pol(b - 1) + (pol(b) - pol(b - 1)) * w;
}

// B0 s(t) dir
void applied_host(const hamr_ms_t h, double t, double B[3]) {
    const double s = polarity_host(h, t);
    for (int d = 0; d < 3; ++d) B[d] = h->D.B0 * s * h->D.dir[d];
}

// |B0 s(t) dir|, the uniform field's magnitude (the m_e solve of a cell is kept while this and
// the cell's temperature are unchanged)
double field_magnitude_host(const hamr_ms_t h, double t) {
    double B[3];
    applied_host(h, t, B);
    return sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
}

// The write field of time t for the kernels: B0 s(t) dir, Bx0 s(t) and the head position
template <typename Real>
Field<Real> field_of(const hamr_ms_t h, double t) {
    double B[3];
    applied_host(h, t, B);
    Field<Real> F;
    F.bx = (Real)B[0];
    F.by = (Real)B[1];
    F.bz = (Real)B[2];
    F.bxs = (Real)(h->P.pBx0 * polarity_host(h, t));
    F.xh = (Real)(h->D.head_x0 + h->D.head_v * t);
    return F;
}

// ---- demagnetising tensor of cuboid cells (Newell, Williams and Dunlop, J. Geophys. Res. 98,
// 9551 (1993)): the second difference over the cell edges of f (diagonal) and g (off-diagonal)
// divided by 4 pi dx dy dz; beyond 40 cell edges the point-dipole tensor
// -(V / 4 pi r^3)(3 r r / r^2 - I), where the second difference cancels to rounding.
double nw_asinh(double a, double b) { return b > 0.0 ? asinh(a / b) : 0.0; }
double nw_atan(double a, double b) { return b != 0.0 ? atan(a / b) : 0.0; }

double newell_f(double x, double y, double z) {
    x = fabs(x);
    y = fabs(y);
    z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    return 0.5 * y * (z2 - x2) * nw_asinh(y, sqrt(x2 + z2)) + 0.5 * z * (y2 - x2) * nw_asinh(z, sqrt(x2 + y2)) -
           x * y * z * nw_atan(y * z, x * R) + (2.0 * x2 - y2 - z2) * R / 6.0;
}

double newell_g(double x, double y, double z) {
    const double sg = (x < 0 ? -1.0 : 1.0) * (y < 0 ? -1.0 : 1.0);   // odd in x and y, even in z
    x = fabs(x);
    y = fabs(y);
    z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    const double r = x * y * z * nw_asinh(z, sqrt(x2 + y2)) + y * (3.0 * z2 - y2) * nw_asinh(x, sqrt(y2 + z2)) / 6.0 +
                     x * (3.0 * z2 - x2) * nw_asinh(y, sqrt(x2 + z2)) / 6.0 - z2 * z * nw_atan(x * y, z * R) / 6.0 -
                     0.5 * z * y2 * nw_atan(x * z, y * R) - 0.5 * z * x2 * nw_atan(y * z, x * R) - x * y * R / 3.0;
    return sg * r;
}

template <typename Fn>
double second_diff(Fn F, double X, double Y, double Z, double d) {
    const double c[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j)
            for (int k = -1; k <= 1; ++k) s += c[i + 1] * c[j + 1] * c[k + 1] * F(X + i * d, Y + j * d, Z + k * d);
    return s;
}

// (xx, yy, zz, xy, xz, yz) between cubic cells of edge d at offset (X, Y, Z)
void demag_tensor(double X, double Y, double Z, double d, double N[6]) {
    const double r = sqrt(X * X + Y * Y + Z * Z);
    if (r > 40.0 * d) {
        const double pre = -d * d * d / (4.0 * M_PI * r * r * r), r2 = r * r;
        N[0] = pre * (3.0 * X * X / r2 - 1.0);
        N[1] = pre * (3.0 * Y * Y / r2 - 1.0);
        N[2] = pre * (3.0 * Z * Z / r2 - 1.0);
        N[3] = pre * 3.0 * X * Y / r2;
        N[4] = pre * 3.0 * X * Z / r2;
        N[5] = pre * 3.0 * Y * Z / r2;
        return;
    }
    const double k = 1.0 / (4.0 * M_PI * d * d * d);
    N[0] = k * second_diff([](double x, double y, double z) { return newell_f(x, y, z); }, X, Y, Z, d);
    N[1] = k * second_diff([](double x, double y, double z) { return newell_f(y, x, z); }, X, Y, Z, d);
    N[2] = k * second_diff([](double x, double y, double z) { return newell_f(z, y, x); }, X, Y, Z, d);
    N[3] = k * second_diff([](double x, double y, double z) { return newell_g(x, y, z); }, X, Y, Z, d);
    N[4] = k * second_diff([](double x, double y, double z) { return newell_g(x, z, y); }, X, Y, Z, d);
    N[5] = k * second_diff([](double x, double y, double z) { return newell_g(y, z, x); }, X, Y, Z, d);
}

// offset of padded index i along an axis of n cells padded to P (INT32_MIN: not a cell offset)
int pad_offset(int i, int n, int P) {
    if (i < n) return i;
    if (i > P - n) return i - P;
    return INT32_MIN;
}

// The tensor of Eq. 7 on the padded grid of ncol columns (host, FP64, in parallel over z
// planes), its transform and the plans.
template <typename Real>
int demag_grid_setup(hamr_ms_t h, DemagGrid &g, int ncol) {
    typedef typename std::conditional<sizeof(Real) == 8, cufftDoubleComplex, cufftComplex>::type C;
    const MsDev &P = h->P;
    Pad &pd = g.pd;
    g.ncol = ncol;
    pd.Px = ncol > 1 ? 2 * ncol : 1;
    pd.Py = P.ncy > 1 ? 2 * P.ncy : 1;
    pd.Pz = P.ncz;
    pd.Ptot = (long long)pd.Px * pd.Py * pd.Pz;
    pd.Pc2 = (long long)(pd.Px / 2 + 1) * pd.Py;
    pd.Pc = pd.Pc2 * pd.Pz;
    // plane d of component c: the tensor at z offset d (>= 0), padded in x and y
    std::vector<double> T(6 * (size_t)pd.Ptot, 0.0);
    const unsigned nth = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            for (int k = (int)w; k < pd.Pz; k += (int)nth) {
                const int Z = k;
                for (int j = 0; j < pd.Py; ++j) {
                    const int Y = pad_offset(j, P.ncy, pd.Py);
                    if (Y == INT32_MIN) continue;
                    for (int i = 0; i < pd.Px; ++i) {
                        const int X = pad_offset(i, ncol, pd.Px);
                        if (X == INT32_MIN) continue;
                        double N[6];
                        demag_tensor(X * P.cell, Y * P.cell, Z * P.cell, P.cell, N);
                        const long long pp = i + (long long)pd.Px * (j + (long long)pd.Py * k);
                        for (int c = 0; c < 6; ++c) T[(size_t)c * pd.Ptot + pp] = N[c];
                    }
                }
            }
        });
    for (auto &t : pool) t.join();
    std::vector<Real> Tr(T.begin(), T.end());
    MSCK(h, cudaMalloc(&g.Nh, sizeof(Real) * 6 * pd.Pc));
    MSCK(h, cudaMalloc(&g.Mh, sizeof(C) * 6 * pd.Pc));
    // [M | H], each 3 padded grids; the tensor's six components pass through it once at setup
    MSCK(h, cudaMalloc(&g.Mpad, sizeof(Real) * 6 * pd.Ptot));
    int n[2] = {pd.Py, pd.Px};
    const bool dbl = sizeof(Real) == 8;
    const int P2 = pd.Px * pd.Py;
    if (cufftPlanMany(&g.plan_f, 2, n, nullptr, 1, P2, nullptr, 1, (int)pd.Pc2, dbl ? CUFFT_D2Z : CUFFT_R2C,
                      3 * pd.Pz) != CUFFT_SUCCESS ||
        cufftPlanMany(&g.plan_b, 2, n, nullptr, 1, (int)pd.Pc2, nullptr, 1, P2, dbl ? CUFFT_Z2D : CUFFT_C2R,
                      3 * pd.Pz) != CUFFT_SUCCESS)
        return msfail(h, HAMR_ERR_CUDA, "cuFFT plan creation failed for %d planes of %d x %d", pd.Pz, pd.Px, pd.Py);
    g.plans = true;
    cufftSetStream(g.plan_f, h->stream);
    cufftSetStream(g.plan_b, h->stream);
    MSCK(h, cudaMemcpyAsync(g.Mpad, Tr.data(), sizeof(Real) * 6 * pd.Ptot, cudaMemcpyHostToDevice, h->stream));
    for (int half = 0; half < 2; ++half) {
        Real *src = (Real *)g.Mpad + (size_t)half * 3 * pd.Ptot;
        C *dst = (C *)g.Mh + (size_t)half * 3 * pd.Pc;
        const cufftResult r = dbl ? cufftExecD2Z(g.plan_f, (cufftDoubleReal *)src, (cufftDoubleComplex *)dst)
                                  : cufftExecR2C(g.plan_f, (cufftReal *)src, (cufftComplex *)dst);
        if (r != CUFFT_SUCCESS) return msfail(h, HAMR_ERR_CUDA, "cuFFT forward transform of the tensor failed");
    }
    k_demag_tensor_compress<C, Real><<<nblk(6 * pd.Pc), BLK, 0, h->stream>>>((Real *)g.Nh, (const C *)g.Mh, pd.Pc);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaMemsetAsync(g.Mpad, 0, sizeof(Real) * 6 * pd.Ptot, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

// The register-blocked z sum for FP32 and a track of 1 to 10 planes (false: not taken).
template <typename C, typename R>
bool demag_zmul_r(C *Hh, const C *Mh, const R *Nr, const Pad &pd, cudaStream_t st) {
    if (!std::is_same<C, cufftComplex>::value) return false;
    const unsigned nb = (unsigned)((pd.Pc2 + 31) / 32);
    float2 *H = (float2 *)Hh;
    const float2 *M = (const float2 *)Mh;
    const float *N = (const float *)Nr;
    switch (pd.Pz) {
#define ZMUL_R(NZ)                                                                    \
    case NZ:                                                                          \
        k_demag_zmul_r<NZ><<<nb, dim3(32, NZ < 4 ? NZ : 4), 0, st>>>(H, M, N, pd.Pc2); \
        return true;
        ZMUL_R(1) ZMUL_R(2) ZMUL_R(3) ZMUL_R(4) ZMUL_R(5)
        ZMUL_R(6) ZMUL_R(7) ZMUL_R(8) ZMUL_R(9) ZMUL_R(10)
#undef ZMUL_R
        default: return false;
    }
}

// The demagnetising field on the target columns [t0, t1) from the sources that `mode` selects
// (k_demag_M), through grid g placed at column g0, into out (plus `add` where given; out null:
// left in the grid's inverse transform, for a BdView).
template <typename Real>
int demag_pass(hamr_ms_t h, DemagGrid &g, int g0, int mode, int s0, int s1, Real *out, int t0, int t1,
               const Real *add, const Real *Mg = nullptr) {
    typedef typename std::conditional<sizeof(Real) == 8, cufftDoubleComplex, cufftComplex>::type C;
    const MsDev &P = h->P;
    const Pad &pd = g.pd;
    const dim3 gc = grid3(g.ncol, P.ncy, P.ncz);
    k_demag_M<Real><<<gc, BLK3, 0, h->stream>>>((Real *)g.Mpad, (const Real *)h->wn, (const Real *)h->m, h->me,
                                                h->grain_d, P, pd, h->ox, g0, g.ncol, s0, s1, mode, Mg);
    MSCK(h, cudaGetLastError());
    const bool dbl = sizeof(Real) == 8;
    cufftResult r = dbl ? cufftExecD2Z(g.plan_f, (cufftDoubleReal *)g.Mpad, (cufftDoubleComplex *)g.Mh)
                        : cufftExecR2C(g.plan_f, (cufftReal *)g.Mpad, (cufftComplex *)g.Mh);
    if (r != CUFFT_SUCCESS) return msfail(h, HAMR_ERR_CUDA, "cuFFT forward transform failed");
    C *Hh = (C *)g.Mh + 3 * pd.Pc;
    if (!demag_zmul_r<C, Real>(Hh, (const C *)g.Mh, (const Real *)g.Nh, pd, h->stream)) {
        const dim3 gz(nblk(pd.Pc2), (unsigned)pd.Pz);
        k_demag_zmul<C, Real><<<gz, BLK, 0, h->stream>>>(Hh, (const C *)g.Mh, (const Real *)g.Nh, pd.Pc2, pd.Pz);
    }
    MSCK(h, cudaGetLastError());
    // H goes to the second half of the buffer: the padding of M (first half) must stay zero
    Real *H = (Real *)g.Mpad + 3 * pd.Ptot;
    r = dbl ? cufftExecZ2D(g.plan_b, (cufftDoubleComplex *)Hh, (cufftDoubleReal *)H)
            : cufftExecC2R(g.plan_b, (cufftComplex *)Hh, (cufftReal *)H);
    if (r != CUFFT_SUCCESS) return msfail(h, HAMR_ERR_CUDA, "cuFFT inverse transform failed");
    if (out) k_demag_extract<Real><<<gc, BLK3, 0, h->stream>>>(out, H, P, pd, g0, g.ncol, t0, t1, add);
    MSCK(h, cudaGetLastError());
    return HAMR_OK;
}

// The simulated region's cell columns [c0, c1): the window and `margin` columns on each side,
// within the track (the whole track when margin < 0).
void ms_region(const hamr_ms_t h, int &c0, int &c1) {
    if (h->margin < 0) {
        c0 = 0;
        c1 = h->P.ncx;
        return;
    }
    c0 = std::max(0, h->ox - h->margin);
    c1 = std::min(h->P.ncx, h->ox + h->P.wx + h->margin);
}

// B_d = -mu0 N * M of the current state (the m_e of each cell must be current).  With a
// simulated region only its cells need B_d: their own part is a convolution over the region's
// padded grid, every step; the frozen cells' part is a convolution over the track's grid with
// the region left out, kept until the region moves or the frozen cells change.
template <typename Real>
BdView<Real> bd_view(const DemagGrid &g, int g0, const Real *add) {
    BdView<Real> V;
    V.H = (const Real *)g.Mpad + 3 * g.pd.Ptot;
    V.add = add;
    V.Ptot = g.pd.Ptot;
    V.Px = g.pd.Px;
    V.Py = g.pd.Py;
    V.g0 = g0;
    V.ncol = g.ncol;
    V.s = (Real)(-1.25663706212e-6 / ((double)g.pd.Px * g.pd.Py));
    return V;
}

template <typename Real>
int ms_demag_step(hamr_ms_t h, BdView<Real> &V) {
    const MsDev &P = h->P;
    int c0, c1;
    ms_region(h, c0, c1);
    const int L = h->margin < 0 ? P.ncx : std::min(P.ncx, P.wx + 2 * h->margin);
    if (L >= P.ncx) {
        V = bd_view<Real>(h->gtrack, 0, nullptr);
        return demag_pass<Real>(h, h->gtrack, 0, 0, 0, P.ncx, (Real *)nullptr, 0, P.ncx, nullptr);
    }
    if (h->gregion.ncol != L) {
        demag_grid_free(h->gregion);
        int rc = demag_grid_setup<Real>(h, h->gregion, L);
        if (rc) return rc;
    }
    if (h->fz_dirty || c0 != h->fz_c0 || c1 != h->fz_c1) {
        int rc = demag_pass<Real>(h, h->gtrack, 0, 2, c0, c1, (Real *)h->Bfz, c0, c1, nullptr);
        if (rc) return rc;
        h->fz_c0 = c0;
        h->fz_c1 = c1;
        h->fz_dirty = false;
    }
    V = bd_view<Real>(h->gregion, c0, (const Real *)h->Bfz);
    return demag_pass<Real>(h, h->gregion, c0, 1, c0, c1, (Real *)nullptr, c0, c1, nullptr);
}

// Thermalise the window sites of cell columns [cx0, cx1) at time t.  m_e(T) is solved first
// on every cell (all = true: a placement, which also gives every frozen cell its m_e) or on
// the simulated region (a move; the cells that just froze keep theirs).
template <typename Real>
int ms_thermalise(hamr_ms_t h, int cx0, int cx1, double t, bool all) {
    const long long n = (long long)(cx1 - cx0) * h->P.r * h->P.nyw * h->P.nzw;
    if (n <= 0) return HAMR_OK;
    int c0 = 0, c1 = h->P.ncx;
    if (!all) ms_region(h, c0, c1);
    const double Bm = field_magnitude_host(h, t);
    k_mm_prep<Real><<<grid3(c1 - c0, h->P.ncy, 1), BLK3, 0, h->stream>>>(
        h->me, h->col, (Real *)h->coef, h->grain_d, h->colmask, h->P, h->D, t, field_of<double>(h, t), h->Bm_last,
        c0, c1 - c0);
    h->Bm_last = Bm;
    k_ms_thermalise<Real><<<nblk(n), BLK, 0, h->stream>>>((Real *)h->S, (const Real *)h->m, h->me, h->grain_d, h->P,
                                                          h->ox, cx0, cx1, (unsigned long long)h->events);
    MSCK(h, cudaGetLastError());
    h->events += 1;
    return HAMR_OK;
}

template <typename Real>
int ms_average(hamr_ms_t h, int cx0, int ncol, cudaStream_t st = nullptr) {
    if (!st) st = h->stream;
    const MsDev &P = h->P;
    const long long n = (long long)ncol * P.ncy * P.ncz;
    Real *m = (Real *)h->m, *wn = (Real *)h->wn;
    const Real *S = (const Real *)h->S;
#define MS_AVG(RT)                                                                                       \
    do {                                                                                                 \
        const long long nthr = 32LL * ((ncol + 32 / RT - 1) / (32 / RT)) * P.ncy * P.ncz;                \
        k_ms_average_w<Real, RT><<<nblk(nthr), BLK, 0, st>>>(m, wn, S, h->grain_d, P, h->ox, cx0, ncol);         \
    } while (0)
    switch (P.r) {
        case 1: MS_AVG(1); break;
        case 2: MS_AVG(2); break;
        case 4: MS_AVG(4); break;
        default:
            k_ms_average<Real><<<nblk(n), BLK, 0, st>>>(m, wn, S, h->grain_d, P, h->ox, cx0, ncol);
            break;
    }
#undef MS_AVG
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
template <typename Real>
int ms_step(hamr_ms_t h) {
    const MsDev &P = h->P;
    cudaStream_t st = h->stream, sd = h->side;
    // Eq. 6 of the window cells (window cells only) and the m_e solve (coefficients only) are
    // independent; the window step reads neither (its x faces see cells outside the window),
    // but with Eq. 7 it reads B_d, which needs both.  RK4 stages 0-2 write only the stage
    // buffers and the accumulator; the last stage writes m, which the window step reads at its
    // faces.  So the side stream takes Eq. 6, the m_e solve (without Eq. 7) and stages 0-2
    // beside the window step, and the last stage waits for both streams.
    MSCK(h, cudaEventRecord(h->ev_fork, st));
    MSCK(h, cudaStreamWaitEvent(sd, h->ev_fork, 0));
    int rc = ms_average<Real>(h, h->ox, P.wx, sd);
    if (rc) return rc;
    cudaStream_t sp = h->demag ? st : sd;  // the m_e solve's stream
    Real *S = (Real *)h->S, *m = (Real *)h->m;
    const double t = (double)h->step * P.dt;
    const Field<Real> F = field_of<Real>(h, t);
    // m_e(T) at t_n of every cell of the simulated region (frozen cells keep theirs), then
    // (optionally) the demagnetising field of the state at t_n
    int c0, c1;
    ms_region(h, c0, c1);
    const int e0 = std::max(0, c0 - 1), e1 = std::min(P.ncx, c1 + 1);
    const double Bm = field_magnitude_host(h, t);
    k_mm_prep<Real><<<grid3(c1 - c0, P.ncy, 1), BLK3, 0, sp>>>(h->me, h->col, (Real *)h->coef, h->grain_d, h->colmask, P,
                                                              h->D, t, field_of<double>(h, t), h->Bm_last, c0, c1 - c0);
    h->Bm_last = Bm;
    MSCK(h, cudaGetLastError());
    BdView<Real> Bd;  // H null: no demagnetising field
    if (h->demag) {
        MSCK(h, cudaEventRecord(h->ev_join, sd));
        MSCK(h, cudaStreamWaitEvent(st, h->ev_join, 0));
        if ((rc = ms_demag_step<Real>(h, Bd))) return rc;
        MSCK(h, cudaEventRecord(h->ev_fork, st));
        MSCK(h, cudaStreamWaitEvent(sd, h->ev_fork, 0));
    }
    const Real cst[4] = {Real(0.5), Real(0.5), Real(1), Real(0)}, wst[4] = {Real(1), Real(2), Real(2), Real(1)};
    auto stage = [&](int s, cudaStream_t ss) {
        const Real *vin = s == 0 ? (const Real *)m : (const Real *)((s & 1) ? h->V1 : h->V0);
        Real *vout = (Real *)((s & 1) ? h->V0 : h->V1);
        k_mm_stage<Real><<<grid3(e1 - e0, P.ncy, P.ncz), BLK3, 0, ss>>>(vin, vout, (Real *)h->acc, m,
                                                                        (const Real *)h->coef, h->grain_d, P, h->ox,
                                                                        F, Bd, cst[s], wst[s], s == 0, s == 3, e0,
                                                                        e1 - e0, c0, c1);
    };
    for (int s = 0; s < 3; ++s) stage(s, sd);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaEventRecord(h->ev_join, sd));
    // both Heun stages of the window in one pass, into the second buffer
    const dim3 gw((unsigned)((P.nxw + MWX - 1) / MWX), (unsigned)((P.nyw + MWY - 1) / MWY),
                  (unsigned)((P.nzw + MWZ - 1) / MWZ));
    const size_t shm = sizeof(V4<Real>) * 7 * MWPOS;
#define MS_HEUN(RT)                                                                                         \
    do {                                                                                                    \
        MSCK(h, cudaFuncSetAttribute(k_ms_fused<Real, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                     (int)shm));                                                           \
        k_ms_fused<Real, RT><<<gw, MWT, shm, st>>>(S, (Real *)h->S2, m, h->grain_d, P, h->D, F, Bd, h->ox, \
                                                   h->step);                                               \
    } while (0)
    switch (P.r) {
        case 1: MS_HEUN(1); break;
        case 2: MS_HEUN(2); break;
        case 4: MS_HEUN(4); break;
        default: MS_HEUN(0); break;
    }
#undef MS_HEUN
    MSCK(h, cudaGetLastError());
    std::swap(h->S, h->S2);
    MSCK(h, cudaStreamWaitEvent(st, h->ev_join, 0));
    stage(3, st);
    MSCK(h, cudaGetLastError());
    h->step += 1;
    return HAMR_OK;
}

template <typename Real>
int ms_shift_forward(hamr_ms_t h, double t) {
    int rc = ms_average<Real>(h, h->ox, 1);
    if (rc) return rc;
    k_ms_shift<Real><<<nblk(h->P.nw), BLK, 0, h->stream>>>((Real *)h->S2, (const Real *)h->S, h->P);
    MSCK(h, cudaGetLastError());
    std::swap(h->S, h->S2);
    h->ox += 1;
    return ms_thermalise<Real>(h, h->ox + h->P.wx - 1, h->ox + h->P.wx, t, false);
}

// host FP64 AoS (already in h->stage) -> state planes, and back
int ms_to_planes(hamr_ms_t h, void *dst, long long n) {
    if (h->prec == HAMR_FP64)
        k_aos_to_planes<double><<<nblk(n), BLK, 0, h->stream>>>(h->stage, (double *)dst, n);
    else
        k_aos_to_planes<float><<<nblk(n), BLK, 0, h->stream>>>(h->stage, (float *)dst, n);
    MSCK(h, cudaGetLastError());
    return HAMR_OK;
}

int ms_from_planes(hamr_ms_t h, const void *src, long long n) {
    if (h->prec == HAMR_FP64)
        k_planes_to_aos<double><<<nblk(n), BLK, 0, h->stream>>>((const double *)src, h->stage, n);
    else
        k_planes_to_aos<float><<<nblk(n), BLK, 0, h->stream>>>((const float *)src, h->stage, n);
    MSCK(h, cudaGetLastError());
    return HAMR_OK;
}

int ms_zero_void(hamr_ms_t h) {
    if (h->prec == HAMR_FP64)
        k_zero_void_cells<double><<<nblk(h->P.nc), BLK, 0, h->stream>>>((double *)h->m, h->grain_d, h->P.nc);
    else
        k_zero_void_cells<float><<<nblk(h->P.nc), BLK, 0, h->stream>>>((float *)h->m, h->grain_d, h->P.nc);
    MSCK(h, cudaGetLastError());
    return HAMR_OK;
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
    // launch grids: (x / 32, y / 4, z) blocks
    if ((long long)d->ncy * d->ratio > 4 * 65535LL || (long long)d->ncz * d->ratio > 65535LL)
        return msfail(nullptr, HAMR_ERR_ARG, "at most 262140 sites across the track and 65535 through it");
    const double vals[] = {d->cell, d->mu_s, d->gamma, d->dt, d->T_C, d->Ms0};
    for (double v : vals)
        if (!(v > 0) || !isfinite(v))
            return msfail(nullptr, HAMR_ERR_ARG, "cell, mu_s, gamma, dt, T_C and Ms0 must be positive");
    if (!isfinite(d->J) || !isfinite(d->ku) || !(d->lambda >= 0) || !isfinite(d->A0) || !isfinite(d->K0))
        return msfail(nullptr, HAMR_ERR_ARG, "J, ku, A0, K0 must be finite and lambda >= 0");
    if (d->precision != HAMR_FP32 && d->precision != HAMR_FP64)
        return msfail(nullptr, HAMR_ERR_ARG, "precision must be HAMR_FP32 or HAMR_FP64");
    hamr_ms_t h = new (std::nothrow) hamr_ms_ctx();
    if (!h) return msfail(nullptr, HAMR_ERR_OOM, "host allocation failed");
    h->device = d->device;
    h->prec = d->precision;
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
    P.cA = 2.0 * d->A0 / d->Ms0;
    P.cK = 2.0 * d->K0 / d->Ms0;
    P.mu_kB = d->mu_s / KB;
    P.i3TC = 1.0 / (3.0 * d->T_C);
    P.J_mu = d->J / d->mu_s;
    P.ku2_mu = 2.0 * d->ku / d->mu_s;
    P.key0 = (unsigned)d->seed;
    P.key1 = (unsigned)(d->seed >> 32);
    h->D.dir[2] = 1.0;
    set_driver_floats(h->D);
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
    {
        cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ms_free(h);
            if (h->own_stream) cudaStreamDestroy(h->stream);
            delete h;
            return msfail(nullptr, HAMR_ERR_CUDA, "side stream or events: %s", cudaGetErrorString(e));
        }
    }
    const size_t el = h->prec == HAMR_FP64 ? sizeof(double) : sizeof(float);
    void **bufs3c[] = {&h->m, &h->V0, &h->V1, &h->acc, &h->coef};
    cudaError_t e = cudaSuccess;
    for (void **b : bufs3c)
        if (e == cudaSuccess) e = cudaMalloc(b, el * 3 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&h->wn, el * nc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->me, sizeof(double) * nc);
    const long long ncol = (long long)h->P.ncx * h->P.ncy;
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->col, sizeof(double) * 3 * ncol);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->colmask, sizeof(unsigned long long) * ncol);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->colmask, 0, sizeof(unsigned long long) * ncol, h->stream);
    void **bufs3w[] = {&h->S, &h->S2};
    for (void **b : bufs3w)
        if (e == cudaSuccess) e = cudaMalloc(b, el * 3 * nw);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->stage, sizeof(double) * 3 * (nw > nc ? nw : nc));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->grain_d, sizeof(int) * nc);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->m, 0, el * 3 * nc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->wn, 0, el * nc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->S, 0, el * 3 * nw, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->grain_d, 0, sizeof(int) * nc, h->stream);
    if (e == cudaSuccess) {
        k_fill<<<nblk(nc), BLK, 0, h->stream>>>(h->me, 1.0, nc);
        k_fill<<<nblk(ncol), BLK, 0, h->stream>>>(h->col, NAN, ncol);
        k_fill<<<nblk(ncol), BLK, 0, h->stream>>>(h->col + ncol, 1.0, ncol);
        k_fill<<<nblk(ncol), BLK, 0, h->stream>>>(h->col + 2 * ncol, NAN, ncol);
        e = cudaGetLastError();
    }
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
    // the magnetic planes of every cell column, and no column's m_e solve kept: cells that
    // turned magnetic get theirs at the next solve
    const long long ncol = (long long)h->P.ncx * h->P.ncy;
    h->colmask_h.assign(ncol, 0ull);
    for (int z = 0; z < h->P.ncz && z < 64; ++z)
        for (long long c = 0; c < ncol; ++c)
            if (cell_grain[c + ncol * z] >= 0) h->colmask_h[c] |= 1ull << z;
    MSCK(h, cudaMemcpyAsync(h->colmask, h->colmask_h.data(), sizeof(unsigned long long) * ncol, cudaMemcpyHostToDevice,
                            h->stream));
    k_fill<<<nblk(ncol), BLK, 0, h->stream>>>(h->col, NAN, ncol);
    MSCK(h, cudaGetLastError());
    int rc = ms_zero_void(h);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    h->grains_set = true;
    h->fz_dirty = true;
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
    set_driver_floats(D);
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
    h->Bm_last = NAN;  // the field law changed: no column keeps its last m_e solve
    D.B0 = B0;
    for (int k = 0; k < 3; ++k) D.dir[k] = dir[k];
    D.n_bits = n_bits;
    D.bits_off = 0;
    D.bit_len = bit_len; D.ramp_len = ramp_len; D.head_x0 = head_x0; D.head_v = head_v;
    set_driver_floats(D);
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

int hamr_ms_set_head_profile(hamr_ms_t h, double Bx0, double wz, double dz, double wx, double dx) {
    if (!h) return HAMR_ERR_ARG;
    if (!(wz > 0)) {
        h->P.profile = 0;
        // every column's m_e was solved with its own profile field: solve them all again
        h->Bm_last = NAN;
        return HAMR_OK;
    }
    if (!isfinite(Bx0) || !isfinite(wz) || !isfinite(dz) || !(wx > 0) || !isfinite(wx) || !isfinite(dx))
        return msfail(h, HAMR_ERR_ARG, "head profile: finite values, widths > 0");
    h->Bm_last = NAN;
    h->P.profile = 1;
    h->P.pBx0 = Bx0;
    h->P.pwz = wz;
    h->P.pdz = dz;
    h->P.pwx = wx;
    h->P.pdx = dx;
    return HAMR_OK;
}

int hamr_ms_set_region(hamr_ms_t h, int32_t margin) {
    if (!h) return HAMR_ERR_ARG;
    h->margin = margin < 0 ? -1 : margin;
    h->fz_dirty = true;
    return HAMR_OK;
}

int hamr_ms_set_demag(hamr_ms_t h, int32_t on) {
    if (!h) return HAMR_ERR_ARG;
    if (!on) {
        h->demag = false;
        return HAMR_OK;
    }
    MsDeviceGuard dg(h->device);
    if (!h->gtrack.plans) {
        const size_t es = h->prec == HAMR_FP64 ? 8 : 4;
        MSCK(h, cudaMalloc(&h->Bfz, es * 3 * h->P.nc));
        const int rc = h->prec == HAMR_FP64 ? demag_grid_setup<double>(h, h->gtrack, h->P.ncx)
                                            : demag_grid_setup<float>(h, h->gtrack, h->P.ncx);
        if (rc) return rc;
    }
    h->demag = true;
    h->fz_dirty = true;
    return HAMR_OK;
}

int hamr_ms_demag_field(hamr_ms_t h, const double *M, double *B_out) {
    if (!h || !M || !B_out) return h ? msfail(h, HAMR_ERR_ARG, "M and B_out must not be NULL") : HAMR_ERR_ARG;
    if (!h->gtrack.plans) return msfail(h, HAMR_ERR_STATE, "Eq. 7 is off: call hamr_ms_set_demag(h, 1) first");
    for (long long q = 0; q < 3 * h->P.nc; ++q)
        if (!isfinite(M[q])) return msfail(h, HAMR_ERR_ARG, "non-finite magnetisation at cell %lld", q / 3);
    MsDeviceGuard dg(h->device);
    // M and B_d pass through the RK4 stage planes, which a step rewrites before it reads them
    MSCK(h, cudaMemcpyAsync(h->stage, M, sizeof(double) * 3 * h->P.nc, cudaMemcpyHostToDevice, h->stream));
    int rc = ms_to_planes(h, h->V0, h->P.nc);
    if (rc) return rc;
    const int nx = h->P.ncx;
    rc = h->prec == HAMR_FP64
             ? demag_pass<double>(h, h->gtrack, 0, 3, 0, nx, (double *)h->V1, 0, nx, nullptr, (const double *)h->V0)
             : demag_pass<float>(h, h->gtrack, 0, 3, 0, nx, (float *)h->V1, 0, nx, nullptr, (const float *)h->V0);
    if (rc) return rc;
    if ((rc = ms_from_planes(h, h->V1, h->P.nc))) return rc;
    MSCK(h, cudaMemcpyAsync(B_out, h->stage, sizeof(double) * 3 * h->P.nc, cudaMemcpyDeviceToHost, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_set_cells(hamr_ms_t h, const double *m) {
    if (!h || !m) return h ? msfail(h, HAMR_ERR_ARG, "m is NULL") : HAMR_ERR_ARG;
    for (long long q = 0; q < 3 * h->P.nc; ++q)
        if (!isfinite(m[q])) return msfail(h, HAMR_ERR_ARG, "non-finite cell value at %lld", q / 3);
    MsDeviceGuard dg(h->device);
    MSCK(h, cudaMemcpyAsync(h->stage, m, sizeof(double) * 3 * h->P.nc, cudaMemcpyHostToDevice, h->stream));
    int rc = ms_to_planes(h, h->m, h->P.nc);
    if (!rc) rc = ms_zero_void(h);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    h->cells_set = true;
    h->window_live = false;
    h->fz_dirty = true;
    return HAMR_OK;
}

int hamr_ms_set_window(hamr_ms_t h, int32_t x0_cells) {
    if (!h) return HAMR_ERR_ARG;
    if (x0_cells < 0 || x0_cells + h->P.wx > h->P.ncx)
        return msfail(h, HAMR_ERR_ARG, "window [%d, %d) outside the track of %d cells", x0_cells, x0_cells + h->P.wx,
                      h->P.ncx);
    if (!h->cells_set) return msfail(h, HAMR_ERR_STATE, "set the cells (hamr_ms_set_cells) before the window");
    MsDeviceGuard dg(h->device);
    // a window already placed hands its sites back to its cells by Eq. 6 first (as the trailing
    // column of a move does), unless the cells have been replaced since
    if (h->ox >= 0 && h->window_live) {
        int rc = h->prec == HAMR_FP64 ? ms_average<double>(h, h->ox, h->P.wx) : ms_average<float>(h, h->ox, h->P.wx);
        if (rc) return rc;
    }
    h->window_live = true;
    h->fz_dirty = true;  // every cell's m_e is solved again at the placement
    h->ox = x0_cells;
    const double t = (double)h->step * h->P.dt;
    int rc = h->prec == HAMR_FP64 ? ms_thermalise<double>(h, h->ox, h->ox + h->P.wx, t, true)
                                  : ms_thermalise<float>(h, h->ox, h->ox + h->P.wx, t, true);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_set_moments(hamr_ms_t h, const double *S) {
    if (!h || !S) return h ? msfail(h, HAMR_ERR_ARG, "S is NULL") : HAMR_ERR_ARG;
    if (h->ox < 0) return msfail(h, HAMR_ERR_STATE, "place the window (hamr_ms_set_window) first");
    MsDeviceGuard dg(h->device);
    MSCK(h, cudaMemcpyAsync(h->stage, S, sizeof(double) * 3 * h->P.nw, cudaMemcpyHostToDevice, h->stream));
    int rc = ms_to_planes(h, h->S, h->P.nw);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_steps(hamr_ms_t h, int64_t n_steps, int32_t follow) {
    if (!h) return HAMR_ERR_ARG;
    if (n_steps < 0) return msfail(h, HAMR_ERR_ARG, "n_steps must be >= 0");
    if (h->ox < 0) return msfail(h, HAMR_ERR_STATE, "place the window (hamr_ms_set_window) first");
    MsDeviceGuard dg(h->device);
    for (int64_t s = 0; s < n_steps; ++s) {
        int rc = h->prec == HAMR_FP64 ? ms_step<double>(h) : ms_step<float>(h);
        if (rc) return rc;
        if (follow) {
            const double t = (double)h->step * h->P.dt;
            const int target = ms_target(h, t);
            while (h->ox < target)
                if ((rc = h->prec == HAMR_FP64 ? ms_shift_forward<double>(h, t) : ms_shift_forward<float>(h, t)))
                    return rc;
        }
    }
    int rc = h->prec == HAMR_FP64 ? ms_average<double>(h, h->ox, h->P.wx) : ms_average<float>(h, h->ox, h->P.wx);
    if (rc) return rc;
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_read_cells(hamr_ms_t h, double *m_out) {
    if (!h || !m_out) return h ? msfail(h, HAMR_ERR_ARG, "m_out is NULL") : HAMR_ERR_ARG;
    MsDeviceGuard dg(h->device);
    int rc = ms_from_planes(h, h->m, h->P.nc);
    if (rc) return rc;
    MSCK(h, cudaMemcpyAsync(m_out, h->stage, sizeof(double) * 3 * h->P.nc, cudaMemcpyDeviceToHost, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_ms_read_moments(hamr_ms_t h, double *S_out) {
    if (!h || !S_out) return h ? msfail(h, HAMR_ERR_ARG, "S_out is NULL") : HAMR_ERR_ARG;
    MsDeviceGuard dg(h->device);
    int rc = ms_from_planes(h, h->S, h->P.nw);
    if (rc) return rc;
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

int hamr_ms_read_track(hamr_ms_t h, double x_start, double bit_len, int32_t n_bits, int32_t cy0, int32_t cy1,
                       double *signal, uint8_t *bits) {
    if (!h) return HAMR_ERR_ARG;
    if (n_bits < 0 || !isfinite(x_start) || !(bit_len > 0) || !isfinite(bit_len) || cy0 < 0 || cy1 > h->P.ncy ||
        cy0 >= cy1)
        return msfail(h, HAMR_ERR_ARG, "bad read-back window (bit_len > 0, 0 <= cy0 < cy1 <= ncy)");
    if (n_bits > 0 && !signal) return msfail(h, HAMR_ERR_ARG, "signal is NULL");
    if ((long long)n_bits > 3 * (h->P.nw > h->P.nc ? h->P.nw : h->P.nc))
        return msfail(h, HAMR_ERR_ARG, "too many bits (%d)", n_bits);
    if (n_bits == 0) return HAMR_OK;
    MsDeviceGuard dg(h->device);
    if (h->prec == HAMR_FP64)
        k_ms_read_track<double><<<n_bits, 256, 0, h->stream>>>((const double *)h->m, h->grain_d, h->P, x_start, bit_len,
                                                              cy0, cy1, h->stage);
    else
        k_ms_read_track<float><<<n_bits, 256, 0, h->stream>>>((const float *)h->m, h->grain_d, h->P, x_start, bit_len,
                                                             cy0, cy1, h->stage);
    MSCK(h, cudaGetLastError());
    MSCK(h, cudaMemcpyAsync(signal, h->stage, sizeof(double) * n_bits, cudaMemcpyDeviceToHost, h->stream));
    MSCK(h, cudaStreamSynchronize(h->stream));
    if (bits)
        for (int32_t b = 0; b < n_bits; ++b) bits[b] = signal[b] < 0.0 ? 1 : 0;
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
