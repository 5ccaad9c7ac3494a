// Two-pass sLLG Heun step (one thread per lattice site, two launches per step).
//
// Pass 1 (predictor) computes, per magnetic site i at step n,
//   T_i(t_n), sigma_i = sqrt(2 alpha kB T_i/(gamma mu_s dt)), B_th,i = sigma_i xi_i,
//   B_i(S) = (1/mu_s) sum_j J_ij S_j + (2 ku/mu_s) S_i,z z + B_app(t_n)        (Eq. 2, 3)
//   f1 = f(S_i, B_i(S) + B_th,i),  S'_i = N(S_i + dt f1)                      (Eq. 1, Heun)
// and stores S', dt f1 and B_th.  Pass 2 (corrector) computes
//   f2 = f(S'_i, B_i(S') + B_th,i),  S_i <- N(S_i + (dt f1 + dt f2)/2)
// in place (it reads S only at i itself, so the update is race-free), and at record steps
// adds the new spin to its grain's FP64 sum.
//
// This is the plain path: FP64 for every precision-FP64 handle, and FP32 for handles that
// use a neighbour list.  Neighbours come from the lattice's implicit stencil (bonds only
// between equal grain codes) or from the packed list.
#include "device_common.cuh"

namespace hamr {

template <typename Real>
struct Drivers;

template <>
struct Drivers<double> {
    __device__ static double pol(const ReplicaDev &R, const uint8_t *bits, long long step, double dt) {
        return field_polarity(R, bits, (double)step * dt);
    }
    __device__ static double temp(const ReplicaDev &R, double x, double y, long long step, double dt) {
        return temperature(R, x, y, (double)step * dt);
    }
    __device__ static double B0(const ReplicaDev &R) { return R.B0; }
    __device__ static double dir(const ReplicaDev &R, int d) { return R.dir[d]; }
    __device__ static double rsq(double v) { return rsqrt(v); }
};

template <>
struct Drivers<float> {
    __device__ static float pol(const ReplicaDev &R, const uint8_t *bits, long long step, float dt) {
        return field_polarity_f(R, bits, (float)step * dt);
    }
    __device__ static float temp(const ReplicaDev &R, float x, float y, long long step, float dt) {
        return temperature_f(R, x, y, (float)step * dt);
    }
    __device__ static float B0(const ReplicaDev &R) { return R.fB0; }
    __device__ static float dir(const ReplicaDev &R, int d) { return R.fdir[d]; }
    __device__ static float rsq(float v) { return rsqrtf(v); }
};

// f(S, B) = pref [S x B + alpha S x (S x B)], written with S x (S x B) = (S.B) S - (S.S) B
template <typename Real>
__device__ __forceinline__ void llg_rhs(Real pref, Real alpha, Real sx, Real sy, Real sz, Real bx, Real by,
                                        Real bz, Real &fx, Real &fy, Real &fz) {
    const Real cx = sy * bz - sz * by, cy = sz * bx - sx * bz, cz = sx * by - sy * bx;
    const Real sb = sx * bx + sy * by + sz * bz, ss = sx * sx + sy * sy + sz * sz;
    fx = pref * (cx + alpha * (sb * sx - ss * bx));
    fy = pref * (cy + alpha * (sb * sy - ss * by));
    fz = pref * (cz + alpha * (sb * sz - ss * bz));
}

struct SiteIdx {
    int x, y, z;
    bool valid;
};

__device__ __forceinline__ SiteIdx decode(const ReplicaDev &R, long long s) {
    const long long loc = s - R.off;
    SiteIdx q;
    q.x = (int)(loc % R.px);
    const long long yz = loc / R.px;
    q.y = (int)(yz % R.ny);
    q.z = (int)(yz / R.ny);
    q.valid = q.x < R.nx && q.z < R.nz;
    return q;
}

// storage slot of the neighbour at (x+dx, y+dy, z+dz), or -1 across an open edge
__device__ __forceinline__ long long stencil_slot(const ReplicaDev &R, const int *per, SiteIdx q, int dx, int dy,
                                                  int dz) {
    int xx = q.x + dx, yy = q.y + dy, zz = q.z + dz;
    if (xx < 0 || xx >= R.nx) {
        if (!per[0]) return -1;
        xx = (xx % R.nx + R.nx) % R.nx;
    }
    if (yy < 0 || yy >= R.ny) {
        if (!per[1]) return -1;
        yy = (yy % R.ny + R.ny) % R.ny;
    }
    if (zz < 0 || zz >= R.nz) {
        if (!per[2]) return -1;
        zz = (zz % R.nz + R.nz) % R.nz;
    }
    return R.off + xx + (long long)R.px * (yy + (long long)R.ny * zz);
}

// sum_j (J_ij / mu_s) V_j over the bonds of slot s
template <typename Real>
__device__ __forceinline__ void exchange(const PlainArgs<Real> &a, const ReplicaDev &R, SiteIdx q, long long s,
                                         unsigned g, const Real *V, Real &ex, Real &ey, Real &ez) {
    const long long NS = a.NS;
    ex = ey = ez = Real(0);
    if (a.ell) {
        for (int k = 0; k < a.ell_w; ++k) {
            const int e = a.ell[(long long)k * NS + s];
            if (e < 0) break;
            const long long j = e & ((1 << ELL_SHELL_SHIFT) - 1);
            const Real cj = (Real)a.ph.cJ[e >> ELL_SHELL_SHIFT];
            ex += cj * V[j];
            ey += cj * V[NS + j];
            ez += cj * V[2 * NS + j];
        }
    } else {
        // the lattice's implicit stencil: SC, 6 nearest neighbours in one shell; L1_0 Fe
        // sublattice, 4 in-plane nearest (shell 0), 2 out of plane (shell 1) and 4 in-plane
        // diagonals (shell 2)
        const bool tet = a.ph.lattice == HAMR_LATTICE_L10;
        const int d[10][4] = {{-1, 0, 0, 0}, {1, 0, 0, 0},  {0, -1, 0, 0},  {0, 1, 0, 0},  {0, 0, -1, 1},
                              {0, 0, 1, 1},  {-1, -1, 0, 2}, {1, -1, 0, 2}, {-1, 1, 0, 2}, {1, 1, 0, 2}};
        const int nb = tet ? 10 : 6;
        for (int k = 0; k < nb; ++k) {
            const long long j = stencil_slot(R, a.ph.per, q, d[k][0], d[k][1], d[k][2]);
            if (j >= 0 && a.gcode[j] == g) {
                const Real cj = (Real)a.ph.cJ[tet ? d[k][3] : 0];
                ex += cj * V[j];
                ey += cj * V[NS + j];
                ez += cj * V[2 * NS + j];
            }
        }
    }
}

template <typename Real>
__global__ void __launch_bounds__(PLAIN_BLOCK) k_predict(PlainArgs<Real> a) {
    const int r = a.blk_rep[blockIdx.x];
    if (r < 0) return;
    const long long s = (long long)blockIdx.x * PLAIN_BLOCK + threadIdx.x;
    const ReplicaDev &R = a.reps[r];
    const SiteIdx q = decode(R, s);
    if (!q.valid) return;
    const unsigned g = a.gcode[s];
    if (g == 0) return;
    const long long NS = a.NS;
    const long long step = a.ctl->step + a.step_off;
    const Real dt = (Real)a.ph.dt;

    // thermal field
    const Real T = Drivers<Real>::temp(R, (Real)((q.x + 0.5) * a.ph.ax), (Real)((q.y + 0.5) * a.ph.ay), step, dt);
    const Real sig = (Real)a.ph.sig0 * sqrt(T);
    const unsigned long long site = (unsigned long long)q.x + (unsigned long long)R.nx * (q.y + (unsigned long long)R.ny * q.z);
    Real n0, n1, n2;
    normals3(philox_site(R.key0, R.key1, site, (unsigned long long)step), n0, n1, n2);
    const Real tx = sig * n0, ty = sig * n1, tz = sig * n2;

    // field at S
    const Real *S = a.S;
    const Real sx = S[s], sy = S[NS + s], sz = S[2 * NS + s];
    Real ex, ey, ez;
    exchange(a, R, q, s, g, S, ex, ey, ez);
    const Real bapp = Drivers<Real>::B0(R) * Drivers<Real>::pol(R, a.bits, step, dt);
    const Real bx = ex + bapp * Drivers<Real>::dir(R, 0) + tx;
    const Real by = ey + bapp * Drivers<Real>::dir(R, 1) + ty;
    const Real bz = ez + (Real)a.ph.cK * sz + bapp * Drivers<Real>::dir(R, 2) + tz;
    Real fx, fy, fz;
    llg_rhs((Real)a.ph.pref, (Real)a.ph.alpha, sx, sy, sz, bx, by, bz, fx, fy, fz);
    fx *= dt;
    fy *= dt;
    fz *= dt;
    Real px = sx + fx, py = sy + fy, pz = sz + fz;
    const Real inv = Drivers<Real>::rsq(px * px + py * py + pz * pz);
    a.SP[s] = px * inv;
    a.SP[NS + s] = py * inv;
    a.SP[2 * NS + s] = pz * inv;
    a.F1[s] = fx;
    a.F1[NS + s] = fy;
    a.F1[2 * NS + s] = fz;
    a.BTH[s] = tx;
    a.BTH[NS + s] = ty;
    a.BTH[2 * NS + s] = tz;
}

template <typename Real, bool RECORD>
__global__ void __launch_bounds__(PLAIN_BLOCK) k_correct(PlainArgs<Real> a) {
    const int r = a.blk_rep[blockIdx.x];
    if (r < 0) return;  // whole block is padding
    const long long s = (long long)blockIdx.x * PLAIN_BLOCK + threadIdx.x;
    const ReplicaDev &R = a.reps[r];
    const SiteIdx q = decode(R, s);
    const unsigned g = q.valid ? a.gcode[s] : 0u;
    const bool act = g != 0;
    const long long NS = a.NS;
    double ox = 0, oy = 0, oz = 0;
    if (act) {
        const long long step = a.ctl->step + a.step_off;
        const Real dt = (Real)a.ph.dt;
        const Real *SP = a.SP;
        const Real spx = SP[s], spy = SP[NS + s], spz = SP[2 * NS + s];
        Real ex, ey, ez;
        exchange(a, R, q, s, g, SP, ex, ey, ez);
        const Real bapp = Drivers<Real>::B0(R) * Drivers<Real>::pol(R, a.bits, step, dt);
        const Real bx = ex + bapp * Drivers<Real>::dir(R, 0) + a.BTH[s];
        const Real by = ey + bapp * Drivers<Real>::dir(R, 1) + a.BTH[NS + s];
        const Real bz = ez + (Real)a.ph.cK * spz + bapp * Drivers<Real>::dir(R, 2) + a.BTH[2 * NS + s];
        Real fx, fy, fz;
        llg_rhs((Real)a.ph.pref, (Real)a.ph.alpha, spx, spy, spz, bx, by, bz, fx, fy, fz);
        const Real h = Real(0.5);
        Real nx = a.S[s] + h * (a.F1[s] + dt * fx);
        Real ny = a.S[NS + s] + h * (a.F1[NS + s] + dt * fy);
        Real nz = a.S[2 * NS + s] + h * (a.F1[2 * NS + s] + dt * fz);
        const Real inv = Drivers<Real>::rsq(nx * nx + ny * ny + nz * nz);
        nx *= inv;
        ny *= inv;
        nz *= inv;
        a.S[s] = nx;
        a.S[NS + s] = ny;
        a.S[2 * NS + s] = nz;
        ox = nx;
        oy = ny;
        oz = nz;
    }
    if (RECORD) grain_accumulate(a.grain_acc, act ? R.grain_off + (int)g - 1 : -1, ox, oy, oz, act);
}

// E = -1/2 sum_i sum_j J_ij S_i.S_j - sum_i ku S_i,z^2 - sum_i mu_s B_app(t).S_i, one thread per
// site of replica r, FP64 block sums, one atomic per block.
template <typename Real>
__global__ void __launch_bounds__(256) k_energy(PlainArgs<Real> a, int r, long long n, long long step, double ku,
                                                double mu_s, double *out) {
    __shared__ double red[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        const ReplicaDev &R = a.reps[r];
        SiteIdx q;
        q.x = (int)(i % R.nx);
        q.y = (int)((i / R.nx) % R.ny);
        q.z = (int)(i / ((long long)R.nx * R.ny));
        q.valid = true;
        const long long s = R.off + q.x + (long long)R.px * (q.y + (long long)R.ny * q.z);
        const unsigned g = a.gcode[s];
        if (g != 0) {
            const long long NS = a.NS;
            const double sx = a.S[s], sy = a.S[NS + s], sz = a.S[2 * NS + s];
            Real ex, ey, ez;
            exchange(a, R, q, s, g, a.S, ex, ey, ez);
            const double b = R.B0 * field_polarity(R, a.bits, (double)step * a.ph.dt);
            e = -0.5 * mu_s * (sx * (double)ex + sy * (double)ey + sz * (double)ez) - ku * sz * sz -
                mu_s * b * (R.dir[0] * sx + R.dir[1] * sy + R.dir[2] * sz);
        }
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

cudaError_t launch_energy(int prec, const void *S, long long NS, const uint16_t *gcode, const ReplicaDev *reps,
                          const ReplicaDev &Rh, int r, const uint8_t *bits, const int *ell, int ell_w,
                          const Phys &ph, long long step, double ku, double mu_s, double *out, cudaStream_t st) {
    const unsigned nb = (unsigned)((Rh.n + 255) / 256);
    if (prec == HAMR_FP64) {
        PlainArgs<double> a{};
        a.S = (double *)S;
        a.NS = NS;
        a.gcode = gcode;
        a.reps = reps;
        a.bits = bits;
        a.ell = ell;
        a.ell_w = ell_w;
        a.ph = ph;
        k_energy<double><<<nb, 256, 0, st>>>(a, r, Rh.n, step, ku, mu_s, out);
    } else {
        PlainArgs<float> a{};
        a.S = (float *)S;
        a.NS = NS;
        a.gcode = gcode;
        a.reps = reps;
        a.bits = bits;
        a.ell = ell;
        a.ell_w = ell_w;
        a.ph = ph;
        k_energy<float><<<nb, 256, 0, st>>>(a, r, Rh.n, step, ku, mu_s, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_step(int prec, const void *args, int n_blocks, bool record, cudaStream_t st) {
    if (prec == HAMR_FP64) {
        const PlainArgs<double> &a = *(const PlainArgs<double> *)args;
        k_predict<double><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
        if (record)
            k_correct<double, true><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
        else
            k_correct<double, false><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
    } else {
        const PlainArgs<float> &a = *(const PlainArgs<float> *)args;
        k_predict<float><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
        if (record)
            k_correct<float, true><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
        else
            k_correct<float, false><<<n_blocks, PLAIN_BLOCK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace hamr
