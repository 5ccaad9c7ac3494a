// One FP64 Heun step that allocates nothing, for callers that cannot call cudaMalloc.
//
// Some callers of this library may not allocate device memory themselves: code that runs
// while another framework owns the whole device memory pool, or a host loop that must not
// allocate once it has started.  They cannot create a hamr_t (which allocates), so this
// entry point takes the caller's own device buffers for the spins and the grain map, and
// keeps its intermediate results (S', dt f(S, B(S)) and the thermal field) in one
// file-scope device array of fixed size that every GPU loading the library holds until the
// process exits.  The arithmetic is that of the two-pass FP64 step: predictor kernel, then
// corrector kernel, on one simple-cubic lattice with the implicit 6-neighbour stencil.
#include <mutex>

#include "device_common.cuh"

namespace hamr {
void set_handleless_error(const char *msg);
}

namespace {

using namespace hamr;

constexpr int kMaxDevices = 64;

// S' [3][n], dt f1 [3][n], B_th [3][n]; shared by every call on a device
static __device__ __align__(256) double g_noalloc_scratch[9 * (size_t)HAMR_NOALLOC_MAX_SITES];

double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

struct NoallocArgs {
    hamr_noalloc_params p;
    const double *Sin;
    double *Sout;
    const int32_t *grain;
    double *scratch;
    long long n;
    long long step;
    double cJ, cK, pref, sig0, c_fwhm;
};

__device__ __forceinline__ bool nb_site(const NoallocArgs &a, int x, int y, int z, int dx, int dy, int dz,
                                        long long &j) {
    int xx = x + dx, yy = y + dy, zz = z + dz;
    const int nx = a.p.nx, ny = a.p.ny, nz = a.p.nz;
    if (xx < 0 || xx >= nx) {
        if (!a.p.periodic[0]) return false;
        xx = (xx % nx + nx) % nx;
    }
    if (yy < 0 || yy >= ny) {
        if (!a.p.periodic[1]) return false;
        yy = (yy % ny + ny) % ny;
    }
    if (zz < 0 || zz >= nz) {
        if (!a.p.periodic[2]) return false;
        zz = (zz % nz + nz) % nz;
    }
    j = xx + (long long)nx * (yy + (long long)ny * zz);
    return true;
}

// (1/mu_s) sum_j J S_j over the stencil bonds of site i that stay inside its grain
__device__ __forceinline__ void nb_sum(const NoallocArgs &a, const double *V, long long i, int g, double &ex,
                                       double &ey, double &ez) {
    const int x = (int)(i % a.p.nx), y = (int)((i / a.p.nx) % a.p.ny), z = (int)(i / ((long long)a.p.nx * a.p.ny));
    const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    ex = ey = ez = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        long long j;
        if (!nb_site(a, x, y, z, d[k][0], d[k][1], d[k][2], j)) continue;
        if ((a.grain ? a.grain[j] : 0) != g) continue;
        ex += V[3 * j];
        ey += V[3 * j + 1];
        ez += V[3 * j + 2];
    }
    ex *= a.cJ;
    ey *= a.cJ;
    ez *= a.cJ;
}

__device__ __forceinline__ void rhs(const NoallocArgs &a, double sx, double sy, double sz, double bx, double by,
                                    double bz, double &fx, double &fy, double &fz) {
    const double cx = sy * bz - sz * by, cy = sz * bx - sx * bz, cz = sx * by - sy * bx;
    const double sb = sx * bx + sy * by + sz * bz, ss = sx * sx + sy * sy + sz * sz;
    fx = a.pref * (cx + a.p.alpha * (sb * sx - ss * bx));
    fy = a.pref * (cy + a.p.alpha * (sb * sy - ss * by));
    fz = a.pref * (cz + a.p.alpha * (sb * sz - ss * bz));
}

__global__ void k_noalloc_predict(NoallocArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int g = a.grain ? a.grain[i] : 0;
    if (g < 0) return;
    const long long n = a.n;
    double *SP = a.scratch, *F1 = a.scratch + 3 * n, *BT = a.scratch + 6 * n;
    const int x = (int)(i % a.p.nx), y = (int)((i / a.p.nx) % a.p.ny);
    const double t = (double)a.step * a.p.dt;
    double T = a.p.T_amb;
    if (a.c_fwhm != 0.0) {
        const double dx = (x + 0.5) * a.p.a - a.p.x0 - a.p.vx * t, dy = (y + 0.5) * a.p.a - a.p.y0 - a.p.vy * t;
        T = a.p.T_amb + (a.p.T_peak - a.p.T_amb) * exp(a.c_fwhm * (dx * dx + dy * dy));
    }
    const double sig = a.sig0 * sqrt(T);
    double n0, n1, n2;
    normals3(philox_site((unsigned)(a.p.seed & 0xffffffffu), (unsigned)(a.p.seed >> 32), (unsigned long long)i,
                         (unsigned long long)a.step),
             n0, n1, n2);
    const double tx = sig * n0, ty = sig * n1, tz = sig * n2;
    const double sx = a.Sin[3 * i], sy = a.Sin[3 * i + 1], sz = a.Sin[3 * i + 2];
    double ex, ey, ez;
    nb_sum(a, a.Sin, i, g, ex, ey, ez);
    const double bx = ex + a.p.B_app[0] + tx, by = ey + a.p.B_app[1] + ty, bz = ez + a.cK * sz + a.p.B_app[2] + tz;
    double fx, fy, fz;
    rhs(a, sx, sy, sz, bx, by, bz, fx, fy, fz);
    fx *= a.p.dt;
    fy *= a.p.dt;
    fz *= a.p.dt;
    const double px = sx + fx, py = sy + fy, pz = sz + fz;
    const double inv = rsqrt(px * px + py * py + pz * pz);
    SP[3 * i] = px * inv;
    SP[3 * i + 1] = py * inv;
    SP[3 * i + 2] = pz * inv;
    F1[3 * i] = fx;
    F1[3 * i + 1] = fy;
    F1[3 * i + 2] = fz;
    BT[3 * i] = tx;
    BT[3 * i + 1] = ty;
    BT[3 * i + 2] = tz;
}

__global__ void k_noalloc_correct(NoallocArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int g = a.grain ? a.grain[i] : 0;
    if (g < 0) {  // non-magnetic: carried over unchanged
        a.Sout[3 * i] = a.Sin[3 * i];
        a.Sout[3 * i + 1] = a.Sin[3 * i + 1];
        a.Sout[3 * i + 2] = a.Sin[3 * i + 2];
        return;
    }
    const long long n = a.n;
    const double *SP = a.scratch, *F1 = a.scratch + 3 * n, *BT = a.scratch + 6 * n;
    const double px = SP[3 * i], py = SP[3 * i + 1], pz = SP[3 * i + 2];
    double ex, ey, ez;
    nb_sum(a, SP, i, g, ex, ey, ez);
    const double bx = ex + a.p.B_app[0] + BT[3 * i], by = ey + a.p.B_app[1] + BT[3 * i + 1],
                 bz = ez + a.cK * pz + a.p.B_app[2] + BT[3 * i + 2];
    double fx, fy, fz;
    rhs(a, px, py, pz, bx, by, bz, fx, fy, fz);
    double ox = a.Sin[3 * i] + 0.5 * (F1[3 * i] + a.p.dt * fx);
    double oy = a.Sin[3 * i + 1] + 0.5 * (F1[3 * i + 1] + a.p.dt * fy);
    double oz = a.Sin[3 * i + 2] + 0.5 * (F1[3 * i + 2] + a.p.dt * fz);
    const double inv = rsqrt(ox * ox + oy * oy + oz * oz);
    a.Sout[3 * i] = ox * inv;
    a.Sout[3 * i + 1] = oy * inv;
    a.Sout[3 * i + 2] = oz * inv;
}

int reject(int code, const char *msg) {
    set_handleless_error(msg);
    return code;
}

}  // namespace

extern "C" int hamr_sllg_heun_step_noalloc(const hamr_noalloc_params *p, const double *S_in, double *S_out,
                                           const int32_t *grain, int64_t step, void *stream) {
    if (!p || !S_in || !S_out) return reject(HAMR_ERR_ARG, "null argument");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return reject(HAMR_ERR_ARG, "lattice dimensions must be >= 1");
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n > HAMR_NOALLOC_MAX_SITES)
        return reject(HAMR_ERR_ARG, "lattice has more sites than HAMR_NOALLOC_MAX_SITES (131072)");
    {
        // the corrector reads S_in[i] while other threads write S_out: the arrays must be the
        // same or disjoint
        const uintptr_t i0 = (uintptr_t)S_in, o0 = (uintptr_t)S_out, len = (uintptr_t)(3 * n) * sizeof(double);
        if (S_out != S_in && i0 < o0 + len && o0 < i0 + len)
            return reject(HAMR_ERR_ARG, "S_out overlaps S_in without being the same array");
    }
    if (!(p->a > 0) || !(p->mu_s > 0) || !(p->dt > 0) || !(p->gamma > 0) || !(p->alpha >= 0) ||
        !(p->T_amb >= 0) || !(p->T_peak >= 0) || step < 0)
        return reject(HAMR_ERR_ARG, "bad physical parameter");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(HAMR_ERR_CUDA, "no usable current CUDA device");
    double *scratch;
    {
        // first call on this device: look up the array's device address (host code only
        // holds a stand-in for it)
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return reject(HAMR_ERR_CUDA, "cudaGetSymbolAddress of the step scratch array failed");
            g_scratch_ptr[dev] = (double *)ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    NoallocArgs a;
    a.p = *p;
    a.Sin = S_in;
    a.Sout = S_out;
    a.grain = grain;
    a.scratch = scratch;
    a.n = n;
    a.step = step;
    a.cJ = p->J / p->mu_s;
    a.cK = 2.0 * p->ku / p->mu_s;
    a.pref = -p->gamma / (1.0 + p->alpha * p->alpha);
    a.sig0 = sqrt(2.0 * p->alpha * KB / (p->gamma * p->mu_s * p->dt));
    a.c_fwhm = p->fwhm > 0 ? -4.0 * log(2.0) / (p->fwhm * p->fwhm) : 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_noalloc_predict<<<nb, 256, 0, st>>>(a);
    k_noalloc_correct<<<nb, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return reject(HAMR_ERR_CUDA, cudaGetErrorString(e));
    return HAMR_OK;
}
