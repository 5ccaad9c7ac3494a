// Fused FP32 sLLG Heun step for simple-cubic lattices: both Heun stages of a step in one
// pass over the spin state, for many replicas of uneven size in one persistent launch.
//
// Work item = a block of bx x by columns of one replica spanning all nz planes.  The CTA
// stages, plane by plane, the spins of the block plus a two-column halo in shared memory and
// marches up the planes.  At march step k it
//   1. predicts S' on plane k for every listed column: the block's interior and its
//      one-column halo, so the corrector never needs another CTA's S';
//   2. corrects plane k-1 on the interior columns from the S' planes k-2, k-1, k;
//   3. stages plane k+2 (loads issued before step 1, stored to shared memory after step 2).
// The list of columns is built on the host per work item: only columns inside the lattice
// that hold a magnetic site are listed (interior first), so lanes are not spent on the
// non-magnetic grain boundaries or on halos beyond an open edge.  Each thread owns the same
// P list entries for the whole march and keeps in registers what the next stage needs from
// its own column: S and the grain code of the previous plane, dt f(S, B(S)) and the thermal
// field of the plane awaiting correction.
// Each site's thermal normals come from its own (replica key, site, step) Philox counter, so
// halo sites computed by two CTAs get the same noise.  Open edges and non-magnetic sites read
// as S = 0 (the state of such sites is kept at 0), so the exchange sum needs no mask unless
// a replica has bonds between two different grains.
// Per step the kernel reads S once (12 B/site) plus the 2-byte grain code and writes S once
// (12 B/site); halo columns are re-read from L2.
#include "device_common.cuh"

namespace hamr {

template <int NT, int P, int CAPS>
struct FusedShape {
    static constexpr int LPT = (CAPS + NT - 1) / NT;  // staged positions per thread
    // S planes k, k+1 | S' planes (3) | grain codes (4 planes)
    static constexpr size_t smem = sizeof(float) * (2 * 3 * CAPS + 3 * 3 * CAPS) + sizeof(uint16_t) * 4 * CAPS;
};

__device__ __forceinline__ int wrap_coord(int v, int n, int per, bool &ok) {
    if (v >= 0 && v < n) return v;
    if (!per) {
        ok = false;
        return 0;
    }
    return ((v % n) + n) % n;
}

template <int NT, int P, int CAPS, bool RECORD>
__global__ void __launch_bounds__(NT, (NT >= 1024 ? 1 : (NT >= 512 ? 2 : 3))) k_fused(FusedArgs a) {
    using Sh = FusedShape<NT, P, CAPS>;
    constexpr int LPT = Sh::LPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sS = reinterpret_cast<float *>(smem_raw);                 // [2][3][CAPS]
    float *sP = sS + 2 * 3 * CAPS;                                    // [3][3][CAPS]
    uint16_t *sG = reinterpret_cast<uint16_t *>(sP + 3 * 3 * CAPS);  // [4][CAPS]
    __shared__ int s_item;
    __shared__ uint4 s_rk[5];  // Philox round keys of the current replica

    const int tid = threadIdx.x;
    const long long NS = a.NS;
    const long long step = a.ctl->step + a.step_off;
    const int par = (int)(step & 1);
    const float *__restrict__ Sin = par ? a.Sbuf1 : a.Sbuf0;
    float *__restrict__ Sout = par ? a.Sbuf0 : a.Sbuf1;
    if (blockIdx.x == 0 && tid == 0) a.ctl->work_ctr[par ^ 1] = 0u;  // next step's counter
    const float t = (float)step * a.dt;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&a.ctl->work_ctr[par], 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= a.n_items) break;
        const WorkItem W = a.items[it];
        const ReplicaDev &R = a.reps[W.r];
        const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px;
        const long long off = R.off;
        const int plane = px * ny;
        const int bx = W.bxy & 0xffff, by = W.bxy >> 16;
        const int WS = bx + 4, SA = WS * (by + 4);
        const int n_act = W.counts & 0xffff, n_int = W.counts >> 16;
        const bool mask = R.cross_grain != 0;
        if (tid < 5) {
            const unsigned k0 = R.key0 + 2u * tid * 0x9E3779B9u, k1 = R.key1 + 2u * tid * 0xBB67AE85u;
            s_rk[tid] = make_uint4(k0, k1, k0 + 0x9E3779B9u, k1 + 0xBB67AE85u);
        }
        // S' of unlisted positions must read as 0 for the whole item
        for (int i = tid; i < 9 * CAPS; i += NT) sP[i] = 0.0f;

        // this thread's list entries (site and storage indices fit in 32 bits: a replica
        // has at most 2^30 sites and the storage fewer than 2^28 slots)
        int pos[P];          // staged-region position, or -1
        bool inner[P];       // interior column: corrected here
        float sig[P];        // thermal-field scale of the column
        unsigned scol[P];    // site index of the column on plane 0
        int ocol[P];         // storage slot of the column on plane 0
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int e = tid + j * NT;
            pos[j] = -1;
            inner[j] = false;
            sig[j] = 0.f;
            scol[j] = 0;
            ocol[j] = 0;
            if (e < n_act) {
                const int p = a.lists[W.list_off + e];
                pos[j] = p;
                inner[j] = e < n_int;
                bool ok = true;
                const int wx = wrap_coord(W.x0 - 2 + p % WS, nx, a.per[0], ok);
                const int wy = wrap_coord(W.y0 - 2 + p / WS, ny, a.per[1], ok);
                const float T = temperature_f(R, (wx + 0.5f) * a.ax, (wy + 0.5f) * a.ay, t);
                sig[j] = a.sig0 * sqrtf(T);
                scol[j] = (unsigned)wx + (unsigned)nx * (unsigned)wy;
                ocol[j] = (int)off + wx + px * wy;
            }
        }
        // staged positions of this thread: column offsets within a plane, -1 if outside
        int lofs[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int idx = tid + l * NT;
            lofs[l] = -1;
            if (idx < SA) {
                bool ok = true;
                const int cx = wrap_coord(W.x0 - 2 + idx % WS, nx, a.per[0], ok);
                const int cy = wrap_coord(W.y0 - 2 + idx / WS, ny, a.per[1], ok);
                if (ok) lofs[l] = cx + px * cy;
            }
        }
        float pre[LPT][3];
        uint16_t preg[LPT];
        auto fetch = [&](int p) {
            bool ok = true;
            const int z = wrap_coord(p, nz, a.per[2], ok);
            const int base = (int)off + z * plane;
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                if (ok && lofs[l] >= 0) {
                    const int j = base + lofs[l];
                    pre[l][0] = __ldg(Sin + j);
                    pre[l][1] = __ldg(Sin + NS + j);
                    pre[l][2] = __ldg(Sin + 2 * NS + j);
                    preg[l] = __ldg(a.gcode + j);
                } else {
                    pre[l][0] = pre[l][1] = pre[l][2] = 0.0f;
                    preg[l] = 0;
                }
            }
        };
        auto stage = [&](int p) {
            float *dst = sS + (p & 1) * 3 * CAPS;
            uint16_t *gd = sG + (p & 3) * CAPS;
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                const int idx = tid + l * NT;
                if (idx < SA) {
                    dst[idx] = pre[l][0];
                    dst[CAPS + idx] = pre[l][1];
                    dst[2 * CAPS + idx] = pre[l][2];
                    gd[idx] = preg[l];
                }
            }
        };

        const float bapp = R.fB0 * field_polarity_f(R, a.bits, t);
        const float bax = bapp * R.fdir[0], bay = bapp * R.fdir[1], baz = bapp * R.fdir[2];
        const unsigned site_plane = (unsigned)nx * (unsigned)ny;
        const float q = a.pref * a.dt;

        // prologue: planes -2 and -1 staged, own S and grain code of plane -2 read
        fetch(-2);
        stage(-2);
        fetch(-1);
        stage(-1);
        __syncthreads();
        float Sm1[P][3];           // S on plane k-1 at this column
        unsigned gm1[P], gm2[P];   // grain codes on planes k-1 and k-2
        float f1[P][3], th[P][3];  // dt f(S, B(S)) and thermal field of plane k-1
        int acc[P][3], gacc[P];    // fixed-point record sums of this column
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int p = pos[j] < 0 ? 0 : pos[j];
            Sm1[j][0] = sS[p];  // plane -2 sits in S slot 0 and grain slot 2
            Sm1[j][1] = sS[CAPS + p];
            Sm1[j][2] = sS[2 * CAPS + p];
            gm1[j] = pos[j] < 0 ? 0u : sG[2 * CAPS + p];
            gm2[j] = 0;
            f1[j][0] = f1[j][1] = f1[j][2] = 0.f;
            th[j][0] = th[j][1] = th[j][2] = 0.f;
            acc[j][0] = acc[j][1] = acc[j][2] = 0;
            gacc[j] = -1;
        }
        __syncthreads();
        fetch(0);
        stage(0);
        __syncthreads();

        for (int k = -1; k <= nz; ++k) {
            fetch(k + 2);
            // ---- predictor on plane k
            const float *P0 = sS + (k & 1) * 3 * CAPS, *Pp = sS + ((k + 1) & 1) * 3 * CAPS;
            const uint16_t *G0 = sG + ((k + 4) & 3) * CAPS, *Gp = sG + ((k + 5) & 3) * CAPS;
            float *Pw = sP + ((k + 3) % 3) * 3 * CAPS;
            bool zok = true;
            const int wz = wrap_coord(k, nz, a.per[2], zok);
            float S0[P][3];
            unsigned g0[P];
            float nf1[P][3], nth[P][3];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int c = pos[j];
                nf1[j][0] = nf1[j][1] = nf1[j][2] = 0.f;
                nth[j][0] = nth[j][1] = nth[j][2] = 0.f;
                S0[j][0] = S0[j][1] = S0[j][2] = 0.f;
                g0[j] = 0;
                if (c < 0) continue;
                g0[j] = G0[c];
                const float sx = P0[c], sy = P0[CAPS + c], sz = P0[2 * CAPS + c];
                S0[j][0] = sx;
                S0[j][1] = sy;
                S0[j][2] = sz;
                float npx = 0.f, npy = 0.f, npz = 0.f;
                if (zok && g0[j] != 0) {
                    float ex, ey, ez;
                    if (!mask) {
                        ex = P0[c - 1] + P0[c + 1] + P0[c - WS] + P0[c + WS] + Sm1[j][0] + Pp[c];
                        ey = P0[CAPS + c - 1] + P0[CAPS + c + 1] + P0[CAPS + c - WS] + P0[CAPS + c + WS] + Sm1[j][1] +
                             Pp[CAPS + c];
                        ez = P0[2 * CAPS + c - 1] + P0[2 * CAPS + c + 1] + P0[2 * CAPS + c - WS] +
                             P0[2 * CAPS + c + WS] + Sm1[j][2] + Pp[2 * CAPS + c];
                    } else {
                        const unsigned g = g0[j];
                        const float w0 = G0[c - 1] == g, w1 = G0[c + 1] == g, w2 = G0[c - WS] == g,
                                    w3 = G0[c + WS] == g, w4 = gm1[j] == g, w5 = Gp[c] == g;
                        ex = w0 * P0[c - 1] + w1 * P0[c + 1] + w2 * P0[c - WS] + w3 * P0[c + WS] + w4 * Sm1[j][0] +
                             w5 * Pp[c];
                        ey = w0 * P0[CAPS + c - 1] + w1 * P0[CAPS + c + 1] + w2 * P0[CAPS + c - WS] +
                             w3 * P0[CAPS + c + WS] + w4 * Sm1[j][1] + w5 * Pp[CAPS + c];
                        ez = w0 * P0[2 * CAPS + c - 1] + w1 * P0[2 * CAPS + c + 1] + w2 * P0[2 * CAPS + c - WS] +
                             w3 * P0[2 * CAPS + c + WS] + w4 * Sm1[j][2] + w5 * Pp[2 * CAPS + c];
                    }
                    float n0, n1, n2;
                    normals3(philox10_rk(philox_ctr(scol[j] + site_plane * (unsigned)wz, (unsigned long long)step),
                                         s_rk),
                             n0, n1, n2);
                    const float tx = sig[j] * n0, ty = sig[j] * n1, tz = sig[j] * n2;
                    nth[j][0] = tx;
                    nth[j][1] = ty;
                    nth[j][2] = tz;
                    const float bx_ = fmaf(a.cJ, ex, bax + tx);
                    const float by_ = fmaf(a.cJ, ey, bay + ty);
                    const float bz_ = fmaf(a.cJ, ez, fmaf(a.cK, sz, baz + tz));
                    const float cx = sy * bz_ - sz * by_, cy = sz * bx_ - sx * bz_, cz = sx * by_ - sy * bx_;
                    const float sb = sx * bx_ + sy * by_ + sz * bz_, ss = sx * sx + sy * sy + sz * sz;
                    nf1[j][0] = q * (cx + a.alpha * (sb * sx - ss * bx_));
                    nf1[j][1] = q * (cy + a.alpha * (sb * sy - ss * by_));
                    nf1[j][2] = q * (cz + a.alpha * (sb * sz - ss * bz_));
                    npx = sx + nf1[j][0];
                    npy = sy + nf1[j][1];
                    npz = sz + nf1[j][2];
                    const float inv = rsqrtf(npx * npx + npy * npy + npz * npz);
                    npx *= inv;
                    npy *= inv;
                    npz *= inv;
                }
                Pw[c] = npx;
                Pw[CAPS + c] = npy;
                Pw[2 * CAPS + c] = npz;
            }
            __syncthreads();

            // ---- corrector on plane k-1
            const int kc = k - 1;
            if (kc >= 0 && kc < nz) {
                const float *Q = sP + ((kc + 3) % 3) * 3 * CAPS, *Qm = sP + ((kc + 2) % 3) * 3 * CAPS,
                            *Qp = sP + ((kc + 4) % 3) * 3 * CAPS;
                const uint16_t *Gc = sG + ((kc + 4) & 3) * CAPS;
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const int c = pos[j];
                    const unsigned g = gm1[j];
                    if (c < 0 || !inner[j] || g == 0) continue;
                    const float sx = Q[c], sy = Q[CAPS + c], sz = Q[2 * CAPS + c];
                    float ex, ey, ez;
                    if (!mask) {
                        ex = Q[c - 1] + Q[c + 1] + Q[c - WS] + Q[c + WS] + Qm[c] + Qp[c];
                        ey = Q[CAPS + c - 1] + Q[CAPS + c + 1] + Q[CAPS + c - WS] + Q[CAPS + c + WS] + Qm[CAPS + c] +
                             Qp[CAPS + c];
                        ez = Q[2 * CAPS + c - 1] + Q[2 * CAPS + c + 1] + Q[2 * CAPS + c - WS] + Q[2 * CAPS + c + WS] +
                             Qm[2 * CAPS + c] + Qp[2 * CAPS + c];
                    } else {
                        const float w0 = Gc[c - 1] == g, w1 = Gc[c + 1] == g, w2 = Gc[c - WS] == g,
                                    w3 = Gc[c + WS] == g, w4 = gm2[j] == g, w5 = g0[j] == g;
                        ex = w0 * Q[c - 1] + w1 * Q[c + 1] + w2 * Q[c - WS] + w3 * Q[c + WS] + w4 * Qm[c] + w5 * Qp[c];
                        ey = w0 * Q[CAPS + c - 1] + w1 * Q[CAPS + c + 1] + w2 * Q[CAPS + c - WS] +
                             w3 * Q[CAPS + c + WS] + w4 * Qm[CAPS + c] + w5 * Qp[CAPS + c];
                        ez = w0 * Q[2 * CAPS + c - 1] + w1 * Q[2 * CAPS + c + 1] + w2 * Q[2 * CAPS + c - WS] +
                             w3 * Q[2 * CAPS + c + WS] + w4 * Qm[2 * CAPS + c] + w5 * Qp[2 * CAPS + c];
                    }
                    const float bx_ = fmaf(a.cJ, ex, bax + th[j][0]);
                    const float by_ = fmaf(a.cJ, ey, bay + th[j][1]);
                    const float bz_ = fmaf(a.cJ, ez, fmaf(a.cK, sz, baz + th[j][2]));
                    const float cx = sy * bz_ - sz * by_, cy = sz * bx_ - sx * bz_, cz = sx * by_ - sy * bx_;
                    const float sb = sx * bx_ + sy * by_ + sz * bz_, ss = sx * sx + sy * sy + sz * sz;
                    const float f2x = q * (cx + a.alpha * (sb * sx - ss * bx_));
                    const float f2y = q * (cy + a.alpha * (sb * sy - ss * by_));
                    const float f2z = q * (cz + a.alpha * (sb * sz - ss * bz_));
                    float ox = Sm1[j][0] + 0.5f * (f1[j][0] + f2x);
                    float oy = Sm1[j][1] + 0.5f * (f1[j][1] + f2y);
                    float oz = Sm1[j][2] + 0.5f * (f1[j][2] + f2z);
                    const float inv = rsqrtf(ox * ox + oy * oy + oz * oz);
                    ox *= inv;
                    oy *= inv;
                    oz *= inv;
                    const int o = ocol[j] + kc * plane;
                    Sout[o] = ox;
                    Sout[NS + o] = oy;
                    Sout[2 * NS + o] = oz;
                    if (RECORD) {
                        const int gg = R.grain_off + (int)g - 1;
                        if (gg != gacc[j] || (kc & 63) == 63) {
                            if (gacc[j] >= 0) {
                                atomicAdd(a.grain_fx + 3 * gacc[j] + 0, (unsigned long long)(long long)acc[j][0]);
                                atomicAdd(a.grain_fx + 3 * gacc[j] + 1, (unsigned long long)(long long)acc[j][1]);
                                atomicAdd(a.grain_fx + 3 * gacc[j] + 2, (unsigned long long)(long long)acc[j][2]);
                            }
                            gacc[j] = gg;
                            acc[j][0] = acc[j][1] = acc[j][2] = 0;
                        }
                        acc[j][0] += __float2int_rn(ox * FX_SCALE);
                        acc[j][1] += __float2int_rn(oy * FX_SCALE);
                        acc[j][2] += __float2int_rn(oz * FX_SCALE);
                    }
                }
            }
            // carry this column's plane-k values to the next march step
#pragma unroll
            for (int j = 0; j < P; ++j) {
                gm2[j] = gm1[j];
                gm1[j] = g0[j];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    Sm1[j][d] = S0[j][d];
                    f1[j][d] = nf1[j][d];
                    th[j][d] = nth[j][d];
                }
            }
            stage(k + 2);
            __syncthreads();
        }
        if (RECORD) {
#pragma unroll
            for (int j = 0; j < P; ++j)
                grain_accumulate_fx(a.grain_fx, gacc[j], acc[j][0], acc[j][1], acc[j][2], gacc[j] >= 0);
        }
    }
}

// Opt in to the variant's dynamic shared memory (done before any stream capture, when the
// work list is built).
template <int NT, int P, int CAPS>
static cudaError_t ensure_attrs() {
    using Sh = FusedShape<NT, P, CAPS>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<NT, P, CAPS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Sh::smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_fused<NT, P, CAPS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Sh::smem);
        if (e != cudaSuccess) return e;
        init = true;
    }
    return cudaSuccess;
}

template <int NT, int P, int CAPS>
static cudaError_t launch_variant(const FusedArgs &a, int grid, bool record, cudaStream_t st) {
    using Sh = FusedShape<NT, P, CAPS>;
    cudaError_t e = ensure_attrs<NT, P, CAPS>();
    if (e != cudaSuccess) return e;
    if (record)
        k_fused<NT, P, CAPS, true><<<grid, NT, Sh::smem, st>>>(a);
    else
        k_fused<NT, P, CAPS, false><<<grid, NT, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

template <int NT, int P, int CAPS>
static int blocks_per_sm() {
    using Sh = FusedShape<NT, P, CAPS>;
    int n = 0;
    if (ensure_attrs<NT, P, CAPS>() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<NT, P, CAPS, false>, NT, Sh::smem) != cudaSuccess)
        return 0;
    return n;
}

// compiled variants: threads per CTA, list entries per thread, staged positions per plane
#define HAMR_FUSED_VARIANTS(X) X(0, 1024, 1, 1536) X(1, 512, 1, 768) X(2, 1024, 1, 1280) X(3, 256, 2, 768)

cudaError_t launch_fused_step(int v, const FusedArgs &a, int grid, bool record, cudaStream_t st) {
#define X(I, NT, P, C) \
    if (v == I) return launch_variant<NT, P, C>(a, grid, record, st);
    HAMR_FUSED_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

bool fused_variant(int v, FusedVariant &out) {
#define X(I, NT, P, C)      \
    if (v == I) {           \
        out.threads = NT;   \
        out.per_thread = P; \
        out.staged = C;     \
        return true;        \
    }
    HAMR_FUSED_VARIANTS(X)
#undef X
    return false;
}

int fused_max_blocks_per_sm(int v) {
#define X(I, NT, P, C) \
    if (v == I) return blocks_per_sm<NT, P, C>();
    HAMR_FUSED_VARIANTS(X)
#undef X
    return 0;
}

}  // namespace hamr
