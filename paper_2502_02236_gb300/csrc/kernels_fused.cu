// Fused FP32 sLLG Heun step for simple-cubic lattices: both Heun stages of a step in one
// pass over the spin state, for many replicas of uneven size in one persistent launch.
//
// Work item = one replica's block of bx x by columns (x, y) spanning all nz planes.  A CTA of
// TX x TY threads owns the block plus a one-column halo: thread (tx, ty) sits on column
// (x0 - 1 + tx, y0 - 1 + ty) and marches up the planes.  At march step k it
//   1. predicts S' on plane k at its column (halo columns included, so the corrector never
//      needs another CTA's S'), from the S planes k-1, k, k+1 staged in shared memory with
//      a two-column halo;
//   2. corrects plane k-1 on interior columns from the S' planes k-2, k-1, k, keeping
//      dt f(S, B(S)) and the thermal field of plane k-1 in registers from step 1;
//   3. stages S plane k+2 (loads issued before step 1, stored to shared memory after 2).
// Each site's thermal normals come from its own (replica key, site, step) Philox counter,
// so sites recomputed in two CTAs' halos get the same noise.  Open edges and non-magnetic
// sites read as S = 0 (the state of such sites is kept at 0), so the exchange sum needs no
// mask unless a replica has bonds between two different grains.
// Per step the kernel reads S once (12 B/site) plus the 2-byte grain code and writes S
// once (12 B/site); halos are re-read from L2.
#include "device_common.cuh"

namespace hamr {

template <int TX, int TY>
struct FusedShape {
    static constexpr int NT = TX * TY;
    static constexpr int SW = TX + 2, SH = TY + 2, SA = SW * SH;
    static constexpr int LPT = (SA + NT - 1) / NT;  // staged positions per thread
    static constexpr size_t smem = sizeof(float) * (4 * 3 * SA + 3 * 3 * NT) + sizeof(uint16_t) * 4 * SA;
};

__device__ __forceinline__ int wrap_coord(int v, int n, int per, bool &ok) {
    if (v >= 0 && v < n) return v;
    if (!per) {
        ok = false;
        return 0;
    }
    return ((v % n) + n) % n;
}

template <int TX, int TY, bool RECORD>
__global__ void __launch_bounds__(TX *TY) k_fused(FusedArgs a) {
    using Sh = FusedShape<TX, TY>;
    constexpr int NT = Sh::NT, SW = Sh::SW, SA = Sh::SA, LPT = Sh::LPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sS = reinterpret_cast<float *>(smem_raw);           // [4][3][SA]
    float *sP = sS + 4 * 3 * SA;                                // [3][3][NT]
    uint16_t *sG = reinterpret_cast<uint16_t *>(sP + 3 * 3 * NT);  // [4][SA]
    __shared__ int s_item;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
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
        const long long plane = (long long)px * ny;
        const int bx = W.bxy & 0xffff, by = W.bxy >> 16;
        const bool mask = R.cross_grain != 0;

        // staged positions of this thread: column offsets within a plane, -1 if outside
        int lofs[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int idx = tid + l * NT;
            lofs[l] = -1;
            if (idx < SA) {
                bool ok = true;
                const int cx = wrap_coord(W.x0 - 2 + idx % SW, nx, a.per[0], ok);
                const int cy = wrap_coord(W.y0 - 2 + idx / SW, ny, a.per[1], ok);
                if (ok) lofs[l] = cx + px * cy;
            }
        }
        auto plane_base = [&](int p, bool &ok) -> long long {
            ok = true;
            const int z = wrap_coord(p, nz, a.per[2], ok);
            return off + (long long)z * plane;
        };
        float pre[LPT][3];
        uint16_t preg[LPT];
        auto fetch = [&](int p) {
            bool ok;
            const long long base = plane_base(p, ok);
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                if (ok && lofs[l] >= 0) {
                    const long long j = base + lofs[l];
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
            const int sl = (p + 4) & 3;
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                const int idx = tid + l * NT;
                if (idx < SA) {
                    sS[(sl * 3 + 0) * SA + idx] = pre[l][0];
                    sS[(sl * 3 + 1) * SA + idx] = pre[l][1];
                    sS[(sl * 3 + 2) * SA + idx] = pre[l][2];
                    sG[sl * SA + idx] = preg[l];
                }
            }
        };

        // this thread's column
        bool colok = tx < bx + 2 && ty < by + 2;
        const int wx = wrap_coord(W.x0 - 1 + tx, nx, a.per[0], colok);
        const int wy = wrap_coord(W.y0 - 1 + ty, ny, a.per[1], colok);
        const bool interior = colok && tx >= 1 && tx <= bx && ty >= 1 && ty <= by;
        const int c = (ty + 1) * SW + (tx + 1);  // centre in the staged region
        float sig = 0.0f;
        if (colok) {
            const float T = temperature_f(R, (wx + 0.5f) * a.ax, (wy + 0.5f) * a.ay, t);
            sig = a.sig0 * sqrtf(T);
        }
        const float bapp = R.fB0 * field_polarity_f(R, a.bits, t);
        const float bax = bapp * R.fdir[0], bay = bapp * R.fdir[1], baz = bapp * R.fdir[2];
        const unsigned long long site_col = (unsigned long long)wx + (unsigned long long)nx * wy;
        const unsigned long long site_plane = (unsigned long long)nx * ny;

        // prologue: planes -2, -1, 0 staged
        fetch(-2);
        stage(-2);
        fetch(-1);
        stage(-1);
        fetch(0);
        stage(0);
        __syncthreads();

        float f1x = 0.f, f1y = 0.f, f1z = 0.f, thx = 0.f, thy = 0.f, thz = 0.f;  // plane k-1
        double accx = 0.0, accy = 0.0, accz = 0.0;
        int gacc = -1;
        unsigned gm2 = 0, gm1 = 0;  // grain codes of this column on planes k-2 and k-1

        for (int k = -1; k <= nz; ++k) {
            fetch(k + 2);
            // ---- predictor on plane k
            const int s0 = (k + 4) & 3, sm = (k + 3) & 3, sp = (k + 5) & 3;
            const int pk = (k + 3) % 3;
            float npx = 0.f, npy = 0.f, npz = 0.f;
            float nf1x = 0.f, nf1y = 0.f, nf1z = 0.f, nthx = 0.f, nthy = 0.f, nthz = 0.f;
            bool zok = true;
            const int wz = wrap_coord(k, nz, a.per[2], zok);
            const unsigned g0 = sG[s0 * SA + c];
            if (colok && zok && g0 != 0) {
                const float *P0 = sS + s0 * 3 * SA, *Pm = sS + sm * 3 * SA, *Pp = sS + sp * 3 * SA;
                const float sx = P0[c], sy = P0[SA + c], sz = P0[2 * SA + c];
                float ex, ey, ez;
                if (!mask) {
                    ex = P0[c - 1] + P0[c + 1] + P0[c - SW] + P0[c + SW] + Pm[c] + Pp[c];
                    ey = P0[SA + c - 1] + P0[SA + c + 1] + P0[SA + c - SW] + P0[SA + c + SW] + Pm[SA + c] + Pp[SA + c];
                    ez = P0[2 * SA + c - 1] + P0[2 * SA + c + 1] + P0[2 * SA + c - SW] + P0[2 * SA + c + SW] +
                         Pm[2 * SA + c] + Pp[2 * SA + c];
                } else {
                    const uint16_t *G0 = sG + s0 * SA;
                    const float w0 = G0[c - 1] == g0, w1 = G0[c + 1] == g0, w2 = G0[c - SW] == g0,
                                w3 = G0[c + SW] == g0, w4 = sG[sm * SA + c] == g0, w5 = sG[sp * SA + c] == g0;
                    ex = w0 * P0[c - 1] + w1 * P0[c + 1] + w2 * P0[c - SW] + w3 * P0[c + SW] + w4 * Pm[c] + w5 * Pp[c];
                    ey = w0 * P0[SA + c - 1] + w1 * P0[SA + c + 1] + w2 * P0[SA + c - SW] + w3 * P0[SA + c + SW] +
                         w4 * Pm[SA + c] + w5 * Pp[SA + c];
                    ez = w0 * P0[2 * SA + c - 1] + w1 * P0[2 * SA + c + 1] + w2 * P0[2 * SA + c - SW] +
                         w3 * P0[2 * SA + c + SW] + w4 * Pm[2 * SA + c] + w5 * Pp[2 * SA + c];
                }
                float n0, n1, n2;
                normals3(philox_site(R.key0, R.key1, site_col + site_plane * (unsigned long long)wz,
                                     (unsigned long long)step),
                         n0, n1, n2);
                nthx = sig * n0;
                nthy = sig * n1;
                nthz = sig * n2;
                const float bx_ = a.cJ * ex + bax + nthx;
                const float by_ = a.cJ * ey + bay + nthy;
                const float bz_ = a.cJ * ez + a.cK * sz + baz + nthz;
                const float cx = sy * bz_ - sz * by_, cy = sz * bx_ - sx * bz_, cz = sx * by_ - sy * bx_;
                const float sb = sx * bx_ + sy * by_ + sz * bz_, ss = sx * sx + sy * sy + sz * sz;
                const float q = a.pref * a.dt;
                nf1x = q * (cx + a.alpha * (sb * sx - ss * bx_));
                nf1y = q * (cy + a.alpha * (sb * sy - ss * by_));
                nf1z = q * (cz + a.alpha * (sb * sz - ss * bz_));
                npx = sx + nf1x;
                npy = sy + nf1y;
                npz = sz + nf1z;
                const float inv = rsqrtf(npx * npx + npy * npy + npz * npz);
                npx *= inv;
                npy *= inv;
                npz *= inv;
            }
            sP[(pk * 3 + 0) * NT + tid] = npx;
            sP[(pk * 3 + 1) * NT + tid] = npy;
            sP[(pk * 3 + 2) * NT + tid] = npz;
            __syncthreads();

            // ---- corrector on plane k-1
            const int kc = k - 1;
            if (interior && kc >= 0 && kc < nz) {
                const int sc = (kc + 4) & 3;
                const unsigned g = gm1;
                if (g != 0) {
                    const int pc = (kc + 3) % 3, pm = (kc + 2) % 3, pp = (kc + 4) % 3;
                    const float *Q = sP + pc * 3 * NT, *Qm = sP + pm * 3 * NT, *Qp = sP + pp * 3 * NT;
                    const int i = tid;
                    const float sx = Q[i], sy = Q[NT + i], sz = Q[2 * NT + i];
                    float ex, ey, ez;
                    if (!mask) {
                        ex = Q[i - 1] + Q[i + 1] + Q[i - TX] + Q[i + TX] + Qm[i] + Qp[i];
                        ey = Q[NT + i - 1] + Q[NT + i + 1] + Q[NT + i - TX] + Q[NT + i + TX] + Qm[NT + i] + Qp[NT + i];
                        ez = Q[2 * NT + i - 1] + Q[2 * NT + i + 1] + Q[2 * NT + i - TX] + Q[2 * NT + i + TX] +
                             Qm[2 * NT + i] + Qp[2 * NT + i];
                    } else {
                        const uint16_t *G0 = sG + sc * SA;
                        // plane kc-1 is being restaged by other threads: use this column's codes
                        const float w0 = G0[c - 1] == g, w1 = G0[c + 1] == g, w2 = G0[c - SW] == g,
                                    w3 = G0[c + SW] == g, w4 = gm2 == g, w5 = g0 == g;
                        ex = w0 * Q[i - 1] + w1 * Q[i + 1] + w2 * Q[i - TX] + w3 * Q[i + TX] + w4 * Qm[i] + w5 * Qp[i];
                        ey = w0 * Q[NT + i - 1] + w1 * Q[NT + i + 1] + w2 * Q[NT + i - TX] + w3 * Q[NT + i + TX] +
                             w4 * Qm[NT + i] + w5 * Qp[NT + i];
                        ez = w0 * Q[2 * NT + i - 1] + w1 * Q[2 * NT + i + 1] + w2 * Q[2 * NT + i - TX] +
                             w3 * Q[2 * NT + i + TX] + w4 * Qm[2 * NT + i] + w5 * Qp[2 * NT + i];
                    }
                    const float bx_ = a.cJ * ex + bax + thx;
                    const float by_ = a.cJ * ey + bay + thy;
                    const float bz_ = a.cJ * ez + a.cK * sz + baz + thz;
                    const float cx = sy * bz_ - sz * by_, cy = sz * bx_ - sx * bz_, cz = sx * by_ - sy * bx_;
                    const float sb = sx * bx_ + sy * by_ + sz * bz_, ss = sx * sx + sy * sy + sz * sz;
                    const float q = a.pref * a.dt;
                    const float f2x = q * (cx + a.alpha * (sb * sx - ss * bx_));
                    const float f2y = q * (cy + a.alpha * (sb * sy - ss * by_));
                    const float f2z = q * (cz + a.alpha * (sb * sz - ss * bz_));
                    const float *O = sS + sc * 3 * SA;
                    float ox = O[c] + 0.5f * (f1x + f2x);
                    float oy = O[SA + c] + 0.5f * (f1y + f2y);
                    float oz = O[2 * SA + c] + 0.5f * (f1z + f2z);
                    const float inv = rsqrtf(ox * ox + oy * oy + oz * oz);
                    ox *= inv;
                    oy *= inv;
                    oz *= inv;
                    const long long j = off + wx + (long long)px * wy + (long long)kc * plane;
                    Sout[j] = ox;
                    Sout[NS + j] = oy;
                    Sout[2 * NS + j] = oz;
                    if (RECORD) {
                        const int gg = R.grain_off + (int)g - 1;
                        if (gg != gacc) {
                            if (gacc >= 0) {
                                atomicAdd(a.grain_acc + 3 * gacc + 0, accx);
                                atomicAdd(a.grain_acc + 3 * gacc + 1, accy);
                                atomicAdd(a.grain_acc + 3 * gacc + 2, accz);
                            }
                            gacc = gg;
                            accx = accy = accz = 0.0;
                        }
                        accx += ox;
                        accy += oy;
                        accz += oz;
                    }
                }
            }
            gm2 = gm1;
            gm1 = g0;
            f1x = nf1x;
            f1y = nf1y;
            f1z = nf1z;
            thx = nthx;
            thy = nthy;
            thz = nthz;
            stage(k + 2);
            __syncthreads();
        }
        if (RECORD) {
            grain_accumulate(a.grain_acc, gacc, accx, accy, accz, gacc >= 0);
        }
    }
}

// Opt in to the shape's dynamic shared memory (done before any stream capture, when the
// work list is built).
template <int TX, int TY>
static cudaError_t ensure_attrs() {
    using Sh = FusedShape<TX, TY>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<TX, TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Sh::smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_fused<TX, TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        init = true;
    }
    return cudaSuccess;
}

template <int TX, int TY>
static cudaError_t launch_shape(const FusedArgs &a, int grid, bool record, cudaStream_t st) {
    using Sh = FusedShape<TX, TY>;
    cudaError_t e = ensure_attrs<TX, TY>();
    if (e != cudaSuccess) return e;
    if (record)
        k_fused<TX, TY, true><<<grid, Sh::NT, Sh::smem, st>>>(a);
    else
        k_fused<TX, TY, false><<<grid, Sh::NT, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY>
static int blocks_per_sm() {
    using Sh = FusedShape<TX, TY>;
    int n = 0;
    if (ensure_attrs<TX, TY>() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<TX, TY, false>, Sh::NT, Sh::smem) != cudaSuccess)
        return 0;
    return n;
}

#define HAMR_FUSED_SHAPES(X) X(32, 8) X(32, 16) X(64, 8) X(64, 16) X(16, 16)

cudaError_t launch_fused_step(int tx, int ty, const FusedArgs &a, int grid, bool record, cudaStream_t st) {
#define X(A, B) \
    if (tx == A && ty == B) return launch_shape<A, B>(a, grid, record, st);
    HAMR_FUSED_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

bool fused_shape_compiled(int tx, int ty) {
#define X(A, B) \
    if (tx == A && ty == B) return true;
    HAMR_FUSED_SHAPES(X)
#undef X
    return false;
}

int fused_max_blocks_per_sm(int tx, int ty) {
#define X(A, B) \
    if (tx == A && ty == B) return blocks_per_sm<A, B>();
    HAMR_FUSED_SHAPES(X)
#undef X
    return 0;
}

void fused_shapes(std::vector<std::pair<int, int>> &out) {
    out.clear();
#define X(A, B) out.push_back({A, B});
    HAMR_FUSED_SHAPES(X)
#undef X
}

}  // namespace hamr
