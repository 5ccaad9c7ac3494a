// Fused FP32 sLLG Heun step for simple-cubic lattices: both Heun stages of a step in one
// pass over the spin state, for many replicas of uneven size in one persistent launch.
//
// Work item = a block of bx x by columns of one replica spanning all nz planes.  The CTA
// stages, plane by plane, the spins of the block plus a two-column halo in shared memory and
// marches up the planes.  Staging runs three planes ahead of the march through a four-slot
// ring with one mbarrier per slot: one thread issues a TMA tile copy of the three spin
// components (zero-filled beyond open edges); replicas whose blocks wrap around a periodic
// edge, or whose grains touch, are staged instead by per-position cp.async copies that arrive
// on the same mbarriers.  At march step k the CTA
//   1. starts staging plane k+3 into the slot that plane k-1 has left;
//   2. waits for plane k+1;
//   3. predicts S' on plane k for every listed column: the block's interior and its
//      one-column halo, so the corrector never needs another CTA's S';
//   4. synchronises once;
//   5. corrects plane k-1 on the interior columns from the S' planes k-2, k-1, k.
// With four S and four S' slots no other barrier is needed: the next step's writes go to
// slots that no thread can still be reading.  The four slot mbarriers are initialised once
// per kernel and keep running phases across work items.
// The list of columns is built on the host per work item: only columns inside the lattice
// that hold a magnetic site are listed, so lanes are not spent on the non-magnetic grain
// boundaries or on halos beyond an open edge; interior columns come first, flagged in the
// list entry.  Each thread owns one list
// entry for the whole march and keeps in registers what the next stage needs from its own
// column: S of the previous plane, dt f(S, B(S)) and the thermal field of the plane awaiting
// correction.  The march is unrolled over the ring period so that ring slots and neighbour
// offsets are compile-time constants.
// Each site's thermal normals come from its own (replica key, site, step) Philox counter, so
// halo sites computed by two CTAs get the same noise.  Open edges and non-magnetic sites read
// as S = 0 (the state of such sites is kept at 0): a zero spin marks a non-magnetic site and
// adds nothing to the exchange sum, so grain codes are read only at record steps (for the
// per-grain sums) and for replicas whose grains touch (the exchange mask).
// Per step the kernel reads S once (12 B/site) and writes S once (12 B/site); halo columns
// are re-read from L2.
#include "device_common.cuh"

namespace hamr {

constexpr int NSLOT = 4;                  // ring depth (planes)
constexpr unsigned WAIT_LIMIT = 1u << 22;  // polls of an mbarrier before the kernel gives up

template <int NT, int SW, int SH>
struct FusedShape {
    static constexpr int CAPS = SW * SH;               // staged positions per plane
    static constexpr int LPT = (CAPS + NT - 1) / NT;  // per-position copies per thread (fallback)
    // one S slot: the TMA box [3 components][SH rows][SW columns], rounded to 128 B
    static constexpr int SLOT_F = ((3 * CAPS * 4 + 127) / 128) * 128 / 4;
    static constexpr size_t smem = 128 + sizeof(float) * NSLOT * SLOT_F + sizeof(float4) * NSLOT * CAPS +
                                   sizeof(uint16_t) * NSLOT * CAPS;
};

template <int V>
struct IC {
    static constexpr int value = V;
};

__device__ __forceinline__ int wrap_coord(int v, int n, int per, bool &ok) {
    if (v >= 0 && v < n) return v;
    if (!per) {
        ok = false;
        return 0;
    }
    return ((v % n) + n) % n;
}

__device__ __forceinline__ bool nonzero3(float x, float y, float z) {
    return ((__float_as_uint(x) | __float_as_uint(y) | __float_as_uint(z)) << 1) != 0u;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}

// this thread's earlier cp.async copies arrive on b once they have landed
__device__ __forceinline__ void mbar_arrive_cp_async(unsigned long long *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false when the phase did not complete within WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    for (unsigned i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

// TMA tile copy of box (x, y, z, component) of a 4-D tensor map into shared memory
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int c,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(c), "r"(smem_u32(bar))
        : "memory");
}

// f(S, B) / (dt pref) = S x B + alpha [(S.B) S - (S.S) B]  (Eq. 1 in Landau-Lifshitz form)
__device__ __forceinline__ float3 rhs_u(float sx, float sy, float sz, float ss, float bx, float by, float bz,
                                        float al) {
    const float cx = sy * bz - sz * by, cy = sz * bx - sx * bz, cz = sx * by - sy * bx;
    const float sb = sx * bx + sy * by + sz * bz;
    return make_float3(fmaf(al, fmaf(sb, sx, -ss * bx), cx), fmaf(al, fmaf(sb, sy, -ss * by), cy),
                       fmaf(al, fmaf(sb, sz, -ss * bz), cz));
}

template <int NT, int SW, int SH, bool RECORD>
__global__ void __launch_bounds__(NT, (NT >= 1024 ? 1 : (NT >= 512 ? 2 : 3))) k_fused(FusedArgs a) {
    using Sh = FusedShape<NT, SW, SH>;
    constexpr int CAPS = Sh::CAPS, LPT = Sh::LPT, SLOT_F = Sh::SLOT_F;
    extern __shared__ unsigned char smem_raw[];
    float *sS = reinterpret_cast<float *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);  // [4][SLOT_F]
    float4 *sP = reinterpret_cast<float4 *>(sS + NSLOT * SLOT_F);                          // [4][CAPS]
    uint16_t *sG = reinterpret_cast<uint16_t *>(sP + NSLOT * CAPS);                        // [4][CAPS]
    __shared__ int s_item;
    __shared__ uint4 s_rk[5];  // Philox round keys of the current replica
    __shared__ __align__(8) unsigned long long s_bar[NSLOT];

    const int tid = threadIdx.x;
    const long long NS = a.NS;
    const long long step = a.ctl->step + a.step_off;
    const int par = (int)(step & 1);
    const float *__restrict__ Sin = par ? a.Sbuf1 : a.Sbuf0;
    float *__restrict__ Sout = par ? a.Sbuf0 : a.Sbuf1;
    if (blockIdx.x == 0 && tid == 0) a.ctl->work_ctr[par ^ 1] = 0u;  // next step's counter
    const float t = (float)step * a.dt;
    const float q = a.pref * a.dt;
    bool stop = false;  // a bounded wait ran out (decided uniformly by barrier vote)
    // The slot barriers live for the whole kernel: every thread arrives once per fill (the TMA
    // issuer with the expected byte count, per-position copies through cp.async), and each
    // thread tracks the parity of the next phase of every slot in ph.
    unsigned ph = 0;
    if (tid < NSLOT) mbar_init(&s_bar[tid], (unsigned)NT);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&a.ctl->work_ctr[par], 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= a.n_items) break;
        const WorkItem W = a.items[it];
        const ReplicaDev &R = a.reps[W.r];
        const int nx = R.nx, ny = R.ny, nz = R.nz, px = R.px;
        const int off = (int)R.off;
        const int plane = px * ny;
        const int bx = W.bxy & 0xffff, by = W.bxy >> 16;
        const int n_act = W.counts & 0xffff;
        const bool mask = R.cross_grain != 0;
        const bool tma = (W.stage & 1) != 0;
        const int xs = W.x0 - 2 - (W.stage >> 8), ys = W.y0 - 2;  // staged-region origin
        const CUtensorMap *map = a.maps + 2 * W.r + par;
        if (tid < 5) {
            const unsigned k0 = R.key0 + 2u * tid * 0x9E3779B9u, k1 = R.key1 + 2u * tid * 0xBB67AE85u;
            s_rk[tid] = make_uint4(k0, k1, k0 + 0x9E3779B9u, k1 + 0xBB67AE85u);
        }
        // S' (and its grain code) of unlisted positions must read as 0 for the whole item
        for (int i = tid; i < NSLOT * CAPS; i += NT) sP[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();

        // this thread's list entry (site and storage indices fit in 32 bits: a replica has at
        // most 2^30 sites and the storage fewer than 2^28 slots)
        const bool act = tid < n_act;
        bool inner = false;  // interior column: corrected by this thread
        int c = 0;           // staged-region position
        float sig = 0.f;     // thermal-field scale of the column
        unsigned scol = 0;   // site index of the column on plane 0
        int ocol = 0;        // storage slot of the column on plane 0
        if (act) {
            const unsigned e = a.lists[W.list_off + tid];
            c = (int)(e & 0x7fffu);
            inner = (e & 0x8000u) != 0;
            bool ok = true;
            const int wx = wrap_coord(xs + c % SW, nx, a.per[0], ok);
            const int wy = wrap_coord(ys + c / SW, ny, a.per[1], ok);
            const float T = temperature_f(R, (wx + 0.5f) * a.ax, (wy + 0.5f) * a.ay, t);
            sig = a.sig0 * sqrtf(T);
            scol = (unsigned)wx + (unsigned)nx * (unsigned)wy;
            ocol = off + wx + px * wy;
        }
        // per-position copies (fallback): column offsets within a plane (-1: zero-filled,
        // -2: outside the block's staged region)
        int lofs[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int idx = tid + l * NT;
            const int sx = idx % SW, sy = idx / SW;
            lofs[l] = -2;
            if (!tma && idx < CAPS && sx < bx + 4 && sy < by + 4) {
                bool ok = true;
                const int cx = wrap_coord(xs + sx, nx, a.per[0], ok);
                const int cy = wrap_coord(ys + sy, ny, a.per[1], ok);
                lofs[l] = ok ? cx + px * cy : -1;
            }
        }
        // stage plane p into ring slot p mod 4 (planes beyond nz + 1 are never needed)
        auto issue = [&](int p) {
            if (p > nz + 1) return;
            const int slot = (p + 4) & 3;
            float *dst = sS + slot * SLOT_F;
            bool ok = true;
            const int z = wrap_coord(p, nz, a.per[2], ok);
            if (tma) {
                if (tid == 0) {
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    mbar_expect_tx(&s_bar[slot], 3u * CAPS * 4u);
                    // an out-of-range plane of an open lattice: every element is zero-filled
                    tma_load_4d(dst, map, xs, ys, ok ? z : -2, 0, &s_bar[slot]);
                } else {
                    mbar_arrive(&s_bar[slot]);
                }
            } else {
                const int base = off + z * plane;
                uint16_t *gd = sG + slot * CAPS;
#pragma unroll
                for (int l = 0; l < LPT; ++l) {
                    if (lofs[l] == -2) continue;
                    const int idx = tid + l * NT;
                    const bool v = ok && lofs[l] >= 0;
                    const float *src = Sin + (v ? base + lofs[l] : 0);
                    cp_async4(dst + idx, src, v);
                    cp_async4(dst + CAPS + idx, src + NS, v);
                    cp_async4(dst + 2 * CAPS + idx, src + 2 * NS, v);
                    if (mask) gd[idx] = v ? __ldg(a.gcode + base + lofs[l]) : (uint16_t)0;
                }
                mbar_arrive_cp_async(&s_bar[slot]);
            }
        };
        // wait until plane p has landed in its slot; a wait that runs out is recorded here and
        // acted on at the next barrier vote
        bool bad = false;
        auto await = [&](int p) {
            const int slot = (p + 4) & 3;
            if (!mbar_wait(&s_bar[slot], (ph >> slot) & 1u)) {
                bad = true;
                atomicOr(&a.ctl->err, 2);
            }
            ph ^= 1u << slot;
        };

        const float bapp = R.fB0 * field_polarity_f(R, a.bits, t);
        const float bax = bapp * R.fdir[0], bay = bapp * R.fdir[1], baz = bapp * R.fdir[2];
        const unsigned site_plane = (unsigned)nx * (unsigned)ny;

        // prologue: planes -2 .. 1 staged; own S (and grain code) of plane -2 read
        issue(-2);
        issue(-1);
        issue(0);
        issue(1);
        await(-2);
        await(-1);
        await(0);
        float m1x = 0.f, m1y = 0.f, m1z = 0.f;     // S on plane k-1 at this column
        float c0x = 0.f, c0y = 0.f, c0z = 0.f;     // S on plane k
        unsigned gm1 = 0;                           // grain code of plane k-1 (masked replicas)
        float amx = 0.f, amy = 0.f, amz = 0.f;     // S + dt f(S, B(S)) / 2 of plane k-1
        float hmx = 0.f, hmy = 0.f, hmz = 0.f;     // B_app + B_th of plane k-1
        int ax_ = 0, ay_ = 0, az_ = 0, gacc = -1;  // fixed-point record sums of this column
        if (act) {
            const float *S2 = sS + 2 * SLOT_F, *S3 = sS + 3 * SLOT_F;  // planes -2 and -1
            m1x = S2[c];
            m1y = S2[CAPS + c];
            m1z = S2[2 * CAPS + c];
            gm1 = sG[2 * CAPS + c];
            c0x = S3[c];
            c0y = S3[CAPS + c];
            c0z = S3[2 * CAPS + c];
        }
        // plane -2's slot is restaged by the first march step; plain grain-code stores become visible
        stop = __syncthreads_or(bad) != 0;

        // one march step; PH fixes the ring slots: plane k sits in slot (PH + 3) % 4
        auto march = [&](auto PHC, int k) {
            constexpr int PH = decltype(PHC)::value;
            constexpr int SK = (PH + 3) & 3, SK1 = PH & 3, SKM1 = (PH + 2) & 3, SKM2 = (PH + 1) & 3;
            issue(k + 3);  // into slot (k + 3) mod 4 = SKM1, left by plane k-1 (kept in registers)
            if (k >= 0) await(k + 1);  // plane 0 was awaited by the prologue
            // ---- predictor on plane k (its own S is in c0, carried from the last step)
            bool zok = true;
            const int wz = wrap_coord(k, nz, a.per[2], zok);
            const float *P0 = sS + SK * SLOT_F + c, *Pp = sS + SK1 * SLOT_F + c;
            const float sx = c0x, sy = c0y, sz = c0z;
            const float ppx = Pp[0], ppy = Pp[CAPS], ppz = Pp[2 * CAPS];
            unsigned g0 = 0;
            float anx = 0.f, any = 0.f, anz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
            float4 sp = make_float4(0.f, 0.f, 0.f, 0.f);
            if (act) {
                if (mask) g0 = sG[SK * CAPS + c];
                const bool mag = mask ? g0 != 0 : nonzero3(sx, sy, sz);
                if (zok && mag) {
                    float n0, n1, n2;
                    normals3(philox10_rk(philox_ctr(scol + site_plane * (unsigned)wz, (unsigned long long)step), s_rk),
                             n0, n1, n2);
                    hx = fmaf(sig, n0, bax);
                    hy = fmaf(sig, n1, bay);
                    hz = fmaf(sig, n2, baz);
                    float ex, ey, ez;
                    if (!mask) {
                        ex = ((P0[-1] + P0[1]) + (P0[-SW] + P0[SW])) + (m1x + ppx);
                        ey = ((P0[CAPS - 1] + P0[CAPS + 1]) + (P0[CAPS - SW] + P0[CAPS + SW])) + (m1y + ppy);
                        ez = ((P0[2 * CAPS - 1] + P0[2 * CAPS + 1]) + (P0[2 * CAPS - SW] + P0[2 * CAPS + SW])) +
                             (m1z + ppz);
                    } else {
                        const uint16_t *G0 = sG + SK * CAPS + c;
                        const float w0 = G0[-1] == g0, w1 = G0[1] == g0, w2 = G0[-SW] == g0, w3 = G0[SW] == g0,
                                    w4 = gm1 == g0, w5 = sG[SK1 * CAPS + c] == g0;
                        ex = w0 * P0[-1] + w1 * P0[1] + w2 * P0[-SW] + w3 * P0[SW] + w4 * m1x + w5 * ppx;
                        ey = w0 * P0[CAPS - 1] + w1 * P0[CAPS + 1] + w2 * P0[CAPS - SW] + w3 * P0[CAPS + SW] +
                             w4 * m1y + w5 * ppy;
                        ez = w0 * P0[2 * CAPS - 1] + w1 * P0[2 * CAPS + 1] + w2 * P0[2 * CAPS - SW] +
                             w3 * P0[2 * CAPS + SW] + w4 * m1z + w5 * ppz;
                    }
                    const float ss = fmaf(sx, sx, fmaf(sy, sy, sz * sz));
                    const float3 u = rhs_u(sx, sy, sz, ss, fmaf(a.cJ, ex, hx), fmaf(a.cJ, ey, hy),
                                           fmaf(a.cJ, ez, fmaf(a.cK, sz, hz)), a.alpha);
                    const float fx = q * u.x, fy = q * u.y, fz = q * u.z;
                    anx = fmaf(0.5f, fx, sx);
                    any = fmaf(0.5f, fy, sy);
                    anz = fmaf(0.5f, fz, sz);
                    const float npx = sx + fx, npy = sy + fy, npz = sz + fz;
                    const float inv = rsqrtf(npx * npx + npy * npy + npz * npz);
                    sp = make_float4(npx * inv, npy * inv, npz * inv, __uint_as_float(g0));
                }
                sP[SK * CAPS + c] = sp;
            }
            stop = __syncthreads_or(bad) != 0;  // the step's one barrier, and the failure vote
            // ---- corrector on plane k-1 from S' planes k-2 (slot SKM2), k-1 (SKM1) and k (own, sp)
            const int kc = k - 1;
            if (inner && kc >= 0 && kc < nz) {
                const float4 *Q = sP + SKM1 * CAPS + c;
                const float4 v = Q[0];
                if (nonzero3(v.x, v.y, v.z)) {
                    const float4 l = Q[-1], r = Q[1], d = Q[-SW], u4 = Q[SW];
                    const float4 zm = sP[SKM2 * CAPS + c];
                    float ex, ey, ez;
                    if (!mask) {
                        ex = ((l.x + r.x) + (d.x + u4.x)) + (zm.x + sp.x);
                        ey = ((l.y + r.y) + (d.y + u4.y)) + (zm.y + sp.y);
                        ez = ((l.z + r.z) + (d.z + u4.z)) + (zm.z + sp.z);
                    } else {
                        const unsigned g = __float_as_uint(v.w);
                        const float w0 = __float_as_uint(l.w) == g, w1 = __float_as_uint(r.w) == g,
                                    w2 = __float_as_uint(d.w) == g, w3 = __float_as_uint(u4.w) == g,
                                    w4 = __float_as_uint(zm.w) == g, w5 = __float_as_uint(sp.w) == g;
                        ex = w0 * l.x + w1 * r.x + w2 * d.x + w3 * u4.x + w4 * zm.x + w5 * sp.x;
                        ey = w0 * l.y + w1 * r.y + w2 * d.y + w3 * u4.y + w4 * zm.y + w5 * sp.y;
                        ez = w0 * l.z + w1 * r.z + w2 * d.z + w3 * u4.z + w4 * zm.z + w5 * sp.z;
                    }
                    // S' is a unit vector: S'.S' = 1 in the damping term
                    const float3 u = rhs_u(v.x, v.y, v.z, 1.f, fmaf(a.cJ, ex, hmx), fmaf(a.cJ, ey, hmy),
                                           fmaf(a.cJ, ez, fmaf(a.cK, v.z, hmz)), a.alpha);
                    const float qh = 0.5f * q;
                    float ox = fmaf(qh, u.x, amx), oy = fmaf(qh, u.y, amy), oz = fmaf(qh, u.z, amz);
                    const float inv = rsqrtf(ox * ox + oy * oy + oz * oz);
                    ox *= inv;
                    oy *= inv;
                    oz *= inv;
                    const int o = ocol + kc * plane;
                    Sout[o] = ox;
                    Sout[NS + o] = oy;
                    Sout[2 * NS + o] = oz;
                    if (RECORD) {
                        const unsigned g = mask ? __float_as_uint(v.w) : (unsigned)__ldg(a.gcode + o);
                        const int gg = R.grain_off + (int)g - 1;
                        if (gg != gacc || (kc & 63) == 63) {
                            if (gacc >= 0) {
                                atomicAdd(a.grain_fx + 3 * gacc + 0, (unsigned long long)(long long)ax_);
                                atomicAdd(a.grain_fx + 3 * gacc + 1, (unsigned long long)(long long)ay_);
                                atomicAdd(a.grain_fx + 3 * gacc + 2, (unsigned long long)(long long)az_);
                            }
                            gacc = gg;
                            ax_ = ay_ = az_ = 0;
                        }
                        ax_ += __float2int_rn(ox * FX_SCALE);
                        ay_ += __float2int_rn(oy * FX_SCALE);
                        az_ += __float2int_rn(oz * FX_SCALE);
                    }
                }
            }
            // carry this column's plane-k values to the next march step
            m1x = sx;
            m1y = sy;
            m1z = sz;
            c0x = ppx;
            c0y = ppy;
            c0z = ppz;
            gm1 = g0;
            amx = anx;
            amy = any;
            amz = anz;
            hmx = hx;
            hmy = hy;
            hmz = hz;
        };

        // k runs from -1 to nz; k = kb + PH with kb = -1 (mod 4), so plane k sits in slot (PH + 3) % 4
        int kend = -2;  // last march step run
        for (int kb = -1; kb <= nz && !stop; kb += 4) {
            march(IC<0>(), kb);
            kend = kb;
            if (!stop && kb + 1 <= nz) march(IC<1>(), kend = kb + 1);
            if (!stop && kb + 2 <= nz) march(IC<2>(), kend = kb + 2);
            if (!stop && kb + 3 <= nz) march(IC<3>(), kend = kb + 3);
        }
        if (stop) {
            // give the fills issued after the last awaited plane a bounded time to land before
            // the CTA's shared memory is released
            if (tid == 0)
                for (int p = max(kend + 2, 1); p <= min(kend + 3, nz + 1); ++p) await(p);
            return;  // uniform: every thread saw the same vote
        }
        if (RECORD) grain_accumulate_fx(a.grain_fx, gacc, ax_, ay_, az_, gacc >= 0);
        __syncthreads();  // all reads of this item's slots are done before they are re-armed
    }
}

// Opt in to the variant's dynamic shared memory (done before any stream capture, when the
// work list is built).
template <int NT, int SW, int SH>
static cudaError_t ensure_attrs() {
    using Sh = FusedShape<NT, SW, SH>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<NT, SW, SH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Sh::smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_fused<NT, SW, SH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Sh::smem);
        if (e != cudaSuccess) return e;
        init = true;
    }
    return cudaSuccess;
}

template <int NT, int SW, int SH>
static cudaError_t launch_variant(const FusedArgs &a, int grid, bool record, cudaStream_t st) {
    using Sh = FusedShape<NT, SW, SH>;
    cudaError_t e = ensure_attrs<NT, SW, SH>();
    if (e != cudaSuccess) return e;
    if (record)
        k_fused<NT, SW, SH, true><<<grid, NT, Sh::smem, st>>>(a);
    else
        k_fused<NT, SW, SH, false><<<grid, NT, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

template <int NT, int SW, int SH>
static int blocks_per_sm() {
    using Sh = FusedShape<NT, SW, SH>;
    int n = 0;
    if (ensure_attrs<NT, SW, SH>() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<NT, SW, SH, false>, NT, Sh::smem) != cudaSuccess)
        return 0;
    return n;
}

// compiled variants: threads per CTA and the staged region's pitch x rows (pitch a multiple
// of 4 so that TMA rows are 16-byte multiples).  A block of bx x by columns fits when
// bx + 4 <= pitch (bx + 7 with TMA, whose origin is rounded down to a multiple of 4),
// by + 4 <= rows and it lists at most one column per thread.
#define HAMR_FUSED_VARIANTS(X) X(0, 1024, 68, 24) X(1, 512, 36, 24) X(2, 256, 36, 14) X(3, 1024, 36, 40)

cudaError_t launch_fused_step(int v, const FusedArgs &a, int grid, bool record, cudaStream_t st) {
#define X(I, NT, SW, SH) \
    if (v == I) return launch_variant<NT, SW, SH>(a, grid, record, st);
    HAMR_FUSED_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

bool fused_variant(int v, FusedVariant &out) {
#define X(I, NT, SW, SH)      \
    if (v == I) {             \
        out.threads = NT;     \
        out.pitch = SW;       \
        out.rows = SH;        \
        out.staged = SW * SH; \
        return true;          \
    }
    HAMR_FUSED_VARIANTS(X)
#undef X
    return false;
}

int fused_max_blocks_per_sm(int v) {
#define X(I, NT, SW, SH) \
    if (v == I) return blocks_per_sm<NT, SW, SH>();
    HAMR_FUSED_VARIANTS(X)
#undef X
    return 0;
}

}  // namespace hamr
