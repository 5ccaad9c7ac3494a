// Fused FP32 sLLG Heun step for the stencil lattices: both Heun stages of a step in one pass
// over the spin state, for many replicas of uneven size in one persistent launch.  The
// simple-cubic lattice has 6 nearest neighbours (one exchange shell); the L1_0 Fe sublattice
// (square nets of spacing a/sqrt2 stacked at c) has 4 in-plane nearest neighbours, 2 out of
// plane and 4 in-plane diagonals (three shells).  Both are stencils over the same staged
// planes: the diagonals are the corners of the halo that the nearest neighbours need anyway.
//
// Work item = a block of bx x by columns of one replica over a range of planes [z0, z0 + nzl)
// (all nz planes unless a lattice has too few column blocks to fill the GPU).  The CTA stages,
// plane by plane, the spins of the block plus a two-column halo in shared memory and marches
// up the planes, from the plane below its range to the plane above it: the predictor on those
// two planes recomputes the S' that the neighbouring ranges compute (the same noise, as the
// counter is the site), so the corrector never needs another CTA's S'.  Planes are numbered
// from z0 within the item (local k = z - z0).  Staging runs three planes ahead of the march through a four-slot
// ring with one mbarrier per slot: one thread (the waiter) issues a TMA tile copy of the
// three spin components (zero-filled beyond open edges), arriving once for the whole CTA;
// replicas whose blocks wrap around a periodic edge, or whose grains touch, are staged instead
// by per-position cp.async copies of every thread that arrive on the same mbarriers.  Only the
// warps that hold list entries march (all of them for per-position copies); the waiter is lane
// 0 of the last of them, whose columns are mostly halo columns with no corrector work.  At
// march step k the marching warps
//   1. start staging plane k+3 into the slot that plane k-1 has left;
//   2. predict S' on plane k for every listed column: the block's interior and its
//      one-column halo (corners included), so the corrector never needs another CTA's S';
//   3. let the waiter wait until plane k+2 has landed (the barrier that follows makes it
//      visible to every thread for the next step);
//   4. synchronise once (a named barrier over the marching warps);
//   5. correct plane k-1 on the interior columns from the S' planes k-2, k-1 (shared
//      memory) and k (the thread's own, in registers).
// With four S and four S' slots no other barrier is needed: the next step's writes go to
// slots that no thread can still be reading.  The four slot mbarriers are initialised once
// per kernel and keep running phases across work items.
// The list of columns is built on the host per work item: only columns inside the lattice
// that hold a magnetic site are listed, so lanes are not spent on the non-magnetic grain
// boundaries or on halos beyond an open edge; interior columns come first, flagged in the
// list entry.  Each thread owns one list entry (or E of them) for the whole march and keeps
// in registers what the next stage needs from its own column: S of planes k-1 and k, the
// corrector base S + dt f(S, B(S)) / 2 and the field terms that do not depend on S (applied
// plus thermal) of the plane awaiting correction.  The march is unrolled over the ring
// period so that ring slots and neighbour offsets are compile-time constants.
// Each site's thermal normals come from its own (replica key, site, step) Philox counter, so
// halo sites computed by two CTAs get the same noise.  Open edges and non-magnetic sites read
// as S = 0 (the state of such sites is kept at 0): a zero spin marks a non-magnetic site and
// adds nothing to the exchange sum, so grain codes are read only for replicas whose grains
// touch (the exchange mask).  The per-grain sums of record steps are taken afterwards by a
// separate coalesced pass over the new state (k_grain_sums_fx).
// Per step the kernel reads S once (12 B/site) and writes S once (12 B/site); halo columns
// are re-read from L2.
#pragma once

#include "device_common.cuh"

namespace hamr {

constexpr int NSLOT = 4;                  // ring depth (planes)


template <int NT, int SW, int SH>
struct FusedShape {
    static constexpr int CAPS = SW * SH;               // staged positions per plane
    static constexpr int LPT = (CAPS + NT - 1) / NT;  // per-position copies per thread (fallback)
    // one S slot: the TMA box [3 components][SH rows][SW columns], rounded to 128 B
    static constexpr int SLOT_F = ((3 * CAPS * 4 + 127) / 128) * 128 / 4;
    static constexpr size_t smem = 128 + sizeof(float) * NSLOT * SLOT_F + sizeof(float4) * NSLOT * CAPS +
                                   sizeof(uint16_t) * NSLOT * CAPS + sizeof(int) * CAPS;
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

// one arrival that stands for `count` threads, with the byte count the TMA copy will deliver
__device__ __forceinline__ void mbar_expect_tx_n(unsigned long long *b, unsigned bytes, unsigned count) {
    asm volatile(
        "mbarrier.expect_tx.shared::cta.b64 [%0], %1;\n"
        "mbarrier.arrive.shared::cta.b64 _, [%0], %2;\n" ::"r"(smem_u32(b)),
        "r"(bytes), "r"(count)
        : "memory");
}

// barrier `id` over the first `nthr` threads of the CTA (a multiple of 32); true on every
// participant when any of them passed v = true
__device__ __forceinline__ bool bar_or(int id, int nthr, bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v), "r"(id), "r"(nthr)
        : "memory");
    return r != 0;
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

// bounded wait: false when the phase did not complete within `polls` polls
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity, unsigned polls) {
    for (unsigned i = 0; i < polls; ++i)
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

// f(S, B) / (dt pref) = S x B + alpha [(S.B) S - (S.S) B]  (Eq. 1 in Landau-Lifshitz form).
// The fused kernels are compiled without implicit multiply-add contraction, and every fused
// multiply-add here is written out, so that all instantiations (every launch shape) round
// identically and a run resumed with different step blocks is bitwise the same.
__device__ __forceinline__ float3 rhs_u(float sx, float sy, float sz, float ss, float bx, float by, float bz,
                                        float al) {
    const float cx = fmaf(sy, bz, -(sz * by)), cy = fmaf(sz, bx, -(sx * bz)), cz = fmaf(sx, by, -(sy * bx));
    const float sb = fmaf(sx, bx, fmaf(sy, by, sz * bz));
    return make_float3(fmaf(al, fmaf(sb, sx, -(ss * bx)), cx), fmaf(al, fmaf(sb, sy, -(ss * by)), cy),
                       fmaf(al, fmaf(sb, sz, -(ss * bz)), cz));
}

// 1 / |v| (v = 0 is not passed)
__device__ __forceinline__ float inv_norm(float x, float y, float z) { return rsqrtf(fmaf(x, x, fmaf(y, y, z * z))); }

// Field at a staged S position: h + sum_s (J_s / mu_s) sum_{j in shell s} S_j, with P0 the
// position in the staged plane (component planes CAPS floats apart) and m / p the own
// column's spins of the planes below and above.  With the mask a neighbour counts only when
// its grain code equals g (codes G0 in the same layout, gm / gp of the planes below and
// above).
template <bool TET, int CAPS, int SW>
__device__ __forceinline__ float3 field_s(const FusedArgs &a, float3 h, const float *P0, float mx, float my, float mz,
                                          float px, float py, float pz, bool mask, const uint16_t *G0, unsigned g,
                                          unsigned gm, unsigned gp) {
    constexpr int D0 = -SW - 1, D1 = -SW + 1, D2 = SW - 1, D3 = SW + 1;  // in-plane diagonals
    float w[10] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
    if (mask) {
        w[0] = G0[-1] == g;
        w[1] = G0[1] == g;
        w[2] = G0[-SW] == g;
        w[3] = G0[SW] == g;
        w[4] = gm == g;
        w[5] = gp == g;
        if (TET) {
            w[6] = G0[D0] == g;
            w[7] = G0[D1] == g;
            w[8] = G0[D2] == g;
            w[9] = G0[D3] == g;
        }
    }
    auto comp = [&](const float *Pd, float zb, float za, float hd) {
        if (!mask) {
            const float nn = (Pd[-1] + Pd[1]) + (Pd[-SW] + Pd[SW]);
            if (TET)
                return fmaf(a.cJ[0], nn, fmaf(a.cJ[1], zb + za, fmaf(a.cJ[2], (Pd[D0] + Pd[D1]) + (Pd[D2] + Pd[D3]), hd)));
            return fmaf(a.cJ[0], nn + (zb + za), hd);
        }
        const float nn = fmaf(w[0], Pd[-1], w[1] * Pd[1]) + fmaf(w[2], Pd[-SW], w[3] * Pd[SW]);
        const float zz = fmaf(w[4], zb, w[5] * za);
        if (TET)
            return fmaf(a.cJ[0], nn,
                        fmaf(a.cJ[1], zz,
                             fmaf(a.cJ[2], fmaf(w[6], Pd[D0], w[7] * Pd[D1]) + fmaf(w[8], Pd[D2], w[9] * Pd[D3]), hd)));
        return fmaf(a.cJ[0], nn + zz, hd);
    };
    return make_float3(comp(P0, mx, px, h.x), comp(P0 + CAPS, my, py, h.y), comp(P0 + 2 * CAPS, mz, pz, h.z));
}

// The same for the staged S' plane (float4 per position, .w = grain code) at Q, with the own
// column's S' of the planes below (zm) and above (zp).
template <bool TET, int SW>
__device__ __forceinline__ float3 field_p(const FusedArgs &a, float3 h, const float4 *Q, const float4 &zm,
                                          const float4 &zp, bool mask, unsigned g) {
    if constexpr (!TET) {  // six nearest neighbours, one shell
        const float4 l = Q[-1], r = Q[1], d = Q[-SW], u = Q[SW];
        float w[6] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
        if (mask) {
            w[0] = __float_as_uint(l.w) == g;
            w[1] = __float_as_uint(r.w) == g;
            w[2] = __float_as_uint(d.w) == g;
            w[3] = __float_as_uint(u.w) == g;
            w[4] = __float_as_uint(zm.w) == g;
            w[5] = __float_as_uint(zp.w) == g;
        }
        auto comp = [&](float vl, float vr, float vd, float vu, float vm, float vp, float hd) {
            if (!mask) return fmaf(a.cJ[0], ((vl + vr) + (vd + vu)) + (vm + vp), hd);
            return fmaf(a.cJ[0], (fmaf(w[0], vl, w[1] * vr) + fmaf(w[2], vd, w[3] * vu)) + fmaf(w[4], vm, w[5] * vp),
                        hd);
        };
        return make_float3(comp(l.x, r.x, d.x, u.x, zm.x, zp.x, h.x), comp(l.y, r.y, d.y, u.y, zm.y, zp.y, h.y),
                           comp(l.z, r.z, d.z, u.z, zm.z, zp.z, h.z));
    }
    constexpr int D0 = -SW - 1, D1 = -SW + 1, D2 = SW - 1, D3 = SW + 1;
    auto wt = [&](const float4 &v) { return mask ? (float)(__float_as_uint(v.w) == g) : 1.f; };
    // nearest in-plane neighbours, then the planes below and above
    float3 nn, zz;
    {
        const float4 l = Q[-1], r = Q[1], d = Q[-SW], u = Q[SW];
        if (!mask) {
            nn = make_float3((l.x + r.x) + (d.x + u.x), (l.y + r.y) + (d.y + u.y), (l.z + r.z) + (d.z + u.z));
            zz = make_float3(zm.x + zp.x, zm.y + zp.y, zm.z + zp.z);
        } else {
            const float w0 = wt(l), w1 = wt(r), w2 = wt(d), w3 = wt(u), w4 = wt(zm), w5 = wt(zp);
            nn = make_float3(fmaf(w0, l.x, w1 * r.x) + fmaf(w2, d.x, w3 * u.x), fmaf(w0, l.y, w1 * r.y) + fmaf(w2, d.y, w3 * u.y),
                             fmaf(w0, l.z, w1 * r.z) + fmaf(w2, d.z, w3 * u.z));
            zz = make_float3(fmaf(w4, zm.x, w5 * zp.x), fmaf(w4, zm.y, w5 * zp.y), fmaf(w4, zm.z, w5 * zp.z));
        }
    }
    // in-plane diagonals (third shell)
    const float4 q0 = Q[D0], q1 = Q[D1], q2 = Q[D2], q3 = Q[D3];
    const float v0 = wt(q0), v1 = wt(q1), v2 = wt(q2), v3 = wt(q3);
    const float3 dg = make_float3(fmaf(v0, q0.x, v1 * q1.x) + fmaf(v2, q2.x, v3 * q3.x),
                                  fmaf(v0, q0.y, v1 * q1.y) + fmaf(v2, q2.y, v3 * q3.y),
                                  fmaf(v0, q0.z, v1 * q1.z) + fmaf(v2, q2.z, v3 * q3.z));
    return make_float3(fmaf(a.cJ[0], nn.x, fmaf(a.cJ[1], zz.x, fmaf(a.cJ[2], dg.x, h.x))),
                       fmaf(a.cJ[0], nn.y, fmaf(a.cJ[1], zz.y, fmaf(a.cJ[2], dg.y, h.y))),
                       fmaf(a.cJ[0], nn.z, fmaf(a.cJ[1], zz.z, fmaf(a.cJ[2], dg.z, h.z))));
}

// ZR: the work items cover plane ranges (false: every item spans all planes of its replica,
// and the range arithmetic compiles away)
template <bool TET, int NT, int E, int SW, int SH, int MINB, bool ZR>
__global__ void __launch_bounds__(NT, MINB) k_fused(FusedArgs a) {
    using Sh = FusedShape<NT, SW, SH>;
    constexpr int CAPS = Sh::CAPS, LPT = Sh::LPT, SLOT_F = Sh::SLOT_F;
    extern __shared__ unsigned char smem_raw[];
    float *sS = reinterpret_cast<float *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);  // [4][SLOT_F]
    float4 *sP = reinterpret_cast<float4 *>(sS + NSLOT * SLOT_F);                          // [4][CAPS]
    uint16_t *sG = reinterpret_cast<uint16_t *>(sP + NSLOT * CAPS);                        // [4][CAPS]
    int *sL = reinterpret_cast<int *>(sG + NSLOT * CAPS);  // [CAPS] per-position copy offsets
    __shared__ int s_item;
    __shared__ uint4 s_rk[5];  // Philox round keys of the current replica
    __shared__ __align__(8) unsigned long long s_bar[NSLOT];
    // staging state that only thread 0 uses (kept out of every thread's registers): the tensor
    // map and origin of the current item's TMA box, the phase parity of the next phase of each
    // slot barrier, and the highest plane staged and the highest awaited
    __shared__ const CUtensorMap *s_map;
    __shared__ int s_xs, s_ys, s_ph, s_hi_issued, s_hi_waited;
    __shared__ float4 s_ba;  // applied field B_app(t) of the current item
    const int tid = threadIdx.x;
    const long long NS = a.NS;
    const long long step = a.ctl->step + a.step_off;
    const int par = (int)(step & 1);
    const float *__restrict__ Sin = par ? a.Sbuf1 : a.Sbuf0;
    float *__restrict__ Sout = par ? a.Sbuf0 : a.Sbuf1;
    if (blockIdx.x == 0 && tid == 0) a.ctl->work_ctr[par ^ 1] = 0u;  // next step's counter
    const float t = (float)step * a.dt;
    const float q = a.pref * a.dt, qh = 0.5f * q;
    bool stop = false;  // a bounded wait ran out (decided uniformly by barrier vote)
    // The slot barriers live for the whole kernel and expect NT arrivals per fill: the TMA
    // issuer arrives once for all NT threads with the expected byte count, per-position copies
    // arrive through cp.async from every thread.  The parity of the next phase of every slot
    // is kept in s_ph (only the waiter of an item reads or changes it).
    if (tid == 0) s_ph = 0;
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
        const int z0 = ZR ? W.zr & 0xffff : 0, nzl = ZR ? W.zr >> 16 : nz;  // the item's planes [z0, z0 + nzl)
        const int off = (int)R.off;
        const int plane = px * ny;
        const int bx = W.bxy & 0xffff, by = W.bxy >> 16;
        const int n_act = W.counts & 0xffff;
        const bool mask = R.cross_grain != 0;
        const bool tma = (W.stage & 1) != 0;
        const int xs = W.x0 - 2 - (W.stage >> 8), ys = W.y0 - 2;  // staged-region origin
        if (tid == 0) {
            s_map = a.maps + 2 * W.r + par;
            s_xs = xs;
            s_ys = ys;
            s_hi_issued = s_hi_waited = -3;
            const float bapp = R.fB0 * field_polarity_f(R, a.bits, t);
            s_ba = make_float4(bapp * R.fdir[0], bapp * R.fdir[1], bapp * R.fdir[2], 0.f);
        }
        if (tid < 5) {
            const unsigned k0 = R.key0 + 2u * tid * 0x9E3779B9u, k1 = R.key1 + 2u * tid * 0xBB67AE85u;
            s_rk[tid] = make_uint4(k0, k1, k0 + 0x9E3779B9u, k1 + 0xBB67AE85u);
        }
        // S' (and its grain code) of unlisted positions must read as 0 for the whole item
        for (int i = tid; i < NSLOT * CAPS; i += NT) sP[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        // per-position copies: each position's column offset within a plane (-1: zero-filled,
        // -2: outside the block's staged region)
        if (!tma)
            for (int idx = tid; idx < CAPS; idx += NT) {
                const int sx = idx % SW, sy = idx / SW;
                int lofs = -2;
                if (sx < bx + 4 && sy < by + 4) {
                    bool in = true;
                    const int cx = wrap_coord(xs + sx, nx, a.per[0], in);
                    const int cy = wrap_coord(ys + sy, ny, a.per[1], in);
                    lofs = in ? cx + px * cy : -1;
                }
                sL[idx] = lofs;
            }
        __syncthreads();

        // this thread's list entries tid, tid + NT, ... (site and storage indices fit in 32
        // bits: a replica has at most 2^30 sites and the storage fewer than 2^28 slots)
        bool act[E], inner[E];  // listed; interior column (corrected by this thread)
        int c[E];               // staged-region position
        float sig[E];           // thermal-field scale of the column
        unsigned scol[E];       // site index of the column on plane 0
        int ocol[E];            // storage slot of the column on the item's first plane z0
#pragma unroll
        for (int j = 0; j < E; ++j) {
            act[j] = tid + j * NT < n_act;
            inner[j] = false;
            c[j] = 0;
            sig[j] = 0.f;
            scol[j] = 0;
            ocol[j] = 0;
            if (act[j]) {
                const unsigned e = a.lists[W.list_off + tid + j * NT];
                c[j] = (int)(e & 0x7fffu);
                inner[j] = (e & 0x8000u) != 0;
                bool ok = true;
                const int wx = wrap_coord(xs + c[j] % SW, nx, a.per[0], ok);
                const int wy = wrap_coord(ys + c[j] / SW, ny, a.per[1], ok);
                const float T = temperature_f(R, (wx + 0.5f) * a.ax, (wy + 0.5f) * a.ay, t);
                sig[j] = a.sig0 * sqrtf(T);
                scol[j] = (unsigned)wx + (unsigned)nx * (unsigned)wy;
                ocol[j] = off + wx + px * (wy + ny * z0);  // the column's slot on plane z0
            }
        }
        // Only the warps that hold list entries march; the others wait at the end of the item.
        // Per-position copies need every thread, so those items march with the whole CTA.  Lane
        // 0 of the last marching warp, whose columns are mostly halo columns without a corrector
        // stage, issues the TMA fills and waits for them (the waiter).
        const int nmarch = tma ? min(NT, (n_act + 31) & ~31) : NT;
        const int waiter = nmarch - 32;
        // stage local plane p into ring slot p mod 4 (planes beyond nzl + 1 are never needed)
        auto issue = [&](int p, bool withhold = false) {
            if (p > nzl + 1) return;
            const int slot = (p + 4) & 3;
            float *dst = sS + slot * SLOT_F;
            bool ok = true;
            const int z = wrap_coord(z0 + p, nz, a.per[2], ok);
            // failure-detection test: the phase of this fill can then never complete
            if (withhold && tid == waiter) return;
            if (tid == waiter) s_hi_issued = p;
            if (tma) {
                if (tid == waiter) {
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    // one arrival for the whole CTA, plus the bytes the copy delivers
                    mbar_expect_tx_n(&s_bar[slot], 3u * CAPS * 4u, (unsigned)NT);
                    // an out-of-range plane of an open lattice: every element is zero-filled
                    tma_load_4d(dst, s_map, s_xs, s_ys, ok ? z : -2, 0, &s_bar[slot]);
                }
            } else {
                const int base = off + z * plane;
                uint16_t *gd = sG + slot * CAPS;
#pragma unroll
                for (int l = 0; l < LPT; ++l) {
                    const int idx = tid + l * NT;
                    if (idx >= CAPS) continue;
                    const int lofs = sL[idx];
                    if (lofs == -2) continue;
                    const bool v = ok && lofs >= 0;
                    const float *src = Sin + (v ? base + lofs : 0);
                    cp_async4(dst + idx, src, v);
                    cp_async4(dst + CAPS + idx, src + NS, v);
                    cp_async4(dst + 2 * CAPS + idx, src + 2 * NS, v);
                    if (mask) gd[idx] = v ? __ldg(a.gcode + base + lofs) : (uint16_t)0;
                }
                mbar_arrive_cp_async(&s_bar[slot]);
            }
        };
        // The waiter alone waits until plane p has landed in its slot (the other threads see the
        // plane after the next barrier); a wait that runs out is recorded here and acted on at
        // that barrier's vote.
        bool bad = false;
        auto await = [&](int p) {
            const int slot = (p + 4) & 3;
            const int ph = s_ph;
            if (!mbar_wait(&s_bar[slot], (ph >> slot) & 1u, a.wait_polls)) {
                bad = true;
                atomicOr(&a.ctl->err, 2);
            }
            s_ph = ph ^ (1 << slot);
            s_hi_waited = p;
        };
        const unsigned site_plane = (unsigned)nx * (unsigned)ny;

        // prologue: planes -2 .. 1 staged; own S (and grain code) of planes -2 and -1 read
        issue(-2);
        issue(-1);
        issue(0);
        issue(1, a.inject && it == 0);
        if (tid == waiter) {
            await(-2);
            await(-1);
            await(0);
        }
        // planes -2 .. 0 become visible to every thread
        stop = __syncthreads_or(bad) != 0;
        float m1x[E], m1y[E], m1z[E];  // S on plane k-1 at each column
        float c0x[E], c0y[E], c0z[E];  // S on plane k
        unsigned gm1[E];               // grain code of plane k-1 (masked replicas)
        float amx[E], amy[E], amz[E];  // S + dt f(S, B(S)) / 2 of plane k-1
        float hmx[E], hmy[E], hmz[E];  // B_app + B_th of plane k-1
#pragma unroll
        for (int j = 0; j < E; ++j) {
            m1x[j] = m1y[j] = m1z[j] = c0x[j] = c0y[j] = c0z[j] = 0.f;
            amx[j] = amy[j] = amz[j] = hmx[j] = hmy[j] = hmz[j] = 0.f;
            gm1[j] = 0;
            if (act[j]) {
                const float *S2 = sS + 2 * SLOT_F + c[j], *S3 = sS + 3 * SLOT_F + c[j];  // planes -2, -1
                m1x[j] = S2[0];
                m1y[j] = S2[CAPS];
                m1z[j] = S2[2 * CAPS];
                gm1[j] = sG[2 * CAPS + c[j]];
                c0x[j] = S3[0];
                c0y[j] = S3[CAPS];
                c0z[j] = S3[2 * CAPS];
            }
        }
        // plane -2's slot is restaged by the first march step
        __syncthreads();
        if (tid < nmarch) {

        // one march step; PH fixes the ring slots: plane k sits in slot (PH + 3) % 4
        auto march = [&](auto PHC, int k) {
            constexpr int PH = decltype(PHC)::value;
            constexpr int SK = (PH + 3) & 3, SK1 = PH & 3, SKM1 = (PH + 2) & 3, SKM2 = (PH + 1) & 3;
            issue(k + 3);  // into slot (k + 3) mod 4 = SKM1, left by plane k-1 (kept in registers)
            bool zok = true;
            const int wz = wrap_coord(z0 + k, nz, a.per[2], zok);
            float4 sp[E];       // S' of plane k (own, for the corrector's z+ neighbour)
            float ppx[E], ppy[E], ppz[E];
            unsigned g0[E];
            float anx[E], any[E], anz[E], hx[E], hy[E], hz[E];
            // ---- predictor on plane k (each column's own S is in c0, carried from the last step)
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const float *P0 = sS + SK * SLOT_F + c[j], *Pp = sS + SK1 * SLOT_F + c[j];
                const float sx = c0x[j], sy = c0y[j], sz = c0z[j];
                ppx[j] = Pp[0];
                ppy[j] = Pp[CAPS];
                ppz[j] = Pp[2 * CAPS];
                g0[j] = 0;
                anx[j] = any[j] = anz[j] = hx[j] = hy[j] = hz[j] = 0.f;
                sp[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (act[j]) {
                    if (mask) g0[j] = sG[SK * CAPS + c[j]];
                    const bool mag = mask ? g0[j] != 0 : nonzero3(sx, sy, sz);
                    if (zok && mag) {
                        float n0, n1, n2;
                        normals3(philox10_rk(philox_ctr(scol[j] + site_plane * (unsigned)wz, (unsigned long long)step),
                                             s_rk),
                                 n0, n1, n2);
                        const float4 ba = s_ba;
                        hx[j] = fmaf(sig[j], n0, ba.x);
                        hy[j] = fmaf(sig[j], n1, ba.y);
                        hz[j] = fmaf(sig[j], n2, ba.z);
                        float3 B;
                        if constexpr (TET) {
                            B = field_s<TET, CAPS, SW>(a, make_float3(hx[j], hy[j], fmaf(a.cK, sz, hz[j])), P0, m1x[j],
                                                       m1y[j], m1z[j], ppx[j], ppy[j], ppz[j], mask, sG + SK * CAPS + c[j],
                                                       g0[j], gm1[j], mask ? sG[SK1 * CAPS + c[j]] : 0u);
                        } else {
                            float ex, ey, ez;
                            if (!mask) {
                                ex = ((P0[-1] + P0[1]) + (P0[-SW] + P0[SW])) + (m1x[j] + ppx[j]);
                                ey = ((P0[CAPS - 1] + P0[CAPS + 1]) + (P0[CAPS - SW] + P0[CAPS + SW])) + (m1y[j] + ppy[j]);
                                ez = ((P0[2 * CAPS - 1] + P0[2 * CAPS + 1]) + (P0[2 * CAPS - SW] + P0[2 * CAPS + SW])) +
                                     (m1z[j] + ppz[j]);
                            } else {
                                const uint16_t *G0 = sG + SK * CAPS + c[j];
                                const unsigned g = g0[j];
                                const float w0 = G0[-1] == g, w1 = G0[1] == g, w2 = G0[-SW] == g, w3 = G0[SW] == g,
                                            w4 = gm1[j] == g, w5 = sG[SK1 * CAPS + c[j]] == g;
                                ex = fmaf(w0, P0[-1], w1 * P0[1]) + fmaf(w2, P0[-SW], w3 * P0[SW]) +
                                     fmaf(w4, m1x[j], w5 * ppx[j]);
                                ey = fmaf(w0, P0[CAPS - 1], w1 * P0[CAPS + 1]) + fmaf(w2, P0[CAPS - SW], w3 * P0[CAPS + SW]) +
                                     fmaf(w4, m1y[j], w5 * ppy[j]);
                                ez = fmaf(w0, P0[2 * CAPS - 1], w1 * P0[2 * CAPS + 1]) +
                                     fmaf(w2, P0[2 * CAPS - SW], w3 * P0[2 * CAPS + SW]) + fmaf(w4, m1z[j], w5 * ppz[j]);
                            }
                            B = make_float3(fmaf(a.cJ[0], ex, hx[j]), fmaf(a.cJ[0], ey, hy[j]),
                                            fmaf(a.cJ[0], ez, fmaf(a.cK, sz, hz[j])));
                        }
                        const float ss = fmaf(sx, sx, fmaf(sy, sy, sz * sz));  // |S|^2
                        const float3 u = rhs_u(sx, sy, sz, ss, B.x, B.y, B.z, a.alpha);
                        // S + dt f / 2 (the corrector's base) and S + dt f, dt f = q u
                        anx[j] = fmaf(qh, u.x, sx);
                        any[j] = fmaf(qh, u.y, sy);
                        anz[j] = fmaf(qh, u.z, sz);
                        const float npx = fmaf(q, u.x, sx), npy = fmaf(q, u.y, sy), npz = fmaf(q, u.z, sz);
                        const float inv = inv_norm(npx, npy, npz);
                        sp[j] = make_float4(npx * inv, npy * inv, npz * inv, __uint_as_float(g0[j]));
                    }
                    sP[SK * CAPS + c[j]] = sp[j];
                }
            }
            // plane k+2 (read by the next step's predictor) is awaited by thread 0 before the
            // step's one barrier, which also carries the failure vote
            if (tid == waiter && k + 2 <= nzl + 1) await(k + 2);
            stop = bar_or(1, nmarch, bad);
            // ---- corrector on plane k-1 from S' planes k-2 (slot SKM2), k-1 (SKM1) and k (own, sp)
            const int kc = k - 1;
            if (kc >= 0 && kc < nzl) {
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    if (!inner[j]) continue;
                    const float4 *Q = sP + SKM1 * CAPS + c[j];
                    const float4 v = Q[0];
                    if (!nonzero3(v.x, v.y, v.z)) continue;
                    // S' is a unit vector: S'.S' = 1 in the damping term
                    float3 B;
                    if constexpr (TET) {
                        B = field_p<TET, SW>(a, make_float3(hmx[j], hmy[j], fmaf(a.cK, v.z, hmz[j])), Q,
                                             sP[SKM2 * CAPS + c[j]], sp[j], mask, __float_as_uint(v.w));
                    } else {
                        const float4 l = Q[-1], r = Q[1], d = Q[-SW], u4 = Q[SW];
                        const float4 zm = sP[SKM2 * CAPS + c[j]], zp = sp[j];
                        float ex, ey, ez;
                        if (!mask) {
                            ex = ((l.x + r.x) + (d.x + u4.x)) + (zm.x + zp.x);
                            ey = ((l.y + r.y) + (d.y + u4.y)) + (zm.y + zp.y);
                            ez = ((l.z + r.z) + (d.z + u4.z)) + (zm.z + zp.z);
                        } else {
                            const unsigned g = __float_as_uint(v.w);
                            const float w0 = __float_as_uint(l.w) == g, w1 = __float_as_uint(r.w) == g,
                                        w2 = __float_as_uint(d.w) == g, w3 = __float_as_uint(u4.w) == g,
                                        w4 = __float_as_uint(zm.w) == g, w5 = __float_as_uint(zp.w) == g;
                            ex = fmaf(w0, l.x, w1 * r.x) + fmaf(w2, d.x, w3 * u4.x) + fmaf(w4, zm.x, w5 * zp.x);
                            ey = fmaf(w0, l.y, w1 * r.y) + fmaf(w2, d.y, w3 * u4.y) + fmaf(w4, zm.y, w5 * zp.y);
                            ez = fmaf(w0, l.z, w1 * r.z) + fmaf(w2, d.z, w3 * u4.z) + fmaf(w4, zm.z, w5 * zp.z);
                        }
                        B = make_float3(fmaf(a.cJ[0], ex, hmx[j]), fmaf(a.cJ[0], ey, hmy[j]),
                                        fmaf(a.cJ[0], ez, fmaf(a.cK, v.z, hmz[j])));
                    }
                    const float3 u = rhs_u(v.x, v.y, v.z, 1.f, B.x, B.y, B.z, a.alpha);
                    float ox = fmaf(qh, u.x, amx[j]), oy = fmaf(qh, u.y, amy[j]), oz = fmaf(qh, u.z, amz[j]);
                    const float inv = inv_norm(ox, oy, oz);
                    ox *= inv;
                    oy *= inv;
                    oz *= inv;
                    const int o = ocol[j] + kc * plane;
                    Sout[o] = ox;
                    Sout[NS + o] = oy;
                    Sout[2 * NS + o] = oz;
                }
            }
            // carry each column's plane-k values to the next march step
#pragma unroll
            for (int j = 0; j < E; ++j) {
                m1x[j] = c0x[j];
                m1y[j] = c0y[j];
                m1z[j] = c0z[j];
                c0x[j] = ppx[j];
                c0y[j] = ppy[j];
                c0z[j] = ppz[j];
                gm1[j] = g0[j];
                amx[j] = anx[j];
                amy[j] = any[j];
                amz[j] = anz[j];
                hmx[j] = hx[j];
                hmy[j] = hy[j];
                hmz[j] = hz[j];
            }
        };

        // k runs from -1 to nzl; k = kb + PH with kb = -1 (mod 4), so plane k sits in slot (PH + 3) % 4
        for (int kb = -1; kb <= nzl && !stop; kb += 4) {
            march(IC<0>(), kb);
            if (!stop && kb + 1 <= nzl) march(IC<1>(), kb + 1);
            if (!stop && kb + 2 <= nzl) march(IC<2>(), kb + 2);
            if (!stop && kb + 3 <= nzl) march(IC<3>(), kb + 3);
        }
        if (stop) {
            // give the fills issued after the last awaited plane a bounded time to land before
            // the CTA's shared memory is released
            if (tid == waiter)
                for (int p = s_hi_waited + 1; p <= s_hi_issued; ++p) {
                    const int slot = (p + 4) & 3;
                    mbar_wait(&s_bar[slot], (s_ph >> slot) & 1, 1u << 22);
                    s_ph ^= 1 << slot;
                }
        }
        }  // marching warps
        // all reads of this item's slots are done before they are re-armed; a failed wait ends
        // the kernel for every thread
        if (__syncthreads_or(stop)) return;
    }
}

// Opt in to the variant's dynamic shared memory (done before any stream capture, when the
// work list is built).
template <bool TET, int NT, int E, int SW, int SH, int MINB, bool ZR>
static cudaError_t ensure_attrs() {
    using Sh = FusedShape<NT, SW, SH>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<TET, NT, E, SW, SH, MINB, ZR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        init = true;
    }
    return cudaSuccess;
}

template <bool TET, int NT, int E, int SW, int SH, int MINB>
static cudaError_t launch_variant(const FusedArgs &a, bool zr, int grid, cudaStream_t st) {
    using Sh = FusedShape<NT, SW, SH>;
    cudaError_t e = zr ? ensure_attrs<TET, NT, E, SW, SH, MINB, true>() : ensure_attrs<TET, NT, E, SW, SH, MINB, false>();
    if (e != cudaSuccess) return e;
    if (zr)
        k_fused<TET, NT, E, SW, SH, MINB, true><<<grid, NT, Sh::smem, st>>>(a);
    else
        k_fused<TET, NT, E, SW, SH, MINB, false><<<grid, NT, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

template <bool TET, int NT, int E, int SW, int SH, int MINB>
static int blocks_per_sm() {
    using Sh = FusedShape<NT, SW, SH>;
    int n = 0, m = 0;
    if (ensure_attrs<TET, NT, E, SW, SH, MINB, false>() != cudaSuccess ||
        ensure_attrs<TET, NT, E, SW, SH, MINB, true>() != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<TET, NT, E, SW, SH, MINB, false>, NT, Sh::smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_fused<TET, NT, E, SW, SH, MINB, true>, NT, Sh::smem) !=
            cudaSuccess)
        return 0;
    return n < m ? n : m;
}

// compiled variants: threads per CTA, listed columns per thread, the staged region's pitch x
// rows (pitch a multiple of 4 so that TMA rows are 16-byte multiples) and the CTAs per SM the
// register budget is sized for.  A block of bx x by columns fits when bx + 4 <= pitch (bx + 7
// with TMA, whose origin is rounded down to a multiple of 4), by + 4 <= rows and it lists at
// most threads x columns-per-thread columns.
#define HAMR_FUSED_VARIANTS(X) \
    X(0, 512, 1, 36, 24, 2) X(1, 1024, 1, 68, 24, 1) X(2, 256, 1, 36, 14, 3) X(3, 256, 2, 36, 24, 2)

template <bool TET>
cudaError_t launch_fused_lattice(int v, bool zr, const FusedArgs &a, int grid, cudaStream_t st) {
#define X(I, NT, E, SW, SH, MINB) \
    if (v == I) return launch_variant<TET, NT, E, SW, SH, MINB>(a, zr, grid, st);
    HAMR_FUSED_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

template <bool TET>
int fused_blocks_lattice(int v) {
#define X(I, NT, E, SW, SH, MINB) \
    if (v == I) return blocks_per_sm<TET, NT, E, SW, SH, MINB>();
    HAMR_FUSED_VARIANTS(X)
#undef X
    return 0;
}

}  // namespace hamr
