// Host side of the C ABI declared in hamr.h: argument checks, device memory layout,
// neighbour-list building, step scheduling through captured CUDA graphs, record
// collection, checkpoints and the tile autotuner.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <memory>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hamr_internal.h"

using namespace hamr;

namespace {

// NVTX range over a host call (setup, step blocks, record collection), visible in a timeline
// profiler; free when no profiler is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

thread_local std::string g_create_err = "no error";

int fail(hamr_t h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_err = buf;
    return code;
}

#define CK(h, call)                                                                               \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(h, e_ == cudaErrorMemoryAllocation ? HAMR_ERR_OOM : HAMR_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

// Makes the handle's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t dalloc(hamr_t h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e == cudaSuccess) h->dev_bytes += count * sizeof(T);
    return e;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

size_t elt(const hamr_t h) { return h->prec == HAMR_FP64 ? 8 : 4; }

// FP32 handles on the implicit stencil (simple cubic or L1_0) run the fused kernel
bool fused_mode(const hamr_t h) { return h->prec == HAMR_FP32 && h->nbr == HAMR_NBR_STENCIL; }

bool tetragonal(const hamr_t h) { return h->lattice == HAMR_LATTICE_L10; }

void clear_graphs(hamr_t h) {
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

bool bad_replica(hamr_t h, int r) { return !h || r < 0 || r >= h->R; }

// ---------------------------------------------------------------- neighbour offsets
struct Off {
    int dx, dy, dz, shell;
};

// Bond offsets in lattice units.  SC: the 6 nearest neighbours (Sec. II).  L1_0 Fe
// sublattice (tetragonal a/sqrt2, a/sqrt2, c): 4 in-plane nearest at a/sqrt2 (shell 0), 2
// out-of-plane at c (shell 1), 4 in-plane diagonals at a (shell 2) (Sec. II, Appendix A).
std::vector<Off> bond_offsets(int lattice) {
    std::vector<Off> o = {{-1, 0, 0, 0}, {1, 0, 0, 0}, {0, -1, 0, 0}, {0, 1, 0, 0}};
    if (lattice == HAMR_LATTICE_SC) {
        o.push_back({0, 0, -1, 0});
        o.push_back({0, 0, 1, 0});
    } else {
        o.push_back({0, 0, -1, 1});
        o.push_back({0, 0, 1, 1});
        o.push_back({-1, -1, 0, 2});
        o.push_back({1, -1, 0, 2});
        o.push_back({-1, 1, 0, 2});
        o.push_back({1, 1, 0, 2});
    }
    return o;
}

bool wrap(int &v, int n, int per) {
    if (v >= 0 && v < n) return true;
    if (!per) return false;
    v = ((v % n) + n) % n;
    return true;
}

long long slot_of(const ReplicaDev &R, long long x, long long y, long long z) {
    return R.off + x + (long long)R.px * (y + (long long)R.ny * z);
}

// Fill this replica's rows of the packed list from the geometry or the user list; bonds only
// between sites with the same non-zero grain code.
int build_ell_replica(hamr_t h, int r, int width) {
    const ReplicaDev &R = h->reps_h[r];
    const long long NS = h->NS;
    const bool user = r < (int)h->ucsr_rp.size() && !h->ucsr_rp[r].empty();
    const std::vector<Off> offs = bond_offsets(h->lattice);
    for (long long z = 0; z < R.nz; ++z)
        for (long long y = 0; y < R.ny; ++y)
            for (long long x = 0; x < R.px; ++x) {
                const long long s = slot_of(R, x, y, z);
                int k = 0;
                const uint16_t g = h->gcode_h[s];
                if (x < R.nx && g != 0) {
                    if (user) {
                        const long long i = x + (long long)R.nx * (y + (long long)R.ny * z);
                        const std::vector<int> &rp = h->ucsr_rp[r], &col = h->ucsr_col[r];
                        const std::vector<uint8_t> &sh = h->ucsr_sh[r];
                        for (int e = rp[i]; e < rp[i + 1]; ++e) {
                            const long long j = col[e];
                            const long long jx = j % R.nx, jy = (j / R.nx) % R.ny, jz = j / ((long long)R.nx * R.ny);
                            const long long sj = slot_of(R, jx, jy, jz);
                            if (h->gcode_h[sj] != g) continue;
                            if (k >= width) return -1;
                            h->ell_h[(size_t)k * NS + s] = (int)(sj | ((long long)sh[e] << ELL_SHELL_SHIFT));
                            ++k;
                        }
                    } else {
                        for (const Off &o : offs) {
                            int jx = (int)x + o.dx, jy = (int)y + o.dy, jz = (int)z + o.dz;
                            if (!wrap(jx, R.nx, h->per[0]) || !wrap(jy, R.ny, h->per[1]) || !wrap(jz, R.nz, h->per[2]))
                                continue;
                            const long long sj = slot_of(R, jx, jy, jz);
                            if (h->gcode_h[sj] != g) continue;
                            h->ell_h[(size_t)k * NS + s] = (int)(sj | ((long long)o.shell << ELL_SHELL_SHIFT));
                            ++k;
                        }
                    }
                }
                for (; k < width; ++k) h->ell_h[(size_t)k * NS + s] = -1;
            }
    return 0;
}

int upload_ell_replica(hamr_t h, int r) {
    const ReplicaDev &R = h->reps_h[r];
    const long long span = (long long)R.px * R.ny * R.nz;
    for (int k = 0; k < h->ell_w; ++k)
        CK(h, cudaMemcpyAsync(h->ell_d + (size_t)k * h->NS + R.off, h->ell_h.data() + (size_t)k * h->NS + R.off,
                              sizeof(int) * span, cudaMemcpyHostToDevice, h->stream));
    return HAMR_OK;
}

// ---------------------------------------------------------------- derived replica data
void set_driver_floats(ReplicaDev &R) {
    R.fT_amb = (float)R.T_amb;
    R.fdT = (float)R.dT;
    R.fc_fwhm = (float)R.c_fwhm;
    R.fx0 = (float)R.x0;
    R.fy0 = (float)R.y0;
    R.fvx = (float)R.vx;
    R.fvy = (float)R.vy;
    R.fB0 = (float)R.B0;
    for (int d = 0; d < 3; ++d) R.fdir[d] = (float)R.dir[d];
    R.fbit_len = (float)R.bit_len;
    R.framp_len = (float)R.ramp_len;
    R.fhead_x0 = (float)R.head_x0;
    R.fhead_v = (float)R.head_v;
}

int upload_replica(hamr_t h, int r) {
    CK(h, cudaMemcpyAsync(h->reps_d + r, &h->reps_h[r], sizeof(ReplicaDev), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

// Site counts of replica r per grain and in total.
void count_grains(hamr_t h, int r) {
    const ReplicaDev &R = h->reps_h[r];
    std::vector<long long> &cnt = h->gcount_rep[r];
    cnt.assign(h->n_grains[r], 0);
    long long nmag = 0;
    for (long long z = 0; z < R.nz; ++z)
        for (long long y = 0; y < R.ny; ++y)
            for (long long x = 0; x < R.nx; ++x) {
                const uint16_t g = h->gcode_h[slot_of(R, x, y, z)];
                if (g) {
                    cnt[g - 1] += 1;
                    ++nmag;
                }
            }
    h->nmag_h[r] = nmag;
}

// grain bins: offsets and counts of all replicas; reallocates when the total grows
int refresh_grains(hamr_t h) {
    int G = 0;
    for (int r = 0; r < h->R; ++r) {
        h->reps_h[r].grain_off = G;
        h->reps_h[r].n_grains = h->n_grains[r];
        G += h->n_grains[r];
    }
    h->G = G;
    h->runs_dirty = true;
    h->gcount_h.assign(std::max(G, 1), 0);
    for (int r = 0; r < h->R; ++r)
        std::copy(h->gcount_rep[r].begin(), h->gcount_rep[r].end(), h->gcount_h.begin() + h->reps_h[r].grain_off);
    if (G > h->G_cap) {
        dfree(h->grain_acc_d);
        dfree(h->grain_fx_d);
        dfree(h->grain_last_d);
        dfree(h->gcount_d);
        const int cap = std::max(G, 2 * h->G_cap);
        CK(h, dalloc(h, &h->grain_acc_d, 3 * (size_t)cap));
        CK(h, dalloc(h, &h->grain_fx_d, 3 * (size_t)cap));
        CK(h, dalloc(h, &h->grain_last_d, 3 * (size_t)cap));
        CK(h, dalloc(h, &h->gcount_d, (size_t)cap));
        h->G_cap = cap;
        clear_graphs(h);
    }
    CK(h, cudaMemsetAsync(h->grain_acc_d, 0, sizeof(double) * 3 * h->G_cap, h->stream));
    CK(h, cudaMemsetAsync(h->grain_fx_d, 0, sizeof(unsigned long long) * 3 * h->G_cap, h->stream));
    CK(h, cudaMemsetAsync(h->grain_last_d, 0, sizeof(double) * 3 * h->G_cap, h->stream));
    CK(h, cudaMemcpyAsync(h->gcount_d, h->gcount_h.data(), sizeof(long long) * G, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->nmag_d, h->nmag_h.data(), sizeof(long long) * h->R, cudaMemcpyHostToDevice, h->stream));
    h->grain_last_h.assign(3 * (size_t)std::max(G, 1), 0.0);
    CK(h, cudaMemcpyAsync(h->reps_d, h->reps_h.data(), sizeof(ReplicaDev) * h->R, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

// Runs of consecutive magnetic slots of one grain (within one row, at most GRAIN_RUN_MAX
// long), grouped by global grain bin, and the items of up to GRAIN_RUN_MAX runs of one grain
// that the per-grain sums of the FP32 fused path take one warp each.
int build_runs(hamr_t h) {
    Range nv("hamr build_runs");
    std::vector<unsigned long long> run;
    std::vector<int> run_grain;
    std::vector<long long> per_grain(std::max(h->G, 1) + 1, 0);
    for (int r = 0; r < h->R; ++r) {
        const ReplicaDev &R = h->reps_h[r];
        for (long long z = 0; z < R.nz; ++z)
            for (long long y = 0; y < R.ny; ++y) {
                const long long row = slot_of(R, 0, y, z);
                long long x = 0;
                while (x < R.nx) {
                    const uint16_t g = h->gcode_h[row + x];
                    long long e = x + 1;
                    while (e < R.nx && e - x < GRAIN_RUN_MAX && h->gcode_h[row + e] == g) ++e;
                    if (g) {
                        run.push_back((unsigned long long)(row + x) << 5 | (unsigned long long)(e - x - 1));
                        run_grain.push_back(R.grain_off + g - 1);
                        per_grain[R.grain_off + g] += 1;
                    }
                    x = e;
                }
            }
    }
    for (size_t g = 1; g < per_grain.size(); ++g) per_grain[g] += per_grain[g - 1];
    std::vector<unsigned long long> sorted(run.size());
    std::vector<long long> fill(per_grain.begin(), per_grain.end() - 1);
    for (size_t i = 0; i < run.size(); ++i) sorted[fill[run_grain[i]]++] = run[i];
    std::vector<GrainRunItem> items;
    for (int g = 0; g < h->G; ++g)
        for (long long k = per_grain[g]; k < per_grain[g + 1]; k += GRAIN_RUN_MAX)
            items.push_back({k, g, (int)std::min<long long>(GRAIN_RUN_MAX, per_grain[g + 1] - k)});
    if ((long long)sorted.size() > h->runs_cap) {
        dfree(h->runs_d);
        const long long cap = std::max<long long>((long long)sorted.size(), 2 * h->runs_cap);
        CK(h, dalloc(h, &h->runs_d, (size_t)cap));
        h->runs_cap = cap;
    }
    if ((int)items.size() > h->gitems_cap) {
        dfree(h->gitems_d);
        const int cap = std::max((int)items.size(), 2 * h->gitems_cap);
        CK(h, dalloc(h, &h->gitems_d, (size_t)cap));
        h->gitems_cap = cap;
    }
    if (!sorted.empty())
        CK(h, cudaMemcpyAsync(h->runs_d, sorted.data(), sizeof(unsigned long long) * sorted.size(),
                              cudaMemcpyHostToDevice, h->stream));
    if (!items.empty())
        CK(h, cudaMemcpyAsync(h->gitems_d, items.data(), sizeof(GrainRunItem) * items.size(), cudaMemcpyHostToDevice,
                              h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->n_gitems = (int)items.size();
    h->runs_dirty = false;
    clear_graphs(h);
    return HAMR_OK;
}

// ---------------------------------------------------------------- fused work list
// Listed columns of the block [x0, x0+bx) x [y0, y0+by) with its one-column halo: columns
// inside the lattice (or wrapping on a periodic axis) that hold a magnetic site; pre is the
// 2-D prefix sum of that column mask (halo columns that wrap are counted through the mask).
struct ColumnMask {
    int nx, ny, per_x, per_y;
    std::vector<uint8_t> m;
    std::vector<int> pre;  // (ny + 1) x (nx + 1)
    int at(int x, int y) const {
        if (!wrap(x, nx, per_x) || !wrap(y, ny, per_y)) return 0;
        return m[x + (size_t)nx * y];
    }
    int rect(int x0, int x1, int y0, int y1) const {  // [x0, x1) x [y0, y1) inside the lattice
        return pre[x1 + (nx + 1) * (size_t)y1] - pre[x0 + (nx + 1) * (size_t)y1] - pre[x1 + (nx + 1) * (size_t)y0] +
               pre[x0 + (nx + 1) * (size_t)y0];
    }
    int listed(int x0, int y0, int bx, int by) const {
        const int xa = std::max(x0 - 1, 0), xb = std::min(x0 + bx + 1, nx);
        const int ya = std::max(y0 - 1, 0), yb = std::min(y0 + by + 1, ny);
        int n = rect(xa, xb, ya, yb);
        // halo columns beyond a periodic edge wrap to columns counted again
        if (per_x || per_y) {
            n = 0;
            for (int y = y0 - 1; y <= y0 + by; ++y)
                for (int x = x0 - 1; x <= x0 + bx; ++x) n += at(x, y);
        }
        return n;
    }
};

ColumnMask column_mask(hamr_t h, int r) {
    const ReplicaDev &R = h->reps_h[r];
    ColumnMask c;
    c.nx = R.nx;
    c.ny = R.ny;
    c.per_x = h->per[0];
    c.per_y = h->per[1];
    c.m.assign((size_t)R.nx * R.ny, 0);
    for (long long z = 0; z < R.nz; ++z)
        for (long long y = 0; y < R.ny; ++y)
            for (long long x = 0; x < R.nx; ++x)
                if (h->gcode_h[slot_of(R, x, y, z)]) c.m[x + (size_t)R.nx * y] = 1;
    c.pre.assign((size_t)(R.nx + 1) * (R.ny + 1), 0);
    for (int y = 0; y < R.ny; ++y)
        for (int x = 0; x < R.nx; ++x)
            c.pre[(x + 1) + (R.nx + 1) * (size_t)(y + 1)] = c.m[x + (size_t)R.nx * y] + c.pre[x + (R.nx + 1) * (size_t)(y + 1)] +
                                                             c.pre[(x + 1) + (R.nx + 1) * (size_t)y] -
                                                             c.pre[x + (R.nx + 1) * (size_t)y];
    return c;
}

// Split of one replica into ntx x nty balanced column blocks for a kernel variant.  A split
// fits when every block's staged region (block + two-column halo) fits the variant's pitch
// and rows and every block lists at most one column per thread.  Among fitting splits the
// one with the least modelled time wins: per block and plane, a fixed cost for the CTA's
// threads, the predictor on the listed columns, the corrector on the interior and the
// staging of the region.
void choose_split(const ReplicaDev &R, const ColumnMask &cm, const FusedVariant &v, int margin, int &bx_out,
                  int &by_out) {
    double best = 1e300;
    bx_out = by_out = 1;
    for (int ntx = 1; ntx <= R.nx; ++ntx) {
        const int bx = (R.nx + ntx - 1) / ntx;
        if (ntx > 1 && bx == (R.nx + ntx - 2) / (ntx - 1)) continue;  // same width as ntx - 1
        if (bx + margin > v.pitch) continue;
        for (int nty = 1; nty <= R.ny; ++nty) {
            const int by = (R.ny + nty - 1) / nty;
            if (nty > 1 && by == (R.ny + nty - 2) / (nty - 1)) continue;
            if (by + 4 > v.rows) continue;
            double cost = 0.0;
            bool fits = true;
            for (int y0 = 0; y0 < R.ny && fits; y0 += by)
                for (int x0 = 0; x0 < R.nx; x0 += bx) {
                    const int wx = std::min(bx, R.nx - x0), wy = std::min(by, R.ny - y0);
                    const int listed = cm.listed(x0, y0, wx, wy);
                    if (listed > v.columns) {
                        fits = false;
                        break;
                    }
                    const int inner = cm.rect(x0, x0 + wx, y0, y0 + wy);
                    cost += 0.25 * v.threads + 2.0 * listed + inner + 0.3 * (wx + 4) * (wy + 4);
                }
            if (fits && cost < best) {
                best = cost;
                bx_out = bx;
                by_out = by;
            }
        }
    }
}

// cuTensorMapEncodeTiled from the driver, found at run time (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// Tensor maps of replica r's spin state in each buffer: a 4-D view (x over the storage pitch,
// y, z, component) whose box is one staged plane of all three components.
int build_maps(hamr_t h, int r, const FusedVariant &v, CUtensorMap out[2]) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(h, HAMR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const ReplicaDev &R = h->reps_h[r];
    const cuuint64_t dim[4] = {(cuuint64_t)R.px, (cuuint64_t)R.ny, (cuuint64_t)R.nz, 3};
    const cuuint64_t stride[3] = {(cuuint64_t)R.px * 4, (cuuint64_t)R.px * R.ny * 4, (cuuint64_t)h->NS * 4};
    const cuuint32_t box[4] = {(cuuint32_t)v.pitch, (cuuint32_t)v.rows, 1, 3};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; ++b) {
        void *base = (float *)h->S[b] + R.off;
        const CUresult e = enc(&out[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dim, stride, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (e != CUDA_SUCCESS)
            return fail(h, HAMR_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for replica %d", (int)e, r);
    }
    return HAMR_OK;
}

// Work items and their column lists for the current variant.  A column is listed when it
// lies inside the lattice (or wraps on a periodic axis) and holds a magnetic site on some
// plane; interior columns come first.
int build_items(hamr_t h) {
    Range nv("hamr build_items");
    FusedVariant v;
    if (!fused_variant(h->variant, v)) return fail(h, HAMR_ERR_ARG, "unknown kernel variant %d", h->variant);
    std::vector<WorkItem> items;
    std::vector<long long> cost;
    std::vector<std::vector<uint16_t>> lists;
    std::vector<CUtensorMap> maps(2 * (size_t)h->R);
    memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    h->tma_ok.assign(h->R, 0);
    for (int r = 0; r < h->R; ++r) {
        const ReplicaDev &R = h->reps_h[r];
        // TMA tiles cannot wrap: replicas with periodic x or y, or touching grains, are staged by
        // per-position copies
        const int tma = !h->per[0] && !h->per[1] && !R.cross_grain;
        h->tma_ok[r] = tma;
        if (tma) {
            int rc = build_maps(h, r, v, &maps[2 * (size_t)r]);
            if (rc) return rc;
        }
        // columns holding a magnetic site on some plane
        const ColumnMask cm = column_mask(h, r);
        const std::vector<uint8_t> &col = cm.m;
        int BX, BY;
        choose_split(R, cm, v, tma ? 7 : 4, BX, BY);
        for (int y0 = 0; y0 < R.ny; y0 += BY)
            for (int x0 = 0; x0 < R.nx; x0 += BX) {
                const int bx = std::min(BX, R.nx - x0), by = std::min(BY, R.ny - y0);
                const int WS = v.pitch;
                // staged origin: x0 - 2, rounded down to a multiple of 4 columns for TMA
                const int dx0 = tma ? (((x0 - 2) % 4) + 4) % 4 : 0;
                std::vector<uint16_t> inner, halo;
                for (int sy = 1; sy <= by + 2; ++sy)
                    for (int sx = 1; sx <= bx + 2; ++sx) {
                        int cx = x0 - 2 + sx, cy = y0 - 2 + sy;
                        if (!wrap(cx, R.nx, h->per[0]) || !wrap(cy, R.ny, h->per[1])) continue;
                        if (!col[cx + (size_t)R.nx * cy]) continue;
                        const bool in = sx >= 2 && sx <= bx + 1 && sy >= 2 && sy <= by + 1;
                        (in ? inner : halo).push_back((uint16_t)(sx + dx0 + WS * sy));
                    }
                if (inner.empty()) continue;  // nothing to update in this block
                WorkItem w;
                w.r = r;
                w.x0 = x0;
                w.y0 = y0;
                w.bxy = bx | (by << 16);
                w.list_off = 0;
                w.counts = (int)(inner.size() + halo.size()) | ((int)inner.size() << 16);
                w.stage = tma | (dx0 << 8);
                // interior columns first, flagged by bit 15 (corrected by the thread that lists them)
                std::vector<uint16_t> mixed;
                mixed.reserve(inner.size() + halo.size());
                for (uint16_t p : inner) mixed.push_back((uint16_t)(p | 0x8000u));
                mixed.insert(mixed.end(), halo.begin(), halo.end());
                w.zr = 0;
                items.push_back(w);
                lists.push_back(std::move(mixed));
                cost.push_back((long long)(2 * (w.counts & 0xffff) + (w.counts >> 16) + 64) * (R.nz + 2));
            }
    }
    // Plane ranges.  A batch whose column blocks are too few to keep the resident CTAs busy is
    // also split along z.  Modelled time of a launch: the larger of the total work over the
    // resident CTAs and the longest item, an item of L planes of a block costing that block's
    // work per plane times L + 4 (its march runs L + 2 steps, the prologue about 2 more).  The
    // range length with the least modelled time wins; a shorter one must gain 5 %.
    const int bps = std::max(1, fused_max_blocks_per_sm(h->variant, tetragonal(h)));
    const double slots = (double)bps * std::max(1, h->num_sms);
    int maxnz = 1;
    for (const ReplicaDev &R : h->reps_h) maxnz = std::max(maxnz, R.nz);
    int Lz = maxnz;
    double best = 1e300;
    for (int L = maxnz; L >= std::min(4, maxnz); --L) {
        double total = 0.0, longest = 0.0;
        for (size_t i = 0; i < items.size(); ++i) {
            const int nz = h->reps_h[items[i].r].nz, nr = (nz + L - 1) / L;
            const double wp = (double)cost[i] / (nz + 2);
            total += wp * (nz + 4.0 * nr);
            longest = std::max(longest, wp * ((nz + nr - 1) / nr + 4));
        }
        const double c = std::max(total / slots, longest);
        if (c < 0.95 * best) {
            best = c;
            Lz = L;
        }
    }
    if (h->z_range_set > 0) Lz = h->z_range_set;
    // replicas by decreasing total cost, the blocks of a replica together and in row order:
    // neighbouring blocks then run at the same time and share their halo planes through L2
    std::vector<long long> rcost(h->R, 0);
    for (size_t i = 0; i < items.size(); ++i) rcost[items[i].r] += cost[i];
    std::vector<size_t> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
        const int ra = items[a].r, rb = items[b].r;
        if (ra != rb) return rcost[ra] != rcost[rb] ? rcost[ra] > rcost[rb] : ra < rb;
        return a < b;
    });
    // each block once per plane range, its ranges in a row (they share the block's column list)
    std::vector<WorkItem> sorted;
    std::vector<uint16_t> flat;
    for (size_t i = 0; i < idx.size(); ++i) {
        WorkItem w = items[idx[i]];
        w.list_off = (int)flat.size();
        flat.insert(flat.end(), lists[idx[i]].begin(), lists[idx[i]].end());
        const int nz = h->reps_h[w.r].nz, nr = (nz + Lz - 1) / Lz;
        for (int j = 0; j < nr; ++j) {
            const int za = (int)((long long)j * nz / nr), zb = (int)((long long)(j + 1) * nz / nr);
            w.zr = za | ((zb - za) << 16);
            sorted.push_back(w);
        }
    }
    if (sorted.size() > (size_t)h->items_cap) {
        dfree(h->items_d);
        CK(h, dalloc(h, &h->items_d, sorted.size()));
        h->items_cap = (int)sorted.size();
    }
    if (flat.size() > h->lists_cap) {
        dfree(h->lists_d);
        CK(h, dalloc(h, &h->lists_d, flat.size()));
        h->lists_cap = flat.size();
    }
    if (!sorted.empty())
        CK(h, cudaMemcpyAsync(h->items_d, sorted.data(), sizeof(WorkItem) * sorted.size(), cudaMemcpyHostToDevice,
                              h->stream));
    if (!flat.empty())
        CK(h, cudaMemcpyAsync(h->lists_d, flat.data(), sizeof(uint16_t) * flat.size(), cudaMemcpyHostToDevice,
                              h->stream));
    if (!h->maps_d) CK(h, dalloc(h, &h->maps_d, 2 * (size_t)h->R));
    CK(h, cudaMemcpyAsync(h->maps_d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->n_items = (int)sorted.size();
    h->z_range = Lz;
    h->z_split = Lz < maxnz;
    h->fused_grid = std::max(1, std::min(h->n_items, bps * h->num_sms));
    h->items_dirty = false;
    clear_graphs(h);
    return HAMR_OK;
}

// ---------------------------------------------------------------- one block of steps
// Enqueue G steps (the last one recording when asked) and the bookkeeping kernel.
int enqueue_block(hamr_t h, int G, bool record) {
    if (fused_mode(h)) {
        FusedArgs a{};
        a.NS = h->NS;
        a.gcode = h->gcode_d;
        a.reps = h->reps_d;
        a.bits = h->bits_d;
        a.items = h->items_d;
        a.lists = h->lists_d;
        a.n_items = h->n_items;
        a.ctl = h->ctl_d;
        for (int s = 0; s < 3; ++s) a.cJ[s] = (float)h->ph.cJ[s];
        a.cK = (float)h->ph.cK;
        a.pref = (float)h->ph.pref;
        a.alpha = (float)h->ph.alpha;
        a.dt = (float)h->ph.dt;
        a.sig0 = (float)h->ph.sig0;
        a.ax = (float)h->ph.ax;
        a.ay = (float)h->ph.ay;
        a.az = (float)h->ph.az;
        for (int d = 0; d < 3; ++d) a.per[d] = h->per[d];
        a.maps = h->maps_d;
        a.wait_polls = h->inject_polls ? h->inject_polls : (1u << 22);
        a.inject = h->inject_polls ? 1 : 0;
        a.Sbuf0 = (float *)h->S[0];
        a.Sbuf1 = (float *)h->S[1];
        for (int i = 0; i < G; ++i) {
            a.step_off = i;
            CK(h, launch_fused_step(h->variant, tetragonal(h), h->z_split, a, h->fused_grid, h->stream));
        }
        if (record)
            CK(h, launch_grain_sums_fx(a.Sbuf0, a.Sbuf1, h->NS, h->runs_d, h->gitems_d, h->n_gitems, h->ctl_d, G,
                                       h->grain_fx_d, h->stream));
    } else {
        const int nb = (int)(h->NS / PLAIN_BLOCK);
        if (h->prec == HAMR_FP64) {
            PlainArgs<double> a{};
            a.S = (double *)h->S[0];
            a.SP = (double *)h->SP;
            a.F1 = (double *)h->F1;
            a.BTH = (double *)h->BTH;
            a.NS = h->NS;
            a.gcode = h->gcode_d;
            a.blk_rep = h->blk_rep_d;
            a.reps = h->reps_d;
            a.bits = h->bits_d;
            a.ell = h->nbr == HAMR_NBR_CSR ? h->ell_d : nullptr;
            a.ell_w = h->ell_w;
            a.ctl = h->ctl_d;
            a.ph = h->ph;
            a.grain_acc = h->grain_acc_d;
            for (int i = 0; i < G; ++i) {
                a.step_off = i;
                CK(h, launch_plain_step(HAMR_FP64, &a, nb, record && i == G - 1, h->stream));
            }
        } else {
            PlainArgs<float> a{};
            a.S = (float *)h->S[0];
            a.SP = (float *)h->SP;
            a.F1 = (float *)h->F1;
            a.BTH = (float *)h->BTH;
            a.NS = h->NS;
            a.gcode = h->gcode_d;
            a.blk_rep = h->blk_rep_d;
            a.reps = h->reps_d;
            a.bits = h->bits_d;
            a.ell = h->nbr == HAMR_NBR_CSR ? h->ell_d : nullptr;
            a.ell_w = h->ell_w;
            a.ctl = h->ctl_d;
            a.ph = h->ph;
            a.grain_acc = h->grain_acc_d;
            for (int i = 0; i < G; ++i) {
                a.step_off = i;
                CK(h, launch_plain_step(HAMR_FP32, &a, nb, record && i == G - 1, h->stream));
            }
        }
    }
    CK(h, launch_bookkeeping(h->ctl_d, G, record, h->R, h->reps_d, h->nmag_d, h->gcount_d, h->G, h->grain_acc_d,
                             h->grain_fx_d, h->grain_last_d, h->rec_d, h->rec_cap, h->rec_step_d, h->stream));
    return HAMR_OK;
}

int run_block(hamr_t h, int G, bool record) {
    if (h->inject_polls) {  // the failure test runs once, outside the graph cache
        int rc = enqueue_block(h, G, record);
        h->inject_polls = 0;
        if (rc) return rc;
        h->step_h += G;
        if (fused_mode(h)) h->cur = (int)(h->step_h & 1);
        return HAMR_OK;
    }
    const auto key = std::make_tuple(G, record ? 1 : 0, 0, h->variant);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        cudaGraph_t graph;
        CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_block(h, G, record);
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (rc != HAMR_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return rc;
        }
        CK(h, e);
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(h, e);
        it = h->graphs.emplace(key, exec).first;
    }
    CK(h, cudaGraphLaunch(it->second, h->stream));
    h->step_h += G;
    if (fused_mode(h)) h->cur = (int)(h->step_h & 1);
    return HAMR_OK;
}

int collect_records(hamr_t h) {
    Range nv("hamr collect_records");
    CK(h, cudaStreamSynchronize(h->stream));
    Ctl c;
    CK(h, cudaMemcpy(&c, h->ctl_d, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (c.err & 2) {
        const int zero = 0;
        CK(h, cudaMemcpy(&h->ctl_d->err, &zero, sizeof zero, cudaMemcpyHostToDevice));
        return fail(h, HAMR_ERR_TIMEOUT, "a bounded wait in the fused kernel ran out; the state is not valid");
    }
    if (c.n_rec > 0) {
        const long long n = std::min(c.n_rec, h->rec_cap);
        const size_t old = h->rec_h.size();
        h->rec_h.resize(old + (size_t)n * h->R * 3);
        CK(h, cudaMemcpy(h->rec_h.data() + old, h->rec_d, sizeof(double) * n * h->R * 3, cudaMemcpyDeviceToHost));
        const size_t olds = h->rec_step_h.size();
        h->rec_step_h.resize(olds + n);
        CK(h, cudaMemcpy(h->rec_step_h.data() + olds, h->rec_step_d, sizeof(long long) * n, cudaMemcpyDeviceToHost));
        if (h->G > 0)
            CK(h, cudaMemcpy(h->grain_last_h.data(), h->grain_last_d, sizeof(double) * 3 * h->G,
                             cudaMemcpyDeviceToHost));
        const long long zero = 0;
        CK(h, cudaMemcpy(&h->ctl_d->n_rec, &zero, sizeof zero, cudaMemcpyHostToDevice));
        if (c.n_rec > h->rec_cap) return fail(h, HAMR_ERR_STATE, "record buffer overflow");
    }
    h->pending_records = false;
    return HAMR_OK;
}

int steps_impl(hamr_t h, int64_t n_steps, int32_t record_every, bool sync) {
    if (!h) return HAMR_ERR_ARG;
    Range nv("hamr sllg_heun_steps");
    if (n_steps < 0 || record_every < 0) return fail(h, HAMR_ERR_ARG, "n_steps and record_every must be >= 0");
    if (!h->shells_set) return fail(h, HAMR_ERR_STATE, "exchange shells not set (hamr_set_neighbour_shells)");
    if (h->max_user_shell >= h->ph.n_shells)
        return fail(h, HAMR_ERR_STATE, "neighbour list uses shell %d but only %d shell(s) are set", h->max_user_shell,
                    h->ph.n_shells);
    DeviceGuard dg(h->device);
    if (fused_mode(h) && h->items_dirty) {
        int rc = build_items(h);
        if (rc) return rc;
    }
    // records this call will make
    long long nrec = 0;
    if (record_every > 0) nrec = (h->step_h + n_steps) / record_every - h->step_h / record_every;
    if (h->pending_records && nrec > 0) {
        int rc = collect_records(h);
        if (rc) return rc;
    }
    if (fused_mode(h) && nrec > 0 && h->runs_dirty) {
        int rc = build_runs(h);
        if (rc) return rc;
    }
    if (nrec > h->rec_cap) {
        dfree(h->rec_d);
        dfree(h->rec_step_d);
        const long long cap = std::max(nrec, 2 * h->rec_cap);
        CK(h, dalloc(h, &h->rec_d, (size_t)cap * h->R * 3));
        CK(h, dalloc(h, &h->rec_step_d, (size_t)cap));
        h->rec_cap = cap;
        clear_graphs(h);
    }
    long long left = n_steps;
    while (left > 0) {
        int G;
        bool rec = false;
        if (record_every > 0) {
            const long long to_rec = record_every - (h->step_h % record_every);
            if (to_rec <= left) {
                G = (int)to_rec;
                rec = true;
            } else {
                G = (int)left;
            }
        } else {
            G = (int)std::min<long long>(left, 64);
        }
        int rc = run_block(h, G, rec);
        if (rc) return rc;
        left -= G;
    }
    if (nrec > 0) h->pending_records = true;
    if (sync) return collect_records(h);
    return HAMR_OK;
}

void destroy_device(hamr_t h) {
    clear_graphs(h);
    dfree(h->reps_d);
    dfree(h->S[0]);
    dfree(h->S[1]);
    dfree(h->SP);
    dfree(h->F1);
    dfree(h->BTH);
    dfree(h->gcode_d);
    dfree(h->blk_rep_d);
    dfree(h->ell_d);
    dfree(h->bits_d);
    dfree(h->ctl_d);
    dfree(h->grain_acc_d);
    dfree(h->grain_fx_d);
    dfree(h->grain_last_d);
    dfree(h->gcount_d);
    dfree(h->nmag_d);
    dfree(h->lists_d);
    dfree(h->maps_d);
    dfree(h->rec_d);
    dfree(h->rec_step_d);
    dfree(h->dscratch_d);
    dfree(h->stage_d);
    dfree(h->items_d);
    dfree(h->runs_d);
    dfree(h->gitems_d);
}

int init_device(hamr_t h, long long NS, long long maxn, const std::vector<int> &blk_rep) {
    // device memory
    const size_t es = elt(h);
    CK(h, dalloc(h, &h->reps_d, h->R));
    CK(h, dalloc(h, (char **)&h->S[0], 3 * NS * es));
    if (fused_mode(h)) {
        CK(h, dalloc(h, (char **)&h->S[1], 3 * NS * es));
    } else {
        CK(h, dalloc(h, (char **)&h->SP, 3 * NS * es));
        CK(h, dalloc(h, (char **)&h->F1, 3 * NS * es));
        CK(h, dalloc(h, (char **)&h->BTH, 3 * NS * es));
        CK(h, cudaMemsetAsync(h->SP, 0, 3 * NS * es, h->stream));
        CK(h, cudaMemsetAsync(h->F1, 0, 3 * NS * es, h->stream));
        CK(h, cudaMemsetAsync(h->BTH, 0, 3 * NS * es, h->stream));
    }
    CK(h, dalloc(h, &h->gcode_d, NS));
    CK(h, dalloc(h, &h->blk_rep_d, blk_rep.size()));
    CK(h, dalloc(h, &h->ctl_d, 1));
    CK(h, dalloc(h, &h->nmag_d, h->R));
    CK(h, dalloc(h, &h->dscratch_d, 8));
    CK(h, dalloc(h, &h->stage_d, 3 * (size_t)maxn));
    h->stage_n = maxn;
    h->bits_cap = 64;
    CK(h, dalloc(h, &h->bits_d, h->bits_cap));
    CK(h, cudaMemsetAsync(h->bits_d, 0, h->bits_cap, h->stream));
    CK(h, cudaMemsetAsync(h->ctl_d, 0, sizeof(Ctl), h->stream));
    CK(h, cudaMemcpyAsync(h->gcode_d, h->gcode_h.data(), sizeof(uint16_t) * NS, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->blk_rep_d, blk_rep.data(), sizeof(int) * blk_rep.size(), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, launch_init_state(h->prec, h->S[0], NS, h->gcode_d, h->stream));
    if (h->S[1]) CK(h, cudaMemsetAsync(h->S[1], 0, 3 * NS * es, h->stream));
    if (h->nbr == HAMR_NBR_CSR) {
        h->ell_w = h->lattice == HAMR_LATTICE_SC ? 6 : 10;
        h->ell_h.assign((size_t)h->ell_w * NS, -1);
        CK(h, dalloc(h, &h->ell_d, (size_t)h->ell_w * NS));
        for (int r = 0; r < h->R; ++r) build_ell_replica(h, r, h->ell_w);
        CK(h, cudaMemcpyAsync(h->ell_d, h->ell_h.data(), sizeof(int) * h->ell_w * NS, cudaMemcpyHostToDevice,
                              h->stream));
    }
    return refresh_grains(h);
}

}  // namespace

// =====================================================================================
namespace hamr {
// error message of a call that has no handle (read back with hamr_last_error(NULL))
void set_handleless_error(const char *msg) { g_create_err = msg; }
}  // namespace hamr

extern "C" {

int hamr_lattice_create(hamr_t *out, const hamr_lattice_desc *d) {
    if (!out || !d) return fail(nullptr, HAMR_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->lattice != HAMR_LATTICE_SC && d->lattice != HAMR_LATTICE_L10)
        return fail(nullptr, HAMR_ERR_ARG, "unknown lattice %d", d->lattice);
    if (d->precision != HAMR_FP32 && d->precision != HAMR_FP64)
        return fail(nullptr, HAMR_ERR_ARG, "unknown precision %d", d->precision);
    if (d->neighbours != HAMR_NBR_STENCIL && d->neighbours != HAMR_NBR_CSR)
        return fail(nullptr, HAMR_ERR_ARG, "unknown neighbour mode %d", d->neighbours);
    if (d->n_replicas < 1 || !d->dims || !d->seeds) return fail(nullptr, HAMR_ERR_ARG, "bad replica description");
    if (!(d->a > 0) || (d->lattice == HAMR_LATTICE_L10 && !(d->c > 0)) || !(d->mu_s > 0) || !(d->dt > 0) ||
        !(d->gamma > 0) || !(d->alpha >= 0) || !isfinite(d->ku))
        return fail(nullptr, HAMR_ERR_ARG, "bad physical parameter (a, c, mu_s, dt, gamma > 0, alpha >= 0)");
    long long NS = 0, maxn = 0;
    for (int r = 0; r < d->n_replicas; ++r) {
        const long long nx = d->dims[3 * r], ny = d->dims[3 * r + 1], nz = d->dims[3 * r + 2];
        if (nx < 1 || ny < 1 || nz < 1 || nx > 65535 || ny > 65535 || nx * ny * nz > (1LL << 30))
            return fail(nullptr, HAMR_ERR_ARG, "replica %d: bad dims %lld x %lld x %lld", r, nx, ny, nz);
        const long long px = (nx + 3) / 4 * 4;
        NS += (px * ny * nz + SLOT_ALIGN - 1) / SLOT_ALIGN * SLOT_ALIGN;
        maxn = std::max(maxn, nx * ny * nz);
    }
    if (NS >= (1LL << ELL_SHELL_SHIFT))
        return fail(nullptr, HAMR_ERR_ARG, "total lattice too large (%lld storage slots, limit 2^28)", NS);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, HAMR_ERR_CUDA, "no CUDA device available");
    if (d->device < 0 || d->device >= ndev) return fail(nullptr, HAMR_ERR_ARG, "bad device ordinal %d", d->device);

    std::unique_ptr<hamr_ctx> hp(new hamr_ctx());
    hamr_t h = hp.get();
    h->device = d->device;
    DeviceGuard dg(h->device);
    h->lattice = d->lattice;
    h->prec = d->precision;
    h->nbr = d->neighbours;
    h->R = d->n_replicas;
    h->dims.assign(d->dims, d->dims + 3 * h->R);
    h->seeds.assign(d->seeds, d->seeds + h->R);
    h->a = d->a;
    h->c = d->c;
    h->mu_s = d->mu_s;
    h->ku = d->ku;
    h->alpha = d->alpha;
    h->dt = d->dt;
    h->gamma = d->gamma;
    for (int k = 0; k < 3; ++k) h->per[k] = d->periodic[k] ? 1 : 0;
    if (d->stream) {
        h->stream = (cudaStream_t)d->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(nullptr, HAMR_ERR_CUDA, "stream creation failed");
        h->own_stream = true;
    }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);

    // physics
    Phys &ph = h->ph;
    ph.cK = 2.0 * h->ku / h->mu_s;
    ph.pref = -h->gamma / (1.0 + h->alpha * h->alpha);
    ph.alpha = h->alpha;
    ph.dt = h->dt;
    ph.sig0 = sqrt(2.0 * h->alpha * KB / (h->gamma * h->mu_s * h->dt));
    if (h->lattice == HAMR_LATTICE_SC) {
        ph.ax = ph.ay = ph.az = h->a;
    } else {
        ph.ax = ph.ay = h->a / sqrt(2.0);
        ph.az = h->c;
    }
    for (int k = 0; k < 3; ++k) ph.per[k] = h->per[k];
    ph.lattice = h->lattice;

    // layout
    h->NS = NS;
    h->reps_h.resize(h->R);
    std::vector<int> blk_rep(NS / PLAIN_BLOCK, -1);
    long long off = 0;
    for (int r = 0; r < h->R; ++r) {
        ReplicaDev &R = h->reps_h[r];
        memset(&R, 0, sizeof R);
        R.nx = h->dims[3 * r];
        R.ny = h->dims[3 * r + 1];
        R.nz = h->dims[3 * r + 2];
        R.px = (R.nx + 3) / 4 * 4;
        R.off = off;
        R.n = (long long)R.nx * R.ny * R.nz;
        R.key0 = (unsigned)(h->seeds[r] & 0xffffffffu);
        R.key1 = (unsigned)(h->seeds[r] >> 32);
        R.dir[2] = 1.0;
        set_driver_floats(R);
        const long long span = ((long long)R.px * R.ny * R.nz + SLOT_ALIGN - 1) / SLOT_ALIGN * SLOT_ALIGN;
        for (long long b = off / PLAIN_BLOCK; b < (off + span) / PLAIN_BLOCK; ++b) blk_rep[b] = r;
        off += span;
    }
    h->gcode_h.assign(NS, 0);
    for (int r = 0; r < h->R; ++r) {
        const ReplicaDev &R = h->reps_h[r];
        for (long long z = 0; z < R.nz; ++z)
            for (long long y = 0; y < R.ny; ++y)
                for (long long x = 0; x < R.nx; ++x) h->gcode_h[slot_of(R, x, y, z)] = 1;
    }
    h->n_grains.assign(h->R, 1);
    h->bits_h.assign(h->R, {});
    h->nmag_h.assign(h->R, 0);
    h->gcount_rep.assign(h->R, {});
    for (int r = 0; r < h->R; ++r) count_grains(h, r);

    int rc = init_device(h, NS, maxn, blk_rep);
    if (rc) {
        g_create_err = h->err;
        destroy_device(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        return rc;
    }
    // default kernel variant; hamr_autotune picks the fastest compiled one
    h->variant = 0;
    *out = hp.release();
    return HAMR_OK;
}

int hamr_set_neighbour_shells(hamr_t h, int32_t n_shells, const double *J) {
    if (!h) return HAMR_ERR_ARG;
    const int want = h->lattice == HAMR_LATTICE_SC ? 1 : 3;
    if (!J || n_shells < 1 || n_shells > MAX_SHELLS)
        return fail(h, HAMR_ERR_ARG, "n_shells must be in [1, %d]", MAX_SHELLS);
    if (h->ucsr_rp.empty() && n_shells != want)
        return fail(h, HAMR_ERR_ARG, "this lattice has %d shell(s), got %d", want, n_shells);
    for (int s = 0; s < n_shells; ++s)
        if (!isfinite(J[s])) return fail(h, HAMR_ERR_ARG, "J[%d] not finite", s);
    h->J.assign(J, J + n_shells);
    for (int s = 0; s < MAX_SHELLS; ++s) h->ph.cJ[s] = s < n_shells ? J[s] / h->mu_s : 0.0;
    h->ph.n_shells = n_shells;
    h->shells_set = true;
    clear_graphs(h);
    return HAMR_OK;
}

int hamr_set_csr(hamr_t h, int32_t replica, const int32_t *row_ptr, const int32_t *col, const uint8_t *shell) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (h->nbr != HAMR_NBR_CSR) return fail(h, HAMR_ERR_STATE, "handle uses the implicit stencil");
    if (!row_ptr || !col || !shell) return fail(h, HAMR_ERR_ARG, "null array");
    const ReplicaDev &R = h->reps_h[replica];
    const long long n = R.n;
    if (row_ptr[0] != 0) return fail(h, HAMR_ERR_ARG, "row_ptr[0] must be 0");
    int maxrow = 0;
    for (long long i = 0; i < n; ++i) {
        const int len = row_ptr[i + 1] - row_ptr[i];
        if (len < 0) return fail(h, HAMR_ERR_ARG, "row_ptr not monotone at %lld", i);
        maxrow = std::max(maxrow, len);
    }
    if (maxrow > ELL_MAX) return fail(h, HAMR_ERR_ARG, "row with %d neighbours (limit %d)", maxrow, ELL_MAX);
    const int nnz = row_ptr[n];
    for (int e = 0; e < nnz; ++e) {
        if (col[e] < 0 || col[e] >= n) return fail(h, HAMR_ERR_ARG, "col[%d] = %d out of range", e, col[e]);
        if (shell[e] >= MAX_SHELLS) return fail(h, HAMR_ERR_ARG, "shell[%d] = %d out of range", e, shell[e]);
    }
    // every bond i -> j of shell s needs its partner j -> i of the same shell (J_ij = J_ji,
    // which the energy and its conservation rely on)
    for (long long i = 0; i < n; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = col[e];
            bool found = false;
            for (int f = row_ptr[j]; f < row_ptr[j + 1] && !found; ++f) found = col[f] == i && shell[f] == shell[e];
            if (!found)
                return fail(h, HAMR_ERR_ARG, "bond %lld -> %d (shell %d) has no partner %d -> %lld", i, j, shell[e], j,
                            i);
        }
    DeviceGuard dg(h->device);
    if ((int)h->ucsr_rp.size() < h->R) {
        h->ucsr_rp.resize(h->R);
        h->ucsr_col.resize(h->R);
        h->ucsr_sh.resize(h->R);
    }
    h->ucsr_rp[replica].assign(row_ptr, row_ptr + n + 1);
    h->ucsr_col[replica].assign(col, col + nnz);
    h->ucsr_sh[replica].assign(shell, shell + nnz);
    for (int e = 0; e < nnz; ++e) h->max_user_shell = std::max(h->max_user_shell, (int)shell[e]);
    if (maxrow > h->ell_w) {
        // widen the list: re-lay the host copy and reallocate
        std::vector<int> wide((size_t)maxrow * h->NS, -1);
        for (int k = 0; k < h->ell_w; ++k)
            std::copy(h->ell_h.begin() + (size_t)k * h->NS, h->ell_h.begin() + (size_t)(k + 1) * h->NS,
                      wide.begin() + (size_t)k * h->NS);
        h->ell_h.swap(wide);
        h->ell_w = maxrow;
        dfree(h->ell_d);
        CK(h, dalloc(h, &h->ell_d, (size_t)h->ell_w * h->NS));
        CK(h, cudaMemcpyAsync(h->ell_d, h->ell_h.data(), sizeof(int) * h->ell_w * h->NS, cudaMemcpyHostToDevice,
                              h->stream));
        clear_graphs(h);
    }
    if (build_ell_replica(h, replica, h->ell_w) != 0) return fail(h, HAMR_ERR_ARG, "neighbour list too wide");
    int rc = upload_ell_replica(h, replica);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_set_grain_map(hamr_t h, int32_t replica, const int32_t *grain, int32_t n_grains) {
    Range nv("hamr set_grain_map");
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!grain || n_grains < 0 || n_grains > 65534) return fail(h, HAMR_ERR_ARG, "bad grain map or n_grains");
    ReplicaDev &R = h->reps_h[replica];
    for (long long i = 0; i < R.n; ++i)
        if (grain[i] < -1 || grain[i] >= n_grains)
            return fail(h, HAMR_ERR_ARG, "grain[%lld] = %d outside [-1, %d)", i, grain[i], n_grains);
    DeviceGuard dg(h->device);
    for (long long z = 0; z < R.nz; ++z)
        for (long long y = 0; y < R.ny; ++y)
            for (long long x = 0; x < R.nx; ++x) {
                const long long i = x + (long long)R.nx * (y + (long long)R.ny * z);
                h->gcode_h[slot_of(R, x, y, z)] = (uint16_t)(grain[i] + 1);
            }
    // does any stencil bond join two different grains?
    int cross = 0;
    for (long long z = 0; z < R.nz && !cross; ++z)
        for (long long y = 0; y < R.ny && !cross; ++y)
            for (long long x = 0; x < R.nx && !cross; ++x) {
                const uint16_t g = h->gcode_h[slot_of(R, x, y, z)];
                if (!g) continue;
                for (const Off &o : bond_offsets(h->lattice)) {
                    int jx = (int)x + o.dx, jy = (int)y + o.dy, jz = (int)z + o.dz;
                    if (!wrap(jx, R.nx, h->per[0]) || !wrap(jy, R.ny, h->per[1]) || !wrap(jz, R.nz, h->per[2]))
                        continue;
                    const uint16_t gj = h->gcode_h[slot_of(R, jx, jy, jz)];
                    if (gj && gj != g) {
                        cross = 1;
                        break;
                    }
                }
            }
    R.cross_grain = cross;
    h->n_grains[replica] = n_grains;
    count_grains(h, replica);
    // the fused path lists only columns that hold a magnetic site: rebuild its work list
    h->items_dirty = true;
    clear_graphs(h);
    const long long span = (long long)R.px * R.ny * R.nz;
    CK(h, cudaMemcpyAsync(h->gcode_d + R.off, h->gcode_h.data() + R.off, sizeof(uint16_t) * span,
                          cudaMemcpyHostToDevice, h->stream));
    // both state buffers: the fused kernel never writes non-magnetic sites
    for (int b = 0; b < 2; ++b)
        if (h->S[b]) CK(h, launch_zero_void(h->prec, h->S[b], h->NS, h->gcode_d, R.off, span, h->stream));
    if (h->nbr == HAMR_NBR_CSR) {
        if (build_ell_replica(h, replica, h->ell_w) != 0) return fail(h, HAMR_ERR_ARG, "neighbour list too wide");
        int rc = upload_ell_replica(h, replica);
        if (rc) return rc;
    }
    return refresh_grains(h);
}

int hamr_set_temperature_profile(hamr_t h, int32_t replica, double T_amb, double T_peak, double fwhm, double x0,
                                 double y0, double vx, double vy) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!(T_amb >= 0) || !(T_peak >= 0) || !isfinite(fwhm) || !isfinite(x0) || !isfinite(y0) || !isfinite(vx) ||
        !isfinite(vy))
        return fail(h, HAMR_ERR_ARG, "temperatures must be >= 0 and all values finite");
    DeviceGuard dg(h->device);
    ReplicaDev &R = h->reps_h[replica];
    R.T_amb = T_amb;
    R.dT = fwhm > 0 ? T_peak - T_amb : 0.0;
    R.c_fwhm = fwhm > 0 ? -4.0 * log(2.0) / (fwhm * fwhm) : 0.0;
    R.x0 = x0;
    R.y0 = y0;
    R.vx = vx;
    R.vy = vy;
    set_driver_floats(R);
    return upload_replica(h, replica);
}

int hamr_set_field_sequence(hamr_t h, int32_t replica, double B0, const double dir[3], const uint8_t *bits,
                            int32_t n_bits, double bit_len, double ramp_len, double head_x0, double head_v) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!dir || !isfinite(B0) || !isfinite(dir[0]) || !isfinite(dir[1]) || !isfinite(dir[2]))
        return fail(h, HAMR_ERR_ARG, "field amplitude and direction must be finite");
    if (n_bits < 0 || (n_bits > 0 && (!bits || !(bit_len > 0) || !(ramp_len >= 0) || !isfinite(head_x0) ||
                                      !isfinite(head_v))))
        return fail(h, HAMR_ERR_ARG, "bad bit sequence (bits, bit_len > 0, ramp_len >= 0)");
    DeviceGuard dg(h->device);
    h->bits_h[replica].assign(bits, bits + n_bits);
    size_t total = 0;
    for (int r = 0; r < h->R; ++r) total += h->bits_h[r].size();
    std::vector<uint8_t> all;
    all.reserve(total);
    for (int r = 0; r < h->R; ++r) {
        h->reps_h[r].bits_off = (int)all.size();
        h->reps_h[r].n_bits = (int)h->bits_h[r].size();
        all.insert(all.end(), h->bits_h[r].begin(), h->bits_h[r].end());
    }
    if (total > h->bits_cap) {
        dfree(h->bits_d);
        h->bits_cap = std::max(total, 2 * h->bits_cap);
        CK(h, dalloc(h, &h->bits_d, h->bits_cap));
        clear_graphs(h);
    }
    if (total) CK(h, cudaMemcpyAsync(h->bits_d, all.data(), total, cudaMemcpyHostToDevice, h->stream));
    ReplicaDev &R = h->reps_h[replica];
    R.B0 = B0;
    for (int d = 0; d < 3; ++d) R.dir[d] = dir[d];
    R.bit_len = n_bits > 0 ? bit_len : 1.0;
    R.ramp_len = n_bits > 0 ? ramp_len : 0.0;
    R.head_x0 = head_x0;
    R.head_v = head_v;
    set_driver_floats(R);
    CK(h, cudaMemcpyAsync(h->reps_d, h->reps_h.data(), sizeof(ReplicaDev) * h->R, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

static int set_moments_impl(hamr_t h, int32_t replica, const double *S, bool host) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!S) return fail(h, HAMR_ERR_ARG, "null spin array");
    DeviceGuard dg(h->device);
    const ReplicaDev &R = h->reps_h[replica];
    const double *src = S;
    if (host) {
        CK(h, cudaMemcpyAsync(h->stage_d, S, sizeof(double) * 3 * R.n, cudaMemcpyHostToDevice, h->stream));
        src = h->stage_d;
    }
    CK(h, launch_aos_to_soa(h->prec, src, h->S[h->cur], h->NS, h->reps_d, replica, h->gcode_d, R.n, h->stream));
    if (host) CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_set_moments(hamr_t h, int32_t replica, const double *S) { return set_moments_impl(h, replica, S, true); }
int hamr_set_moments_device(hamr_t h, int32_t replica, const double *S) {
    return set_moments_impl(h, replica, S, false);
}

int hamr_sllg_heun_steps(hamr_t h, int64_t n_steps, int32_t record_every) {
    return steps_impl(h, n_steps, record_every, true);
}

int hamr_sllg_heun_steps_async(hamr_t h, int64_t n_steps, int32_t record_every) {
    return steps_impl(h, n_steps, record_every, false);
}

int hamr_synchronize(hamr_t h) {
    if (!h) return HAMR_ERR_ARG;
    DeviceGuard dg(h->device);
    return collect_records(h);
}

static int read_moments_impl(hamr_t h, int32_t replica, double *S, bool host) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!S) return fail(h, HAMR_ERR_ARG, "null output array");
    DeviceGuard dg(h->device);
    const ReplicaDev &R = h->reps_h[replica];
    double *dst = host ? h->stage_d : S;
    CK(h, launch_soa_to_aos(h->prec, h->S[h->cur], h->NS, h->reps_d, replica, dst, R.n, h->stream));
    if (host) {
        CK(h, cudaMemcpyAsync(S, h->stage_d, sizeof(double) * 3 * R.n, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return HAMR_OK;
}

int hamr_read_moments(hamr_t h, int32_t replica, double *S_out) { return read_moments_impl(h, replica, S_out, true); }
int hamr_read_moments_device(hamr_t h, int32_t replica, double *S_dev) {
    return read_moments_impl(h, replica, S_dev, false);
}

int hamr_read_magnetisation(hamr_t h, int32_t replica, double *M_t, int64_t capacity, int64_t *n_rec,
                            double *M_grain, int64_t *step_of_rec) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!n_rec || capacity < 0) return fail(h, HAMR_ERR_ARG, "n_rec must not be null");
    if (h->pending_records) {
        DeviceGuard dg(h->device);
        int rc = collect_records(h);
        if (rc) return rc;
    }
    const long long n = (long long)h->rec_step_h.size();
    *n_rec = n;
    if (M_t) {
        const long long m = std::min<long long>(n, capacity);
        for (long long k = 0; k < m; ++k)
            for (int d = 0; d < 3; ++d) M_t[3 * k + d] = h->rec_h[((size_t)k * h->R + replica) * 3 + d];
        if (step_of_rec)
            for (long long k = 0; k < m; ++k) step_of_rec[k] = h->rec_step_h[k];
    }
    if (M_grain) {
        const ReplicaDev &R = h->reps_h[replica];
        for (int g = 0; g < R.n_grains; ++g)
            for (int d = 0; d < 3; ++d) M_grain[3 * g + d] = h->grain_last_h[3 * (size_t)(R.grain_off + g) + d];
    }
    return HAMR_OK;
}

int hamr_clear_records(hamr_t h) {
    if (!h) return HAMR_ERR_ARG;
    if (h->pending_records) {
        DeviceGuard dg(h->device);
        int rc = collect_records(h);
        if (rc) return rc;
    }
    h->rec_h.clear();
    h->rec_step_h.clear();
    return HAMR_OK;
}

int hamr_read_energy(hamr_t h, int32_t replica, double *E) {
    if (bad_replica(h, replica)) return h ? fail(h, HAMR_ERR_ARG, "bad replica %d", replica) : HAMR_ERR_ARG;
    if (!E) return fail(h, HAMR_ERR_ARG, "null output");
    if (!h->shells_set) return fail(h, HAMR_ERR_STATE, "exchange shells not set");
    DeviceGuard dg(h->device);
    CK(h, cudaMemsetAsync(h->dscratch_d, 0, sizeof(double), h->stream));
    CK(h, launch_energy(h->prec, h->S[h->cur], h->NS, h->gcode_d, h->reps_d, h->reps_h[replica], replica, h->bits_d,
                        h->nbr == HAMR_NBR_CSR ? h->ell_d : nullptr, h->ell_w, h->ph, h->step_h, h->ku, h->mu_s,
                        h->dscratch_d, h->stream));
    CK(h, cudaMemcpyAsync(E, h->dscratch_d, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return HAMR_OK;
}

int hamr_get_step(hamr_t h, int64_t *step) {
    if (!h || !step) return HAMR_ERR_ARG;
    *step = h->step_h;
    return HAMR_OK;
}

int hamr_set_step(hamr_t h, int64_t step) {
    if (!h) return HAMR_ERR_ARG;
    if (step < 0) return fail(h, HAMR_ERR_ARG, "step must be >= 0");
    DeviceGuard dg(h->device);
    CK(h, cudaStreamSynchronize(h->stream));
    Ctl c;
    CK(h, cudaMemcpy(&c, h->ctl_d, sizeof c, cudaMemcpyDeviceToHost));
    c.step = step;
    c.work_ctr[0] = c.work_ctr[1] = 0;
    CK(h, cudaMemcpy(h->ctl_d, &c, sizeof c, cudaMemcpyHostToDevice));
    h->step_h = step;
    if (fused_mode(h) && h->cur != (int)(step & 1)) {
        // the fused kernel finds the state of step n in buffer n & 1
        CK(h, launch_copy_state(h->prec, h->S[h->cur], h->S[step & 1], h->NS, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->cur = (int)(step & 1);
    }
    return HAMR_OK;
}

int hamr_check_finite(hamr_t h) {
    if (!h) return HAMR_ERR_ARG;
    DeviceGuard dg(h->device);
    CK(h, cudaMemsetAsync(&h->ctl_d->err, 0, sizeof(int), h->stream));
    CK(h, launch_check_finite(h->prec, h->S[h->cur], h->NS, h->gcode_d, h->ctl_d, h->stream));
    int err = 0;
    CK(h, cudaMemcpyAsync(&err, &h->ctl_d->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (err) return fail(h, HAMR_ERR_NUMERIC, "non-finite or non-unit spin found");
    return HAMR_OK;
}

static const char kMagic[8] = {'H', 'A', 'M', 'R', 'S', 'T', '0', '1'};

int hamr_save_state(hamr_t h, const char *path) {
    if (!h || !path) return HAMR_ERR_ARG;
    std::ofstream f(path, std::ios::binary);
    if (!f) return fail(h, HAMR_ERR_IO, "cannot open %s", path);
    const int32_t hdr[4] = {h->prec, h->lattice, h->R, 0};
    f.write(kMagic, 8);
    f.write((const char *)hdr, sizeof hdr);
    f.write((const char *)h->dims.data(), sizeof(int) * h->dims.size());
    f.write((const char *)h->seeds.data(), sizeof(uint64_t) * h->seeds.size());
    const int64_t step = h->step_h;
    f.write((const char *)&step, sizeof step);
    std::vector<double> buf;
    for (int r = 0; r < h->R; ++r) {
        buf.resize(3 * (size_t)h->reps_h[r].n);
        int rc = hamr_read_moments(h, r, buf.data());
        if (rc) return rc;
        f.write((const char *)buf.data(), sizeof(double) * buf.size());
    }
    if (!f) return fail(h, HAMR_ERR_IO, "write to %s failed", path);
    return HAMR_OK;
}

int hamr_load_state(hamr_t h, const char *path) {
    if (!h || !path) return HAMR_ERR_ARG;
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(h, HAMR_ERR_IO, "cannot open %s", path);
    char magic[8];
    int32_t hdr[4];
    f.read(magic, 8);
    f.read((char *)hdr, sizeof hdr);
    if (!f || memcmp(magic, kMagic, 8) != 0) return fail(h, HAMR_ERR_IO, "%s is not a state file", path);
    if (hdr[0] != h->prec || hdr[1] != h->lattice || hdr[2] != h->R)
        return fail(h, HAMR_ERR_ARG, "state file shape or precision differs from the handle");
    std::vector<int> dims(3 * (size_t)h->R);
    std::vector<uint64_t> seeds(h->R);
    f.read((char *)dims.data(), sizeof(int) * dims.size());
    f.read((char *)seeds.data(), sizeof(uint64_t) * seeds.size());
    int64_t step = 0;
    f.read((char *)&step, sizeof step);
    if (!f || dims != h->dims) return fail(h, HAMR_ERR_ARG, "state file dimensions differ from the handle");
    if (seeds != h->seeds) return fail(h, HAMR_ERR_ARG, "state file seeds differ from the handle");
    std::vector<double> buf;
    for (int r = 0; r < h->R; ++r) {
        buf.resize(3 * (size_t)h->reps_h[r].n);
        f.read((char *)buf.data(), sizeof(double) * buf.size());
        if (!f) return fail(h, HAMR_ERR_IO, "%s is truncated", path);
        int rc = hamr_set_moments(h, r, buf.data());
        if (rc) return rc;
    }
    return hamr_set_step(h, step);
}

static int find_variant(int threads, int staged) {
    FusedVariant v;
    for (int i = 0; fused_variant(i, v); ++i)
        if (v.threads == threads && v.staged == staged) return i;
    return -1;
}

int hamr_set_tile(hamr_t h, int32_t threads, int32_t staged) {
    if (!h) return HAMR_ERR_ARG;
    const int v = find_variant(threads, staged);
    if (v < 0) return fail(h, HAMR_ERR_ARG, "no compiled kernel variant with %d threads, %d staged positions", threads,
                           staged);
    DeviceGuard dg(h->device);
    if (fused_max_blocks_per_sm(v, tetragonal(h)) < 1) return fail(h, HAMR_ERR_ARG, "variant %d cannot launch", v);
    if (v != h->variant) {
        h->variant = v;
        h->items_dirty = true;
        clear_graphs(h);
    }
    return HAMR_OK;
}

int hamr_get_tile(hamr_t h, int32_t *threads, int32_t *staged) {
    if (!h || !threads || !staged) return HAMR_ERR_ARG;
    FusedVariant v;
    fused_variant(h->variant, v);
    *threads = v.threads;
    *staged = v.staged;
    return HAMR_OK;
}

int hamr_set_plane_range(hamr_t h, int32_t planes) {
    if (!h) return HAMR_ERR_ARG;
    if (planes < 0) return fail(h, HAMR_ERR_ARG, "planes must be >= 0");
    if (planes != h->z_range_set) {
        h->z_range_set = planes;
        h->items_dirty = true;
        clear_graphs(h);
    }
    return HAMR_OK;
}

int hamr_autotune(hamr_t h, int32_t steps_per_trial) {
    if (!h) return HAMR_ERR_ARG;
    Range nv("hamr autotune");
    if (steps_per_trial < 1) return fail(h, HAMR_ERR_ARG, "steps_per_trial must be >= 1");
    if (!fused_mode(h)) return HAMR_OK;  // the two-pass path has a single launch shape
    if (!h->shells_set) return fail(h, HAMR_ERR_STATE, "exchange shells not set");
    DeviceGuard dg(h->device);
    // keep the state, step and records: trials run on a copy and are undone
    void *backup = nullptr;
    CK(h, cudaMalloc(&backup, 3 * h->NS * sizeof(float)));
    CK(h, launch_copy_state(h->prec, h->S[h->cur], backup, h->NS, h->stream));
    const long long step0 = h->step_h;
    const int cur0 = h->cur;
    float best = 1e30f;
    int bestv = h->variant;
    // with the range length left to the work model (z_range_set 0), a shape the model splits
    // along z is also timed on whole columns: the model does not know every shape's costs
    const int zset0 = h->z_range_set;
    int maxnz = 1;
    for (const ReplicaDev &R : h->reps_h) maxnz = std::max(maxnz, R.nz);
    int bestz = zset0;
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    int rc = HAMR_OK;
    auto trial = [&](int zset, float &ms) -> int {
        int r = hamr_set_plane_range(h, zset);
        if (!r) r = steps_impl(h, steps_per_trial, 0, true);  // warm-up, graph capture
        if (r) return r;
        cudaError_t e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess && !(r = steps_impl(h, steps_per_trial, 0, false))) {
            e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (r) return r;
        return e == cudaSuccess ? HAMR_OK : fail(h, HAMR_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
    };
    FusedVariant v;
    for (int i = 0; fused_variant(i, v); ++i) {
        if (fused_max_blocks_per_sm(i, tetragonal(h)) < 1) continue;
        if ((rc = hamr_set_tile(h, v.threads, v.staged))) break;
        float ms = 0;
        if ((rc = trial(zset0, ms))) break;
        if (ms < best) {
            best = ms;
            bestv = i;
            bestz = zset0;
        }
        if (zset0 == 0 && h->z_split && maxnz > 1) {
            if ((rc = trial(maxnz, ms))) break;
            if (ms < best) {
                best = ms;
                bestv = i;
                bestz = maxnz;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cur = cur0;
    CK(h, launch_copy_state(h->prec, backup, h->S[h->cur], h->NS, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(backup);
    int rc2 = hamr_set_step(h, step0);
    if (rc) return rc;
    if (rc2) return rc2;
    fused_variant(bestv, v);
    if ((rc = hamr_set_plane_range(h, bestz))) return rc;
    return hamr_set_tile(h, v.threads, v.staged);
}

int hamr_query(hamr_t h, int32_t key, int64_t *value) {
    if (!h || !value) return HAMR_ERR_ARG;
    switch (key) {
        case 0: {
            long long n = 0;
            for (auto &R : h->reps_h) n += R.n;
            *value = n;
            return HAMR_OK;
        }
        case 1: {
            long long n = 0;
            for (long long m : h->nmag_h) n += m;
            *value = n;
            return HAMR_OK;
        }
        case 2:
            *value = (int64_t)h->dev_bytes;
            return HAMR_OK;
        case 3:
            *value = fused_mode(h) ? 1 : 2;
            return HAMR_OK;
        case 4:
            *value = h->NS;
            return HAMR_OK;
        case 5:
        case 6: {
            if (fused_mode(h) && h->items_dirty) {
                DeviceGuard dg(h->device);
                int rc = build_items(h);
                if (rc) return rc;
            }
            *value = key == 5 ? h->n_items : h->z_range;
            return HAMR_OK;
        }
        default:
            return fail(h, HAMR_ERR_ARG, "unknown query key %d", key);
    }
}

int hamr_inject_wait_timeout(hamr_t h, int32_t polls) {
    if (!h) return HAMR_ERR_ARG;
    if (polls < 1) return fail(h, HAMR_ERR_ARG, "polls must be >= 1");
    if (!fused_mode(h)) return fail(h, HAMR_ERR_STATE, "only the fused FP32 stencil kernel has bounded waits");
    h->inject_polls = (unsigned)polls;
    return HAMR_OK;
}

const char *hamr_last_error(hamr_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void hamr_destroy(hamr_t h) {
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        destroy_device(h);
    }
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
