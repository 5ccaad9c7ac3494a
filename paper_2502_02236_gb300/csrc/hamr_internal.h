// Internal types of the GB300 sLLG library: device-side replica table, physical
// constants, kernel argument blocks and the host context behind a hamr_t.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "hamr.h"

namespace hamr {

constexpr double KB = 1.380649e-23;   // Boltzmann constant [J/K]
constexpr int SLOT_ALIGN = 256;       // replica storage offsets are multiples of this
constexpr int PLAIN_BLOCK = 256;      // threads per block of the two-pass kernels
constexpr int MAX_SHELLS = 4;
constexpr int ELL_MAX = 32;           // neighbours per site in the list format
constexpr int ELL_SHELL_SHIFT = 28;   // packed neighbour: storage index | shell << 28

// Per-replica constants, read by every kernel (one entry per replica in device memory).
struct ReplicaDev {
    int nx, ny, nz, px;        // logical dimensions and storage pitch along x
    long long off;             // storage slot of site (0,0,0)
    long long n;               // nx * ny * nz
    unsigned key0, key1;       // Philox key = replica seed (low, high)
    int grain_off, n_grains;   // this replica's grain bins in the global accumulator
    int cross_grain;           // 1 when a stencil bond joins two different grains
    int n_bits, bits_off;      // write-field bit pattern in the global bit buffer
    int pad_;
    // laser spot: T = T_amb + dT exp(c_fwhm r^2), c_fwhm = -4 ln2 / fwhm^2 (0: uniform)
    double T_amb, dT, c_fwhm, x0, y0, vx, vy;
    // write field B0 * s(t) * dir
    double B0, dir[3], bit_len, ramp_len, head_x0, head_v;
    // FP32 copies used by the FP32 kernels
    float fT_amb, fdT, fc_fwhm, fx0, fy0, fvx, fvy;
    float fB0, fdir[3], fbit_len, framp_len, fhead_x0, fhead_v;
};

// Constants shared by all replicas.
struct Phys {
    double cJ[MAX_SHELLS];  // J_s / mu_s [T]
    double cK;              // 2 ku / mu_s [T]
    double pref;            // -gamma / (1 + alpha^2)
    double alpha, dt;
    double sig0;            // sqrt(2 alpha kB / (gamma mu_s dt)); sigma_i = sig0 sqrt(T_i) [T]
    double ax, ay, az;      // site spacing [m]
    int per[3];
    int n_shells;
    int lattice;            // HAMR_LATTICE_SC or HAMR_LATTICE_L10 (the implicit stencil's shape)
};

// Device control block.
struct Ctl {
    long long step;          // completed steps
    long long n_rec;         // records written since the host last collected them
    unsigned work_ctr[2];    // work-list counters of the persistent kernel (by step parity)
    int err;                 // error flags (bit 0: bad value found by the finite check;
                             // bit 1: a bounded wait of the fused kernel ran out)
    int ticket;              // blocks of a record's bookkeeping that are done (0 between launches)
};

// One unit of work of the fused kernel: a block of columns of one replica.
// Runs of consecutive storage slots of one grain (at most GRAIN_RUN_MAX slots, within one
// row), packed as slot << 5 | (length - 1) and grouped by global grain bin; an item is up
// to GRAIN_RUN_MAX runs of one grain, summed by one warp.
constexpr int GRAIN_RUN_MAX = 32;
struct GrainRunItem {
    long long run0;  // first run of the item
    int grain;       // global grain bin
    int n_runs;      // 1 .. GRAIN_RUN_MAX
};

struct WorkItem {
    int r;         // replica
    int x0, y0;    // first interior column
    int bxy;       // interior width | height << 16
    int list_off;  // first entry of its column list
    int counts;    // listed columns | interior columns << 16
    int stage;     // 1: staged by TMA | columns between the staged origin and x0 - 2, << 8
    int zr;        // first plane | planes << 16
};

// A compiled variant of the fused kernel.
struct FusedVariant {
    int threads;  // CTA size
    int columns;  // listed columns per work item at most (a whole number per thread)
    int pitch;    // staged-region row pitch: bx + 4 <= pitch
    int rows;     // staged-region rows: by + 4 <= rows
    int staged;   // pitch * rows
};

template <typename Real>
struct PlainArgs {
    Real *S, *SP, *F1, *BTH;      // component planes [3][NS]
    long long NS;
    const uint16_t *gcode;        // grain code per slot: 0 = non-magnetic, else grain + 1
    const int *blk_rep;           // replica of each PLAIN_BLOCK-slot block
    const ReplicaDev *reps;
    const uint8_t *bits;
    const int *ell;               // packed neighbour list [ell_w][NS], or null (stencil)
    int ell_w;
    const Ctl *ctl;
    int step_off;
    Phys ph;
    double *grain_acc;            // [G][3] sums at record steps
};

struct FusedArgs {
    float *Sbuf0, *Sbuf1;       // state at step n lives in Sbuf[n & 1]
    long long NS;
    const uint16_t *gcode;
    const ReplicaDev *reps;
    const uint8_t *bits;
    const WorkItem *items;
    const uint16_t *lists;      // column lists of all items (staged-region positions)
    int n_items;
    Ctl *ctl;
    int step_off;
    float cJ[3];                // J_s / mu_s of the stencil's shells (SC: shell 0 only) [T]
    float cK, pref, alpha, dt, sig0, ax, ay, az;
    int per[3];
    const CUtensorMap *maps;       // [R][2] tensor maps of each replica's state in each buffer
    unsigned wait_polls;           // a bounded device wait fails after this many polls
    int inject;                    // failure-detection test: 1 = the CTA of work item 0 withholds
                                   // one arrival on the staging barrier of plane 1
};

// kernel launchers (kernels_*.cu)
cudaError_t launch_plain_step(int prec, const void *args, int n_blocks, bool record, cudaStream_t st);
// tet: the L1_0 (tetragonal three-shell) stencil instead of the simple-cubic one; zr: some work
// items cover plane ranges (WorkItem::zr)
cudaError_t launch_fused_step(int variant, bool tet, bool zr, const FusedArgs &a, int grid, cudaStream_t st);
// exact per-grain sums (fixed point, 2^-24) of the FP32 state after G steps from ctl->step,
// into grain_fx (read by k_bookkeeping at a record point)
cudaError_t launch_grain_sums_fx(const float *S0, const float *S1, long long NS, const unsigned long long *runs,
                                 const GrainRunItem *items, int n_items, const Ctl *ctl, int G,
                                 unsigned long long *grain_fx, cudaStream_t st);
bool fused_variant(int variant, FusedVariant &out);
int fused_max_blocks_per_sm(int variant, bool tet);
cudaError_t launch_bookkeeping(Ctl *ctl, int G, bool record, int R, const ReplicaDev *reps,
                               const long long *nmag, const long long *gcount, int Gtot, double *grain_acc,
                               unsigned long long *grain_fx, double *grain_last, double *rec, long long rec_cap,
                               long long *rec_step, cudaStream_t st);
cudaError_t launch_init_state(int prec, void *S, long long NS, const uint16_t *gcode, cudaStream_t st);
cudaError_t launch_zero_void(int prec, void *S, long long NS, const uint16_t *gcode, long long first,
                             long long count, cudaStream_t st);
cudaError_t launch_aos_to_soa(int prec, const double *src, void *S, long long NS, const ReplicaDev *reps,
                              int r, const uint16_t *gcode, long long n, cudaStream_t st);
cudaError_t launch_soa_to_aos(int prec, const void *S, long long NS, const ReplicaDev *reps, int r,
                              double *dst, long long n, cudaStream_t st);
cudaError_t launch_energy(int prec, const void *S, long long NS, const uint16_t *gcode,
                          const ReplicaDev *reps, const ReplicaDev &Rh, int r, const uint8_t *bits,
                          const int *ell, int ell_w, const Phys &ph, long long step, double ku, double mu_s,
                          double *out, cudaStream_t st);
cudaError_t launch_check_finite(int prec, const void *S, long long NS, const uint16_t *gcode, Ctl *ctl,
                                cudaStream_t st);
cudaError_t launch_copy_state(int prec, const void *src, void *dst, long long NS, cudaStream_t st);

}  // namespace hamr

// The host context behind a hamr_t.
struct hamr_ctx {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int lattice = 0, prec = 0, nbr = 0, R = 0;
    std::vector<int> dims;            // 3R
    std::vector<uint64_t> seeds;
    double a = 0, c = 0, mu_s = 0, ku = 0, alpha = 0, dt = 0, gamma = 0;
    int per[3] = {0, 0, 0};
    hamr::Phys ph{};
    bool shells_set = false;
    std::vector<double> J;

    long long NS = 0;                 // storage slots per component
    std::vector<hamr::ReplicaDev> reps_h;
    hamr::ReplicaDev *reps_d = nullptr;
    void *S[2] = {nullptr, nullptr};  // state planes [3][NS] (FP32 fused path ping-pongs)
    int cur = 0;
    void *SP = nullptr, *F1 = nullptr, *BTH = nullptr;   // two-pass intermediates
    uint16_t *gcode_d = nullptr;
    std::vector<uint16_t> gcode_h;
    int *blk_rep_d = nullptr;
    int *ell_d = nullptr;
    int ell_w = 0;
    std::vector<int> ell_h;           // host copy of the packed list (rebuilt per replica)
    // user-supplied lists (logical site indices), kept to re-filter when grains change
    std::vector<std::vector<int>> ucsr_rp, ucsr_col;
    std::vector<std::vector<uint8_t>> ucsr_sh;
    int max_user_shell = -1;
    uint8_t *bits_d = nullptr;
    std::vector<std::vector<uint8_t>> bits_h;
    size_t bits_cap = 0;
    hamr::Ctl *ctl_d = nullptr;

    // reductions
    std::vector<int> n_grains;        // per replica
    int G = 0, G_cap = 0;             // total grain bins and allocated capacity
    double *grain_acc_d = nullptr, *grain_last_d = nullptr;
    unsigned long long *grain_fx_d = nullptr;
    long long *gcount_d = nullptr, *nmag_d = nullptr;
    std::vector<long long> gcount_h, nmag_h;
    std::vector<std::vector<long long>> gcount_rep;   // per replica, per grain
    double *rec_d = nullptr;
    long long *rec_step_d = nullptr;
    long long rec_cap = 0;
    std::vector<double> rec_h;        // [n][R][3]
    std::vector<long long> rec_step_h;
    std::vector<double> grain_last_h;
    bool pending_records = false;
    double *dscratch_d = nullptr;     // small FP64 scratch (energy)
    double *stage_d = nullptr;        // FP64 AoS staging for host copies (3 x max replica)
    long long stage_n = 0;
    long long step_h = 0;             // host mirror of the step counter

    // fused kernel tiling
    int variant = 0;
    hamr::WorkItem *items_d = nullptr;
    int n_items = 0, items_cap = 0;
    uint16_t *lists_d = nullptr;
    size_t lists_cap = 0;
    CUtensorMap *maps_d = nullptr;    // [R][2] (variant-dependent box)
    std::vector<int> tma_ok;          // replica staged by TMA (open in x and y, no grain mask)
    int fused_grid = 0;
    int z_range = 0;                  // planes per work item (the longest; 0 until items are built)
    int z_range_set = 0;              // > 0: plane range fixed by hamr_set_plane_range
    bool z_split = false;             // some work items cover plane ranges (the range kernel runs)
    unsigned inject_polls = 0;        // >0: the next step block runs the failure test
    bool items_dirty = true;
    // per-grain runs for the record sums of the FP32 fused path (rebuilt after grain changes)
    unsigned long long *runs_d = nullptr;
    hamr::GrainRunItem *gitems_d = nullptr;
    long long runs_cap = 0;
    int gitems_cap = 0, n_gitems = 0;
    bool runs_dirty = true;
    int num_sms = 0;
    size_t dev_bytes = 0;

    // captured step blocks: (steps, record, start parity, tile) -> executable graph
    std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
};
