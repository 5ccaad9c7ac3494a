// Record bookkeeping after a block of steps, layout conversion between the FP64 site-major
// boundary format and the internal component planes, state initialisation and the
// finite-value scan.
#include "device_common.cuh"

namespace hamr {

// After a block of G steps: advance the step counter and, at a record point, turn the
// per-grain FP64 sums into the replica magnetisation M = sum S / N_mag (Eq. 6 as an
// average over magnetic sites), per-grain averages, and clear the sums.  A record launch has
// one block per replica: the block folds the FP32 path's exact fixed-point sums (units of
// 2^-24) of its grains into their FP64 sums, writes the grain averages, clears both and
// reduces its replica's M over a fixed tree.  Every block reads the step counter and the
// record index before any is changed: the last block to finish (a ticket counted in ctl)
// advances them.
constexpr int BK_THREADS = 128;
__global__ void __launch_bounds__(BK_THREADS) k_bookkeeping(Ctl *ctl, int G, int record, const ReplicaDev *reps,
                                                             const long long *nmag, const long long *gcount,
                                                             double *grain_acc, unsigned long long *grain_fx,
                                                             double *grain_last, double *rec, long long rec_cap,
                                                             long long *rec_step, int R) {
    const long long after = ctl->step + G;
    if (!record) {
        if (threadIdx.x == 0) ctl->step = after;
        return;
    }
    const long long idx = ctl->n_rec;
    const int r = blockIdx.x;
    const int g0 = reps[r].grain_off, ng = reps[r].n_grains;
    double mx = 0, my = 0, mz = 0;
    for (int g = g0 + (int)threadIdx.x; g < g0 + ng; g += BK_THREADS) {
        double t[3];
        for (int d = 0; d < 3; ++d) {
            t[d] = grain_acc[3 * g + d] + (double)(long long)grain_fx[3 * g + d] * 5.9604644775390625e-08;
            grain_acc[3 * g + d] = 0.0;
            grain_fx[3 * g + d] = 0ull;
        }
        mx += t[0];
        my += t[1];
        mz += t[2];
        const double c = (double)gcount[g];
        for (int d = 0; d < 3; ++d) grain_last[3 * g + d] = c > 0 ? t[d] / c : 0.0;
    }
    __shared__ double sm[3][BK_THREADS];
    sm[0][threadIdx.x] = mx;
    sm[1][threadIdx.x] = my;
    sm[2][threadIdx.x] = mz;
    __syncthreads();
    for (int w = BK_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int d = 0; d < 3; ++d) sm[d][threadIdx.x] += sm[d][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nm = (double)nmag[r];
        if (idx < rec_cap) {
            double *o = rec + (idx * R + r) * 3;
            for (int d = 0; d < 3; ++d) o[d] = nm > 0 ? sm[d][0] / nm : 0.0;
        }
        __threadfence();
        if (atomicAdd(&ctl->ticket, 1) == (int)gridDim.x - 1) {  // every block has read ctl
            if (idx < rec_cap) rec_step[idx] = after;
            ctl->n_rec = idx + 1;
            ctl->step = after;
            ctl->ticket = 0;
        }
    }
}

cudaError_t launch_bookkeeping(Ctl *ctl, int G, bool record, int R, const ReplicaDev *reps, const long long *nmag,
                               const long long *gcount, int Gtot, double *grain_acc, unsigned long long *grain_fx,
                               double *grain_last, double *rec, long long rec_cap, long long *rec_step,
                               cudaStream_t st) {
    (void)Gtot;
    k_bookkeeping<<<record ? R : 1, BK_THREADS, 0, st>>>(ctl, G, record ? 1 : 0, reps, nmag, gcount, grain_acc,
                                                         grain_fx, grain_last, rec, rec_cap, rec_step, R);
    return cudaGetLastError();
}

// Per-grain sums of the FP32 state after a block of G steps from ctl->step (the new state is
// in buffer (step + G) mod 2): every magnetic slot adds its spin, rounded to a multiple of 2^-24,
// to its grain's 64-bit fixed-point sums.  One warp takes one item (up to 32 runs of one grain):
// lane k holds run k's descriptor; each run is read by the lanes of the warp in one coalesced
// pass per component; a lane's partial sums (at most 32 sites of magnitude <= 2^24) fit in 32
// bits; the warp reduces them in 64 bits and adds them to the grain once.  The sums are
// integers, so the result does not depend on the order of the additions.
__global__ void __launch_bounds__(PLAIN_BLOCK) k_grain_sums_fx(
    const float *__restrict__ S0, const float *__restrict__ S1, long long NS,
    const unsigned long long *__restrict__ runs, const GrainRunItem *__restrict__ items, int n_items,
    const Ctl *__restrict__ ctl, int G, unsigned long long *__restrict__ grain_fx) {
    const int w = blockIdx.x * (PLAIN_BLOCK / 32) + (threadIdx.x >> 5);
    if (w >= n_items) return;   // uniform over the warp
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const GrainRunItem it = items[w];
    const unsigned long long mine = lane < it.n_runs ? runs[it.run0 + lane] : 0ull;
    const float *__restrict__ S = ((ctl->step + G) & 1) ? S1 : S0;
    int sx = 0, sy = 0, sz = 0;
    // eight runs at a time, every load issued before any is used: a lane past its run's end
    // (or past the item's last run) reads the run's first slot, a valid address, and drops it
    constexpr int RB = 8;
    for (int k0 = 0; k0 < it.n_runs; k0 += RB) {
        float vx[RB], vy[RB], vz[RB];
        bool on[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int k = k0 + u;
            const unsigned long long rw = __shfl_sync(full, mine, k & 31);
            on[u] = k < it.n_runs && lane <= (int)(rw & 31ull);
            const long long j = (long long)(rw >> 5) + (on[u] ? lane : 0);
            vx[u] = S[j];
            vy[u] = S[NS + j];
            vz[u] = S[2 * NS + j];
        }
#pragma unroll
        for (int u = 0; u < RB; ++u)
            if (on[u]) {
                sx += __float2int_rn(vx[u] * FX_SCALE);
                sy += __float2int_rn(vy[u] * FX_SCALE);
                sz += __float2int_rn(vz[u] * FX_SCALE);
            }
    }
    long long tx = sx, ty = sy, tz = sz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tx += __shfl_xor_sync(full, tx, o);
        ty += __shfl_xor_sync(full, ty, o);
        tz += __shfl_xor_sync(full, tz, o);
    }
    if (lane == 0) {
        atomicAdd(grain_fx + 3 * (long long)it.grain + 0, (unsigned long long)tx);
        atomicAdd(grain_fx + 3 * (long long)it.grain + 1, (unsigned long long)ty);
        atomicAdd(grain_fx + 3 * (long long)it.grain + 2, (unsigned long long)tz);
    }
}

cudaError_t launch_grain_sums_fx(const float *S0, const float *S1, long long NS, const unsigned long long *runs,
                                 const GrainRunItem *items, int n_items, const Ctl *ctl, int G,
                                 unsigned long long *grain_fx, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const int per = PLAIN_BLOCK / 32;
    k_grain_sums_fx<<<(unsigned)((n_items + per - 1) / per), PLAIN_BLOCK, 0, st>>>(S0, S1, NS, runs, items, n_items,
                                                                               ctl, G, grain_fx);
    return cudaGetLastError();
}

template <typename Real>
__global__ void k_aos_to_soa(const double *src, Real *S, long long NS, const ReplicaDev *reps, int r,
                             const uint16_t *gcode, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ReplicaDev &R = reps[r];
    const long long x = i % R.nx, yz = i / R.nx, y = yz % R.ny, z = yz / R.ny;
    const long long j = R.off + x + R.px * (y + R.ny * z);
    const bool mag = gcode[j] != 0;
    S[j] = mag ? (Real)src[3 * i] : Real(0);
    S[NS + j] = mag ? (Real)src[3 * i + 1] : Real(0);
    S[2 * NS + j] = mag ? (Real)src[3 * i + 2] : Real(0);
}

template <typename Real>
__global__ void k_soa_to_aos(const Real *S, long long NS, const ReplicaDev *reps, int r, double *dst, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ReplicaDev &R = reps[r];
    const long long x = i % R.nx, yz = i / R.nx, y = yz % R.ny, z = yz / R.ny;
    const long long j = R.off + x + R.px * (y + R.ny * z);
    dst[3 * i] = (double)S[j];
    dst[3 * i + 1] = (double)S[NS + j];
    dst[3 * i + 2] = (double)S[2 * NS + j];
}

template <typename Real>
__global__ void k_init_state(Real *S, long long NS, const uint16_t *gcode) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NS) return;
    S[j] = Real(0);
    S[NS + j] = Real(0);
    S[2 * NS + j] = gcode[j] ? Real(1) : Real(0);
}

template <typename Real>
__global__ void k_zero_void(Real *S, long long NS, const uint16_t *gcode, long long first, long long count) {
    const long long j = first + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= first + count || gcode[j] != 0) return;
    S[j] = Real(0);
    S[NS + j] = Real(0);
    S[2 * NS + j] = Real(0);
}

template <typename Real>
__global__ void k_check_finite(const Real *S, long long NS, const uint16_t *gcode, Ctl *ctl) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NS || gcode[j] == 0) return;
    const double x = S[j], y = S[NS + j], z = S[2 * NS + j];
    const double n2 = x * x + y * y + z * z;
    if (!isfinite(n2) || fabs(n2 - 1.0) > 1e-3) atomicOr(&ctl->err, 1);
}

static unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_aos_to_soa(int prec, const double *src, void *S, long long NS, const ReplicaDev *reps, int r,
                              const uint16_t *gcode, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (prec == HAMR_FP64)
        k_aos_to_soa<double><<<nblk(n, 256), 256, 0, st>>>(src, (double *)S, NS, reps, r, gcode, n);
    else
        k_aos_to_soa<float><<<nblk(n, 256), 256, 0, st>>>(src, (float *)S, NS, reps, r, gcode, n);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(int prec, const void *S, long long NS, const ReplicaDev *reps, int r, double *dst,
                              long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (prec == HAMR_FP64)
        k_soa_to_aos<double><<<nblk(n, 256), 256, 0, st>>>((const double *)S, NS, reps, r, dst, n);
    else
        k_soa_to_aos<float><<<nblk(n, 256), 256, 0, st>>>((const float *)S, NS, reps, r, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int prec, void *S, long long NS, const uint16_t *gcode, cudaStream_t st) {
    if (prec == HAMR_FP64)
        k_init_state<double><<<nblk(NS, 256), 256, 0, st>>>((double *)S, NS, gcode);
    else
        k_init_state<float><<<nblk(NS, 256), 256, 0, st>>>((float *)S, NS, gcode);
    return cudaGetLastError();
}

cudaError_t launch_zero_void(int prec, void *S, long long NS, const uint16_t *gcode, long long first,
                             long long count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (prec == HAMR_FP64)
        k_zero_void<double><<<nblk(count, 256), 256, 0, st>>>((double *)S, NS, gcode, first, count);
    else
        k_zero_void<float><<<nblk(count, 256), 256, 0, st>>>((float *)S, NS, gcode, first, count);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(int prec, const void *S, long long NS, const uint16_t *gcode, Ctl *ctl,
                                cudaStream_t st) {
    if (prec == HAMR_FP64)
        k_check_finite<double><<<nblk(NS, 256), 256, 0, st>>>((const double *)S, NS, gcode, ctl);
    else
        k_check_finite<float><<<nblk(NS, 256), 256, 0, st>>>((const float *)S, NS, gcode, ctl);
    return cudaGetLastError();
}

cudaError_t launch_copy_state(int prec, const void *src, void *dst, long long NS, cudaStream_t st) {
    const size_t bytes = (size_t)3 * NS * (prec == HAMR_FP64 ? 8 : 4);
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
}

}  // namespace hamr
