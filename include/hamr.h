/*
 * hamr.h -- C ABI of the GB300 stochastic-LLG library.
 *
 * One library call advances the atomistic spin lattice of the laser-heated write
 * window of a HAMR model (arXiv 2502.02236) by Heun steps of the stochastic
 * Landau-Lifshitz-Gilbert equation (Sec. II, Eq. 1), with
 *   - exchange from a neighbour list: simple cubic, 6 nearest neighbours, or the L1_0
 *     FePt Fe sublattice, 4 nearest + 6 next-nearest neighbours in up to 3 shells
 *     (Sec. II, Eq. 2; Appendix A);
 *   - uniaxial anisotropy along z (Eq. 3);
 *   - a spatially uniform write field whose polarity follows a bit pattern (Sec. III);
 *   - a thermal field, Gaussian with standard deviation
 *     sqrt(2 alpha kB T_i / (gamma mu_s dt)) (Sec. II, text under Eq. 1), where T_i is the
 *     local temperature of a Gaussian laser spot moving at constant velocity (Sec. III);
 * and FP64 reductions of the magnetisation, total and per grain (Eq. 6 as an average).
 *
 * Units: SI, fields in tesla (B = mu0 H), so gamma is in rad/(s T) and the thermal
 * standard deviation above is in tesla.  Equation of motion, per site i:
 *   dS/dt = -gamma/(1+alpha^2) [S x B + alpha S x (S x B)],
 *   B = (1/mu_s) sum_j J_ij S_j + (2 ku/mu_s)(S.z) z + B_app(t) + B_th,i.
 * One step from t_n = n dt (drivers frozen at t_n, the same thermal field in both stages):
 *   S'    = N(S + dt f(S, B(S)))
 *   S_new = N(S + dt/2 [f(S, B(S)) + f(S', B(S'))]),   N(v) = v/|v|.
 * Thermal normals: Philox4x32-10 (Salmon et al., SC'11) with key = the replica's 64-bit
 * seed (low word, high word) and counter = (site low, site high, step low, step high),
 * site = ix + nx (iy + ny iz); u_k = (x_k + 1/2) 2^-32; Box-Muller on (u0, u1) gives the x
 * and y normals, on (u2, u3) the z normal.  Results therefore do not depend on how the
 * lattice is tiled or batched.
 *
 * Conventions for every call:
 *   - Return value: HAMR_OK (0) or a negative hamr_status; no call aborts or throws.
 *     hamr_last_error(h) then describes the failure; the handle stays usable unless the
 *     status is HAMR_ERR_CUDA after a device fault.
 *   - Host arrays passed in are copied before the call returns; the caller keeps
 *     ownership.  Output arrays are caller-allocated.
 *   - Spin arrays at the boundary are FP64, site-major with three components
 *     (AoS: S[3*i + d]), sites ordered x fastest, then y, then z, whatever the internal
 *     precision.
 *   - Calls run on the stream given at creation and return when their work is done
 *     (host-synchronous), except where stated.
 *   - Non-magnetic sites (grain id -1) hold S = 0, are never updated and do not count
 *     in any average.
 */
#ifndef HAMR_H
#define HAMR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hamr_ctx *hamr_t;

typedef enum {
    HAMR_OK = 0,
    HAMR_ERR_ARG = -1,      /* invalid argument; nothing was changed */
    HAMR_ERR_OOM = -2,      /* device or host allocation failed */
    HAMR_ERR_CUDA = -3,     /* a CUDA call failed (message names it) */
    HAMR_ERR_STATE = -4,    /* call out of order (e.g. step before the exchange is set) */
    HAMR_ERR_TIMEOUT = -5,  /* a bounded device wait ran out */
    HAMR_ERR_NUMERIC = -6,  /* NaN or Inf found in the spin state */
    HAMR_ERR_IO = -7        /* file could not be read or written, or is malformed */
} hamr_status;

enum { HAMR_LATTICE_SC = 0, HAMR_LATTICE_L10 = 1 };
enum { HAMR_FP32 = 0, HAMR_FP64 = 1 };
enum { HAMR_NBR_STENCIL = 0, HAMR_NBR_CSR = 1 };

typedef struct {
    int32_t lattice;      /* HAMR_LATTICE_SC: sites at ((i+1/2)a, (j+1/2)a, (k+1/2)a).
                             HAMR_LATTICE_L10: Fe sublattice of the L1_0 fct cell (a, c):
                             square nets of spacing a/sqrt(2) stacked at c, sites at
                             ((i+1/2)a/sqrt2, (j+1/2)a/sqrt2, (k+1/2)c) (Appendix A). */
    int32_t precision;    /* HAMR_FP32: spin state and field arithmetic in FP32, FP64
                             reductions.  HAMR_FP64: everything in FP64. */
    int32_t neighbours;   /* HAMR_NBR_STENCIL: the lattice's implicit stencil (SC: 6
                             nearest neighbours; L1_0: 4 in-plane nearest, 2 out of plane,
                             4 in-plane diagonals); FP32 stencil handles run the fused
                             kernel.  HAMR_NBR_CSR: neighbour list, built from the geometry
                             at creation or replaced per replica by hamr_set_csr. */
    int32_t n_replicas;   /* independent lattices advanced together, >= 1 */
    const int32_t *dims;  /* [3 * n_replicas]: nx, ny, nz of each replica, each >= 1 */
    const uint64_t *seeds;/* [n_replicas]: Philox key of each replica */
    double a;             /* SC spacing, or the L1_0 in-plane fct constant [m], > 0 */
    double c;             /* L1_0 fct constant along z [m]; ignored for SC */
    int32_t periodic[3];  /* periodic boundary along x, y, z (0 = open) */
    double mu_s;          /* atomic moment [J/T], > 0 */
    double ku;            /* uniaxial anisotropy energy per atom [J] (K_1 of Eq. 3) */
    double alpha;         /* damping, the paper's lambda, >= 0 */
    double dt;            /* time step [s], > 0 */
    double gamma;         /* gyromagnetic ratio [rad/(s T)], > 0 */
    int32_t device;       /* CUDA device ordinal */
    void *stream;         /* cudaStream_t for all work of this handle.  NULL: the library
                             creates its own non-blocking stream (the legacy default stream
                             cannot be captured into CUDA graphs); callers that pass device
                             pointers must then order their own work with it. */
} hamr_lattice_desc;

/* Create a handle: allocates device state for all replicas (all spins +z, every site
 * magnetic and in grain 0, T = 0, no field, step counter 0).  *out is set on success and
 * owned by the caller until hamr_destroy.  Errors: ARG (bad descriptor), OOM, CUDA. */
int hamr_lattice_create(hamr_t *out, const hamr_lattice_desc *d);

/* Exchange energies J_s [J] of the neighbour shells (Eq. 2; Eq. 8 relates J to T_C).
 * SC: n_shells = 1 (bond length a).  L1_0: n_shells = 3, bond lengths a/sqrt2 (4 in-plane
 * nearest), c (2 out of plane) and a (4 in-plane diagonals); the paper uses one J for all
 * ten.  Must be called before the first step.  Errors: ARG. */
int hamr_set_neighbour_shells(hamr_t h, int32_t n_shells, const double *J);

/* Replace the neighbour list of one replica (HAMR_NBR_CSR only): row_ptr[n+1], col[nnz]
 * site indices of that replica (x fastest), shell[nnz] in [0, n_shells).  At most 32
 * neighbours per site.  Bonds touching a non-magnetic site are ignored.  Every bond i -> j
 * of shell s must have its partner j -> i of the same shell (J_ij = J_ji); a list without
 * is rejected.  Errors: ARG, STATE (stencil handle), OOM. */
int hamr_set_csr(hamr_t h, int32_t replica, const int32_t *row_ptr, const int32_t *col,
                 const uint8_t *shell);

/* Grain map of one replica (Sec. II: exchange-decoupled grains): grain[n] with ids in
 * [0, n_grains) or -1 for a non-magnetic site.  Exchange bonds join only sites of the
 * same grain; spins of non-magnetic sites are set to 0.  A site that turns magnetic keeps
 * its stored spin, which is 0 if it was non-magnetic: after changing a map in the middle
 * of a run, set the replica's moments (hamr_set_moments) before the next step.
 * n_grains <= 65534.  Errors: ARG. */
int hamr_set_grain_map(hamr_t h, int32_t replica, const int32_t *grain, int32_t n_grains);

/* Laser temperature of one replica (Sec. III, Fig. 2):
 * T(x, y, t) = T_amb + (T_peak - T_amb) exp(-4 ln2 [(x - x0 - vx t)^2 + (y - y0 - vy t)^2] / fwhm^2),
 * uniform in z; fwhm <= 0 gives the uniform T_amb.  Kelvin, metres, m/s.  Errors: ARG
 * (negative temperature). */
int hamr_set_temperature_profile(hamr_t h, int32_t replica, double T_amb, double T_peak,
                                 double fwhm, double x0, double y0, double vx, double vy);

/* Write field of one replica (Sec. III): B_app(t) = B0 s(t) dir, where the head at
 * x_h = head_x0 + head_v t sits in bit b = floor(x_h / bit_len) and s ramps linearly from
 * the polarity of bit b-1 to that of bit b over the first ramp_len of bit b (bit 1 ->
 * polarity -1, bit 0 -> +1; before the first bit and after the last the end bits hold).
 * n_bits = 0 gives the static field B0 dir.  dir is used as given (not normalised).
 * Errors: ARG. */
int hamr_set_field_sequence(hamr_t h, int32_t replica, double B0, const double dir[3],
                            const uint8_t *bits, int32_t n_bits, double bit_len,
                            double ramp_len, double head_x0, double head_v);

/* Spin state of one replica from host memory, S[3n] FP64 AoS (converted to the handle's
 * precision; non-magnetic sites are stored as 0).  Errors: ARG, CUDA. */
int hamr_set_moments(hamr_t h, int32_t replica, const double *S);

/* As hamr_set_moments, from device memory on the handle's device (S_dev[3n] FP64 AoS);
 * stream-ordered, returns without waiting. */
int hamr_set_moments_device(hamr_t h, int32_t replica, const double *S_dev);

/* Advance every replica by n_steps Heun steps (n_steps >= 0).  With record_every > 0 the
 * magnetisation of each replica is recorded after every completed step whose global
 * count is a multiple of record_every, and per-grain sums are kept for the latest
 * record.  Steps run as CUDA-graph replays of record_every steps (or 64 without
 * records).  Errors: STATE (exchange not set), CUDA, TIMEOUT, NUMERIC (only when
 * hamr_check_finite finds a bad value). */
int hamr_sllg_heun_steps(hamr_t h, int64_t n_steps, int32_t record_every);

/* As hamr_sllg_heun_steps but stream-ordered: returns after enqueueing the work. Records
 * become readable after hamr_synchronize. */
int hamr_sllg_heun_steps_async(hamr_t h, int64_t n_steps, int32_t record_every);

/* Wait for all work of the handle; moves pending records to the host record list. */
int hamr_synchronize(hamr_t h);

/* Spin state of one replica to host memory, S_out[3n] FP64 AoS.  Errors: ARG, CUDA. */
int hamr_read_moments(hamr_t h, int32_t replica, double *S_out);

/* As hamr_read_moments, into device memory S_dev[3n] on the handle's device;
 * stream-ordered, returns without waiting. */
int hamr_read_moments_device(hamr_t h, int32_t replica, double *S_dev);

/* Magnetisation records of one replica since creation or hamr_clear_records: M_t gets up
 * to `capacity` records of 3 doubles (M = sum over magnetic sites of S / their number),
 * *n_rec the number available (call with M_t = NULL to size the buffer).  M_grain, if not
 * NULL, gets n_grains x 3 doubles: each grain's average spin at the latest record.
 * step_of_rec, if not NULL, gets the completed-step count of each returned record.
 * Errors: ARG. */
int hamr_read_magnetisation(hamr_t h, int32_t replica, double *M_t, int64_t capacity,
                            int64_t *n_rec, double *M_grain, int64_t *step_of_rec);

/* Forget all stored records. */
int hamr_clear_records(hamr_t h);

/* Energy of one replica at the current state and step [J]:
 * E = -1/2 sum_i sum_j J_ij S_i.S_j - sum_i ku (S_i.z)^2 - sum_i mu_s B_app(t).S_i,
 * accumulated in FP64.  Errors: ARG, STATE, CUDA. */
int hamr_read_energy(hamr_t h, int32_t replica, double *E);

/* Count of completed steps (the n of t_n = n dt for the next step). */
int hamr_get_step(hamr_t h, int64_t *step);
int hamr_set_step(hamr_t h, int64_t step);

/* Scan the spin state for NaN/Inf (and |S| far from 1 on magnetic sites).  Returns
 * HAMR_OK or HAMR_ERR_NUMERIC. */
int hamr_check_finite(hamr_t h);

/* Checkpoint: spins, step counter, seeds and lattice shape to a binary file.  Because the
 * thermal field is counter-based, a run resumed from a checkpoint is bitwise identical to
 * an uninterrupted one.  Load requires a handle of the same shape and precision.
 * Errors: IO, ARG, CUDA. */
int hamr_save_state(hamr_t h, const char *path);
int hamr_load_state(hamr_t h, const char *path);

/* Launch shape of the fused FP32 stencil kernel (both lattices): CTA size `threads` and
 * `staged`, the number
 * of positions per plane a CTA stages in shared memory (row pitch x rows).  Each replica is
 * split into column blocks that fit the shape: the block plus a two-column halo within the
 * staged region, and the block plus a one-column halo within the columns the CTA lists
 * (one or two per thread); the split is chosen per replica by a work model.  Compiled
 * (threads, columns per thread, pitch x rows): (512, 1, 36 x 24), (1024, 1, 68 x 24),
 * (256, 1, 36 x 14), (256, 2, 36 x 24).  hamr_autotune times every compiled shape on the
 * current state (advancing nothing: state and step are restored) and keeps the fastest.  With
 * the plane-range length left to the work model (hamr_set_plane_range 0), a shape that the
 * model splits along z is timed on whole columns as well; if whole columns win, the range
 * length is then fixed at the deepest replica's plane count (hamr_query key 6).
 * Errors: ARG (shape not compiled), STATE, CUDA. */
int hamr_set_tile(hamr_t h, int32_t threads, int32_t staged);
int hamr_get_tile(hamr_t h, int32_t *threads, int32_t *staged);
/* Planes per work item of the fused FP32 kernel.  A column block spans all planes of its
 * replica unless the batch has too few blocks to keep every resident CTA busy; then each
 * block is also split into ranges of at most `planes` planes (at least 4, chosen by a work
 * model that weighs the resident CTAs against the two recomputed halo planes per range).  The
 * results do not depend on the split: the S' of a range's boundary planes is recomputed with
 * the same noise.  planes = 0 (the default): chosen by the work model; > 0: fixed.
 * hamr_query key 6 reports the length in use, key 5 the number of work items.  Errors: ARG. */
int hamr_set_plane_range(hamr_t h, int32_t planes);
int hamr_autotune(hamr_t h, int32_t steps_per_trial);

/* Failure-detection test hook (no counterpart in the paper).  The next step call makes the
 * CTA that takes the first work item of its first step withhold one arrival on the staging
 * barrier of plane 1, so that its bounded waits run out after `polls` polls (instead of
 * 2^22).  That call returns HAMR_ERR_TIMEOUT and leaves the spin state invalid (set it
 * again); the device context stays usable.  Nothing faults.  Fused FP32 stencil handles
 * only.  Errors: ARG (polls < 1), STATE (other handles). */
int hamr_inject_wait_timeout(hamr_t h, int32_t polls);

/* Sizes: key 0 = total lattice sites, 1 = magnetic sites, 2 = device bytes held,
 * 3 = kernel launches per step (excluding records), 4 = storage slots, 5 = work items of the
 * fused FP32 kernel, 6 = its planes per work item (5 and 6 build the work list if needed). */
int hamr_query(hamr_t h, int32_t key, int64_t *value);

/* ---- One step without allocation ------------------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot allocate device
 * memory themselves (code running while another framework owns the whole device memory
 * pool, or a host loop that must not allocate after start-up) and so cannot create a
 * hamr_t.  It advances one simple-cubic lattice (implicit 6-neighbour stencil, one exchange
 * energy J) by one FP64 Heun step, with the same arithmetic and the same Philox stream as
 * the FP64 path of hamr_sllg_heun_steps, a static applied field B_app and the laser spot of
 * hamr_set_temperature_profile.
 *   S_in, S_out: caller-owned device arrays of 3 n doubles (site-major, x fastest); they
 *                are the same array or do not overlap (a partial overlap is ARG).
 *                Non-magnetic sites are copied unchanged.
 *   grain:       caller-owned device array of n int32 grain ids (-1 = non-magnetic), or
 *                NULL for one grain.
 *   step:        the n of t_n = n dt (thermal-field counter and laser position).
 *   stream:      cudaStream_t; the call only enqueues two kernels and returns.
 * Intermediate results live in one fixed device array (9 doubles per site, for at most
 * HAMR_NOALLOC_MAX_SITES sites, about 9.4 MB) that every GPU loading the library holds until
 * the process exits.  No call allocates or frees memory.  The first call on a device looks
 * up that array's address (cudaGetSymbolAddress) and should come before any stream capture.
 * All calls share the array and it keeps the last call's contents (nothing in it needs to
 * start at zero): calls that overlap on the GPU race.  Errors (hamr_last_error(NULL) holds
 * the message): ARG (null pointer, bad parameter, more than HAMR_NOALLOC_MAX_SITES sites,
 * S_out partly overlapping S_in), CUDA. */
#define HAMR_NOALLOC_MAX_SITES 131072

typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
    double a, mu_s, J, ku, alpha, dt, gamma;   /* as in hamr_lattice_desc; J of the one shell */
    uint64_t seed;                             /* Philox key */
    double T_amb, T_peak, fwhm, x0, y0, vx, vy; /* as in hamr_set_temperature_profile */
    double B_app[3];                           /* static applied field [T] */
} hamr_noalloc_params;

int hamr_sllg_heun_step_noalloc(const hamr_noalloc_params *p, const double *S_in, double *S_out,
                                const int32_t *grain, int64_t step, void *stream);

/* Message of the last failed call on this handle (never NULL). */
const char *hamr_last_error(hamr_t h);

/* Free all device and host memory of the handle.  NULL is allowed. */
void hamr_destroy(hamr_t h);


/* ------------------------------------------------------------------------------------
 * Multiscale write window (Sec. II and Fig. 1 of the paper).
 *
 * A micromagnetic track of ncx x ncy x ncz cubic cells (edge `cell`) holds an atomistic
 * simple-cubic window of spacing a = cell / ratio: the window is wx cell columns long,
 * starts at cell column x0 and spans every cell in y and z, so each of its cells holds
 * ratio^3 sites.  A cell's grain id (-1 = non-magnetic) is shared by its sites.  FP64.
 * One coupled step n -> n+1, drivers frozen at t_n:
 *   1. every window cell takes the direction of the sum of its spins (Eq. 6);
 *   2. the window takes one sLLG Heun step as in hamr_sllg_heun_steps (Eq. 1-3, damping
 *      lambda, thermal normals keyed by the seed with the site's index on the whole track,
 *      X + (ncx ratio)(j + (ncy ratio) k), X = x0 ratio + i); a bond across the window's
 *      x faces sees the direction m of the micromagnetic cell holding the neighbour
 *      position (Eq. 2 with the cell's m).  Bonds join equal grain ids only;
 *   3. the cells outside the window take one classical RK4 step of the micromagnetic LLG
 *      (Eq. 1 without thermal field) in the field
 *        B = (2 A(T)/Ms(T)) lap(m) + (2 K(T)/Ms(T)) (m.z) z + B_app          (Eq. 4, 5)
 *      with the 6-point finite-difference Laplacian over same-grain magnetic cells (a
 *      missing neighbour adds nothing; window cells enter with their Eq. 6 directions),
 *      Ms(T) = Ms0 m_e, A(T) = A0 m_e^2, K(T) = K0 m_e^3, damping
 *      lambda (1 - T / 3 T_C) with T capped at T_C, and m_e(T) the root in [0, 1] of
 *      m = L(3 T_C m / T + mu_s |B_app| / kB T), L(x) = coth x - 1/x (Sec. II); T is the
 *      laser temperature at the cell centre; m is renormalised after the step.
 * With hamr_ms_set_demag the demagnetising field of Eq. 7 is added to both regions; with
 * hamr_ms_set_head_profile the write field varies along the track.
 * Moving the window one column forward (hamr_ms_steps with follow): the trailing column
 * is handed to the micromagnetic side by Eq. 6, the sites shift back by one cell column
 * and the new leading column is thermalised: each site gets a spin whose polar angle from
 * the cell's m is uniform in [0, theta_max], theta_max = (5 pi/9) sqrt(1 - sqrt(1 +
 * 6 (m_e - 1)/5)) with the root's argument held in [0, 1] (Sec. II, M/Ms0 = m_e of the
 * cell), and whose azimuth is uniform; u0, u1 are the first two words of Philox4x32-10
 * with key = seed and counter = (site low, site high, event low, event high | 2^31),
 * event = the number of thermalisations so far (window placements and moves).
 * Conventions are those of the rest of this header; cell and site arrays at the boundary
 * are FP64 AoS, x fastest.  Sites of the window: i + nxw (j + nyw k) with nxw = wx ratio,
 * nyw = ncy ratio.
 * ------------------------------------------------------------------------------------ */
typedef struct hamr_ms_ctx *hamr_ms_t;

typedef struct {
    int32_t ncx, ncy, ncz;   /* micromagnetic cells along x (the track), y, z */
    double cell;             /* cell edge [m] */
    int32_t ratio;           /* atomistic sites per cell edge, >= 1 */
    int32_t wx;              /* window length in cells, 1 <= wx <= ncx */
    double J, mu_s, ku;      /* atomistic exchange [J], moment [J/T], anisotropy per atom [J] */
    double Ms0, A0, K0;      /* micromagnetic Ms [A/m], A [J/m], K [J/m^3] at 0 K */
    double lambda;           /* atomistic damping (the paper's lambda) */
    double T_C;              /* Curie temperature of the m_e(T) law [K] */
    double gamma, dt;        /* [rad/(s T)], [s] */
    uint64_t seed;           /* Philox key */
    int32_t precision;       /* HAMR_FP64: everything in FP64.  HAMR_FP32: spins, cells and
                                field arithmetic in FP32 (m_e(T) is solved in FP64) */
    int32_t device;
    void *stream;            /* cudaStream_t, or NULL for a library-owned stream.  Work is
                                ordered on this stream; within a step the handle also runs
                                the parts that do not depend on one another on a second,
                                library-owned stream, forked from and joined back to it */
} hamr_ms_desc;

/* Allocates the track and the window (errors: ARG, OOM, CUDA; message in
 * hamr_ms_last_error(NULL)).  Cells start at m = 0, every cell in grain 0. */
int hamr_ms_create(hamr_ms_t *out, const hamr_ms_desc *d);
/* Grain id per cell (ncx ncy ncz int32, -1 = non-magnetic; copied).  ARG on ids < -1. */
int hamr_ms_set_grain_map(hamr_ms_t h, const int32_t *cell_grain);
/* Laser spot and write field, as hamr_set_temperature_profile / hamr_set_field_sequence
 * (Sec. III, Fig. 2), shared by both regions. */
int hamr_ms_set_temperature_profile(hamr_ms_t h, double T_amb, double T_peak, double fwhm, double x0, double y0,
                                    double vx, double vy);
int hamr_ms_set_field_sequence(hamr_ms_t h, double B0, const double dir[3], const uint8_t *bits, int32_t n_bits,
                               double bit_len, double ramp_len, double head_x0, double head_v);
/* Spatial profile of the write field along the track (Sec. III, Fig. 2, where the head
 * field is drawn as tanh profiles of its out-of-plane and in-plane components; the paper gives
 * no formula, this is the reading): with wz > 0 the field at x is
 *   B0 s(t) dir P(x - x_h(t) - dz, wz) + Bx0 s(t) P(x - x_h(t) - dx, wx) x,
 *   P(u, w) = (1 - tanh(u / w)) / 2,   x_h(t) = head_x0 + head_v t,
 * full under the pole upstream of the head and zero downstream, in both regions and in the
 * m_e(T) law.  wz <= 0 restores the spatially uniform field B0 s(t) dir.  ARG on non-finite
 * values or wx <= 0. */
int hamr_ms_set_head_profile(hamr_ms_t h, double Bx0, double wz, double dz, double wx, double dx);
/* Simulated region (Sec. II, Fig. 1): margin >= 0 evolves only the micromagnetic cells of
 * the cell columns [x0 - margin, x0 + wx + margin) around the window (x0 its first column),
 * a region that moves with the window; every other cell is frozen: it keeps its m and the
 * m_e(T) of its last evolved step, or of the window's last placement (its magnetisation in
 * Eq. 7).  The cost of a step then follows the region, not the track.  margin < 0 (the
 * default) evolves the whole track.  Takes effect from the next step.  Errors: ARG (NULL). */
int hamr_ms_set_region(hamr_ms_t h, int32_t margin);
/* Demagnetising and stray field (Eq. 7) in both regions: B_d = -mu0 N * M on every cell,
 * with N the demagnetising tensor of cubic cells (Newell, Williams and Dunlop, J. Geophys.
 * Res. 98, 9551 (1993); the point-dipole tensor beyond 40 cell edges), M = Ms0 m_e(T) m on
 * micromagnetic cells and M = (mu_s / V) sum of its spins on window cells (Eq. 6, Sec. II),
 * recomputed every step from the state at t_n and added to the field of every cell and of
 * every site in it.  The convolution: in x and y by FFT on a grid zero-padded to twice the
 * columns and rows (cuFFT, one in-plane transform per plane and component), along z by the
 * direct sum over the track's planes at every in-plane frequency; the first call with
 * on != 0 builds the tensor (host, FP64) and its transforms.  on = 0 switches it off.
 * Errors: OOM, CUDA. */
int hamr_ms_set_demag(hamr_ms_t h, int32_t on);
/* B_d = -mu0 N * M (Eq. 7, the convolution of hamr_ms_set_demag over the whole track) for a
 * given magnetisation M [A/m] of every cell (3 ncx ncy ncz doubles, AoS, non-magnetic cells
 * included; read only) into B_out [T] (same layout, caller-owned), computed in the handle's
 * precision.  The state is not touched.  ARG on NULL or non-finite M, STATE while Eq. 7 is
 * off (hamr_ms_set_demag(h, 1) first), CUDA on a failed transform. */
int hamr_ms_demag_field(hamr_ms_t h, const double *M, double *B_out);
/* Micromagnetic directions m (3 ncx ncy ncz doubles, AoS; copied; non-magnetic cells are
 * set to 0).  ARG on non-finite values. */
int hamr_ms_set_cells(hamr_ms_t h, const double *m);
/* Places the window at cell column x0_cells and thermalises all of it from the cells (one
 * thermalisation event).  A window already placed first hands its sites back to its cells by
 * Eq. 6, as the trailing column does when the window moves (Sec. II), unless set_cells has
 * replaced the cells since.  A second pass along a parallel track (Sec. III) is a new spot
 * centre y0 (set_temperature_profile), spot and head starting points for the current time
 * (set_temperature_profile, set_field_sequence) and this call at the new spot.
 * ARG if the window leaves the track, STATE before set_cells. */
int hamr_ms_set_window(hamr_ms_t h, int32_t x0_cells);
/* Overwrites the window's spins (3 nxw nyw nzw doubles, AoS; copied).  STATE before the
 * window is placed. */
int hamr_ms_set_moments(hamr_ms_t h, const double *S);
/* n_steps coupled steps; follow != 0 moves the window forward after each step until it is
 * centred on the laser spot, x0 = floor(x_spot / cell - wx/2 + 1/2) kept on the track.
 * Window cells then hold the Eq. 6 directions of the current spins.  ARG on n_steps < 0,
 * STATE before the window is placed. */
int hamr_ms_steps(hamr_ms_t h, int64_t n_steps, int32_t follow);
/* Reads m (3 ncx ncy ncz doubles) or the window spins (3 nxw nyw nzw doubles). */
int hamr_ms_read_cells(hamr_ms_t h, double *m_out);
int hamr_ms_read_moments(hamr_ms_t h, double *S_out);
/* Read-back of the written track, a stand-in for the read head of Sec. III (its tunnel-
 * junction model is not part of the paper).  Bit b (0 <= b < n_bits) covers the cells whose
 * centre x lies in [x_start + b bit_len, x_start + (b + 1) bit_len) and whose row lies in
 * [cy0, cy1), all layers; signal[b] = mean m_z over its magnetic cells (window cells count
 * with their Eq. 6 directions; 0 when there is no magnetic cell), bits[b] = 1 where the signal
 * is negative (a '1' is written along -z), else 0.  signal: caller-owned n_bits doubles;
 * bits: caller-owned n_bits bytes, or NULL.  ARG on bit_len <= 0, an empty or out-of-range
 * row band, or a NULL signal. */
int hamr_ms_read_track(hamr_ms_t h, double x_start, double bit_len, int32_t n_bits, int32_t cy0, int32_t cy1,
                       double *signal, uint8_t *bits);
/* Window column (-1 before placement) and completed steps; either pointer may be NULL. */
int hamr_ms_get_window(hamr_ms_t h, int32_t *x0_cells, int64_t *step);
const char *hamr_ms_last_error(hamr_ms_t h);
void hamr_ms_destroy(hamr_ms_t h);

#ifdef __cplusplus
}
#endif

#endif /* HAMR_H */
